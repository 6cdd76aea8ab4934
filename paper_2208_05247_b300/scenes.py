"""Seeded synthetic scenes for the shortwave Monte Carlo tracer.

The paper traces cloud fields from its LES runs (38.4 km square at 50 m
horizontal spacing, Sec. 2.2), which are not available here. These seeded
generators stand in for them with fields of the same kind: a stratified gas
profile plus compact cumulus-like cloud bodies near 1 km, a grey Lambertian
surface, and the paper's grid spacings.

This module only draws inputs. It holds none of the transport arithmetic: the
CUDA path and the CPU oracle both consume the arrays it returns, so that the
two sides see identical inputs.

Every field is float32 with layout [nz][ny][nx] (x fastest); the surface
albedo is [ny][nx].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import ndtri

GAS_K0 = 2e-5          # gas extinction at z = 0 [m^-1]
GAS_SCALE_HEIGHT = 8000.0
GAS_SSA = 0.9
CLOUD_SSA = 0.999999
CLOUD_G = 0.86


@dataclass
class Scene:
    """One periodic 3D scene: grid, five optics fields and the surface albedo."""

    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    k_gas: np.ndarray
    ssa_gas: np.ndarray
    k_cld: np.ndarray
    ssa_cld: np.ndarray
    g_cld: np.ndarray
    albedo: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def ncol(self) -> int:
        return self.nx * self.ny

    def fields(self):
        """The five optics arrays in the order the tracer's set-optics call takes them."""
        return (self.k_gas, self.ssa_gas, self.k_cld, self.ssa_cld, self.g_cld)

    def cloud_fraction(self) -> float:
        """Projected (column) cloud fraction."""
        return float((self.k_cld.max(axis=0) > 0).mean())


def _empty(nx, ny, nz):
    return np.zeros((nz, ny, nx), dtype=np.float32)


def gas_profile(nz: int, dz: float, scale: float = 1.0) -> np.ndarray:
    """Gas extinction k(z) = scale * 2e-5 * exp(-z/8000) m^-1 at cell centres."""
    zc = (np.arange(nz, dtype=np.float64) + 0.5) * dz
    return (scale * GAS_K0 * np.exp(-zc / GAS_SCALE_HEIGHT)).astype(np.float32)


def _gas_fields(nx, ny, nz, dz, scale=1.0, ssa=GAS_SSA):
    k = np.broadcast_to(gas_profile(nz, dz, scale)[:, None, None], (nz, ny, nx)).astype(np.float32)
    return np.ascontiguousarray(k), np.full((nz, ny, nx), ssa, dtype=np.float32)


def _periodic_offset(coord, centre, length):
    """Signed periodic distance coord - centre folded into [-L/2, L/2)."""
    return np.mod(coord - centre + 0.5 * length, length) - 0.5 * length


def ellipsoid_scene(seed: int = 0, n: int = 32, d: float = 100.0, nblobs: int = 3,
                    k_cloud: float = 0.05, albedo: float = 0.2) -> Scene:
    """Small cube with a few cloud ellipsoids (the oracle-sized workload).

    32^3 cells of 100 m; gas as `gas_profile`; `nblobs` ellipsoids with radii
    U(200, 500) m per axis, bases at 800 m, centres uniform in x and y with
    periodic wrap; inside a blob k_cld = 0.05 m^-1, ssa 0.999999, g 0.86.
    """
    rng = np.random.default_rng(seed)
    nx = ny = nz = n
    L = n * d
    k_gas, ssa_gas = _gas_fields(nx, ny, nz, d)
    k_cld = _empty(nx, ny, nz)
    xc = (np.arange(nx) + 0.5) * d
    zc = (np.arange(nz) + 0.5) * d
    blobs = []
    for _ in range(nblobs):
        rx, ry, rz = rng.uniform(200.0, 500.0, size=3)
        cx, cy = rng.uniform(0.0, L, size=2)
        cz = 800.0 + rz
        ox = _periodic_offset(xc, cx, L) / rx
        oy = _periodic_offset(xc, cy, L) / ry
        oz = (zc - cz) / rz
        inside = (oz[:, None, None] ** 2 + oy[None, :, None] ** 2 + ox[None, None, :] ** 2) <= 1.0
        k_cld[inside] = k_cloud
        blobs.append((rx, ry, rz, cx, cy, cz))
    cloudy = k_cld > 0
    ssa_cld = np.where(cloudy, CLOUD_SSA, 0.0).astype(np.float32)
    g_cld = np.where(cloudy, CLOUD_G, 0.0).astype(np.float32)
    alb = np.full((ny, nx), albedo, dtype=np.float32)
    return Scene("ellipsoids32", nx, ny, nz, d, d, d, k_gas, ssa_gas, k_cld, ssa_cld, g_cld, alb,
                 meta={"seed": seed, "blobs": blobs})


def cumulus_scene(seed: int = 1, nx: int = 256, ny: int = 256, nz: int = 128,
                  dx: float = 50.0, dy: float = 50.0, dz: float = 25.0,
                  nblobs: int | None = None, cloud_fraction: float = 0.20,
                  k_median: float = 0.03, k_sigma: float = 0.8,
                  gas_scale: float = 1.0) -> Scene:
    """LES-like cumulus field from a seeded sum of Gaussian blobs.

    400 blobs for a 256x256 domain (scaled with area otherwise): horizontal
    sigma U(100, 400) m, vertical sigma U(100, 300) m, base U(700, 1000) m with
    the centre at base + 2 sigma_z, periodic in x and y. Cells below the base of
    the blob that dominates them are cleared, then the sum is thresholded so
    that the projected cloud fraction is `cloud_fraction`. In-cloud extinction is
    the rank map of the blob sum onto lognormal(median 0.03 m^-1, sigma 0.8),
    which keeps the spatial coherence of the blobs. Cloud ssa 0.999999, g 0.86;
    surface albedo U(0.15, 0.25) per column.
    """
    rng = np.random.default_rng(seed)
    if nblobs is None:
        nblobs = max(1, int(round(400 * (nx * dx) * (ny * dy) / (256 * 50.0) ** 2)))
    Lx, Ly = nx * dx, ny * dy
    f = np.zeros((nz, ny, nx), dtype=np.float32)
    dom = np.zeros((nz, ny, nx), dtype=np.float32)       # largest single-blob contribution
    base_of_dom = np.zeros((nz, ny, nx), dtype=np.float32)
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    zc = (np.arange(nz) + 0.5) * dz
    sig_h = rng.uniform(100.0, 400.0, size=nblobs)
    sig_z = rng.uniform(100.0, 300.0, size=nblobs)
    base = rng.uniform(700.0, 1000.0, size=nblobs)
    cxs = rng.uniform(0.0, Lx, size=nblobs)
    cys = rng.uniform(0.0, Ly, size=nblobs)
    for b in range(nblobs):
        sh, sz, cz = sig_h[b], sig_z[b], base[b] + 2.0 * sig_z[b]
        # periodic +-3 sigma box in x and y, clipped box in z
        rx = min(nx // 2, int(np.ceil(3 * sh / dx)))
        ry = min(ny // 2, int(np.ceil(3 * sh / dy)))
        i0 = int(np.floor(cxs[b] / dx))
        j0 = int(np.floor(cys[b] / dy))
        ii = np.unique(np.mod(np.arange(i0 - rx, i0 + rx + 1), nx))
        jj = np.unique(np.mod(np.arange(j0 - ry, j0 + ry + 1), ny))
        kk = np.nonzero(np.abs(zc - cz) <= 3 * sz)[0]
        if kk.size == 0:
            continue
        gx = np.exp(-0.5 * (_periodic_offset(xc[ii], cxs[b], Lx) / sh) ** 2)
        gy = np.exp(-0.5 * (_periodic_offset(yc[jj], cys[b], Ly) / sh) ** 2)
        gz = np.exp(-0.5 * ((zc[kk] - cz) / sz) ** 2)
        blob = (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).astype(np.float32)
        ix = np.ix_(kk, jj, ii)
        f[ix] += blob
        cur = dom[ix]
        win = blob > cur
        dom[ix] = np.where(win, blob, cur)
        base_of_dom[ix] = np.where(win, np.float32(base[b]), base_of_dom[ix])
    f[zc[:, None, None] < base_of_dom] = 0.0
    colmax = f.max(axis=0)
    thr = np.quantile(colmax, 1.0 - cloud_fraction)
    mask = f > thr
    k_gas, ssa_gas = _gas_fields(nx, ny, nz, dz, gas_scale)
    k_cld = _empty(nx, ny, nz)
    vals = f[mask]
    if vals.size:
        order = np.argsort(vals, kind="stable")
        q = (np.arange(vals.size) + 0.5) / vals.size
        ln = (k_median * np.exp(k_sigma * ndtri(q))).astype(np.float32)
        mapped = np.empty_like(vals)
        mapped[order] = ln
        k_cld[mask] = mapped
    ssa_cld = np.where(mask, CLOUD_SSA, 0.0).astype(np.float32)
    g_cld = np.where(mask, CLOUD_G, 0.0).astype(np.float32)
    alb = rng.uniform(0.15, 0.25, size=(ny, nx)).astype(np.float32)
    return Scene(f"cumulus{nx}x{ny}x{nz}", nx, ny, nz, dx, dy, dz, k_gas, ssa_gas, k_cld, ssa_cld,
                 g_cld, alb, meta={"seed": seed, "nblobs": nblobs, "threshold": float(thr)})


def layered_scene(nx: int, ny: int, nz: int, dx: float, dy: float, dz: float,
                  k_gas, ssa_gas, k_cld=0.0, ssa_cld=0.0, g_cld=0.0, albedo=0.0,
                  name: str = "layered") -> Scene:
    """Horizontally homogeneous scene from per-layer values (scalars or length-nz)."""
    def lay(v):
        v = np.broadcast_to(np.asarray(v, dtype=np.float32), (nz,))
        return np.ascontiguousarray(np.broadcast_to(v[:, None, None], (nz, ny, nx))).astype(np.float32)
    alb = np.ascontiguousarray(np.broadcast_to(np.asarray(albedo, dtype=np.float32), (ny, nx))).astype(np.float32)
    return Scene(name, nx, ny, nz, dx, dy, dz, lay(k_gas), lay(ssa_gas), lay(k_cld), lay(ssa_cld),
                 lay(g_cld), alb)


def random_scene(nx: int, ny: int, nz: int, seed: int, d: float = 100.0) -> Scene:
    """Cell-by-cell random optics on a small grid (edge-case parity tests):
    gas k U(0, 5e-3) m^-1 with albedo U(0.3, 1); cloud in half of the cells,
    k U(0.005, 0.05) m^-1, albedo U(0.9, 1), g U(0, 0.9); surface albedo
    U(0, 0.6) per column."""
    rng = np.random.default_rng(seed)
    s3 = (nz, ny, nx)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)   # noqa: E731
    cloudy = rng.random(s3) < 0.5
    k_cld = np.where(cloudy, rng.uniform(0.005, 0.05, s3), 0.0)
    return Scene("random%dx%dx%d" % (nx, ny, nz), nx, ny, nz, d, d, d,
                 f32(rng.uniform(0.0, 5e-3, s3)), f32(rng.uniform(0.3, 1.0, s3)), f32(k_cld),
                 f32(np.where(cloudy, rng.uniform(0.9, 1.0, s3), 0.0)),
                 f32(np.where(cloudy, rng.uniform(0.0, 0.9, s3), 0.0)), f32(rng.uniform(0.0, 0.6, (ny, nx))))


# --- batched spectral + multi-scene workload ---------------------------------------

BATCH_SCENE_SHAPES = ((128, 128, 96), (192, 96, 128), (256, 256, 128), (64, 64, 64))
N_GPOINTS = 112


def gpoint_table(seed: int = 2, n: int = N_GPOINTS, total_flux: float = 1000.0):
    """Per-g-point gas extinction scale (log-uniform 1e-3..10) and TOA flux.

    TOA weights are U(0.1, 1), normalised so that the fluxes sum to
    `total_flux` W m^-2. Returns (gas_scale[n], toa_flux[n]) as float64.
    """
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(np.log(1e-3), np.log(10.0), size=n))
    w = rng.uniform(0.1, 1.0, size=n)
    return scale, w / w.sum() * total_flux


def batch_scenes(seed0: int = 20):
    """The four uneven scenes of the batched workload (C1-style, same spacing)."""
    return [cumulus_scene(seed=seed0 + s, nx=nx, ny=ny, nz=nz)
            for s, (nx, ny, nz) in enumerate(BATCH_SCENE_SHAPES)]
