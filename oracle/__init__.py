"""CPU oracle for the shortwave Monte Carlo ray tracer (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this package. The CUDA library never imports, links or calls it, and it never
imports the CUDA library.

It wraps `mcrt_oracle.c` (an FP64 analog tracer with its own Philox4x32-10
stream, fine-cell DDA and analog collisions; see that file's header) and adds
the flux normalisation of the paper in numpy FP64.

Normalisation (Sec. 2.3, the experiments' definition of samples per pixel):
N photons enter the domain top; with a flux F0 normal to the beam and solar
zenith angle theta0, each carries E = F0 cos(theta0) Lx Ly / N watts. A surface
or top tally of n photons in a column is n E / (dx dy) W m^-2, and an
absorption tally in a cell is n E / (dx dy dz) W m^-3.

Heating rates use c_p = 1004 J kg^-1 K^-1 and rho(z) = 1.225 exp(-z/8000)
kg m^-3 (the paper states heating in K/d without a density profile).

Parity status of each function is stated in its docstring; every function is
pinned by the tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcrt_oracle.c")
_LIB = os.path.join(_HERE, "libmcrt_oracle.so")
_lib = None

CP_AIR = 1004.0
RHO0 = 1.225
RHO_SCALE_HEIGHT = 8000.0
SECONDS_PER_DAY = 86400.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc/OpenMP (in-tree shared object)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        u64, i32, f64 = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_sample_mu.argtypes = [i32, f64, u64, u64, P]
        lib.or_sample_mu.restype = i32
        lib.or_turn.argtypes = [P, u64, P, P, P]
        lib.or_trace.argtypes = ([i32, i32, i32, f64, f64, f64] + [P] * 6 +
                                 [f64, f64, u64, u64, u64, u64, i32, i32, u64, f64, i32] + [P] * 9)
        lib.or_trace.restype = i32
        lib.or_direct_beam.argtypes = [i32, i32, i32, f64, f64, f64, P, P, f64, f64, i32, i32, P]
        lib.or_direct_beam.restype = i32
        lib.or_sobol2.argtypes = [u64, i32, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11); pinned by the published KAT."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample_mu(kind: str, n: int, seed: int = 1, g: float = 0.0) -> np.ndarray:
    """Scattering-angle cosines from the oracle's samplers (Sec. 2.3 phase functions).

    kind: 'rayleigh' (rejection), 'hg' (inverse CDF) or 'lambert' (cosine law).
    """
    k = {"rayleigh": 0, "hg": 1, "lambert": 2}[kind]
    out = np.empty(n, dtype=np.float64)
    if _load().or_sample_mu(k, float(g), n, seed, _ptr(out)) != 0:
        raise ValueError(kind)
    return out


def turn(d, mu, phi) -> np.ndarray:
    """Directions at angle acos(mu) from unit vector d, azimuth phi about d."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.empty((mu.size, 3), dtype=np.float64)
    _load().or_turn(_ptr(d), mu.size, _ptr(mu), _ptr(phi), _ptr(out))
    return out


def sobol2(n: int, k0: int = 0) -> np.ndarray:
    """(n, 2) uint32: points k0..k0+n-1 of the 2D Sobol sequence (Sec. 2.3 start
    positions), as 32-bit binary fractions."""
    out = np.empty((n, 2), dtype=np.uint32)
    _load().or_sobol2(int(k0), int(n), _ptr(out))
    return out


def sun_mu0(sza_deg: float) -> float:
    return float(np.cos(np.deg2rad(sza_deg)))


def photon_energy(scene, sza_deg: float, toa_flux: float, photons_total: int) -> float:
    """Energy per photon E = F0 mu0 Lx Ly / N [W]."""
    return toa_flux * sun_mu0(sza_deg) * (scene.nx * scene.dx) * (scene.ny * scene.dy) / photons_total


def air_density(nz: int, dz: float) -> np.ndarray:
    zc = (np.arange(nz, dtype=np.float64) + 0.5) * dz
    return RHO0 * np.exp(-zc / RHO_SCALE_HEIGHT)


def heating_rate(abs_w_m3: np.ndarray, dz: float) -> np.ndarray:
    """K/day from absorbed power density [W m^-3], layout [nz][ny][nx]."""
    rho = air_density(abs_w_m3.shape[0], dz)
    return SECONDS_PER_DAY * abs_w_m3 / (rho[:, None, None] * CP_AIR)


def homogenize(field: np.ndarray) -> np.ndarray:
    """Horizontal homogenisation of the "-hom" and "-hom-hr" experiments
    (Sec. 2.4): every horizontal layer of a [nz][ny][nx] field, or the single
    layer of a [ny][nx] field, replaced by its mean over the layer's columns."""
    f = np.asarray(field, dtype=np.float64)
    layers = f.reshape(-1, f.shape[-2] * f.shape[-1])
    out = np.empty_like(layers)
    for k in range(layers.shape[0]):
        out[k, :] = layers[k].sum() / layers.shape[1]
    return out.reshape(f.shape)


@dataclass
class OracleResult:
    """Fields in physical units (W m^-2 for 2D, W m^-3 for 3D) plus raw counts."""

    abs_dir: np.ndarray      # track-length estimator, never-scattered photons
    abs_dif: np.ndarray      # track-length estimator, scattered photons
    abs_dir_cnt: np.ndarray  # analog-absorption estimator
    abs_dif_cnt: np.ndarray
    sfc_dir: np.ndarray
    sfc_dif: np.ndarray
    sfc_abs: np.ndarray
    toa_up: np.ndarray
    counts: dict
    totals: dict
    energy: float

    @property
    def abs3d(self) -> np.ndarray:
        return self.abs_dir + self.abs_dif


def trace(scene, sza_deg: float, az_deg: float, toa_flux: float, photons: int, seed: int,
          id_begin: int = 0, photons_total: int | None = None, col_offset: int = 0,
          pcld_mode: int = 0, nthreads: int = 0, max_steps: int = 10**9,
          diffuse_fraction: float = 0.0, birth: str = "philox") -> OracleResult:
    """Analog FP64 Monte Carlo estimate (Sec. 2.3) for photon ids [id_begin, id_begin+photons).

    `photons_total` (default `photons`) sets the energy per photon, so that
    disjoint id ranges traced separately add up to one run. A share
    `diffuse_fraction` of the photons starts diffuse (isotropic downwelling
    radiance at the domain top, Sec. 2.3). `birth` "sobol" starts the photons of
    each column at its scrambled Sobol points (Sec. 2.3) instead of uniform
    random positions.
    """
    lib = _load()
    birth_mode = {"philox": 0, "sobol": 1}[birth]
    nx, ny, nz = scene.nx, scene.ny, scene.nz
    ncell, ncol = nx * ny * nz, nx * ny
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in
            (scene.k_gas, scene.ssa_gas, scene.k_cld, scene.ssa_cld, scene.g_cld, scene.albedo)]
    tl_dir = np.zeros(ncell); tl_dif = np.zeros(ncell)
    n_adir = np.zeros(ncell, np.uint64); n_adif = np.zeros(ncell, np.uint64)
    n_sdir = np.zeros(ncol, np.uint64); n_sdif = np.zeros(ncol, np.uint64)
    n_sabs = np.zeros(ncol, np.uint64); n_toa = np.zeros(ncol, np.uint64)
    tot = np.zeros(8, np.uint64)
    st = lib.or_trace(nx, ny, nz, scene.dx, scene.dy, scene.dz, *[_ptr(a) for a in arrs],
                      float(sza_deg), float(az_deg), int(id_begin), int(id_begin + photons),
                      int(col_offset), int(seed), int(pcld_mode), int(nthreads), int(max_steps),
                      float(diffuse_fraction), birth_mode,
                      _ptr(tl_dir), _ptr(tl_dif), _ptr(n_adir), _ptr(n_adif), _ptr(n_sdir),
                      _ptr(n_sdif), _ptr(n_sabs), _ptr(n_toa), _ptr(tot))
    if st != 0:
        raise RuntimeError(f"oracle trace failed with status {st}")
    E = photon_energy(scene, sza_deg, toa_flux, photons_total or photons)
    f2 = E / (scene.dx * scene.dy)
    f3 = E / (scene.dx * scene.dy * scene.dz)
    shp3, shp2 = (nz, ny, nx), (ny, nx)
    names = ["photons", "toa", "atm_abs", "sfc_abs", "collisions", "scatters", "surface_hits", "steps"]
    return OracleResult(
        abs_dir=(tl_dir * f3).reshape(shp3), abs_dif=(tl_dif * f3).reshape(shp3),
        abs_dir_cnt=(n_adir * f3).reshape(shp3), abs_dif_cnt=(n_adif * f3).reshape(shp3),
        sfc_dir=(n_sdir * f2).reshape(shp2), sfc_dif=(n_sdif * f2).reshape(shp2),
        sfc_abs=(n_sabs * f2).reshape(shp2), toa_up=(n_toa * f2).reshape(shp2),
        counts={"abs_dir": n_adir.reshape(shp3), "abs_dif": n_adif.reshape(shp3),
                "sfc_dir": n_sdir.reshape(shp2), "sfc_dif": n_sdif.reshape(shp2),
                "sfc_abs": n_sabs.reshape(shp2), "toa": n_toa.reshape(shp2)},
        totals={k: int(v) for k, v in zip(names, tot)}, energy=E)


def direct_beam(scene, sza_deg: float, az_deg: float, nsub: int = 8, nthreads: int = 0) -> np.ndarray:
    """Column-mean direct-beam transmittance exp(-int k_ext ds) toward the sun, [ny][nx].

    Deterministic (FP64 DDA, midpoint nsub x nsub grid of surface points per
    column). F0 mu0 times this is the expected direct surface irradiance.
    """
    out = np.zeros(scene.nx * scene.ny)
    kg = np.ascontiguousarray(scene.k_gas, dtype=np.float32)
    kc = np.ascontiguousarray(scene.k_cld, dtype=np.float32)
    st = _load().or_direct_beam(scene.nx, scene.ny, scene.nz, scene.dx, scene.dy, scene.dz,
                                _ptr(kg), _ptr(kc), float(sza_deg), float(az_deg), int(nsub),
                                int(nthreads), _ptr(out))
    if st != 0:
        raise ValueError("invalid direct-beam arguments")
    return out.reshape(scene.ny, scene.nx)


FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")


def batch_means(scene, sza_deg, az_deg, toa_flux, photons, seeds, **kw):
    """Mean and standard error over independent batches (one seed each).

    Returns {field: (mean, se)} for the FIELDS plus the list of per-batch results.
    """
    runs = [trace(scene, sza_deg, az_deg, toa_flux, photons, s, **kw) for s in seeds]
    out = {}
    B = len(runs)
    for f in FIELDS:
        stack = np.stack([getattr(r, f) for r in runs])
        out[f] = (stack.mean(0), stack.std(0, ddof=1) / np.sqrt(B))
    return out, runs
