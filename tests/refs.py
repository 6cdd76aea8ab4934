"""Closed-form and deterministic references that pin the oracle (and the GPU path).

Nothing here shares arithmetic with the oracle or the CUDA library: each result
is derived from the radiative-transfer definitions directly.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate
from scipy.special import expn


def hg_pdf(mu, g):
    """Henyey-Greenstein density of mu = cos(scattering angle), normalised on [-1,1]."""
    return 0.5 * (1 - g * g) / (1 + g * g - 2 * g * mu) ** 1.5


def rayleigh_pdf(mu):
    return 0.375 * (1 + mu * mu)


def hg_cdf(mu, g):
    """Closed-form HG CDF (integral of hg_pdf from -1)."""
    if abs(g) < 1e-12:
        return 0.5 * (mu + 1)
    return (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * mu) ** -0.5 - 1 / (1 + g))


def rayleigh_cdf(mu):
    return (mu ** 3 + 3 * mu + 4) / 8.0


def upward_density(pdf, mu0, mu):
    """Density over outgoing direction cosine mu for a beam travelling downward
    with cosine -mu0, averaging the phase density over the outgoing azimuth."""
    s0 = np.sqrt(1 - mu0 * mu0)
    s = np.sqrt(max(0.0, 1 - mu * mu))

    def f(phi):
        cos_theta = -mu0 * mu + s0 * s * np.cos(phi)
        return pdf(cos_theta)
    val, _ = integrate.quad(f, 0.0, 2 * np.pi, limit=200, epsabs=1e-13)
    return val / (2 * np.pi)


def single_scatter_reflectance(pdf, mu0, tau, omega=1.0):
    """Exact single-scattering reflectance of a homogeneous slab over a black
    surface: omega * int_0^1 q(mu) (1/mu0) (1 - e^{-tau(1/mu0+1/mu)}) / (1/mu0+1/mu) dmu."""
    def f(mu):
        a = 1 / mu0 + 1 / mu
        return upward_density(pdf, mu0, mu) * (1 / mu0) * (-np.expm1(-tau * a)) / a
    val, _ = integrate.quad(f, 0.0, 1.0, limit=200, epsabs=1e-14)
    return omega * val


def single_scatter_transmittance(pdf, mu0, tau, omega=1.0):
    """Exact single-scattering diffuse transmittance (downward outgoing directions)."""
    def f(mu):  # mu > 0 is the cosine below the horizontal
        # the density for a downward outgoing cosine -mu equals the upward density of
        # a mirrored incident beam: pdf(mu0*mu + s0 s cos phi)
        s0 = np.sqrt(1 - mu0 * mu0)
        s = np.sqrt(max(0.0, 1 - mu * mu))
        q = integrate.quad(lambda phi: pdf(mu0 * mu + s0 * s * np.cos(phi)), 0.0, 2 * np.pi,
                           limit=200, epsabs=1e-13)[0] / (2 * np.pi)
        if abs(mu - mu0) < 1e-12:
            path = tau * np.exp(-tau / mu0)
        else:
            path = (np.exp(-tau / mu0) - np.exp(-tau / mu)) / (1 / mu - 1 / mu0)
        return q * (1 / mu0) * path
    val, _ = integrate.quad(f, 0.0, 1.0, limit=200, epsabs=1e-14, points=[mu0])
    return omega * val


def e3(x):
    return expn(3, x)


def layered_tau(k_layers, dz):
    """Optical depth from the top down to each layer interface (top first)."""
    k = np.asarray(k_layers, dtype=np.float64)[::-1]   # top layer first
    return np.concatenate([[0.0], np.cumsum(k * dz)])


def absorber_with_lambert(k_layers, dz, mu0, albedo, F0=1.0):
    """Purely absorbing layered atmosphere over a Lambertian surface.

    Returns dict with the direct surface irradiance, the upward flux at the top,
    and absorbed flux per layer (bottom layer first) split into the direct beam
    part and the surface-reflected (diffuse) part. The reflected radiance is
    isotropic, so its flux after optical depth t is F_up * 2 E3(t).
    """
    tau = layered_tau(k_layers, dz)                 # interfaces from the top
    ts = tau[-1]
    Fdir_iface = F0 * mu0 * np.exp(-tau / mu0)
    abs_direct_top_first = Fdir_iface[:-1] - Fdir_iface[1:]
    Fsfc = Fdir_iface[-1]
    Fup0 = albedo * Fsfc
    # upward flux at each interface: depth below the interface to the surface = ts - tau
    Fup_iface = Fup0 * 2 * e3(ts - tau)
    abs_diffuse_top_first = Fup_iface[1:] - Fup_iface[:-1]
    return {
        "sfc_dir": Fsfc,
        "toa_up": Fup_iface[0],
        "abs_dir_layers": abs_direct_top_first[::-1],
        "abs_dif_layers": abs_diffuse_top_first[::-1],
    }


def isotropic_slab_cp(tau_star, omega, mu0, M=400):
    """Homogeneous slab, isotropic scattering, black surface, collimated beam.

    Collision-probability solution: the slab is cut into M layers with a flat
    collision density in each; P[n, m] is the probability that a photon emitted
    isotropically from a uniform point of layer n has its next collision in
    layer m (exact slab kernels in E3). With f the direct beam's first-collision
    probabilities, collisions C solve C = f + omega P^T C. Returns per incident
    photon: R, T_dir, T_dif, absorbed fraction per layer (top first), and the
    layer edges in optical depth.
    """
    D = tau_star / M
    edges = np.linspace(0.0, tau_star, M + 1)
    f = np.exp(-edges[:-1] / mu0) - np.exp(-edges[1:] / mu0)
    idx = np.arange(M)
    gap = (np.abs(idx[:, None] - idx[None, :]) - 1) * D
    gap = np.maximum(gap, 0.0)
    P = (e3(gap) - 2 * e3(gap + D) + e3(gap + 2 * D)) / (2 * D)
    np.fill_diagonal(P, 1.0 - (0.5 - e3(D)) / D)
    esc_top = (e3(edges[:-1]) - e3(edges[1:])) / (2 * D)
    esc_bot = (e3(tau_star - edges[1:]) - e3(tau_star - edges[:-1])) / (2 * D)
    C = np.linalg.solve(np.eye(M) - omega * P.T, f)
    return {
        "R": omega * C @ esc_top,
        "T_dir": np.exp(-tau_star / mu0),
        "T_dif": omega * C @ esc_bot,
        "A_layers": (1 - omega) * C,
        "edges": edges,
        "row_sum": P.sum(1) + esc_top + esc_bot,
    }


def box_chord(p, d, lo, hi):
    """Length of the ray p + s d (s >= 0) inside the axis-aligned box [lo, hi]."""
    t0, t1 = 0.0, np.inf
    for a in range(3):
        if abs(d[a]) < 1e-300:
            if p[a] < lo[a] or p[a] > hi[a]:
                return 0.0
            continue
        ta, tb = (lo[a] - p[a]) / d[a], (hi[a] - p[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def zscores(m1, se1, m2, se2):
    den = np.sqrt(se1 ** 2 + se2 ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(den > 0, (m1 - m2) / den, np.where(m1 == m2, 0.0, np.inf))
    return z


class BatchMoments:
    """Running per-cell moments of independent batch results (one field).

    add(x) takes one batch ([nz, ny, nx] or [ny, nx]); the per-cell mean and
    standard error of the mean follow from the sums. `rare` (a boolean mask of
    the cells that are tested pooled, not alone) makes add() also keep each
    batch's sum over those cells, per layer of a 3D field or in one for a 2D
    field; the domain sum of every batch is kept as well. Streaming keeps the
    full-size scene (8.4 M cells) within a few hundred MB however many batches.
    """

    def __init__(self, rare=None):
        self.n, self.s, self.ss, self.rare = 0, None, None, rare
        self.pooled, self.totals = [], []

    def add(self, x):
        x = np.asarray(x, dtype=np.float64)
        if self.s is None:
            self.s, self.ss = np.zeros_like(x), np.zeros_like(x)
        self.n += 1
        self.s += x
        self.ss += x * x
        self.totals.append(float(x.sum()))
        if self.rare is not None:
            r = np.where(self.rare, x, 0.0)
            self.pooled.append(r.sum(axis=(1, 2)) if x.ndim == 3 else np.array([r.sum()]))

    def mean(self):
        return self.s / self.n

    def se(self):
        m = self.mean()
        var = np.maximum(self.ss / self.n - m * m, 0.0) * self.n / (self.n - 1)
        return np.sqrt(var / self.n)


def parity_from_moments(mg, mo, good, z_limit=4.0):
    """The parity statistic of two BatchMoments (built with rare = ~good)."""
    from scipy import stats as st
    B1, B2 = mg.n, mo.n
    m1, m2 = mg.mean(), mo.mean()
    sg, so = mg.se(), mo.se()
    z = zscores(m1, sg, m2, so)[good].ravel()
    n = z.size
    frac = float(np.mean(np.abs(z) > z_limit)) if n else 0.0
    dof = min(B1, B2) - 1
    bound = max(3.0 / max(n, 1), 2.0 * 2.0 * st.t.sf(z_limit, dof))
    # Under parity each z follows Student's t with the Welch-Satterthwaite
    # degrees of freedom of its cell, so 2 F_t(|z|) - 1 is uniform on (0,1)
    # whatever the cell's dof. |z| rather than z: the batch means of sparsely
    # sampled cells are skewed, which moves the signed z but hardly its size.
    vg, vo = (sg ** 2)[good].ravel(), (so ** 2)[good].ravel()
    with np.errstate(divide="ignore", invalid="ignore"):
        nu = (vg + vo) ** 2 / (vg ** 2 / (B1 - 1) + vo ** 2 / (B2 - 1))
    ok = np.isfinite(z) & np.isfinite(nu) & (nu > 0)
    u = 2.0 * st.t.cdf(np.abs(z[ok]), nu[ok]) - 1.0
    ks = st.kstest(u, "uniform") if u.size > 1 else None
    ks_p = float(ks.pvalue) if ks is not None else 1.0
    ks_d = float(ks.statistic) if ks is not None else 0.0
    # The uniform law of those values is itself an approximation (Welch-t,
    # mildly skewed batch means), and with tens of thousands of cells the KS
    # p-value detects that alone. The bound is on the distance instead: the
    # KS 1 % critical value for n values plus 0.03 for the approximation,
    # calibrated on independent oracle runs of the 32^3 ellipsoid scene with
    # 32-128 photons per column per batch (distance <= 0.018 over 3D fields,
    # <= 0.040 over 2D fields; a 3 % cloud-absorption error gives 0.44-0.82).
    ks_bound = 0.03 + 1.63 / np.sqrt(max(u.size, 1))
    # pooled rare cells: per-batch sums over them, per layer (3D) or in one (2D)
    pg, po = np.array(mg.pooled), np.array(mo.pooled)
    vpg, vpo = pg.var(0, ddof=1) / B1, po.var(0, ddof=1) / B2
    zp = zscores(pg.mean(0), np.sqrt(vpg), po.mean(0), np.sqrt(vpo))
    used = (pg != 0).any(0) | (po != 0).any(0)
    zp, vpg, vpo = zp[used], vpg[used], vpo[used]
    # Each pooled z is Welch-t (the SEs come from B batches a side); where one
    # side's spread dominates, as the collision estimator's does against the
    # oracle's, it is close to Student's t with B-1 dof, whose tail at 4.5 is
    # 40x the normal one. So the pooled groups are judged by their two-sided
    # t p-values, Bonferroni-corrected for the number of groups (layers).
    with np.errstate(divide="ignore", invalid="ignore"):
        nup = (vpg + vpo) ** 2 / (vpg ** 2 / (B1 - 1) + vpo ** 2 / (B2 - 1))
    nup = np.where(np.isfinite(nup) & (nup > 0), nup, min(B1, B2) - 1)
    pp = 2.0 * st.t.sf(np.abs(zp), nup)
    pooled_p_family = float(min(1.0, pp.min() * pp.size)) if pp.size else 1.0
    tot_g, tot_o = np.array(mg.totals), np.array(mo.totals)
    rel = float((tot_g.mean() - tot_o.mean()) / tot_o.mean()) if tot_o.mean() != 0 else 0.0
    se_rel = float(np.sqrt(tot_g.var(ddof=1) / B1 + tot_o.var(ddof=1) / B2) / abs(tot_o.mean())) \
        if tot_o.mean() != 0 else 0.0
    return {"frac_over": frac, "bound": bound, "max_abs_z": float(np.max(np.abs(z))) if n else 0.0,
            "n": n, "n_total": int(good.size), "pooled_max_abs_z": float(np.max(np.abs(zp))) if zp.size else 0.0,
            "pooled_p_family": pooled_p_family, "pooled_groups": int(zp.size),
            "domain_rel": rel, "domain_rel_se": se_rel, "z": z, "ks_p": ks_p, "ks_d": ks_d,
            "ks_bound": float(ks_bound)}


def domain_from_moments(mg, mo):
    """Relative difference of the mean domain sums of two BatchMoments and its SE."""
    tg, to = np.array(mg.totals), np.array(mo.totals)
    m = to.mean()
    if m == 0:
        return {"domain_rel": 0.0, "domain_rel_se": 0.0}
    return {"domain_rel": float((tg.mean() - m) / m),
            "domain_rel_se": float(np.sqrt(tg.var(ddof=1) / tg.size + to.var(ddof=1) / to.size) / abs(m))}


def parity_report(gpu_batches, orc_batches, z_limit=4.0, min_nonzero=0.9, pilot=None):
    """Cell-wise statistical parity of two sets of independent batch results.

    gpu_batches, orc_batches: arrays [B, ...] (3D fields [B, nz, ny, nx] or 2D
    [B, ny, nx]). A cell is well sampled when both sides score in at least
    `min_nonzero` of their batches of `pilot` = (gpu_pilot, orc_pilot), which
    must be independent of the batches under test: choosing cells from the
    tested batches themselves would select cells where one side happened to
    score low and bias the pooled sums. For well-sampled cells,
    z = (m1 - m2) / sqrt(se1^2 + se2^2)
    with batch standard errors. Cells that a collision estimator scores only
    rarely have no usable per-cell variance, so they are pooled (summed) per
    layer of a 3D field, or all together for a 2D field, and the pooled sums get
    the same z test. The shape of the z distribution is tested too: each |z|
    goes through the t-CDF of its cell's Welch-Satterthwaite degrees of
    freedom, and the KS distance of the results from the uniform law (ks_d)
    is held to ks_bound. Returns the fraction of well-sampled cells with
    |z| > z_limit and the bound it is held to (the larger of 3 cells and twice
    the two-sided Student-t tail with B-1 dof), the largest pooled |z| with the
    Bonferroni-corrected Welch-t p-value of the pooled groups
    (pooled_p_family), and the relative difference of the domain sums with its standard error.
    (The same statistic as parity_from_moments, which streams the batches.)
    """
    if pilot is None:
        raise ValueError("parity_report needs independent pilot batches for cell selection")
    pg_, po_ = (np.asarray(x, dtype=np.float64) for x in pilot)
    good = ((pg_ != 0).mean(0) >= min_nonzero) & ((po_ != 0).mean(0) >= min_nonzero)
    mg, mo = BatchMoments(~good), BatchMoments(~good)
    for x in np.asarray(gpu_batches, dtype=np.float64):
        mg.add(x)
    for x in np.asarray(orc_batches, dtype=np.float64):
        mo.add(x)
    return parity_from_moments(mg, mo, good, z_limit)


def domain_compare(gpu_batches, orc_batches):
    """Relative difference of the domain sums of two batch sets and its SE."""
    g = np.asarray(gpu_batches, dtype=np.float64)
    o = np.asarray(orc_batches, dtype=np.float64)
    tg, to = g.reshape(g.shape[0], -1).sum(1), o.reshape(o.shape[0], -1).sum(1)
    m = to.mean()
    if m == 0:
        return 0.0, 0.0
    se = np.sqrt(tg.var(ddof=1) / tg.size + to.var(ddof=1) / to.size) / abs(m)
    return float((tg.mean() - m) / m), float(se)
