"""GPU tests of the CUDA tracer through the C ABI.

Parity is statistical (Monte Carlo): the GPU's weighted null-collision
estimator and the oracle's analog estimator have the same expectation, so
results are compared cell by cell in units of their combined standard error
(independent batches on each side), plus domain means within 0.5 %. Closed
forms (Beer-Lambert, absorber + Lambertian surface, isotropic slab) pin the
GPU path directly as well.
"""
import copy

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2208_05247_b300 import scenes
from paper_2208_05247_b300 import rt
from tests import refs

pytestmark = pytest.mark.gpu

FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")


def gpu_batches(scene, sza, az, flux, photons, seeds, cxyz=(0, 0, 0), **opts):
    out = {f: [] for f in FIELDS}
    stats_list = []
    with rt.Tracer.from_scene(scene, *cxyz, **opts) as t:
        for s in seeds:
            t.reset()
            t.trace(sza, az, flux, photons, s)
            f = t.fields(split=True)
            for k in FIELDS:
                out[k].append(f[k])
            stats_list.append(t.stats())
    return {k: np.stack(v) for k, v in out.items()}, stats_list


def oracle_batches(scene, sza, az, flux, photons, seeds, **kw):
    out = {f: [] for f in FIELDS}
    for s in seeds:
        r = oracle.trace(scene, sza, az, flux, photons, s, **kw)
        for k in FIELDS:
            out[k].append(getattr(r, k))
    return {k: np.stack(v) for k, v in out.items()}


# --- RNG and samplers ------------------------------------------------------------------

def test_philox_known_answers_on_gpu():
    from tests.test_oracle_pins import PHILOX_KAT
    ctr = np.array([c for c, _, _ in PHILOX_KAT], dtype=np.uint32)
    key = np.array([k for _, k, _ in PHILOX_KAT], dtype=np.uint32)
    want = np.array([w for _, _, w in PHILOX_KAT], dtype=np.uint32)
    assert np.array_equal(rt.rt_debug_philox(ctr, key), want)


def _chi2(samples, cdf, lo=-1.0, nbins=100):
    edges = np.linspace(lo, 1, nbins + 1)
    obs, _ = np.histogram(samples, bins=edges)
    exp = np.diff([cdf(e) for e in edges]) * samples.size
    return stats.chisquare(obs, exp).pvalue


def test_gpu_rayleigh_sampler():
    mu = rt.rt_debug_sample("rayleigh", 4_000_000, seed=3).astype(np.float64)
    assert np.all(np.abs(mu) <= 1)
    assert abs(mu.mean()) < 4 * np.sqrt(0.4 / mu.size)
    assert abs((mu ** 2).mean() - 0.4) < 4 * np.sqrt((12 / 35 - 0.16) / mu.size)
    assert _chi2(mu, refs.rayleigh_cdf) > 1e-4


@pytest.mark.parametrize("g", [0.0, 0.3, 0.86, -0.5, 0.98])
def test_gpu_hg_sampler(g):
    mu = rt.rt_debug_sample("hg", 4_000_000, seed=5, g=g).astype(np.float64)
    assert abs(mu.mean() - g) < 4 * mu.std() / np.sqrt(mu.size) + 2e-6
    p2 = 1.5 * mu ** 2 - 0.5
    assert abs(p2.mean() - g * g) < 4 * p2.std() / np.sqrt(mu.size) + 2e-6
    assert _chi2(mu, lambda m: refs.hg_cdf(m, g)) > 1e-4


def test_gpu_lambert_sampler():
    mu = rt.rt_debug_sample("lambert", 4_000_000, seed=9).astype(np.float64)
    assert mu.min() > 0 and mu.max() <= 1
    assert abs(mu.mean() - 2 / 3) < 4 * np.sqrt(1 / 18 / mu.size)
    assert _chi2(mu, lambda m: m * m, lo=0.0) > 1e-4


@pytest.mark.parametrize("d", [(0, 0, -1), (0.6, 0, 0.8), (0.3, -0.4, np.sqrt(0.75)), (1, 0, 0),
                               (0, 0, 1)])
def test_gpu_turn(d):
    d = np.asarray(d, float) / np.linalg.norm(d)
    rng = np.random.default_rng(1)
    n = 200_000
    mu = rng.uniform(-1, 1, n)
    phi = rng.uniform(-np.pi, np.pi, n)
    out = rt.rt_debug_turn(d, mu, phi).astype(np.float64)
    assert np.allclose(np.linalg.norm(out, axis=1), 1, atol=1e-6)
    assert np.allclose(out @ d, mu, atol=2e-6)
    assert np.all(np.abs(out.mean(0)) < 4 / np.sqrt(3 * n))


# --- closed forms through the full path ----------------------------------------------

def test_gpu_absorber_over_lambertian_surface():
    k = np.array([2e-3, 1e-3, 5e-4, 2e-4], dtype=np.float32)
    dz = 200.0
    sc = scenes.layered_scene(4, 4, k.size, 100.0, 100.0, dz, k_gas=k, ssa_gas=0.0, albedo=0.6)
    sza, F0 = 35.0, 1000.0
    mu0 = np.cos(np.deg2rad(sza))
    ref = refs.absorber_with_lambert(k, dz, mu0, 0.6, F0)
    g, st = gpu_batches(sc, sza, 17.0, F0, 1_000_000, range(16), cxyz=(2, 2, 2))
    # Ten expectations are checked at once (4 + 4 layers, surface, top), so the
    # bound is family-wise: 4.5 SE per comparison keeps the chance that any
    # one of them fails by noise near 1e-4 (4 SE per comparison would be 6e-4).
    def check(arr, want):
        m = arr.mean(0)
        se = arr.std(0, ddof=1) / np.sqrt(arr.shape[0])
        assert np.all(np.abs(m - want) < 4.5 * se + 1e-9 * abs(want)), (m, want, se)
    check(g["sfc_dir"].mean(axis=(1, 2)), ref["sfc_dir"])
    check(g["toa_up"].mean(axis=(1, 2)), ref["toa_up"])
    assert np.all(g["sfc_dif"] == 0)
    check(g["abs_dir"].mean(axis=(2, 3)) * dz, ref["abs_dir_layers"])
    check(g["abs_dif"].mean(axis=(2, 3)) * dz, ref["abs_dif_layers"])


def test_gpu_isotropic_slab_against_collision_probabilities():
    tau_star, omega, sza = 1.0, 0.9, 36.87
    mu0 = np.cos(np.deg2rad(sza))
    nz, k = 10, 1e-3
    dz = tau_star / (k * nz)
    sc = scenes.layered_scene(4, 4, nz, 100.0, 100.0, dz, k_gas=0.0, ssa_gas=0.0, k_cld=k,
                              ssa_cld=omega, g_cld=0.0)
    ref = refs.isotropic_slab_cp(tau_star, omega, mu0, M=400)
    g, _ = gpu_batches(sc, sza, 0.0, 1.0, 1_000_000, range(16))
    norm = mu0   # fluxes are per unit horizontal incoming flux mu0 * F0
    for arr, want in ((g["toa_up"].mean(axis=(1, 2)) / norm, ref["R"]),
                      (g["sfc_dif"].mean(axis=(1, 2)) / norm, ref["T_dif"]),
                      (g["sfc_dir"].mean(axis=(1, 2)) / norm, ref["T_dir"])):
        se = arr.std(ddof=1) / np.sqrt(arr.size)
        assert abs(arr.mean() - want) < 4 * se, (arr.mean(), want, se)
    A = ref["A_layers"].reshape(nz, -1).sum(1)[::-1]
    lay = (g["abs_dir"] + g["abs_dif"]).mean(axis=(2, 3)) * dz / norm
    se = lay.std(0, ddof=1) / np.sqrt(lay.shape[0])
    assert np.all(np.abs(lay.mean(0) - A) < 4 * se)


@pytest.mark.parametrize("phase", ["rayleigh", "hg"])
def test_gpu_thin_slab_single_scattering_oblique(phase):
    tau, omega, g, sza = 2e-3, 0.5, 0.86, 60.0
    if phase == "rayleigh":
        sc = scenes.layered_scene(2, 2, 1, 100.0, 100.0, tau, k_gas=1.0, ssa_gas=omega)
        pdf = refs.rayleigh_pdf
    else:
        sc = scenes.layered_scene(2, 2, 1, 100.0, 100.0, tau, k_gas=0.0, ssa_gas=0.0, k_cld=1.0,
                                  ssa_cld=omega, g_cld=g)
        pdf = lambda m: refs.hg_pdf(m, g)   # noqa: E731
    mu0 = np.cos(np.deg2rad(sza))
    R1 = refs.single_scatter_reflectance(pdf, mu0, tau, omega)
    T1 = refs.single_scatter_transmittance(pdf, mu0, tau, omega)
    res, _ = gpu_batches(sc, sza, 10.0, 1.0, 8_000_000, range(8), cxyz=(1, 1, 1))
    for arr, want in ((res["toa_up"].mean(axis=(1, 2)) / mu0, R1),
                      (res["sfc_dif"].mean(axis=(1, 2)) / mu0, T1)):
        se = arr.std(ddof=1) / np.sqrt(arr.size)
        assert abs(arr.mean() - want) < 4 * se + 3 * (omega * tau / mu0) * want, (arr.mean(), want, se)


# --- parity with the oracle on the 32^3 ellipsoid scene ------------------------------

@pytest.fixture(scope="module")
def c0_parity():
    sc = scenes.ellipsoid_scene(seed=0)
    B = 24
    g, st = gpu_batches(sc, 30.0, 0.0, 1000.0, 2 ** 22, range(100, 100 + B))
    o = oracle_batches(sc, 30.0, 0.0, 1000.0, 2 ** 18, range(500, 500 + B))
    # independent pilot batches decide which cells are sampled well enough to test alone
    gp, _ = gpu_batches(sc, 30.0, 0.0, 1000.0, 2 ** 22, range(200, 208))
    op = oracle_batches(sc, 30.0, 0.0, 1000.0, 2 ** 18, range(600, 608))
    return sc, g, o, st, (gp, op)


@pytest.mark.parametrize("field", FIELDS)
def test_parity_cellwise_with_oracle(c0_parity, field):
    _, g, o, _, (gp, op) = c0_parity
    rep = refs.parity_report(g[field], o[field], pilot=(gp[field], op[field]))
    assert rep["frac_over"] <= rep["bound"], (field, rep["frac_over"], rep["bound"], rep["max_abs_z"])
    assert rep["n"] >= 0.8 * rep["n_total"], (field, rep["n"], rep["n_total"])
    assert rep["pooled_p_family"] >= 1e-3, (field, rep["pooled_max_abs_z"], rep["pooled_p_family"])
    # the standardised differences are distributed as noise alone makes them
    # (KS distance of their Welch-t CDF values from the uniform law)
    assert rep["ks_d"] <= rep["ks_bound"], (field, rep["ks_d"], rep["ks_bound"])


@pytest.mark.parametrize("field", FIELDS)
def test_parity_domain_means_within_half_percent(c0_parity, field):
    _, g, o, _, (gp, op) = c0_parity
    rep = refs.parity_report(g[field], o[field], pilot=(gp[field], op[field]))
    assert abs(rep["domain_rel"]) < 0.005, (field, rep["domain_rel"], rep["domain_rel_se"])
    assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-9


def test_energy_ledger_closes(c0_parity):
    _, _, _, st, _ = c0_parity
    for s in st:
        lhs = s["energy_in"] + s["energy_created"] - s["energy_destroyed"] - s["energy_capped"]
        rhs = s["energy_toa_up"] + s["energy_atm_abs"] + s["energy_sfc_abs"]
        assert abs(lhs - rhs) < 1e-9 * s["energy_in"], (lhs, rhs)
        assert s["status"] == 0 and s["capped"] == 0
        assert s["photons"] == 2 ** 22


# --- conservation and symmetry pins ---------------------------------------------------

def test_gpu_conservative_black_surface_and_white_surface():
    """omega = 1 everywhere: weights never drop in the atmosphere, so nothing
    is absorbed there. Over a black surface every photon ends at the surface or
    the top; over a white one every photon leaves through the top (R = 1).
    Both hold to rounding, not only statistically (Sec. 2.3); the rounding is
    that of the FP32 product of weight and per-call photon energy that every
    tally adds (about 1e-8 relative), far below the sampling noise (~1e-3)."""
    sc = scenes.ellipsoid_scene(seed=0)
    sc.ssa_gas[:] = 1.0
    sc.ssa_cld[sc.k_cld > 0] = 1.0
    F = 1000.0 * np.cos(np.deg2rad(30.0))
    sc.albedo[:] = 0.0
    with rt.Tracer.from_scene(sc) as t:
        t.trace(30.0, 0.0, 1000.0, 1_000_000, 41)
        f, st = t.fields(split=True), t.stats()
    assert np.all(f["abs_dir"] == 0) and np.all(f["abs_dif"] == 0)
    assert st["energy_atm_abs"] == 0 and st["capped"] == 0
    arrived = f["sfc_dir"].mean() + f["sfc_dif"].mean()
    assert np.isclose(arrived + f["toa_up"].mean(), F, rtol=1e-6)
    sc.albedo[:] = 1.0
    with rt.Tracer.from_scene(sc) as t:
        t.trace(30.0, 0.0, 1000.0, 1_000_000, 42)
        f, st = t.fields(split=True), t.stats()
    assert st["energy_atm_abs"] == 0 and st["energy_sfc_abs"] == 0 and st["capped"] == 0
    assert np.isclose(f["toa_up"].mean(), F, rtol=1e-6)


def test_gpu_horizontally_homogeneous_scene_is_translation_invariant():
    """A layered scene with scattering: every column sees the same expectation,
    so column means differ from the domain mean only by sampling noise."""
    sc = scenes.layered_scene(12, 10, 8, 60.0, 60.0, 80.0, k_gas=2e-4, ssa_gas=0.9,
                              k_cld=[0, 0, 0.01, 0.02, 0.01, 0, 0, 0], ssa_cld=0.99, g_cld=0.8, albedo=0.3)
    g, _ = gpu_batches(sc, 40.0, 75.0, 1000.0, 399_960, range(300, 324))     # 3333 photons per column
    for field in ("sfc_dir", "sfc_dif", "toa_up"):
        a = g[field]                                   # [B][ny][nx]
        m = a.mean(0)
        se = a.std(0, ddof=1) / np.sqrt(a.shape[0])
        z = (m - m.mean()) / se
        # chi^2 of the column means about the domain mean: consistent with noise
        chi2 = float((z ** 2).sum())
        dof = z.size - 1
        assert chi2 < dof + 5 * np.sqrt(2 * dof), (field, chi2, dof)
        assert np.abs(z).max() < 6.5, (field, np.abs(z).max())


def test_gpu_overhead_sun_commutes_with_swapping_x_and_y():
    """With the sun overhead the transport has no preferred horizontal axis:
    tracing the x-y transposed scene gives the transposed fields (cell-wise
    parity statistic between two independent GPU runs)."""
    sc = scenes.ellipsoid_scene(seed=3)
    sw = copy.deepcopy(sc)
    for name in ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld"):
        setattr(sw, name, np.ascontiguousarray(np.swapaxes(getattr(sc, name), 1, 2)))
    sw.albedo = np.ascontiguousarray(sc.albedo.T)
    sw.nx, sw.ny, sw.dx, sw.dy = sc.ny, sc.nx, sc.dy, sc.dx
    a, _ = gpu_batches(sc, 0.0, 0.0, 1000.0, 2 ** 20, range(700, 716))
    b, _ = gpu_batches(sw, 0.0, 0.0, 1000.0, 2 ** 20, range(800, 816))
    # independent pilot batches choose the well-sampled cells
    ap, _ = gpu_batches(sc, 0.0, 0.0, 1000.0, 2 ** 20, range(900, 908))
    bp, _ = gpu_batches(sw, 0.0, 0.0, 1000.0, 2 ** 20, range(950, 958))
    for field in FIELDS:
        bt = np.swapaxes(b[field], -1, -2)
        rep = refs.parity_report(bt, a[field], pilot=(np.swapaxes(bp[field], -1, -2), ap[field]))
        assert rep["frac_over"] <= rep["bound"], (field, rep["frac_over"], rep["bound"])
        assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-9, (field, rep["domain_rel"])


def test_gpu_scene_shifted_by_whole_cells_gives_shifted_fields():
    """Periodic x and y: rolling the scene by (11, 5) cells, which carries the
    clouds across both lateral edges, rolls the fields by the same cells
    (cell-wise parity statistic between independent runs, slanted sun so that
    paths cross the edges)."""
    sc = scenes.ellipsoid_scene(seed=2)
    sh = copy.deepcopy(sc)
    dy, dx = 5, 11
    for name in ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld"):
        setattr(sh, name, np.ascontiguousarray(np.roll(getattr(sc, name), (dy, dx), axis=(1, 2))))
    sh.albedo = np.ascontiguousarray(np.roll(sc.albedo, (dy, dx), axis=(0, 1)))
    a, _ = gpu_batches(sc, 45.0, 60.0, 1000.0, 2 ** 20, range(1100, 1116))
    b, _ = gpu_batches(sh, 45.0, 60.0, 1000.0, 2 ** 20, range(1200, 1216))
    ap, _ = gpu_batches(sc, 45.0, 60.0, 1000.0, 2 ** 20, range(1300, 1308))
    bp, _ = gpu_batches(sh, 45.0, 60.0, 1000.0, 2 ** 20, range(1400, 1408))
    for field in FIELDS:
        back = np.roll(b[field], (-dy, -dx), axis=(-2, -1))
        back_p = np.roll(bp[field], (-dy, -dx), axis=(-2, -1))
        rep = refs.parity_report(back, a[field], pilot=(back_p, ap[field]))
        assert rep["frac_over"] <= rep["bound"], (field, rep["frac_over"], rep["bound"])
        assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-9, (field, rep["domain_rel"])


# --- reproducibility, launch-geometry and partition invariance -----------------------

def _run(sc, seed, N, **opts):
    with rt.Tracer.from_scene(sc, **opts) as t:
        t.trace(30.0, 0.0, 1000.0, N, seed)
        return t.fields(split=True), t.stats()


def test_same_seed_same_histories_any_launch_shape(small_scene):
    N = 300_000
    f1, s1 = _run(small_scene, 7, N)
    f2, s2 = _run(small_scene, 7, N, block_size=128, blocks_per_sm=1, refill_chunk=8)
    for k in ("photons", "events", "scatters", "crossings", "surface_hits", "roulette_kills", "max_events_photon"):
        assert s1[k] == s2[k], k
    for k in FIELDS:
        assert np.allclose(f1[k], f2[k], rtol=1e-12, atol=1e-12 * np.abs(f1[k]).max()), k
    f3, s3 = _run(small_scene, 8, N)
    assert s3["events"] != s1["events"]


def test_partition_invariance(small_scene):
    N = 200_000
    full, sf = _run(small_scene, 3, N)
    with rt.Tracer.from_scene(small_scene) as t:
        t.trace_range(30.0, 0.0, 1000.0, 0, 70_001, N, 3)
        t.trace_range(30.0, 0.0, 1000.0, 70_001, N - 70_001, N, 3)
        part, sp = t.fields(split=True), t.stats()
    for k in ("photons", "events", "scatters", "crossings"):
        assert sf[k] == sp[k]
    for k in FIELDS:
        assert np.allclose(full[k], part[k], rtol=1e-12, atol=1e-12 * np.abs(full[k]).max())
    assert np.isclose(sf["energy_in"], sp["energy_in"], rtol=1e-14)


def test_photon_ids_beyond_2_32(small_scene):
    """Photon ids that cross 2^32 (the kernel's 64-bit id, column and launch-
    order arithmetic), with the thick-first schedule engaged (whole rounds of
    >= 64 photons per column): one call over the range equals two calls over
    its halves, and the domain means match the oracle's over the same ids."""
    sc = small_scene
    ncol = sc.ncol
    B = (1 << 32) - 96 * ncol            # a multiple of ncol; the range crosses 2^32
    n = 192 * ncol
    total = B + n
    with rt.Tracer.from_scene(sc) as t:
        t.trace_range(30.0, 0.0, 1000.0, B, n, total, 5)
        full, sf = t.fields(split=True), t.stats()
    with rt.Tracer.from_scene(sc) as t:
        t.trace_range(30.0, 0.0, 1000.0, B, n // 2, total, 5)
        t.trace_range(30.0, 0.0, 1000.0, B + n // 2, n // 2, total, 5)
        part, sp = t.fields(split=True), t.stats()
    for k in ("photons", "events", "scatters", "crossings"):
        assert sf[k] == sp[k], k
    for k in FIELDS:
        assert np.allclose(full[k], part[k], rtol=1e-12, atol=1e-12 * np.abs(full[k]).max())
    # statistics: 8 disjoint sub-ranges a side, each normalised by the whole range
    g, o = {k: [] for k in FIELDS}, {k: [] for k in FIELDS}
    m = n // 8
    with rt.Tracer.from_scene(sc) as t:
        for i in range(8):
            t.reset()
            t.trace_range(30.0, 0.0, 1000.0, B + i * m, m, B + 8 * m, 5)
            f = t.fields(split=True)
            for k in FIELDS:
                g[k].append(8 * f[k].sum())
    for i in range(8):
        r = oracle.trace(sc, 30.0, 0.0, 1000.0, m, 17, id_begin=B + i * m, photons_total=B + 8 * m)
        for k in FIELDS:
            o[k].append(8 * getattr(r, k).sum())
    for k in FIELDS:
        a, b = np.array(g[k]), np.array(o[k])
        se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
        assert abs(a.mean() - b.mean()) < 4 * se + 1e-12 * abs(b.mean()), (k, a.mean(), b.mean(), se)


def test_coarse_factors_do_not_change_the_expectation(small_scene):
    """Any majorant grid (1x1x1 up to one coarse cell per axis) is unbiased."""
    res = {}
    for c in ((1, 1, 1), (4, 4, 4), (3, 5, 7), (32, 32, 32)):
        g, _ = gpu_batches(small_scene, 30.0, 0.0, 1000.0, 2 ** 17, range(8), cxyz=c)
        res[c] = g
    base = res[(4, 4, 4)]
    for c, g in res.items():
        for f in ("sfc_dif", "toa_up", "abs_dif"):
            rel, se = refs.domain_compare(g[f], base[f])
            assert abs(rel) < 4 * se + 1e-12, (c, f, rel, se)


# --- precision, modes and buffers ----------------------------------------------------

def test_fp32_tallies_follow_the_same_histories(small_scene):
    N = 200_000
    f64, s64 = _run(small_scene, 5, N)
    with rt.Tracer.from_scene(small_scene, tally_precision=rt.RT_TALLY_FP32) as t:
        t.reset()
        t.trace(30.0, 0.0, 1000.0, N, 5)
        f32, s32 = t.fields(split=True), t.stats()
    assert s32["events"] == s64["events"]
    for k in FIELDS:
        scale = np.abs(f64[k]).max()
        assert np.max(np.abs(f32[k] - f64[k])) < 1e-4 * scale, k


def test_paper_literal_scatterer_choice_mode():
    tau = 2e-3
    sc = scenes.layered_scene(2, 2, 1, 100.0, 100.0, tau, k_gas=0.5, ssa_gas=1.0, k_cld=0.5,
                              ssa_cld=0.2, g_cld=0.86)
    mu0 = 1.0 - 1e-12
    Rr = refs.single_scatter_reflectance(refs.rayleigh_pdf, mu0, tau)
    Rh = refs.single_scatter_reflectance(lambda m: refs.hg_pdf(m, 0.86), mu0, tau)
    for mode, want in ((0, 0.5 * Rr + 0.1 * Rh), (1, 0.6 * (0.5 * Rr + 0.5 * Rh))):
        g, _ = gpu_batches(sc, 0.0, 0.0, 1.0, 8_000_000, range(8), cxyz=(1, 1, 1), pcld_mode=mode)
        R = g["toa_up"].mean(axis=(1, 2))
        se = R.std(ddof=1) / np.sqrt(R.size)
        assert abs(R.mean() - want) < 4 * se + 3 * tau * want, (mode, R.mean(), want)


def test_device_buffers_match_host_buffers(small_scene):
    torch = pytest.importorskip("torch")
    N = 100_000
    fh, sh = _run(small_scene, 11, N)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in small_scene.fields()]
    alb = torch.from_numpy(small_scene.albedo).cuda()
    with rt.Tracer(small_scene.nx, small_scene.ny, small_scene.nz, small_scene.dx, small_scene.dy,
                   small_scene.dz, stream=torch.cuda.current_stream()) as t:
        t.set_optics(*dev)
        t.set_surface(alb)
        t.build_accel()
        t.trace(30.0, 0.0, 1000.0, N, 11)
        out = torch.empty(small_scene.ncell, dtype=torch.float64, device="cuda")
        sd = torch.empty(small_scene.ncol, dtype=torch.float64, device="cuda")
        rt.rt_fields(t.h, t.ncell, t.ncol, abs3d=out, sfc_dir=sd)
        torch.cuda.synchronize()
        assert np.allclose(out.cpu().numpy().reshape(fh["abs3d"].shape), fh["abs3d"], rtol=1e-12,
                           atol=1e-12 * fh["abs3d"].max())
        assert np.allclose(sd.cpu().numpy().reshape(fh["sfc_dir"].shape), fh["sfc_dir"], rtol=1e-12)


def test_heating_rate_conversion(small_scene):
    with rt.Tracer.from_scene(small_scene) as t:
        t.trace(30.0, 0.0, 1000.0, 100_000, 2)
        f = t.fields(split=True)
        hr = t.heating_rate(0)
        hr_dir = t.heating_rate(1)
    want = oracle.heating_rate(f["abs3d"], small_scene.dz)
    assert np.allclose(hr, want, rtol=1e-12, atol=0)
    assert np.allclose(hr_dir, oracle.heating_rate(f["abs_dir"], small_scene.dz), rtol=1e-12, atol=0)


# --- error paths (host-detected or device status; nothing faults) ----------------------

def test_errors_are_reported_not_faulted(small_scene):
    with rt.Tracer(8, 8, 8, 10.0, 10.0, 10.0) as t:
        with pytest.raises(rt.RtError) as e:
            t.trace(30.0, 0.0, 1000.0, 100, 1)
        assert e.value.code == rt.RT_E_STATE
        bad = [np.full(512, v, np.float32) for v in (1e-3, 0.5, 0.0, 0.0, 0.0)]
        bad[0][17] = np.nan
        with pytest.raises(rt.RtError) as e:
            t.set_optics(*bad)
        assert e.value.code == rt.RT_E_INVAL
        bad[0][17] = 1e-3
        bad[4][3] = 1.0          # |g| = 1
        with pytest.raises(rt.RtError):
            t.set_optics(*bad)
        bad[4][3] = 0.0
        t.set_optics(*bad)
        with pytest.raises(rt.RtError):
            t.set_surface(np.full(64, 1.5, np.float32))
        t.set_surface(np.full(64, 0.3, np.float32))
        with pytest.raises(rt.RtError):
            t.build_accel(9, 1, 1)
        t.build_accel()
        for args in ((90.0, 0.0, 1.0, 10, 1), (-1.0, 0.0, 1.0, 10, 1), (10.0, 0.0, -1.0, 10, 1)):
            with pytest.raises(rt.RtError) as e:
                t.trace(*args)
            assert e.value.code == rt.RT_E_INVAL
        with pytest.raises(rt.RtError):
            t.trace_range(10.0, 0.0, 1.0, 5, 10, 12, 1)
        t.trace(30.0, 0.0, 1000.0, 1000, 1)
        t.synchronize()


def test_step_cap_sets_budget_status_and_returns(small_scene):
    with rt.Tracer.from_scene(small_scene, max_steps=5) as t:
        t.trace(30.0, 0.0, 1000.0, 50_000, 1)
        with pytest.raises(rt.RtError) as e:
            t.synchronize()
        assert e.value.code == rt.RT_E_BUDGET
        s = t.stats()
        assert s["capped"] > 0 and s["status"] == rt.RT_E_BUDGET
        lhs = s["energy_in"] + s["energy_created"] - s["energy_destroyed"] - s["energy_capped"]
        rhs = s["energy_toa_up"] + s["energy_atm_abs"] + s["energy_sfc_abs"]
        assert abs(lhs - rhs) < 1e-9 * s["energy_in"]
        t.reset()
        t.set_options(max_steps=0)
        t.trace(30.0, 0.0, 1000.0, 50_000, 1)
        t.synchronize()


# --- the full-size LES-like scene, in the benchmark's launch configuration -------------

@pytest.fixture(scope="module")
def c1_scene():
    return scenes.cumulus_scene(seed=1)


def test_fullsize_cumulus_direct_beam_and_closure(c1_scene):
    """256x256x128 scene at 64 photons per column, default launch shape: the
    direct surface irradiance of 256 sampled columns matches the oracle's
    deterministic Beer-Lambert transmittance, and the energy ledger closes."""
    sc = c1_scene
    sza, az, F0 = 30.0, 0.0, 1000.0
    N = 64 * sc.ncol
    B = 6
    g, st = gpu_batches(sc, sza, az, F0, N, range(B))
    for s in st:
        lhs = s["energy_in"] + s["energy_created"] - s["energy_destroyed"] - s["energy_capped"]
        rhs = s["energy_toa_up"] + s["energy_atm_abs"] + s["energy_sfc_abs"]
        assert abs(lhs - rhs) < 1e-9 * s["energy_in"]
        assert s["capped"] == 0
    rng = np.random.default_rng(0)
    cols = rng.choice(sc.ncol, 256, replace=False)
    sub = copy.copy(sc)
    T = oracle.direct_beam(sub, sza, az, nsub=16).ravel()[cols]
    want = F0 * np.cos(np.deg2rad(sza)) * T
    arr = g["sfc_dir"].reshape(B, -1)[:, cols]
    m = arr.mean(0)
    se = arr.std(0, ddof=1) / np.sqrt(B)
    # Shadowed columns may see no direct photon in any batch; bound the standard
    # error from below by that of the direct-arrival fraction (weights <= 1).
    Tm = np.clip(T, 0.0, 1.0)
    se = np.maximum(se, F0 * np.cos(np.deg2rad(sza)) * np.sqrt(Tm * (1 - Tm) / (64 * B)) + 1e-9)
    z = (m - want) / se
    assert np.mean(np.abs(z) > 4.5) <= 0.02, np.sort(np.abs(z))[-5:]
    assert abs(m.mean() / want.mean() - 1) < 0.005


# --- parity with the oracle on the full 256x256x128 cumulus scene -------------------

# the benchmark's launch configuration (majorant boxes on a 2x2x2 grid)
C1_LAUNCH = dict(ready_threshold=16, max_inner=64, refill_chunk=128, block_size=64)
C1_PPC, C1_B, C1_PILOT = 64, 16, 8


@pytest.fixture(scope="module")
def c1_parity(c1_scene):
    """Streamed per-cell moments of 16 GPU and 16 oracle batches of 64 photons
    per column (4.2 M photons each), and the cells that independent pilots (8
    batches a side) find well sampled."""
    sc = c1_scene
    N = C1_PPC * sc.ncol
    cnt_g = {f: 0 for f in FIELDS}
    cnt_o = {f: 0 for f in FIELDS}
    with rt.Tracer.from_scene(sc, 2, 2, 2, **C1_LAUNCH) as t:
        for s in range(C1_PILOT):
            t.reset()
            t.trace(30.0, 0.0, 1000.0, N, 7000 + s)
            f = t.fields(split=True)
            for k in FIELDS:
                cnt_g[k] = cnt_g[k] + (f[k] != 0)
        for s in range(C1_PILOT):
            r = oracle.trace(sc, 30.0, 0.0, 1000.0, N, 8000 + s)
            for k in FIELDS:
                cnt_o[k] = cnt_o[k] + (getattr(r, k) != 0)
        good = {k: (cnt_g[k] >= 0.9 * C1_PILOT) & (cnt_o[k] >= 0.9 * C1_PILOT) for k in FIELDS}
        mg = {k: refs.BatchMoments(~good[k]) for k in FIELDS}
        mo = {k: refs.BatchMoments(~good[k]) for k in FIELDS}
        stats_list = []
        for s in range(C1_B):
            t.reset()
            t.trace(30.0, 0.0, 1000.0, N, 7100 + s)
            f = t.fields(split=True)
            for k in FIELDS:
                mg[k].add(f[k])
            stats_list.append(t.stats())
    for s in range(C1_B):
        r = oracle.trace(sc, 30.0, 0.0, 1000.0, N, 8100 + s)
        for k in FIELDS:
            mo[k].add(getattr(r, k))
    return good, mg, mo, stats_list


@pytest.mark.parametrize("field", FIELDS)
def test_fullsize_parity_cellwise_with_oracle(c1_parity, field):
    """Cell-wise parity on the full scene (8.4 M cells), where the majorant
    boxes, the launch order and L2 eviction all act: the same criterion as on
    the 32^3 scene."""
    good, mg, mo, _ = c1_parity
    rep = refs.parity_from_moments(mg[field], mo[field], good[field])
    assert rep["frac_over"] <= rep["bound"], (field, rep["frac_over"], rep["bound"], rep["max_abs_z"])
    assert rep["pooled_p_family"] >= 1e-3, (field, rep["pooled_max_abs_z"], rep["pooled_p_family"])
    assert rep["ks_d"] <= rep["ks_bound"], (field, rep["ks_d"], rep["ks_bound"])
    assert rep["n"] > 0


@pytest.mark.parametrize("field", FIELDS)
def test_fullsize_domain_means_within_half_percent(c1_parity, field):
    """Domain means within 0.5 % of the oracle's, with enough oracle photons
    (16 x 4.2 M) that 4 standard errors stay well below that."""
    _, mg, mo, _ = c1_parity
    rep = refs.domain_from_moments(mg[field], mo[field])
    assert 4 * rep["domain_rel_se"] < 0.005, (field, rep["domain_rel_se"])
    assert abs(rep["domain_rel"]) < 0.005, (field, rep["domain_rel"])
    assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-12, (field, rep["domain_rel"], rep["domain_rel_se"])


@pytest.mark.parametrize("sza", [0.0, 60.0])
def test_fullsize_domain_means_at_other_sun_angles(c1_scene, sza):
    """The full scene at the other two sun angles of the workload, bench launch
    shape, 8 + 8 batches of 64 photons per column: every field's domain mean
    within 0.5 % of the oracle's and within 4 combined SE, the SE small enough
    for the 0.5 % bound to mean something, and the ledger closed."""
    sc = c1_scene
    N = C1_PPC * sc.ncol
    B = 8
    tg, to = {f: [] for f in FIELDS}, {f: [] for f in FIELDS}
    with rt.Tracer.from_scene(sc, 2, 2, 2, **C1_LAUNCH) as t:
        for s in range(B):
            t.reset()
            t.trace(sza, 0.0, 1000.0, N, 7300 + s)
            f = t.fields(split=True)
            for k in FIELDS:
                tg[k].append(f[k].sum())
            st = t.stats()
            lhs = st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
            rhs = st["energy_toa_up"] + st["energy_atm_abs"] + st["energy_sfc_abs"]
            assert abs(lhs - rhs) < 1e-9 * st["energy_in"] and st["status"] == 0
    for s in range(B):
        r = oracle.trace(sc, sza, 0.0, 1000.0, N, 8300 + s)
        for k in FIELDS:
            to[k].append(getattr(r, k).sum())
    for k in FIELDS:
        a, b = np.array(tg[k]), np.array(to[k])
        rel = (a.mean() - b.mean()) / b.mean()
        se = np.sqrt(a.var(ddof=1) / B + b.var(ddof=1) / B) / abs(b.mean())
        assert 4 * se < 0.005, (k, sza, se)
        assert abs(rel) < 0.005 and abs(rel) < 4 * se + 1e-12, (k, sza, rel, se)


def test_fullsize_ledger_closes(c1_parity):
    for st in c1_parity[3]:
        lhs = st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
        rhs = st["energy_toa_up"] + st["energy_atm_abs"] + st["energy_sfc_abs"]
        assert abs(lhs - rhs) < 1e-9 * st["energy_in"], (lhs - rhs) / st["energy_in"]
        assert st["status"] == 0 and st["capped"] == 0




# --- degenerate and tiny grids ------------------------------------------------------

TINY = [((1, 1, 1), 11), ((1, 1, 6), 12), ((3, 1, 4), 13), ((1, 4, 3), 14), ((2, 3, 7), 15)]


@pytest.mark.parametrize("shape, seed", TINY)
def test_tiny_and_degenerate_grids_match_the_oracle(shape, seed):
    """Random cell-by-cell optics on a single cell, a single column, grids one
    cell wide in x or in y and a ragged 2x3x7 grid, each with the default,
    the finest and a single coarse cell: cell-wise parity with the oracle
    and domain means within 4 SE, ledger closed."""
    nx, ny, nz = shape
    sc = scenes.random_scene(nx, ny, nz, seed)
    B = 16
    o = oracle_batches(sc, 40.0, 30.0, 1000.0, 2 ** 16, range(9000, 9000 + B))
    op = oracle_batches(sc, 40.0, 30.0, 1000.0, 2 ** 16, range(9100, 9108))
    for cxyz in ((0, 0, 0), (1, 1, 1), (nx, ny, nz)):
        g, st = gpu_batches(sc, 40.0, 30.0, 1000.0, 2 ** 18, range(9200, 9200 + B), cxyz=cxyz)
        gp, _ = gpu_batches(sc, 40.0, 30.0, 1000.0, 2 ** 18, range(9300, 9308), cxyz=cxyz)
        for s in st:
            lhs = s["energy_in"] + s["energy_created"] - s["energy_destroyed"] - s["energy_capped"]
            rhs = s["energy_toa_up"] + s["energy_atm_abs"] + s["energy_sfc_abs"]
            # one photon deposits many times into one cell of these grids (a
            # single column keeps it in a layer's cell for long stretches), and
            # its FP32 partial of that cell rounds at ~6e-8 per addition before
            # the FP64 flush: 3.6e-9 measured on 1x1x6, against <= 1e-11 on the
            # workload scenes, where photons change cells every few events
            assert abs(lhs - rhs) < 1e-7 * s["energy_in"] and s["status"] == 0, (shape, cxyz)
        for field in FIELDS:
            rep = refs.parity_report(g[field], o[field], pilot=(gp[field], op[field]))
            assert rep["frac_over"] <= rep["bound"], (shape, cxyz, field, rep["max_abs_z"])
            assert rep["pooled_p_family"] >= 1e-3, (shape, cxyz, field, rep["pooled_max_abs_z"])
            assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-9, (shape, cxyz, field, rep["domain_rel"])


def test_empty_atmosphere_and_zero_photons_are_exact():
    """No extinction anywhere: every photon reaches the surface unscattered.
    With the sun overhead and whole rounds of photons per column, each column
    receives exactly its own photons: its direct irradiance is exactly F, its
    surface absorption F (1 - albedo), and the reflected share leaves through
    the top untouched (its roulette below weight 1/2 makes the domain mean
    upward flux F times the mean albedo in expectation). Under a slanted sun photons land in other columns, but the
    domain mean direct irradiance is still exactly F cos(sza). Nothing is
    absorbed in the atmosphere, and a trace of zero photons tallies nothing."""
    nx, ny, nz = 12, 10, 8
    sc = scenes.layered_scene(nx, ny, nz, 80.0, 80.0, 60.0, k_gas=0.0, ssa_gas=0.0)
    rng = np.random.default_rng(3)
    sc.albedo = rng.uniform(0.0, 0.8, (ny, nx)).astype(np.float32)
    alb = sc.albedo.astype(np.float64)
    with rt.Tracer.from_scene(sc) as t:
        t.trace(37.0, 123.0, 1000.0, 0, 5)
        f = t.fields(split=True)
        assert all(float(np.abs(f[k]).max()) == 0.0 for k in f), "zero photons must tally nothing"
        assert t.stats()["photons"] == 0
        t.trace(0.0, 0.0, 1000.0, 64 * sc.ncol, 5)
        f, st = t.fields(split=True), t.stats()
        assert st["status"] == 0 and st["scatters"] == 0
        assert np.allclose(f["sfc_dir"], 1000.0, rtol=1e-12)
        assert np.allclose(f["sfc_abs"], 1000.0 * (1.0 - alb), rtol=1e-6)
        # the reflected weight goes through roulette when it is below 1/2 (Sec.
        # 2.3): survival with probability a at weight 1, so the top flux is
        # exact only in expectation; per photon the variance is a (1 - a)
        var = np.where(alb < 0.5, alb * (1.0 - alb), 0.0)
        se = 1000.0 * np.sqrt(64 * var.sum()) / (64 * sc.ncol)
        assert abs(f["toa_up"].mean() - 1000.0 * alb.mean()) < 4 * se + 1e-9, (f["toa_up"].mean(), alb.mean(), se)
        for k in ("sfc_dif", "abs3d"):
            assert float(np.abs(f[k]).max()) == 0.0, k
        t.reset()
        t.trace(37.0, 123.0, 1000.0, 64 * sc.ncol, 6)
        f = t.fields(split=True)
        assert np.isclose(f["sfc_dir"].mean(), 1000.0 * np.cos(np.deg2rad(37.0)), rtol=1e-12)
        assert float(np.abs(f["abs3d"]).max()) == 0.0
