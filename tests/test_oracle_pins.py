"""Pins of the CPU oracle to results the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms of radiative transfer, exact invariants, or
an independent deterministic solver (collision probabilities). They are chosen
so that a plausible mistake (a dropped term, a wrong sign of the sun azimuth,
a mis-sampled phase function, a transposed index) fails at least one.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2208_05247_b300 import scenes
from tests import refs

NT = 0  # oracle threads: all cores


# --- random numbers -----------------------------------------------------------------

# Published known-answer vectors of Philox4x32-10 (Random123 distribution, kat_vectors).
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(ctr, key, want):
    assert tuple(int(v) for v in oracle.philox4x32_10(ctr, key)) == want


# --- phase functions and the Lambertian surface (Sec. 2.3) ---------------------------

def _chi2_pvalue(samples, cdf, nbins=100):
    edges = np.linspace(-1, 1, nbins + 1) if samples.min() < 0 else np.linspace(0, 1, nbins + 1)
    obs, _ = np.histogram(samples, bins=edges)
    p = np.diff([cdf(e) for e in edges])
    exp = p * samples.size
    return stats.chisquare(obs, exp).pvalue


def test_rayleigh_sampler():
    mu = oracle.sample_mu("rayleigh", 2_000_000, seed=3)
    assert abs(mu.mean()) < 4 * np.sqrt(0.4 / mu.size)
    # E[mu^2] = 2/5 for p = 3/8 (1 + mu^2); Var(mu^2) = E[mu^4] - 4/25 = 12/35 - 4/25
    assert abs((mu ** 2).mean() - 0.4) < 4 * np.sqrt((12 / 35 - 0.16) / mu.size)
    assert _chi2_pvalue(mu, refs.rayleigh_cdf) > 1e-4


@pytest.mark.parametrize("g", [0.0, 0.5, 0.86, -0.3])
def test_hg_sampler(g):
    mu = oracle.sample_mu("hg", 2_000_000, seed=5, g=g)
    # E[mu] = g and E[P2(mu)] = g^2 for Henyey-Greenstein
    assert abs(mu.mean() - g) < 4 * mu.std() / np.sqrt(mu.size)
    p2 = 1.5 * mu ** 2 - 0.5
    assert abs(p2.mean() - g * g) < 4 * p2.std() / np.sqrt(mu.size)
    assert _chi2_pvalue(mu, lambda m: refs.hg_cdf(m, g)) > 1e-4


def test_lambert_sampler():
    mu = oracle.sample_mu("lambert", 2_000_000, seed=9)
    assert mu.min() > 0 and mu.max() < 1
    assert abs(mu.mean() - 2 / 3) < 4 * np.sqrt(1 / 18 / mu.size)
    assert _chi2_pvalue(mu, lambda m: m * m) > 1e-4


@pytest.mark.parametrize("d", [(0, 0, -1), (0.6, 0, 0.8), (0.3, -0.4, np.sqrt(0.75)), (1, 0, 0)])
def test_turn_preserves_angle_and_is_uniform_in_azimuth(d):
    d = np.asarray(d, float) / np.linalg.norm(d)
    rng = np.random.default_rng(0)
    n = 200_000
    mu = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    out = oracle.turn(d, mu, phi)
    assert np.allclose(np.linalg.norm(out, axis=1), 1, atol=1e-12)
    assert np.allclose(out @ d, mu, atol=1e-12)
    # uniform mu and phi give an isotropic direction: mean 0, second moment I/3
    assert np.all(np.abs(out.mean(0)) < 4 / np.sqrt(3 * n))
    assert np.allclose(out.T @ out / n, np.eye(3) / 3, atol=4 * np.sqrt(4 / 45 / n) + 1e-3)


# --- direct beam: Beer-Lambert and geometry ----------------------------------------

@pytest.mark.parametrize("sza,az", [(0, 0), (30, 0), (60, 228.1), (75, 90), (45, 333)])
def test_direct_beam_beer_lambert_layered(sza, az):
    k = np.array([3e-4, 1e-3, 5e-4, 2e-5, 7e-4, 0.0, 1e-4], dtype=np.float32)
    sc = scenes.layered_scene(5, 3, k.size, 70.0, 40.0, 55.0, k_gas=k, ssa_gas=0.0)
    mu0 = np.cos(np.deg2rad(sza))
    exact = np.exp(-np.sum(k.astype(np.float64) * 55.0) / mu0)
    T = oracle.direct_beam(sc, sza, az, nsub=3)
    assert np.max(np.abs(T / exact - 1)) < 1e-12


@pytest.mark.parametrize("az", [0.0, 90.0, 200.0])
def test_direct_beam_shadow_of_one_cell(az):
    """One absorbing cell in an empty domain: the transmittance of every sub-ray
    is exp(-k * chord), with the chord from an independent box intersection over
    the periodic images. A wrong azimuth convention moves the shadow."""
    n, d = 8, 100.0
    sc = scenes.layered_scene(n, n, n, d, d, d, k_gas=0.0, ssa_gas=0.0)
    k_cell = float(np.float32(4e-3))      # the scene stores float32 optics
    ci, cj, ck = 5, 2, 3
    sc.k_cld[ck, cj, ci] = k_cell
    sza = 40.0
    nsub = 4
    T = oracle.direct_beam(sc, sza, az, nsub=nsub)
    t, p = np.deg2rad(sza), np.deg2rad(az)
    to_sun = np.array([np.sin(t) * np.sin(p), np.sin(t) * np.cos(p), np.cos(t)])
    L = n * d
    want = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            acc = 0.0
            for a in range(nsub):
                for b in range(nsub):
                    p0 = np.array([(i + (a + 0.5) / nsub) * d, (j + (b + 0.5) / nsub) * d, 0.0])
                    chord = 0.0
                    for sx in (-2, -1, 0, 1, 2):
                        for sy in (-2, -1, 0, 1, 2):
                            lo = np.array([ci * d + sx * L, cj * d + sy * L, ck * d])
                            chord += refs.box_chord(p0, to_sun, lo, lo + d)
                    acc += np.exp(-k_cell * chord)
            want[j, i] = acc / nsub ** 2
    assert np.max(np.abs(T - want)) < 1e-12
    assert T.min() < 0.9        # the shadow is really there


# --- Monte Carlo closed forms --------------------------------------------------------

def test_mc_pure_absorber_over_lambertian_surface():
    """Absorbing layers (no scattering) over a Lambertian surface of albedo a:
    direct surface flux F0 mu0 e^{-tau/mu0}, top upward flux a F_sfc 2E3(tau),
    and per-layer absorption of the beam and of the reflected diffuse flux."""
    k = np.array([2e-3, 1e-3, 5e-4, 2e-4], dtype=np.float32)    # bottom first
    dz = 200.0
    sc = scenes.layered_scene(4, 4, k.size, 100.0, 100.0, dz, k_gas=k, ssa_gas=0.0, albedo=0.6)
    sza, F0, N = 35.0, 1000.0, 2_000_000
    mu0 = np.cos(np.deg2rad(sza))
    r = oracle.trace(sc, sza, 17.0, F0, N, seed=11, nthreads=NT)
    ref = refs.absorber_with_lambert(k, dz, mu0, 0.6, F0)
    area_cols = sc.ncol
    # surface direct: binomial counts
    n_dir = r.counts["sfc_dir"].sum()
    p = ref["sfc_dir"] / (F0 * mu0)
    assert abs(n_dir - N * p) < 4 * np.sqrt(N * p * (1 - p))
    assert r.counts["sfc_dif"].sum() == 0          # nothing scatters back down
    n_toa = r.counts["toa"].sum()
    q = ref["toa_up"] / (F0 * mu0)
    assert abs(n_toa - N * q) < 4 * np.sqrt(N * q * (1 - q))
    # per-layer absorption (track length), W m^-2 per layer = mean over columns * dz
    lay_dir = r.abs_dir.mean(axis=(1, 2)) * dz
    lay_dif = r.abs_dif.mean(axis=(1, 2)) * dz
    for got, want in ((lay_dir, ref["abs_dir_layers"]), (lay_dif, ref["abs_dif_layers"])):
        # track-length scores per photon are bounded by k dz / mu; SE bound from Bernoulli
        se = F0 * mu0 * np.sqrt(want / (F0 * mu0) / N) + 1e-9
        assert np.all(np.abs(got - want) < 6 * se), (got, want)
    # analog absorption counts estimate the same thing
    cnt = (r.abs_dir_cnt + r.abs_dif_cnt).mean(axis=(1, 2)) * dz
    tot = ref["abs_dir_layers"] + ref["abs_dif_layers"]
    se = F0 * mu0 * np.sqrt(tot / (F0 * mu0) / N)
    assert np.all(np.abs(cnt - tot) < 4 * se)
    assert area_cols == 16


def test_mc_no_atmosphere_normalisation():
    """Empty atmosphere, black surface: every photon lands as direct light, so
    the domain-mean direct irradiance is exactly F0 mu0 (normalisation, Sec. 2.3)."""
    sc = scenes.layered_scene(6, 5, 3, 50.0, 80.0, 100.0, k_gas=0.0, ssa_gas=0.0)
    r = oracle.trace(sc, 50.0, 123.0, 1000.0, 30_000, seed=2, nthreads=NT)
    assert np.isclose(r.sfc_dir.mean(), 1000.0 * np.cos(np.deg2rad(50.0)), rtol=1e-12)
    assert r.totals["sfc_abs"] == 30_000


def test_heating_rate_conversion_literal_factors():
    """The K/day conversion (reading c15 of the heating rates the paper quotes in
    K/day, Sec. 3): HR = 86400 A / (rho(z_c) c_p) with c_p = 1004 J/(kg K) and
    rho = 1.225 exp(-z_c / 8000 m) at the layer CENTRE. The factors below were
    evaluated by hand (not by the oracle) for dz = 25 m at z_c = 12.5 m (layer
    0) and z_c = 3187.5 m (layer 127), and for dz = 300 m at z_c = 150 m. A
    density taken at layer bottoms (z = 0, 3175 m), a wrong c_p, a missing
    86400, or a conversion broadcast along y or x instead of z fails here."""
    nz, ny, nx = 128, 2, 3
    a = np.zeros((nz, ny, nx))
    a[0, 1, 2] = 2.0          # W m^-3 in layer 0
    a[127, 0, 1] = 0.5        # W m^-3 in layer 127
    hr = oracle.heating_rate(a, 25.0)
    assert hr.shape == (nz, ny, nx)
    assert np.isclose(hr[0, 1, 2], 2.0 * 70.3594646098895, rtol=1e-12)
    assert np.isclose(hr[127, 0, 1], 0.5 * 104.63648654442953, rtol=1e-12)
    assert np.count_nonzero(hr) == 2
    # density profile itself: sea-level value 1.225 kg m^-3, scale height 8 km
    rho = oracle.air_density(2, 300.0)
    assert np.allclose(rho, [1.2022452424910, 1.1579959062988], rtol=1e-9)
    assert np.isclose(oracle.heating_rate(np.ones((1, 1, 1)), 300.0)[0, 0, 0], 71.57922015488663, rtol=1e-12)


def test_mc_conservative_black_surface_and_white_surface():
    """omega = 1 everywhere: nothing is absorbed in the atmosphere; with a white
    surface every photon leaves through the top (R = 1)."""
    sc = scenes.ellipsoid_scene(seed=0)
    sc.ssa_gas[:] = 1.0
    sc.ssa_cld[sc.k_cld > 0] = 1.0
    sc.albedo[:] = 0.0
    r = oracle.trace(sc, 30.0, 0.0, 1000.0, 100_000, seed=4, nthreads=NT)
    t = r.totals
    assert t["atm_abs"] == 0 and t["toa"] + t["sfc_abs"] == t["photons"]
    assert np.all(r.abs_dir == 0) and np.all(r.abs_dif == 0)
    sc.albedo[:] = 1.0
    r = oracle.trace(sc, 30.0, 0.0, 1000.0, 50_000, seed=5, nthreads=NT)
    assert r.totals["toa"] == 50_000
    assert np.isclose(r.toa_up.mean(), 1000.0 * np.cos(np.deg2rad(30.0)), rtol=1e-12)


def test_mc_energy_closure_per_photon(small_scene):
    r = oracle.trace(small_scene, 30.0, 0.0, 1000.0, 2 ** 17, seed=21, nthreads=NT)
    t = r.totals
    assert t["photons"] == t["toa"] + t["atm_abs"] + t["sfc_abs"]
    assert t["atm_abs"] == int(r.counts["abs_dir"].sum() + r.counts["abs_dif"].sum())
    assert t["sfc_abs"] == int(r.counts["sfc_abs"].sum())
    assert t["toa"] == int(r.counts["toa"].sum())


def _thin_slab(k_gas, w_gas, k_cld, w_cld, g_cld, tau):
    nz = 1
    dz = tau / (k_gas + k_cld)
    return scenes.layered_scene(2, 2, nz, 100.0, 100.0, dz, k_gas=k_gas, ssa_gas=w_gas,
                                k_cld=k_cld, ssa_cld=w_cld, g_cld=g_cld)


@pytest.mark.parametrize("sza,phase", [(0.0, "rayleigh"), (60.0, "rayleigh"), (0.0, "hg"),
                                       (60.0, "hg")])
def test_mc_thin_slab_single_scattering(sza, phase):
    """Optically thin slab (tau = 2e-3): reflectance and diffuse transmittance
    equal the exact single-scattering integrals up to O(tau^2) multiple
    scattering. The oblique HG case pins the direction rotation."""
    tau, omega, g = 2e-3, 0.5, 0.86
    if phase == "rayleigh":
        sc = _thin_slab(1.0, omega, 0.0, 0.0, 0.0, tau)
        pdf = refs.rayleigh_pdf
    else:
        sc = _thin_slab(0.0, 0.0, 1.0, omega, g, tau)
        pdf = lambda m: refs.hg_pdf(m, g)   # noqa: E731
    mu0 = np.cos(np.deg2rad(sza)) if sza > 0 else 1.0 - 1e-12
    N = 8_000_000
    r = oracle.trace(sc, sza, 10.0, 1.0, N, seed=31, nthreads=NT)
    R = r.totals["toa"] / N
    Td = r.counts["sfc_dif"].sum() / N
    R1 = refs.single_scatter_reflectance(pdf, mu0, tau, omega)
    T1 = refs.single_scatter_transmittance(pdf, mu0, tau, omega)
    for got, want in ((R, R1), (Td, T1)):
        se = np.sqrt(want / N)
        bias = 3 * (omega * tau / mu0) * want   # generous bound on double scattering
        assert abs(got - want) < 4 * se + bias, (got, want, se)


@pytest.mark.parametrize("mode", [0, 1])
def test_mc_scatterer_choice(mode):
    """Gas (Rayleigh, omega 1) and cloud (HG g=0.86, omega 0.2) mixed with equal
    extinction: the probability of a cloud scattering is k_sca,cloud / k_sca
    (mode 0, the reading adopted here) or k_ext,cloud / k_ext (mode 1, the
    paper's literal ratio). The thin-slab reflectance differs by 1.6x."""
    tau = 2e-3
    sc = _thin_slab(0.5, 1.0, 0.5, 0.2, 0.86, tau)
    mu0 = 1.0 - 1e-12
    N = 8_000_000
    r = oracle.trace(sc, 0.0, 0.0, 1.0, N, seed=41, nthreads=NT, pcld_mode=mode)
    Rr = refs.single_scatter_reflectance(refs.rayleigh_pdf, mu0, tau)
    Rh = refs.single_scatter_reflectance(lambda m: refs.hg_pdf(m, 0.86), mu0, tau)
    if mode == 0:
        want = 0.5 * 1.0 * Rr + 0.5 * 0.2 * Rh
    else:
        want = 0.6 * (0.5 * Rr + 0.5 * Rh)
    R = r.totals["toa"] / N
    assert abs(R - want) < 4 * np.sqrt(want / N) + 3 * tau * want


def test_mc_isotropic_slab_against_collision_probabilities():
    """Multiple scattering: homogeneous slab (tau 1, omega 0.9, isotropic = HG
    with g 0) over a black surface against the collision-probability solution."""
    tau_star, omega, sza = 1.0, 0.9, 36.87
    mu0 = np.cos(np.deg2rad(sza))
    nz = 10
    k = 1e-3
    dz = tau_star / (k * nz)
    sc = scenes.layered_scene(2, 2, nz, 100.0, 100.0, dz, k_gas=0.0, ssa_gas=0.0, k_cld=k,
                              ssa_cld=omega, g_cld=0.0)
    ref = refs.isotropic_slab_cp(tau_star, omega, mu0, M=400)
    ref2 = refs.isotropic_slab_cp(tau_star, omega, mu0, M=800)
    assert abs(ref["R"] - ref2["R"]) < 1e-5 and abs(ref["T_dif"] - ref2["T_dif"]) < 1e-5
    N = 4_000_000
    r = oracle.trace(sc, sza, 0.0, 1.0, N, seed=51, nthreads=NT)
    cnt = r.counts
    for got_n, want in ((r.totals["toa"], ref["R"]), (cnt["sfc_dif"].sum(), ref["T_dif"]),
                        (cnt["sfc_dir"].sum(), ref["T_dir"])):
        assert abs(got_n / N - want) < 4 * np.sqrt(want * (1 - want) / N)
    # absorbed fraction per grid layer (bottom first in the grid; top first in ref)
    A = ref["A_layers"].reshape(nz, -1).sum(1)[::-1]
    got = (cnt["abs_dir"] + cnt["abs_dif"]).sum(axis=(1, 2)) / N
    assert np.all(np.abs(got - A) < 4 * np.sqrt(A / N))
    # the track-length estimator of the same absorption, in photons per layer
    tl = (r.abs_dir + r.abs_dif).sum(axis=(1, 2)) * (sc.dx * sc.dy * dz) / r.energy / N
    assert np.all(np.abs(tl - A) < 4 * np.sqrt(A / N))


# --- reproducibility and partition invariance -----------------------------------------

def test_partition_and_thread_invariance(small_scene):
    N = 40_000
    full = oracle.trace(small_scene, 30.0, 0.0, 1000.0, N, seed=8, nthreads=4)
    one = oracle.trace(small_scene, 30.0, 0.0, 1000.0, N, seed=8, nthreads=1)
    a = oracle.trace(small_scene, 30.0, 0.0, 1000.0, N // 2, seed=8, photons_total=N, nthreads=3)
    b = oracle.trace(small_scene, 30.0, 0.0, 1000.0, N - N // 2, seed=8, id_begin=N // 2,
                     photons_total=N, nthreads=2)
    for key in full.counts:
        assert np.array_equal(full.counts[key], one.counts[key])
        assert np.array_equal(full.counts[key], a.counts[key] + b.counts[key])
    assert np.allclose(full.abs_dif, a.abs_dif + b.abs_dif, rtol=1e-12, atol=0)
    assert np.allclose(full.sfc_dif, a.sfc_dif + b.sfc_dif, rtol=1e-12, atol=0)


def test_track_length_matches_analog_counts(small_scene):
    """Both absorption estimators have the same expectation (column sums)."""
    means = []
    for s in range(8):
        r = oracle.trace(small_scene, 30.0, 0.0, 1000.0, 2 ** 16, seed=100 + s, nthreads=NT)
        means.append((r.abs3d.sum(), (r.abs_dir_cnt + r.abs_dif_cnt).sum()))
    m = np.array(means)
    d = m[:, 0] - m[:, 1]
    assert abs(d.mean()) < 4 * d.std(ddof=1) / np.sqrt(len(d)) + 1e-12


# --- diffuse share of the top boundary (Sec. 2.3) --------------------------------------

def test_mc_diffuse_fraction_in_an_empty_atmosphere():
    """No atmosphere, black surface: the surface receives (1-f) F mu0 direct and
    f F mu0 diffuse, exactly in expectation (binomial in the photon counts)."""
    sc = scenes.layered_scene(4, 4, 3, 50.0, 50.0, 100.0, k_gas=0.0, ssa_gas=0.0)
    N, f = 400_000, 0.3
    r = oracle.trace(sc, 40.0, 0.0, 1000.0, N, seed=3, nthreads=NT, diffuse_fraction=f)
    nd = r.counts["sfc_dif"].sum()
    assert abs(nd - f * N) < 4 * np.sqrt(N * f * (1 - f))
    assert r.counts["sfc_dir"].sum() + nd == N


def test_mc_diffuse_fraction_through_an_absorbing_slab():
    """Isotropic downwelling radiance crosses a purely absorbing slab of optical
    depth tau with flux transmittance 2 E3(tau)."""
    k = np.array([1e-3, 3e-3], dtype=np.float32)
    dz = 150.0
    sc = scenes.layered_scene(3, 3, 2, 100.0, 100.0, dz, k_gas=k, ssa_gas=0.0)
    N = 1_000_000
    r = oracle.trace(sc, 20.0, 0.0, 1.0, N, seed=9, nthreads=NT, diffuse_fraction=1.0)
    tau = float(np.sum(k.astype(np.float64)) * dz)
    p = 2 * refs.e3(tau)
    n = r.counts["sfc_dif"].sum()
    assert r.counts["sfc_dir"].sum() == 0
    assert abs(n - p * N) < 4 * np.sqrt(N * p * (1 - p))


def test_homogenize_layer_means():
    """Sec. 2.4 homogenisation: a field that already is horizontally uniform is
    left alone (a mean over the wrong axis would change it), a field varying
    only in x becomes its x-mean in every layer, and layer sums are kept."""
    nz, ny, nx = 4, 3, 5
    zonly = np.broadcast_to(np.arange(1.0, nz + 1)[:, None, None], (nz, ny, nx)).copy()
    assert np.array_equal(oracle.homogenize(zonly), zonly)
    xonly = np.broadcast_to(np.array([1.0, 2.0, 4.0, 8.0, 16.0])[None, None, :], (nz, ny, nx)).copy()
    assert np.allclose(oracle.homogenize(xonly), 31.0 / 5.0, rtol=0, atol=1e-15)
    rng = np.random.default_rng(0)
    f = rng.random((nz, ny, nx))
    h = oracle.homogenize(f)
    for k in range(nz):                      # brute force: each layer's own mean
        tot = 0.0
        for j in range(ny):
            for i in range(nx):
                tot += f[k, j, i]
        assert np.allclose(h[k], tot / (nx * ny), rtol=1e-15, atol=0)
    assert np.allclose(oracle.homogenize(h), h, rtol=1e-15, atol=0)
    s2 = rng.random((ny, nx))
    assert np.allclose(oracle.homogenize(s2), s2.mean(), rtol=1e-15, atol=0)


# --- Sobol start positions (Sec. 2.3) -------------------------------------------------

# Natural-order points 0..7 of the first two Sobol dimensions (dimension 1 is the
# van der Corput sequence; dimension 2 from the polynomial x + 1), as fractions.
SOBOL2_FIRST8 = [(0, 0), (1 / 2, 1 / 2), (1 / 4, 3 / 4), (3 / 4, 1 / 4), (1 / 8, 5 / 8), (5 / 8, 1 / 8),
                 (3 / 8, 3 / 8), (7 / 8, 7 / 8)]


def _is_net(pts: np.ndarray, m: int) -> bool:
    """Each of the 2^m elementary boxes of every shape 2^-a x 2^-b (a + b = m)
    holds exactly one of the 2^m points."""
    x, y = pts[:, 0].astype(np.uint64), pts[:, 1].astype(np.uint64)
    for a in range(m + 1):
        b = m - a
        box = (x >> np.uint64(32 - a)) * np.uint64(1 << b) + (y >> np.uint64(32 - b)) if m else x * 0
        if np.unique(box).size != (1 << m):
            return False
    return True


def test_sobol_points_and_net_property():
    pts = oracle.sobol2(1 << 12)
    assert [tuple(p) for p in pts[:8] / 2.0 ** 32] == SOBOL2_FIRST8
    for m in range(1, 11):
        for blk in range(2):                   # the first two aligned blocks of 2^m points
            assert _is_net(pts[blk << m:(blk + 1) << m], m), m
    # a random digital shift (XOR with one word per axis) keeps the net property
    rng = np.random.default_rng(4)
    sx, sy = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
    sh = pts ^ np.array([sx, sy], dtype=np.uint32)
    for m in (3, 6, 9):
        assert _is_net(sh[:1 << m], m)
    # a plain random sample is not a net (the check has teeth)
    assert not _is_net(rng.integers(0, 2 ** 32, size=(512, 2), dtype=np.uint64).astype(np.uint32), 9)
    # the continuation far along the sequence: points 2^20 .. 2^20 + 2^8 form a net too
    assert _is_net(oracle.sobol2(256, 1 << 20), 8)


def test_sobol_birth_is_unbiased_and_stratifies_the_direct_beam(small_scene):
    """With Sobol start points the surface direct irradiance still has the
    deterministic Beer-Lambert column means as its expectation, and its error
    per column is smaller than with uniform random starts at equal photons."""
    sc = small_scene
    F, sza, az = 1000.0, 30.0, 30.0
    truth = F * np.cos(np.deg2rad(sza)) * oracle.direct_beam(sc, sza, az, nsub=16)
    N = 16 * sc.ncol
    err = {}
    for birth in ("philox", "sobol"):
        runs = [oracle.trace(sc, sza, az, F, N, 900 + s, birth=birth).sfc_dir for s in range(8)]
        r = np.stack(runs)
        m = r.mean(axis=0)
        se = r.std(axis=0, ddof=1).mean() / np.sqrt(len(runs))
        assert abs(m.mean() - truth.mean()) < 4 * se + 1e-9, birth
        err[birth] = np.sqrt(((r - truth) ** 2).mean())
    assert err["sobol"] < 0.7 * err["philox"], err


# --- symmetries of the periodic domain ------------------------------------------------

_SYM_FIELDS = ("abs_dir", "abs_dif", "sfc_dir", "sfc_dif", "toa_up")


def _oracle_batches(scene, sza, az, photons, seeds):
    out = {f: [] for f in _SYM_FIELDS}
    for s in seeds:
        r = oracle.trace(scene, sza, az, 1000.0, photons, s)
        for k in _SYM_FIELDS:
            out[k].append(getattr(r, k))
    return {k: np.stack(v) for k, v in out.items()}


def _with_fields(scene, fn):
    """A copy of `scene` with `fn` applied to every optics field ([nz][ny][nx])
    and to the albedo ([ny][nx])."""
    import copy
    sc = copy.deepcopy(scene)
    for name in ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld"):
        setattr(sc, name, np.ascontiguousarray(fn(getattr(scene, name))))
    sc.albedo = np.ascontiguousarray(fn(scene.albedo[None])[0])
    return sc


def _assert_same_expectation(a, b, pa, pb):
    for field in _SYM_FIELDS:
        rep = refs.parity_report(a[field], b[field], pilot=(pa[field], pb[field]))
        assert rep["frac_over"] <= rep["bound"], (field, rep["frac_over"], rep["bound"])
        assert rep["pooled_p_family"] >= 1e-3, (field, rep["pooled_p_family"])
        assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-9, (field, rep["domain_rel"])


def test_oracle_overhead_sun_commutes_with_swapping_x_and_y():
    """With the sun overhead no horizontal axis is preferred: the x-y transposed
    scene gives the transposed fields (independent batches, the parity
    statistic). A swapped index or spacing in the fine-cell walk fails it."""
    sc = scenes.ellipsoid_scene(seed=3)
    sw = _with_fields(sc, lambda a: np.swapaxes(a, -1, -2))
    sw.nx, sw.ny, sw.dx, sw.dy = sc.ny, sc.nx, sc.dy, sc.dx
    n = 2 ** 19
    a = _oracle_batches(sc, 0.0, 0.0, n, range(3100, 3112))
    b = _oracle_batches(sw, 0.0, 0.0, n, range(3200, 3212))
    pa = _oracle_batches(sc, 0.0, 0.0, n, range(3300, 3306))
    pb = _oracle_batches(sw, 0.0, 0.0, n, range(3400, 3406))
    t = lambda d: {k: np.swapaxes(v, -1, -2) for k, v in d.items()}   # noqa: E731
    _assert_same_expectation(t(b), a, t(pb), pa)


def test_oracle_scene_rolled_by_whole_cells_gives_rolled_fields():
    """Periodic x and y: rolling the scene by (11, 5) cells, which carries the
    clouds across both lateral edges, rolls the fields by the same cells under
    a slanted sun whose paths cross the edges. A wrong wrap in the walk or in
    the birth column fails it."""
    sc = scenes.ellipsoid_scene(seed=2)
    dy, dx = 5, 11
    sh = _with_fields(sc, lambda a: np.roll(a, (dy, dx), axis=(-2, -1)))
    n = 2 ** 19
    a = _oracle_batches(sc, 45.0, 60.0, n, range(3500, 3512))
    b = _oracle_batches(sh, 45.0, 60.0, n, range(3600, 3612))
    pa = _oracle_batches(sc, 45.0, 60.0, n, range(3700, 3706))
    pb = _oracle_batches(sh, 45.0, 60.0, n, range(3800, 3806))
    back = lambda d: {k: np.roll(v, (-dy, -dx), axis=(-2, -1)) for k, v in d.items()}   # noqa: E731
    _assert_same_expectation(back(b), a, back(pb), pa)
