"""The cell-wise parity criterion, calibrated on the CPU: two independent
oracle runs of the same scene must pass it (no false alarm), and a run with a
planted 3 % error in the cloud scattering albedo must fail it."""
import numpy as np

import oracle
from tests import refs


def _batches(scene, seeds, n):
    out = {f: [] for f in oracle.FIELDS}
    for s in seeds:
        r = oracle.trace(scene, 30.0, 0.0, 1000.0, n, s)
        for f in oracle.FIELDS:
            out[f].append(getattr(r, f))
    return {f: np.stack(v) for f, v in out.items()}


def test_criterion_passes_for_independent_oracle_runs(small_scene):
    a = _batches(small_scene, range(1000, 1016), 2 ** 15)
    b = _batches(small_scene, range(2000, 2016), 2 ** 15)
    pa = _batches(small_scene, range(1100, 1108), 2 ** 15)
    pb = _batches(small_scene, range(2100, 2108), 2 ** 15)
    for f in oracle.FIELDS:
        rep = refs.parity_report(a[f], b[f], pilot=(pa[f], pb[f]))
        assert rep["frac_over"] <= rep["bound"], (f, rep["frac_over"], rep["bound"])
        assert rep["pooled_p_family"] >= 1e-3, (f, rep["pooled_max_abs_z"], rep["pooled_p_family"])
        assert abs(rep["domain_rel"]) < 4 * rep["domain_rel_se"] + 1e-12
        assert rep["ks_d"] <= rep["ks_bound"], (f, rep["ks_d"], rep["ks_bound"])


def test_criterion_catches_a_planted_error(small_scene):
    import copy
    wrong = copy.deepcopy(small_scene)
    cloudy = wrong.k_cld > 0
    wrong.ssa_cld[cloudy] = np.float32(0.97)          # planted: 3 % cloud absorption
    a = _batches(small_scene, range(3000, 3016), 2 ** 15)
    b = _batches(wrong, range(4000, 4016), 2 ** 15)
    pa = _batches(small_scene, range(3100, 3104), 2 ** 15)
    pb = _batches(wrong, range(4100, 4104), 2 ** 15)
    rep = refs.parity_report(a["sfc_dif"], b["sfc_dif"], pilot=(pa["sfc_dif"], pb["sfc_dif"]))
    assert rep["frac_over"] > rep["bound"] or abs(rep["domain_rel"]) > 4 * rep["domain_rel_se"]
    # each criterion alone also catches it
    assert rep["ks_d"] > rep["ks_bound"], (rep["ks_d"], rep["ks_bound"])
    rep3 = refs.parity_report(a["abs_dif"], b["abs_dif"], pilot=(pa["abs_dif"], pb["abs_dif"]))
    assert rep3["frac_over"] > rep3["bound"] and rep3["ks_d"] > rep3["ks_bound"]
