"""The time-to-RMSE arithmetic behind the denoiser speed-ups (CPU only):
the plain tracer's RMSE is modelled as a / sqrt(ppc) (Monte Carlo error falls
as N^-1/2, Sec. 3.2); its wall time is interpolated between the measured
runs (a least-squares line is reported beside it). Also the training loop's
guard bookkeeping, driven by a fake network."""
import math

import numpy as np
import pytest

from paper_2208_05247_b300 import denoise

PPC = (4, 16, 64, 256, 1024)


def test_exact_model_is_recovered():
    a, t0, t1 = 417.0, 2.6, 0.0167
    rmse = [a / math.sqrt(p) for p in PPC]
    ms = [t0 + t1 * p for p in PPC]
    f0, f1 = denoise.plain_time_fit(PPC, ms)
    assert math.isclose(f0, t0, rel_tol=1e-9) and math.isclose(f1, t1, rel_tol=1e-9)
    for target in (200.0, 13.0, 8.0, 0.5):
        assert math.isclose(denoise.plain_ppc_to_match(PPC, rmse, target), (a / target) ** 2, rel_tol=1e-12)


def test_prefactor_is_the_geometric_mean():
    """Run-to-run scatter whose factors multiply to one leaves a unchanged."""
    a = 7.25
    f = [1.1, 1 / 1.1, 1.0, 1.05, 1 / 1.05]
    rmse = [a / math.sqrt(p) * k for p, k in zip(PPC, f)]
    assert math.isclose(denoise.plain_ppc_to_match(PPC, rmse, 0.0785), (a / 0.0785) ** 2, rel_tol=1e-12)
    # halving the target error needs four times the photons
    r1 = denoise.plain_ppc_to_match(PPC, rmse, 0.2)
    assert math.isclose(denoise.plain_ppc_to_match(PPC, rmse, 0.1), 4 * r1, rel_tol=1e-12)


def test_time_fit_is_least_squares():
    rng = np.random.default_rng(0)
    ms = [2.6 + 0.0167 * p + e for p, e in zip(PPC, rng.normal(0, 0.05, len(PPC)))]
    t0, t1 = denoise.plain_time_fit(PPC, ms)
    A = np.stack([np.ones(len(PPC)), np.array(PPC, float)], 1)
    want = np.linalg.lstsq(A, np.array(ms), rcond=None)[0]
    assert np.allclose([t0, t1], want, rtol=1e-10, atol=1e-12)


def test_truth_noise_term():
    """Errors against a noisy truth of Nt photons/column: rmse^2 =
    a^2 (1/p + 1/Nt) for plain runs. The prefactor and the match are then
    recovered exactly, and the match lies beyond the naive a/sqrt(p) one
    (part of the measured target error is the truth's own noise)."""
    a, nt = 331.0, 16384
    rmse = [a * math.sqrt(1.0 / p + 1.0 / nt) for p in PPC]
    for n_true in (100.0, 1810.0, 8000.0):
        target = a * math.sqrt(1.0 / n_true + 1.0 / nt)      # a run of n_true photons, measured the same way
        got = denoise.plain_ppc_to_match(PPC, rmse, target, truth_ppc=nt)
        assert math.isclose(got, n_true, rel_tol=1e-9)
        if n_true > 1000:    # where the truth's noise is a visible part of the target error
            assert got > 1.08 * denoise.plain_ppc_to_match(PPC, rmse, target)
    # at or below the truth's noise floor no plain run can be matched
    assert denoise.plain_ppc_to_match(PPC, rmse, a / math.sqrt(nt), truth_ppc=nt) == math.inf
    # the noise-free-truth limit is the plain a / sqrt(p) model
    assert math.isclose(denoise.plain_ppc_to_match(PPC, [a / math.sqrt(p) for p in PPC], 8.0, truth_ppc=None),
                        (a / 8.0) ** 2, rel_tol=1e-12)


class _FakeNet:
    """Stands in for the U-Net in `denoise.train`: plays back a loss sequence
    and records the learning rate of every optimizer step and every rollback."""

    def __init__(self, losses):
        self.losses = list(losses)
        self.rates, self.rollbacks_at, self.decays, self.k = [], [], [], 0

    def forward(self, x, shape):
        pass

    def loss_and_grad(self, target, shape, chw):
        self.k += 1
        return _Scalar(self.losses[self.k - 1])

    def backward(self, x, shape):
        pass

    def step(self, rate):
        self.rates.append((self.k, rate))

    def ema(self, decay):
        self.decays.append(decay)

    def apply_ema(self):
        pass

    def rollback(self):
        self.rollbacks_at.append(self.k)


class _Scalar:
    def __init__(self, v):
        self.v = v

    def item(self):
        return self.v


def test_training_recovers_after_a_rollback(monkeypatch):
    """32 non-finite losses in a row roll the weights back to their average.
    The averaged weights may score far above the best running loss; the
    running loss and its lowest value restart, so the loop trains on instead
    of skipping and rolling back for ever, and the learning rate rises from
    the ramp's start again instead of resuming at full rate."""
    from types import SimpleNamespace

    import torch

    from paper_2208_05247_b300 import denoise
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    n = 600
    losses = [0.02] * 300 + [float("nan")] * 32 + [0.5] * (n - 332)
    net = _FakeNet(losses)
    samples = [SimpleNamespace(x=None, shape=None, target=None)] * n
    denoise.train(net, samples, epochs=1, lr=1e-3, lr_final=1e-3, chw=[1.0], warmup=0.1)
    assert net.rollbacks_at == [332]
    assert net.train_log == {"skipped_steps": 32, "rollbacks": 1}
    rate = dict(net.rates)
    ramp = 0.1 * n
    # before: the ramp from step 1, full rate once it ends
    assert rate[1] == pytest.approx(1e-3 / ramp)
    assert rate[300] == pytest.approx(1e-3)
    # skipped steps take no optimizer step; every step after the rollback does
    assert not any(301 <= k <= 332 for k in rate)
    assert all(k in rate for k in range(333, n + 1))
    # after the rollback the ramp starts again
    assert rate[333] == pytest.approx(1e-3 / ramp)
    assert rate[350] == pytest.approx(1e-3 * 18 / ramp)
    assert rate[332 + int(ramp)] == pytest.approx(1e-3)
    # the moving average follows the weights early on: decay (1 + n) / (10 + n)
    assert net.decays[0] == pytest.approx(2 / 11)
    assert net.decays[-1] == pytest.approx(1 - 10 / n)


def test_speedup_bracket_from_the_runs_either_side():
    ppc = (4, 16, 64, 256)
    rmse = (8.0, 4.0, 2.0, 1.0)
    ms = (1.0, 2.0, 5.0, 17.0)
    # target 1.5 lies between the 64- and 256-photon runs
    assert denoise.speedup_bracket(ppc, rmse, ms, 1.5, 0.5) == [10.0, 34.0]
    # the direct-beam solve is added to every plain time
    assert denoise.speedup_bracket(ppc, rmse, ms, 1.5, 0.5, extra_ms=0.5) == [11.0, 35.0]
    # an error equal to a run's counts as reached by that run
    assert denoise.speedup_bracket(ppc, rmse, ms, 2.0, 1.0) == [2.0, 5.0]
    # below every run: only a lower bound; above every run: only an upper one
    assert denoise.speedup_bracket(ppc, rmse, ms, 0.5, 1.0) == [17.0, None]
    assert denoise.speedup_bracket(ppc, rmse, ms, 9.0, 1.0) == [None, 1.0]
    # the order of the runs does not matter
    assert denoise.speedup_bracket(ppc[::-1], rmse[::-1], ms[::-1], 1.5, 0.5) == [10.0, 34.0]


def test_plain_time_interpolates_between_the_runs():
    ppc = (4, 16, 64, 256)
    ms = (1.5, 2.0, 3.0, 7.0)
    # at a run: its time; between two runs: linear in photons/column
    assert denoise.plain_time_at(ppc, ms, 16) == 2.0
    assert denoise.plain_time_at(ppc, ms, 40) == pytest.approx(2.5)
    assert denoise.plain_time_at(ppc, ms, 160) == pytest.approx(5.0)
    # below the smallest run: that run's time (the launch floor)
    assert denoise.plain_time_at(ppc, ms, 1) == 1.5
    # beyond the largest: at the rate of the last two runs (4 ms per 192)
    assert denoise.plain_time_at(ppc, ms, 448) == pytest.approx(11.0)
    assert denoise.plain_time_at(ppc, ms, math.inf) == math.inf
    # measured plain times of one short evaluation: the least-squares line
    # through them, pulled by the 16384-photon run, starts below zero
    runs = (4, 16, 64, 256, 1024, 4096, 16384)
    times = (1.50, 1.79, 2.47, 4.09, 10.08, 36.21, 192.79)
    t0, t1 = denoise.plain_time_fit(runs, times)
    assert t0 + t1 * 4 < 0.0
    assert denoise.plain_time_at(runs, times, 4) == 1.50
    assert denoise.plain_time_at(runs, times, 2048) == pytest.approx(10.08 + (36.21 - 10.08) / 3)
