"""Pins of the numpy FP64 reference of the denoiser's layers: brute-force sums,
finite differences of the loss through every layer, and adjoint identities."""
import numpy as np
import pytest

from oracle import nn_ref


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3d_against_brute_force_sum():
    rng = _rng(1)
    x = rng.normal(size=(2, 3, 4, 5, 3))
    W = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    out = nn_ref.conv3d(x, W, b)
    N, D, H, Wd, C = x.shape
    for (n, z, y, xx, o) in [(0, 0, 0, 0, 0), (1, 2, 3, 4, 1), (0, 1, 2, 2, 1), (1, 0, 3, 0, 0)]:
        s = b[o]
        for t, (dz, dy, dx) in enumerate(nn_ref.taps(3)):
            zz, yy, xq = z + dz, y + dy, xx + dx
            if 0 <= zz < D and 0 <= yy < H and 0 <= xq < Wd:
                s += sum(x[n, zz, yy, xq, i] * W[t, i, o] for i in range(C))
        assert np.isclose(out[n, z, y, xx, o], s, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("ksize", [1, 3])
def test_conv3d_gradients_by_finite_differences(ksize):
    rng = _rng(2)
    x = rng.normal(size=(1, 3, 3, 4, 2))
    W = rng.normal(size=(len(nn_ref.taps(ksize)), 2, 3))
    b = rng.normal(size=3)
    gout = rng.normal(size=(1, 3, 3, 4, 3))
    f = lambda x_, W_, b_: float((gout * nn_ref.conv3d(x_, W_, b_, ksize)).sum())  # noqa: E731
    gx, gW, gb = nn_ref.conv3d_backward(x, W, gout, ksize)
    h = 1e-6
    for idx in [(0, 0, 0, 0, 0), (0, 2, 1, 3, 1), (0, 1, 2, 2, 0)]:
        e = np.zeros_like(x); e[idx] = h
        assert np.isclose((f(x + e, W, b) - f(x - e, W, b)) / (2 * h), gx[idx], rtol=1e-6, atol=1e-8)
    for idx in [(0, 0, 0), (len(gW) - 1, 1, 2), (len(gW) // 2, 1, 0)]:
        e = np.zeros_like(W); e[idx] = h
        assert np.isclose((f(x, W + e, b) - f(x, W - e, b)) / (2 * h), gW[idx], rtol=1e-6, atol=1e-8)
    for o in range(3):
        e = np.zeros_like(b); e[o] = h
        assert np.isclose((f(x, W, b + e) - f(x, W, b - e)) / (2 * h), gb[o], rtol=1e-6, atol=1e-8)


def test_pool_and_upsample_adjoints():
    rng = _rng(3)
    x = rng.normal(size=(2, 4, 6, 2, 3))
    y = rng.normal(size=(2, 2, 3, 1, 3))
    # <pool2(x), y> = <x, pool2_backward(y)> and <up2(y), x> = <y, up2_backward(x)>
    assert np.isclose((nn_ref.pool2(x) * y).sum(), (x * nn_ref.pool2_backward(y)).sum(), rtol=1e-13)
    assert np.isclose((nn_ref.up2(y) * x).sum(), (y * nn_ref.up2_backward(x)).sum(), rtol=1e-13)
    assert np.isclose(nn_ref.pool2(x)[1, 1, 2, 0, 2], x[1, 2:4, 4:6, 0:2, 2].mean())


def test_mse_gradient_by_finite_differences():
    rng = _rng(4)
    pred = rng.normal(size=(5, 4))
    target = rng.normal(size=(5, 3))
    w = np.array([1.0, 2.0, 0.5])
    loss, g = nn_ref.mse(pred, target, w)
    assert np.all(g[:, 3] == 0)
    h = 1e-6
    e = np.zeros_like(pred); e[2, 1] = h
    assert np.isclose((nn_ref.mse(pred + e, target, w)[0] - nn_ref.mse(pred - e, target, w)[0]) / (2 * h), g[2, 1], rtol=1e-6)


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-30], np.float32)
    r = nn_ref.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0                  # 1 + 2^-8 is a tie: rounds to even
    assert r[2] == np.float32(1.0078125)
    assert abs(r[3] / vals[3] - 1) < 2 ** -8
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
