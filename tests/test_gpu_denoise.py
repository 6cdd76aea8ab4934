"""The learned denoiser end to end: pairs traced by the tracer itself, the
U-Net trained with the library's own forward/backward kernels, and what it
gains over the method without it (the plain 4-photon field) on held-out scenes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2208_05247_b300 import build, denoise  # noqa: E402


def test_unet_gradient_matches_finite_difference_of_the_loss():
    """Directional derivative of the loss through the whole U-Net (BF16
    forward) against the kernels' backward pass, on a small volume."""
    build.build()
    shape = (8, 16, 16)
    rng = np.random.default_rng(0)
    net = denoise.UNet(seed=1)
    V = int(np.prod(shape))
    x = torch.from_numpy(rng.normal(size=V * 16).astype(np.float32)).cuda().to(torch.bfloat16)
    tgt = torch.from_numpy(rng.normal(size=V * 3).astype(np.float32)).cuda()
    chw = torch.ones(3, device="cuda")
    net.forward(x, shape)
    net.loss_and_grad(tgt, shape, chw)
    net.backward(x, shape)
    layer = net.dec[2][1]                       # a full-resolution decoder convolution
    d = torch.from_numpy(rng.normal(size=layer.W.numel()).astype(np.float32)).cuda().view_as(layer.W)
    d *= 0.05 * layer.W.abs().mean() / d.abs().mean()
    analytic = float((layer.gW * d).sum())
    W0 = layer.W.clone()
    vals = []
    for s in (+1.0, -1.0):
        layer.W.copy_(W0 + s * d)
        layer.refresh()
        net.forward(x, shape)
        vals.append(float(net.loss_and_grad(tgt, shape, chw).item()))
    layer.W.copy_(W0)
    layer.refresh()
    numeric = (vals[0] - vals[1]) / 2.0
    assert np.sign(numeric) == np.sign(analytic)
    assert abs(numeric - analytic) < 0.1 * abs(analytic) + 1e-5, (numeric, analytic)


def test_trained_denoiser_beats_the_noisy_input_on_held_out_scenes():
    build.build()
    shape = (128, 64, 64)
    pairs = denoise.make_pairs(list(range(2000, 2064)), shape, workers=8)
    net = denoise.UNet(seed=0)
    losses = denoise.train(net, pairs, epochs=12, lr=1e-3)
    assert losses[-1][1] < 0.7 * losses[0][1]
    res = denoise.evaluate(net, list(range(2100, 2106)), shape, truth_ppc=2048, plain_ppc=(4, 16, 64),
                           workers=8, repeats=1)
    d, n = res["denoised"], res["noisy_input"]
    # what the network gains over the plain 4-photon field (the method without it)
    assert d["rmse_ghi"] < 0.9 * n["rmse_ghi"], res
    assert d["rmse_hr"] < 0.6 * n["rmse_hr"], res
    # the exact pixel-mean direct beam is far closer to the truth than the 4-photon tally
    c = res["surface"]["rmse"]
    assert c["exact_dir"] < 0.3 * c["noisy_dir"], res["surface"]
