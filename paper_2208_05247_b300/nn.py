"""Python binding of the denoiser kernels declared in include/nn.h.

Argument marshalling only: tensors are CUDA torch tensors (device memory and
streams come from torch); every computation runs in librt_b300.so.
"""
from __future__ import annotations

import ctypes

from .rt import library

NN_OK = 0
NN_CONV_AUTO, NN_CONV_MMA_SYNC, NN_CONV_TCGEN05, NN_CONV_TCGEN05_TAP, NN_CONV_TCGEN05_HALO = 0, 1, 2, 3, 4

_sig_done = False


def _lib():
    global _sig_done
    lib = library()
    if not _sig_done:
        P, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_float, ctypes.c_double
        sig = {
            "nn_last_error": ([], ctypes.c_char_p),
            "nn_set_conv_path": ([i32], i32),
            "nn_status": ([P], i32),
            "nn_conv3d_fwd": ([P, P, P, P, P] + [i32] * 8 + [P], i32),
            "nn_conv3d_wgrad": ([P, P, P, P] + [i32] * 7 + [P], i32),
            "nn_relu_bwd": ([P, P, i64, P], i32),
            "nn_pool2_fwd": ([P, P] + [i32] * 5 + [P], i32),
            "nn_pool2_bwd": ([P, P] + [i32] * 5 + [P], i32),
            "nn_up2_fwd": ([P, P] + [i32] * 7 + [P], i32),
            "nn_up2_bwd": ([P, P] + [i32] * 7 + [P], i32),
            "nn_copy_channels": ([P, i32, i32, P, i32, i32, i64, i32, i32, P], i32),
            "nn_mse": ([P, i32, P, i32, P, P, i64, P, P], i32),
            "nn_adam": ([P, P, P, P, i64, f32, f32, f32, f32, i32, f32, P], i32),
            "nn_ema": ([P, P, i64, f32, P], i32),
            "nn_weights_bf16": ([P, P, P, i32, i32, i32, P], i32),
            "nn_pack_inputs": ([P] * 11 + [i32] * 3 + [f64, f64, P], i32),
            "nn_direct_transmittance": ([P, P] + [i32] * 3 + [f64] * 5 + [P, P, P], i32),
            "nn_direct_surface": ([P, P] + [i32] * 3 + [f64] * 5 + [i32, P, P], i32),
            "nn_pack_targets": ([P] * 7 + [i32] * 3 + [f64, f64, P], i32),
            "nn_unpack": ([P, P, i32, P, P, P] + [i32] * 3 + [f64, f64, P], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _sig_done = True
    return lib


class NnError(RuntimeError):
    pass


def _check(rc):
    if rc != NN_OK:
        raise NnError(_lib().nn_last_error().decode())


def _p(t):
    return None if t is None else t.data_ptr()


def _s(stream):
    return None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)


def nn_set_conv_path(path: int) -> int:
    """Select the 3x3x3 convolution kernel (NN_CONV_*); returns the previous choice."""
    old = _lib().nn_set_conv_path(int(path))
    if old < 0:
        raise NnError(_lib().nn_last_error().decode())
    return old


def nn_status(stream=None):
    """Wait for the stream; raise if a tcgen05 convolution gave up waiting."""
    _check(_lib().nn_status(_s(stream)))


def nn_conv3d_fwd(x, wt, bias, out_bf16, out_f32, N, D, H, W, Cin, Cout, ksize, relu, stream=None):
    _check(_lib().nn_conv3d_fwd(_p(x), _p(wt), _p(bias), _p(out_bf16), _p(out_f32), N, D, H, W, Cin, Cout, ksize,
                                int(relu), _s(stream)))


def nn_conv3d_wgrad(x, gout, gw, gb, N, D, H, W, Cin, Cout, ksize, stream=None):
    _check(_lib().nn_conv3d_wgrad(_p(x), _p(gout), _p(gw), _p(gb), N, D, H, W, Cin, Cout, ksize, _s(stream)))


def nn_relu_bwd(y, g, stream=None):
    _check(_lib().nn_relu_bwd(_p(y), _p(g), g.numel(), _s(stream)))


def nn_pool2_fwd(x, out, N, D, H, W, C, stream=None):
    _check(_lib().nn_pool2_fwd(_p(x), _p(out), N, D, H, W, C, _s(stream)))


def nn_pool2_bwd(gout, gin, N, D, H, W, C, stream=None):
    _check(_lib().nn_pool2_bwd(_p(gout), _p(gin), N, D, H, W, C, _s(stream)))


def nn_up2_fwd(x, out, N, d, h, w, C, Cdst, c0, stream=None):
    _check(_lib().nn_up2_fwd(_p(x), _p(out), N, d, h, w, C, Cdst, c0, _s(stream)))


def nn_up2_bwd(gout, gin, N, d, h, w, C, Csrc, c0, stream=None):
    _check(_lib().nn_up2_bwd(_p(gout), _p(gin), N, d, h, w, C, Csrc, c0, _s(stream)))


def nn_copy_channels(src, Csrc, s0, dst, Cdst, d0, vox, C, accumulate=False, stream=None):
    _check(_lib().nn_copy_channels(_p(src), Csrc, s0, _p(dst), Cdst, d0, vox, C, int(accumulate), _s(stream)))


def nn_mse(pred, Cp, target, Cuse, chw, grad, vox, loss, stream=None):
    _check(_lib().nn_mse(_p(pred), Cp, _p(target), Cuse, _p(chw), _p(grad), vox, _p(loss), _s(stream)))


def nn_adam(W, m, v, grad, lr, step, b1=0.9, b2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    _check(_lib().nn_adam(_p(W), _p(m), _p(v), _p(grad), W.numel(), lr, b1, b2, eps, step, weight_decay,
                          _s(stream)))


def nn_ema(avg, W, decay, stream=None):
    """avg = decay * avg + (1 - decay) * W (FP32 CUDA tensors of equal size)."""
    _check(_lib().nn_ema(_p(avg), _p(W), W.numel(), float(decay), _s(stream)))


def nn_weights_bf16(W, wt, wd, ksize, Cin, Cout, stream=None):
    _check(_lib().nn_weights_bf16(_p(W), _p(wt), _p(wd), ksize, Cin, Cout, _s(stream)))


def nn_pack_inputs(abs3d, sfc_dir, sfc_dif, k_gas, ssa_gas, k_cld, ssa_cld, g_cld, out, D, H, W, dz, flux,
                   stream=None, t3d=None, t2d=None):
    _check(_lib().nn_pack_inputs(*[_p(t) for t in (abs3d, sfc_dir, sfc_dif, k_gas, ssa_gas, k_cld, ssa_cld, g_cld,
                                                    t3d, t2d, out)], D, H, W, float(dz), float(flux), _s(stream)))


def nn_direct_transmittance(k_gas, k_cld, D, H, W, dx, dy, dz, sza_deg, azimuth_deg, t3d, t2d, stream=None):
    _check(_lib().nn_direct_transmittance(_p(k_gas), _p(k_cld), D, H, W, float(dx), float(dy), float(dz),
                                          float(sza_deg), float(azimuth_deg), _p(t3d), _p(t2d), _s(stream)))


def nn_direct_surface(k_gas, k_cld, D, H, W, dx, dy, dz, sza_deg, azimuth_deg, nsub, t2d, stream=None):
    _check(_lib().nn_direct_surface(_p(k_gas), _p(k_cld), D, H, W, float(dx), float(dy), float(dz), float(sza_deg),
                                    float(azimuth_deg), int(nsub), _p(t2d), _s(stream)))


def nn_pack_targets(abs_hi, sdir_hi, sdif_hi, abs_lo, sdir_lo, sdif_lo, out, D, H, W, dz, flux, stream=None):
    _check(_lib().nn_pack_targets(*[_p(t) for t in (abs_hi, sdir_hi, sdif_hi, abs_lo, sdir_lo, sdif_lo, out)],
                                  D, H, W, float(dz), float(flux), _s(stream)))


def nn_unpack(x, pred, Cp, abs3d, sfc_dir, sfc_dif, D, H, W, dz, flux, stream=None):
    _check(_lib().nn_unpack(_p(x), _p(pred), Cp, _p(abs3d), _p(sfc_dir), _p(sfc_dif), D, H, W, float(dz),
                            float(flux), _s(stream)))


def nn_last_error() -> str:
    return _lib().nn_last_error().decode()
