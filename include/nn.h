/*
 * nn.h -- C ABI of the BF16 tensor-core kernels behind the learned denoiser.
 *
 * The paper traces every field at 256 samples per pixel and reports that the
 * error falls only as N^-1/2 while the cost grows as N (Sec. 3.2). The denoiser
 * built on these kernels (a 3D U-Net) maps a field traced with few photons,
 * plus the optics, to the field a high photon count would give. The paper has
 * no denoiser; these kernels are its training and inference path.
 *
 * Conventions
 *   - Activations and activation gradients: BF16, channels last,
 *     [N][D][H][W][C] (C fastest), device memory. Convolutions need C_in a
 *     multiple of 16.
 *   - Master weights and weight gradients: FP32 [taps][C_in][C_out] with
 *     taps = 27 (3x3x3, tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)) or 1 (1x1x1).
 *     The convolution kernel reads BF16 weights in [taps][C_out][C_in]
 *     ("wt") and, for the input gradient, [taps][C_in][C_out] with the taps
 *     reversed ("wd"); nn_weights_bf16 writes both.
 *   - Padding is "same" with zeros outside the volume.
 *   - All products are accumulated in FP32 (BF16 inputs). 3x3x3 convolutions
 *     with output channels a multiple of 16 run on tcgen05.mma with
 *     tensor-memory accumulators and TMA-staged operands; the others, the
 *     1x1x1 convolutions and the weight gradient use mma.sync.
 *   - Every call is ordered on `stream` (NULL = default stream) and returns
 *     NN_OK or a negative NN_E_* code; nn_last_error() gives the message.
 */
#ifndef NN_B300_H
#define NN_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { NN_OK = 0, NN_E_INVAL = -1, NN_E_CUDA = -3, NN_E_DEVICE = -4 };

const char *nn_last_error(void);

/* Which kernel nn_conv3d_fwd uses for 3x3x3 convolutions:
 *   NN_CONV_AUTO         tcgen05 where supported (Cin and Cout multiples of 16),
 *                        else mma.sync
 *   NN_CONV_MMA_SYNC     always the mma.sync kernel
 *   NN_CONV_TCGEN05      always tcgen05 (NN_E_INVAL for unsupported shapes): the
 *                        halo-tiled persistent kernel when its shared memory
 *                        fits (at most 64 output channels per tile), else the
 *                        per-tap kernel
 *   NN_CONV_TCGEN05_TAP  always the per-tap tcgen05 kernel
 *   NN_CONV_TCGEN05_HALO always the halo-tiled kernel; NN_E_INVAL where it does
 *                        not fit
 * 1x1x1 convolutions always use the mma.sync kernel. Process-wide; returns the
 * previous setting. */
enum { NN_CONV_AUTO = 0, NN_CONV_MMA_SYNC = 1, NN_CONV_TCGEN05 = 2, NN_CONV_TCGEN05_TAP = 3,
       NN_CONV_TCGEN05_HALO = 4 };
int nn_set_conv_path(int path);

/* Wait for `stream`, then report and clear device-side failures of the
 * tcgen05 kernels: NN_E_DEVICE if one of their bounded waits gave up (the
 * outputs of that launch are then incomplete), else NN_OK. */
int nn_status(void *stream);

/* out[p][o] = act(bias[o] + sum_t sum_i in[p + off(t)][i] W[t][i][o]) with
 * act = ReLU if relu != 0. wt: BF16 [taps][Cout][Cin]. bias may be NULL.
 * Writes out_bf16 (BF16 [vox][Cout], Cout even) and/or out_f32 (FP32). With
 * the input gradient of a convolution as `in` and its "wd" weights, this is
 * the gradient with respect to that convolution's input (Cin, Cout swapped). */
int nn_conv3d_fwd(const void *in, const void *wt, const float *bias, void *out_bf16, float *out_f32, int N, int D,
                  int H, int W, int Cin, int Cout, int ksize, int relu, void *stream);

/* gw[t][i][o] += sum_p in[p + off(t)][i] gout[p][o]; gb[o] += sum_p gout[p][o]
 * (gb may be NULL). FP32 atomics: zero gw and gb first. Channels multiples of 8.
 * 3x3x3 kernels with channel counts that are multiples of 16 run on tcgen05
 * (unless NN_CONV_MMA_SYNC is selected): the (tap, input channel) rows and the
 * voxel reduction are transposed into the tensor core's operand layout in
 * shared memory by the CTA's threads. */
int nn_conv3d_wgrad(const void *in, const void *gout, float *gw, float *gb, int N, int D, int H, int W, int Cin,
                    int Cout, int ksize, void *stream);

/* g[i] = 0 where y[i] <= 0 (gradient through ReLU, y the ReLU output). */
int nn_relu_bwd(const void *y, void *g, long long n, void *stream);

/* 2x2x2 average pooling [N][D][H][W][C] -> [N][D/2][H/2][W/2][C] and its gradient. */
int nn_pool2_fwd(const void *in, void *out, int N, int D, int H, int W, int C, void *stream);
int nn_pool2_bwd(const void *gout, void *gin, int N, int D, int H, int W, int C, void *stream);

/* Nearest 2x upsampling of [N][d][h][w][C] into channels [c0, c0+C) of a
 * [N][2d][2h][2w][Cdst] tensor, and its gradient (sum over the 8 children). */
int nn_up2_fwd(const void *in, void *out, int N, int d, int h, int w, int C, int Cdst, int c0, void *stream);
int nn_up2_bwd(const void *gout, void *gin, int N, int d, int h, int w, int C, int Csrc, int c0, void *stream);

/* dst[v][d0 + c] (+)= src[v][s0 + c] for c < C over vox voxels (concatenation
 * and its gradient). */
int nn_copy_channels(const void *src, int Csrc, int s0, void *dst, int Cdst, int d0, long long vox, int C,
                     int accumulate, void *stream);

/* Mean weighted squared error of FP32 pred [vox][Cp] (channels < Cuse) against
 * FP32 target [vox][Cuse], channel weights chw (NULL = 1); writes the BF16
 * gradient [vox][Cp] and ADDS the loss to *loss (device double). */
int nn_mse(const float *pred, int Cp, const float *target, int Cuse, const float *chw, void *grad, long long vox,
           double *loss, void *stream);

/* One Adam step (bias-corrected, optional decoupled-style L2 term) on FP32
 * master parameters; step counts from 1. */
int nn_adam(float *W, float *m, float *v, const float *grad, long long n, float lr, float b1, float b2, float eps,
            int step, float weight_decay, void *stream);

/* Exponential moving average of parameters: avg = decay avg + (1 - decay) W
 * over n FP32 values (weights averaged over the last steps of training). */
int nn_ema(float *avg, const float *W, long long n, float decay, void *stream);

/* BF16 copies of FP32 W [taps][Cin][Cout]: wt [taps][Cout][Cin] for the
 * forward pass and wd [taps][Cin][Cout] with reversed taps for the input
 * gradient (either may be NULL). */
int nn_weights_bf16(const float *W, void *wt, void *wd, int ksize, int Cin, int Cout, void *stream);

/* Direct-beam transmittance toward the sun (Sec. 2.3: "direct" radiation is
 * the never-scattered part, whose expectation is Beer-Lambert along the sun
 * ray): exp(-integral of k_gas + k_cld) from each voxel centre to the domain
 * top, t3d FP32 [D][H][W], and from each column's centre at the surface,
 * t2d FP32 [H][W]. An exact walk over the fine cells (cell sizes dx, dy, dz,
 * periodic in x and y) in FP32; optical depths above 30 give 0. A feature
 * of the optics for the denoiser. */
int nn_direct_transmittance(const float *k_gas, const float *k_cld, int D, int H, int W, double dx, double dy,
                            double dz, double sza_deg, double azimuth_deg, float *t3d, float *t2d, void *stream);

/* Pixel-mean direct-beam transmittance at the surface, t2d FP32 [H][W]: the
 * mean of exp(-integral of (k_gas + k_cld) ds) toward the sun over nsub x nsub
 * surface points on a midpoint grid of each column (Sec. 2.3: direct radiation
 * is the never-scattered part, so toa_flux cos(sza) t2d is the expectation of
 * the traced surface direct irradiance). The march through the fine cells
 * (periodic in x and y) runs in FP32; one warp per column sums its points in a
 * fixed order, so the result is deterministic. Optical depths above 30 give 0.
 * nsub 1..32; NN_E_INVAL otherwise or for a solar zenith angle outside
 * [0, 90). k_gas, k_cld [D][H][W] and t2d are device buffers. */
int nn_direct_surface(const float *k_gas, const float *k_cld, int D, int H, int W, double dx, double dy, double dz,
                      double sza_deg, double azimuth_deg, int nsub, float *t2d, void *stream);

/* Denoiser inputs from a traced field (FP64 [D][H][W] absorption [W m^-3],
 * [H][W] surface direct/diffuse [W m^-2]) and the optics (FP32 [D][H][W]):
 * BF16 [D][H][W][16] with channels 0: 100 A dz / F, 1: direct / F, 2: diffuse
 * / F (surface values repeated in every layer), 3: log(tau_cell + 1e-4) / 5,
 * 4: k_sca / k_ext, 5: cloud g, 6: direct transmittance of the voxel (t3d),
 * 7: direct transmittance of the column at the surface (t2d), 8..15: 0.
 * t3d and t2d may be NULL (channels 6 and 7 then 0). F = toa_flux cos(sza)
 * [W m^-2]. */
int nn_pack_inputs(const double *abs3d, const double *sfc_dir, const double *sfc_dif, const float *k_gas,
                   const float *ssa_gas, const float *k_cld, const float *ssa_cld, const float *g_cld,
                   const float *t3d, const float *t2d, void *out, int D, int H, int W, double dz, double flux,
                   void *stream);

/* Training targets FP32 [D][H][W][3]: channels 0..2 of the high-photon field
 * minus those of the low-photon field (as BF16-rounded inputs hold them). */
int nn_pack_targets(const double *abs_hi, const double *sdir_hi, const double *sdif_hi, const double *abs_lo,
                    const double *sdir_lo, const double *sdif_lo, float *out, int D, int H, int W, double dz,
                    double flux, void *stream);

/* Denoised fields: input channel + predicted correction (pred FP32 [vox][Cp]),
 * back to W m^-3 and W m^-2. Every layer of a column predicts the surface
 * correction (channels 1 and 2); the surface fields take the column mean. */
int nn_unpack(const void *in, const float *pred, int Cp, double *abs3d, double *sfc_dir, double *sfc_dif, int D,
              int H, int W, double dz, double flux, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NN_B300_H */
