// nn_kernels.cu -- BF16 tensor-core kernels of the 3D U-Net denoiser.
//
// Activations are channels-last BF16, [N][D][H][W][C] with C a multiple of 16.
// A 3x3x3 ("same" padding) or 1x1x1 convolution is an implicit GEMM:
//   out[p][o] = bias[o] + sum_t sum_i in[p + off(t)][i] * W[t][i][o]
// with M = voxels, N = output channels, K = taps * input channels. Tiles of
// 128 voxels x 32 output channels are staged in shared memory with cp.async
// (zero fill outside the volume) and multiplied with mma.sync m16n8k16
// (BF16 inputs, FP32 accumulation).
//
// The kernel reads weights as Wt[t][o][i] (input channels contiguous). The
// gradient with respect to the input is the same kernel applied to the output
// gradient with Wd[t][o'][i'] = W[26 - t][o'][i'] (taps reversed, no transpose).
// The weight gradient gW[t][i][o] = sum_p in[p + off(t)][i] gout[p][o] is a
// GEMM over voxels, split across blocks and reduced with FP32 atomics.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nn.h"

namespace nn_tc {   // conv_tc.cu
bool supported(int Cin, int Cout);
int conv3d_fwd(const void *in, const void *wt, const float *bias, void *out_bf16, float *out_f32, int N, int D, int H,
               int W, int Cin, int Cout, int relu, cudaStream_t st, char *err, size_t errlen, int variant);
int take_status(cudaStream_t st, unsigned *out);
bool wgrad_supported(int Cin, int Cout);
int conv3d_wgrad(const void *in, const void *gout, float *gw, float *gb, int N, int D, int H, int W, int Cin,
                 int Cout, cudaStream_t st, char *err, size_t errlen);
}  // namespace nn_tc

namespace {

int g_conv_path = NN_CONV_AUTO;

constexpr int kBM = 128, kChunk = 16, kStageChunks = 2;
constexpr int kRow = 24;   // bf16 per staged row: 16 used + 8 pad (48 B: conflict-free fragment reads)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const int bytes = valid ? 16 : 0;   // 0 bytes read: the destination is zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ldmatrix: lane l supplies the address of row (l % 8) of 8x8 matrix (l / 8);
// register j receives this lane's part of matrix j (transposed with .trans).
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int tap_offset(int t, int taps, int &dz, int &dy, int &dx)
{
    if (taps == 1) { dz = dy = dx = 0; return 0; }
    dz = t / 9 - 1; dy = (t / 3) % 3 - 1; dx = t % 3 - 1;
    return 0;
}

// ---------------------------------------------------------------------------
// Convolution forward (also the input gradient with tap-reversed weights).
// Block tile 128 voxels x BN output channels; warps 4 (voxels) x BN/32
// (channels), each 32 x 32. Fragments come from shared memory by ldmatrix.
// grid (ceil(M/128), ceil(Cout/BN)), 4 * BN threads.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void __launch_bounds__(4 * BN) conv_fwd_kernel(const __nv_bfloat16 *__restrict__ in,
                                                          const __nv_bfloat16 *__restrict__ wt,
                                                          const float *__restrict__ bias, __nv_bfloat16 *out_bf,
                                                          float *out_f, int N, int D, int H, int W, int Cin,
                                                          int Cout, int taps, int relu)
{
    constexpr int NT = 4 * BN;
    __shared__ __align__(16) __nv_bfloat16 sA[2][kStageChunks][kBM][kRow];
    __shared__ __align__(16) __nv_bfloat16 sB[2][kStageChunks][BN][kRow];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, q = lane & 3;
    const int wm = warp & 3, wn = warp >> 2;
    const long long M = (long long)N * D * H * W;
    const long long m0 = (long long)blockIdx.x * kBM;
    const int co0 = blockIdx.y * BN;
    const int cpt = Cin / kChunk;           // chunks per tap
    const int nchunks = taps * cpt;

    // this thread stages voxel row `arow` of the A tile (halves ahalf0.. of it)
    const int arow = tid % kBM;
    const long long mv = m0 + arow;
    const bool mvalid = mv < M;
    int vz = 0, vy = 0, vx = 0;
    if (mvalid) {
        long long r = mv % ((long long)D * H * W);
        vz = (int)(r / (H * W)); r -= (long long)vz * H * W;
        vy = (int)(r / W); vx = (int)(r - (long long)vy * W);
    }

    auto stage = [&](int buf, int c0) {
        for (int c = 0; c < kStageChunks; ++c) {
            const int kc = c0 + c;
            const bool live = kc < nchunks;
            const int t = live ? kc / cpt : 0, ci0 = live ? (kc % cpt) * kChunk : 0;
            int dz, dy, dx;
            tap_offset(t, taps, dz, dy, dx);
            const int z = vz + dz, y = vy + dy, x = vx + dx;
            const bool ok = live && mvalid && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
            const long long nb = ok ? mv + ((long long)dz * H + dy) * W + dx : 0;
            const __nv_bfloat16 *src = in + nb * Cin + ci0;
            for (int h = tid / kBM; h < 2; h += NT / kBM)
                cp_async16(&sA[buf][c][arow][h * 8], src + h * 8, ok);
            if (tid < 2 * BN) {
                const int row = tid >> 1, half = tid & 1;
                const bool okb = live && (co0 + row) < Cout;
                const __nv_bfloat16 *wsrc = wt + ((long long)(t * Cout + (okb ? co0 + row : 0)) * Cin + ci0 + half * 8);
                cp_async16(&sB[buf][c][row][half * 8], wsrc, okb);
            }
        }
        cp_async_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;

    // ldmatrix row/column of this lane: A (16x16) and B (two 8-wide n tiles)
    const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lcol = (lane >> 4) * 8;
    const int brow = (lane & 7) + (lane >> 4) * 8, bcol = ((lane >> 3) & 1) * 8;

    const int nstages = (nchunks + kStageChunks - 1) / kStageChunks;
    stage(0, 0);
    for (int s = 0; s < nstages; ++s) {
        const int buf = s & 1;
        if (s + 1 < nstages) {
            stage(buf ^ 1, (s + 1) * kStageChunks);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kStageChunks; ++c) {
            if (s * kStageChunks + c < nchunks) {
                unsigned af[2][4], bf[2][4];
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) ldsm_x4(af[mi], &sA[buf][c][wm * 32 + mi * 16 + lrow][lcol]);
#pragma unroll
                for (int jp = 0; jp < 2; ++jp) ldsm_x4(bf[jp], &sB[buf][c][wn * 32 + jp * 16 + brow][bcol]);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                    for (int nj = 0; nj < 4; ++nj) {
                        const unsigned b2[2] = {bf[nj >> 1][(nj & 1) * 2], bf[nj >> 1][(nj & 1) * 2 + 1]};
                        mma_bf16(acc[mi][nj], af[mi], b2);
                    }
            }
        }
        __syncthreads();
    }

    // epilogue: bias, optional ReLU, BF16 and/or FP32 store
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long m = m0 + wm * 32 + mi * 16 + g + half * 8;
            if (m >= M) continue;
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) {
                const int co = co0 + wn * 32 + nj * 8 + q * 2;
                if (co >= Cout) continue;
                float v0 = acc[mi][nj][half * 2], v1 = acc[mi][nj][half * 2 + 1];
                if (bias) { v0 += bias[co]; v1 += (co + 1 < Cout) ? bias[co + 1] : 0.f; }
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                if (out_bf) {
                    if (co + 1 < Cout)
                        *reinterpret_cast<__nv_bfloat162 *>(out_bf + m * Cout + co) = __floats2bfloat162_rn(v0, v1);
                    else
                        out_bf[m * Cout + co] = __float2bfloat16_rn(v0);
                }
                if (out_f) {
                    out_f[m * Cout + co] = v0;
                    if (co + 1 < Cout) out_f[m * Cout + co + 1] = v1;
                }
            }
        }
}

// ---------------------------------------------------------------------------
// Weight gradient gW[t][i][o] += sum_p in[p + off(t)][i] * gout[p][o] (FP32),
// and (tap 0 blocks only, when gb != null) the bias gradient gb[o] += sum_p gout[p][o].
// grid (taps * ceil(Cin/32), ceil(Cout/32), splits), 128 threads: 2 x 2 warps of
// 16 input x 16 output channels; voxels in chunks of 32.
// ---------------------------------------------------------------------------
constexpr int kWV = 32;   // voxels per chunk
constexpr int kWRow = 40; // bf16 per staged row (32 channels + 8 pad, 80 B)

__global__ void __launch_bounds__(128) conv_wgrad_kernel(const __nv_bfloat16 *__restrict__ in,
                                                         const __nv_bfloat16 *__restrict__ gout, float *gw,
                                                         float *gb, int N, int D, int H, int W, int Cin, int Cout,
                                                         int taps, long long vox_per_split)
{
    __shared__ __align__(16) __nv_bfloat16 sI[kWV][kWRow];
    __shared__ __align__(16) __nv_bfloat16 sG[kWV][kWRow];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, q = lane & 3;
    const int iblocks = (Cin + 31) / 32;
    const int t = blockIdx.x / iblocks, i0 = (blockIdx.x % iblocks) * 32;
    const int o0 = blockIdx.y * 32;
    const long long M = (long long)N * D * H * W;
    const long long p_begin = (long long)blockIdx.z * vox_per_split;
    const long long p_end = min(M, p_begin + vox_per_split);
    int dz, dy, dx;
    tap_offset(t, taps, dz, dy, dx);
    const int wi = (warp >> 1) * 16, wo = (warp & 1) * 16;   // warp tile origin within the block tile
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    float bacc = 0.f;   // bias gradient: thread tid < 32 sums output channel o0 + tid

    // staging: thread -> (voxel row r = tid / 4, 16-byte column c16 = tid % 4)
    const int r = tid >> 2, c16 = tid & 3;
    for (long long p0 = p_begin; p0 < p_end; p0 += kWV) {
        const long long p = p0 + r;
        bool okg = p < p_end;
        bool oki = okg;
        long long nb = 0;
        if (okg) {
            long long rr = p % ((long long)D * H * W);
            const int z = (int)(rr / (H * W));
            rr -= (long long)z * H * W;
            const int y = (int)(rr / W), x = (int)(rr - (long long)y * W);
            oki = z + dz >= 0 && z + dz < D && y + dy >= 0 && y + dy < H && x + dx >= 0 && x + dx < W;
            nb = p + ((long long)dz * H + dy) * W + dx;
        }
        const int ci = i0 + c16 * 8, co = o0 + c16 * 8;
        cp_async16(&sI[r][c16 * 8], in + (oki && ci < Cin ? nb * Cin + ci : 0), oki && ci < Cin);
        cp_async16(&sG[r][c16 * 8], gout + (okg && co < Cout ? p * Cout + co : 0), okg && co < Cout);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kWV; kk += 16) {
            // A[m=i][k=p] = sI[p][i] and B[k=p][n=o] = sG[p][o]: both are the
            // transposes of the staged (voxel-major) tiles, read with ldmatrix.trans.
            // Matrix j of the A load: voxels kk + 8 (j >> 1) .., channels wi + 8 (j & 1) ..
            // Matrix j of the B load: voxels kk + 8 (j & 1) .., channels wo + 8 (j >> 1) ..
            unsigned a[4], bb[4];
            const int mj = lane >> 3, mr = lane & 7;
            ldsm_x4_trans(a, &sI[kk + (mj >> 1) * 8 + mr][wi + (mj & 1) * 8]);
            ldsm_x4_trans(bb, &sG[kk + (mj & 1) * 8 + mr][wo + (mj >> 1) * 8]);
            const unsigned b0[2] = {bb[0], bb[1]}, b1[2] = {bb[2], bb[3]};
            mma_bf16(acc[0], a, b0);
            mma_bf16(acc[1], a, b1);
        }
        if (gb && t == 0 && i0 == 0 && tid < 32)
            for (int v = 0; v < kWV; ++v) bacc += __bfloat162float(sG[v][tid]);
        __syncthreads();
    }
#pragma unroll
    for (int nj = 0; nj < 2; ++nj)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + wi + g + (e >> 1) * 8;
            const int o = o0 + wo + nj * 8 + q * 2 + (e & 1);
            if (i < Cin && o < Cout) atomicAdd(&gw[((long long)t * Cin + i) * Cout + o], acc[nj][e]);
        }
    if (gb && t == 0 && i0 == 0 && tid < 32 && o0 + tid < Cout) atomicAdd(&gb[o0 + tid], bacc);
}

// ---------------------------------------------------------------------------
// Elementwise and resampling kernels (grid-stride).
// ---------------------------------------------------------------------------
#define GRID_LOOP(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
                             i += (long long)gridDim.x * blockDim.x)

__global__ void relu_bwd_kernel(const __nv_bfloat16 *y, __nv_bfloat16 *g, long long n)
{
    GRID_LOOP(i, n) if (!(__bfloat162float(y[i]) > 0.f)) g[i] = __float2bfloat16_rn(0.f);
}

// 2x2x2 average pooling of [N][D][H][W][C] into [N][D/2][H/2][W/2][C]
__global__ void pool2_fwd_kernel(const __nv_bfloat16 *in, __nv_bfloat16 *out, int N, int D, int H, int W, int C)
{
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)N * d * h * w * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % w); v /= w;
        const int y = (int)(v % h); v /= h;
        const int z = (int)(v % d);
        const long long b = v / d;
        float s = 0.f;
        for (int e = 0; e < 8; ++e) {
            const long long src = (((b * D + 2 * z + (e >> 2)) * H + 2 * y + ((e >> 1) & 1)) * W + 2 * x + (e & 1)) * C + c;
            s += __bfloat162float(in[src]);
        }
        out[i] = __float2bfloat16_rn(0.125f * s);
    }
}

// gradient of the pooling: each fine voxel gets 1/8 of its coarse gradient
__global__ void pool2_bwd_kernel(const __nv_bfloat16 *gout, __nv_bfloat16 *gin, int N, int D, int H, int W, int C)
{
    const long long n = (long long)N * D * H * W * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % W); v /= W;
        const int y = (int)(v % H); v /= H;
        const int z = (int)(v % D);
        const long long b = v / D;
        const long long src = (((b * (D / 2) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c;
        gin[i] = __float2bfloat16_rn(0.125f * __bfloat162float(gout[src]));
    }
}

// nearest-neighbour 2x upsampling of [N][d][h][w][C] into channels [c0, c0+C) of
// a [N][2d][2h][2w][Cdst] tensor (the first half of a concatenation)
__global__ void up2_fwd_kernel(const __nv_bfloat16 *in, __nv_bfloat16 *out, int N, int d, int h, int w, int C,
                               int Cdst, int c0)
{
    const long long n = (long long)N * 8 * d * h * w * C;
    const int D = 2 * d, H = 2 * h, W = 2 * w;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % W); v /= W;
        const int y = (int)(v % H); v /= H;
        const int z = (int)(v % D);
        const long long b = v / D;
        const long long src = (((b * d + z / 2) * h + y / 2) * w + x / 2) * C + c;
        out[(((b * D + z) * H + y) * W + x) * (long long)Cdst + c0 + c] = in[src];
    }
}

// gradient of the upsampling: sum of the 8 fine gradients, read from channels
// [c0, c0+C) of the concatenated gradient
__global__ void up2_bwd_kernel(const __nv_bfloat16 *gout, __nv_bfloat16 *gin, int N, int d, int h, int w, int C,
                               int Csrc, int c0)
{
    const long long n = (long long)N * d * h * w * C;
    GRID_LOOP(i, n) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % w); v /= w;
        const int y = (int)(v % h); v /= h;
        const int z = (int)(v % d);
        const long long b = v / d;
        float s = 0.f;
        for (int e = 0; e < 8; ++e) {
            const long long src = (((b * 2 * d + 2 * z + (e >> 2)) * 2 * h + 2 * y + ((e >> 1) & 1)) * 2 * w +
                                   2 * x + (e & 1)) * (long long)Csrc + c0 + c;
            s += __bfloat162float(gout[src]);
        }
        gin[i] = __float2bfloat16_rn(s);
    }
}

// ---- 8-channel (16-byte) variants of the resampling and copy kernels ----
// Used when every channel count and offset is a multiple of 8 and the buffers
// are 16-byte aligned. One thread handles 8 channels of one coarse voxel (of
// one voxel for the copy), so the index arithmetic runs once per 16 bytes
// instead of once per element; I is the index type (32-bit when the counts
// fit). Per channel the arithmetic and its order are those of the scalar
// kernels above, so the results are bit-identical.
struct bf8 { __nv_bfloat162 h[4]; };

__device__ __forceinline__ void bf8_to_f(const uint4 &q, float (&f)[8])
{
    const bf8 b = *reinterpret_cast<const bf8 *>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(b.h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 f_to_bf8(const float (&f)[8])
{
    bf8 b;
#pragma unroll
    for (int j = 0; j < 4; ++j) b.h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return *reinterpret_cast<const uint4 *>(&b);
}

// coarse voxel (b, z, y, x) of i / G over a [N][d][h][w] grid
template <typename I>
__device__ __forceinline__ void coarse_index(I v, int d, int h, int w, I &b, int &z, int &y, int &x)
{
    x = (int)(v % (I)w); v /= (I)w;
    y = (int)(v % (I)h); v /= (I)h;
    z = (int)(v % (I)d);
    b = v / (I)d;
}

template <typename I>
__global__ void pool2_fwd_vec_kernel(const uint4 *in, uint4 *out, int N, int d, int h, int w, int G)
{
    const I n = (I)N * d * h * w * G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int g = (int)(i % (I)G);
        I b; int z, y, x;
        coarse_index<I>(i / (I)G, d, h, w, b, z, y, x);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int e = 0; e < 8; ++e) {
            const I src = ((b * (2 * d) + 2 * z + (e >> 2)) * (2 * h) + 2 * y + ((e >> 1) & 1)) * (2 * w) + 2 * x + (e & 1);
            float f[8];
            bf8_to_f(in[src * G + g], f);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += f[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] *= 0.125f;
        out[i] = f_to_bf8(s);
    }
}

template <typename I>
__global__ void pool2_bwd_vec_kernel(const uint4 *gout, uint4 *gin, int N, int d, int h, int w, int G)
{
    const I n = (I)N * d * h * w * G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int g = (int)(i % (I)G);
        I b; int z, y, x;
        coarse_index<I>(i / (I)G, d, h, w, b, z, y, x);
        float f[8];
        bf8_to_f(gout[i], f);
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] *= 0.125f;
        const uint4 q = f_to_bf8(f);
        for (int e = 0; e < 8; ++e) {
            const I dst = ((b * (2 * d) + 2 * z + (e >> 2)) * (2 * h) + 2 * y + ((e >> 1) & 1)) * (2 * w) + 2 * x + (e & 1);
            gin[dst * G + g] = q;
        }
    }
}

template <typename I>
__global__ void up2_fwd_vec_kernel(const uint4 *in, uint4 *out, int N, int d, int h, int w, int G, int Gdst, int g0)
{
    const I n = (I)N * d * h * w * G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int g = (int)(i % (I)G);
        I b; int z, y, x;
        coarse_index<I>(i / (I)G, d, h, w, b, z, y, x);
        const uint4 q = in[i];
        for (int e = 0; e < 8; ++e) {
            const I dst = ((b * (2 * d) + 2 * z + (e >> 2)) * (2 * h) + 2 * y + ((e >> 1) & 1)) * (2 * w) + 2 * x + (e & 1);
            out[dst * Gdst + g0 + g] = q;
        }
    }
}

template <typename I>
__global__ void up2_bwd_vec_kernel(const uint4 *gout, uint4 *gin, int N, int d, int h, int w, int G, int Gsrc, int g0)
{
    const I n = (I)N * d * h * w * G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int g = (int)(i % (I)G);
        I b; int z, y, x;
        coarse_index<I>(i / (I)G, d, h, w, b, z, y, x);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int e = 0; e < 8; ++e) {
            const I src = ((b * (2 * d) + 2 * z + (e >> 2)) * (2 * h) + 2 * y + ((e >> 1) & 1)) * (2 * w) + 2 * x + (e & 1);
            float f[8];
            bf8_to_f(gout[src * Gsrc + g0 + g], f);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += f[j];
        }
        gin[i] = f_to_bf8(s);
    }
}

template <typename I>
__global__ void copy_channels_vec_kernel(const uint4 *src, int Gs, int s0, uint4 *dst, int Gd, int d0, I vox, int G,
                                         int accumulate)
{
    const I n = vox * (I)G;
    for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const I v = i / (I)G;
        const int g = (int)(i - v * (I)G);
        const uint4 x = src[v * Gs + s0 + g];
        uint4 &y = dst[v * Gd + d0 + g];
        if (accumulate) {
            float a[8], c[8];
            bf8_to_f(y, a);
            bf8_to_f(x, c);
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] += c[j];
            y = f_to_bf8(a);
        } else {
            y = x;
        }
    }
}

// copy C channels between tensors with channel strides Csrc / Cdst and offsets
__global__ void copy_channels_kernel(const __nv_bfloat16 *src, int Csrc, int s0, __nv_bfloat16 *dst, int Cdst, int d0,
                                     long long vox, int C, int accumulate)
{
    GRID_LOOP(i, vox * C) {
        const long long v = i / C;
        const int c = (int)(i % C);
        const __nv_bfloat16 x = src[v * Csrc + s0 + c];
        __nv_bfloat16 &y = dst[v * Cdst + d0 + c];
        y = accumulate ? __float2bfloat16_rn(__bfloat162float(y) + __bfloat162float(x)) : x;
    }
}

// weighted squared error on channels [0, Cuse) of pred [vox][Cp] (FP32) against
// target [vox][Cuse] (FP32); writes d loss / d pred (BF16, zero in unused
// channels) and adds the loss to *loss. mask[v] (optional) weights voxels.
__global__ void mse_kernel(const float *pred, int Cp, const float *target, int Cuse, const float *chw,
                           __nv_bfloat16 *grad, long long vox, double inv_count, double *loss)
{
    double local = 0.0;
    GRID_LOOP(i, vox * Cp) {
        const long long v = i / Cp;
        const int c = (int)(i % Cp);
        float gval = 0.f;
        if (c < Cuse) {
            const float d = pred[i] - target[v * Cuse + c];
            const float wgt = chw ? chw[c] : 1.f;
            local += (double)(wgt * d * d);
            gval = (float)(2.0 * inv_count) * wgt * d;
        }
        grad[i] = __float2bfloat16_rn(gval);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local != 0.0) atomicAdd(loss, local * inv_count);
}

// Adam (FP32 master weights) followed by the two BF16 layouts the kernels read:
// wt[t][o][i] for the forward pass, wd[t][o'=i][i'=o] with reversed taps for the
// input gradient. W, m, v, grad: [taps][Cin][Cout]. Bias uses the same update
// with taps = 1, Cin = 1 and no BF16 copies.
__global__ void adam_kernel(float *W, float *m, float *v, const float *grad, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2, float wdecay)
{
    GRID_LOOP(i, n) {
        const float gr = grad[i] + wdecay * W[i];
        const float mi = b1 * m[i] + (1.f - b1) * gr;
        const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        W[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void ema_kernel(float *avg, const float *W, long long n, float decay)
{
    GRID_LOOP(i, n) avg[i] = fmaf(decay, avg[i] - W[i], W[i]);
}

__global__ void weights_bf16_kernel(const float *W, __nv_bfloat16 *wt, __nv_bfloat16 *wd, int taps, int Cin, int Cout)
{
    GRID_LOOP(idx, (long long)taps * Cin * Cout) {
        const int o = (int)(idx % Cout);
        const long long r = idx / Cout;
        const int i = (int)(r % Cin), t = (int)(r / Cin);
        const __nv_bfloat16 b = __float2bfloat16_rn(W[idx]);
        if (wt) wt[((long long)t * Cout + o) * Cin + i] = b;
        if (wd) wd[((long long)(taps - 1 - t) * Cin + i) * Cout + o] = b;
    }
}

// ---------------------------------------------------------------------------
// Denoiser input/output packing. Fields are the tracer's: FP64 [D][H][W] 3D
// absorption [W m^-3] and [H][W] surface direct/diffuse [W m^-2]; optics FP32
// [D][H][W]. F = toa_flux * cos(sza) is the horizontal flux into the domain.
// Channels (BF16, 16 per voxel):
//   0 absorbed fraction per cell, 100 * A dz / F   (noisy)
//   1 surface direct / F  (noisy; the column's value in every layer)
//   2 surface diffuse / F (noisy; likewise)
//   3 log(tau_cell + 1e-4) / 5 with tau_cell = (k_gas + k_cld) dz
//   4 single-scattering albedo of the cell, k_sca / k_ext (1 where k_ext = 0)
//   5 cloud asymmetry g
//   6..15 zero
// Targets (FP32, 3 per voxel) are the same first three quantities of the
// high-photon field MINUS the noisy input (the network predicts a correction).
// ---------------------------------------------------------------------------
// Direct-beam transmittance exp(-integral of k_ext) from each voxel centre,
// and from each column's centre at the surface, to the domain top along the
// direction toward the sun (vx, vy, vz), vz > 0: an exact walk over the fine
// cells with periodic x and y. Walks stop once the optical depth passes 30
// (transmittance below 1e-13, stored as 0) or after a bound on the steps.
__global__ void direct_transmittance_kernel(const float *kg, const float *kc, int D, int H, int W, float dx,
                                            float dy, float dz, float vx, float vy, float vz, float *t3, float *t2)
{
    const long long n3 = (long long)D * H * W, n = n3 + (long long)H * W;
    const int max_steps = 4 * (D + H + W) + 64;
    const float ax = fabsf(vx), ay = fabsf(vy);
    const float stx = ax > 0.f ? dx / ax : INFINITY, sty = ay > 0.f ? dy / ay : INFINITY, stz = dz / vz;
    const int sx = vx > 0.f ? 1 : -1, sy = vy > 0.f ? 1 : -1;
    GRID_LOOP(q, n) {
        int i, j, k;
        float fz;                                  // start height within the first cell, in cells
        if (q < n3) {
            i = (int)(q % W); j = (int)((q / W) % H); k = (int)(q / ((long long)W * H)); fz = 0.5f;
        } else {
            const long long c = q - n3;
            i = (int)(c % W); j = (int)(c / W); k = 0; fz = 0.f;
        }
        // distances along the ray to the next face per axis (start at the cell's centre in x and y)
        float tx = ax > 0.f ? 0.5f * stx : INFINITY, ty = ay > 0.f ? 0.5f * sty : INFINITY;
        float tz = (1.f - fz) * stz, t = 0.f, tau = 0.f;
        for (int s = 0; s < max_steps; ++s) {
            const long long cell = ((long long)k * H + j) * W + i;
            const float tm = fminf(tx, fminf(ty, tz));
            tau = fmaf(kg[cell] + kc[cell], tm - t, tau);
            t = tm;
            if (tau > 30.f) break;
            if (tm == tz) {
                if (++k >= D) break;
                tz += stz;
            } else if (tm == tx) {
                i += sx;
                i = i < 0 ? W - 1 : i >= W ? 0 : i;
                tx += stx;
            } else {
                j += sy;
                j = j < 0 ? H - 1 : j >= H ? 0 : j;
                ty += sty;
            }
        }
        const float T = tau > 30.f ? 0.f : expf(-tau);
        if (q < n3) t3[q] = T;
        else t2[q - n3] = T;
    }
}

// One warp per surface column: lane l marches the sub-points l, l + 32, ...
// of the column's nsub x nsub midpoint grid toward the sun; the warp sums in
// a fixed butterfly order.
__global__ void direct_surface_kernel(const float *kg, const float *kc, int D, int H, int W, float dx, float dy,
                                      float dz, float vx, float vy, float vz, int nsub, float *t2)
{
    const int lane = threadIdx.x & 31;
    const long long ncol = (long long)H * W;
    const int max_steps = 4 * (D + H + W) + 64;
    const float ax = fabsf(vx), ay = fabsf(vy);
    const float stx = ax > 0.f ? dx / ax : INFINITY, sty = ay > 0.f ? dy / ay : INFINITY, stz = dz / vz;
    const int sx = vx > 0.f ? 1 : -1, sy = vy > 0.f ? 1 : -1;
    const int npts = nsub * nsub;
    for (long long col = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; col < ncol;
         col += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int ci = (int)(col % W), cj = (int)(col / W);
        float acc = 0.f;
        for (int q = lane; q < npts; q += 32) {
            const float fx = ((q % nsub) + 0.5f) / nsub, fy = ((q / nsub) + 0.5f) / nsub;
            int i = ci, j = cj, k = 0;
            float tx = ax > 0.f ? (vx > 0.f ? 1.f - fx : fx) * stx : INFINITY;
            float ty = ay > 0.f ? (vy > 0.f ? 1.f - fy : fy) * sty : INFINITY;
            float tz = stz, t = 0.f, tau = 0.f;
            for (int s = 0; s < max_steps; ++s) {
                const long long cell = ((long long)k * H + j) * W + i;
                const float tm = fminf(tx, fminf(ty, tz));
                tau = fmaf(kg[cell] + kc[cell], tm - t, tau);
                t = tm;
                if (tau > 30.f) break;
                if (tm == tz) {
                    if (++k >= D) break;
                    tz += stz;
                } else if (tm == tx) {
                    i += sx;
                    i = i < 0 ? W - 1 : i >= W ? 0 : i;
                    tx += stx;
                } else {
                    j += sy;
                    j = j < 0 ? H - 1 : j >= H ? 0 : j;
                    ty += sty;
                }
            }
            acc += tau > 30.f ? 0.f : expf(-tau);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) t2[col] = acc / (float)npts;
    }
}

// s_abs = 100 dz / F and s_sfc = 1 / F come from the host: FP64 divisions
// are slow on this GPU, and a product with the reciprocal moves the value by
// at most an FP64 ulp or two before it is rounded to FP32 and BF16.
__global__ void pack_inputs_kernel(const double *abs3d, const double *sdir, const double *sdif, const float *kg,
                                   const float *wg, const float *kc, const float *wc, const float *gc,
                                   const float *t3, const float *t2, __nv_bfloat16 *out, int D, int H, int W,
                                   float dz, double s_abs, double s_sfc)
{
    const long long n = (long long)D * H * W;
    GRID_LOOP(v, n) {
        const long long col = v % ((long long)H * W);
        const float ke = kg[v] + kc[v];
        const float ks = kg[v] * wg[v] + kc[v] * wc[v];
        float ch[16];
        ch[0] = (float)(abs3d[v] * s_abs);
        ch[1] = (float)(sdir[col] * s_sfc);
        ch[2] = (float)(sdif[col] * s_sfc);
        ch[3] = logf(ke * dz + 1e-4f) / 5.0f;
        ch[4] = ke > 0.f ? ks / ke : 1.0f;
        ch[5] = gc[v];
        ch[6] = t3 ? t3[v] : 0.f;
        ch[7] = t2 ? t2[col] : 0.f;
        for (int c = 8; c < 16; ++c) ch[c] = 0.f;
        __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(out + v * 16);
        for (int c = 0; c < 8; ++c) o[c] = __floats2bfloat162_rn(ch[2 * c], ch[2 * c + 1]);
    }
}

__global__ void pack_targets_kernel(const double *abs_hi, const double *sdir_hi, const double *sdif_hi,
                                    const double *abs_lo, const double *sdir_lo, const double *sdif_lo,
                                    float *out, int D, int H, int W, double s_abs, double s_sfc)
{
    const long long n = (long long)D * H * W;
    GRID_LOOP(v, n) {
        const long long col = v % ((long long)H * W);
        // the noisy value exactly as the input channel holds it (BF16-rounded)
        const float lo0 = __bfloat162float(__float2bfloat16_rn((float)(abs_lo[v] * s_abs)));
        const float lo1 = __bfloat162float(__float2bfloat16_rn((float)(sdir_lo[col] * s_sfc)));
        const float lo2 = __bfloat162float(__float2bfloat16_rn((float)(sdif_lo[col] * s_sfc)));
        out[v * 3 + 0] = (float)(abs_hi[v] * s_abs) - lo0;
        out[v * 3 + 1] = (float)(sdir_hi[col] * s_sfc) - lo1;
        out[v * 3 + 2] = (float)(sdif_hi[col] * s_sfc) - lo2;
    }
}

// denoised fields: noisy input channel + predicted correction, back to
// physical units; surface fields from the mean correction over each column
// s_out = F / (100 dz) from the host (see pack_inputs_kernel)
__global__ void unpack_kernel(const __nv_bfloat16 *in, const float *pred, int Cp, double *abs3d, double *sdir,
                              double *sdif, int D, int H, int W, double s_out, double F)
{
    const long long n = (long long)D * H * W;
    GRID_LOOP(v, n) {
        const float a = __bfloat162float(in[v * 16 + 0]) + pred[v * Cp + 0];
        abs3d[v] = (double)a * s_out;
    }
    // every layer of a column is trained to predict the same surface
    // correction; their mean is the surface estimate. One warp per column:
    // lane l sums layers l, l + 32, ...; the warp adds the partial sums in a
    // fixed order (blockDim is a multiple of 32, so every warp is whole).
    const long long nc = (long long)H * W;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nc; c += nwarps) {
        float s1 = 0.f, s2 = 0.f;
        for (int k = lane; k < D; k += 32) {
            s1 += pred[(k * nc + c) * Cp + 1];
            s2 += pred[(k * nc + c) * Cp + 2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            sdir[c] = (double)(__bfloat162float(in[c * 16 + 1]) + s1 / D) * F;
            sdif[c] = (double)(__bfloat162float(in[c * 16 + 2]) + s2 / D) * F;
        }
    }
}

int grid1d(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148 * 16)); }

bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// the 8-channel kernels index with 32 bits when every index they form fits
bool fits32(long long elems16) { return elems16 < (1LL << 31); }

thread_local char g_err[256] = "";

int check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
        return NN_E_CUDA;
    }
    return NN_OK;
}

int inval(const char *msg)
{
    snprintf(g_err, sizeof g_err, "%s", msg);
    return NN_E_INVAL;
}

}  // namespace

extern "C" {

const char *nn_last_error(void) { return g_err; }

int nn_set_conv_path(int path)
{
    if (path != NN_CONV_AUTO && path != NN_CONV_MMA_SYNC && path != NN_CONV_TCGEN05 && path != NN_CONV_TCGEN05_TAP &&
        path != NN_CONV_TCGEN05_HALO)
        return inval("nn_set_conv_path: unknown path");
    const int old = g_conv_path;
    g_conv_path = path;
    return old;
}

int nn_status(void *stream)
{
    unsigned v = 0;
    if (nn_tc::take_status((cudaStream_t)stream, &v) != NN_OK) return check_launch("nn_status");
    if (v) {
        snprintf(g_err, sizeof g_err, "a tcgen05 convolution gave up waiting for its operands (status %u)", v);
        return NN_E_DEVICE;
    }
    return NN_OK;
}

int nn_conv3d_fwd(const void *in, const void *wt, const float *bias, void *out_bf16, float *out_f32, int N, int D,
                  int H, int W, int Cin, int Cout, int ksize, int relu, void *stream)
{
    if (!in || !wt || (!out_bf16 && !out_f32) || N <= 0 || D <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cout <= 0)
        return inval("nn_conv3d_fwd: bad argument");
    if (Cin % 16 != 0) return inval("nn_conv3d_fwd: Cin must be a multiple of 16");
    if (out_bf16 && Cout % 2 != 0) return inval("nn_conv3d_fwd: BF16 output needs an even Cout");
    if (ksize != 1 && ksize != 3) return inval("nn_conv3d_fwd: ksize must be 1 or 3");
    const bool forced = g_conv_path == NN_CONV_TCGEN05 || g_conv_path == NN_CONV_TCGEN05_TAP ||
                        g_conv_path == NN_CONV_TCGEN05_HALO;
    if (ksize == 3 && g_conv_path != NN_CONV_MMA_SYNC && (forced || nn_tc::supported(Cin, Cout))) {
        const int variant = g_conv_path == NN_CONV_TCGEN05_TAP ? 1 : g_conv_path == NN_CONV_TCGEN05_HALO ? 2 : 0;
        return nn_tc::conv3d_fwd(in, wt, bias, out_bf16, out_f32, N, D, H, W, Cin, Cout, relu, (cudaStream_t)stream,
                                 g_err, sizeof g_err, variant);
    }
    if (forced && ksize == 3) return inval("nn_conv3d_fwd: channel counts the tcgen05 kernels do not take");
    const long long M = (long long)N * D * H * W;
    if (Cout >= 64) {
        dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((Cout + 63) / 64));
        conv_fwd_kernel<64><<<grid, 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16 *)in, (const __nv_bfloat16 *)wt, bias, (__nv_bfloat16 *)out_bf16, out_f32, N, D, H,
            W, Cin, Cout, ksize == 3 ? 27 : 1, relu);
    } else {
        dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((Cout + 31) / 32));
        conv_fwd_kernel<32><<<grid, 128, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16 *)in, (const __nv_bfloat16 *)wt, bias, (__nv_bfloat16 *)out_bf16, out_f32, N, D, H,
            W, Cin, Cout, ksize == 3 ? 27 : 1, relu);
    }
    return check_launch("nn_conv3d_fwd");
}

int nn_conv3d_wgrad(const void *in, const void *gout, float *gw, float *gb, int N, int D, int H, int W, int Cin,
                    int Cout, int ksize, void *stream)
{
    if (!in || !gout || !gw || N <= 0 || D <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cout <= 0)
        return inval("nn_conv3d_wgrad: bad argument");
    if (Cin % 8 != 0 || Cout % 8 != 0) return inval("nn_conv3d_wgrad: channels must be multiples of 8");
    if (ksize != 1 && ksize != 3) return inval("nn_conv3d_wgrad: ksize must be 1 or 3");
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(gout) |
                           reinterpret_cast<uintptr_t>(gw)) & 15u) == 0;
    if (ksize == 3 && g_conv_path != NN_CONV_MMA_SYNC && aligned && nn_tc::wgrad_supported(Cin, Cout))
        return nn_tc::conv3d_wgrad(in, gout, gw, gb, N, D, H, W, Cin, Cout, (cudaStream_t)stream, g_err,
                                   sizeof g_err);
    const int taps = ksize == 3 ? 27 : 1;
    const long long M = (long long)N * D * H * W;
    const long long tiles = (long long)taps * ((Cin + 31) / 32) * ((Cout + 31) / 32);
    long long splits = std::max<long long>(1, (148LL * 8) / tiles);
    splits = std::min<long long>(splits, (M + kWV - 1) / kWV);
    const long long per = ((M + splits - 1) / splits + kWV - 1) / kWV * kWV;
    splits = (M + per - 1) / per;
    dim3 grid((unsigned)(taps * ((Cin + 31) / 32)), (unsigned)((Cout + 31) / 32), (unsigned)splits);
    conv_wgrad_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)in,
                                                             (const __nv_bfloat16 *)gout, gw, gb, N, D, H, W, Cin,
                                                             Cout, taps, per);
    return check_launch("nn_conv3d_wgrad");
}

int nn_relu_bwd(const void *y, void *g, long long n, void *stream)
{
    if (!y || !g || n < 0) return inval("nn_relu_bwd: bad argument");
    relu_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)y, (__nv_bfloat16 *)g, n);
    return check_launch("nn_relu_bwd");
}

int nn_pool2_fwd(const void *in, void *out, int N, int D, int H, int W, int C, void *stream)
{
    if (!in || !out || D % 2 || H % 2 || W % 2) return inval("nn_pool2_fwd: bad argument");
    const long long n = (long long)N * (D / 2) * (H / 2) * (W / 2) * C;
    if (C % 8 == 0 && al16(in) && al16(out)) {
        const long long big = (long long)N * D * H * W * (C / 8);
        if (fits32(big))
            pool2_fwd_vec_kernel<uint32_t><<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)in, (uint4 *)out, N, D / 2, H / 2, W / 2, C / 8);
        else
            pool2_fwd_vec_kernel<long long><<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)in, (uint4 *)out, N, D / 2, H / 2, W / 2, C / 8);
        return check_launch("nn_pool2_fwd");
    }
    pool2_fwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)in, (__nv_bfloat16 *)out, N, D,
                                                                  H, W, C);
    return check_launch("nn_pool2_fwd");
}

int nn_pool2_bwd(const void *gout, void *gin, int N, int D, int H, int W, int C, void *stream)
{
    if (!gout || !gin || D % 2 || H % 2 || W % 2) return inval("nn_pool2_bwd: bad argument");
    const long long n = (long long)N * D * H * W * C;
    if (C % 8 == 0 && al16(gout) && al16(gin)) {
        if (fits32(n / 8))
            pool2_bwd_vec_kernel<uint32_t><<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)gout, (uint4 *)gin, N, D / 2, H / 2, W / 2, C / 8);
        else
            pool2_bwd_vec_kernel<long long><<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)gout, (uint4 *)gin, N, D / 2, H / 2, W / 2, C / 8);
        return check_launch("nn_pool2_bwd");
    }
    pool2_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)gout, (__nv_bfloat16 *)gin, N,
                                                                  D, H, W, C);
    return check_launch("nn_pool2_bwd");
}

int nn_up2_fwd(const void *in, void *out, int N, int d, int h, int w, int C, int Cdst, int c0, void *stream)
{
    if (!in || !out || c0 < 0 || c0 + C > Cdst) return inval("nn_up2_fwd: bad argument");
    const long long n = (long long)N * 8 * d * h * w * C;
    if (C % 8 == 0 && Cdst % 8 == 0 && c0 % 8 == 0 && al16(in) && al16(out)) {
        const long long big = (long long)N * 8 * d * h * w * (Cdst / 8);
        if (fits32(big))
            up2_fwd_vec_kernel<uint32_t><<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)in, (uint4 *)out, N, d, h, w, C / 8, Cdst / 8, c0 / 8);
        else
            up2_fwd_vec_kernel<long long><<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)in, (uint4 *)out, N, d, h, w, C / 8, Cdst / 8, c0 / 8);
        return check_launch("nn_up2_fwd");
    }
    up2_fwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)in, (__nv_bfloat16 *)out, N, d, h,
                                                                w, C, Cdst, c0);
    return check_launch("nn_up2_fwd");
}

int nn_up2_bwd(const void *gout, void *gin, int N, int d, int h, int w, int C, int Csrc, int c0, void *stream)
{
    if (!gout || !gin || c0 < 0 || c0 + C > Csrc) return inval("nn_up2_bwd: bad argument");
    const long long n = (long long)N * d * h * w * C;
    if (C % 8 == 0 && Csrc % 8 == 0 && c0 % 8 == 0 && al16(gout) && al16(gin)) {
        const long long big = (long long)N * 8 * d * h * w * (Csrc / 8);
        if (fits32(big))
            up2_bwd_vec_kernel<uint32_t><<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)gout, (uint4 *)gin, N, d, h, w, C / 8, Csrc / 8, c0 / 8);
        else
            up2_bwd_vec_kernel<long long><<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)gout, (uint4 *)gin, N, d, h, w, C / 8, Csrc / 8, c0 / 8);
        return check_launch("nn_up2_bwd");
    }
    up2_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)gout, (__nv_bfloat16 *)gin, N, d,
                                                                h, w, C, Csrc, c0);
    return check_launch("nn_up2_bwd");
}

int nn_copy_channels(const void *src, int Csrc, int s0, void *dst, int Cdst, int d0, long long vox, int C,
                     int accumulate, void *stream)
{
    if (!src || !dst || s0 < 0 || d0 < 0 || s0 + C > Csrc || d0 + C > Cdst) return inval("nn_copy_channels: bad argument");
    if (C % 8 == 0 && Csrc % 8 == 0 && Cdst % 8 == 0 && s0 % 8 == 0 && d0 % 8 == 0 && al16(src) && al16(dst)) {
        const long long big = vox * (std::max(Csrc, Cdst) / 8);
        if (fits32(big))
            copy_channels_vec_kernel<uint32_t><<<grid1d(vox * C / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)src, Csrc / 8, s0 / 8, (uint4 *)dst, Cdst / 8, d0 / 8, (uint32_t)vox, C / 8, accumulate);
        else
            copy_channels_vec_kernel<long long><<<grid1d(vox * C / 8), 256, 0, (cudaStream_t)stream>>>(
                (const uint4 *)src, Csrc / 8, s0 / 8, (uint4 *)dst, Cdst / 8, d0 / 8, vox, C / 8, accumulate);
        return check_launch("nn_copy_channels");
    }
    copy_channels_kernel<<<grid1d(vox * C), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)src, Csrc, s0, (__nv_bfloat16 *)dst, Cdst, d0, vox, C, accumulate);
    return check_launch("nn_copy_channels");
}

int nn_mse(const float *pred, int Cp, const float *target, int Cuse, const float *chw, void *grad, long long vox,
           double *loss, void *stream)
{
    if (!pred || !target || !grad || !loss || Cuse > Cp || vox <= 0) return inval("nn_mse: bad argument");
    mse_kernel<<<grid1d(vox * Cp), 256, 0, (cudaStream_t)stream>>>(pred, Cp, target, Cuse, chw, (__nv_bfloat16 *)grad,
                                                                   vox, 1.0 / ((double)vox * Cuse), loss);
    return check_launch("nn_mse");
}

int nn_adam(float *W, float *m, float *v, const float *grad, long long n, float lr, float b1, float b2, float eps,
            int step, float weight_decay, void *stream)
{
    if (!W || !m || !v || !grad || n <= 0 || step <= 0) return inval("nn_adam: bad argument");
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(W, m, v, grad, n, lr, b1, b2, eps, c1, c2, weight_decay);
    return check_launch("nn_adam");
}

int nn_direct_transmittance(const float *k_gas, const float *k_cld, int D, int H, int W, double dx, double dy,
                            double dz, double sza_deg, double azimuth_deg, float *t3d, float *t2d, void *stream)
{
    if (!k_gas || !k_cld || !t3d || !t2d || D <= 0 || H <= 0 || W <= 0 || !(dx > 0) || !(dy > 0) || !(dz > 0) ||
        !(sza_deg >= 0.0 && sza_deg < 90.0) || !std::isfinite(azimuth_deg))
        return inval("nn_direct_transmittance: bad argument");
    const double t = sza_deg * 3.14159265358979323846 / 180.0, p = azimuth_deg * 3.14159265358979323846 / 180.0;
    const long long n = (long long)D * H * W + (long long)H * W;
    direct_transmittance_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(
        k_gas, k_cld, D, H, W, (float)dx, (float)dy, (float)dz, (float)(std::sin(t) * std::sin(p)),
        (float)(std::sin(t) * std::cos(p)), (float)std::cos(t), t3d, t2d);
    return check_launch("nn_direct_transmittance");
}

int nn_direct_surface(const float *k_gas, const float *k_cld, int D, int H, int W, double dx, double dy, double dz,
                      double sza_deg, double azimuth_deg, int nsub, float *t2d, void *stream)
{
    if (!k_gas || !k_cld || !t2d || D <= 0 || H <= 0 || W <= 0 || !(dx > 0) || !(dy > 0) || !(dz > 0) ||
        !(sza_deg >= 0.0 && sza_deg < 90.0) || !std::isfinite(azimuth_deg) || nsub < 1 || nsub > 32)
        return inval("nn_direct_surface: bad argument");
    const double t = sza_deg * 3.14159265358979323846 / 180.0, p = azimuth_deg * 3.14159265358979323846 / 180.0;
    const long long ncol = (long long)H * W;
    const long long blocks = std::min<long long>((ncol * 32 + 255) / 256, 148LL * 64);
    direct_surface_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        k_gas, k_cld, D, H, W, (float)dx, (float)dy, (float)dz, (float)(std::sin(t) * std::sin(p)),
        (float)(std::sin(t) * std::cos(p)), (float)std::cos(t), nsub, t2d);
    return check_launch("nn_direct_surface");
}

int nn_pack_inputs(const double *abs3d, const double *sfc_dir, const double *sfc_dif, const float *k_gas,
                   const float *ssa_gas, const float *k_cld, const float *ssa_cld, const float *g_cld,
                   const float *t3d, const float *t2d, void *out, int D, int H, int W, double dz, double flux,
                   void *stream)
{
    if (!abs3d || !sfc_dir || !sfc_dif || !k_gas || !ssa_gas || !k_cld || !ssa_cld || !g_cld || !out || !(flux > 0))
        return inval("nn_pack_inputs: bad argument");
    pack_inputs_kernel<<<grid1d((long long)D * H * W), 256, 0, (cudaStream_t)stream>>>(
        abs3d, sfc_dir, sfc_dif, k_gas, ssa_gas, k_cld, ssa_cld, g_cld, t3d, t2d, (__nv_bfloat16 *)out, D, H, W,
        (float)dz, 100.0 * dz / flux, 1.0 / flux);
    return check_launch("nn_pack_inputs");
}

int nn_pack_targets(const double *abs_hi, const double *sdir_hi, const double *sdif_hi, const double *abs_lo,
                    const double *sdir_lo, const double *sdif_lo, float *out, int D, int H, int W, double dz,
                    double flux, void *stream)
{
    if (!abs_hi || !sdir_hi || !sdif_hi || !abs_lo || !sdir_lo || !sdif_lo || !out || !(flux > 0))
        return inval("nn_pack_targets: bad argument");
    pack_targets_kernel<<<grid1d((long long)D * H * W), 256, 0, (cudaStream_t)stream>>>(
        abs_hi, sdir_hi, sdif_hi, abs_lo, sdir_lo, sdif_lo, out, D, H, W, 100.0 * dz / flux, 1.0 / flux);
    return check_launch("nn_pack_targets");
}

int nn_unpack(const void *in, const float *pred, int Cp, double *abs3d, double *sfc_dir, double *sfc_dif, int D,
              int H, int W, double dz, double flux, void *stream)
{
    if (!in || !pred || !abs3d || !sfc_dir || !sfc_dif || Cp < 3 || !(flux > 0)) return inval("nn_unpack: bad argument");
    unpack_kernel<<<grid1d((long long)D * H * W), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)in, pred, Cp, abs3d, sfc_dir, sfc_dif, D, H, W, flux / (100.0 * dz), flux);
    return check_launch("nn_unpack");
}

int nn_ema(float *avg, const float *W, long long n, float decay, void *stream)
{
    if (!avg || !W || n < 0 || !(decay >= 0.f && decay <= 1.f)) return inval("nn_ema: bad argument");
    if (n == 0) return NN_OK;
    ema_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(avg, W, n, decay);
    return check_launch("nn_ema");
}

int nn_weights_bf16(const float *W, void *wt, void *wd, int ksize, int Cin, int Cout, void *stream)
{
    if (!W || (!wt && !wd) || (ksize != 1 && ksize != 3)) return inval("nn_weights_bf16: bad argument");
    const int taps = ksize == 3 ? 27 : 1;
    weights_bf16_kernel<<<grid1d((long long)taps * Cin * Cout), 256, 0, (cudaStream_t)stream>>>(
        W, (__nv_bfloat16 *)wt, (__nv_bfloat16 *)wd, taps, Cin, Cout);
    return check_launch("nn_weights_bf16");
}

}  // extern "C"
