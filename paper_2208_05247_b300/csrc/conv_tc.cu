// conv_tc.cu -- 3x3x3 "same" convolution on the fifth-generation tensor cores.
//
// The convolution is the implicit GEMM of nn_kernels.cu,
//   out[p][o] = bias[o] + sum_t sum_i in[p + off(t)][i] * Wt[t][o][i],
// with M = voxels, N = output channels, K = 27 taps x input channels. One CTA
// computes a tile of 128 voxels (a Wt x Ht x Dt box of the volume) by BN
// output channels:
//
//   - one thread streams the operands with TMA: for every (tap, channel chunk)
//     the activation box shifted by the tap offset (5D tensor map over
//     [N][D][H][W][C]; coordinates outside the volume read as zeros, which is
//     the "same" padding) and the weight slice Wt[t][n0:n0+BN][c0:c0+CK];
//   - one thread issues tcgen05.mma (kind::f16, BF16 operands, FP32
//     accumulator of 128 lanes x BN columns in tensor memory), releasing each
//     stage back to the producer with tcgen05.commit;
//   - all four warps read the accumulator with tcgen05.ld (warp w owns tensor
//     memory lanes 32w..32w+31 = voxel rows), add the bias, apply ReLU and
//     write FP32 and/or BF16 channels-last outputs.
//
// Operand tiles are K-major with the TMA swizzle that matches the channel
// chunk (CK = 16, 32 or 64 BF16 = 32, 64 or 128 bytes per row), so the same
// bytes are the canonical tcgen05 shared-memory layout. Every wait on an
// mbarrier is bounded; on time-out the CTA records an error, waits (bounded)
// for its own copies and products in flight, frees its tensor memory and
// returns.
//
// The weight gradient (conv3d_wgrad) is the GEMM with the (tap, input
// channel) pairs as M, output channels as N and voxels as K. Activations and
// output gradients are voxel-major, which is the MN-major operand layout for
// that GEMM, so its TMA boxes feed tcgen05.mma directly (see the kernel's
// own comment).
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "nn.h"

namespace nn_tc {

__device__ unsigned int g_status;   // bit 0: an mbarrier wait timed out

// kernel variants of conv3d_fwd (0: the halo kernel where it fits, else per tap)
constexpr int kVariantTap = 1, kVariantHalo = 2;

namespace {

constexpr int kThreads = 128;
constexpr uint32_t kMaxDynSmem = 232448;   // opt-in shared memory per block (227 KB)

// Let a kernel use all the opt-in shared memory its static shared memory leaves.
cudaError_t allow_max_smem(const void *kern)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kMaxDynSmem - (uint32_t)fa.sharedSizeBytes));
}

constexpr long long kSpinCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete, for at most ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kSpinCycles) {
            atomicOr(&g_status, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2, int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6, %7}], [%2];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
        "%5}], [%2];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: start address, leading byte offset
// (unused by swizzled K-major operands), stride byte offset between 8-row
// groups, descriptor version 1 (bit 46) and the swizzle mode (bits 61-63).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo_bytes, uint64_t layout)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | (layout << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 lanes x 16 columns of 32-bit words from tensor memory: this thread gets
// its lane's 16 consecutive columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// tensor memory is allocated in powers of two of at least 32 columns
__host__ __device__ constexpr uint32_t tmem_cols(int bn) { return bn <= 32 ? 32u : bn <= 64 ? 64u : bn <= 128 ? 128u : 256u; }

struct ConvTile {
    int N, D, H, W, Cin, Cout;
    int Wt, Ht, Dt;             // box of 128 voxels
    int tw, th, td;             // tiles per axis
    int relu;
};

// BN output channels per CTA (16..256), CK input channels per K stage
// (16/32/64 -> 32/64/128-byte swizzle), S pipeline stages.
template <int BN, int CK, int S>
__global__ void __launch_bounds__(kThreads) conv3d_tc_kernel(const __grid_constant__ CUtensorMap map_x,
                                                             const __grid_constant__ CUtensorMap map_w,
                                                             const float *__restrict__ bias,
                                                             __nv_bfloat16 *__restrict__ out_bf16,
                                                             float *__restrict__ out_f32, const ConvTile P)
{
    constexpr uint32_t kRowBytes = CK * 2;                 // = swizzle span
    constexpr uint32_t kABytes = 128 * kRowBytes, kBBytes = BN * kRowBytes;
    constexpr uint32_t kStageBytes = kABytes + kBBytes;
    constexpr uint64_t kLayout = CK == 64 ? 2 : CK == 32 ? 4 : 6;   // SWIZZLE_128B / 64B / 32B
    constexpr uint32_t kCols = tmem_cols(BN);
    // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | (8u << 24);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage buffers (the swizzle pattern repeats every 1024 B)
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - smem_u32(smem_raw));
    __shared__ __align__(8) unsigned long long bar_full[S], bar_empty[S], bar_acc;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kchunks = P.Cin / CK, kb_total = 27 * kchunks;

    // tile coordinates
    int tile = blockIdx.x;
    const int tx = tile % P.tw; tile /= P.tw;
    const int ty = tile % P.th; tile /= P.th;
    const int tz = tile % P.td; tile /= P.td;
    const int n = tile;
    const int w0 = tx * P.Wt, h0 = ty * P.Ht, d0 = tz * P.Dt;
    const int n0 = blockIdx.y * BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    int issued = 0;      // producer: stages loaded
    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: TMA loads of (tap, channel chunk) stages ----
            for (int kb = 0; kb < kb_total; ++kb) {
                const int s = kb % S;
                if (kb >= S && !mbar_wait(smem_u32(&bar_empty[s]), ((kb / S) - 1) & 1)) {
                    s_abort = 1;
                    break;
                }
                if (*(volatile int *)&s_abort) break;
                const int t = kb / kchunks, c0 = (kb % kchunks) * CK;
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                const uint32_t a = base + s * kStageBytes, b = a + kABytes, fb = smem_u32(&bar_full[s]);
                mbar_expect_tx(fb, kStageBytes);
                tma_load_5d(a, &map_x, fb, c0, w0 + dx, h0 + dy, d0 + dz, n);
                tma_load_3d(b, &map_w, fb, c0, n0, t);
                ++issued;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            int kb = 0;
            for (; kb < kb_total; ++kb) {
                const int s = kb % S;
                if (!mbar_wait(smem_u32(&bar_full[s]), (kb / S) & 1)) {
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a = base + s * kStageBytes, b = a + kABytes;
#pragma unroll
                for (int k = 0; k < CK / 16; ++k)
                    umma_f16(tmem, umma_desc(a + 32 * k, 8 * kRowBytes, kLayout),
                             umma_desc(b + 32 * k, 8 * kRowBytes, kLayout), kIdesc, (kb | k) != 0);
                umma_commit(smem_u32(&bar_empty[s]));
            }
            // the accumulator barrier fires once every product issued so far is done
            umma_commit(smem_u32(&bar_acc));
        }
        __syncwarp();
    }

    // ---- epilogue: tensor memory -> registers -> global ----
    const bool done = mbar_wait(smem_u32(&bar_acc), 0);
    tc_fence_after();
    const int r = warp * 32 + lane;
    const int w = w0 + r % P.Wt, h = h0 + (r / P.Wt) % P.Ht, d = d0 + r / (P.Wt * P.Ht);
    const bool valid = done && !*(volatile int *)&s_abort && w < P.W && h < P.H && d < P.D;
    const long long vox = (((long long)n * P.D + d) * P.H + h) * P.W + w;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
        float v[16];
        // every lane of the warp takes part in the load (.sync.aligned)
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        if (!valid) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float x = v[j] + (bias ? __ldg(bias + n0 + c + j) : 0.f);
            v[j] = P.relu ? fmaxf(x, 0.f) : x;
        }
        const long long o = vox * P.Cout + n0 + c;
        if (out_f32) {
            float4 *dst = reinterpret_cast<float4 *>(out_f32 + o);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        if (out_bf16) {
            uint4 pk[2];
            uint32_t *pw = reinterpret_cast<uint32_t *>(pk);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                __nv_bfloat162 t2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                pw[q] = *reinterpret_cast<uint32_t *>(&t2);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(out_bf16 + o);
            dst[0] = pk[0];
            dst[1] = pk[1];
        }
    }

    // ---- after an abort: let this CTA's copies land before its memory goes ----
    if (threadIdx.x == 0 && *(volatile int *)&s_abort) {
        for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb)
            mbar_wait(smem_u32(&bar_full[kb % S]), (kb / S) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
    }
}

// ---------------------------------------------------------------------------
// Halo-tiled persistent variant for narrow layers (at most 64 output channels
// per tile). The per-tap kernel above reloads a 128-row box from L2 for each
// of the 27 taps, which bounds the 32-channel layers by L2 throughput. Here a
// tile is 8 (x) x 16 (y) voxels of one z slice, and one TMA box of
// 8 x 18 x 3 voxels (the tile's y and z halo) per (x offset, channel chunk)
// serves nine taps: tap (dy, dz) reads the 128 rows that start
// 8 (dy + 1) + 144 (dz + 1) rows into the box, a multiple of the 8-row swizzle
// atom, so the tcgen05 descriptor just starts there. The weights of the nine
// taps come as one 4D box per stage, or stay resident in shared memory for the
// whole launch when they fit (RESW). The CTA is persistent (one per SM) and
// double-buffers the accumulator in tensor memory, so the epilogue of one tile
// overlaps the products of the next. Warps 0-3 drain the accumulator, warp 4
// loads, warp 5 issues the products and owns the tensor memory.
// ---------------------------------------------------------------------------
constexpr int kHaloW = 8, kHaloH = 16;                    // tile: 8 x 16 voxels = 128 rows
constexpr int kHaloRows = kHaloW * (kHaloH + 2) * 3;       // 432 rows per halo box
constexpr int kHaloThreads = 192;

struct HaloTile {
    int N, D, H, W, Cin, Cout;
    int tw, th, ntn;            // tiles along x and y; output-channel tiles
    long long ntiles;           // ntn * tw * th * D * N
    int relu;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Bytes of dynamic shared memory the halo kernel needs (plus alignment slack).
__host__ __device__ constexpr uint32_t halo_stage_bytes(int BN, int CK, bool resw)
{
    return (uint32_t)(kHaloRows * CK * 2) + (resw ? 0u : (uint32_t)(9 * BN * CK * 2));
}

template <int BN, int CK, int S, bool RESW>
__global__ void __launch_bounds__(kHaloThreads, 1) conv3d_tc_halo_kernel(
    const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
    const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out_bf16, float *__restrict__ out_f32,
    const HaloTile P)
{
    constexpr uint32_t kRow = CK * 2;
    constexpr uint32_t kA = kHaloRows * kRow;
    constexpr uint32_t kBtap = BN * kRow;                     // one tap's weight tile
    constexpr uint32_t kStage = halo_stage_bytes(BN, CK, RESW);
    constexpr uint64_t kLayout = CK == 64 ? 2 : CK == 32 ? 4 : 6;
    constexpr uint32_t kCols = tmem_cols(BN);
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | (8u << 24);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t wres = base + S * kStage;                  // resident weights (RESW)
    __shared__ __align__(8) unsigned long long bar_full[S], bar_empty[S], bar_accf[2], bar_acce[2], bar_w,
        bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kchunks = P.Cin / CK, KB = 3 * kchunks;

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(smem_u32(&bar_full[q]), 1);
            mbar_init(smem_u32(&bar_empty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&bar_accf[q]), 1);
            mbar_init(smem_u32(&bar_acce[q]), 4);   // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&bar_w), 1);
        mbar_init(smem_u32(&bar_drain), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(2 * kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // tile -> (output-channel tile, x tile, y tile, z slice, sample); the
    // channel tile varies fastest so concurrent CTAs share halo boxes in L2
    auto decode = [&](long long tile, int &tn, int &w0, int &h0, int &d, int &n) {
        tn = (int)(tile % P.ntn); tile /= P.ntn;
        w0 = (int)(tile % P.tw) * kHaloW; tile /= P.tw;
        h0 = (int)(tile % P.th) * kHaloH; tile /= P.th;
        d = (int)(tile % P.D);
        n = (int)(tile / P.D);
    };

    if (warp == 4) {
        if (lane == 0) {
            // ---- producer ----
            if (RESW) {
                mbar_expect_tx(smem_u32(&bar_w), (uint32_t)(3 * kchunks * 9) * kBtap);
                for (int dxp = 0; dxp < 3; ++dxp)
                    for (int ch = 0; ch < kchunks; ++ch)
                        tma_load_4d(wres + (uint32_t)((dxp * kchunks + ch) * 9) * kBtap, &map_w,
                                    smem_u32(&bar_w), ch * CK, 0, dxp, 0);
            }
            long long g = 0;
            for (long long tile = blockIdx.x; tile < P.ntiles && !*(volatile int *)&s_abort; tile += gridDim.x) {
                int tn, w0, h0, d, n;
                decode(tile, tn, w0, h0, d, n);
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int q = (int)(g % S);
                    if (g >= S && !mbar_wait(smem_u32(&bar_empty[q]), (uint32_t)((g / S) - 1) & 1u)) {
                        s_abort = 1;
                        break;
                    }
                    const int dxp = kb / kchunks, ch = kb % kchunks;
                    const uint32_t a = base + (uint32_t)q * kStage, fb = smem_u32(&bar_full[q]);
                    mbar_expect_tx(fb, kStage);
                    tma_load_5d(a, &map_x, fb, ch * CK, w0 + dxp - 1, h0 - 1, d - 1, n);
                    if (!RESW) tma_load_4d(a + kA, &map_w, fb, ch * CK, tn * BN, dxp, 0);
                }
            }
        }
        __syncwarp();
    } else if (warp == 5) {
        if (lane == 0) {
            // ---- MMA issuer ----
            bool ok = !RESW || mbar_wait(smem_u32(&bar_w), 0);
            if (!ok) s_abort = 1;
            long long g = 0;
            int i = 0;
            for (long long tile = blockIdx.x; ok && tile < P.ntiles; tile += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(&bar_acce[b]), (uint32_t)((i >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)b * kCols;
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int q = (int)(g % S);
                    if (!mbar_wait(smem_u32(&bar_full[q]), (uint32_t)(g / S) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int dxp = kb / kchunks, ch = kb % kchunks;
                    const uint32_t a = base + (uint32_t)q * kStage;
#pragma unroll 1
                    for (int m = 0; m < 9; ++m) {
                        const uint32_t ra = a + (uint32_t)(kHaloW * (m % 3) + kHaloW * (kHaloH + 2) * (m / 3)) * kRow;
                        const uint32_t rb = RESW ? wres + (uint32_t)((dxp * kchunks + ch) * 9 + m) * kBtap
                                                 : a + kA + (uint32_t)m * kBtap;
#pragma unroll
                        for (int k = 0; k < CK / 16; ++k)
                            umma_f16(dt, umma_desc(ra + 32 * k, 8 * kRow, kLayout),
                                     umma_desc(rb + 32 * k, 8 * kRow, kLayout), kIdesc, (kb | m | k) != 0);
                    }
                    umma_commit(smem_u32(&bar_empty[q]));
                }
                if (!ok) break;
                umma_commit(smem_u32(&bar_accf[b]));
            }
            if (!ok) s_abort = 1;
            umma_commit(smem_u32(&bar_drain));     // fires once every product issued is done
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 0-3, tensor memory lanes 32 warp .. 32 warp + 31 ----
        int i = 0;
        for (long long tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            int ok = 0;
            if (lane == 0) ok = mbar_wait(smem_u32(&bar_accf[b]), (uint32_t)(i >> 1) & 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok || *(volatile int *)&s_abort) break;
            tc_fence_after();
            int tn, w0, h0, d, n;
            decode(tile, tn, w0, h0, d, n);
            const int r = warp * 32 + lane;
            const int w = w0 + r % kHaloW, h = h0 + r / kHaloW;
            const bool valid = w < P.W && h < P.H;
            const long long vox = (((long long)n * P.D + d) * P.H + h) * P.W + w;
            const int n0 = tn * BN;
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                float v[16];
                tmem_ld16(tmem + (uint32_t)b * kCols + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float x = v[j] + (bias ? __ldg(bias + n0 + c + j) : 0.f);
                    v[j] = P.relu ? fmaxf(x, 0.f) : x;
                }
                const long long o = vox * P.Cout + n0 + c;
                if (out_f32) {
                    float4 *dst = reinterpret_cast<float4 *>(out_f32 + o);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                if (out_bf16) {
                    uint4 pk[2];
                    uint32_t *pw = reinterpret_cast<uint32_t *>(pk);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        __nv_bfloat162 t2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        pw[q] = *reinterpret_cast<uint32_t *>(&t2);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(out_bf16 + o);
                    dst[0] = pk[0];
                    dst[1] = pk[1];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acce[b]));
        }
    }

    // ---- teardown: every product done, copies landed, then free tensor memory ----
    if (warp == 5 && lane == 0) mbar_wait(smem_u32(&bar_drain), 0);
    if (warp == 4 && lane == 0 && *(volatile int *)&s_abort) {
        // copies in flight at an abort: wait (bounded) for the stages' last phases
        for (int q = 0; q < S; ++q) mbar_wait(smem_u32(&bar_full[q]), 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * kCols));
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05: gW[t][i][o] += sum_p in[p + off(t)][i] gout[p][o].
// As a GEMM the rows (M) are the 27 * Cin (tap, input channel) pairs in the
// order of gW, the columns (N) the output channels, and the reduction (K) runs
// over voxels. Both tensors are stored voxel-major with channels contiguous,
// which is the MN-major operand layout: a TMA box of KV voxels x CK channels
// (rows of CK * 2 bytes with the matching swizzle) is a stack of tcgen05
// MN-major swizzle atoms with the voxel as K index, so no thread touches the
// operands. For every tile of KV voxels the producer loads, per row block of
// 128 (tap, channel) rows, 128 / CK activation boxes shifted by their tap's
// offset (zeros outside the volume: the "same" padding) and once the gout box
// of NT output channels, which the CTA's MG row blocks share; each row block
// accumulates into its own 128 x NT tensor-memory accumulator. A CTA reduces
// over a range of voxel tiles and adds its partial sums to gW with FP32
// atomics.
//
// Shared-memory descriptors of an MN-major swizzled operand: the leading byte
// offset is the distance between swizzle atoms along M (or N), the stride
// byte offset the distance between groups of 8 K rows.
// ---------------------------------------------------------------------------
struct WgradArgs {
    int N, D, H, W, Cin, Cout;
    int Wb, Hb, Db, KV;          // voxel box (Wb * Hb * Db = KV voxels = K per stage)
    int tw, th, td;              // boxes per axis
    int ntiles, stride;          // voxel tiles; CTA z takes tiles z, z + stride, ...
    int groups, MG, NT, S;       // 128-row blocks, row blocks per CTA, N tile, stages
    int CK, CKB;                 // channels per activation / gout box
    uint32_t stage_bytes, cols;  // bytes per stage, tensor-memory columns per accumulator
};

__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes,
                                                 uint64_t layout)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | (layout << 61);
}

__device__ __forceinline__ uint64_t swizzle_layout(int ck) { return ck == 64 ? 2 : ck == 32 ? 4 : 6; }

constexpr int kWgMaxStages = 8;

__global__ void __launch_bounds__(kThreads) conv3d_wgrad_tc_kernel(const __grid_constant__ CUtensorMap map_x,
                                                                   const __grid_constant__ CUtensorMap map_g,
                                                                   float *__restrict__ gw, const WgradArgs P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    __shared__ __align__(8) unsigned long long bar_full[kWgMaxStages], bar_empty[kWgMaxStages], bar_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.S, NT = P.NT;
    const int g0 = blockIdx.x * P.MG;                               // first row block of this CTA
    const int mg = min(P.MG, P.groups - g0);                        // row blocks held
    const int n0 = blockIdx.y * NT;
    // all CTAs sweep the volume together (tile z, z + stride, ...), so the
    // planes that the z taps read again stay in L2
    const int t_begin = blockIdx.z;
    const int nt_local = t_begin < P.ntiles ? (P.ntiles - t_begin + P.stride - 1) / P.stride : 0;
    const int atoms = 128 / P.CK, chunks = P.Cin / P.CK, batoms = NT / P.CKB;
    const uint32_t a_atom = (uint32_t)P.KV * P.CK * 2, b_atom = (uint32_t)P.KV * P.CKB * 2;
    const uint32_t a_block = 128u * P.KV * 2;                       // bytes of one 128-row block
    const uint32_t bytes = ((uint32_t)mg * 128 + NT) * P.KV * 2;    // bytes landing per stage

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(P.MG * P.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    int issued = 0;
    if (warp == 0) {
        // ---- producer: the lanes of warp 0 share a stage's boxes (at most 36) ----
        // box b < mg * atoms: activation atom (row block b / atoms, tap and
        // channel chunk of its rows); the rest: gout atoms of NT / batoms channels
        const int nbox = mg * atoms + batoms;
        int bc[2], bdx[2], bdy[2], bdz[2], bmap[2];
        uint32_t boff[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int bx = lane + 32 * q;
            bc[q] = bdx[q] = bdy[q] = bdz[q] = 0;
            bmap[q] = -1;                                  // -1: no box for this lane
            boff[q] = 0;
            if (bx < mg * atoms) {
                const int m = bx / atoms, j = bx - m * atoms;
                int a = (g0 + m) * atoms + j;              // global (tap, chunk) atom
                int tap = a / chunks;
                if (tap > 26) { tap = 26; a = 26 * chunks; }   // rows past 27 * Cin: loaded, not stored
                bc[q] = (a - tap * chunks) * P.CK;
                bdz[q] = tap / 9 - 1; bdy[q] = (tap / 3) % 3 - 1; bdx[q] = tap % 3 - 1;
                bmap[q] = 0;
                boff[q] = (uint32_t)m * a_block + (uint32_t)j * a_atom;
            } else if (bx < nbox) {
                const int j = bx - mg * atoms;
                bc[q] = n0 + j * P.CKB;
                bmap[q] = 1;
                boff[q] = (uint32_t)P.MG * a_block + (uint32_t)j * b_atom;
            }
        }
        // first tile's coordinates; later tiles add the stride digit by digit
        int t = t_begin;
        int tx = t % P.tw; t /= P.tw;
        int ty = t % P.th; t /= P.th;
        int tz = t % P.td;
        int n = t / P.td;
        t = P.stride;
        const int sx = t % P.tw; t /= P.tw;
        const int sy = t % P.th; t /= P.th;
        const int sz = t % P.td;
        const int sn = t / P.td;
        int s = 0;
        uint32_t ph = 0;                                   // parity of the stage's next reuse wait
        for (int i = 0; i < nt_local; ++i) {
            int ok = 1;
            if (lane == 0) {
                if (i >= S && !mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u)) ok = 0;
                if (*(volatile int *)&s_abort) ok = 0;
                if (!ok) s_abort = 1;
                else mbar_expect_tx(smem_u32(&bar_full[s]), bytes);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const uint32_t st = base + (uint32_t)s * P.stage_bytes, fb = smem_u32(&bar_full[s]);
            const int w0 = tx * P.Wb, h0 = ty * P.Hb, d0 = tz * P.Db;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (bmap[q] == 0)
                    tma_load_5d(st + boff[q], &map_x, fb, bc[q], w0 + bdx[q], h0 + bdy[q], d0 + bdz[q], n);
                else if (bmap[q] == 1)
                    tma_load_5d(st + boff[q], &map_g, fb, bc[q], w0, h0, d0, n);
            }
            ++issued;
            if (++s == S) { s = 0; ph ^= 1u; }
            int c = 0;
            tx += sx; if (tx >= P.tw) { tx -= P.tw; c = 1; }
            ty += sy + c; c = 0; if (ty >= P.th) { ty -= P.th; c = 1; }
            tz += sz + c; c = 0; if (tz >= P.td) { tz -= P.td; c = 1; }
            n += sn + c;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: KV / 16 products per row block and stage ----
            // kind::f16, FP32 accumulator, BF16 A and B, both MN-major (bits 15, 16)
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                   ((uint32_t)(NT >> 3) << 17) | (8u << 24);
            // descriptors of stage 0; a stage's own differ in the start-address field only
            const uint64_t da = umma_desc_mn(base, a_atom, 8 * P.CK * 2, swizzle_layout(P.CK));
            const uint64_t db = umma_desc_mn(base + (uint32_t)P.MG * a_block, b_atom, 8 * P.CKB * 2,
                                             swizzle_layout(P.CKB));
            const uint32_t ka = 16 * P.CK * 2 >> 4, kb = 16 * P.CKB * 2 >> 4, mb = a_block >> 4;
            const int ksteps = P.KV / 16;
            int s = 0;
            uint32_t ph = 0;
            for (int i = 0; i < nt_local; ++i) {
                if (*(volatile int *)&s_abort || !mbar_wait(smem_u32(&bar_full[s]), ph)) {
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t so = (uint64_t)((uint32_t)s * P.stage_bytes >> 4);
                for (int m = 0; m < mg; ++m)
                    for (int k = 0; k < ksteps; ++k)
                        umma_f16(tmem + (uint32_t)m * P.cols, da + so + (uint64_t)(m * mb + k * ka),
                                 db + so + (uint64_t)(k * kb), idesc, (i | k) != 0);
                umma_commit(smem_u32(&bar_empty[s]));
                if (++s == S) { s = 0; ph ^= 1u; }
            }
            umma_commit(smem_u32(&bar_done));
        }
        __syncwarp();
    }

    // ---- epilogue: each row block's 128 x NT partial sums into gW ----
    const bool done = mbar_wait(smem_u32(&bar_done), 0);
    tc_fence_after();
    const bool valid = done && nt_local > 0 && !*(volatile int *)&s_abort;
    const int rows = 27 * P.Cin;
#pragma unroll 1
    for (int m = 0; m < mg; ++m) {
        const int r = (g0 + m) * 128 + warp * 32 + lane;
#pragma unroll 1
        for (int cc = 0; cc < NT; cc += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)m * P.cols + (uint32_t)cc, v);
            if (!valid || r >= rows) continue;
            float4 *dst = reinterpret_cast<float4 *>(gw + (long long)r * P.Cout + n0 + cc);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 t = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) atomicAdd(dst + q, t);
            }
        }
    }

    // ---- after an abort: let this CTA's copies land before its memory goes ----
    if (threadIdx.x == 0 && *(volatile int *)&s_abort) {
        for (int i = (issued > S ? issued - S : 0); i < issued; ++i)
            mbar_wait(smem_u32(&bar_full[i % S]), (i / S) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(P.MG * P.cols));
    }
}

// gb[o] += sum over voxels of gout[p][o]. Thread t of a block owns the 8
// channels 8 (t mod Cout/8) .. +7 and every (blockDim / (Cout/8))-th voxel of
// the block's share; partial sums meet in shared memory, then one global
// atomic per channel and block.
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ gout, float *__restrict__ gb, long long V, int Cout)
{
    extern __shared__ float part[];
    for (int o = threadIdx.x; o < Cout; o += blockDim.x) part[o] = 0.f;
    __syncthreads();
    const int cbs = Cout / 8, lanes = blockDim.x / cbs;
    const int cb = threadIdx.x % cbs, lv = threadIdx.x / cbs;
    if (lv < lanes) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (long long v = (long long)blockIdx.x * lanes + lv; v < V; v += (long long)gridDim.x * lanes) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(gout + v * Cout + cb * 8));
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(e[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&part[cb * 8 + j], acc[j]);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < Cout; o += blockDim.x)
        if (part[o] != 0.f) atomicAdd(gb + o, part[o]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int pow2_at_least(int x, int cap)
{
    int p = 1;
    while (p < x && p < cap) p <<= 1;
    return p;
}

template <int BN, int CK, int S>
int launch(const CUtensorMap &mx, const CUtensorMap &mw, const float *bias, __nv_bfloat16 *ob, float *of,
           const ConvTile &P, int ntiles, int ny, cudaStream_t st, char *err, size_t errlen)
{
    constexpr uint32_t kStage = (128 + BN) * CK * 2;
    constexpr int kCols = (int)tmem_cols(BN);
    // at most 512 / kCols CTAs may hold tensor memory on one SM at a time:
    // ask for enough shared memory that no more than that become resident
    const int min_smem = 232448 / (512 / kCols) + 1024;
    int smem = (int)(S * kStage + 1024);
    if (smem < min_smem) smem = min_smem;
    auto kern = conv3d_tc_kernel<BN, CK, S>;
    static bool attr_set = false;   // once per instantiation: allow the full opt-in shared memory
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = allow_max_smem(reinterpret_cast<const void *>(kern));
        attr_set = e == cudaSuccess;
    }
    if (e == cudaSuccess) {
        kern<<<dim3((unsigned)ntiles, (unsigned)ny), kThreads, smem, st>>>(mx, mw, bias, ob, of, P);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "conv3d_tc: %s", cudaGetErrorString(e));
        return NN_E_CUDA;
    }
    return NN_OK;
}

template <int CK>
int dispatch_bn(int BN, const CUtensorMap &mx, const CUtensorMap &mw, const float *bias, __nv_bfloat16 *ob,
                float *of, const ConvTile &P, int ntiles, int ny, cudaStream_t st, char *err, size_t errlen)
{
    switch (BN) {
    case 16: return launch<16, CK, 4>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    case 32: return launch<32, CK, 4>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    case 48: return launch<48, CK, 4>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    case 64: return launch<64, CK, 4>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    case 128: return launch<128, CK, 4>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    case 256: return launch<256, CK, 3>(mx, mw, bias, ob, of, P, ntiles, ny, st, err, errlen);
    default: break;
    }
    snprintf(err, errlen, "conv3d_tc: no kernel for %d output channels per tile", BN);
    return NN_E_INVAL;
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            n = 148;
    }
    return n;
}

template <int BN, int CK, int S, bool RESW>
int launch_halo(const CUtensorMap &mx, const CUtensorMap &mw, const float *bias, __nv_bfloat16 *ob, float *of,
                const HaloTile &P, uint32_t smem, cudaStream_t st, char *err, size_t errlen)
{
    auto kern = conv3d_tc_halo_kernel<BN, CK, S, RESW>;
    static bool attr_set = false;   // once per instantiation: allow the full opt-in shared memory
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = allow_max_smem(reinterpret_cast<const void *>(kern));
        attr_set = e == cudaSuccess;
    }
    if (e == cudaSuccess) {
        // persistent: as many CTAs as shared memory (228 KB per SM, 1 KB reserved
        // per CTA) and tensor memory allow
        const int fit = (int)(233472 / (smem + 1024 + 1024));
        const int per_sm = std::max(1, std::min(fit, (int)(512 / (2 * tmem_cols(BN)))));
        const long long grid = std::min<long long>(P.ntiles, (long long)num_sms() * per_sm);
        kern<<<(unsigned)grid, kHaloThreads, smem, st>>>(mx, mw, bias, ob, of, P);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "conv3d_tc (halo): %s", cudaGetErrorString(e));
        return NN_E_CUDA;
    }
    return NN_OK;
}

// Stages and weight residency of the halo kernel for this shape, or 0 stages
// when it does not fit in shared memory.
struct HaloPlan {
    int stages;
    bool resw;
    uint32_t smem;
};

// Measured on the U-Net layers at 128^3: two resident CTAs per SM (one's
// epilogue and loads overlapping the other's products) beat one CTA with a
// deeper ring, so the plan first looks for the deepest ring that still lets two
// CTAs share an SM, then for the deepest one that fits alone. Resident weights
// win ties.
HaloPlan plan_halo(int BN, int CK, int Cin, int ntn)
{
    const uint32_t wbytes = 27u * (uint32_t)Cin * (uint32_t)BN * 2u;
    const uint32_t sa = halo_stage_bytes(BN, CK, true), sb = halo_stage_bytes(BN, CK, false);
    const uint32_t two = 233472u / 2u - 2048u;   // per-CTA budget for two CTAs per SM
    for (uint32_t budget : {two, kMaxDynSmem}) {
        for (int st = 4; st >= 2; --st) {
            const uint32_t r = (uint32_t)st * sa + wbytes + 1024, t = (uint32_t)st * sb + 1024;
            if (ntn == 1 && r <= budget) return {st, true, r};
            if (t <= budget) return {st, false, t};
        }
    }
    return {0, false, 0};
}

template <int BN, int CK>
int dispatch_halo_stages(const HaloPlan &pl, const CUtensorMap &mx, const CUtensorMap &mw, const float *bias,
                         __nv_bfloat16 *ob, float *of, const HaloTile &P, cudaStream_t st, char *err, size_t errlen)
{
    if (pl.resw) {
        if (pl.stages == 4) return launch_halo<BN, CK, 4, true>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
        if (pl.stages == 3) return launch_halo<BN, CK, 3, true>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
        return launch_halo<BN, CK, 2, true>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
    }
    if (pl.stages == 4) return launch_halo<BN, CK, 4, false>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
    if (pl.stages == 3) return launch_halo<BN, CK, 3, false>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
    return launch_halo<BN, CK, 2, false>(mx, mw, bias, ob, of, P, pl.smem, st, err, errlen);
}

template <int CK>
int dispatch_halo(int BN, const HaloPlan &pl, const CUtensorMap &mx, const CUtensorMap &mw, const float *bias,
                  __nv_bfloat16 *ob, float *of, const HaloTile &P, cudaStream_t st, char *err, size_t errlen)
{
    switch (BN) {
    case 16: return dispatch_halo_stages<16, CK>(pl, mx, mw, bias, ob, of, P, st, err, errlen);
    case 32: return dispatch_halo_stages<32, CK>(pl, mx, mw, bias, ob, of, P, st, err, errlen);
    case 48: return dispatch_halo_stages<48, CK>(pl, mx, mw, bias, ob, of, P, st, err, errlen);
    case 64: return dispatch_halo_stages<64, CK>(pl, mx, mw, bias, ob, of, P, st, err, errlen);
    default: break;
    }
    snprintf(err, errlen, "conv3d_tc (halo): no kernel for %d output channels per tile", BN);
    return NN_E_INVAL;
}

}  // namespace

// Shapes the tensor-core path takes: 3x3x3 kernels with input and output
// channel counts that are positive multiples of 16.
bool supported(int Cin, int Cout) { return Cin > 0 && Cout > 0 && Cin % 16 == 0 && Cout % 16 == 0; }

namespace {
// Channels per K stage: the widest of 64, 32, 16 that divides Cin.
int chunk_for(int Cin) { return Cin % 64 == 0 ? 64 : Cin % 32 == 0 ? 32 : 16; }
// Output channels per CTA: the widest tile width that divides Cout.
int tile_n_for(int Cout)
{
    for (int bn : {256, 128, 64, 48, 32, 16})
        if (Cout % bn == 0) return bn;
    return 0;
}
// The same for the halo kernel, which takes at most 64 channels per tile.
int halo_n_for(int Cout)
{
    for (int bn : {64, 48, 32, 16})
        if (Cout % bn == 0) return bn;
    return 0;
}

// Halo kernel for this shape if it fits (stages > 0), with its tensor maps.
int run_halo(const void *in, const void *wt, const float *bias, void *out_bf16, float *out_f32, int N, int D, int H,
             int W, int Cin, int Cout, int relu, cudaStream_t st, char *err, size_t errlen, bool *taken)
{
    *taken = false;
    const int CK = chunk_for(Cin), BN = halo_n_for(Cout);
    if (!BN) return NN_OK;
    const int ntn = Cout / BN;
    const HaloPlan pl = plan_halo(BN, CK, Cin, ntn);
    if (!pl.stages) return NN_OK;
    HaloTile P{};
    P.N = N; P.D = D; P.H = H; P.W = W; P.Cin = Cin; P.Cout = Cout; P.relu = relu;
    P.tw = (W + kHaloW - 1) / kHaloW;
    P.th = (H + kHaloH - 1) / kHaloH;
    P.ntn = ntn;
    P.ntiles = (long long)ntn * P.tw * P.th * D * N;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    const CUtensorMapSwizzle sw = CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : CK == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
    CUtensorMap mx, mw;
    const cuuint64_t gx[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t sx[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2,
                              (cuuint64_t)D * H * W * Cin * 2};
    const cuuint32_t bx[5] = {(cuuint32_t)CK, (cuuint32_t)kHaloW, (cuuint32_t)(kHaloH + 2), 3, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    CUresult r1 = enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(in), gx, sx, bx, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // weights [27][Cout][Cin] viewed as [9][3][Cout][Cin]: tap t = dx' + 3 m
    const cuuint64_t gw[4] = {(cuuint64_t)Cin, (cuuint64_t)Cout, 3, 9};
    const cuuint64_t swd[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)Cout * Cin * 2, 3ull * Cout * Cin * 2};
    const cuuint32_t bw[4] = {(cuuint32_t)CK, (cuuint32_t)BN, 1, 9};
    CUresult r2 = enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(wt), gw, swd, bw, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
        snprintf(err, errlen, "conv3d_tc (halo): tensor map encoding failed (%d, %d)", (int)r1, (int)r2);
        return NN_E_INVAL;
    }
    *taken = true;
    auto *ob = static_cast<__nv_bfloat16 *>(out_bf16);
    if (CK == 64) return dispatch_halo<64>(BN, pl, mx, mw, bias, ob, out_f32, P, st, err, errlen);
    if (CK == 32) return dispatch_halo<32>(BN, pl, mx, mw, bias, ob, out_f32, P, st, err, errlen);
    return dispatch_halo<16>(BN, pl, mx, mw, bias, ob, out_f32, P, st, err, errlen);
}
}  // namespace

int conv3d_fwd(const void *in, const void *wt, const float *bias, void *out_bf16, float *out_f32, int N, int D, int H,
               int W, int Cin, int Cout, int relu, cudaStream_t st, char *err, size_t errlen, int variant)
{
    if (!supported(Cin, Cout)) {
        snprintf(err, errlen, "conv3d_tc: unsupported channels %d -> %d", Cin, Cout);
        return NN_E_INVAL;
    }
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(wt) | reinterpret_cast<uintptr_t>(out_bf16) |
         reinterpret_cast<uintptr_t>(out_f32)) & 15u) {
        snprintf(err, errlen, "conv3d_tc: buffers must be 16-byte aligned");
        return NN_E_INVAL;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        snprintf(err, errlen, "conv3d_tc: cuTensorMapEncodeTiled is not available");
        return NN_E_CUDA;
    }
    if (variant != kVariantTap) {
        bool taken = false;
        const int rc = run_halo(in, wt, bias, out_bf16, out_f32, N, D, H, W, Cin, Cout, relu, st, err, errlen, &taken);
        if (taken || rc != NN_OK) return rc;
        if (variant == kVariantHalo) {
            snprintf(err, errlen, "conv3d_tc: the halo kernel does not take %d -> %d channels", Cin, Cout);
            return NN_E_INVAL;
        }
    }
    const int CK = chunk_for(Cin);
    const int BN = tile_n_for(Cout);
    ConvTile P{};
    P.N = N; P.D = D; P.H = H; P.W = W; P.Cin = Cin; P.Cout = Cout; P.relu = relu;
    P.Wt = pow2_at_least(W, 128);
    P.Ht = pow2_at_least(H, 128 / P.Wt);
    P.Dt = 128 / (P.Wt * P.Ht);
    P.tw = (W + P.Wt - 1) / P.Wt;
    P.th = (H + P.Ht - 1) / P.Ht;
    P.td = (D + P.Dt - 1) / P.Dt;
    const long long ntiles = (long long)P.tw * P.th * P.td * N;
    if (ntiles > 0x7FFFFFFFLL) {
        snprintf(err, errlen, "conv3d_tc: volume too large");
        return NN_E_INVAL;
    }
    const CUtensorMapSwizzle sw = CK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : CK == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_32B;
    CUtensorMap mx, mw;
    const cuuint64_t gx[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t sx[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2,
                              (cuuint64_t)D * H * W * Cin * 2};
    const cuuint32_t bx[5] = {(cuuint32_t)CK, (cuuint32_t)P.Wt, (cuuint32_t)P.Ht, (cuuint32_t)P.Dt, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    CUresult r1 = enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(in), gx, sx, bx, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const cuuint64_t gw[3] = {(cuuint64_t)Cin, (cuuint64_t)Cout, 27};
    const cuuint64_t sw_[2] = {(cuuint64_t)Cin * 2, (cuuint64_t)Cout * Cin * 2};
    const cuuint32_t bw[3] = {(cuuint32_t)CK, (cuuint32_t)BN, 1};
    CUresult r2 = enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(wt), gw, sw_, bw, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
        snprintf(err, errlen, "conv3d_tc: tensor map encoding failed (%d, %d)", (int)r1, (int)r2);
        return NN_E_INVAL;
    }
    const int ny = Cout / BN;
    auto *ob = static_cast<__nv_bfloat16 *>(out_bf16);
    if (CK == 64) return dispatch_bn<64>(BN, mx, mw, bias, ob, out_f32, P, (int)ntiles, ny, st, err, errlen);
    if (CK == 32) return dispatch_bn<32>(BN, mx, mw, bias, ob, out_f32, P, (int)ntiles, ny, st, err, errlen);
    return dispatch_bn<16>(BN, mx, mw, bias, ob, out_f32, P, (int)ntiles, ny, st, err, errlen);
}

// Weight gradient of a 3x3x3 convolution on tcgen05 (Cin, Cout multiples of
// 16). gw and gb accumulate (FP32).
bool wgrad_supported(int Cin, int Cout) { return supported(Cin, Cout); }

namespace {
CUtensorMapSwizzle swizzle_for(int ck)
{
    return ck == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : ck == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}
}  // namespace

int conv3d_wgrad(const void *in, const void *gout, float *gw, float *gb, int N, int D, int H, int W, int Cin,
                 int Cout, cudaStream_t st, char *err, size_t errlen)
{
    if (!wgrad_supported(Cin, Cout)) {
        snprintf(err, errlen, "conv3d_wgrad_tc: unsupported channels %d -> %d", Cin, Cout);
        return NN_E_INVAL;
    }
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(gout) | reinterpret_cast<uintptr_t>(gw)) &
        15u) {
        snprintf(err, errlen, "conv3d_wgrad_tc: buffers must be 16-byte aligned");
        return NN_E_INVAL;
    }
    if (Cout / 8 > 256) {
        snprintf(err, errlen, "conv3d_wgrad_tc: bias gradient takes at most 2048 channels");
        return NN_E_INVAL;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        snprintf(err, errlen, "conv3d_wgrad_tc: cuTensorMapEncodeTiled unavailable");
        return NN_E_CUDA;
    }
    WgradArgs P{};
    P.N = N; P.D = D; P.H = H; P.W = W; P.Cin = Cin; P.Cout = Cout;
    // N tile: the widest of 256, 192, 128, 96, 64, 48, 32, 16 dividing Cout
    for (int c : {256, 192, 128, 96, 64, 48, 32, 16})
        if (Cout % c == 0) { P.NT = c; break; }
    P.CK = Cin % 64 == 0 ? 64 : Cin % 32 == 0 ? 32 : 16;
    P.CKB = P.NT % 64 == 0 ? 64 : P.NT % 32 == 0 ? 32 : 16;
    P.cols = tmem_cols(P.NT);
    P.groups = (27 * Cin + 127) / 128;
    // Launch plan (measured on the U-Net's layers; TMA issue of many small
    // boxes, not the tensor core, bounds the narrow layers, so the plan keeps
    // boxes at 64 voxels where it can and several producers per SM):
    //   N tile 192-256: two row blocks share each gout box, one CTA per SM;
    //   N tile 128: one row block, four CTAs per SM;
    //   narrower: two row blocks, two CTAs per SM.
    int per_sm;
    uint32_t budget;                                   // stage-ring bytes per CTA
    if (P.cols == 256) { P.MG = 2; per_sm = 1; budget = 200 * 1024; }
    else if (P.NT == 128) { P.MG = 1; per_sm = 4; budget = 40 * 1024; }
    else { P.MG = 2; per_sm = 2; budget = 96 * 1024; }
    if (P.MG > P.groups) P.MG = 1;
    // voxel box of KV voxels (x first, then y, then z): 64 if two stages fit
    P.KV = (uint32_t)(P.MG * 128 + P.NT) * 64 * 2 * 2 <= budget ? 64 : 32;
    P.Wb = pow2_at_least(W, P.KV);
    P.Hb = pow2_at_least(H, P.KV / P.Wb);
    P.Db = P.KV / (P.Wb * P.Hb);
    P.tw = (W + P.Wb - 1) / P.Wb;
    P.th = (H + P.Hb - 1) / P.Hb;
    P.td = (D + P.Db - 1) / P.Db;
    const long long ntiles = (long long)N * P.td * P.th * P.tw;
    if (ntiles > 0x7fffffffLL) {
        snprintf(err, errlen, "conv3d_wgrad_tc: volume too large");
        return NN_E_INVAL;
    }
    P.ntiles = (int)ntiles;
    P.stage_bytes = (uint32_t)(P.MG * 128 + P.NT) * P.KV * 2;
    P.S = (int)std::min<uint32_t>(kWgMaxStages, budget / P.stage_bytes);
    if (P.S < 2) {
        snprintf(err, errlen, "conv3d_wgrad_tc: no stage plan for %d -> %d", Cin, Cout);
        return NN_E_INVAL;
    }
    // one wave of CTAs, per_sm on each SM
    const long long xy = (long long)((P.groups + P.MG - 1) / P.MG) * (Cout / P.NT);
    long long splits = std::max<long long>(1, (long long)num_sms() * per_sm / xy);
    splits = std::min<long long>(splits, P.ntiles);
    P.stride = (int)splits;
    // Shared memory caps the CTAs per SM at the number whose tensor
    // memory (MG * cols columns each) fits in 512 columns: one more CTA of
    // this size would exceed the SM's shared memory.
    static int sm_smem = 0;
    if (!sm_smem) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
            sm_smem = 233472;
    }
    const int tmem_fit = sm_smem / (512 / (P.MG * (int)P.cols) + 1) + 1;
    // ... and at per_sm, so that the wave spreads evenly over the SMs
    const int wave_fit = sm_smem / (per_sm + 1) + 1;
    const int smem = std::max<int>((int)(P.S * P.stage_bytes) + 1024, std::max(tmem_fit, wave_fit));

    CUtensorMap mx, mg;
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    const cuuint64_t gx[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t sx[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2,
                              (cuuint64_t)D * H * W * Cin * 2};
    const cuuint32_t bx[5] = {(cuuint32_t)P.CK, (cuuint32_t)P.Wb, (cuuint32_t)P.Hb, (cuuint32_t)P.Db, 1};
    CUresult r1 = enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(in), gx, sx, bx, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(P.CK), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const cuuint64_t gg[5] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t sg[4] = {(cuuint64_t)Cout * 2, (cuuint64_t)W * Cout * 2, (cuuint64_t)H * W * Cout * 2,
                              (cuuint64_t)D * H * W * Cout * 2};
    const cuuint32_t bg[5] = {(cuuint32_t)P.CKB, (cuuint32_t)P.Wb, (cuuint32_t)P.Hb, (cuuint32_t)P.Db, 1};
    CUresult r2 = enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(gout), gg, sg, bg, ones,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(P.CKB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
        snprintf(err, errlen, "conv3d_wgrad_tc: tensor map encoding failed (%d, %d)", (int)r1, (int)r2);
        return NN_E_INVAL;
    }
    static bool attr_set = false;
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = allow_max_smem(reinterpret_cast<const void *>(conv3d_wgrad_tc_kernel));
        attr_set = e == cudaSuccess;
    }
    if (e == cudaSuccess) {
        conv3d_wgrad_tc_kernel<<<dim3((unsigned)((P.groups + P.MG - 1) / P.MG), (unsigned)(Cout / P.NT),
                                      (unsigned)splits),
                                 kThreads, smem, st>>>(mx, mg, gw, P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && gb) {
        const long long V = (long long)N * D * H * W;
        bias_grad_kernel<<<num_sms() * 4, 256, Cout * sizeof(float), st>>>((const __nv_bfloat16 *)gout, gb, V, Cout);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "conv3d_wgrad_tc: %s", cudaGetErrorString(e));
        return NN_E_CUDA;
    }
    return NN_OK;
}

// Read and clear the device-side status word (bit 0: an mbarrier wait timed out).
int take_status(cudaStream_t st, unsigned *out)
{
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_status, sizeof v, 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbolAsync(g_status, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    *out = v;
    return e == cudaSuccess ? NN_OK : NN_E_CUDA;
}

}  // namespace nn_tc
