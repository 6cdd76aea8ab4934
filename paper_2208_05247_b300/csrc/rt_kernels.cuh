// rt_kernels.cuh -- kernels of the shortwave Monte Carlo tracer
// (Veerman et al. 2022, Sec. 2.3).
//
//   derive_optics   per-cell record {k_abs, k_sca, k_sca*P(cloud|scatter), g}
//                   from the five gas/cloud fields, with validation
//   build_majorant  coarse-grid maximum of k_ext (the null-collision coefficient)
//   box_*           majorant boxes: per coarse cell a cube of low optical depth
//                   that one walk step may cross
//   trace_kernel    persistent photon transport with warp-level refill:
//                   null-collision tracking over the majorant boxes, weights,
//                   roulette, Lambertian surface, FP32 partial -> FP64 tallies
//   fields kernels  FP64 normalisation of the tallies into output fields
//
// Everything here has internal linkage: the files that include this header
// each compile their own copy of the kernels they launch.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "rt_device.cuh"

namespace rt {
namespace {   // internal linkage: each .cu file that includes this header has its own copy

constexpr int kStatusBudget = 1;
constexpr int kStatusInput = 2;                        // an rt_step launch found invalid inputs
constexpr int kStatusBounds = 4;                       // an index check failed (RT_CHECK_BOUNDS builds)

// Index i into an array of n elements. Unchanged in normal builds. A build
// with RT_CHECK_BOUNDS=1 (the library's bounds-checking variant, for tests:
// compute-sanitizer is not available) checks it: an index outside [0, n) sets
// kStatusBounds in the launch's status word and is replaced by 0, so the access
// stays inside the array and nothing traps.
#ifndef RT_CHECK_BOUNDS
#define RT_CHECK_BOUNDS 0
#endif
__device__ __forceinline__ long long checked_index(long long i, long long n, int *status)
{
#if RT_CHECK_BOUNDS
    if (i < 0 || i >= n) {
        atomicOr(status, kStatusBounds);
        return 0;
    }
#else
    (void)n;
    (void)status;
#endif
    return i;
}
constexpr unsigned long long kQueueClosed = 1ull << 62; // queue head that no launch ever reaches

// Per-handle device scratch: the photon queue head, counters and ledger.
struct Scratch {
    unsigned long long queue_head;
    unsigned long long photons, events, scatters, crossings, surface_hits, roulette_kills, capped,
        max_events;
    double created, destroyed, capped_energy;
    double e_toa, e_atm, e_sfc;
    int status;
    int bad;
};

template <typename T>
struct Tallies {
    T *abs_dir, *abs_dif;           // [ncell]
    T *sfc_dir, *sfc_dif, *toa;     // [ncol]
};

constexpr int kMaxBatchScenes = 16;
constexpr int kMaxBatchJobs = 512;

// How a launch reads the optics of a cell at an event.
enum : int {
    kOpticsRecord = 0,   // single scene: derived record {k_abs, k_sca, k_sca*P(cloud), g}
    kOpticsSplit = 1,    // batched: {k_abs,gas, k_sca,gas, k_abs,cloud, k_sca,cloud} and cloud g,
                         // gas scaled per quadrature point
    kOpticsFields = 2    // the five input fields themselves (no derived record in memory)
};

// One scene as the transport kernel sees it.
template <typename T>
struct SceneDev {
    const float4 *rec;     // kOpticsRecord / kOpticsSplit record per cell
    const float *gcl;      // kOpticsSplit and kOpticsFields: cloud asymmetry per cell
    const float *f_kg, *f_wg, *f_kc, *f_wc;   // kOpticsFields: gas/cloud extinction and albedo
    const uint32_t *box;   // majorant box word per coarse cell (single scene)
    const uint2 *box2;     // batched: {gas, cloud} majorant box words per coarse cell
    const float *alb;      // [ny][nx]
    Tallies<T> tal;
    Scratch *scr;
    int nx, ny, nz, NX, NY, NZ, cx, cy, cz, pcld_mode;
    float dx, dy, dz, inv_dx, inv_dy, inv_dz, Lx, Ly, H;
    float cdx, cdy, cdz;   // coarse cell size [m] (the last cell may be smaller)
    float inv_cdx, inv_cdy, inv_cdz;
    int birth;             // start positions: 0 Philox uniforms, 1 scrambled Sobol
    // face caps: with a shorter last coarse cell along x (or y) the face at NX
    // is the domain edge (xcap = Lx, fxcap = nx); otherwise +inf / INT_MAX
    float xcap, ycap;
    int fxcap, fycap;
};

// One traced job: a scene, a sun position, an energy per photon and a range of
// photon ids; in a batched launch one job per (scene, g-point).
struct JobDev {
    unsigned long long start;      // first queue index of the job
    unsigned long long id_begin;   // photon id of that queue index
    unsigned long long ncol;
    float sx, sy, sz;              // travel direction of the direct beam
    float gas_scale;               // multiplies the gas extinction (batched launches)
    uint32_t key0, key1;           // Philox key
    int scene;
    float diffuse;                 // fraction of photons that start diffuse (isotropic downwelling)
    double energy;                 // W per unit photon weight
    double scale2, scale3;         // energy / (dx dy), energy / (dx dy dz)
};

static_assert(sizeof(SceneDev<double>) % 16 == 0 && sizeof(SceneDev<float>) % 16 == 0,
              "scene descriptors are copied to shared memory in 16-byte words");
static_assert(sizeof(JobDev) % 16 == 0, "job descriptors are copied in 16-byte words");

template <typename T>
struct TraceArgs {
    SceneDev<T> scene;             // single-scene launches
    JobDev job;
    const SceneDev<T> *scenes;     // batched launches (copied into shared memory)
    const JobDev *jobs;
    int nscenes, njobs;
    unsigned long long count;      // photons of the launch
    Scratch *scr;                  // queue head; counters of single-scene launches
    uint32_t max_steps;
    uint32_t chunk;
    int ready_threshold;           // lanes that must be ready before an interaction sweep
    int max_inner;                 // bound on walk sweeps per interaction sweep
    int refill_min;                // dead lanes a warp gathers before it refills
    // single-scene launches of whole photon rounds: queue index q takes photon
    // (order_k0 + q mod order_ppc) * ncol + order[q div order_ppc], i.e. all
    // photons of one column in turn, columns in the order of `order`
    const uint32_t *order;
    uint32_t order_ppc;
    unsigned long long order_k0;
};

// ---------------------------------------------------------------------------
// a1 for one cell, shared by the derivation kernel and the launches that read
// the five input fields directly: explicit roundings (no contraction into
// fused multiply-adds), so both give the same bits.
// ---------------------------------------------------------------------------
struct CellOptics {
    float kabs, ksca, kscl;   // absorption, scattering, scattering by cloud
};

__device__ __forceinline__ CellOptics cell_optics(float kg, float wg, float kc, float wc, int pcld_mode)
{
    const float ksg = __fmul_rn(kg, wg), ksc = __fmul_rn(kc, wc);
    CellOptics o;
    o.ksca = __fadd_rn(ksg, ksc);
    o.kabs = __fadd_rn(__fmul_rn(kg, __fsub_rn(1.0f, wg)), __fmul_rn(kc, __fsub_rn(1.0f, wc)));
    o.kscl = ksc;
    if (pcld_mode == 1) {
        const float ke = __fadd_rn(kg, kc);
        o.kscl = ke > 0.0f ? __fmul_rn(o.ksca, __fdiv_rn(kc, ke)) : 0.0f;
    }
    return o;
}

// ---------------------------------------------------------------------------
// a1: optics record. k_abs = k_g (1 - w_g) + k_c (1 - w_c); k_sca = k_g w_g + k_c w_c;
// the third entry is k_sca times the probability that a scattering is by cloud:
// k_c w_c (scattering ratio) or k_sca k_c / (k_g + k_c) (the paper's extinction
// ratio, Sec. 2.3). Invalid inputs raise `bad` (no trap).
// ---------------------------------------------------------------------------
__global__ void derive_optics(const float *__restrict__ kg, const float *__restrict__ wg,
                              const float *__restrict__ kc, const float *__restrict__ wc,
                              const float *__restrict__ gc, float4 *__restrict__ rec, size_t n,
                              int pcld_mode, int *bad)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float a = kg[i], b = wg[i], c = kc[i], d = wc[i], g = gc[i];
        const bool ok = (a >= 0.0f) && (a <= 3.0e38f) && (c >= 0.0f) && (c <= 3.0e38f) &&
                        (b >= 0.0f) && (b <= 1.0f) && (d >= 0.0f) && (d <= 1.0f) &&
                        (fabsf(g) < 1.0f);
        if (!ok) atomicOr(bad, 1);
        const CellOptics o = cell_optics(a, b, c, d, pcld_mode);
        rec[i] = make_float4(o.kabs, o.ksca, o.kscl, g);
    }
}

// The paper's own inputs (Sec. 2.3): total extinction, cloud extinction, one
// single-scattering albedo and g. The record follows: k_sca = w k_ext,
// k_abs = k_ext - k_sca, and the cloud share of scattering is k_ext,cloud/k_ext.
__global__ void derive_optics_total(const float *__restrict__ ke, const float *__restrict__ kc,
                                    const float *__restrict__ w, const float *__restrict__ gc,
                                    float4 *__restrict__ rec, size_t n, int *bad)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float e = ke[i], c = kc[i], a = w[i], g = gc[i];
        const bool ok = (e >= 0.0f) && (e <= 3.0e38f) && (c >= 0.0f) && (c <= e) && (a >= 0.0f) && (a <= 1.0f) &&
                        (fabsf(g) < 1.0f);
        if (!ok) atomicOr(bad, 1);
        const float ksca = e * a;
        const float kabs = e * (1.0f - a);
        const float zc = e > 0.0f ? ksca * (c / e) : 0.0f;
        rec[i] = make_float4(kabs, ksca, zc, g);
    }
}

__global__ void check_albedo(const float *__restrict__ alb, size_t n, int *bad)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float a = alb[i];
        if (!(a >= 0.0f && a <= 1.0f)) atomicOr(bad, 1);
    }
}

// ---------------------------------------------------------------------------
// a2: majorant grid (Sec. 2.3: each coarse cell holds the highest extinction of
// the fine cells it covers). One thread per coarse cell; the last coarse cell
// along an axis covers the remainder.
// ---------------------------------------------------------------------------
// Grid-stride loops over coarse cells count with an unsigned index: n < 2^31,
// and q + stride (at most 148 * 32 blocks of 256 threads) then stays below
// 2^32, where a signed index could overflow on grids of nearly 2^31 cells.
__global__ void build_majorant(const float4 *__restrict__ rec, float *__restrict__ kmax, int nx,
                               int ny, int nz, int cx, int cy, int cz, int NX, int NY, int NZ)
{
    const int n = NX * NY * NZ;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const int I = q % NX, J = (q / NX) % NY, K = q / (NX * NY);
        const int i1 = min(I * cx + cx, nx), j1 = min(J * cy + cy, ny), k1 = min(K * cz + cz, nz);
        float m = 0.0f;
        for (int k = K * cz; k < k1; ++k)
            for (int j = J * cy; j < j1; ++j) {
                const float4 *row = rec + ((size_t)k * ny + j) * nx;
                for (int i = I * cx; i < i1; ++i) {
                    const float4 o = __ldg(row + i);
                    m = fmaxf(m, o.x + o.y);
                }
            }
        kmax[q] = m;
    }
}

// ---------------------------------------------------------------------------
// Launch order. A launch lasts as long as its longest photon history, and the
// longest histories are random walks through thick cloud. Starting the photons
// of the optically thickest columns first lets those histories overlap with
// the rest of the launch instead of trailing it. A photon's history depends
// only on its id, so the order changes no result (FP64 atomic rounding aside).
// ---------------------------------------------------------------------------
constexpr int kOrderKeys = 256;

// Key of each coarse column: 255 - min(255, 16 log2(1 + tau)), with tau the
// majorant optical depth of the column (sum of k_max times coarse cell height).
// Thick columns get low keys.
__global__ void column_keys(const float *__restrict__ kmax, int NX, int NY, int NZ, float cdz, float H,
                            unsigned char *__restrict__ key)
{
    const int n = NX * NY;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        float tau = 0.f;
        for (int K = 0; K < NZ; ++K)
            tau = fmaf(__ldg(kmax + (size_t)K * n + q), fminf(cdz, H - (float)K * cdz), tau);
        key[q] = (unsigned char)(255 - min(255, (int)(16.f * log2f(1.f + tau))));
    }
}

// One block of 1024 threads: counting sort of the fine columns by the key of
// their coarse column; order[r] is the fine column of rank r. Columns with
// equal keys come in an unspecified order. Most columns share a few keys
// (clear sky), so lanes with equal keys add to a counter once per warp.
// Slot for this lane's key k in counter array cnt: lanes of the warp with equal
// keys share one atomic. Every lane of the warp must call it; k >= kOrderKeys
// marks a lane without a column.
__device__ __forceinline__ unsigned int warp_claim(unsigned int *cnt, unsigned int k)
{
    const unsigned int lane = threadIdx.x & 31u;
    const unsigned int peers = __match_any_sync(0xffffffffu, k);
    const int leader = __ffs(peers) - 1;
    unsigned int base = 0;
    if ((int)lane == leader && k < (unsigned int)kOrderKeys) base = atomicAdd(&cnt[k], (unsigned int)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(1024) order_columns(const unsigned char *__restrict__ key, int nx, int ny, int cx,
                                                      int cy, int NX, uint32_t *__restrict__ order)
{
    __shared__ unsigned int cnt[kOrderKeys];
    const int ncol = nx * ny;
    const int rounds = (ncol + (int)blockDim.x - 1) / (int)blockDim.x;   // equal for every thread
    for (int b = threadIdx.x; b < kOrderKeys; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
        const int c = r * (int)blockDim.x + (int)threadIdx.x;
        warp_claim(cnt, c < ncol ? key[(c / nx / cy) * NX + (c % nx) / cx] : (unsigned int)kOrderKeys);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int b = 0; b < kOrderKeys; ++b) {
            const unsigned int v = cnt[b];
            cnt[b] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
        const int c = r * (int)blockDim.x + (int)threadIdx.x;
        const unsigned int k = c < ncol ? key[(c / nx / cy) * NX + (c % nx) / cx] : (unsigned int)kOrderKeys;
        const unsigned int pos = warp_claim(cnt, k);
        if (c < ncol) order[pos] = (uint32_t)c;
    }
}

// ---------------------------------------------------------------------------
// Batched launches scale the gas extinction per g-point, so they keep gas and
// cloud apart: {k_abs,gas, k_sca,gas, k_abs,cloud, k_sca,cloud} and g per cell,
// and a factored majorant s * max(k_ext,gas) + max(k_ext,cloud) per coarse
// cell, which bounds s k_ext,gas + k_ext,cloud of every fine cell for any gas
// scale s >= 0. Both maxima are raised by 2^-20 relative so the bound still
// holds after the FP32 rounding of the per-cell sums.
// ---------------------------------------------------------------------------
__global__ void derive_split(const float *__restrict__ kg, const float *__restrict__ wg,
                             const float *__restrict__ kc, const float *__restrict__ wc,
                             const float *__restrict__ gc, float4 *__restrict__ rec2, float *__restrict__ gcl,
                             size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float a = kg[i], b = wg[i], c = kc[i], d = wc[i];
        rec2[i] = make_float4(a * (1.0f - b), a * b, c * (1.0f - d), c * d);
        gcl[i] = gc[i];
    }
}

__global__ void build_majorant_split(const float4 *__restrict__ rec2, float2 *__restrict__ kmax2, int nx,
                                     int ny, int nz, int cx, int cy, int cz, int NX, int NY, int NZ)
{
    const int n = NX * NY * NZ;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const int I = q % NX, J = (q / NX) % NY, K = q / (NX * NY);
        const int i1 = min(I * cx + cx, nx), j1 = min(J * cy + cy, ny), k1 = min(K * cz + cz, nz);
        float mg = 0.0f, mc = 0.0f;
        for (int k = K * cz; k < k1; ++k)
            for (int j = J * cy; j < j1; ++j) {
                const float4 *row = rec2 + ((size_t)k * ny + j) * nx;
                for (int i = I * cx; i < i1; ++i) {
                    const float4 o = __ldg(row + i);
                    mg = fmaxf(mg, o.x + o.y);
                    mc = fmaxf(mc, o.z + o.w);
                }
            }
        const float up = 1.0f + 9.5367431640625e-7f;   // 1 + 2^-20
        kmax2[q] = make_float2(mg * up, mc * up);
    }
}

// ---------------------------------------------------------------------------
// Majorant boxes (a2, a4). A walk that crosses one coarse cell per step spends
// most of its steps in clear air, where tens of crossings add up to an optical
// depth of a few hundredths. Every coarse cell therefore also carries a box:
// the cube of coarse cells within Chebyshev radius r of it (periodic in x and
// y, clipped at the surface and the domain top) and the largest extinction in
// that cube. A photon in the cell crosses the whole cube in one step with the
// cube's maximum as its majorant. The bound is >= the extinction everywhere on
// the step, and it may be chosen anew at every step from the photon's current
// position (thinning with a piecewise-constant dominating rate, Sec. 2.3's
// null collisions), so the estimator is unchanged in expectation. r is the
// largest of 0, 1, 3, 7, 15 for which the cube's maximum times the cube's
// diagonal stays below box_tau: a step through a box adds at most about
// box_tau null collisions, while in clear air it replaces up to 2r + 1
// crossings.
//
// Box word: the float bits of the cube maximum with the low four mantissa
// bits replaced by r. Read back with those bits set to one, the majorant is
// >= the cube maximum (at most 15 units in the last place above it).
// ---------------------------------------------------------------------------
constexpr int kBoxLevels = 4;                    // radii 1, 3, 7, 15 (dilation by 1, 2, 4, 8)
constexpr int kDefaultCoarse = 2;                // coarsening factor per axis selected by 0,0,0
// launch defaults shared by rt_create's options and rt_trace_noalloc
constexpr uint32_t kDefaultMaxSteps = 10000000u;
constexpr int kDefaultReadyThreshold = 16;
constexpr int kDefaultMaxInner = 16;
constexpr int kDefaultRefillMin = 8;
constexpr int kDefaultBoxLevels = 4;
constexpr float kDefaultBoxTau = 0.5f;

__device__ __forceinline__ uint32_t box_word(float k, int r) { return (__float_as_uint(k) & ~0xFu) | (uint32_t)r; }
__device__ __forceinline__ float box_kmaj(uint32_t w) { return __uint_as_float(w | 0xFu); }
__device__ __forceinline__ int box_radius(uint32_t w) { return (int)(w & 0xFu); }

// radius 0: every box is its own coarse cell
__global__ void box_init(const float *__restrict__ kmax, float *__restrict__ cur, uint32_t *__restrict__ box, int n)
{
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const float k = kmax[q];
        cur[q] = k;
        box[q] = box_word(k, 0);
    }
}

__global__ void box_init2(const float2 *__restrict__ kmax2, float *__restrict__ curg, float *__restrict__ curc,
                          uint2 *__restrict__ box2, int n)
{
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const float2 m = kmax2[q];
        curg[q] = m.x;
        curc[q] = m.y;
        box2[q] = make_uint2(box_word(m.x, 0), __float_as_uint(m.y) | 0xFu);
    }
}

// One axis of a running-maximum filter of radius rho over the coarse grid:
// axis 0 (x) and 1 (y) periodic, axis 2 (z) clipped. Callers keep rho < NX, NY.
__global__ void box_dilate(const float *__restrict__ in, float *__restrict__ out, int NX, int NY, int NZ, int axis,
                           int rho)
{
    const int n = NX * NY * NZ;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const int I = q % NX, J = (q / NX) % NY, K = q / (NX * NY);
        float m = in[q];
        if (axis == 0) {
            const int row = q - I;
            for (int d = 1; d <= rho; ++d) {
                const int a = I + d >= NX ? I + d - NX : I + d, b = I - d < 0 ? I - d + NX : I - d;
                m = fmaxf(m, fmaxf(in[row + a], in[row + b]));
            }
        } else if (axis == 1) {
            const int base = q - J * NX;
            for (int d = 1; d <= rho; ++d) {
                const int a = J + d >= NY ? J + d - NY : J + d, b = J - d < 0 ? J - d + NY : J - d;
                m = fmaxf(m, fmaxf(in[base + a * NX], in[base + b * NX]));
            }
        } else {
            const int base = q - K * NX * NY;
            for (int k = max(K - rho, 0); k <= min(K + rho, NZ - 1); ++k) m = fmaxf(m, in[base + k * NX * NY]);
        }
        out[q] = m;
    }
}

// Cells whose box still has radius r_prev take radius r_new where the dilated
// maximum m is at most `limit` = box_tau / ((2 r_new + 1) * cell diagonal).
__global__ void box_select(const float *__restrict__ m, uint32_t *__restrict__ box, int n, int r_prev, int r_new,
                           float limit)
{
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const uint32_t w = box[q];
        if (box_radius(w) == r_prev && m[q] <= limit) box[q] = box_word(m[q], r_new);
    }
}

// Batched launches: the radius follows from gas (at scale 1) plus cloud; the
// gas and cloud maxima of the box are kept apart for the per-job gas scale.
__global__ void box_select2(const float *__restrict__ mg, const float *__restrict__ mc, uint2 *__restrict__ box2,
                            int n, int r_prev, int r_new, float limit)
{
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const uint2 w = box2[q];
        if (box_radius(w.x) == r_prev && mg[q] + mc[q] <= limit)
            box2[q] = make_uint2(box_word(mg[q], r_new), __float_as_uint(mc[q]) | 0xFu);
    }
}

// ---------------------------------------------------------------------------
// Tally accumulation (a5, a9, a10): an FP32 partial of photon weight, times
// the job's energy per unit weight in FP64, added to the FP64 (or, for the
// precision study, FP32) global accumulator.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tally_add(double *p, float v, double scale) { atomicAdd(p, (double)v * scale); }
__device__ __forceinline__ void tally_add(float *p, float v, double scale) { atomicAdd(p, (float)((double)v * scale)); }

__device__ __forceinline__ unsigned long long warp_sum_u32(uint32_t v)
{
    return (unsigned long long)__reduce_add_sync(0xffffffffu, v);
}

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Flush of the absorption partials of the lanes with `fl` set (every lane of
// the warp calls it). With `aggregate`, lanes that flush the same (cell,
// direct/diffuse) are grouped (__match_any_sync); the group's lowest lane adds
// the members' partials in lane order and issues the one atomic. Otherwise
// every flushing lane issues its own. Grouping depends on which photons share
// a warp, so aggregated sums are reproducible across launch shapes only to
// FP32 rounding; unaggregated ones to the order of FP64 additions.
template <typename T, bool AGG>
__device__ __forceinline__ void flush_partials(bool fl, T *t_dir, T *t_dif, int cell, bool dir, float acc,
                                               double scale)
{
    if constexpr (!AGG) {
        if (fl) tally_add((dir ? t_dir : t_dif) + cell, acc, scale);
        return;
    }
    const unsigned flm = __ballot_sync(0xffffffffu, fl);
    if (!flm) return;
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t key = fl ? ((uint32_t)cell << 1 | (uint32_t)dir) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(0xffffffffu, key) & flm;
    const int leader = grp ? __ffs(grp) - 1 : (int)lane;
    unsigned rest = grp & ~(1u << leader);
    float sum = acc;
    while (__any_sync(0xffffffffu, rest != 0u)) {
        const int src = rest ? __ffs(rest) - 1 : (int)lane;
        const float v = __shfl_sync(0xffffffffu, acc, src);
        if (rest) sum += v;
        rest &= rest - 1u;
    }
    if (fl && (int)lane == leader) tally_add((dir ? t_dir : t_dif) + cell, sum, scale);
}

// ---------------------------------------------------------------------------
// Geometry of the periodic coarse grid. Boxes of radius r > 0 exist only when
// the coarse cells along x and y all have one size (box_grid_uniform), so a
// coarse face e along x, for any integer e, lies at e * cdx, and the fine cell
// beyond it has index e * cx (both in the periodic extension of the domain).
// With a shorter last coarse cell the radius is 0 everywhere, faces are those
// of the cell itself (e in [0, NX]) and the face at NX is the domain edge:
// min(e * cdx, xcap) with xcap = Lx (fine index min(e * cx, fxcap), fxcap =
// nx), the caps being +inf and INT_MAX otherwise. z is not periodic: a face
// at min(e * cdz, H).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float wrap_coord(float p, float L) { return p < 0.f ? p + L : (p >= L ? p - L : p); }

// ---------------------------------------------------------------------------
// a3-a11: persistent transport kernel.
//
// Every warp loops until the photon queue is empty. One iteration has three
// phases, each warp-synchronous:
//
//  1. refill: once at least refill_min lanes hold no photon (births run with
//     only those lanes active), they flush the ended photons' absorption
//     partials and take new photon ids (one atomicAdd per warp for a chunk of
//     ids, handed out by ballot rank); a new photon is born at the domain top
//     along the sun beam;
//  2. walk: lanes without a pending interaction take box steps (subtracting
//     k_box * l from the remaining optical depth) until the free path ends
//     inside a box (an event), the photon reaches the surface or leaves the
//     top. Sweeps repeat until `ready_threshold` lanes are ready (or none is
//     left to walk, or `max_inner` sweeps), so the costly interaction code
//     runs with most lanes active;
//  3. interact: ready lanes handle their event, surface hit or exit; lanes
//     whose absorption partial moved to another cell flush the old one.
//
// A walk step starts at the photon's position o in coarse cell (I,J,K) with
// box radius r: the distance to the box face ahead along each axis, the
// nearest of the three, and either the event inside the box or the move to
// the neighbouring coarse cell across that face (x and y wrap periodically).
// The crossed axis takes its index from the face. The others take the cell of
// the position, but moved from the start cell only in the direction of travel
// and within the box: a position on a face then stays in the cell the photon
// moves into (the plain cell of the position can put it back behind a face it
// crossed, and two axes can then undo each other's steps forever).
//
// Events (Sec. 2.3, weights after Iwabuchi 2006): at every majorant event the
// cell absorbs w k_abs/k_maj (heating tally) and w shrinks by the same amount;
// the photon then scatters with probability k_sca/(k_maj - k_abs), by cloud
// (HG) or gas (Rayleigh), or has a null collision; below w = 0.5 roulette ends
// it with probability 1 - w or resets w = 1. The surface adds w to the direct
// or diffuse irradiance of its column, multiplies w by the albedo and reflects
// Lambertian. Leaving the top adds w to the upward flux of its column.
// Events and surface hits share one code path.
//
// Random numbers: block b of photon p is Philox(ctr = (p lo, p hi, b, slot)).
// A uniform takes the top 24 bits of a word; the low 8 bits of words 0, 1 and
// 2 form a fifth, independent uniform (u01_low). Birth uses block 0 (x, y,
// first free path, diffuse choice); each event or surface hit uses the next
// block: (choice, mu, phi, next free path) at an event, (-, mu, phi, next free
// path) at the surface, and the fifth uniform for roulette.
//
// Counters: per photon (events, scatterings, box steps) into per-block shared
// totals when the photon ends; per block into the launch scratch at the end.
// ---------------------------------------------------------------------------
enum : int { kNone = 0, kEvent = 1, kSurface = 2, kTop = 3, kCap = 4 };
// per-scene block counters: surface hits, roulette kills, capped photons,
// photons, events, scatterings, box steps, largest event count of a photon
enum : int { kCntSurface = 0, kCntKills, kCntCapped, kCntPhotons, kCntEvents, kCntScatters, kCntSteps, kCntMax, kCnt };

// Scene and job fields of the lane's photon: kernel parameters in single-scene
// launches, shared memory in batched ones (folded at compile time).
#define RT_SC(f) (BATCH ? s_scenes[sid].f : A.scene.f)
#define RT_JB(f) (BATCH ? s_jobs[jid].f : A.job.f)

// Scrambled Sobol start point k of column col (Sec. 2.3): the column's two
// scramble words come from Philox counter (col, 0, 0, 2) under the job's key.
// Kept out of line: it runs once per photon.
__device__ __noinline__ uint2 sobol_start(uint32_t k, uint32_t col, uint32_t k0, uint32_t k1)
{
    const uint4 h = philox4x32_10(make_uint4(col, 0u, 0u, 2u), k0, k1);
    return make_uint2(sobol_dim1(k) ^ h.x, sobol_dim2(k) ^ h.y);
}

constexpr int kMaxWarpsPerBlock = 8;          // blocks of up to 256 threads

// Five blocks of 256 threads per SM (register budget 48 per thread).
// AGG (single-scene launches with rt_options.tally_aggregate) compiles the
// grouped flush as a separate instantiation.
// Five resident blocks of 256 threads per SM (48 registers) for single-scene
// launches; batched launches carry more per-lane state (scene, job, gas
// scale) and run faster at four blocks without spills.
template <typename T, int MODE, bool AGG = false>
__global__ void __launch_bounds__(256, MODE == kOpticsSplit ? 4 : 5) trace_kernel(const __grid_constant__ TraceArgs<T> A)
{
    constexpr bool BATCH = MODE == kOpticsSplit;
    static_assert(!(AGG && BATCH), "batched launches flush per lane (jobs differ in energy)");
    constexpr unsigned kFull = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    const int wid = threadIdx.x >> 5;

    // batched launches: scene and job descriptors in dynamic shared memory
    extern __shared__ __align__(16) unsigned char s_dyn[];
    SceneDev<T> *s_scenes = reinterpret_cast<SceneDev<T> *>(s_dyn);
    JobDev *s_jobs = reinterpret_cast<JobDev *>(s_dyn + (BATCH ? A.nscenes : 0) * sizeof(SceneDev<T>));
    constexpr int NS = BATCH ? kMaxBatchScenes : 1;
    __shared__ unsigned long long s_cnt[NS][kCnt];
    __shared__ double s_led[NS][3];          // roulette created, destroyed, capped energy
    // each warp's share of the photon queue: next and end index, queue empty
    __shared__ unsigned long long s_q[kMaxWarpsPerBlock][2];
    __shared__ int s_exh[kMaxWarpsPerBlock];
    for (int q = threadIdx.x; q < NS * kCnt; q += blockDim.x) s_cnt[q / kCnt][q % kCnt] = 0;
    for (int q = threadIdx.x; q < NS * 3; q += blockDim.x) s_led[q / 3][q % 3] = 0.0;
    if (lane == 0) {
        s_q[wid][0] = s_q[wid][1] = 0;
        s_exh[wid] = 0;
    }
    if (BATCH) {
        const int4 *src = reinterpret_cast<const int4 *>(A.scenes);
        int4 *dst = reinterpret_cast<int4 *>(s_scenes);
        for (int q = threadIdx.x; q < (int)(A.nscenes * sizeof(SceneDev<T>) / 16); q += blockDim.x) dst[q] = src[q];
        const int4 *js = reinterpret_cast<const int4 *>(A.jobs);
        int4 *jd = reinterpret_cast<int4 *>(s_jobs);
        for (int q = threadIdx.x; q < (int)(A.njobs * sizeof(JobDev) / 16); q += blockDim.x) jd[q] = js[q];
    }
    __syncthreads();

    int sid = 0, jid = 0;                     // scene and job of the lane's photon
    float ox = 0.f, oy = 0.f, oz = 0.f;       // photon position at the start of the walk step
    float ux = 0.f, uy = 0.f, uz = -1.f;      // direction
    float ivx = 0.f, ivy = 0.f, ivz = 0.f;    // 1/u per axis (used only on axes that move)
    float w = 0.f, kmaj = 0.f;                // weight, box majorant
    float tau = 0.f;                          // optical depth left; once an event is found,
                                              // its distance from o
    int I = 0, J = 0, K = 0, r = 0;           // coarse cell and its box radius
    unsigned long long gid = 0;
    uint32_t blk = 0, nev = 0, ncr = 0, nsc = 0;   // Philox block; events, box steps, scatterings
    bool alive = false, direct = false;
    int ready = kNone;
    int pcell = -1;                           // absorption partial: cell, direct flag, FP32 sum
    bool pdir = false;
    float pacc = 0.f;

    using BoxWord = typename std::conditional<BATCH, uint2, uint32_t>::type;
    auto set_box = [&](BoxWord b) {
        if constexpr (BATCH) {
            r = box_radius(b.x);
            kmaj = fmaf(RT_JB(gas_scale), box_kmaj(b.x), box_kmaj(b.y));
        } else {
            r = box_radius(b);
            kmaj = box_kmaj(b);
        }
    };
    // coarse cell of a position inside the periodic domain (cell_of: its
    // index only; locate: make it the walk's current cell)
    auto cell_of = [&](float px, float py, float pz, int &i, int &j, int &k) {
        i = min(max((int)(px * RT_SC(inv_cdx)), 0), RT_SC(NX) - 1);
        j = min(max((int)(py * RT_SC(inv_cdy)), 0), RT_SC(NY) - 1);
        k = min(max((int)(pz * RT_SC(inv_cdz)), 0), RT_SC(NZ) - 1);
        return (int)checked_index((k * RT_SC(NY) + j) * RT_SC(NX) + i,
                                  (long long)RT_SC(NX) * RT_SC(NY) * RT_SC(NZ), &RT_SC(scr)->status);
    };
    auto locate = [&](float px, float py, float pz) { cell_of(px, py, pz, I, J, K); };
    auto load_box = [&]() {
        const int q = (int)checked_index((K * RT_SC(NY) + J) * RT_SC(NX) + I,
                                         (long long)RT_SC(NX) * RT_SC(NY) * RT_SC(NZ), &RT_SC(scr)->status);
        if constexpr (BATCH) set_box(__ldg(RT_SC(box2) + q));
        else set_box(__ldg(RT_SC(box) + q));
    };
    auto set_recip = [&]() {
        ivx = __fdividef(1.0f, ux);
        ivy = __fdividef(1.0f, uy);
        ivz = __fdividef(1.0f, uz);
    };
    auto flush = [&](bool fl, int cell, bool dir, float acc) {
        flush_partials<T, AGG>(fl, RT_SC(tal.abs_dir), RT_SC(tal.abs_dif), cell, dir, acc, RT_JB(scale3));
    };
    auto end_photon = [&]() {
        // the lane flushes the photon's absorption partial at the end of the pass
        alive = false;
        atomicAdd(&s_cnt[sid][kCntPhotons], 1ull);
        atomicAdd(&s_cnt[sid][kCntEvents], (unsigned long long)nev);
        atomicAdd(&s_cnt[sid][kCntScatters], (unsigned long long)nsc);
        atomicAdd(&s_cnt[sid][kCntSteps], (unsigned long long)ncr);
        atomicMax(&s_cnt[sid][kCntMax], (unsigned long long)nev);
    };
    auto roulette = [&](float xi) -> bool {   // true: the photon dies
        if (xi > w) {
            atomicAdd(&s_led[sid][1], (double)w * RT_JB(energy));
            atomicAdd(&s_cnt[sid][kCntKills], 1ull);
            return true;
        }
        atomicAdd(&s_led[sid][0], (1.0 - (double)w) * RT_JB(energy));
        w = 1.f;
        return false;
    };

    for (;;) {
        // ---------------- 1. refill (a3, a11) ----------------
        // Births run with only the empty lanes active, so they wait until at
        // least refill_min lanes are empty (or all are, or the queue is empty).
        const unsigned dead = __ballot_sync(kFull, !alive);
        if (dead && (dead == kFull ||
                     ((!s_exh[wid] || s_q[wid][0] < s_q[wid][1]) && __popc(dead) >= A.refill_min))) {
            unsigned long long pool_next = s_q[wid][0], pool_end = s_q[wid][1];
            bool exhausted = s_exh[wid] != 0;
            const unsigned ndead = __popc(dead);
            const unsigned rank = __popc(dead & below);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long mine = ~0ull;
            if (!alive && rank < avail) mine = pool_next + rank;
            if (ndead <= avail) {
                pool_next += ndead;
            } else {
                const unsigned long long need = ndead - avail;
                pool_next = pool_end;
                if (!exhausted) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(&A.scr->queue_head, (unsigned long long)A.chunk);
                    base = __shfl_sync(kFull, base, 0);
                    if (base >= A.count) {
                        exhausted = true;
                    } else {
                        const unsigned long long end = min(base + A.chunk, A.count);
                        if (!alive && rank >= avail && base + (rank - avail) < end)
                            mine = base + (rank - avail);
                        pool_next = min(base + need, end);
                        pool_end = end;
                        if (end >= A.count) exhausted = true;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                s_q[wid][0] = pool_next;
                s_q[wid][1] = pool_end;
                s_exh[wid] = exhausted;
            }
            __syncwarp();
            if (mine != ~0ull) {
                // ---- a11: which job (batched launches: binary search of job starts) ----
                if constexpr (BATCH) {
                    int lo = 0, hi = A.njobs - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_jobs[mid].start <= mine) lo = mid; else hi = mid - 1;
                    }
                    jid = (int)checked_index(lo, A.njobs, &A.scr->status);
                    sid = (int)checked_index(s_jobs[jid].scene, A.nscenes, &A.scr->status);
                }
                // ---- a3: birth at the domain top, along the sun beam ----
                if (!BATCH && A.order) {
                    const unsigned long long cr =
                        (mine >> 32) ? mine / A.order_ppc : (unsigned long long)((uint32_t)mine / A.order_ppc);
                    gid = (A.order_k0 + (mine - cr * A.order_ppc)) * RT_JB(ncol) +
                          __ldg(A.order + checked_index((long long)cr, (long long)RT_JB(ncol), &A.scr->status));
                } else {
                    gid = RT_JB(id_begin) + (mine - RT_JB(start));
                }
                const unsigned long long ncol = RT_JB(ncol);
                const unsigned col = (gid >> 32) ? (unsigned)(gid % ncol) : (uint32_t)gid % (uint32_t)ncol;
                const int ci = (int)(col % (unsigned)RT_SC(nx)), cj = (int)(col / (unsigned)RT_SC(nx));
                const uint4 rb = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 0u),
                                               RT_JB(key0), RT_JB(key1));
                uint32_t bx = rb.x, by = rb.y;
                if (RT_SC(birth)) {
                    // photon k = gid / ncol of its column takes the column's k-th
                    // Sobol point, shifted by that column's scramble words
                    const uint32_t k = (gid >> 32) ? (uint32_t)(gid / ncol) : (uint32_t)gid / (uint32_t)ncol;
                    const uint2 p = sobol_start(k, col, RT_JB(key0), RT_JB(key1));
                    bx = p.x;
                    by = p.y;
                }
                // position inside the column (the product can round up to the
                // column's far edge; the cell index comes from the column)
                ox = ((float)ci + u01(bx)) * RT_SC(dx);
                oy = ((float)cj + u01(by)) * RT_SC(dy);
                oz = RT_SC(H);
                ux = RT_JB(sx); uy = RT_JB(sy); uz = RT_JB(sz);
                direct = true;
                if (RT_JB(diffuse) > 0.f && u01(rb.w) < RT_JB(diffuse)) {
                    // diffuse share of the top boundary: isotropic downwelling
                    // radiance, i.e. cosine-weighted downward directions (Sec. 2.3)
                    const uint4 d = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 1u),
                                                  RT_JB(key0), RT_JB(key1));
                    lambert_up(ux, uy, uz, u01(d.x), u01(d.y));
                    uz = -uz;
                    direct = false;
                }
                set_recip();
                tau = -__logf(u01(rb.z));
                w = 1.f;
                alive = true;
                ready = kNone;
                I = min(ci / RT_SC(cx), RT_SC(NX) - 1);
                J = min(cj / RT_SC(cy), RT_SC(NY) - 1);
                K = RT_SC(NZ) - 1;
                load_box();
                blk = 1; nev = 0; ncr = 0; nsc = 0;
            }
            if (!__any_sync(kFull, alive)) break;
        }

        // ---------------- 2. walk (a4) ----------------
        for (int it = 0; it < A.max_inner; ++it) {
            const bool pend = alive && ready == kNone;
            const unsigned pm = __ballot_sync(kFull, pend);
            if (!pm) break;
            if (it > 0 && __popc(__ballot_sync(kFull, ready != kNone)) >= A.ready_threshold) break;
            if (!pend) continue;
            if (ncr + nev >= A.max_steps) { ready = kCap; continue; }
            const int NX = RT_SC(NX), NY = RT_SC(NY), NZ = RT_SC(NZ);
            const int ex = ux > 0.f ? I + r + 1 : I - r;
            const int ey = uy > 0.f ? J + r + 1 : J - r;
            const int ez = uz > 0.f ? min(K + r + 1, NZ) : max(K - r, 0);
            const float fx = fminf(small_int_to_float(ex) * RT_SC(cdx), RT_SC(xcap));
            const float fy = fminf(small_int_to_float(ey) * RT_SC(cdy), RT_SC(ycap));
            const float fz = fminf(small_int_to_float(ez) * RT_SC(cdz), RT_SC(H));
            const float tx = ux != 0.f ? (fx - ox) * ivx : INFINITY;
            const float ty = uy != 0.f ? (fy - oy) * ivy : INFINITY;
            const float tz = uz != 0.f ? (fz - oz) * ivz : INFINITY;
            const bool cz_ = tz <= tx && tz <= ty, cx_ = !cz_ && tx <= ty, cy_ = !cz_ && !cx_;
            const float tm = fmaxf(cz_ ? tz : (cx_ ? tx : ty), 0.f);
            if (kmaj * tm > tau) {
                tau = __fdividef(tau, kmaj);      // the free path ends inside this box, tau from o
                ready = kEvent;
                continue;
            }
            tau = fmaf(-kmaj, tm, tau);
            ++ncr;
            // Written without branches (selects only), so lanes that cross
            // different faces do not diverge. On the crossed axis the position
            // is the face and the cell the one beyond it; on the others the
            // cell of the position, moved only forward and within the box (with
            // r = 0 that is the current cell).
            float px = cx_ ? fx : fmaf(ux, tm, ox);
            float py = cy_ ? fy : fmaf(uy, tm, oy);
            const float pz = cz_ ? fz : fmaf(uz, tm, oz);
            int ci = (int)floorf(px * RT_SC(inv_cdx));
            ci = cx_ ? (ux > 0.f ? ex : ex - 1)
                     : (ux > 0.f ? min(max(ci, I), I + r) : (ux < 0.f ? min(max(ci, I - r), I) : I));
            int cj = (int)floorf(py * RT_SC(inv_cdy));
            cj = cy_ ? (uy > 0.f ? ey : ey - 1)
                     : (uy > 0.f ? min(max(cj, J), J + r) : (uy < 0.f ? min(max(cj, J - r), J) : J));
            int ck = (int)floorf(pz * RT_SC(inv_cdz));
            ck = cz_ ? (uz > 0.f ? ez : ez - 1)
                     : (uz > 0.f ? min(max(ck, K), min(K + r, NZ - 1))
                                 : (uz < 0.f ? min(max(ck, max(K - r, 0)), K) : K));
            // periodic x and y: the cell index and the position shift together
            px += ci < 0 ? RT_SC(Lx) : (ci >= NX ? -RT_SC(Lx) : 0.f);
            ci += ci < 0 ? NX : (ci >= NX ? -NX : 0);
            py += cj < 0 ? RT_SC(Ly) : (cj >= NY ? -RT_SC(Ly) : 0.f);
            cj += cj < 0 ? NY : (cj >= NY ? -NY : 0);
            ox = px; oy = py; oz = pz;
            I = ci; J = cj;
            K = min(max(ck, 0), NZ - 1);
            // below the surface or above the top: that boundary's interaction;
            // the box then loaded is not used
            ready = ck < 0 ? kSurface : (ck >= NZ ? kTop : kNone);
            load_box();
        }

        // ---------------- 3. interact ----------------
        bool fl = false;                     // a partial to flush: the photon left its cell
        bool ended = false;                  // the photon ended in this pass
        int fcell = 0;
        bool fdir = false;
        float facc = 0.f;
        if (ready == kEvent || ready == kSurface) {
            // Events (a5-a8) and surface hits (a9) share one path: a position, a
            // Philox block, possibly a new direction, the next free path, a new
            // walk origin and roulette.
            const bool sfc = ready == kSurface;
            const int nx = RT_SC(nx), ny = RT_SC(ny);
            float px, py, pz;
            if (sfc) {
                px = wrap_coord(ox, RT_SC(Lx)); py = wrap_coord(oy, RT_SC(Ly)); pz = 0.f;
            } else {
                px = wrap_coord(fmaf(ux, tau, ox), RT_SC(Lx));
                py = wrap_coord(fmaf(uy, tau, oy), RT_SC(Ly));
                pz = fmaf(uz, tau, oz);
            }
            const int fi = min(max((int)(px * RT_SC(inv_dx)), 0), nx - 1);
            const int fj = min(max((int)(py * RT_SC(inv_dy)), 0), ny - 1);
            const long long ncell = (long long)nx * ny * RT_SC(nz);
            int cell = (int)checked_index((min(max((int)(pz * RT_SC(inv_dz)), 0), RT_SC(nz) - 1) * ny + fj) * nx + fi,
                                          ncell, &RT_SC(scr)->status);
            // Both gathers of this pass are issued before the Philox block so
            // that their latencies overlap it and each other: the optics of the
            // event cell (record mode; a surface hit loads layer 0 and ignores
            // it) and the box word of the coarse cell the next walk starts in,
            // decoded after the event, whose acceptance uses the current box.
            float4 orec;
            if constexpr (MODE == kOpticsRecord) orec = __ldg(RT_SC(rec) + cell);
            BoxWord bnext;
            {
                int i, j, k;
                const int q = cell_of(px, py, pz, i, j, k);
                if constexpr (BATCH) bnext = __ldg(RT_SC(box2) + q);
                else bnext = __ldg(RT_SC(box) + q);
            }
            const uint4 rn = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u),
                                           RT_JB(key0), RT_JB(key1));
            ++blk;
            bool turned = sfc;
            float mu = 0.f;
            if (!sfc) {
                // ---- a5: majorant event at distance tau, inside the box ----
                float kabs, ksca, kscl;   // absorption, scattering, scattering by cloud
                auto optics = [&]() {
                    if constexpr (MODE == kOpticsRecord) {
                        kabs = orec.x; ksca = orec.y; kscl = orec.z;
                    } else if constexpr (MODE == kOpticsSplit) {
                        const float4 o = __ldg(RT_SC(rec) + cell);
                        const float s = RT_JB(gas_scale);
                        kabs = fmaf(s, o.x, o.z);
                        ksca = fmaf(s, o.y, o.w);
                        if (RT_SC(pcld_mode) == 1) {
                            const float kc = o.z + o.w, kext = fmaf(s, o.x + o.y, kc);
                            kscl = kext > 0.f ? ksca * (kc / kext) : 0.f;
                        } else {
                            kscl = o.w;
                        }
                    } else {
                        const CellOptics c = cell_optics(__ldg(RT_SC(f_kg) + cell), __ldg(RT_SC(f_wg) + cell),
                                                         __ldg(RT_SC(f_kc) + cell), __ldg(RT_SC(f_wc) + cell), 0);
                        kabs = c.kabs; ksca = c.ksca; kscl = c.kscl;
                    }
                };
                optics();
                if (kabs + ksca > kmaj) {
                    // The event point lies in the box up to rounding; when rounding
                    // put it in a neighbouring cell whose extinction the box
                    // majorant does not bound, take the nearest cell of the box.
                    const int cx = RT_SC(cx), cy = RT_SC(cy), cz = RT_SC(cz);
                    int gi = (int)floorf(fmaf(ux, tau, ox) * RT_SC(inv_dx));
                    gi = min(max(gi, (I - r) * cx), min((I + r + 1) * cx, RT_SC(fxcap)) - 1);
                    gi += gi < 0 ? nx : (gi >= nx ? -nx : 0);
                    int gj = (int)floorf(fmaf(uy, tau, oy) * RT_SC(inv_dy));
                    gj = min(max(gj, (J - r) * cy), min((J + r + 1) * cy, RT_SC(fycap)) - 1);
                    gj += gj < 0 ? ny : (gj >= ny ? -ny : 0);
                    const int gk = min(max((int)(pz * RT_SC(inv_dz)), max(K - r, 0) * cz),
                                       min((K + r + 1) * cz, RT_SC(nz)) - 1);
                    cell = (int)checked_index((gk * ny + gj) * nx + gi, ncell, &RT_SC(scr)->status);
                    if constexpr (MODE == kOpticsRecord) orec = __ldg(RT_SC(rec) + cell);
                    optics();
                }
                // the weight splits exactly into the deposit and what goes on
                // (w = dep + wn in FP32): the smaller share is rounded, the
                // larger is the exact difference (Sterbenz)
                const float pabs = fminf(__fdividef(kabs, kmaj), 1.0f);
                const float wa = w * (1.0f - pabs), wb = w * pabs;
                const bool keep = pabs <= 0.5f;
                const float wn = keep ? wa : w - wb;
                const float dep = keep ? w - wa : wb;
                if (cell != pcell || direct != pdir) {
                    fl = pcell >= 0;
                    fcell = pcell; fdir = pdir; facc = pacc;
                    pcell = cell; pdir = direct; pacc = 0.f;
                }
                pacc += dep;
                w = wn;
                ++nev;
                // ---- a6/a7: real scattering or null collision ----
                // scatter if xi < k_sca/(k_max - k_abs), by cloud if xi < k_sca,cloud/(k_max - k_abs)
                const float den = kmaj - kabs;
                const float xd = u01(rn.x) * den;
                if (den > 0.f && xd < ksca) {
                    const bool cloud = xd < kscl;
                    float g = 0.f;
                    if (cloud) {
                        if constexpr (MODE == kOpticsRecord) g = orec.w;
                        else g = __ldg(RT_SC(gcl) + cell);
                    }
                    const float xi = u01(rn.y);
                    // the scattering lanes of this pass agree on the scatterer more often
                    // than not (a warp's lanes share a column): then only one sampler runs
                    const unsigned am = __activemask();
                    const unsigned cm = __ballot_sync(am, cloud);
                    if (cm == am) {
                        mu = hg_mu(g, xi);
                    } else if (cm == 0u) {
                        mu = rayleigh_mu(xi);
                    } else {
                        const float mh = hg_mu(g, xi), mr = rayleigh_mu(xi);
                        mu = cloud ? mh : mr;
                    }
                    turned = true;
                    direct = false;
                    ++nsc;
                }
            } else {
                // ---- a9: Lambertian surface ----
                const int col = (int)checked_index(fj * nx + fi, (long long)nx * ny, &RT_SC(scr)->status);
                tally_add((direct ? RT_SC(tal.sfc_dir) : RT_SC(tal.sfc_dif)) + col, w, RT_JB(scale2));
                atomicAdd(&s_cnt[sid][kCntSurface], 1ull);
                w *= __ldg(RT_SC(alb) + col);
                direct = false;
            }
            if (turned) {
                // new direction: polar cosine mu about the old direction (a7), or
                // cosine-law about the surface normal, mu = sqrt(xi) (a9)
                float sp, cp;
                azimuth(u01(rn.z), sp, cp);
                if (sfc) {
                    const float xi = u01(rn.y), st = sqrt_fast(1.0f - xi);
                    ux = st * cp; uy = st * sp; uz = sqrt_fast(xi);
                } else {
                    turn(ux, uy, uz, mu, sp, cp);
                }
                set_recip();
            }
            tau = -__logf(u01(rn.w));
            ox = px; oy = py; oz = pz;
            locate(px, py, pz);       // the cell of that box word, recomputed
            set_box(bnext);
            // ---- a8: roulette, with the fifth uniform of the block ----
            if (w < 0.5f && roulette(u01_low(rn))) {
                end_photon();
                ended = true;
            }
        } else if (ready == kTop) {
            // ---- a10: leaves through the domain top ----
            const int nx = RT_SC(nx), ny = RT_SC(ny);
            const float px = wrap_coord(ox, RT_SC(Lx)), py = wrap_coord(oy, RT_SC(Ly));
            const int fi = min(max((int)(px * RT_SC(inv_dx)), 0), nx - 1);
            const int fj = min(max((int)(py * RT_SC(inv_dy)), 0), ny - 1);
            tally_add(RT_SC(tal.toa) + checked_index(fj * nx + fi, (long long)nx * ny, &RT_SC(scr)->status), w,
                      RT_JB(scale2));
            end_photon();
            ended = true;
        } else if (ready == kCap) {
            // step cap: record, stop the photon, never spin
            atomicAdd(&s_cnt[sid][kCntCapped], 1ull);
            atomicAdd(&s_led[sid][2], (double)w * RT_JB(energy));
            atomicOr(&RT_SC(scr)->status, kStatusBudget);
            end_photon();
            ended = true;
        }
        ready = kNone;
        flush(fl, fcell, fdir, facc);
        // an ended photon's partial (a lane may flush two in one pass)
        flush(ended && pcell >= 0, pcell, pdir, pacc);
        if (ended) pcell = -1;
    }
    // the last photons' absorption partials
    flush(pcell >= 0, pcell, pdir, pacc);

    // ---- block totals into the launch scratch, once per block and scene ----
    __syncthreads();
    const int nsc_blk = BATCH ? A.nscenes : 1;
    for (int q = threadIdx.x; q < nsc_blk; q += blockDim.x) {
        Scratch *S = BATCH ? s_scenes[q].scr : A.scene.scr;
        const unsigned long long *c = s_cnt[q];
        if (c[kCntSurface]) atomicAdd(&S->surface_hits, c[kCntSurface]);
        if (c[kCntKills]) atomicAdd(&S->roulette_kills, c[kCntKills]);
        if (c[kCntCapped]) atomicAdd(&S->capped, c[kCntCapped]);
        if (c[kCntPhotons]) atomicAdd(&S->photons, c[kCntPhotons]);
        if (c[kCntEvents]) atomicAdd(&S->events, c[kCntEvents]);
        if (c[kCntScatters]) atomicAdd(&S->scatters, c[kCntScatters]);
        if (c[kCntSteps]) atomicAdd(&S->crossings, c[kCntSteps]);
        if (c[kCntMax]) atomicMax(&S->max_events, c[kCntMax]);
        if (s_led[q][0] != 0.0) atomicAdd(&S->created, s_led[q][0]);
        if (s_led[q][1] != 0.0) atomicAdd(&S->destroyed, s_led[q][1]);
        if (s_led[q][2] != 0.0) atomicAdd(&S->capped_energy, s_led[q][2]);
    }
}

#undef RT_SC
#undef RT_JB

// One device word into mapped pinned host memory (status reads that must not
// wait behind copies on the copy engines).
__global__ void store_flag(const int *__restrict__ src, int *dst)
{
    *reinterpret_cast<volatile int *>(dst) = *src;
}

// ---------------------------------------------------------------------------
// a12: FP64 normalisation and output fields. Tallies already hold W m^-3 and
// W m^-2 (the per-call photon energy is applied when they are accumulated).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void sum_fields(const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)a[i] + (b ? (double)b[i] : 0.0);
}

template <typename T>
__global__ void surface_absorption(const T *__restrict__ dir, const T *__restrict__ dif,
                                   const float *__restrict__ alb, double *__restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (1.0 - (double)alb[i]) * ((double)dir[i] + (double)dif[i]);
}

// HR = A * f(k), f(k) = 86400 / (rho(z_k) c_p) precomputed per layer.
template <typename T>
__global__ void heating_rate(const T *__restrict__ a, const T *__restrict__ b,
                             const double *__restrict__ layer_factor, double *__restrict__ out,
                             size_t ncol, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = (a ? (double)a[i] : 0.0) + (b ? (double)b[i] : 0.0);
        out[i] = v * layer_factor[i / ncol];
    }
}

// Energy ledger from the tallies: W absorbed in the atmosphere, leaving the top,
// absorbed by the surface.
template <typename T>
__global__ void ledger_reduce(Tallies<T> t, const float *__restrict__ alb, size_t ncell, size_t ncol,
                              double vol, double area, Scratch *S)
{
    double atm = 0.0, toa = 0.0, sfc = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ncell; i += stride)
        atm += (double)t.abs_dir[i] + (double)t.abs_dif[i];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ncol; i += stride) {
        toa += (double)t.toa[i];
        sfc += (1.0 - (double)alb[i]) * ((double)t.sfc_dir[i] + (double)t.sfc_dif[i]);
    }
    atm = warp_sum_f64(atm); toa = warp_sum_f64(toa); sfc = warp_sum_f64(sfc);
    if ((threadIdx.x & 31u) == 0) {
        atomicAdd(&S->e_atm, atm * vol);
        atomicAdd(&S->e_toa, toa * area);
        atomicAdd(&S->e_sfc, sfc * area);
    }
}

// ---------------------------------------------------------------------------
// Coupled-model step (Sec. 2.2: one radiation call per model step).
// ---------------------------------------------------------------------------

// Runs after the step's inputs were validated into *bad: on invalid input the
// photon queue is closed, so the transport launch that follows takes no photon,
// and the status records why.
__global__ void step_gate(const int *__restrict__ bad, Scratch *scr)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && *bad) {
        scr->queue_head = kQueueClosed;
        scr->status |= kStatusInput;
    }
}

// Horizontal homogenisation of the "-hom" experiments (Sec. 2.4): every value
// of a layer of n_layer values becomes the layer's mean. One block per layer;
// each thread sums a fixed strided subset, then a fixed shuffle tree, so the
// result does not depend on scheduling.
__global__ void homogenize_layers(double *__restrict__ f, size_t n_layer)
{
    __shared__ double part[32];
    double *row = f + (size_t)blockIdx.x * n_layer;
    double s = 0.0;
    for (size_t i = threadIdx.x; i < n_layer; i += blockDim.x) s += row[i];
    s = warp_sum_f64(s);
    if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        v = warp_sum_f64(v);
        if (threadIdx.x == 0) part[0] = v / (double)n_layer;
    }
    __syncthreads();
    const double m = part[0];
    for (size_t i = threadIdx.x; i < n_layer; i += blockDim.x) row[i] = m;
}

// ---------------------------------------------------------------------------
// Test kernels: the device RNG, samplers and rotation on small arrays.
// ---------------------------------------------------------------------------
__global__ void debug_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key[i].x, key[i].y);
}

__global__ void debug_sample(int kind, float g, unsigned long long n, uint32_t k0, uint32_t k1, float *out)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 2u), k0, k1);
    float mu;
    if (kind == 0) mu = rayleigh_mu(u01(r.x));
    else if (kind == 1) mu = hg_mu(g, u01(r.x));
    else { float x, y, z; lambert_up(x, y, z, u01(r.x), u01(r.y)); mu = z; }
    out[i] = mu;
}

__global__ void debug_sobol(unsigned long long k0, int n, uint32_t sx, uint32_t sy, uint32_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = (uint32_t)(k0 + i);
    out[2 * i] = sobol_dim1(k) ^ sx;
    out[2 * i + 1] = sobol_dim2(k) ^ sy;
}

__global__ void debug_turn(float dx, float dy, float dz, const float *mu, const float *phi, float *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = dx, y = dy, z = dz, sp, cp;
    sincosf(phi[i], &sp, &cp);
    turn(x, y, z, mu[i], sp, cp);
    out[3 * i] = x; out[3 * i + 1] = y; out[3 * i + 2] = z;
}


// ---------------------------------------------------------------------------
// Majorant grid straight from the five input fields, for launches that keep no
// derived record: the per-cell values are formed by cell_optics as
// derive_optics forms them, so the maxima equal build_majorant's. Invalid
// optics or albedo (as derive_optics and check_albedo judge them) set *bad.
// ---------------------------------------------------------------------------
__global__ void majorant_from_fields(const float *__restrict__ kg, const float *__restrict__ wg,
                                     const float *__restrict__ kc, const float *__restrict__ wc,
                                     const float *__restrict__ gc, const float *__restrict__ alb,
                                     float *__restrict__ kmax, int *bad, int nx, int ny, int nz, int cx, int cy,
                                     int cz, int NX, int NY, int NZ)
{
    const int n = NX * NY * NZ;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)n; q += gridDim.x * blockDim.x) {
        const int I = q % NX, J = (q / NX) % NY, K = q / (NX * NY);
        const int i1 = min(I * cx + cx, nx), j1 = min(J * cy + cy, ny), k1 = min(K * cz + cz, nz);
        float m = 0.0f;
        bool ok = true;
        for (int k = K * cz; k < k1; ++k)
            for (int j = J * cy; j < j1; ++j)
                for (int i = I * cx; i < i1; ++i) {
                    const size_t c = ((size_t)k * ny + j) * nx + i;
                    const float a = kg[c], b = wg[c], cc = kc[c], d = wc[c], g = gc[c];
                    ok = ok && (a >= 0.0f) && (a <= 3.0e38f) && (cc >= 0.0f) && (cc <= 3.0e38f) &&
                         (b >= 0.0f) && (b <= 1.0f) && (d >= 0.0f) && (d <= 1.0f) && (fabsf(g) < 1.0f);
                    const CellOptics o = cell_optics(a, b, cc, d, 0);
                    m = fmaxf(m, o.kabs + o.ksca);
                }
        if (K == 0)
            for (int j = J * cy; j < j1; ++j)
                for (int i = I * cx; i < i1; ++i) {
                    const float al = alb[(size_t)j * nx + i];
                    ok = ok && (al >= 0.0f) && (al <= 1.0f);
                }
        if (!ok) atomicOr(bad, 1);
        kmax[q] = m;
    }
}

// ---------------------------------------------------------------------------
// Host side of the majorant-box build: kmax -> box words, `levels` dilation
// levels (radii 1, 3, 7, 15; a level is skipped once 2r + 1 exceeds the
// smaller horizontal coarse count, so a box never wraps onto itself). Boxes
// need coarse cells of one size along x and y (uniform_xy: the coarsening
// factors divide nx and ny); otherwise every radius stays 0. w0 and w1 are
// scratch arrays of NX*NY*NZ floats.
// ---------------------------------------------------------------------------
inline int box_grid(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 32)); }

inline cudaError_t build_boxes(const float *kmax, uint32_t *box, float *w0, float *w1, int NX, int NY, int NZ,
                               double cdx, double cdy, double cdz, int levels, double box_tau, bool uniform_xy,
                               cudaStream_t st)
{
    const int n = NX * NY * NZ, g = box_grid((size_t)n);
    if (!uniform_xy) levels = 0;
    box_init<<<g, 256, 0, st>>>(kmax, w0, box, n);
    const double diag = std::sqrt(cdx * cdx + cdy * cdy + cdz * cdz);
    float *cur = w0, *tmp = w1;
    int r_prev = 0;
    for (int L = 0; L < std::min(levels, kBoxLevels); ++L) {
        const int rho = 1 << L, r_new = r_prev + rho;
        if (2 * r_new + 1 > std::min(NX, NY)) break;
        box_dilate<<<g, 256, 0, st>>>(cur, tmp, NX, NY, NZ, 0, rho);
        box_dilate<<<g, 256, 0, st>>>(tmp, cur, NX, NY, NZ, 1, rho);
        box_dilate<<<g, 256, 0, st>>>(cur, tmp, NX, NY, NZ, 2, rho);
        std::swap(cur, tmp);
        box_select<<<g, 256, 0, st>>>(cur, box, n, r_prev, r_new, (float)(box_tau / ((2 * r_new + 1) * diag)));
        r_prev = r_new;
    }
    return cudaGetLastError();
}

// Batched launches: gas and cloud channels dilated apart (w0..w3 scratch).
inline cudaError_t build_boxes2(const float2 *kmax2, uint2 *box2, float *w0, float *w1, float *w2, float *w3, int NX,
                                int NY, int NZ, double cdx, double cdy, double cdz, int levels, double box_tau,
                                bool uniform_xy, cudaStream_t st)
{
    const int n = NX * NY * NZ, g = box_grid((size_t)n);
    if (!uniform_xy) levels = 0;
    box_init2<<<g, 256, 0, st>>>(kmax2, w0, w2, box2, n);
    const double diag = std::sqrt(cdx * cdx + cdy * cdy + cdz * cdz);
    float *cg = w0, *tg = w1, *cc = w2, *tc = w3;
    int r_prev = 0;
    for (int L = 0; L < std::min(levels, kBoxLevels); ++L) {
        const int rho = 1 << L, r_new = r_prev + rho;
        if (2 * r_new + 1 > std::min(NX, NY)) break;
        for (int ch = 0; ch < 2; ++ch) {
            float *&c = ch ? cc : cg, *&t = ch ? tc : tg;
            box_dilate<<<g, 256, 0, st>>>(c, t, NX, NY, NZ, 0, rho);
            box_dilate<<<g, 256, 0, st>>>(t, c, NX, NY, NZ, 1, rho);
            box_dilate<<<g, 256, 0, st>>>(c, t, NX, NY, NZ, 2, rho);
            std::swap(c, t);
        }
        box_select2<<<g, 256, 0, st>>>(cg, cc, box2, n, r_prev, r_new, (float)(box_tau / ((2 * r_new + 1) * diag)));
        r_prev = r_new;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace rt
