// rt_kernels.cuh -- kernels of the shortwave Monte Carlo tracer
// (Veerman et al. 2022, Sec. 2.3).
//
//   derive_optics   per-cell record {k_abs, k_sca, k_sca*P(cloud|scatter), g}
//                   from the five gas/cloud fields, with validation
//   build_majorant  coarse-grid maximum of k_ext (the null-collision coefficient)
//   trace_kernel    persistent photon transport with warp-level refill:
//                   null-collision tracking over the coarse grid, weights,
//                   roulette, Lambertian surface, FP32 partial -> FP64 tallies
//   fields kernels  FP64 normalisation of the tallies into output fields
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rt_device.cuh"

namespace rt {

constexpr int kStatusBudget = 1;
constexpr int kStatusInput = 2;                        // an rt_step launch found invalid inputs
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

// One scene as the transport kernel sees it.
template <typename T>
struct SceneDev {
    const float4 *rec;     // single-scene launches: {k_abs, k_sca, k_sca*P(cloud), g} per cell;
                           // batched launches: {k_abs,gas, k_sca,gas, k_abs,cloud, k_sca,cloud}
    const float *gcl;      // batched launches: cloud asymmetry per cell
    const float *kmax;     // single-scene: max k_ext per coarse cell
    const float2 *kmax2;   // batched: {max gas k_ext, max cloud k_ext} per coarse cell
    const float *alb;      // [ny][nx]
    Tallies<T> tal;
    Scratch *scr;
    int nx, ny, nz, NX, NY, NZ, cx, cy, cz, pcld_mode;
    float dx, dy, dz, inv_dx, inv_dy, inv_dz, Lx, Ly, H;
    float cdx, cdy, cdz;   // coarse cell size [m] (the last cell may be smaller)
    int birth;             // start positions: 0 Philox uniforms, 1 scrambled Sobol
    int pad_[3];
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
    int max_inner;                 // bound on face-crossing sweeps per interaction sweep
    // single-scene launches of whole photon rounds: queue index q takes photon
    // (order_k0 + q mod order_ppc) * ncol + order[q div order_ppc], i.e. all
    // photons of one column in turn, columns in the order of `order`
    const uint32_t *order;
    uint32_t order_ppc;
    unsigned long long order_k0;
};

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
        const float ksg = a * b, ksc = c * d;
        const float ksca = ksg + ksc;
        const float kabs = fmaf(a, 1.0f - b, c * (1.0f - d));
        float zc = ksc;
        if (pcld_mode == 1) zc = (a + c > 0.0f) ? ksca * (c / (a + c)) : 0.0f;
        rec[i] = make_float4(kabs, ksca, zc, g);
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
__global__ void build_majorant(const float4 *__restrict__ rec, float *__restrict__ kmax, int nx,
                               int ny, int nz, int cx, int cy, int cz, int NX, int NY, int NZ)
{
    const int n = NX * NY * NZ;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
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
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
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
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
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
// Tally accumulation: FP32 partial times the per-call energy, added into the
// FP64 (or, for the precision study, FP32) global accumulator.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tally_add(double *p, float v, double scale)
{
    // the partial is FP32 already; scaling it in FP32 keeps the thin FP64 pipe
    // to the one conversion the FP64 accumulator needs
    atomicAdd(p, (double)(v * (float)scale));
}
__device__ __forceinline__ void tally_add(float *p, float v, double scale)
{
    atomicAdd(p, v * (float)scale);
}

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

// ---------------------------------------------------------------------------
// a3-a11: persistent transport kernel.
//
// Every warp loops until the photon queue is empty. One iteration has three
// phases, each warp-synchronous:
//
//  1. refill: lanes whose photon ended take new photon ids (one atomicAdd per
//     warp for a chunk of ids, handed out by ballot rank) and are born at the
//     domain top along the sun beam;
//  2. advance: lanes without a pending interaction cross faces of their coarse
//     cell (subtracting k_max * l from the remaining optical depth) until the
//     free path ends inside a cell (an event), the photon reaches the surface
//     or leaves the top. The sweep repeats until `ready_threshold` lanes are
//     ready (or none is left to advance, or `max_inner` sweeps), so the costly
//     interaction code below runs with most lanes active;
//  3. interact: ready lanes handle their event, surface hit or exit.
//
// The walk over the coarse grid is parametric: along a straight segment from
// origin o with direction u, tn[a] is the distance to the next face on axis a;
// a crossing updates only the crossed axis. x and y wrap periodically (the
// origin shifts by the domain length).
//
// Events (Sec. 2.3, weights after Iwabuchi 2006): at every majorant event the
// cell absorbs w k_abs/k_max (heating tally) and w shrinks by the same amount;
// the photon then scatters with probability k_sca/(k_max - k_abs), by cloud
// (HG) or gas (Rayleigh), or has a null collision; below w = 0.5 roulette ends
// it with probability 1 - w or resets w = 1. The surface adds w to the direct
// or diffuse irradiance of its column, multiplies w by the albedo and reflects
// Lambertian. Leaving the top adds w to the upward flux of its column.
//
// Random numbers: block b of photon p is Philox(ctr = (p lo, p hi, b, slot)).
// Birth uses block 0 (x, y, first free path); each event or surface hit uses
// the next block (choice, mu, phi, next free path) and slot 1 of the same
// block for roulette.
// ---------------------------------------------------------------------------
enum : int { kNone = 0, kEvent = 1, kSurface = 2, kTop = 3, kCap = 4 };

// Scene and job fields of the lane's photon: kernel parameters in single-scene
// launches, shared memory in batched ones (folded at compile time).
#define RT_SC(f) (BATCH ? s_scenes[sid].f : A.scene.f)
#define RT_JB(f) (BATCH ? s_jobs[jid].f : A.job.f)

// Scrambled Sobol start point k of column col (Sec. 2.3): the column's two
// scramble words come from Philox counter (col, 0, 0, 2) under the job's key.
// Kept out of line: it runs once per photon, and inlining it into the refill
// phase made the batched kernel spill.
__device__ __noinline__ uint2 sobol_start(uint32_t k, uint32_t col, uint32_t k0, uint32_t k1)
{
    const uint4 h = philox4x32_10(make_uint4(col, 0u, 0u, 2u), k0, k1);
    return make_uint2(sobol_dim1(k) ^ h.x, sobol_dim2(k) ^ h.y);
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ TraceArgs<T> A)
{
    constexpr unsigned kFull = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;

    // batched launches: scene and job descriptors in dynamic shared memory
    extern __shared__ __align__(16) unsigned char s_dyn[];
    SceneDev<T> *s_scenes = reinterpret_cast<SceneDev<T> *>(s_dyn);
    JobDev *s_jobs = reinterpret_cast<JobDev *>(s_dyn + (BATCH ? A.nscenes : 0) * sizeof(SceneDev<T>));
    // rare counters and the energy ledger per scene: surface hits, roulette
    // kills, capped | created, destroyed, capped energy; batched launches also
    // keep photons, events, scatters and crossings per scene here
    constexpr int NS = BATCH ? kMaxBatchScenes : 1;
    __shared__ unsigned long long s_cnt[NS][7];
    __shared__ double s_led[NS][3];
    for (int q = threadIdx.x; q < NS * 7; q += blockDim.x) s_cnt[q / 7][q % 7] = 0;
    for (int q = threadIdx.x; q < NS * 3; q += blockDim.x) s_led[q / 3][q % 3] = 0.0;
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
    float ox = 0.f, oy = 0.f, oz = 0.f;       // origin of the current straight segment
    float ux = 0.f, uy = 0.f, uz = -1.f;      // direction
    float ivx = 0.f, ivy = 0.f, ivz = 0.f;    // 1/u per axis (used only on axes that move)
    float tnx = 0.f, tny = 0.f, tnz = 0.f;    // distance from o to the next face per axis
    float tcur = 0.f;                         // distance from o to the photon
    float w = 0.f, tau = 0.f, kmaj = 0.f;
    int I = 0, J = 0, K = 0;
    unsigned long long gid = 0;
    uint32_t blk = 0, steps = 0, nev = 0, nsc = 0, ncr = 0;
    bool alive = false, direct = false;
    int ready = kNone;
    int pcell = -1;
    bool pdir = false;
    float pacc = 0.f;

    uint32_t c_ph = 0, c_ev = 0, c_sc = 0, c_cr = 0, c_max = 0;

    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;

    auto load_kmaj = [&]() -> float {
        const size_t q = ((size_t)K * RT_SC(NY) + J) * RT_SC(NX) + I;
        if constexpr (BATCH) {
            const float2 m = __ldg(RT_SC(kmax2) + q);
            return fmaf(RT_JB(gas_scale), m.x, m.y);
        } else {
            return __ldg(RT_SC(kmax) + q);
        }
    };
    auto flush = [&]() {
        if (pcell >= 0)
            tally_add((pdir ? RT_SC(tal.abs_dir) : RT_SC(tal.abs_dif)) + pcell, pacc, RT_JB(scale3));
        pcell = -1;
    };

    // distances to the next coarse faces from origin o along u, for cell (I,J,K).
    // An axis along which the photon does not move gets an infinite distance and
    // is never crossed, so its reciprocal is never used.
    auto start_segment = [&]() {
        tcur = 0.f;
        ivx = __frcp_rn(ux); ivy = __frcp_rn(uy); ivz = __frcp_rn(uz);
        tnx = ux > 0.f ? (fminf((float)(I + 1) * RT_SC(cdx), RT_SC(Lx)) - ox) * ivx
            : ux < 0.f ? ((float)I * RT_SC(cdx) - ox) * ivx : INFINITY;
        tny = uy > 0.f ? (fminf((float)(J + 1) * RT_SC(cdy), RT_SC(Ly)) - oy) * ivy
            : uy < 0.f ? ((float)J * RT_SC(cdy) - oy) * ivy : INFINITY;
        tnz = uz > 0.f ? (fminf((float)(K + 1) * RT_SC(cdz), RT_SC(H)) - oz) * ivz
            : uz < 0.f ? ((float)K * RT_SC(cdz) - oz) * ivz : INFINITY;
        tnx = fmaxf(tnx, 0.f); tny = fmaxf(tny, 0.f); tnz = fmaxf(tnz, 0.f);
    };

    for (;;) {
        // ---------------- 1. refill ----------------
        const unsigned dead = __ballot_sync(kFull, !alive);
        if (dead) {
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
            if (mine != ~0ull) {
                // ---- a11: which job (batched launches: binary search of job starts) ----
                if constexpr (BATCH) {
                    int lo = 0, hi = A.njobs - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_jobs[mid].start <= mine) lo = mid; else hi = mid - 1;
                    }
                    jid = lo;
                    sid = s_jobs[jid].scene;
                }
                // ---- a3: birth at the domain top, along the sun beam ----
                if (!BATCH && A.order) {
                    const unsigned long long cr =
                        (mine >> 32) ? mine / A.order_ppc : (unsigned long long)((uint32_t)mine / A.order_ppc);
                    gid = (A.order_k0 + (mine - cr * A.order_ppc)) * RT_JB(ncol) + __ldg(A.order + cr);
                } else {
                    gid = RT_JB(id_begin) + (mine - RT_JB(start));
                }
                const unsigned long long ncol = RT_JB(ncol);
                const unsigned col = (gid >> 32) ? (unsigned)(gid % ncol) : (uint32_t)gid % (uint32_t)ncol;
                const int ci = (int)(col % (unsigned)RT_SC(nx)), cj = (int)(col / (unsigned)RT_SC(nx));
                const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 0u),
                                              RT_JB(key0), RT_JB(key1));
                uint32_t bx = r.x, by = r.y;
                if (RT_SC(birth)) {
                    // photon k = gid / ncol of its column takes the column's k-th
                    // Sobol point, shifted by that column's scramble words
                    const uint32_t k = (gid >> 32) ? (uint32_t)(gid / ncol) : (uint32_t)gid / (uint32_t)ncol;
                    const uint2 p = sobol_start(k, col, RT_JB(key0), RT_JB(key1));
                    bx = p.x;
                    by = p.y;
                }
                ox = ((float)ci + u01(bx)) * RT_SC(dx);
                oy = ((float)cj + u01(by)) * RT_SC(dy);
                oz = RT_SC(H);
                ux = RT_JB(sx); uy = RT_JB(sy); uz = RT_JB(sz);
                direct = true;
                if (RT_JB(diffuse) > 0.f && u01(r.w) < RT_JB(diffuse)) {
                    // diffuse share of the top boundary: isotropic downwelling
                    // radiance, i.e. cosine-weighted downward directions (Sec. 2.3)
                    const uint4 d = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 1u),
                                                  RT_JB(key0), RT_JB(key1));
                    lambert_up(ux, uy, uz, u01(d.x), u01(d.y));
                    uz = -uz;
                    direct = false;
                }
                tau = -__logf(u01(r.z));
                w = 1.f;
                alive = true;
                ready = kNone;
                I = ci / RT_SC(cx); J = cj / RT_SC(cy); K = RT_SC(NZ) - 1;
                kmaj = load_kmaj();
                start_segment();
                blk = 1; steps = 0; nev = 0; nsc = 0; ncr = 0;
                ++c_ph;
            }
            if (!__any_sync(kFull, alive)) break;
        }

        // ---------------- 2. advance (a4) ----------------
        for (int it = 0; it < A.max_inner; ++it) {
            const bool pend = alive && ready == kNone;
            const unsigned pm = __ballot_sync(kFull, pend);
            if (!pm) break;
            if (it > 0 && __popc(__ballot_sync(kFull, ready != kNone)) >= A.ready_threshold) break;
            if (!pend) continue;
            if (++steps > A.max_steps) { ready = kCap; continue; }
            float tm;
            int ax;
            if (tnx <= tny && tnx <= tnz) { tm = tnx; ax = 0; }
            else if (tny <= tnz) { tm = tny; ax = 1; }
            else { tm = tnz; ax = 2; }
            const float dt = fmaxf(tm - tcur, 0.f);
            if (kmaj * dt > tau) {
                tcur += __fdividef(tau, kmaj);     // the free path ends in this coarse cell
                ready = kEvent;
                continue;
            }
            tau = fmaf(-kmaj, dt, tau);
            tcur = tm;
            ++c_cr;
            if (BATCH) ++ncr;
            if (ax == 0) {
                if (ux > 0.f) {
                    if (++I == RT_SC(NX)) { I = 0; ox -= RT_SC(Lx); }
                    tnx = (fminf((float)(I + 1) * RT_SC(cdx), RT_SC(Lx)) - ox) * ivx;
                } else {
                    if (--I < 0) { I = RT_SC(NX) - 1; ox += RT_SC(Lx); }
                    tnx = ((float)I * RT_SC(cdx) - ox) * ivx;
                }
            } else if (ax == 1) {
                if (uy > 0.f) {
                    if (++J == RT_SC(NY)) { J = 0; oy -= RT_SC(Ly); }
                    tny = (fminf((float)(J + 1) * RT_SC(cdy), RT_SC(Ly)) - oy) * ivy;
                } else {
                    if (--J < 0) { J = RT_SC(NY) - 1; oy += RT_SC(Ly); }
                    tny = ((float)J * RT_SC(cdy) - oy) * ivy;
                }
            } else {
                if (uz > 0.f) {
                    if (++K == RT_SC(NZ)) { ready = kTop; continue; }
                    tnz = (fminf((float)(K + 1) * RT_SC(cdz), RT_SC(H)) - oz) * ivz;
                } else {
                    if (--K < 0) { ready = kSurface; continue; }
                    tnz = ((float)K * RT_SC(cdz) - oz) * ivz;
                }
            }
            kmaj = load_kmaj();
        }

        // ---------------- 3. interact ----------------
        if (ready == kNone) continue;
        bool end_photon = false;
        const int ilo = I * RT_SC(cx), ihi = min(ilo + RT_SC(cx), RT_SC(nx));
        const int jlo = J * RT_SC(cy), jhi = min(jlo + RT_SC(cy), RT_SC(ny));
        const float px = fmaf(ux, tcur, ox), py = fmaf(uy, tcur, oy);
        const int fi = min(max((int)(px * RT_SC(inv_dx)), ilo), ihi - 1);
        const int fj = min(max((int)(py * RT_SC(inv_dy)), jlo), jhi - 1);
        if (ready == kEvent) {
            // ---- a5: majorant event: absorb a fraction of the weight ----
            ++steps;
            const float pz = fmaf(uz, tcur, oz);
            const int klo = K * RT_SC(cz), khi = min(klo + RT_SC(cz), RT_SC(nz));
            const int fk = min(max((int)(pz * RT_SC(inv_dz)), klo), khi - 1);
            const int cell = (fk * RT_SC(ny) + fj) * RT_SC(nx) + fi;
            float kabs, ksca, kscl;   // absorption, scattering, scattering times P(cloud)
            const float4 o = __ldg(RT_SC(rec) + cell);
            if constexpr (BATCH) {
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
                kabs = o.x; ksca = o.y; kscl = o.z;
            }
            const float pabs = fminf(__fdividef(kabs, kmaj), 1.0f);
            const float wn = w * (1.0f - pabs);
            if (cell != pcell || direct != pdir) {
                flush();
                pcell = cell; pdir = direct; pacc = 0.f;
            }
            pacc += w - wn;
            w = wn;
            ++c_ev; ++nev;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u),
                                          RT_JB(key0), RT_JB(key1));
            ++blk;
            // ---- a6/a7: real scattering or null collision ----
            // scatter if xi < k_sca/(k_max - k_abs), by cloud if xi < k_sca,cloud/(k_max - k_abs)
            ox = px; oy = py; oz = pz;
            const float den = kmaj - kabs;
            bool scattered = false;
            if (den > 0.f) {
                const float xd = u01(r.x) * den;
                if (xd < ksca) {
                    float mu;
                    if (xd < kscl) {
                        float g;
                        if constexpr (BATCH) g = __ldg(RT_SC(gcl) + cell);
                        else g = o.w;
                        mu = hg_mu(g, u01(r.y));
                    } else {
                        mu = rayleigh_mu(u01(r.y));
                    }
                    float sp, cp;
                    azimuth(u01(r.z), sp, cp);
                    turn(ux, uy, uz, mu, sp, cp);
                    direct = false;
                    scattered = true;
                    ++c_sc;
                    if (BATCH) ++nsc;
                }
            }
            if (scattered) {
                start_segment();
            } else {
                tnx -= tcur; tny -= tcur; tnz -= tcur;
                tcur = 0.f;
            }
            tau = -__logf(u01(r.w));
            // ---- a8: roulette ----
            if (w < 0.5f) {
                const uint4 q = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk - 1u, 1u),
                                              RT_JB(key0), RT_JB(key1));
                if (u01(q.x) > w) {
                    atomicAdd(&s_led[sid][1], (double)w * RT_JB(energy));
                    atomicAdd(&s_cnt[sid][1], 1ull);
                    end_photon = true;
                } else {
                    atomicAdd(&s_led[sid][0], (double)(1.0f - w) * RT_JB(energy));
                    w = 1.f;
                }
            }
        } else if (ready == kSurface) {
            // ---- a9: Lambertian surface ----
            ++steps;
            const int col = fj * RT_SC(nx) + fi;
            tally_add((direct ? RT_SC(tal.sfc_dir) : RT_SC(tal.sfc_dif)) + col, w, RT_JB(scale2));
            atomicAdd(&s_cnt[sid][0], 1ull);
            w *= __ldg(RT_SC(alb) + col);
            direct = false;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u),
                                          RT_JB(key0), RT_JB(key1));
            ++blk;
            lambert_up(ux, uy, uz, u01(r.x), u01(r.y));
            tau = -__logf(u01(r.w));
            K = 0;
            ox = px; oy = py; oz = 0.f;
            start_segment();
            if (w < 0.5f) {
                if (u01(r.z) > w) {
                    atomicAdd(&s_led[sid][1], (double)w * RT_JB(energy));
                    atomicAdd(&s_cnt[sid][1], 1ull);
                    end_photon = true;
                } else {
                    atomicAdd(&s_led[sid][0], (double)(1.0f - w) * RT_JB(energy));
                    w = 1.f;
                }
            }
        } else if (ready == kTop) {
            // ---- a10: leaves through the domain top ----
            tally_add(RT_SC(tal.toa) + (fj * RT_SC(nx) + fi), w, RT_JB(scale2));
            end_photon = true;
        } else {
            // step cap: record, stop the photon, never spin
            atomicAdd(&s_cnt[sid][2], 1ull);
            atomicAdd(&s_led[sid][2], (double)w * RT_JB(energy));
            atomicOr(&RT_SC(scr)->status, kStatusBudget);
            end_photon = true;
        }
        ready = kNone;
        if (end_photon) {
            flush();
            alive = false;
            c_max = max(c_max, nev);
            if (BATCH) {
                atomicAdd(&s_cnt[sid][3], 1ull);
                atomicAdd(&s_cnt[sid][4], (unsigned long long)nev);
                atomicAdd(&s_cnt[sid][5], (unsigned long long)nsc);
                atomicAdd(&s_cnt[sid][6], (unsigned long long)ncr);
                atomicMax(&RT_SC(scr)->max_events, (unsigned long long)nev);
            }
        }
    }

    // ---- counters: warp reduction, one atomic per warp; block totals once ----
    if (!BATCH) {
        const unsigned long long s_ph = warp_sum_u32(c_ph), s_ev = warp_sum_u32(c_ev),
                                 s_sc = warp_sum_u32(c_sc), s_cr = warp_sum_u32(c_cr);
        const unsigned m_ev = __reduce_max_sync(kFull, c_max);
        Scratch *S = A.scene.scr;
        if (lane == 0) {
            if (s_ph) atomicAdd(&S->photons, s_ph);
            if (s_ev) atomicAdd(&S->events, s_ev);
            if (s_sc) atomicAdd(&S->scatters, s_sc);
            if (s_cr) atomicAdd(&S->crossings, s_cr);
            if (m_ev) atomicMax(&S->max_events, (unsigned long long)m_ev);
        }
    }
    __syncthreads();
    const int nsc_blk = BATCH ? A.nscenes : 1;
    for (int q = threadIdx.x; q < nsc_blk; q += blockDim.x) {
        Scratch *S = BATCH ? s_scenes[q].scr : A.scene.scr;
        if (s_cnt[q][0]) atomicAdd(&S->surface_hits, s_cnt[q][0]);
        if (s_cnt[q][1]) atomicAdd(&S->roulette_kills, s_cnt[q][1]);
        if (s_cnt[q][2]) atomicAdd(&S->capped, s_cnt[q][2]);
        if (BATCH) {
            if (s_cnt[q][3]) atomicAdd(&S->photons, s_cnt[q][3]);
            if (s_cnt[q][4]) atomicAdd(&S->events, s_cnt[q][4]);
            if (s_cnt[q][5]) atomicAdd(&S->scatters, s_cnt[q][5]);
            if (s_cnt[q][6]) atomicAdd(&S->crossings, s_cnt[q][6]);
        }
        if (s_led[q][0] != 0.0) atomicAdd(&S->created, s_led[q][0]);
        if (s_led[q][1] != 0.0) atomicAdd(&S->destroyed, s_led[q][1]);
        if (s_led[q][2] != 0.0) atomicAdd(&S->capped_energy, s_led[q][2]);
    }
}

#undef RT_SC
#undef RT_JB

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

}  // namespace rt
