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

template <typename T>
struct TraceArgs {
    const float4 *__restrict__ rec;   // [nz][ny][nx] {k_abs, k_sca, k_sca*P(cloud), g}
    const float *__restrict__ kmax;   // [NZ][NY][NX]
    const float *__restrict__ alb;    // [ny][nx]
    Tallies<T> tal;
    Scratch *scr;
    unsigned long long id_begin, count, ncol;
    int nx, ny, nz, NX, NY, NZ, cx, cy, cz;
    float dx, dy, dz, inv_dx, inv_dy, inv_dz, Lx, Ly, H;
    float sx, sy, sz;                 // travel direction of the direct beam
    uint32_t key0, key1;
    double energy;                    // W per unit photon weight
    double scale2, scale3;            // energy / (dx dy), energy / (dx dy dz)
    uint32_t max_steps;
    uint32_t chunk;
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
// Tally accumulation: FP32 partial times the per-call energy, added into the
// FP64 (or, for the precision study, FP32) global accumulator.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tally_add(double *p, float v, double scale)
{
    atomicAdd(p, (double)v * scale);
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
// Every warp loops until the photon queue is empty. Each iteration: lanes
// whose photon has ended take new photon ids (one atomicAdd per warp for a
// chunk of ids, handed out by ballot rank), then every live lane makes ONE
// step: either it crosses a face of its coarse cell (subtracting k_max * l from
// its remaining optical depth) or it has an event inside it. Steps are short
// and alike, so lanes stay busy even though photon lifetimes differ by orders
// of magnitude.
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
template <typename T>
__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ TraceArgs<T> A)
{
    constexpr unsigned kFull = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;

    float px = 0.f, py = 0.f, pz = 0.f, ux = 0.f, uy = 0.f, uz = -1.f;
    float w = 0.f, tau = 0.f, kmaj = 0.f;
    int I = 0, J = 0, K = 0;
    unsigned long long gid = 0;
    uint32_t blk = 0, steps = 0, nev = 0;
    bool alive = false, direct = false;
    int pcell = -1;
    bool pdir = false;
    float pacc = 0.f;

    uint32_t c_ph = 0, c_ev = 0, c_sc = 0, c_cr = 0, c_sf = 0, c_rk = 0, c_cap = 0, c_max = 0;
    double e_cr = 0.0, e_de = 0.0, e_cap = 0.0;

    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;

    const uint32_t k0 = A.key0, k1 = A.key1;

    for (;;) {
        const unsigned dead = __ballot_sync(kFull, !alive);
        if (dead) {
            // ---- warp-level refill ----
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
                // ---- a3: birth at the domain top, along the sun beam ----
                gid = A.id_begin + mine;
                const unsigned col = (unsigned)(gid % A.ncol);
                const int ci = (int)(col % (unsigned)A.nx), cj = (int)(col / (unsigned)A.nx);
                const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 0u), k0, k1);
                px = ((float)ci + u01(r.x)) * A.dx;
                py = ((float)cj + u01(r.y)) * A.dy;
                pz = A.H;
                ux = A.sx; uy = A.sy; uz = A.sz;
                tau = -__logf(u01(r.z));
                w = 1.f;
                direct = true;
                alive = true;
                I = ci / A.cx; J = cj / A.cy; K = A.NZ - 1;
                kmaj = __ldg(A.kmax + ((size_t)K * A.NY + J) * A.NX + I);
                blk = 1; steps = 0; nev = 0;
                ++c_ph;
            }
            if (!__any_sync(kFull, alive)) break;
        }
        if (!alive) continue;

        bool end_photon = false;
        if (++steps > A.max_steps) {
            // step cap: record, stop the photon, never spin
            ++c_cap;
            e_cap += (double)w * A.energy;
            atomicOr(&A.scr->status, kStatusBudget);
            end_photon = true;
        } else {
            const int ilo = I * A.cx, ihi = min(ilo + A.cx, A.nx);
            const int jlo = J * A.cy, jhi = min(jlo + A.cy, A.ny);
            const int klo = K * A.cz, khi = min(klo + A.cz, A.nz);
            const float bx = (float)(ux > 0.f ? ihi : ilo) * A.dx;
            const float by = (float)(uy > 0.f ? jhi : jlo) * A.dy;
            const float bz = (float)(uz > 0.f ? khi : klo) * A.dz;
            const float tx = ux != 0.f ? fmaxf(0.f, __fdividef(bx - px, ux)) : INFINITY;
            const float ty = uy != 0.f ? fmaxf(0.f, __fdividef(by - py, uy)) : INFINITY;
            const float tz = uz != 0.f ? fmaxf(0.f, __fdividef(bz - pz, uz)) : INFINITY;
            float smin = tx;
            int axis = 0;
            if (ty < smin) { smin = ty; axis = 1; }
            if (tz < smin) { smin = tz; axis = 2; }

            if (kmaj * smin > tau) {
                // ---- a4/a5: majorant event inside this coarse cell ----
                const float s = __fdividef(tau, kmaj);
                px = fmaf(ux, s, px); py = fmaf(uy, s, py); pz = fmaf(uz, s, pz);
                const int fi = min(max((int)(px * A.inv_dx), ilo), ihi - 1);
                const int fj = min(max((int)(py * A.inv_dy), jlo), jhi - 1);
                const int fk = min(max((int)(pz * A.inv_dz), klo), khi - 1);
                const int cell = (fk * A.ny + fj) * A.nx + fi;
                const float4 o = __ldg(A.rec + cell);
                const float wn = w * (1.0f - __fdividef(o.x, kmaj));
                const float dep = w - wn;
                if (cell != pcell || direct != pdir) {
                    if (pcell >= 0) tally_add((pdir ? A.tal.abs_dir : A.tal.abs_dif) + pcell, pacc, A.scale3);
                    pcell = cell; pdir = direct; pacc = 0.f;
                }
                pacc += dep;
                w = wn;
                ++c_ev; ++nev;
                const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u), k0, k1);
                ++blk;
                // ---- a6/a7: real scattering or null collision ----
                const float den = kmaj - o.x;
                if (den > 0.f) {
                    const float rd = 1.0f / den;
                    const float xi = u01(r.x);
                    if (xi < o.y * rd) {
                        const float mu = (xi < o.z * rd) ? hg_mu(o.w, u01(r.y)) : rayleigh_mu(u01(r.y));
                        float sp, cp;
                        azimuth(u01(r.z), sp, cp);
                        turn(ux, uy, uz, mu, sp, cp);
                        direct = false;
                        ++c_sc;
                    }
                }
                tau = -__logf(u01(r.w));
                // ---- a8: roulette ----
                if (w < 0.5f) {
                    const uint4 q = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk - 1u, 1u), k0, k1);
                    if (u01(q.x) > w) {
                        e_de += (double)w * A.energy;
                        ++c_rk;
                        end_photon = true;
                    } else {
                        e_cr += (double)(1.0f - w) * A.energy;
                        w = 1.f;
                    }
                }
            } else {
                // ---- a4: cross a face of the coarse cell ----
                tau = fmaf(-kmaj, smin, tau);
                ++c_cr;
                if (axis == 0) {
                    py = fmaf(uy, smin, py); pz = fmaf(uz, smin, pz);
                    px = bx;
                    if (ux > 0.f) { if (++I == A.NX) { I = 0; px = 0.f; } }
                    else { if (--I < 0) { I = A.NX - 1; px = A.Lx; } }
                } else if (axis == 1) {
                    px = fmaf(ux, smin, px); pz = fmaf(uz, smin, pz);
                    py = by;
                    if (uy > 0.f) { if (++J == A.NY) { J = 0; py = 0.f; } }
                    else { if (--J < 0) { J = A.NY - 1; py = A.Ly; } }
                } else {
                    px = fmaf(ux, smin, px); py = fmaf(uy, smin, py);
                    pz = bz;
                    K += (uz > 0.f) ? 1 : -1;
                }
                if (K < 0) {
                    // ---- a9: Lambertian surface ----
                    K = 0; pz = 0.f;
                    const int fi = min(max((int)(px * A.inv_dx), ilo), ihi - 1);
                    const int fj = min(max((int)(py * A.inv_dy), jlo), jhi - 1);
                    const int col = fj * A.nx + fi;
                    tally_add((direct ? A.tal.sfc_dir : A.tal.sfc_dif) + col, w, A.scale2);
                    ++c_sf;
                    w *= __ldg(A.alb + col);
                    direct = false;
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u), k0, k1);
                    ++blk;
                    lambert_up(ux, uy, uz, u01(r.x), u01(r.y));
                    tau = -__logf(u01(r.w));
                    if (w < 0.5f) {
                        if (u01(r.z) > w) {
                            e_de += (double)w * A.energy;
                            ++c_rk;
                            end_photon = true;
                        } else {
                            e_cr += (double)(1.0f - w) * A.energy;
                            w = 1.f;
                        }
                    }
                } else if (K >= A.NZ) {
                    // ---- a10: leaves through the domain top ----
                    const int fi = min(max((int)(px * A.inv_dx), ilo), ihi - 1);
                    const int fj = min(max((int)(py * A.inv_dy), jlo), jhi - 1);
                    tally_add(A.tal.toa + (fj * A.nx + fi), w, A.scale2);
                    end_photon = true;
                } else {
                    kmaj = __ldg(A.kmax + ((size_t)K * A.NY + J) * A.NX + I);
                }
            }
        }
        if (end_photon) {
            if (pcell >= 0) {
                tally_add((pdir ? A.tal.abs_dir : A.tal.abs_dif) + pcell, pacc, A.scale3);
                pcell = -1;
            }
            alive = false;
            c_max = max(c_max, nev);
        }
    }

    // ---- counters: warp reduction, one atomic per warp ----
    const unsigned long long s_ph = warp_sum_u32(c_ph), s_ev = warp_sum_u32(c_ev),
                             s_sc = warp_sum_u32(c_sc), s_cr = warp_sum_u32(c_cr),
                             s_sf = warp_sum_u32(c_sf), s_rk = warp_sum_u32(c_rk),
                             s_cap = warp_sum_u32(c_cap);
    const unsigned m_ev = __reduce_max_sync(kFull, c_max);
    const double d_cr = warp_sum_f64(e_cr), d_de = warp_sum_f64(e_de), d_cap = warp_sum_f64(e_cap);
    if (lane == 0) {
        Scratch *S = A.scr;
        if (s_ph) atomicAdd(&S->photons, s_ph);
        if (s_ev) atomicAdd(&S->events, s_ev);
        if (s_sc) atomicAdd(&S->scatters, s_sc);
        if (s_cr) atomicAdd(&S->crossings, s_cr);
        if (s_sf) atomicAdd(&S->surface_hits, s_sf);
        if (s_rk) atomicAdd(&S->roulette_kills, s_rk);
        if (s_cap) atomicAdd(&S->capped, s_cap);
        if (m_ev) atomicMax(&S->max_events, (unsigned long long)m_ev);
        if (d_cr != 0.0) atomicAdd(&S->created, d_cr);
        if (d_de != 0.0) atomicAdd(&S->destroyed, d_de);
        if (d_cap != 0.0) atomicAdd(&S->capped_energy, d_cap);
    }
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
