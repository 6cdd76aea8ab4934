// rt_noalloc.cu -- rt_trace_noalloc: the transport of rt_trace for callers that
// cannot allocate device memory.
//
// Some callers own every byte of device memory themselves: an atmospheric model
// that sets up one memory pool at start-up and may not allocate inside its time
// loop, a framework whose allocator is the only one allowed to touch the GPU,
// or code with a fixed memory budget. They cannot create an rt_handle, because
// the handle allocates its optics record, majorant grid, tallies and per-launch
// scratch with cudaMalloc. This entry point takes the caller's own device
// buffers for every input and output and reads the five optics fields
// directly. The only other memory it needs -- the photon queue head, an event
// counter, a status word and the majorant grid -- lives in one file-scope
// device array of fixed size that every GPU loading the library holds until
// the process exits.
//
// Each photon follows exactly the arithmetic of trace_kernel (same Philox
// counters, same walk over the coarse grid, same event and surface handling),
// so for equal seeds the results equal rt_trace's up to the order of the FP64
// atomic additions. The photons are scheduled more simply (one photon per
// thread at a time), which is slower than rt_trace.
#include <cmath>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "rt.h"
#include "rt_device.cuh"

namespace rt {
int record_error(int code, const char *msg);   // rt_api.cu: sets rt_last_error()
}

namespace {

constexpr size_t kMaxCoarseCells = size_t(1) << 20;      // majorant cells (4 MiB)
constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + kMaxCoarseCells * sizeof(float);
constexpr int kMaxDevices = 64;
constexpr int kBadInput = 2;
constexpr int kBudget = 1;
constexpr uint32_t kMaxSteps = 10000000u;

struct Header {
    unsigned long long queue_head;
    unsigned long long events;
    int status;
};

// Shared by every call on a device: the header first, then the majorant grid.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Args {
    const float *__restrict__ kg, *__restrict__ wg, *__restrict__ kc, *__restrict__ wc, *__restrict__ gc;
    const float *__restrict__ alb;
    double *abs_dir, *abs_dif, *sfc_dir, *sfc_dif, *toa;
    Header *hdr;
    const float *kmax;
    unsigned long long count, ncol;
    int nx, ny, nz, NX, NY, NZ, cx, cy, cz;
    float dx, dy, dz, inv_dx, inv_dy, inv_dz, Lx, Ly, H, cdx, cdy, cdz, sx, sy, sz;
    uint32_t key0, key1;
    double scale2, scale3;
};

// Majorant grid straight from the optics fields, with the per-cell values
// formed as rt_set_optics forms them; invalid inputs set kBadInput.
__global__ void majorant_from_fields(const float *__restrict__ kg, const float *__restrict__ wg,
                                     const float *__restrict__ kc, const float *__restrict__ wc,
                                     const float *__restrict__ gc, const float *__restrict__ alb, float *kmax,
                                     Header *hdr, int nx, int ny, int nz, int cx, int cy, int cz, int NX, int NY,
                                     int NZ)
{
    const int n = NX * NY * NZ;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
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
                    const float ksg = a * b, ksc = cc * d;
                    const float ksca = ksg + ksc;
                    const float kabs = fmaf(a, 1.0f - b, cc * (1.0f - d));
                    m = fmaxf(m, kabs + ksca);
                }
        if (K == 0)
            for (int j = J * cy; j < j1; ++j)
                for (int i = I * cx; i < i1; ++i) {
                    const float al = alb[(size_t)j * nx + i];
                    ok = ok && (al >= 0.0f) && (al <= 1.0f);
                }
        if (!ok) atomicOr(&hdr->status, kBadInput);
        kmax[q] = m;
    }
}

__global__ void __launch_bounds__(256) trace_fields(const __grid_constant__ Args A)
{
    if (A.hdr->status & kBadInput) return;
    const uint32_t k0 = A.key0, k1 = A.key1;
    unsigned long long n_ev = 0;
    for (;;) {
        const unsigned long long gid = atomicAdd(&A.hdr->queue_head, 1ull);
        if (gid >= A.count) break;
        // birth at the domain top along the sun beam
        const unsigned col0 = (gid >> 32) ? (unsigned)(gid % A.ncol) : (uint32_t)gid % (uint32_t)A.ncol;
        const int ci = (int)(col0 % (unsigned)A.nx), cj = (int)(col0 / (unsigned)A.nx);
        const uint4 r0 = rt::philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), 0u, 0u), k0, k1);
        float ox = ((float)ci + rt::u01(r0.x)) * A.dx;
        float oy = ((float)cj + rt::u01(r0.y)) * A.dy;
        float oz = A.H;
        float ux = A.sx, uy = A.sy, uz = A.sz;
        float tau = -__logf(rt::u01(r0.z));
        float w = 1.f;
        bool direct = true;
        int I = ci / A.cx, J = cj / A.cy, K = A.NZ - 1;
        float kmaj = A.kmax[((size_t)K * A.NY + J) * A.NX + I];
        float ivx, ivy, ivz, tnx, tny, tnz, tcur;
        auto start_segment = [&]() {
            tcur = 0.f;
            ivx = __frcp_rn(ux); ivy = __frcp_rn(uy); ivz = __frcp_rn(uz);
            tnx = ux > 0.f ? (fminf((float)(I + 1) * A.cdx, A.Lx) - ox) * ivx
                : ux < 0.f ? ((float)I * A.cdx - ox) * ivx : INFINITY;
            tny = uy > 0.f ? (fminf((float)(J + 1) * A.cdy, A.Ly) - oy) * ivy
                : uy < 0.f ? ((float)J * A.cdy - oy) * ivy : INFINITY;
            tnz = uz > 0.f ? (fminf((float)(K + 1) * A.cdz, A.H) - oz) * ivz
                : uz < 0.f ? ((float)K * A.cdz - oz) * ivz : INFINITY;
            tnx = fmaxf(tnx, 0.f); tny = fmaxf(tny, 0.f); tnz = fmaxf(tnz, 0.f);
        };
        start_segment();
        uint32_t blk = 1, steps = 0;
        int pcell = -1;
        bool pdir = false;
        float pacc = 0.f;
        bool alive = true;
        while (alive) {
            // advance over coarse faces until an event, the surface or the top
            int what = 0;   // 1 event, 2 surface, 3 top, 4 step cap
            while (what == 0) {
                if (++steps > kMaxSteps) { what = 4; break; }
                float tm;
                int ax;
                if (tnx <= tny && tnx <= tnz) { tm = tnx; ax = 0; }
                else if (tny <= tnz) { tm = tny; ax = 1; }
                else { tm = tnz; ax = 2; }
                const float dt = fmaxf(tm - tcur, 0.f);
                if (kmaj * dt > tau) {
                    tcur += __fdividef(tau, kmaj);
                    what = 1;
                    break;
                }
                tau = fmaf(-kmaj, dt, tau);
                tcur = tm;
                if (ax == 0) {
                    if (ux > 0.f) {
                        if (++I == A.NX) { I = 0; ox -= A.Lx; }
                        tnx = (fminf((float)(I + 1) * A.cdx, A.Lx) - ox) * ivx;
                    } else {
                        if (--I < 0) { I = A.NX - 1; ox += A.Lx; }
                        tnx = ((float)I * A.cdx - ox) * ivx;
                    }
                } else if (ax == 1) {
                    if (uy > 0.f) {
                        if (++J == A.NY) { J = 0; oy -= A.Ly; }
                        tny = (fminf((float)(J + 1) * A.cdy, A.Ly) - oy) * ivy;
                    } else {
                        if (--J < 0) { J = A.NY - 1; oy += A.Ly; }
                        tny = ((float)J * A.cdy - oy) * ivy;
                    }
                } else {
                    if (uz > 0.f) {
                        if (++K == A.NZ) { what = 3; break; }
                        tnz = (fminf((float)(K + 1) * A.cdz, A.H) - oz) * ivz;
                    } else {
                        if (--K < 0) { what = 2; break; }
                        tnz = ((float)K * A.cdz - oz) * ivz;
                    }
                }
                kmaj = A.kmax[((size_t)K * A.NY + J) * A.NX + I];
            }
            const int ilo = I * A.cx, ihi = min(ilo + A.cx, A.nx);
            const int jlo = J * A.cy, jhi = min(jlo + A.cy, A.ny);
            const float px = fmaf(ux, tcur, ox), py = fmaf(uy, tcur, oy);
            const int fi = min(max((int)(px * A.inv_dx), ilo), ihi - 1);
            const int fj = min(max((int)(py * A.inv_dy), jlo), jhi - 1);
            bool end_photon = false;
            if (what == 1) {
                ++steps;
                const float pz = fmaf(uz, tcur, oz);
                const int klo = K * A.cz, khi = min(klo + A.cz, A.nz);
                const int fk = min(max((int)(pz * A.inv_dz), klo), khi - 1);
                const int cell = (fk * A.ny + fj) * A.nx + fi;
                const float a = A.kg[cell], b = A.wg[cell], cc = A.kc[cell], d = A.wc[cell];
                const float ksg = a * b, ksc = cc * d;
                const float ksca = ksg + ksc;
                const float kabs = fmaf(a, 1.0f - b, cc * (1.0f - d));
                const float pabs = fminf(__fdividef(kabs, kmaj), 1.0f);
                const float wn = w * (1.0f - pabs);
                if (cell != pcell || direct != pdir) {
                    if (pcell >= 0) atomicAdd((pdir ? A.abs_dir : A.abs_dif) + pcell, (double)(pacc * (float)A.scale3));
                    pcell = cell; pdir = direct; pacc = 0.f;
                }
                pacc += w - wn;
                w = wn;
                ++n_ev;
                const uint4 r = rt::philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u), k0, k1);
                ++blk;
                ox = px; oy = py; oz = pz;
                const float den = kmaj - kabs;
                bool scattered = false;
                if (den > 0.f) {
                    const float xd = rt::u01(r.x) * den;
                    if (xd < ksca) {
                        const float mu = (xd < ksc) ? rt::hg_mu(A.gc[cell], rt::u01(r.y))
                                                    : rt::rayleigh_mu(rt::u01(r.y));
                        float sp, cp;
                        rt::azimuth(rt::u01(r.z), sp, cp);
                        rt::turn(ux, uy, uz, mu, sp, cp);
                        direct = false;
                        scattered = true;
                    }
                }
                if (scattered) {
                    start_segment();
                } else {
                    tnx -= tcur; tny -= tcur; tnz -= tcur;
                    tcur = 0.f;
                }
                tau = -__logf(rt::u01(r.w));
                if (w < 0.5f) {
                    const uint4 q = rt::philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk - 1u, 1u), k0, k1);
                    if (rt::u01(q.x) > w) end_photon = true;
                    else w = 1.f;
                }
            } else if (what == 2) {
                ++steps;
                const int col = fj * A.nx + fi;
                atomicAdd((direct ? A.sfc_dir : A.sfc_dif) + col, (double)(w * (float)A.scale2));
                w *= A.alb[col];
                direct = false;
                const uint4 r = rt::philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), blk, 0u), k0, k1);
                ++blk;
                rt::lambert_up(ux, uy, uz, rt::u01(r.x), rt::u01(r.y));
                tau = -__logf(rt::u01(r.w));
                K = 0;
                ox = px; oy = py; oz = 0.f;
                start_segment();
                if (w < 0.5f) {
                    if (rt::u01(r.z) > w) end_photon = true;
                    else w = 1.f;
                }
            } else if (what == 3) {
                atomicAdd(A.toa + (fj * A.nx + fi), (double)(w * (float)A.scale2));
                end_photon = true;
            } else {
                atomicOr(&A.hdr->status, kBudget);
                end_photon = true;
            }
            if (end_photon) {
                if (pcell >= 0) atomicAdd((pdir ? A.abs_dir : A.abs_dif) + pcell, (double)(pacc * (float)A.scale3));
                alive = false;
            }
        }
    }
    if (n_ev) atomicAdd(&A.hdr->events, n_ev);
}

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rt::record_error(RT_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rt::record_error(RT_E_CUDA, "rt_trace_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "rt_trace_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return rt::record_error(RT_E_CUDA, msg);
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RT_OK;
}

}  // namespace

extern "C" int rt_trace_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, const float *k_gas,
                                const float *ssa_gas, const float *k_cld, const float *ssa_cld,
                                const float *g_cld, const float *albedo, int cx, int cy, int cz,
                                double sza_deg, double azimuth_deg, double toa_flux, uint64_t photons,
                                uint64_t seed, double *abs_dir, double *abs_dif, double *sfc_dir,
                                double *sfc_dif, double *toa_up, void *stream, uint64_t *events_out)
{
    char msg[256];
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) ||
        !std::isfinite(dy) || !std::isfinite(dz))
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: sizes must be positive");
    const size_t ncell = (size_t)nx * ny * nz;
    if (ncell >= (size_t)1 << 31) return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: nx*ny*nz must be below 2^31");
    if (!k_gas || !ssa_gas || !k_cld || !ssa_cld || !g_cld || !albedo || !abs_dir || !abs_dif || !sfc_dir ||
        !sfc_dif || !toa_up)
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: null buffer");
    if (cx == 0 && cy == 0 && cz == 0) { cx = nx < 4 ? nx : 4; cy = ny < 4 ? ny : 4; cz = nz < 4 ? nz : 4; }
    if (cx <= 0 || cy <= 0 || cz <= 0 || cx > nx || cy > ny || cz > nz)
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: coarsening factors must be in [1, n] per axis");
    const int NX = (nx + cx - 1) / cx, NY = (ny + cy - 1) / cy, NZ = (nz + cz - 1) / cz;
    const size_t ncoarse = (size_t)NX * NY * NZ;
    if (ncoarse > kMaxCoarseCells) {
        snprintf(msg, sizeof msg, "rt_trace_noalloc: %zu coarse cells exceed the fixed maximum of %zu; "
                 "use larger coarsening factors or rt_trace", ncoarse, kMaxCoarseCells);
        return rt::record_error(RT_E_INVAL, msg);
    }
    if (!(sza_deg >= 0.0 && sza_deg < 90.0)) return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: sza must be in [0, 90)");
    if (!std::isfinite(azimuth_deg)) return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: azimuth must be finite");
    if (!(toa_flux >= 0.0) || !std::isfinite(toa_flux)) return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: toa_flux must be >= 0");
    if (events_out) *events_out = 0;
    if (photons == 0) return RT_OK;

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Header *hdr = static_cast<Header *>(base);
    float *kmax = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + kHeaderBytes);

    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(Header), st);
    if (e == cudaSuccess) {
        majorant_from_fields<<<(unsigned)((ncoarse + 255) / 256), 256, 0, st>>>(k_gas, ssa_gas, k_cld, ssa_cld, g_cld,
                                                                                 albedo, kmax, hdr, nx, ny, nz, cx, cy, cz,
                                                                                 NX, NY, NZ);
        e = cudaGetLastError();
    }
    int dev = 0, sms = 1, bps = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, trace_fields, 256, 0);
    if (e == cudaSuccess) {
        Args A{};
        A.kg = k_gas; A.wg = ssa_gas; A.kc = k_cld; A.wc = ssa_cld; A.gc = g_cld; A.alb = albedo;
        A.abs_dir = abs_dir; A.abs_dif = abs_dif; A.sfc_dir = sfc_dir; A.sfc_dif = sfc_dif; A.toa = toa_up;
        A.hdr = hdr; A.kmax = kmax;
        A.count = photons; A.ncol = (unsigned long long)nx * ny;
        A.nx = nx; A.ny = ny; A.nz = nz; A.NX = NX; A.NY = NY; A.NZ = NZ; A.cx = cx; A.cy = cy; A.cz = cz;
        A.dx = (float)dx; A.dy = (float)dy; A.dz = (float)dz;
        A.inv_dx = (float)(1.0 / dx); A.inv_dy = (float)(1.0 / dy); A.inv_dz = (float)(1.0 / dz);
        A.Lx = (float)(nx * dx); A.Ly = (float)(ny * dy); A.H = (float)(nz * dz);
        A.cdx = (float)(cx * dx); A.cdy = (float)(cy * dy); A.cdz = (float)(cz * dz);
        const double t = sza_deg * 3.14159265358979323846 / 180.0, p = azimuth_deg * 3.14159265358979323846 / 180.0;
        A.sx = (float)(-std::sin(t) * std::sin(p));
        A.sy = (float)(-std::sin(t) * std::cos(p));
        A.sz = (float)(-std::cos(t));
        A.key0 = (uint32_t)seed; A.key1 = (uint32_t)(seed >> 32);
        const double energy = toa_flux * std::cos(t) * (nx * dx) * (ny * dy) / (double)photons;
        A.scale2 = energy / (dx * dy);
        A.scale3 = energy / (dx * dy * dz);
        trace_fields<<<sms * (bps > 0 ? bps : 1), 256, 0, st>>>(A);
        e = cudaGetLastError();
    }
    Header h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, hdr, sizeof(Header), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "rt_trace_noalloc: %s", cudaGetErrorString(e));
        return rt::record_error(RT_E_CUDA, msg);
    }
    if (events_out) *events_out = h.events;
    if (h.status & kBadInput)
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: invalid optical property (NaN, negative "
                                            "extinction, albedo outside [0,1] or |g| >= 1); outputs unchanged");
    if (h.status & kBudget)
        return rt::record_error(RT_E_BUDGET, "rt_trace_noalloc: a photon reached the step cap; outputs incomplete");
    return RT_OK;
}
