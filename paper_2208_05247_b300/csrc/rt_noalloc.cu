// rt_noalloc.cu -- rt_trace_noalloc: the transport of rt_trace for callers that
// cannot allocate device memory.
//
// Some callers own every byte of device memory themselves: an atmospheric model
// that sets up one memory pool at start-up and may not allocate inside its time
// loop, a framework whose allocator is the only one allowed to touch the GPU,
// or code with a fixed memory budget. They cannot create an rt_handle, because
// the handle allocates its optics record, majorant grid, tallies and per-launch
// scratch with cudaMalloc. This entry point takes the caller's own device
// buffers for every input and output, and the transport reads the five optics
// fields directly instead of a derived record. The only other memory it needs
// -- the launch scratch (photon queue head, counters, energy ledger, status),
// the majorant grid, its boxes and the two arrays their build works in -- lives
// in one file-scope device array of fixed size that every GPU loading the
// library holds until the process exits.
//
// The photons run through the same trace_kernel as rt_trace's (its
// kOpticsFields mode), and the per-cell optics are formed by the same
// cell_optics arithmetic as rt_set_optics forms the record, so for equal seeds
// and default options the results equal rt_trace's up to the order of the FP64
// atomic additions. Photons start in id order (rt_trace may start thick
// columns first; a photon's history does not depend on that order).
#include <climits>
#include <cmath>
#include <cstdio>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "rt.h"
#include "rt_kernels.cuh"

namespace rt {
int record_error(int code, const char *msg);   // rt_api.cu: sets rt_last_error()
}

namespace {

constexpr size_t kMaxCoarseCells = size_t(1) << 20;      // majorant cells
constexpr size_t kHeaderBytes = 256;                     // rt::Scratch, padded
// header, then four arrays of kMaxCoarseCells words: majorant, box words and
// the two scratch arrays of the box build (16 MiB + 256 B in all)
constexpr size_t kScratchBytes = kHeaderBytes + 4 * kMaxCoarseCells * sizeof(float);
static_assert(sizeof(rt::Scratch) <= kHeaderBytes, "launch scratch must fit the header");

// Shared by every call on a device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch in the current context. It is looked up on every
// call rather than cached: after cudaDeviceReset, or under another context on
// the same device ordinal, the module is loaded again and the array can move.
// The lookup costs far less than the call's launches and synchronisation.
int scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        char msg[256];
        snprintf(msg, sizeof msg, "rt_trace_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return rt::record_error(RT_E_CUDA, msg);
    }
    *out = p;
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
    nvtxRangePushA("rt_trace_noalloc");
    struct PopRange { ~PopRange() { nvtxRangePop(); } } nvtx_pop;
    char msg[256];
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) ||
        !std::isfinite(dy) || !std::isfinite(dz))
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: sizes must be positive");
    const size_t ncell = (size_t)nx * ny * nz;
    if (ncell >= (size_t)1 << 31) return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: nx*ny*nz must be below 2^31");
    if (!k_gas || !ssa_gas || !k_cld || !ssa_cld || !g_cld || !albedo || !abs_dir || !abs_dif || !sfc_dir ||
        !sfc_dif || !toa_up)
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: null buffer");
    if (cx == 0 && cy == 0 && cz == 0) {
        cx = nx < rt::kDefaultCoarse ? nx : rt::kDefaultCoarse;
        cy = ny < rt::kDefaultCoarse ? ny : rt::kDefaultCoarse;
        cz = nz < rt::kDefaultCoarse ? nz : rt::kDefaultCoarse;
    }
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
    unsigned char *b8 = static_cast<unsigned char *>(base);
    rt::Scratch *scr = reinterpret_cast<rt::Scratch *>(b8);
    float *kmax = reinterpret_cast<float *>(b8 + kHeaderBytes);
    uint32_t *box = reinterpret_cast<uint32_t *>(b8 + kHeaderBytes + kMaxCoarseCells * sizeof(float));
    float *w0 = reinterpret_cast<float *>(b8 + kHeaderBytes + 2 * kMaxCoarseCells * sizeof(float));
    float *w1 = reinterpret_cast<float *>(b8 + kHeaderBytes + 3 * kMaxCoarseCells * sizeof(float));

    // the header keeps the last call's contents: clear it (queue head,
    // counters, ledger, status and the invalid-input flag)
    cudaError_t e = cudaMemsetAsync(scr, 0, sizeof(rt::Scratch), st);
    if (e == cudaSuccess) {
        rt::majorant_from_fields<<<rt::box_grid(ncoarse), 256, 0, st>>>(k_gas, ssa_gas, k_cld, ssa_cld, g_cld, albedo,
                                                                         kmax, &scr->bad, nx, ny, nz, cx, cy, cz, NX,
                                                                         NY, NZ);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = rt::build_boxes(kmax, box, w0, w1, NX, NY, NZ, cx * dx, cy * dy, cz * dz, rt::kDefaultBoxLevels,
                            rt::kDefaultBoxTau, nx % cx == 0 && ny % cy == 0, st);
    if (e == cudaSuccess) {
        // invalid inputs close the photon queue: the transport then traces nothing
        rt::step_gate<<<1, 32, 0, st>>>(&scr->bad, scr);
        e = cudaGetLastError();
    }
    int dev = 0, sms = 1, bps = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rt::trace_kernel<double, rt::kOpticsFields>, 256, 0);
    if (e == cudaSuccess) {
        rt::TraceArgs<double> A{};
        rt::SceneDev<double> &S = A.scene;
        S.f_kg = k_gas; S.f_wg = ssa_gas; S.f_kc = k_cld; S.f_wc = ssa_cld; S.gcl = g_cld;
        S.box = box;
        S.alb = albedo;
        S.tal.abs_dir = abs_dir; S.tal.abs_dif = abs_dif;
        S.tal.sfc_dir = sfc_dir; S.tal.sfc_dif = sfc_dif; S.tal.toa = toa_up;
        S.scr = scr;
        S.nx = nx; S.ny = ny; S.nz = nz; S.NX = NX; S.NY = NY; S.NZ = NZ; S.cx = cx; S.cy = cy; S.cz = cz;
        S.pcld_mode = RT_PCLD_SCATTERING;
        S.birth = RT_BIRTH_PHILOX;
        S.dx = (float)dx; S.dy = (float)dy; S.dz = (float)dz;
        S.inv_dx = (float)(1.0 / dx); S.inv_dy = (float)(1.0 / dy); S.inv_dz = (float)(1.0 / dz);
        S.Lx = (float)(nx * dx); S.Ly = (float)(ny * dy); S.H = (float)(nz * dz);
        S.cdx = (float)(cx * dx); S.cdy = (float)(cy * dy); S.cdz = (float)(cz * dz);
        S.inv_cdx = (float)(1.0 / (cx * dx)); S.inv_cdy = (float)(1.0 / (cy * dy)); S.inv_cdz = (float)(1.0 / (cz * dz));
        S.xcap = nx % cx ? S.Lx : INFINITY;
        S.ycap = ny % cy ? S.Ly : INFINITY;
        S.fxcap = nx % cx ? nx : INT_MAX;
        S.fycap = ny % cy ? ny : INT_MAX;
        rt::JobDev &J = A.job;
        const double t = sza_deg * 3.14159265358979323846 / 180.0, p = azimuth_deg * 3.14159265358979323846 / 180.0;
        J.sx = (float)(-std::sin(t) * std::sin(p));
        J.sy = (float)(-std::sin(t) * std::cos(p));
        J.sz = (float)(-std::cos(t));
        J.gas_scale = 1.0f;
        J.key0 = (uint32_t)seed;
        J.key1 = (uint32_t)(seed >> 32);
        J.ncol = (unsigned long long)nx * ny;
        J.energy = toa_flux * std::cos(t) * (nx * dx) * (ny * dy) / (double)photons;
        J.scale2 = J.energy / (dx * dy);
        J.scale3 = J.energy / (dx * dy * dz);
        A.count = photons;
        A.scr = scr;
        A.max_steps = rt::kDefaultMaxSteps;
        A.chunk = 32;
        A.ready_threshold = rt::kDefaultReadyThreshold;
        A.max_inner = rt::kDefaultMaxInner;
        A.refill_min = rt::kDefaultRefillMin;
        rt::trace_kernel<double, rt::kOpticsFields><<<sms * (bps > 0 ? bps : 1), 256, 0, st>>>(A);
        e = cudaGetLastError();
    }
    rt::Scratch h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, scr, sizeof(rt::Scratch), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "rt_trace_noalloc: %s", cudaGetErrorString(e));
        return rt::record_error(RT_E_CUDA, msg);
    }
    if (events_out) *events_out = h.events;
    if (h.status & rt::kStatusBounds)
        return rt::record_error(RT_E_BOUNDS, "rt_trace_noalloc: an index check of the bounds-checking build failed");
    if (h.status & rt::kStatusInput)
        return rt::record_error(RT_E_INVAL, "rt_trace_noalloc: invalid optical property (NaN, negative "
                                            "extinction, albedo outside [0,1] or |g| >= 1); outputs unchanged");
    if (h.status & rt::kStatusBudget)
        return rt::record_error(RT_E_BUDGET, "rt_trace_noalloc: a photon reached the step cap; outputs incomplete");
    return RT_OK;
}
