/*
 * rt.h -- C ABI of the B300 shortwave Monte Carlo ray tracer.
 *
 * The method is that of Veerman, van Stratum & van Heerwaarden (2022),
 * "Shallow cumulus convection over land in cloud-resolving simulations with a
 * coupled ray tracer", Sec. 2.3 ("The ray tracer"): photons enter at the
 * domain top, move by null-collision tracking over a coarse grid of maximum
 * extinction, scatter by Rayleigh (gas) or Henyey-Greenstein (cloud) phase
 * functions, lose weight by absorption at every event, are rescaled by
 * Russian roulette below weight 0.5, reflect from a Lambertian surface, and
 * are tallied into 3D absorption, upward flux at the domain top and surface
 * direct and diffuse irradiance.
 *
 * Conventions used throughout
 *   - Grids are [nz][ny][nx] with x fastest; 2D surface fields are [ny][nx].
 *     x points east, y north, z up; cell (i,j,k) spans [i dx,(i+1) dx) x
 *     [j dy,(j+1) dy) x [k dz,(k+1) dz). The domain is periodic in x and y, the
 *     surface is z = 0 and the domain top z = nz dz.
 *   - Angles are degrees. The solar zenith angle must lie in [0, 90). The
 *     azimuth is clockwise from north and names where the sun stands (the
 *     paper's "south-west" sun is 228.1), so photons travel along
 *     (-sin sza sin az, -sin sza cos az, -cos sza).
 *   - toa_flux is the solar flux normal to the beam [W m^-2]; the flux through
 *     the horizontal domain top is toa_flux cos(sza).
 *   - Output units: W m^-2 for surface and top fluxes, W m^-3 for absorption,
 *     K day^-1 for heating rates.
 *   - mem arguments say where a pointer lives: RT_HOST (pageable or pinned host
 *     memory) or RT_DEVICE (device memory of the handle's GPU).
 *
 * Ownership and ordering
 *   - A handle owns all device memory it allocates; rt_destroy frees it.
 *   - Inputs are copied (host) or read (device) before the call returns to the
 *     stream order, so the caller may free or overwrite them once the handle's
 *     stream has passed the call.
 *   - Every call is ordered on the handle's stream (rt_set_stream; default the
 *     legacy default stream). Calls that write host memory synchronise it.
 *   - A handle is not thread-safe; distinct handles may be used from distinct
 *     threads.
 *
 * Errors
 *   - Every int-returning call returns RT_OK (0) or a negative RT_E_* code and
 *     records a message for rt_last_error() (thread-local).
 *   - Conditions found on the device (an event budget exhausted; invalid inputs
 *     of an rt_step launch) are recorded in the handle's status and returned by
 *     rt_synchronize, rt_stats and rt_fields; the kernels never trap and every
 *     loop in them is bounded.
 */
#ifndef RT_B300_H
#define RT_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_scene *rt_handle;

enum {
    RT_OK = 0,
    RT_E_INVAL = -1,   /* bad argument or invalid optical property */
    RT_E_STATE = -2,   /* call made in the wrong order (e.g. trace before optics) */
    RT_E_CUDA = -3,    /* CUDA runtime error */
    RT_E_OOM = -4,     /* device allocation failed */
    RT_E_BUDGET = -5,  /* a photon hit the per-photon step cap; tallies are incomplete */
    RT_E_BOUNDS = -6   /* the bounds-checking build (librt_b300_checked.so) found an index
                          outside its array; that access was redirected in bounds and the
                          results are invalid (a library bug, never expected) */
};

enum { RT_HOST = 0, RT_DEVICE = 1 };

/* Choice of scatterer at a real scattering event. The paper (Sec. 2.3) gives
 * the cloud probability as k_ext,cloud / k_ext; with separate gas and cloud
 * single-scattering albedos the unbiased choice is k_sca,cloud / k_sca. */
enum { RT_PCLD_SCATTERING = 0, RT_PCLD_EXTINCTION = 1 };

/* Tally precision: FP64 global accumulators (default) or FP32 (precision study). */
enum { RT_TALLY_FP64 = 0, RT_TALLY_FP32 = 1 };

/* Start positions at the domain top. Sec. 2.3 starts photons at the points of a
 * scrambled Sobol sequence. RT_BIRTH_PHILOX draws each photon's position in its
 * column from its own Philox stream. RT_BIRTH_SOBOL gives photon p, the k-th
 * photon (k = p div nx*ny) of column c = p mod nx*ny, the k-th point of the
 * two-dimensional Sobol sequence, XORed per axis with a 32-bit word drawn for
 * (column, seed) from Philox counter (c, 0, 0, 2); the photons of a column then
 * stratify its area, and each start point is still uniform. */
enum { RT_BIRTH_PHILOX = 0, RT_BIRTH_SOBOL = 1 };

/* Order in which a launch starts its photons. A launch lasts as long as its
 * longest photon history, typically a random walk through thick cloud.
 * RT_SCHEDULE_IDS starts photons in id order. RT_SCHEDULE_THICK_FIRST starts
 * all photons of one column in turn (a warp's lanes then share a column and
 * follow similar paths), columns in decreasing majorant optical depth, so the
 * long histories overlap the rest of the launch. It is used by single-scene
 * launches of whole rounds (photon range start and count multiples of nx*ny)
 * with at least 64 photons per column; other launches use id order. A
 * photon's history depends only on its id, so results are the same either way
 * up to the order of FP64 additions. */
enum { RT_SCHEDULE_IDS = 0, RT_SCHEDULE_THICK_FIRST = 1 };

typedef struct {
    int block_size;              /* threads per block of the transport kernel; 0 = 256 */
    int blocks_per_sm;           /* resident blocks per SM; 0 = as many as fit */
    int refill_chunk;            /* photon ids a warp takes from the queue at once; 0 = 32 */
    uint32_t max_steps;          /* per-photon cap on events + cell crossings; 0 = 10,000,000 */
    int pcld_mode;               /* RT_PCLD_*; applies from the next rt_set_optics */
    int tally_precision;         /* RT_TALLY_*; applies from the next rt_reset_tallies */
    int ready_threshold;         /* lanes of a warp that must have an event, surface hit or exit
                                    pending before the warp handles them together; 0 = 16 */
    int max_inner;               /* bound on walk sweeps between two such passes; 0 = 16 */
    int batch_optics;            /* 1: rt_set_optics also keeps gas and cloud apart and
                                    rt_build_accel builds the factored majorant, as
                                    rt_trace_batch needs (+20 B per cell); 0 (default): not */
    int birth;                   /* RT_BIRTH_*; default RT_BIRTH_PHILOX */
    int schedule;                /* RT_SCHEDULE_*; applies from the next rt_build_accel;
                                    default RT_SCHEDULE_THICK_FIRST */
    int box_levels;              /* majorant boxes (see rt_build_accel): 0..4 dilation levels,
                                    i.e. box radii up to 0, 1, 3, 7 or 15 coarse cells; 0 = every
                                    walk step crosses one coarse cell; applies from the next
                                    rt_build_accel; default 4 */
    float box_tau;               /* largest majorant optical depth across a box diagonal; 0 selects
                                    the default 0.5; applies from the next rt_build_accel */
    int tally_aggregate;         /* 1: in single-scene launches, lanes of a warp that flush
                                    absorption into the same cell sum their FP32 partials first and
                                    issue one FP64 atomic (fewer atomics; results then reproduce
                                    across launch shapes to FP32 rounding only); 0 (default): one
                                    atomic per photon and cell, reproducible to FP64 rounding */
    int refill_min;              /* lanes of a warp whose photons ended that it gathers before it
                                    starts new photons (births run with only those lanes active);
                                    0 = 8 */
} rt_options;

typedef struct {
    uint64_t photons;            /* photons traced since the last reset */
    uint64_t events;             /* majorant events (real scatterings + null collisions) */
    uint64_t scatters;           /* real scattering events */
    uint64_t crossings;          /* walk steps that crossed a box face (see rt_build_accel) */
    uint64_t surface_hits;
    uint64_t roulette_kills;
    uint64_t capped;             /* photons stopped by the step cap */
    uint64_t max_events_photon;  /* largest event count of a single photon */
    double energy_in;            /* W entering through the domain top */
    double energy_toa_up;        /* W leaving through the domain top (from the tallies) */
    double energy_atm_abs;       /* W absorbed in the atmosphere (from the tallies) */
    double energy_sfc_abs;       /* W absorbed by the surface (from the tallies) */
    double energy_created;       /* W added by roulette survivors (w -> 1) */
    double energy_destroyed;     /* W removed by roulette kills */
    double energy_capped;        /* W carried by photons stopped by the step cap */
    int status;                  /* device-side error: RT_OK, RT_E_BUDGET, or RT_E_INVAL (an
                                    rt_step launch found invalid inputs) */
} rt_stats_t;

/* Create a scene of nx*ny*nz cells of size dx*dy*dz metres on the current CUDA
 * device. Sizes must be positive and nx*ny*nz < 2^31. Returns NULL on error
 * (see rt_last_error). Allocates the derived optics, the tallies and the
 * per-launch scratch (about 32 B per cell). */
rt_handle rt_create(int nx, int ny, int nz, double dx, double dy, double dz);

/* Free everything the handle owns. NULL is accepted. */
int rt_destroy(rt_handle h);

/* Order all following calls of this handle on `stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream); NULL selects the default stream.
 * Handles share no device state, so the calls of two handles on two streams
 * may run at the same time: repeated steps that alternate between two handles
 * start one step's transport on the SMs that the previous step's last, longest
 * histories leave idle. */
int rt_set_stream(rt_handle h, void *stream);

int rt_set_options(rt_handle h, const rt_options *opt);
int rt_get_options(rt_handle h, rt_options *opt);

/* Per-cell optics for one spectral quadrature point (Sec. 2.3: the tracer needs
 * full-domain extinction, single-scattering albedo and asymmetry; gas and cloud
 * are given separately). Five float arrays of nx*ny*nz values, layout
 * [nz][ny][nx]: gas extinction [m^-1], gas single-scattering albedo, cloud
 * extinction [m^-1], cloud single-scattering albedo, cloud asymmetry g.
 * Validates (finite, extinction >= 0, albedos in [0,1], |g| < 1) and derives
 * the per-cell record used by the transport kernel. Synchronises the stream to
 * report RT_E_INVAL; after an error the handle holds no valid optics (rt_trace
 * returns RT_E_STATE) until a call succeeds. Invalidates the acceleration grid. */
int rt_set_optics(rt_handle h, const float *k_gas, const float *ssa_gas, const float *k_cld,
                  const float *ssa_cld, const float *g_cld, int mem);

/* The paper's own optics inputs (Sec. 2.3: total extinction, cloud extinction,
 * single-scattering albedo and asymmetry): four float arrays [nz][ny][nx] of
 * total k_ext [m^-1], cloud k_ext,cloud (<= k_ext), albedo and cloud g. A
 * scattering is by cloud with probability k_ext,cloud / k_ext, the paper's
 * ratio. Equivalent to rt_set_optics with k_gas = k_ext - k_ext,cloud and both
 * albedos equal. Not usable with rt_trace_batch (no gas/cloud split of the
 * albedo). Errors and state as rt_set_optics. */
int rt_set_optics_total(rt_handle h, const float *k_ext, const float *k_ext_cld, const float *ssa,
                        const float *g_cld, int mem);

/* Lambertian surface albedo per column (Sec. 2.3), nx*ny floats in [0,1]. */
int rt_set_surface(rt_handle h, const float *albedo, int mem);

/* Build the maximum-extinction acceleration grid (Sec. 2.3: a coarser grid whose
 * cells hold the largest extinction of the fine cells they cover, used as the
 * null-collision coefficient, without recursion). cx, cy, cz are the coarsening
 * factors (fine cells per coarse cell); the last coarse cell along an axis
 * covers the remainder. 0,0,0 selects the library default, 2,2,2 clipped to
 * the grid (the fastest factors measured on the 256 x 256 x 128 cumulus scene;
 * the caller-side autotuner in the Python package picks factors for other
 * scenes by timing trial launches).
 *
 * With rt_options.box_levels > 0 the grid also gets majorant boxes: each coarse
 * cell carries the cube of coarse cells within radius r of it (r one of 0, 1,
 * 3, 7, 15; periodic in x and y, clipped at the surface and the top) and the
 * largest extinction in that cube, with r the largest radius whose maximum
 * times the cube's diagonal stays below rt_options.box_tau. A walk step from
 * that cell crosses the whole cube with the cube's maximum as its majorant:
 * still an upper bound everywhere on the step, so the null-collision estimator
 * keeps its expectation, while a step through clear air replaces up to 31
 * coarse-cell crossings. */
int rt_build_accel(rt_handle h, int cx, int cy, int cz);

/* Trace `photons` photons of one spectral quadrature point and ADD their
 * contribution to the tallies (Sec. 2.3). Photon p starts in column
 * p mod (nx*ny) (samples per pixel = photons / (nx*ny), Sec. 2.4) at a uniform
 * position at the domain top, along the sun beam, with weight 1. Each photon
 * carries toa_flux cos(sza) nx dx ny dy / photons watts, so calls for different
 * quadrature points sum. `seed` keys the counter-based random streams: equal
 * seeds and photon ids give equal histories. Requires optics, surface and an
 * acceleration grid (RT_E_STATE otherwise). Asynchronous. */
int rt_trace(rt_handle h, double sza_deg, double azimuth_deg, double toa_flux,
             uint64_t photons, uint64_t seed);

/* As rt_trace for photon ids [photon_begin, photon_begin + photon_count) of a
 * run of photons_total photons: disjoint ranges traced by separate calls (or
 * separate GPUs) add up to the full run. */
int rt_trace_range(rt_handle h, double sza_deg, double azimuth_deg, double toa_flux,
                   uint64_t photon_begin, uint64_t photon_count, uint64_t photons_total,
                   uint64_t seed);

/* One traced (scene, quadrature point) pair of a batched launch. */
typedef struct {
    rt_handle scene;       /* optics, surface and grid set with batch_optics = 1; tallies add here */
    double sza_deg;        /* solar zenith angle of this job [deg, 0..90) */
    double azimuth_deg;
    double toa_flux;       /* flux of this quadrature point normal to the beam [W m^-2] */
    double gas_scale;      /* factor on the scene's gas extinction (absorption and scattering) */
    uint64_t photons;      /* photons of this job when total_photons is 0 */
    double diffuse_fraction; /* share of the top flux entering diffuse (as rt_trace_ex) */
} rt_job;

/* Trace all jobs -- every spectral quadrature point of several scenes of
 * different sizes -- in one persistent launch (Sec. 2.3 traces each quadrature
 * point independently; the tallies of a scene sum over its jobs as they would
 * over separate rt_trace calls). With total_photons > 0 the photons are split in
 * proportion to the energy each job brings into its domain (toa_flux cos(sza)
 * times the domain area), the largest remainders taking the leftovers;
 * otherwise each job traces its own `photons`. Job j uses Philox key
 * (seed lo, seed hi + j * 0x9E3779B9), so job 0 with gas_scale 1 draws the same
 * streams as rt_trace(seed). Per cell, k_abs = s k_abs,gas + k_abs,cloud and
 * k_sca = s k_sca,gas + k_sca,cloud with s = gas_scale; the majorant is
 * s max k_ext,gas + max k_ext,cloud per coarse cell. Up to 16 distinct scenes;
 * jobs are launched 512 at a time. Ordered on the first job's scene's stream;
 * other scenes' streams must not overlap with it. Counters and the energy
 * ledger are added to each job's own scene. Asynchronous. Errors: RT_E_INVAL,
 * RT_E_STATE (a scene without batch_optics or grid), RT_E_CUDA, RT_E_OOM. */
int rt_trace_batch(const rt_job *jobs, int njobs, uint64_t total_photons, uint64_t seed);

/* ---- a batched launch recorded once, replayed per model step ---- */

/* The paper's coupled runs make one radiation call per model step (Sec. 2.2),
 * each tracing all spectral quadrature points (Sec. 2.3). An rt_batch_step
 * records what rt_trace_batch(jobs, njobs, total_photons, seed) does -- the
 * photon budgets, the scene and job descriptors and the persistent launches
 * (one per 512 jobs) -- as one CUDA graph, preceded by a reset of every
 * scene's tallies, counters and energy ledger. Each rt_batch_step_launch
 * uploads the job keys for `seed` (one host-to-device copy of the
 * descriptors) and replays the graph on the first job's scene's stream:
 * results equal those of rt_trace_batch with that seed after
 * rt_reset_tallies on every scene, up to the order of FP64 additions. The
 * graph reads the scenes' device buffers, so optics rewritten in place are
 * traced by the next replay; the calls that reallocate or change a scene
 * (rt_set_optics, rt_build_accel, rt_set_options, rt_trace*, rt_step_create,
 * rt_destroy) return RT_E_STATE while a batch step uses it, and a scene takes
 * part in at most one batch step. Errors as rt_trace_batch; *out receives the
 * step. */
typedef struct rt_batch_step_s *rt_batch_step;
int rt_batch_step_create(const rt_job *jobs, int njobs, uint64_t total_photons, rt_batch_step *out);

/* Replay the recorded batch for `seed`; asynchronous. */
int rt_batch_step_launch(rt_batch_step s, uint64_t seed);

/* Synchronise, free the graph and give the scenes back. NULL is accepted. */
int rt_batch_step_destroy(rt_batch_step s);

/* As rt_trace_range, with a fraction `diffuse_fraction` in [0,1] of the
 * photons starting diffuse (Sec. 2.3: the diffuse part of the top-of-domain
 * flux enters as isotropic downwelling radiance, so those photons start with
 * cosine-weighted downward directions and count as scattered). Photon p is
 * diffuse when the fourth uniform of its birth block is below the fraction. */
int rt_trace_ex(rt_handle h, double sza_deg, double azimuth_deg, double toa_flux, double diffuse_fraction,
                uint64_t photon_begin, uint64_t photon_count, uint64_t photons_total, uint64_t seed);

/* Copy the accumulated fields out, normalised (Sec. 2.3 fluxes from mean
 * weights; absorption per cell volume). abs3d: nx*ny*nz doubles [W m^-3], the
 * sum of direct and diffuse absorption; sfc_dir, sfc_dif, toa_up: nx*ny doubles
 * [W m^-2]. Any pointer may be NULL. With RT_HOST the call synchronises and
 * returns the device status (RT_E_BUDGET if a photon was capped). */
int rt_fields(rt_handle h, double *abs3d, double *sfc_dir, double *sfc_dif, double *toa_up, int mem);

/* Absorption split by photons never scattered (direct) and scattered (diffuse),
 * nx*ny*nz doubles each [W m^-3], and surface absorption per column
 * (1 - albedo) (direct + diffuse) [W m^-2]. Any pointer may be NULL. */
int rt_fields_split(rt_handle h, double *abs_dir, double *abs_dif, double *sfc_abs, int mem);

/* Heating rate [K day^-1] = 86400 A / (rho(z) c_p) with c_p = 1004 J kg^-1 K^-1
 * and rho(z) = 1.225 exp(-z_c / 8000 m) kg m^-3 at cell centres. which: 0 total,
 * 1 direct, 2 diffuse. hr: nx*ny*nz doubles. */
int rt_heating_rate(rt_handle h, double *hr, int which, int mem);

/* Zero all tallies, counters, the energy ledger and the device status. */
int rt_reset_tallies(rt_handle h);

/* Counters and energy ledger since the last reset. Synchronises. */
int rt_stats(rt_handle h, rt_stats_t *out);

/* Wait for the handle's stream; returns the device status (RT_OK, RT_E_BUDGET,
 * or RT_E_INVAL after an rt_step launch with invalid inputs). */
int rt_synchronize(rt_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *rt_last_error(void);

/* RT_E_* code of the last failed call on this thread (RT_OK if none); the only
 * way to learn why rt_create returned NULL. */
int rt_last_error_code(void);

/* ---- coupled-model step: one graph replay per radiation call ---- */

/* In the paper's coupled runs the tracer is called every 60 s of model time with
 * the optics of the current model state (Sec. 2.2), and two experiments replace
 * the surface fluxes or the heating rates by their horizontal means
 * ("-hom" and "-hom-hr" runs, Sec. 2.4). An rt_step binds device input and
 * output buffers once and records the whole radiation call -- validation and
 * derivation of the optics, the majorant grid, a tally reset, the transport,
 * the normalised outputs and the optional homogenisation -- as one CUDA graph.
 * Each rt_step_launch replays it for the current contents of the inputs with
 * no host synchronisation and no allocation.
 *
 * optics selects the meaning of field[0..4] (device float arrays [nz][ny][nx],
 * read at every launch):
 *   RT_OPTICS_SPLIT  k_gas, ssa_gas, k_cld, ssa_cld, g_cld (as rt_set_optics)
 *   RT_OPTICS_TOTAL  k_ext, k_ext_cld, ssa, g; field[4] unused (as rt_set_optics_total)
 * albedo: device [ny][nx] floats read at every launch, or NULL to use the
 * handle's surface (which rt_set_surface may change between launches).
 * Outputs (device doubles, each may be NULL) are overwritten at every launch:
 * abs3d [W m^-3] and hr [K day^-1] nx*ny*nz; sfc_dir, sfc_dif, toa_up
 * [W m^-2] nx*ny.
 * homogenize: RT_HOM_SURFACE replaces sfc_dir and sfc_dif by their domain
 * means (upward surface flux albedo * (dir + dif) then follows for a uniform
 * albedo); RT_HOM_HEATING replaces every layer of abs3d and hr by its mean.
 * Means are summed in a fixed order, so a replay is reproducible up to the
 * order of the transport's atomic additions. */
enum { RT_OPTICS_SPLIT = 0, RT_OPTICS_TOTAL = 1 };
enum { RT_HOM_SURFACE = 1, RT_HOM_HEATING = 2 };

typedef struct {
    int optics;                  /* RT_OPTICS_* */
    const float *field[5];
    const float *albedo;
    uint64_t photons;            /* photons per launch (> 0) */
    double *abs3d, *hr, *sfc_dir, *sfc_dif, *toa_up;
    int homogenize;              /* RT_HOM_* bits */
} rt_step_desc;

typedef struct rt_step_s *rt_step;

/* Record the step of handle h. The handle must hold valid optics, a surface and
 * an acceleration grid (RT_E_STATE otherwise): the grid's coarsening factors,
 * the handle's options and its tally precision are fixed at this call. While
 * the step exists the handle belongs to it: rt_set_optics, rt_set_optics_total,
 * rt_build_accel, rt_set_options, rt_trace*, and rt_destroy return RT_E_STATE;
 * rt_fields, rt_fields_split, rt_heating_rate, rt_stats and rt_synchronize
 * report the last launch. One step per handle. *out receives the step. */
int rt_step_create(rt_handle h, const rt_step_desc *desc, rt_step *out);

/* Replay the step on the handle's stream for one sun position, top flux,
 * diffuse fraction (as rt_trace_ex) and seed; asynchronous. Invalid values in
 * the bound inputs are found on the device: the launch then traces nothing,
 * writes zero outputs and rt_synchronize / rt_stats of the handle report
 * RT_E_INVAL. */
int rt_step_launch(rt_step s, double sza_deg, double azimuth_deg, double toa_flux, double diffuse_fraction,
                   uint64_t seed);

/* Free the step's graph and give the handle back to the ordinary calls. NULL is
 * accepted. */
int rt_step_destroy(rt_step s);

/* ---- tracing without any allocation ---- */

/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory -- for example an atmospheric model that reserves all
 * of its GPU memory in one pool at start-up and may not allocate inside its
 * time loop, or a host framework whose own allocator must own every buffer.
 * rt_create allocates, so such callers cannot hold a handle.
 *
 * Traces `photons` photons exactly as rt_trace does (Sec. 2.3; same random
 * streams for the same seed, scatterer choice RT_PCLD_SCATTERING) and ADDS
 * their contribution to the caller's output buffers, in the units of
 * rt_fields / rt_fields_split. Every pointer is device memory of the current
 * device and is owned by the caller:
 *   inputs  k_gas, ssa_gas, k_cld, ssa_cld, g_cld: nx*ny*nz floats [nz][ny][nx];
 *           albedo: nx*ny floats
 *   outputs abs_dir, abs_dif: nx*ny*nz doubles [W m^-3]; sfc_dir, sfc_dif,
 *           toa_up: nx*ny doubles [W m^-2]; zero them before the first call.
 * cx, cy, cz are the coarsening factors of the majorant grid (0,0,0 = 4,4,4
 * clipped). `stream` orders the work (NULL = default stream); the call waits
 * for it to finish, then returns. events_out (host, may be NULL) receives the
 * number of majorant events.
 *
 * Memory: the call allocates nothing. The photon queue head, an event counter,
 * a status word and the majorant grid live in one fixed device array of
 * 4 MiB + 256 B inside the library, which every GPU that loads the library
 * holds until the process exits. The majorant grid must fit in it: at most
 * 1,048,576 coarse cells, otherwise RT_E_INVAL. Every call looks the array's
 * device address up in the current context (cudaGetSymbolAddress) and
 * synchronises `stream` before it returns. All calls on a device share the array
 * and it keeps the last call's contents (each call clears what must start at
 * zero), so calls whose work overlaps on the GPU race: serialise them.
 * Errors: RT_E_INVAL (sizes, pointers, angles, too many coarse cells, invalid
 * optical property -- outputs then unchanged), RT_E_BUDGET (a photon hit the
 * step cap), RT_E_CUDA. */
int rt_trace_noalloc(int nx, int ny, int nz, double dx, double dy, double dz, const float *k_gas,
                     const float *ssa_gas, const float *k_cld, const float *ssa_cld, const float *g_cld,
                     const float *albedo, int cx, int cy, int cz, double sza_deg, double azimuth_deg,
                     double toa_flux, uint64_t photons, uint64_t seed, double *abs_dir, double *abs_dif,
                     double *sfc_dir, double *sfc_dif, double *toa_up, void *stream, uint64_t *events_out);

/* ---- test entry points: the device RNG and samplers, on host buffers ---- */

/* n Philox4x32-10 blocks computed on the GPU: ctr[4n], key[2n] in, out[4n]. */
int rt_debug_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n);

/* n direction cosines from the device samplers (kind 0 Rayleigh, 1
 * Henyey-Greenstein with asymmetry g, 2 Lambertian), drawn with the transport
 * kernel's own functions; out: n floats on the host. */
int rt_debug_sample(int kind, float g, uint64_t n, uint64_t seed, float *out);

/* n two-dimensional Sobol points k0 .. k0+n-1 as the transport kernel computes
 * them, XORed with sx and sy: out[2i], out[2i+1] are 32-bit binary fractions
 * (host array of 2n words). */
int rt_debug_sobol(uint64_t k0, int n, uint32_t sx, uint32_t sy, uint32_t *out);

/* n rotations by the transport kernel's own turn: out[3i..3i+2] is the unit
 * vector at angle acos(mu[i]) from d and azimuth phi[i] about it (host arrays). */
int rt_debug_turn(const float d[3], const float *mu, const float *phi, float *out, int n);

/* Memory-system probe (measurement of the GPU, not part of the method): one
 * launch reads `bytes` of device buffer buf `reps` times over with 16-byte
 * loads cached in L2 only (ld.global.cg), on `stream`; the caller times it.
 * Swept over buffer sizes it gives the L2 read bandwidth below the L2
 * capacity and the DRAM bandwidth above it. bytes: a positive multiple of 16;
 * buf 16-byte aligned; sink: one device word, written only so that the
 * loads are not removed. RT_E_INVAL otherwise. */
int rt_probe_read(const void *buf, uint64_t bytes, int reps, unsigned *sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_B300_H */
