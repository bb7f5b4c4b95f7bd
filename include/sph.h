/*
 * sph.h - C ABI of the GB300 weakly-compressible SPH hot path.
 *
 * The library runs, on one sm_103a GPU, the per-step pipeline of a
 * weakly-compressible SPH solver (arXiv 2207.11328, Sections 2.1-2.3):
 * cell hash -> key sort -> particle reorder -> cell start/end tables ->
 * split neighbour list -> particle interactions (continuity, momentum with
 * the Tait/Cole equation of state, Wendland C2 gradient, artificial or
 * laminar viscosity, dynamic boundary particles) -> predictor-corrector
 * integration with the CFL time-step reduction.
 *
 * Conventions
 *  - Every call returns SPH_OK (0) or a negative SPH_ERR_* code.  Device
 *    errors found by kernels (neighbour overflow, non-finite state) are
 *    recorded in a sticky device error word; they are reported by the next
 *    call that synchronises (sph_get_stats, sph_download*, sph_sync) and
 *    stay set until sph_clear_error.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - Host arrays are read or written during the call only (copied);
 *    pointers named *_dev are device pointers that the caller owns.
 *  - Particle arrays are particle-major: pos[3*i + axis].
 *  - The library allocates all its device buffers once, in sph_create, for
 *    max_particles particles (paper, "The GPU in GPUSPH": arrays are
 *    allocated once; particles that leave the domain are dropped during the
 *    sort; a capacity overflow is an error, not a reallocation).
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define SPH_OK                  0
#define SPH_ERR_ARG            -1  /* bad argument (NULL, size, layout, physics out of range) */
#define SPH_ERR_CUDA           -2  /* CUDA runtime error (allocation, launch) */
#define SPH_ERR_CAPACITY       -3  /* more particles than max_particles */
#define SPH_ERR_NEIB_OVERFLOW  -4  /* a particle has more neighbours than max_neibs (list truncated) */
#define SPH_ERR_OUT_OF_DOMAIN  -5  /* uploaded particle outside its scene's domain */
#define SPH_ERR_NONFINITE      -6  /* non-finite value in the uploaded or integrated state */
#define SPH_ERR_TIMEOUT        -7  /* a bounded device wait gave up */
#define SPH_ERR_STATE          -8  /* call out of order (e.g. step before upload) */
#define SPH_ERR_SKIN           -9  /* a particle moved more than skin/2 since the last list build */
#define SPH_ERR_BOUNDS        -10  /* checked build only: an index out of range or a buffer's canary tail
                                      overwritten (the access was skipped) */

/* device error word bits (sph_stats.error_bits) */
#define SPH_EBIT_NEIB_OVERFLOW  1u
#define SPH_EBIT_NONFINITE      2u
#define SPH_EBIT_TIMEOUT        4u
#define SPH_EBIT_SKIN           8u
#define SPH_EBIT_BOUNDS        16u  /* checked build (compiled with SPH_CHECKED) */

/* viscosity models (paper Table 1 "viscous model", Sections 2.1 and 3).  The laminar models
 * use the neighbour weight omega_ij = m_j/(rho_i rho_j) and mubar_ij, the average (visc_avg)
 * of the dynamic viscosities rho nu of i and j: */
#define SPH_VISC_ARTIFICIAL     0  /* Monaghan artificial viscosity Pi_ij inside the pressure bracket */
#define SPH_VISC_LAMINAR        1  /* Morris: sum_j omega 2 mubar F u_ij */
#define SPH_VISC_MORRIS         1
#define SPH_VISC_MONAGHAN       2  /* K sum_j omega 2 mubar F (x.u/x.x) x_ij, K = 5 (3D) */
#define SPH_VISC_ESPANOL_REVENGA 3 /* sum_j omega F ((5/3 mubar - zetabar) u_ij
                                      + 5 (mubar/3 + zetabar)(x.u/x.x) x_ij), zeta = bulk */

/* smoothing kernels (Table 1; kernel-templates listing of Section 4), 3D, normalised to
 * unit integral; F = (1/r) dW/dr */
#define SPH_KERNEL_WENDLAND     0  /* (2q+1)(1-q/2)^4, support 2h */
#define SPH_KERNEL_CUBIC_SPLINE 1  /* 1 - 3/2 q^2 + 3/4 q^3 (q<1), (2-q)^3/4 (q<2) */
#define SPH_KERNEL_QUADRATIC    2  /* (2-q)^2, support 2h */
#define SPH_KERNEL_GAUSSIAN     3  /* exp(-q^2) - exp(-Q^2), cut at Q = kernel_radius */

/* SPH formulations (Section 2.1) */
#define SPH_FORM_1              0  /* drho_i = sum m_j u_ij.x_ij F; P_i/rho_i^2 + P_j/rho_j^2 */
#define SPH_FORM_2              1  /* drho_i = sum (rho_i/rho_j) m_j u_ij.x_ij F; (P_i+P_j)/(rho_i rho_j) */

/* averaging operator of the laminar viscosity (Table 1) */
#define SPH_AVG_HARMONIC        0
#define SPH_AVG_ARITHMETIC      1
#define SPH_AVG_GEOMETRIC       2

/* density diffusion (Table 1) */
#define SPH_DDIFF_NONE          0
#define SPH_DDIFF_MOLTENI       1  /* Molteni & Colagrossi: + 2 xi h c0 sum_j (rho_i - rho_j) F_ij m_j/rho_j
                                      over fluid neighbours of fluid particles */

/* particle types (paper Section 4, split neighbour list: fluid and boundary) */
#define SPH_FLUID               0
#define SPH_BOUNDARY            1  /* dynamic boundary particle: fixed, continuity + EOS only */

typedef struct sph_ctx sph_ctx;  /* opaque; owned by the library */

/* Run parameters, copied by sph_create.  All lengths in metres, SI units. */
typedef struct {
    double   dp;             /* particle spacing (informative) */
    double   h;              /* smoothing length */
    double   kernel_radius;  /* influence radius = kernel_radius*h; Wendland C2 needs 2 */
    double   rho0;           /* rest density */
    double   c0;             /* sound speed of scene 0 (per-scene values: sph_set_scenes) */
    double   gamma;          /* EOS exponent: an integer in [1, 8] */
    int32_t  visc_model;     /* SPH_VISC_* */
    int32_t  pad0;
    double   alpha;          /* artificial-viscosity coefficient */
    double   nu;             /* kinematic viscosity (laminar) */
    double   g[3];           /* body force per unit mass on fluid particles */
    double   cfl;            /* CFL factor of the adaptive time step: dt = min(cfl*min(sqrt(h/|a|max), h/c0),
                                0.125 h^2/nu [laminar models]) */
    double   dt_fixed;       /* > 0: constant time step; <= 0: adaptive (CFL) */
    double   origin[3];      /* domain of scene 0 */
    double   size[3];
    uint32_t periodic_mask;  /* bit0 x, bit1 y, bit2 z; a periodic axis needs >= 3 cells */
    uint32_t max_particles;  /* capacity, <= 2^26 */
    uint32_t max_neibs;      /* neighbour-list slots per particle, 8..1024 */
    uint32_t n_scenes;       /* 1, or the number of scenes given to sph_set_scenes */
    uint32_t rebuild_every;  /* 0 or 1: neighbour pipeline every step.  k > 1: list radius enlarged
                                by `skin` (paper Section 7: GPUSPH rebuilds every 10 steps with an
                                enlarged radius); the device runs the pipeline when a particle has
                                moved skin/4 since the last build, or after k steps, so the list
                                covers every pair within the influence radius (a displacement past
                                skin/2 is reported: SPH_ERR_SKIN).  Not with sph_record. */
    uint32_t pad1;
    double   skin;           /* added to the list radius when rebuild_every > 1 (>= 0) */
    /* model options (Table 1); all zero = Wendland C2, formulation 1, harmonic mean, no
     * density diffusion.  Other choices run the general interaction kernels; sph_record
     * (the adjoint) takes only the all-zero options with SPH_VISC_ARTIFICIAL or _LAMINAR. */
    int32_t  kernel_type;    /* SPH_KERNEL_* (the Gaussian is cut at kernel_radius*h) */
    int32_t  formulation;    /* SPH_FORM_* */
    int32_t  visc_avg;       /* SPH_AVG_*, laminar models only */
    int32_t  ddiff;          /* SPH_DDIFF_* */
    double   ddiff_coef;     /* density-diffusion coefficient xi (>= 0) */
    double   zeta;           /* kinematic bulk viscosity, SPH_VISC_ESPANOL_REVENGA (>= 0) */
} sph_params;

/* One independent scene of a batch: its own domain, grid and sound speed. */
typedef struct {
    double   origin[3];
    double   size[3];
    uint32_t periodic_mask;
    uint32_t pad0;
    double   c0;
} sph_scene;

/* Counters read back from the device (sph_get_stats synchronises). */
typedef struct {
    uint32_t n_active;        /* particles in the domain (after the last sort) */
    uint32_t n_removed;       /* particles dropped because they left the domain (cumulative) */
    uint32_t max_neibs_seen;  /* largest neighbour count found by the last build (before truncation) */
    uint32_t error_bits;      /* SPH_EBIT_* (sticky) */
    uint64_t steps;           /* steps taken since upload */
    double   dt;              /* time step of scene 0 for the next step */
    double   time;            /* simulated time of scene 0 */
    uint32_t n_cells;         /* cells over all scenes */
    uint32_t kernels_per_step;/* kernel launches in one captured step (0 before the first step) */
    uint64_t list_entries;    /* neighbour-list entries written by all builds since upload;
                                 each step's two force passes read its build's entries twice */
    uint64_t interactions;    /* pairs within the influence radius evaluated by the first force
                                 pass of each step since upload, counted when rebuild_every > 1 */
    uint32_t builds;          /* neighbour-list builds run by the upload and the steps since upload
                                 (one per step when rebuild_every <= 1) */
    uint32_t pad;
} sph_stats;

/* Create a context on the current CUDA device and allocate every device
 * buffer for p->max_particles particles.  The grid of scene 0 comes from
 * p->origin/size/periodic_mask with cell side size/floor(size/(kernel_radius*h))
 * (>= the influence radius, paper Section 2.3).  Returns SPH_ERR_ARG for
 * invalid physics or sizes, SPH_ERR_CUDA if allocation fails; *out is set
 * only on success. */
int sph_create(const sph_params* p, sph_ctx** out);

/* Replace the scene table by n_scenes independent scenes (batched stepping).
 * Must precede sph_upload; reallocates the cell tables (host call, syncs).
 * Each scene keeps its own grid, sound speed, dt and time; scenes never
 * interact. */
int sph_set_scenes(sph_ctx* ctx, uint32_t n_scenes, const sph_scene* scenes);

/* Upload n particles from HOST arrays (copied):
 *   pos   n*3 FP64 absolute positions (converted on the device to a cell index
 *         plus an FP32 offset from the cell centre, paper Section 2.3),
 *   vel   n*3 FP32 (ignored, i.e. zero, for boundary particles),
 *   delta n   FP32 relative density rho/rho0 - 1,
 *   mass  n   FP32 (> 0),
 *   type  n   SPH_FLUID / SPH_BOUNDARY,
 *   scene n   scene index, or NULL for all-zero.
 * Particle i keeps id i for sph_download.  Sorts the particles and resets
 * step count, time and dt (the first sph_step computes dt0 from one forces
 * call).  Errors: SPH_ERR_CAPACITY (n > max_particles), SPH_ERR_ARG (bad
 * type/scene/mass), SPH_ERR_OUT_OF_DOMAIN (a position outside its scene's
 * domain on a non-periodic axis), SPH_ERR_NONFINITE.  Synchronises `stream`. */
int sph_upload(sph_ctx* ctx, uint32_t n, const double* pos, const float* vel, const float* delta,
               const float* mass, const uint8_t* type, const uint32_t* scene, void* stream);

/* Same as sph_upload with DEVICE arrays of the same layouts. */
int sph_upload_device(sph_ctx* ctx, uint32_t n, const double* pos_dev, const float* vel_dev,
                      const float* delta_dev, const float* mass_dev, const uint8_t* type_dev,
                      const uint32_t* scene_dev, void* stream);

/* Neighbour pipeline on the current state: cell hash, key sort by (cell,
 * type, id), reorder, cell start/end, split neighbour list (paper
 * Sections 2.3 and 4: fixed-size, neighbour-major in chunks of two entries,
 * fluid neighbours from the front and boundary neighbours from the back;
 * sph_download_neighbors returns it by upload id). */
int sph_build_neighbors(sph_ctx* ctx, void* stream);

/* Particle interactions on the current state with the current neighbour
 * list (paper Section 2.1): acceleration and density rate of every
 * particle into the library's force buffer (read with sph_download_forces). */
int sph_forces(sph_ctx* ctx, void* stream);

/* nsteps predictor-corrector steps, each: neighbour pipeline, forces at n,
 * predictor (dt/2), forces at the predicted state, corrector (dt), CFL dt
 * for the next step.  Paper: Section 2.1 (the method), Section 3 "Code
 * structure" (the integrator runs forces and euler twice per step, the
 * first stage over dt/2, the second over dt) and Section 3 "The GPU in
 * GPUSPH" (the time step is a minimum over particles by parallel reduction);
 * the update formulas are reading C6, the dt formula reading C7 (not
 * printed in the paper).  Replays a captured CUDA graph per step: no host
 * round trip, the counters GPUSPH downloads every step stay on the device
 * until sph_get_stats.  Errors: SPH_ERR_STATE before an upload,
 * SPH_ERR_CUDA on a launch failure; device-found errors are sticky (see
 * Conventions). */
int sph_step(sph_ctx* ctx, uint32_t nsteps, void* stream);

/* Domain decomposition support (paper Section "Multi-GPU": each device holds
 * its own particles plus copies of the neighbouring devices' particles near the
 * boundary, the "halo").  Particles uploaded with an id >= n_owned are halo
 * copies: they interact and are integrated like the others, but their forces
 * are incomplete (their own neighbours beyond the halo are missing), so they
 * are left out of the CFL time-step reduction.  UINT32_MAX (the default): no
 * halo.  Synchronises the device. */
int sph_set_owned(sph_ctx* ctx, uint32_t n_owned);

/* Take dt (> 0, finite; else SPH_ERR_ARG) as the time step of the next step
 * of every scene instead of the step's own CFL value (reading C7): a
 * decomposed run agrees on one dt, the minimum of the devices' proposals
 * (paper Section "The GPU in GPUSPH": the time step is a minimum over all
 * particles, downloaded to the host).  Later steps return to their own CFL
 * value.  Synchronises the device. */
int sph_set_dt(sph_ctx* ctx, double dt);

/* The CFL time step of the current state (reading C7, halo copies left out):
 * one forces-only pass with its |a| reduction, without a step; scene 0's value
 * into *dt (HOST).  For the first step of a decomposed run, whose dt is the
 * minimum of every device's value before any step.  The step count and time
 * are unchanged.  Synchronises `stream`. */
int sph_cfl_dt(sph_ctx* ctx, double* dt, void* stream);

/* The CFL time step the next step of scene 0 would take (reading C7: from the
 * corrector-stage accelerations of the last step, halo copies left out),
 * into *dt (HOST), without changing any state: a decomposed run reduces these
 * proposals to their minimum and passes it to sph_set_dt.  Synchronises
 * `stream`; SPH_ERR_STATE before an upload. */
int sph_next_dt(sph_ctx* ctx, double* dt, void* stream);

/* Run the neighbour-list build and the predictor pass as one kernel (on != 0)
 * or as two (0): each thread writes its particle's list (the thread-per-
 * particle build) and evaluates the predictor pass over it at once, while
 * the list and the candidates it has just tested are in cache.  The same list
 * and the same results, to the bit.  sph_autotune fuses them when that is at
 * least 2% faster.  Only with the list rebuilt every step and the default model
 * (SPH_ERR_ARG otherwise); the paper runs the two as separate commands
 * (Section 3 "Code structure").  Synchronises the device. */
int sph_set_fused_predict(sph_ctx* ctx, int on);

/* The step options in use (outputs nullable): the fused build + predictor
 * kernel (sph_set_fused_predict) and the persistent step kernel
 * (sph_set_persistent). */
int sph_get_step_options(sph_ctx* ctx, int* fused_predict, int* persistent);

/* Step all scenes with one persistent kernel instead of the captured graph of
 * per-phase kernels (on != 0), or back (0).  The persistent kernel runs every
 * phase of the step (dt, hash, scan, scatter, reorder, list build, predictor
 * pass, corrector pass) over all scenes' particles, with a grid-wide barrier
 * between phases, for all the steps of one sph_step call: one cooperative
 * launch (every block resident, so every barrier completes; it is launched as
 * such each time, not replayed from a captured graph).  Same arithmetic as
 * the graph path: the same results, to the bit.  Batching of independent scenes is not in the paper (its GPU
 * section runs one scene per device); this is the single-launch form of the
 * batched step.  Only with the list rebuilt every step and the default model
 * (SPH_ERR_ARG otherwise).  Synchronises the device. */
int sph_set_persistent(sph_ctx* ctx, int on);

/* ---- differentiable run (reverse mode) --------------------------------
 * Loss L on the state after T steps; gradients w.r.t. the initial state and
 * the artificial-viscosity coefficient alpha.  The paper has no adjoint; it
 * differentiates the step of Section 2.1 with readings C1-C7 as implemented
 * here, with dt frozen (no gradient through dt) and the neighbour list of
 * each step held fixed within the step (F and F' vanish at the cutoff, so
 * the step map is C1 across list changes). */

/* Set alpha (artificial viscosity only; SPH_ERR_ARG otherwise).  Host call,
 * synchronises the device; invalidates a recording. */
int sph_set_alpha(sph_ctx* ctx, double alpha);

/* Forward of a differentiable run: T predictor-corrector steps from the
 * uploaded state with dt frozen at params.dt_fixed, or (if that is <= 0) at
 * the CFL dt of one forces call on the initial state (*dt_out, nullable),
 * storing a checkpoint of the state every K steps (T % K == 0).  One scene
 * only.  Allocates its checkpoints and tape: 48 B per particle per
 * checkpoint, and per step of one segment 80 B per particle of states plus
 * a neighbour-list slot (8 * (max_neibs/2 + 1) + 4 B per particle), where
 * sph_backward keeps each recomputed step's list for its reversal.  Afterwards
 * the context holds the state after T steps.  Synchronises `stream`. */
int sph_record(sph_ctx* ctx, uint32_t T, uint32_t K, void* stream, double* dt_out);

/* Reverse of the last sph_record.  Inputs: DEVICE arrays in upload order
 * with the adjoints of the final state, dL/dx_T (n*3), dL/du_T (n*3),
 * dL/ddelta_T (n); any may be NULL (zero).  Outputs: DEVICE arrays dL/dx_0,
 * dL/du_0 (n*3), dL/ddelta_0 (n), nullable; *alphabar (host, nullable) =
 * dL/dalpha.  Boundary particles' x and u are constants (zero adjoint).
 * Each segment of K steps is recomputed from its checkpoint and reversed
 * step by step; the vector-Jacobian products are gathers over the
 * symmetric neighbour lists (deterministic, no atomics).  Leaves the
 * context at the recorded initial state.  Synchronises `stream`. */
int sph_backward(sph_ctx* ctx, const float* xbar_T, const float* ubar_T, const float* dbar_T, float* xbar_0,
                 float* ubar_0, float* dbar_0, double* alphabar, void* stream);

/* Generation of the recording sph_backward would reverse: every successful
 * sph_record numbers its tape 1, 2, 3, ... per context; *gen = 0 when no
 * valid recording exists (none yet, a failed sph_record, sph_set_alpha).
 * A caller that holds several recordings' results (e.g. an autograd graph
 * with two rollouts on one context) stores the generation after its
 * sph_record and checks it before sph_backward: a mismatch means the tape
 * now belongs to a later recording.  The paper has no counterpart.  Host
 * call, no synchronisation; SPH_ERR_ARG for a null argument. */
int sph_tape_generation(sph_ctx* ctx, uint64_t* gen);

/* Autotuner (launch shapes only; results are unchanged): times each
 * neighbour-build variant (one thread per particle with 128 or 256 threads
 * per block, or one warp per cell with 2, 4 or 8 cells per block) and each
 * force-kernel shape (64, 128 or 256 threads per block with at most 64
 * registers; 128 threads with at most 85 or 128) on the uploaded state, the
 * predictor and the corrector pass apart (3 timed launches each, CUDA events
 * on `stream`; the corrector runs on a scratch copy of the state), then the
 * list build and the predictor pass fused against apart (every-step list,
 * default model), keeps the fastest and re-captures the step graph on the
 * next sph_step.  The
 * particle state and the next time step are as before the call (the list
 * counters include the timed builds).  Outputs (nullable): the build
 * variant and the predictor pass's shape (names: sph_build_variant_name,
 * sph_forces_variant_name; sph_get_variants gives the corrector's too).
 * Synchronises `stream`; SPH_ERR_STATE before an upload. */
int sph_autotune(sph_ctx* ctx, void* stream, int* build_variant, int* forces_variant);

/* Select the neighbour-build variant (0..4) and the force-kernel launch shape
 * (0..4, for every pass) directly, as sph_autotune would (-1 keeps the
 * current one).  Every variant computes the same bits.  Synchronises the
 * device; SPH_ERR_ARG for an index out of range. */
int sph_set_variants(sph_ctx* ctx, int build_variant, int forces_variant);

/* The force-kernel launch shapes (0..4) of the forces-only and predictor
 * passes and of the corrector pass, set apart (-1 keeps one).  sph_autotune
 * picks them apart too: the fastest shape of the two passes can differ.
 * Synchronises the device; SPH_ERR_ARG for an index out of range. */
int sph_set_forces_variants(sph_ctx* ctx, int forces_predict, int forces_correct);

/* The variants in use: build, predictor-pass shape, corrector-pass shape
 * (outputs nullable). */
int sph_get_variants(sph_ctx* ctx, int* build_variant, int* forces_predict, int* forces_correct);

/* Names of the variants of sph_autotune (static storage). */
const char* sph_build_variant_name(int variant);
const char* sph_forces_variant_name(int variant);

/* Same work as sph_step, launched kernel by kernel (no graph) with CUDA
 * events recorded on `stream` between the launches; adds the elapsed
 * milliseconds of each phase to phase_ms[0..7]: 0 dt, 1 hash, 2 scan,
 * 3 scatter, 4 in-cell sort + reorder, 5 neighbour-list build (with the
 * predictor pass when they are fused, see sph_set_fused_predict),
 * 6 forces + predictor (0 when fused), 7 forces + corrector.  Synchronises after each
 * step (measurement aid; sph_step is the production path). */
int sph_step_profiled(sph_ctx* ctx, uint32_t nsteps, void* stream, double* phase_ms);

/* Download the state in upload order into HOST arrays (any may be NULL):
 * pos n*3 FP64, vel n*3 FP32, delta n FP32.  Paper: Section 3 "The GPU in
 * GPUSPH" (particle data is downloaded to the host only at fixed simulated
 * time intervals, with the simulation suspended meanwhile): a host call
 * between steps, never inside one.  Particles removed from the domain read
 * as NaN.  n must equal the uploaded count (else SPH_ERR_ARG).
 * Synchronises `stream`; returns the sticky device error as sph_get_stats
 * does. */
int sph_download(sph_ctx* ctx, uint32_t n, double* pos, float* vel, float* delta, void* stream);

/* Same as sph_download into DEVICE arrays (no host synchronisation). */
int sph_download_device(sph_ctx* ctx, uint32_t n, double* pos_dev, float* vel_dev,
                        float* delta_dev, void* stream);

/* Download the last sph_forces result in upload order: acc n*3, drho n
 * (FP32, density rate d rho/dt).  HOST arrays; synchronises. */
int sph_download_forces(sph_ctx* ctx, uint32_t n, float* acc, float* drho, void* stream);

/* Download the neighbour lists in upload order (for checking): counts
 * n*2 (fluid, boundary neighbours written), ids n*max_neibs upload ids of
 * the neighbours, fluid first then boundary, unused slots 0xFFFFFFFF.
 * HOST arrays; synchronises. */
int sph_download_neighbors(sph_ctx* ctx, uint32_t n, uint32_t* counts, uint32_t* ids, void* stream);

/* The neighbour lists of m sampled particles, by upload id: sample[0..m) (HOST)
 * upload ids; counts m*2 (fluid, boundary neighbours of sample[k]), ids
 * m*max_neibs upload ids in the layout of sph_download_neighbors, row k for
 * sample[k] (HOST outputs).  For checking a few lists of a state too large to
 * download whole.  Allocates per-call device staging (4 B per uploaded
 * particle plus the outputs) and frees it; SPH_ERR_ARG for an id out of
 * range (the other rows are still written).  Synchronises `stream`. */
int sph_download_neighbors_of(sph_ctx* ctx, uint32_t m, const uint32_t* sample, uint32_t* counts, uint32_t* ids,
                              void* stream);

/* Same result as sph_download_neighbors, without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * must not call cudaMalloc/cudaFree while they run, e.g. a process whose
 * device memory is already held by another allocator (a framework's caching
 * allocator), or a loop that cannot afford the device-wide synchronisation
 * cudaMalloc and cudaFree may cause.  The device staging sph_download_neighbors
 * allocates per call lives here in one fixed device array of 24 MiB that
 * every GPU loading the library holds until the process exits.
 * Limits: n <= 2^20 particles and n * max_neibs <= 2^22 entries, else
 * SPH_ERR_CAPACITY (nothing is done).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (this call clears what it reads
 * back), so calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.  The current device must be the
 * context's device (else SPH_ERR_STATE).  HOST output arrays as in
 * sph_download_neighbors; synchronises `stream`. */
int sph_download_neighbors_noalloc(sph_ctx* ctx, uint32_t n, uint32_t* counts, uint32_t* ids, void* stream);

/* Conservation sums at the current state (paper Section 2.1 invariants), from one
 * forces-only pass (its results also land where sph_download_forces reads them):
 *   out[0..2] momentum sum_i m_i u_i (fluid),  out[3..5] force sum_i m_i a_i,
 *   out[6] sum_i m_i drho_i/dt,  out[7] kinetic energy sum_i m_i |u_i|^2 / 2,
 *   out[8] total mass sum_i m_i (particles in the domain),
 * masses taken positive.  With no boundary particles and no gravity the pair forces
 * cancel: out[3..5] vanish to rounding.  FP64 sums in a fixed order (bitwise
 * reproducible).  HOST out[9]; synchronises `stream`; returns the sticky device
 * error as sph_get_stats does. */
int sph_conservation(sph_ctx* ctx, double* out, void* stream);

/* Read device counters into *out (synchronises `stream`).  Paper: Section 3
 * "The GPU in GPUSPH" (the only data that returns to the host between
 * steps: the particle count after the sort, which shows removed particles,
 * the largest neighbour count of the list build, which shows an overflow,
 * and the time step of the reduction).  Returns the sticky device error as
 * a code (SPH_ERR_NEIB_OVERFLOW, SPH_ERR_NONFINITE, SPH_ERR_SKIN,
 * SPH_ERR_TIMEOUT) if one is set, else SPH_OK; *out is filled either way.
 * SPH_ERR_ARG for a null context or output. */
int sph_get_stats(sph_ctx* ctx, sph_stats* out, void* stream);

/* Per-scene dt and simulated time (n_scenes entries each, HOST, nullable). */
int sph_get_scene_times(sph_ctx* ctx, double* dt, double* time, void* stream);

/* Clear the sticky device error word. */
int sph_clear_error(sph_ctx* ctx, void* stream);

/* Wait for the stream and return the sticky device error (as sph_get_stats). */
int sph_sync(sph_ctx* ctx, void* stream);

/* FP32 CUDA-core throughput of the current device in TFLOP/s (FMA = 2 flops),
 * measured with a kernel of independent FMA chains on every SM (best of 5
 * timed launches on `stream`, synchronises it).  The ALU roof against which
 * the interaction kernels are reported; the paper has no counterpart.
 * Returns SPH_ERR_ARG for a null output, SPH_ERR_CUDA on a CUDA failure. */
int sph_fp32_peak(void* stream, double* tflops);

/* Human-readable text of a return code (static storage). */
const char* sph_strerror(int code);

/* Free every buffer of the context (synchronises the device).  Paper:
 * Section 3 "The GPU in GPUSPH" (arrays are allocated once, at
 * initialisation, and never reallocated while the simulation runs): the
 * buffers sph_create allocated live until this call; apart from them only
 * sph_set_scenes (the cell tables of a new scene table), sph_record (its
 * tape) and sph_download_neighbors (per-call staging) allocate device
 * memory.  A null context is ignored.  The context must not be used
 * afterwards; work still queued on its streams is waited for first. */
void sph_destroy(sph_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */
