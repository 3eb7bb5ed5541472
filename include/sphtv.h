/*
 * sphtv.h -- C ABI of libsphtv, a single-GPU (sm_103a) library for one
 * kick-drift-kick step of weakly-compressible SPH with the limited,
 * h^2-scaled transport-velocity correction of Wang, Haidn & Hu, "The
 * efficient implementation of transport velocity formulation"
 * (arXiv 2411.13992).
 *
 * What one step computes (paper sections / equations):
 *   1. half kick  v += dt/2 a;  drift  x += dt v + dr  (kick-drift-kick,
 *      Sec. 1 and Sec. 3; dr is the transport-velocity displacement of the
 *      previous step, applied once per step, Sec. 3);
 *   2. cell-linked list: particles counting-sorted by cell index, ties broken
 *      by particle id, so the order is deterministic;
 *   3. density summation rho_i = rho0 sum_j W_ij / sigma0_i (Eq. 8) with the
 *      equation of state p = c^2 (rho - rho0) (Eq. 2), Wendland C2 kernel
 *      with support 2h (Sec. 4);
 *   4. one fused pair pass: Riemann pressure force with the dissipation
 *      limiter (Eq. 3 second row, Eq. 5-6), viscous force (Eq. 7), the
 *      residual R_i = sum_j V_j grad_i W_ij and the limited displacement
 *      dr_i = xi chi_i h^2 R_i (Eq. 14-16);
 *   5. closing half kick, FP64 diagnostics and the next step size
 *      min(dt_ad, dt_ac) (Eq. 9-11, h = h_min).
 * The dual-criteria integrator of Sec. 2.4 (SPH_INT_DUAL) is the other
 * choice: one advection step with the density reinitialisation and the
 * correction, then acoustic substeps with the Riemann continuity equation.
 *
 * Conventions.
 *   - Vectors crossing the ABI are row-major [n][3] doubles (x, y, z per
 *     particle; z is ignored in 2-D).  Scalars are [n] arrays.
 *   - Every pointer argument may be host or device memory (the library
 *     copies with cudaMemcpyKind Default); host memory should be pinned for
 *     asynchronous transfers.  Arrays passed in are read during the call's
 *     stream work only; the library keeps its own copy in the workspace.
 *   - Results are always returned in the particle order given to
 *     sph_set_state, whatever the internal (cell-sorted) order is.
 *   - The caller owns the device workspace and the stream.  The library
 *     allocates no device memory: it carves every buffer out of the
 *     workspace given to sph_create, whose size sph_query_workspace reports.
 *     The context itself is a small host object.
 *   - All calls enqueue work on the context's stream and return without
 *     waiting, except sph_sync, sph_get_diag, and sph_get_state /
 *     sph_step_adjoint when they write to host memory.
 *   - Every call returns a status.  Host-detectable errors (bad arguments,
 *     call order, workspace too small, CUDA launch errors) return at once.
 *     Device-detected errors (cell overflow, non-finite values, particle
 *     outside a non-periodic box, h outside [h_min, h_max]) set a sticky
 *     error word that sph_sync returns.  Nothing is thrown across the ABI; no call traps the GPU.
 */
#ifndef SPHTV_H
#define SPHTV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPH_API __attribute__((visibility("default")))
#else
#define SPH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sph_status {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,        /* invalid argument (host check) */
    SPH_ERR_CUDA = 2,       /* a CUDA call failed */
    SPH_ERR_WORKSPACE = 3,  /* workspace NULL, misaligned or too small */
    SPH_ERR_OVERFLOW = 4,   /* device: a cell held more particles than supported, or (SPH_INT_DUAL)
                               a particle had more neighbours than its frozen list holds
                               (128 in 3-D, 96 in 2-D) */
    SPH_ERR_NAN = 5,        /* device: non-finite position or velocity */
    SPH_ERR_DOMAIN = 6,     /* device: particle left a non-periodic box */
    SPH_ERR_STATE = 7,      /* call order: e.g. sph_step before sph_build_cells */
    SPH_ERR_INPUT = 8       /* device: a particle's h outside [h_min, h_max] or mass not positive */
} sph_status;

enum { SPH_TV_OFF = 0, SPH_TV_LIMITED = 1, SPH_TV_UNLIMITED = 2, SPH_TV_BACKGROUND = 3 };
enum { SPH_TVH_MIN = 0, SPH_TVH_PARTICLE = 1 };
enum { SPH_HPAIR_MEAN = 0, SPH_HPAIR_MAX = 1 };
/* Time integrators. */
enum {
    SPH_INT_KDK = 0,    /* single-rate kick-drift-kick, dt = min(dt_ad, dt_ac), the
                           correction applied in every drift (Sec. 1, Sec. 3) */
    SPH_INT_DUAL = 1    /* dual-criteria time stepping (Sec. 2.4): one sph_step is one
                           advection step Dt_ad (Eq. 9-10) -- cell list rebuilt and its
                           neighbour set frozen for the step, density reinitialised by
                           summation (Eq. 8), viscous force (Eq. 7) held, transport
                           correction (Eq. 14-16; Eq. 12 with p0 = 7 rho0 |v|_ad^2 of
                           Eq. 13) added to the positions once -- followed by acoustic
                           substeps dt = min(dt_ac, Dt_ad - t) (Eq. 11) of drift dt/2,
                           kick with the Riemann pressure force (Eq. 3 row 2, Eq. 5-6),
                           drift dt/2, and the Riemann continuity equation (Eq. 3 row 1,
                           U* of Eq. 5 row 1) integrating the density by halves */
};

/* Plain-data parameter block.  sph_default_params fills the paper's
 * constants; the caller sets the domain and the fluid. */
typedef struct sph_params {
    int32_t dim;            /* 2 or 3 */
    int32_t precision;      /* 64: FP64 throughout; 32: FP32 pair sums with
                               Kahan compensation, FP32 cell-relative positions,
                               FP64 positions (each step's displacement in FP32,
                               accumulated in FP64) and FP64 reductions */
    int32_t periodic[3];    /* 1: periodic along that axis */
    int32_t tv_mode;        /* SPH_TV_*: none / limited (Eq. 16) / unlimited (Eq. 14) /
                               background pressure p0 = rho0 c^2 (Eq. 12): the drift
                               adds dt^2/2 a_bg, a_bg = -2 sum_j m_j p0/(rho_i rho_j) grad W_ij,
                               with the dt of the step that computed it */
    double lo[3];           /* domain lower corner */
    double L[3];            /* domain lengths; every particle must stay in
                               [lo, lo+L] along non-periodic axes */
    double rho0;            /* reference density (Eq. 2, 8) */
    double c0;              /* artificial sound speed c (Eq. 2) */
    double eta;             /* dynamic viscosity (Eq. 7) */
    double g[3];            /* body force per unit mass */
    double h_min;           /* minimum smoothing length (Eq. 9-11, 15-16) */
    double h_max;           /* maximum smoothing length: sets the cell edge >= h_max */
    double riemann_eta;     /* dissipation limiter slope, 3 (Eq. 6) */
    double tv_xi;           /* -0.2 (Eq. 14, 16) */
    double tv_C;            /* 1e3 (Eq. 15) */
    double tv_thresh;       /* 5e-4 (Eq. 15) */
    double cfl_ad;          /* 0.25 (Eq. 9) */
    double cfl_ac;          /* 0.6 (Eq. 11) */
    double u_ref;           /* reference velocity U_ref (Eq. 10) */
    double fixed_dt;        /* > 0: every step uses this dt; 0: Eq. 9-11 */
    int32_t tv_h;           /* SPH_TVH_*: h in Eq. 14-16 is h_min (paper) or h_i */
    int32_t h_pair;         /* SPH_HPAIR_*: h_ij = (h_i+h_j)/2 (default) or max */
    int32_t kahan;          /* FP32 form: 1 = compensated pair sums (default) */
    int32_t adjoint_steps;  /* longest segment sph_step_adjoint will replay
                               (0: no adjoint buffers in the workspace; must be 0
                               with SPH_INT_DUAL); each step of it takes a tape
                               slot in the workspace, which in the FP32 form also
                               holds that step's neighbour list (128 entries per
                               particle in 3-D, 96 in 2-D, 4 bytes each) */
    int32_t integrator;     /* SPH_INT_*: kick-drift-kick (default) or dual-criteria;
                               SPH_INT_DUAL requires fixed_dt = 0 */
    int32_t graphs;         /* 1 (default): sph_step replays kick-drift-kick steps two at a
                               time from a captured CUDA graph on a library-owned stream,
                               ordered after and before the context's stream by events
                               (same results, fewer launches); 0: always launch directly */
    int32_t pair_tiles;     /* FP32 form at uniform resolution (h_min == h_max), the density
                               pass: 0 (default, the fastest measured) walks the cell rows in
                               global memory, one thread per particle; 1 stages a block of cells
                               and the two cells around it in shared memory per thread block
                               and walks that tile, one thread per particle (the same results as
                               0 bit for bit); 2 walks the tile with groups of lanes sharing each
                               particle's candidates (the same neighbour lists, sigma summed in
                               another order); 3 walks the tile with each thread's cell rows taken
                               as one sequence (the same results as 0 bit for bit).  The tiles
                               hold whole cells: with x_subcells > 1, 1 and 3 visit the row walk's
                               pairs in its order plus the candidates of the sub-cells that its
                               cut drops, whose zero terms enter the compensated sums, so their
                               results equal 0's bit for bit only with x_subcells = 1.  Ignored
                               otherwise */
    int32_t body_force;     /* 1: the force pass also sums the force of the fluid on the wall
                               particles (the body force of Eq. 18, e.g. the cylinder of
                               Sec. 4.4), reported in sph_diag.body_force; 0 (default): not */
    double fringe_lambda;   /* free stream in a periodic box (Sec. 4.4 names a free-stream
                               boundary without giving it): the fringe-region forcing of
                               Nordstrom, Nordin & Henningson (SIAM J. Sci. Comput. 20, 1999)
                               adds lambda(x) (fringe_u - v) to the acceleration of fluid
                               particles, lambda(x) = fringe_lambda [S((x - x0)/rise)
                               - S((x - x1)/fall + 1)] along axis 0, S(t) = 1/(1 + exp(1/(t-1)
                               + 1/t)) on (0, 1), 0 below, 1 above.  0 (default): off.
                               Kick-drift-kick only (SPH_ERR_ARG with SPH_INT_DUAL) */
    double fringe_u[3];     /* free-stream velocity U_inf */
    double fringe_x[4];     /* x0, x1, rise > 0, fall > 0 of the fringe region */
    int32_t x_subcells;     /* 1, 2 or 4 (default 4; 0 means 1): the counting sort refines each
                               cell along axis 0 into this many sub-cells (particles ordered by
                               sub-cell, then by id, within their cell), and the row walks of the
                               density passes cut each row's x extent at sub-cell instead of cell
                               granularity: fewer candidate tests for the same neighbours in the
                               same order (only the order of particles within a cell changes, and
                               with it the rounding of the sums).  Reduced to 2, then 1, where the
                               cells times the sub-cells would exceed 2^30.  SPH_ERR_ARG for other
                               values */
} sph_params;

/* FP64 diagnostics of the fluid particles after a step (or after
 * sph_build_cells). */
typedef struct sph_diag {
    double mass;            /* sum m */
    double momentum[3];     /* sum m v */
    double kinetic;         /* 1/2 sum m |v|^2 */
    double vmax;            /* max |v| */
    double vt_max;          /* max |v + dr/dt|: transport velocity (Sec. 3) */
    double dr_max;          /* max |dr| */
    double n_chi;           /* number of particles with chi > 0 (Eq. 15) */
    double dt;              /* step size used by the last step */
    double dt_next;         /* step size the next step will use */
    double steps;           /* steps taken since sph_build_cells */
    double substeps;        /* SPH_INT_DUAL: acoustic substeps of the last advection step */
    double body_force[3];   /* params.body_force: force of the fluid on the wall particles in
                               the last force pass (minus the fluid's momentum rate from its
                               pair terms, which cancel between fluid pairs): the F of the
                               drag and lift coefficients of Eq. 18, C = 2 F / (rho0 U^2 D) */
    double body_impulse[3]; /* kick-drift-kick with params.body_force: sum over the steps since
                               sph_build_cells of each step's body force times its dt (its
                               differences over an interval, divided by the interval's time,
                               give the force averaged over every step of it) */
    double time;            /* kick-drift-kick: simulated time since sph_build_cells (sum of dt) */
} sph_diag;

typedef struct sph_ctx sph_ctx;

/* Fill *p with the paper's constants: riemann_eta 3, tv_xi -0.2, tv_C 1e3,
 * tv_thresh 5e-4, cfl_ad 0.25, cfl_ac 0.6, tv_mode limited, tv_h h_min,
 * h_pair mean, kahan on, graphs on, pair_tiles 0, body_force off, no fringe forcing,
 * x_subcells 4,
 * precision 64, dim 2, rho0 1.  Returns
 * SPH_ERR_ARG on NULL. */
SPH_API sph_status sph_default_params(sph_params* p);

/* Bytes of device workspace a context for n particles needs, 1 <= n <= 2^25.
 * The cell grid follows from dim, lo, L, periodic and h_max: along each
 * axis floor(L / h_max) cells of edge >= h_max, so the neighbours of a
 * particle lie in the 5^D cells around its own (at least 5 cells along
 * periodic axes, else SPH_ERR_ARG).  The grid may have at most 2^20 cells
 * along an axis and 2^30 cells in all (else SPH_ERR_ARG, before anything is
 * sized or enqueued).  Returns SPH_ERR_ARG on invalid parameters. */
SPH_API sph_status sph_query_workspace(const sph_params* p, int64_t n, size_t* bytes);

/* Create a context on the current CUDA device.  workspace: device memory
 * of at least the queried size, 256-byte aligned, owned by the caller and
 * kept alive until sph_destroy.  stream: a cudaStream_t (NULL = legacy
 * default stream) on which every call of this context enqueues its work. */
SPH_API sph_status sph_create(const sph_params* p, int64_t n, void* workspace, size_t bytes, void* stream,
                      sph_ctx** out);

/* Load the particle state (Sec. 2; Eq. 8 reference sums).
 *   x  [n][3] positions (required)            v  [n][3] velocities (required)
 *   a  [n][3] accelerations or NULL           dr [n][3] displacements or NULL
 *   h  [n] smoothing lengths (required)       m  [n] masses (required)
 *   kind [n] int8: 0 fluid, 1 wall, or NULL (all fluid)
 *   vw [n][3] prescribed wall velocities or NULL (zero)
 *   sigma0 [n] reference sums of Eq. 8 or NULL: then sigma0_i is the
 *     perfect-lattice sum at spacing dp_i = (m_i/rho0)^(1/D) and h_i.
 * With a and dr NULL, sph_build_cells computes them from x and v (initial
 * force pass).  Velocities of walls are their prescribed velocities. */
SPH_API sph_status sph_set_state(sph_ctx* ctx, const double* x, const double* v, const double* a, const double* dr,
                         const double* h, const double* m, const int8_t* kind, const double* vw,
                         const double* sigma0);

/* Sort the loaded state into cells and run the density pass; when a/dr
 * were not given, also the force pass (a, dr from x and v).  Then compute
 * the diagnostics and the first dt (Eq. 9-11, or fixed_dt).  Kick-drift-kick
 * with a and dr given: only the diagnostics and the first dt, which need
 * neither cells nor densities; the first sph_step sorts the particles and
 * runs the density pass as every step does, and sph_get_state with rho
 * before any step sorts them and runs the density pass first. */
SPH_API sph_status sph_build_cells(sph_ctx* ctx);

/* Advance nsteps >= 0 steps on the context's stream: kick-drift-kick steps,
 * or with SPH_INT_DUAL advection steps, each with its acoustic substeps.  The
 * dual integrator decides on the device when an advection step is complete;
 * the host waits for the stream once per advection step to learn it. */
SPH_API sph_status sph_step(sph_ctx* ctx, int32_t nsteps);

/* SPH_INT_DUAL: set or read the density rate d rho/dt that the integrator
 * carries from one acoustic substep to the next and across advection steps
 * ([n] doubles, caller's particle order, walls 0).  sph_set_state sets it to
 * zero; call sph_set_density_rate after sph_set_state and before
 * sph_build_cells.  Reading waits for the copy when drho is host memory.
 * SPH_ERR_ARG with the kick-drift-kick integrator or a NULL pointer;
 * SPH_ERR_STATE before sph_set_state. */
SPH_API sph_status sph_set_density_rate(sph_ctx* ctx, const double* drho);
SPH_API sph_status sph_get_density_rate(sph_ctx* ctx, double* drho);

/* Override the step size of the next step (> 0). */
SPH_API sph_status sph_set_dt(sph_ctx* ctx, double dt);

/* Set the dynamic viscosity eta (>= 0, Eq. 7) used from the next launch on
 * (for example to evaluate a rollout at another viscosity). */
SPH_API sph_status sph_set_eta(sph_ctx* ctx, double eta);

/* Copy the state out in the caller's original particle order.  Any pointer
 * may be NULL.  x, v, a, dr: [n][3]; rho: [n] (walls report rho0).  Waits
 * for the copy when a destination is host memory. */
SPH_API sph_status sph_get_state(sph_ctx* ctx, double* x, double* v, double* a, double* dr, double* rho);

/* Wait for the stream and copy the diagnostics of the last step. */
SPH_API sph_status sph_get_diag(sph_ctx* ctx, sph_diag* out);

/* A checkpoint of the kick-drift-kick state after a step: what
 * sph_step_adjoint replays a segment from (its x0, v0, a0, dr0).  The four
 * arrays are the caller's ([n][3] doubles, caller's particle order, host or
 * device memory); the library writes them and the two scalars. */
typedef struct sph_ckpt {
    double* x;          /* positions */
    double* v;          /* velocities (walls: prescribed velocity) */
    double* a;          /* accelerations of the last force pass (Eq. 3, 7) */
    double* dr;         /* transport displacements the next drift adds (Eq. 16) */
    double dt_next;     /* step size the next step takes (Eq. 9-11, or fixed_dt) */
    double steps;       /* steps taken since sph_build_cells */
} sph_ckpt;

/* Save a checkpoint (the state as sph_get_state writes it, with the next
 * step size and the step count of sph_get_diag).  Waits for the stream.
 * SPH_ERR_ARG for a NULL context, checkpoint or array; SPH_ERR_STATE before
 * sph_build_cells. */
SPH_API sph_status sph_save_ckpt(sph_ctx* ctx, sph_ckpt* ck);

/* Wait for the context's stream; return the sticky device error word as a
 * status (SPH_OK if none), then clear it. */
SPH_API sph_status sph_sync(sph_ctx* ctx);

/* Destroy the host context (the workspace stays the caller's). */
SPH_API void sph_destroy(sph_ctx* ctx);

/* Static description of a status code. */
SPH_API const char* sph_status_str(sph_status s);

/* Number of kernel launches this context has enqueued since creation. */
SPH_API int64_t sph_launch_count(const sph_ctx* ctx);

/* Kernel classes of one step, for per-kernel timing. */
enum {
    SPH_K_KICKDRIFT = 0,   /* kick + drift + cell key + histogram */
    SPH_K_SCAN = 1,        /* exclusive scan of the cell counts */
    SPH_K_ORDER = 2,       /* scatter into cells + per-cell order by id */
    SPH_K_PERMUTE = 3,     /* permute the particle arrays */
    SPH_K_DENSITY = 4,     /* density summation (Eq. 8) */
    SPH_K_FORCES = 5,      /* fused pair pass (Eq. 3, 5-7, 14-16) + closing kick */
    SPH_K_FINALIZE = 6,    /* FP64 reductions and dt (Eq. 9-11) */
    SPH_K_ADVECT = 7,      /* SPH_INT_DUAL: viscous force + transport correction of an advection step */
    SPH_K_ACOUSTIC = 8,    /* SPH_INT_DUAL: all acoustic substeps of an advection step */
    SPH_K_NCLASS = 9
};

/* Per-kernel timing (tracing).  After sph_profile_begin, each of the next
 * max_steps steps records a CUDA event before and after every kernel class
 * on the context's stream (events are host-created driver objects; no device
 * memory is allocated).  sph_profile_end waits for the stream and writes,
 * per class, the summed elapsed milliseconds (ms[SPH_K_NCLASS]) and the
 * number of timed launches (count[SPH_K_NCLASS]); either may be NULL.
 * Returns SPH_ERR_STATE if no profile is open, SPH_ERR_ARG if max_steps < 1. */
SPH_API sph_status sph_profile_begin(sph_ctx* ctx, int32_t max_steps);
SPH_API sph_status sph_profile_end(sph_ctx* ctx, double* ms, int64_t* count);

/* Static name of a kernel class ("forces", ...), or "?" when out of range. */
SPH_API const char* sph_kernel_class_name(int32_t k);

/* Measurement aid (not in the paper): the fused multiply-add throughput of
 * this GPU, the denominator of the pair kernels' ALU roofline.  Enqueues on
 * `stream` one launch of `blocks` blocks x 256 threads; each thread runs
 * `iters` rounds of 8 independent FMA chains in the precision given (32:
 * float, 64: double) and writes one value to sink[thread] so that the work
 * is live.
 *   sink    device memory, blocks * 256 elements of float (32) or double (64)
 *   flops   host; receives the floating-point operations of the launch
 *           (blocks * 256 * iters * 8 FMAs, an FMA counting 2)
 * The caller times the launch with CUDA events on the same stream; the call
 * does not wait.  SPH_ERR_ARG for precision not 32 or 64, blocks < 1,
 * iters < 1 or a NULL pointer; SPH_ERR_CUDA if the launch fails. */
SPH_API sph_status sph_fma_peak(int32_t precision, int32_t blocks, int32_t iters, void* sink, void* stream,
                                double* flops);

/* Adjoint of a segment of nsteps steps (reverse mode), with every step's
 * neighbour set and step size frozen (not in the paper; the derivatives of
 * Eq. 2-8 and 14-16 are taken by hand).  Subgradients at the kinks: the
 * Riemann limiter (Eq. 6) has d beta / d dU = eta_R / c inside
 * 0 < eta_R dU / c < 1 and 0 elsewhere; the transport-velocity limiter
 * (Eq. 15) has d chi / d s = C inside thresh < s < 1/C and 0 elsewhere.
 *
 *   x0, v0, a0, dr0  [n][3] checkpoint state at the start of the segment, in
 *                    the caller's order (host or device): the arrays of an
 *                    sph_save_ckpt (or sph_get_state) at that step of the
 *                    forward run
 *   nsteps           1 <= nsteps <= params.adjoint_steps
 *   xbar, vbar, abar, drbar  [n][3] (host or device, caller order): on entry
 *                    the cotangents of the state after the segment, on
 *                    return those of the checkpoint state
 *   etabar           on return d(loss)/d(eta) accumulated over the segment
 *                    (host double; may be NULL)
 * The library replays the segment from the checkpoint (the cell sort is
 * deterministic, so the replay reproduces the forward run bit for bit),
 * keeping per-step values in its workspace, then runs the reverse steps.
 * On return the context holds the replayed state after the segment.  The
 * FP32 form computes pair derivatives in FP32 with compensated sums and
 * keeps the cotangents in FP64.  Waits for the stream.  SPH_ERR_ARG for
 * nsteps outside [1, adjoint_steps], NULL arrays, or tv_mode
 * SPH_TV_BACKGROUND (no adjoint for that mode). */
SPH_API sph_status sph_step_adjoint(sph_ctx* ctx, const double* x0, const double* v0, const double* a0,
                                    const double* dr0, int32_t nsteps, double* xbar, double* vbar, double* abar,
                                    double* drbar, double* etabar);

/* Adjoint of the initial force pass of sph_build_cells (a and dr from x and
 * v, no a/dr given): with abar, drbar the cotangents of that pass's a and dr
 * ([n][3], caller order), ADD the cotangents of x and v to xbar and vbar and
 * write d/d(eta) to *etabar (may be NULL).  Loads x and v into the context
 * (as sph_set_state + sph_build_cells would, with the smoothing lengths,
 * masses, kinds and prescribed wall velocities of the last sph_set_state;
 * the walls' entries of v are ignored).  Waits for the stream.
 * Requires params.adjoint_steps >= 1. */
SPH_API sph_status sph_force_pass_adjoint(sph_ctx* ctx, const double* x, const double* v, const double* abar,
                                          const double* drbar, double* xbar, double* vbar, double* etabar);

/* Limits of sph_density_noalloc's fixed scratch. */
#define SPH_NOALLOC_MAX_PARTICLES 65536
#define SPH_NOALLOC_MAX_CELLS 65536

/* Density pass without any device allocation.  This entry point has no
 * counterpart in the paper; it exists for callers that cannot give the
 * library a workspace: a host framework that owns all device memory and does
 * not let its plug-ins call cudaMalloc outside its allocator, or a real-time
 * loop where a cudaMalloc/cudaFree could synchronise the device and stall it.
 *
 * It computes the summation density rho_i = rho0 sum_j W_ij / sigma0_i of
 * sph_build_cells (FP64, same kernels, same result) for n particles:
 *   p       parameters; precision must be 64 (else SPH_ERR_ARG)
 *   x       [n][3] positions, device memory
 *   h, m    [n] smoothing lengths and masses, device memory
 *   kind    [n] 0 fluid / 1 wall, device memory, or NULL (all fluid)
 *   sigma0  [n] reference sums, device memory, or NULL (perfect-lattice sums)
 *   rho     [n] output, device memory, in the caller's particle order
 *   stream  cudaStream_t on which the work is enqueued; returns without waiting
 * Its scratch is one fixed array in device memory inside the library,
 * 24 MiB on every GPU that loads it, held until the process exits; n above
 * SPH_NOALLOC_MAX_PARTICLES or a cell grid above SPH_NOALLOC_MAX_CELLS cells
 * returns SPH_ERR_WORKSPACE before any work is enqueued.  A call made
 * outside stream capture looks up the scratch's device address on the
 * current device (cudaGetSymbolAddress) and remembers it; a call made while
 * the stream is being captured uses the remembered address, so make a first
 * call on each device before any capture (otherwise SPH_ERR_STATE).  After a
 * device reset, make a call outside capture before capturing again.  All calls share the one
 * scratch: the call clears the counters it sums into, but two calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller.  Device-side input checks
 * (particles outside a non-periodic box, h outside [h_min, h_max]) are not
 * reported by this entry point. */
SPH_API sph_status sph_density_noalloc(const sph_params* p, int64_t n, const double* x, const double* h,
                                       const double* m, const int8_t* kind, const double* sigma0, double* rho,
                                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPHTV_H */
