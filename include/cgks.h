/*
 * cgks.h -- C ABI of the GB300 (sm_103a) library for one two-stage
 * fourth-order (S2O4) time step of the compact gas-kinetic scheme with
 * adaptive stencil extension and discontinuity feedback factor (ASE-DFF-CGKS)
 * on structured 1-D / 2-D Cartesian meshes.
 *
 * Method (paper sections, equations and algorithms):
 *   S2O4 stepping of cell averages and gradients ........ Sec. 2.2, Eq. 2.13-2.30
 *   gas-kinetic flux and interface state ................. Sec. 2.1, Eq. 2.6-2.8, 2.11-2.12
 *   discontinuity feedback factor (DFF) .................. Sec. 3.1, Eq. 3.1-3.5
 *   ASE-DFF Hermite reconstruction (r5/r7/r9, HWENO-AO) .. Sec. 3.2, Eq. 3.6-3.19, Algorithm 1
 *   2-D dimension-by-dimension reconstruction (Steps 1-4)  Sec. 3.3
 *   collision time and CFL time step ..................... Sec. 4 (opening paragraphs)
 *
 * Conventions
 *   - Every call returns 0 (CGKS_OK) or a negative CGKS_E* code; nothing throws.
 *   - Host arrays are FP64, structure of arrays, C order:
 *       W, Wx, Wy            [nvar][ny][nx]     nvar = 3 (1-D: rho, rho U, rho E)
 *                                                    = 4 (2-D: rho, rho U, rho V, rho E)
 *       Wx_line, Wy_line     [m][nvar][ny][nx]  m = 2, 3, 4 Gauss points per face
 *                                               for order 5, 7, 9 (2-D only)
 *       sigma_x              [ny][nx+1]         DFF strength of x-faces (face f lies
 *                                               between cells f-1 and f)
 *       sigma_y              [ny+1][nx]         DFF strength of y-faces
 *     1-D meshes use ny = 1 and pass NULL for every y array.
 *   - Wx / Wy are cell averages of the x / y derivative; Wx_line[l] is the
 *     x-derivative averaged along the l-th Gauss line y = y_j + xi_l dy of the
 *     cell (Sec. 3.3, "line averaged slopes").
 *   - The library owns the solver and all device memory.  A solver is not
 *     thread safe; distinct solvers are independent.  Results are
 *     deterministic: the same inputs give bitwise identical outputs.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL means
 *     the legacy default stream).
 */
#ifndef CGKS_H
#define CGKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define CGKS_OK 0
#define CGKS_EINVAL (-1)     /* invalid argument (order, size, gamma, cfl, pointer) */
#define CGKS_ENOMEM (-2)     /* device allocation failed */
#define CGKS_ECUDA (-3)      /* a CUDA runtime call failed */
#define CGKS_ENONPHYS (-4)   /* non-positive density / pressure or non-finite value */
#define CGKS_ETIMEOUT (-5)   /* reserved: a bounded device wait gave up (no kernel here waits on
                                another block or launch, so none is returned) */
#define CGKS_ENOTSUP (-6)    /* combination of options not supported */

/* precision of the reconstruction and kinetic arithmetic */
#define CGKS_FP64 0          /* everything in FP64 */
#define CGKS_FP32_BULK 1     /* reconstruction / kinetics in FP32; cell averages,
                                their accumulation, DFF and positivity tests in FP64 */
/* collision time (Sec. 4) */
#define CGKS_TAU_ZERO 0      /* tau = 0 (smooth inviscid tests, Sec. 4.6) */
#define CGKS_TAU_HGKS 1      /* tau = c1 dt + c2 |pl - pr| / (pl + pr) dt */
#define CGKS_TAU_NS 2        /* viscous flow (Sec. 4): tau = mu / p + c2 |pl - pr| / (pl + pr) dt,
                                p the pressure of the equilibrium state at the face point;
                                the time step adds the limit dx^2 / (4 nu), nu = mu / rho */
/* time lag of the DFF's sigma (Sec. 3.1, "from the previous time step"): */
#define CGKS_DFF_LAG_STEP 0  /* (default) sigma of stage 1 of step n-1 in both stages of step n */
#define CGKS_DFF_LAG_STAGE 1 /* the same in stage 1; stage 2 uses the sigma of stage 1 of
                                step n, half a step old.  Neither carries every case: with
                                the step lag a strong wave that enters a cell within one
                                step meets stencils that still see sigma = 0 (the Sec. 4.9
                                shock tube loses positivity in step 2), while the stage lag
                                lets the two stages pick different stencils and loses
                                positivity late in Configuration 3 (Sec. 4.7, 500^2, FP32
                                bulk).  Smooth data take the same branches under both */
/* boundary conditions, per side: bc[0..3] = x-low, x-high, y-low, y-high */
#define CGKS_BC_PERIODIC 0
#define CGKS_BC_TRANSMISSIVE 1  /* ghost = nearest interior cell, normal slopes zero */
#define CGKS_BC_FIXED 2         /* 1-D only: ghost cells fixed by cgks_set_ghost */
#define CGKS_BC_REFLECTIVE 3    /* slip wall (Sec. 4.4, and the symmetry plane of Sec. 4.9):
                                   ghost cell k = mirror image of interior cell k (the
                                   cell and line averages and slopes reflected, the
                                   normal momentum reversed); ghost faces mirror sigma */
#define CGKS_BC_NOSLIP 4        /* adiabatic no-slip wall (Sec. 4.9): the same mirror with
                                   both momentum components reversed */
#define CGKS_BC_INFLOW 5        /* 2-D: ghost cells hold a prescribed state with zero slopes
                                   (the supersonic inflow and the exact shock motion of
                                   Sec. 4.8): bc_state[side][0] where the ghost cell's centre
                                   coordinate along the side (y on x-sides, x on y-sides)
                                   lies below split(t) = bc_split[side][0] + bc_split[side][1] t,
                                   bc_state[side][1] elsewhere, t the stage's time (t^n in
                                   stage 1, t^n + dt/2 in stage 2); beyond the side sigma is 0
                                   at the faces parallel to it and copies the nearest row or
                                   column along it, as at a transmissive side */
#define CGKS_BC_INFLOW_REFLECTIVE 6 /* 2-D: bc_state[side][0] below split(t), a slip wall
                                   beyond it (the bottom of Sec. 4.8); sigma mirrors as at
                                   a wall along the whole side */
/* first-order fallback at face Gauss points (not a step of the paper, which
   states no limiter; off by default) */
#define CGKS_PT_FALLBACK_OFF 0
#define CGKS_PT_FALLBACK_FIRST_ORDER 1 /* a side of a face Gauss point whose reconstructed
                                   state has rho <= 0 or p <= 0 (tested in the bulk
                                   precision) takes the average of the cell it was
                                   reconstructed from, with every derivative zero; sigma
                                   then comes from the states used; counted in
                                   cgks_stats.fallbacks.  Compiled into the flux of
                                   the collision-time modes only: with CGKS_TAU_ZERO
                                   it is rejected with CGKS_ENOTSUP */

typedef struct {
    int dim;            /* 1 or 2 */
    int order;          /* 5, 7 or 9: ASE-DFF(5,3), (7,5,3), (9,7,5,3) */
    int precision;      /* CGKS_FP64 or CGKS_FP32_BULK */
    int tau_mode;       /* CGKS_TAU_ZERO or CGKS_TAU_HGKS */
    int bc[4];          /* CGKS_BC_* per side */
    double gamma;       /* ratio of specific heats, > 1 */
    double cfl;         /* CFL number of the time-step rule, > 0 */
    double sigma_thres; /* DFF threshold, Eq. 3.3 (1.0 for compact stencils) */
    double gamma_hi;    /* HWENO-AO linear weight of the big stencil, Eq. 3.12 (0.85) */
    double gamma_lo;    /* HWENO-AO low-order split, Eq. 3.12 (0.6) */
    double weno_eps;    /* epsilon of the WENO-Z weights, Eq. 3.14 (1e-8) */
    double tau_c1;      /* c1 of the HGKS collision time (0.05) */
    double tau_c2;      /* c2 of the HGKS collision time (1.0) */
    double mu;          /* dynamic viscosity of CGKS_TAU_NS (constant), >= 0 */
    int dff_lag;        /* CGKS_DFF_LAG_STEP (default) or CGKS_DFF_LAG_STAGE */
    int pt_fallback;    /* CGKS_PT_FALLBACK_OFF (default) or CGKS_PT_FALLBACK_FIRST_ORDER */
    double bc_state[4][2][4]; /* prescribed ghost states of CGKS_BC_INFLOW* sides, conservative
                                 (rho, rho U, rho V, rho E), rho > 0 and p > 0 */
    double bc_split[4][2];    /* split point along each such side: [0] + [1] t */
} cgks_params;

typedef struct cgks_solver cgks_solver;
typedef struct cgks_batch cgks_batch;

typedef struct {
    double t;            /* simulated time */
    long long steps;     /* completed steps */
    double min_rho, min_p;
    double mass[4];      /* sum over cells of W * dx * dy, per variable */
    long long branch[4]; /* normal-reconstruction branches (per cell and Gauss
                            line, both directions) of the latest step's two
                            stages: HWENO-AO, linear r5, r7, r9 (batches: summed) */
    long long fallbacks; /* face-point sides that took CGKS_PT_FALLBACK_FIRST_ORDER since
                            the last set_state (both stages and directions) */
} cgks_stats;

/* Fill *p with the paper's defaults for (dim, order): gamma 1.4, CFL 0.5,
 * sigma_thres 1, gamma_hi 0.85, gamma_lo 0.6, eps 1e-8, c1 0.05, c2 1, mu 0,
 * FP64, tau = 0, periodic, step-lag DFF, no point fallback, zero inflow
 * states.  Returns CGKS_EINVAL for a NULL p. */
int cgks_default_params(cgks_params* p, int dim, int order);

/* Create a solver for an nx x ny mesh on [x0,x1] x [y0,y1] (1-D: ny = 1,
 * y bounds ignored).  All device buffers are allocated here on `stream`'s
 * device; the CUDA graph of one step is captured on first use.
 * Errors: CGKS_EINVAL (NULL out/p, dim not 1/2, order not 5/7/9, nx or ny < 1,
 * ny != 1 in 1-D, gamma <= 1, cfl <= 0, non-positive extent, FIXED bc in 2-D,
 * INFLOW bc in 1-D, an inflow side whose states are not physical or whose
 * split is not finite, a wall or inflow side across fewer than 3 cells,
 * pt_fallback not 0/1,
 * a mesh with 2^31 or more face Gauss points: about 16000^2 cells at order 9,
 * more than the device memory holds), CGKS_ENOTSUP (pt_fallback with
 * CGKS_TAU_ZERO), CGKS_ENOMEM, CGKS_ECUDA.  On error *out is NULL. */
int cgks_init_mesh(cgks_solver** out, const cgks_params* p, int nx, int ny,
                   double x0, double x1, double y0, double y1, void* stream);

/* Copy a host state in (synchronous); the simulated time and the fallback
 * count restart from 0.  sigma_x / sigma_y may be NULL: sigma is then
 * initialised from Eq. 3.2 applied to the two cell averages adjacent to each
 * face (ghost cells of inflow sides taken at t = 0).  Returns CGKS_ENONPHYS if
 * some cell has rho <= 0 or p <= 0, CGKS_EINVAL for a NULL required array. */
int cgks_set_state(cgks_solver* s, const double* W, const double* Wx, const double* Wy,
                   const double* Wx_line, const double* Wy_line,
                   const double* sigma_x, const double* sigma_y);

/* As cgks_set_state, with device pointers (same layouts), enqueued on the
 * solver's stream.  sigma pointers may be NULL (initialised on the device). */
int cgks_set_state_device(cgks_solver* s, const double* W, const double* Wx, const double* Wy,
                          const double* Wx_line, const double* Wy_line,
                          const double* sigma_x, const double* sigma_y);

/* Set the simulated time (the t^n of the next step), e.g. to resume a run or
 * to place the split points of inflow sides; enqueued on the solver's stream.
 * If the last set_state initialised sigma (NULL sigma arrays) and no step has
 * run since, sigma is initialised again with the ghost states of inflow sides
 * taken at t, as if the state had been set at time t.
 * CGKS_EINVAL for a NULL solver or a non-finite t. */
int cgks_set_time(cgks_solver* s, double t);

/* 1-D, CGKS_BC_FIXED sides: ghost cells [2 sides][3 layers][2 fields W,Wx][3 vars]
 * (layer 0 touches the boundary).  Host pointer; copied. */
int cgks_set_ghost(cgks_solver* s, const double* ghost);

/* Time step of the CFL rule: dt = cfl * min over cells of min(dx,dy) / (|U| + a),
 * a = sqrt(gamma p / rho).  Synchronous. */
int cgks_compute_dt(cgks_solver* s, double* dt);

/* Enqueue one S2O4 step (two stages) on the solver's stream as one CUDA graph
 * launch.  dt > 0: use it; dt <= 0: use the CFL rule, evaluated on the device
 * (no host round trip).  Returns only host-detectable errors; device status
 * (non-physical states) is reported by cgks_sync. */
int cgks_step(cgks_solver* s, double dt);

/* Enqueue n steps of fixed dt (> 0) or CFL steps (dt <= 0). */
int cgks_advance(cgks_solver* s, int n, double dt);

/* Wait for the solver's stream.  t_out (may be NULL) receives the simulated
 * time; bad_cell (may be NULL) the first cell index flagged.  Returns
 * CGKS_ENONPHYS if any stage met rho <= 0, p <= 0 or a non-finite value. */
int cgks_sync(cgks_solver* s, double* t_out, long long* bad_cell);

/* Copy the state out (synchronous), FP64 whatever the precision.  Any output
 * pointer may be NULL to skip that array. */
int cgks_get_state(cgks_solver* s, double* W, double* Wx, double* Wy, double* Wx_line,
                   double* Wy_line, double* sigma_x, double* sigma_y);

/* Device-pointer variant of cgks_get_state, enqueued on the solver's stream. */
int cgks_get_state_device(cgks_solver* s, double* W, double* Wx, double* Wy, double* Wx_line,
                          double* Wy_line, double* sigma_x, double* sigma_y);

/* Diagnostics (synchronous). */
int cgks_get_stats(cgks_solver* s, cgks_stats* st);

/* Autotuner: times every stage kernel on the solver's current state and keeps
 * the fastest launch shape; the step graph is rebuilt on the next step.  The
 * 2-D Steps 1-2 (one fused kernel per direction over tiles held in shared
 * memory) are timed over tile shapes TA x TB (cells along the face normal x
 * across it: 28x8, 60x4, 12x16, 28x4, 12x8, 124x2) at 128 and 256 threads;
 * the other kernels over block sizes 64..512 (persistent grid = SM count x
 * resident blocks), the FP64 flux kernels also in a register-capped variant (more
 * resident warps, some spilling).  The state is not advanced (only scratch is
 * written; the simulated time, the status word and the fallback count are
 * restored) and results do not depend on the choice: every work item is
 * computed by one thread.  threads_out (may be NULL) receives 10 ints: the
 * block sizes of Steps 1-2 along x and y (1-D: 0 and Step 2), flux (stage 1,
 * 2), update (stage 1, 2), then the tile shapes (TA, TB) along x and y (0 in
 * 1-D); a negative flux entry marks the capped variant.  Requires a state
 * (CGKS_EINVAL otherwise). */
int cgks_autotune(cgks_solver* s, int* threads_out);
int cgks_batch_autotune(cgks_batch* b, int* threads_out);

/* Number of graph nodes (kernel launches) one CFL step makes. */
int cgks_step_info(cgks_solver* s, int* kernels_per_step);

/* Diagnostics: run one fixed-dt step (dt > 0) kernel by kernel outside the
 * graph, with CUDA events on the solver's stream between launches.  ms[k]
 * receives the device time of launch k and ids[k] its kernel:
 * 0 Steps 1-2 along x (2-D), 1 Steps 1-2 along y (2-D) or Step 2 (1-D),
 * 2 flux, 3 update, 4 dt (stage s launches carry 10*s + id).  *n is the capacity on entry and the count on exit (<= 16).
 * Advances the state like cgks_step. */
int cgks_profile_step(cgks_solver* s, double dt, float* ms, int* ids, int* n);

/* Diagnostics for the roofline of the stage kernels (no counterpart in the
 * paper): the measured fused multiply-add throughput of the current GPU in
 * precision CGKS_FP32_BULK (FP32) or CGKS_FP64, from a kernel of independent
 * FMA chains on every SM (2 flops per FMA), timed with CUDA events at the
 * clock the GPU runs at; *tflops receives TFLOP/s, ms (may be NULL) the best
 * launch time.  Allocates a small output buffer; synchronous; changes no
 * GPU setting.  CGKS_EINVAL for a NULL tflops or another precision. */
int cgks_fma_peak(int precision, double* tflops, float* ms);

void cgks_destroy(cgks_solver* s);
const char* cgks_strerror(int code);

/* ---------------------------------------------------------------- batch
 * Many independent 2-D meshes advanced together: every kernel of a stage is
 * one persistent launch over a device work list of all instances, and the
 * two-stage step is one CUDA graph.  Instance k has nx[k] x ny[k] cells on
 * [ext[4k], ext[4k+1]] x [ext[4k+2], ext[4k+3]]; all share *p.  States are
 * concatenated per instance in the single-mesh layouts above.  An instance
 * agrees with the same mesh stepped alone to rounding, not bitwise: a single
 * mesh runs its own compilation of the stage kernels (the mesh descriptor
 * passed by value), which may contract multiply-adds differently. */
int cgks_batch_init(cgks_batch** out, const cgks_params* p, int n, const int* nx, const int* ny,
                    const double* ext, void* stream);
int cgks_batch_set_state(cgks_batch* b, int k, const double* W, const double* Wx, const double* Wy,
                         const double* Wx_line, const double* Wy_line);
/* Device-pointer variants for instance k (same layouts), enqueued on the
 * batch's stream without waiting.  set: sigma is initialised from the cell
 * averages and the state's positivity is checked on the device; a
 * non-physical state is reported by cgks_batch_sync.  get: FP64 copies of the
 * state (upcast from the float planes in the FP32-bulk form). */
int cgks_batch_set_state_device(cgks_batch* b, int k, const double* W, const double* Wx, const double* Wy,
                                const double* Wx_line, const double* Wy_line);
int cgks_batch_get_state_device(cgks_batch* b, int k, double* W, double* Wx, double* Wy,
                                double* Wx_line, double* Wy_line);
/* one step of all instances; dt[k] > 0 fixed per instance, or NULL: each
 * instance takes its own CFL dt on the device. */
int cgks_batch_step(cgks_batch* b, const double* dt);
int cgks_batch_sync(cgks_batch* b);
int cgks_batch_get_state(cgks_batch* b, int k, double* W, double* Wx, double* Wy,
                         double* Wx_line, double* Wy_line);
void cgks_batch_destroy(cgks_batch* b);

/* ---------------------------------------------------------------- no-allocation step
 * One S2O4 step of a 1-D mesh that allocates no device memory.  The paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc, for
 * example code running under another framework's memory manager that owns
 * the whole device (and forbids raw allocations), or code on a latency-bound
 * path where an allocation (which may synchronise the device) is not allowed.
 *
 * All intermediate data (stage state, accumulator, face data, descriptors)
 * lives in one file-scope device array of CGKS_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library keeps until process exit; meshes are limited to
 * nx <= CGKS_NOALLOC_MAX_CELLS (larger nx returns CGKS_EINVAL).
 *
 * Arguments: p (dim must be 1; FIXED boundaries are not supported here and
 * return CGKS_ENOTSUP), nx cells on [x0, x1]; device pointers state_in and
 * state_out of 6*nx doubles ([W(3 vars)][nx] then [Wx(3 vars)][nx]; they may
 * be equal), sigma_in (nx+1 doubles, or NULL: initialised from the cell
 * averages as in cgks_set_state) and sigma_out (nx+1 doubles); dt > 0 fixed,
 * dt <= 0 the CFL rule; status_out (device unsigned int, may be NULL)
 * receives the step's status word (nonzero: non-physical state met).  The
 * work is enqueued on `stream` (NULL: the legacy default stream) and the call
 * returns without waiting.  It enqueues kernel launches and device-to-device
 * copies only: the descriptor and dt travel as kernel arguments, so no host
 * memory is read after the call returns.  With CGKS_PT_FALLBACK_FIRST_ORDER
 * the fallback runs but its count is not reported by this entry point.
 *
 * The first call on a device does its set-up there (finds the scratch array's
 * device address, loads the reconstruction tables): make that first call
 * before any stream capture.  The set-up is guarded by a lock, so first calls
 * from several host threads are safe.  Every call uses the same scratch array and
 * clears the parts that must start at zero; calls that overlap on the GPU
 * (different streams, or devices sharing nothing but this array's contents
 * per device) race on it and must be serialised by the caller. */
#define CGKS_NOALLOC_MAX_CELLS 4096
#define CGKS_NOALLOC_SCRATCH_BYTES (4u << 20)
int cgks_step_1d_noalloc(const cgks_params* p, int nx, double x0, double x1,
                         const double* state_in, const double* sigma_in,
                         double* state_out, double* sigma_out, double dt,
                         unsigned* status_out, void* stream);

/* ---------------------------------------------------------------- host tables
 * The reconstruction functionals the kernels use, for inspection (no GPU
 * needed).  Stencil st: 0 S0, 1 S1, 2 S2, 3 r5, 4 r7, 5 r9 (Sec. 3.2); row:
 * 0..2 value, d/dxi, d2/dxi2 at xi = +1/2; 3..5 the same at xi = -1/2;
 * 6..9 values at the m Gauss nodes of `order`.  out[10] multiplies
 * [Qbar_{i-2..i+2}, dx*Qx_{i-2..i+2}]. */
int cgks_stencil_row(int order, int st, int row, double* out);

#ifdef __cplusplus
}
#endif
#endif
