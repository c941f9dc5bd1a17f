/*
 * ibm.h -- C ABI of libibm, the GB300 (sm_103a) hot path of the immersed-
 * boundary fractional-step solver of arXiv 2406.19920 ("A Python-based flow
 * solver for numerical simulations using an immersed boundary method on
 * single GPUs").
 *
 * Problem statement (Sec. 2.1, Eq. 2a-2h): incompressible flow on a uniform
 * staggered (MAC) grid, periodic in x and z and bounded by no-slip walls in
 * y, advanced by a three-stage semi-implicit RK scheme with Uhlmann's
 * direct-forcing immersed boundary.  Each stage needs three Helmholtz solves
 * (Eq. 2e), one Poisson solve (Eq. 2f), the interpolation / spreading pair
 * between Eulerian grid and Lagrangian markers (Eq. 2b-2d) and a projection
 * (Eq. 2g, 2h).  The linear systems are solved directly as in the paper's
 * doubly periodic branch (Sec. 2.3.3, S1.1/S1.2/S2.1/S2.2): real FFT along x,
 * complex FFT along z, one tridiagonal (Thomas) solve per Fourier pencil
 * along y, inverse transforms.
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid: nx x ny x nz cells, spacings h = {hx, hy, hz}.  nx and nz must be
 *   2^a 3^b with b <= 1 and 8 <= n <= 512; 8 <= ny <= 512.
 * Layout: every field is a dense C array [ny][nz][nx] (x fastest, then z,
 *   then y) in DEVICE memory, of the plan's precision (float for
 *   IBM_FP32_REFINED, double for IBM_FP64).
 *   - cell-centred fields (p, phi, Poisson rhs) at ((i+1/2)hx,(j+1/2)hy,(k+1/2)hz)
 *   - u on x-faces (i hx, (j+1/2)hy, (k+1/2)hz)
 *   - w on z-faces ((i+1/2)hx, (j+1/2)hy, k hz)
 *   - v on y-faces ((i+1/2)hx, j hy, (k+1/2)hz): plane j is face j, plane 0
 *     is the bottom wall and the top wall face j = ny is not stored.  Both
 *     wall faces carry v = 0: plane 0 is ignored on input and written as 0.
 * Markers: positions X and velocities/forces are arrays [n][3] (x, y, z),
 *   volumes dV are [n], all in device memory, plan precision.  The wall
 *   rule: the support of delta_h (Eq. 2b, 2d) reaches 1.5 hy (3-point
 *   kernel) / 2 hy (4-point kernel) from a marker along y, and a marker
 *   closer than that to a wall (Y < 1.5 hy or Y > Ly - 1.5 hy; 2 hy for the
 *   4-point kernel; NaN too) would need values beyond the wall.  Marker
 *   positions live on the device, so the kernels apply the rule: such a
 *   marker is neither interpolated (its U and F are written as 0) nor
 *   spread, and the plan's error word counts it.  ibm_plan_check, and the
 *   next call with a non-NULL info, then return IBM_ERR_ARG with the count.
 * Alignment: field pointers must be 16-byte aligned (they are moved with
 *   bulk asynchronous copies); marker arrays need their element alignment.
 * Ownership: all field and marker pointers belong to the caller; the plan
 *   owns its workspace, twiddle and eigenvalue tables.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Every
 *   call is asynchronous on it, except that when `info` is non-NULL the call
 *   synchronises the stream before returning so that `info` is filled.
 * Errors: every entry point returns an IBM_* code and never throws.  Bad
 *   arguments are rejected with IBM_ERR_ARG before any launch; CUDA failures
 *   give IBM_ERR_CUDA.  ibm_last_error() returns a thread-local message.
 * Thread safety: a plan may be used from one host thread / stream at a time.
 */
#ifndef IBM_H
#define IBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_plan_s *ibm_plan;
typedef struct ibm_batch_s *ibm_batch;
typedef struct ibm_server_s *ibm_server;

enum {
  IBM_OK = 0,
  IBM_PENDING = 1,
  IBM_ERR_ARG = -1,
  IBM_ERR_OOM = -2,
  IBM_ERR_CUDA = -3,
  IBM_ERR_TIMEOUT = -4,
  IBM_ERR_BUSY = -5,
  IBM_ERR_UNSUPPORTED = -6,
  IBM_ERR_CANCELLED = -7
};

/* Domain boundary conditions.
 * IBM_BC_PXZ_WALL_Y: periodic x and z, walls in y (the paper's doubly
 *   periodic branch, Sec. 2.3.3, with its wall axis renamed y): every entry
 *   point.
 * IBM_BC_TRIPLY_PERIODIC: periodic in all three axes (Sec. 2.3.3, S2): the
 *   Poisson and Helmholtz solves only (ny must then be 2^a 3^b, b <= 1, in
 *   [8, 512]); ibm_substep, ibm_interp and ibm_spread return
 *   IBM_ERR_UNSUPPORTED for such plans. */
enum { IBM_BC_PXZ_WALL_Y = 1, IBM_BC_TRIPLY_PERIODIC = 2 };

/* Precision of fields and of the bulk arithmetic. */
enum { IBM_FP64 = 0, IBM_FP32_REFINED = 1 };

/* Wall rows of a Helmholtz field (Appendix B). */
enum {
  IBM_FIELD_CELL_NEUMANN = 0,   /* cell-centred, ghost = first value        */
  IBM_FIELD_CELL_DIRICHLET = 1, /* cell-centred no-slip: alpha = 2, A11 = A1 - A2 */
  IBM_FIELD_FACE_DIRICHLET = 2, /* wall-normal faces: alpha = 1, walls = 0   */
  IBM_FIELD_PERIODIC = 3        /* no walls: the triply periodic branch's only kind */
};

/* Regularised delta kernels (Sec. 2.1 cites Peskin and Roma et al.). */
enum { IBM_DELTA_ROMA3 = 0, IBM_DELTA_PESKIN4 = 1 };

/* Prescribed marker motion (L2, Sec. 2.3.2). */
enum { IBM_MOTION_STATIC = 0, IBM_MOTION_TRANSLATE = 1, IBM_MOTION_HEAVE = 2 };

enum {
  IBM_K_FORWARD = 0,   /* x/z forward transform of a right-hand side      */
  IBM_K_PENCIL = 1,    /* tridiagonal solves along y                      */
  IBM_K_INVERSE = 2,   /* z/x inverse transform                           */
  IBM_K_RESIDUAL = 3,  /* refinement residual                             */
  IBM_K_EXPLICIT = 4,  /* E1 explicit terms                               */
  IBM_K_MOTION = 5,    /* L2 marker motion (fused into IBM_K_INTERP: no   */
                       /* launches of its own)                            */
  IBM_K_INTERP = 6,    /* L2 motion + L1 interpolation + force            */
  IBM_K_SPREAD = 7,    /* L1 spreading                                    */
  IBM_K_DIVERGENCE = 8,/* E2 divergence                                   */
  IBM_K_PROJECT = 9,   /* E3 projection + pressure update                 */
  IBM_K_OUTFLOW = 10,  /* outlet update + mass balance (inflow-outflow)   */
  IBM_K_COUNT = 11
};

typedef struct {
  double rel_residual;  /* ||b - A x||_2 / ||b||_2 of the returned x (FP64 sums)  */
  double removed_mean;  /* Poisson: mean(b) removed to make b compatible          */
  double div_max;       /* substep: max |D u^n| after projection (float-float)    */
  double div_before;    /* substep: max |D u*| before projection                  */
  double t_ms;          /* device time of the call (events), when info is given   */
  int refine_iters;     /* refinement steps applied                              */
  int reserved;
  double phase_ms[IBM_K_COUNT]; /* device time of each kernel kind (IBM_K_*) in   */
                        /* the call, from events around its launches (the      */
                        /* per-task split the paper reports in Sec. 4)          */
} ibm_info;

/* ---------------------------------------------------------------------------
 * Plans
 * ------------------------------------------------------------------------- */

/* Create a plan for an nx x ny x nz grid with spacings h[3] = {hx, hy, hz}.
 * bc: IBM_BC_PXZ_WALL_Y or IBM_BC_TRIPLY_PERIODIC.  precision: IBM_FP64 or
 * IBM_FP32_REFINED.
 * refine_iters: iterative-refinement steps on the residual for the FP32 path
 * (0..4; ignored for FP64).  Allocates the plan's device workspace
 * (about 4 fields) and its FP64-derived twiddle and modified-wavenumber
 * tables (Appendix A) on the current device.  Errors: IBM_ERR_ARG for an
 * unsupported size or spacing, IBM_ERR_OOM when the workspace does not fit. */
int ibm_plan_create(int nx, int ny, int nz, int bc, const double h[3],
                    int precision, int refine_iters, ibm_plan *out);
int ibm_plan_destroy(ibm_plan plan);
/* Select the delta kernel used by ibm_interp / ibm_spread / ibm_substep. */
int ibm_plan_set_delta(ibm_plan plan, int kernel);
/* Spreading (Eq. 2d) used by ibm_spread / ibm_substep.
 *   IBM_SPREAD_ATOMIC  (default) atomic spreading.  From 40,000 markers on,
 *                      with shared-memory pre-aggregation: a CTA of 256
 *                      (marker, component) entries whose stencils fit a small
 *                      box adds them into shared memory first and then each
 *                      non-zero box point to f with one global atomic; other
 *                      CTAs, and smaller marker sets, add directly as
 *                      IBM_SPREAD_ATOMIC_DIRECT.  The order of the additions,
 *                      and so the last bits of f, vary from run to run.
 *   IBM_SPREAD_ATOMIC_DIRECT  the paper's L1 kernel (Sec. 2.3.2) as it
 *                      stands: one thread per (marker, component) adds its
 *                      S^3 shares with global atomics.
 *   IBM_SPREAD_GATHER  the alternative Sec. 2.3.2 describes and sets aside:
 *                      one thread per Eulerian point gathers the shares of the
 *                      markers whose stencils cover it.  Markers are binned by
 *                      stencil origin into 4^3 bricks per component (counting
 *                      sort, each brick's entries ordered by marker index), so
 *                      every point sums its shares in a fixed order: f is
 *                      bitwise the same on every run.  Needs plan workspace of
 *                      about 12 bytes per brick and 40 bytes per marker
 *                      component (allocated on first use; IBM_ERR_OOM if it
 *                      cannot be). */
enum { IBM_SPREAD_ATOMIC = 0, IBM_SPREAD_GATHER = 1, IBM_SPREAD_ATOMIC_DIRECT = 2 };
int ibm_plan_set_spread(ibm_plan plan, int mode);
/* Bytes of device memory the plan holds. */
size_t ibm_plan_workspace_bytes(ibm_plan plan);

/* Synchronise the device and report the plan's device error word, then
 * clear it: IBM_ERR_TIMEOUT when a kernel gave up one of its bounded waits,
 * IBM_ERR_ARG when markers were rejected by the wall rule (the message gives
 * their count, summed over the calls since the last check), IBM_OK
 * otherwise.  Calls with a non-NULL info perform the same check. */
int ibm_plan_check(ibm_plan plan);

/* Diagnostic of the bounded waits (no fault is involved).  Every wait of the
 * library's kernels on an mbarrier (bulk copies, tensor-core commits) gives
 * up after a fixed wall time (100 ms), records IBM_ERR_TIMEOUT in the plan's
 * error word, waits once more (bounded) for work in flight and returns.
 * This launches one CTA that takes that way out on purpose, after limit_ms
 * milliseconds (0 < limit_ms <= 5000), on one of two paths:
 *   IBM_SELFTEST_TENSOR_MEMORY  holds tensor memory and waits on an mbarrier
 *                               that nothing completes, then frees the memory;
 *   IBM_SELFTEST_BULK_COPY      issues one in-bounds 16-byte bulk copy whose
 *                               barrier expects twice its bytes, so the wait
 *                               cannot complete, then waits once more.
 * The next ibm_plan_check (after the stream has drained) returns
 * IBM_ERR_TIMEOUT; the plan and the context stay usable. */
enum { IBM_SELFTEST_TENSOR_MEMORY = 0, IBM_SELFTEST_BULK_COPY = 1 };
int ibm_selftest_timeout(ibm_plan plan, int path, double limit_ms, void *stream);

/* Per-kernel timing (tracing).  While enabled, every kernel the plan
 * launches is bracketed by a pair of CUDA events on its stream; the pairs
 * are accumulated per kernel kind (IBM_K_*).  ibm_plan_profile_read
 * synchronises the device, writes the summed milliseconds and launch counts
 * of the first max_kinds kinds to ms[] / launches[] (either may be NULL),
 * clears the record and returns IBM_K_COUNT.  The paper reports per-task
 * time shares (Sec. 4); this gives the same breakdown per kernel. */

int ibm_plan_profile(ibm_plan plan, int enable);
int ibm_plan_profile_read(ibm_plan plan, int max_kinds, double *ms, int *launches);

/* Poisson solve, Eq. 2f (S2.1 + S2.2): L_h phi = rhs - mean(rhs) with the
 * 7-point Laplacian, periodic x/z, homogeneous Neumann y (Appendix B,
 * A3 + A2 corner rows), mean(phi) = 0.  rhs and phi are [ny][nz][nx]; rhs may
 * equal phi.  The zero-wavenumber pencil is eliminated in FP64 with the
 * paper's pin (phi_hat = 0 at the first interior point, Sec. 2.3.3), then
 * its FP64 mean is removed.  On an IBM_BC_TRIPLY_PERIODIC plan y is periodic
 * too (Sec. 2.3.3, S2): every (kx, kz) pencil is Fourier-transformed along y
 * and divided by its eigenvalue, the (0,0,0) mode set to 0. */
int ibm_poisson_solve(ibm_plan plan, const void *rhs, void *phi, void *stream,
                      ibm_info *info);

/* Poisson solve for callers that cannot allocate device memory.  The paper
 * has no counterpart: it exists for hosts that own the GPU's memory budget
 * (memory pools, frameworks that hand out only their own buffers) or must
 * not call cudaMalloc mid-run.  Same FP32 method, kernels and result as
 * ibm_poisson_solve on an IBM_FP32_REFINED plan with refine_iters steps, but
 * no plan: the workspace lives in one static 24 MiB device array that the
 * library holds on every GPU that loads it until the process exits, enough
 * for a 128^3 grid with one refinement step.  Larger grids return
 * IBM_ERR_ARG with the bytes needed, before any CUDA call.  rhs and phi are
 * distinct float fields [ny][nz][nx] in device memory (16-byte aligned).
 * status (optional, host memory) receives the solve's device error word
 * through a copy queued on `stream` after the solve: 0 when every bounded
 * wait of the solve completed, non-zero (bit 0: a wait gave up) when phi is
 * not valid.  Read it once the stream has reached the end of the call; with
 * pinned memory the copy is asynchronous, with pageable memory the call
 * returns only after the solve has finished.  The first call on a device
 * looks up the array's device address; make that first call before
 * capturing a stream into a CUDA graph.  All calls share the array and it
 * keeps the last call's contents: calls that overlap on the GPU race, so
 * serialise them (one stream, one host thread at a time). */
int ibm_poisson_solve_noalloc(int nx, int ny, int nz, const double h[3], int refine_iters,
                              const float *rhs, float *phi, int *status, void *stream);

/* Helmholtz solve, Eq. 2e (S1.1 + S1.2): (I - c L_h) u = rhs, c > 0, with the
 * wall rows selected by field_bc (Appendix B; IBM_FIELD_PERIODIC, and only
 * that, on an IBM_BC_TRIPLY_PERIODIC plan).  Eq. 2e is this system with
 * c = beta_n dt / Re.  rhs may equal u. */
int ibm_helmholtz_solve(ibm_plan plan, double c, int field_bc, const void *rhs,
                        void *u, void *stream, ibm_info *info);

/* The same solves with non-homogeneous wall data (Appendix B: the first and
 * last rows of each pencil carry the boundary values on their right-hand
 * sides; the paper's BC2.2 forms those terms from the 2D FFT of the ghost
 * planes, here they are added to a copy of rhs before the forward transform,
 * which is the same by linearity).  g_lo / g_hi are [nz][nx] planes in the
 * plan precision (device, 16-byte aligned) at the wall y = 0 / y = Ly; NULL
 * means 0 on that wall.
 *   ibm_poisson_solve_bc    q = dphi/dy at the walls (inhomogeneous
 *                           Neumann; the mean of the resulting right-hand
 *                           side is removed and reported as for
 *                           ibm_poisson_solve).
 *   ibm_helmholtz_solve_bc  g is the wall value of u for the Dirichlet kinds
 *                           (cell-centred: ghost = 2 g - u_0; wall faces: the
 *                           face value, written to plane 0 of u) and du/dy
 *                           at the wall for IBM_FIELD_CELL_NEUMANN.
 * rhs is not modified (the plan's scratch field holds the copy); rhs may
 * equal the output.  IBM_ERR_UNSUPPORTED on a triply periodic plan. */
int ibm_poisson_solve_bc(ibm_plan plan, const void *rhs, void *phi, const void *q_lo,
                         const void *q_hi, void *stream, ibm_info *info);
int ibm_helmholtz_solve_bc(ibm_plan plan, double c, int field_bc, const void *rhs,
                           void *u, const void *g_lo, const void *g_hi, void *stream,
                           ibm_info *info);

/* Interpolation, Eq. 2b: U[m] = sum over the kernel support of u_c(x) *
 * phi(dx/hx) phi(dy/hy) phi(dz/hz) for each component c on its own staggered
 * sub-grid, periodic in x and z.  X, U: [n][3]; u, v, w: fields. */
int ibm_interp(ibm_plan plan, int n, const void *X, const void *u, const void *v,
               const void *w, void *U, void *stream);

/* Spreading, Eq. 2d: f_c(x) += F_c(X) phi phi phi dV / (hx hy hz), accumulated
 * with atomics into fu, fv, fw (not cleared first).  X, F: [n][3]; dV: [n]. */
int ibm_spread(ibm_plan plan, int n, const void *X, const void *F, const void *dV,
               void *fu, void *fv, void *fw, void *stream);

/* State of the flow for ibm_substep (device pointers, plan precision). */
typedef struct {
  void *u, *v, *w, *p; /* velocity on faces and pressure, updated in place   */
  void *Nu, *Nv, *Nw;  /* advection term of the previous stage; read for the
                          zeta_n term and overwritten with this stage's      */
  double t;            /* time at the start of the stage; advanced by
                          (alpha_n + beta_n) dt                              */
} ibm_state;

/* Lagrangian markers for ibm_substep (device pointers, plan precision). */
typedef struct {
  int n;
  const void *X0; /* [n][3] reference positions                          */
  const void *dV; /* [n] volume of each marker                            */
  void *X;        /* [n][3] out: positions at the stage time (L2)         */
  void *Ud;       /* [n][3] out: surface velocity at the stage time (L2)  */
  void *F;        /* [n][3] out: Lagrangian force of the stage, or NULL   */
  int motion;     /* IBM_MOTION_*                                         */
  double params[4]; /* TRANSLATE: (Ux,Uy,Uz); HEAVE: (amplitude, period) */
} ibm_markers;

/* One RK stage (rk_stage = 1, 2, 3) of Eq. 2a-2h with the low-storage
 * coefficients of Rai & Moin (cited in Sec. 2.1; the paper does not print
 * them): E1 explicit terms, L2 marker update at the stage start time, L1
 * interpolation + force + spreading, three Helmholtz solves, divergence,
 * Poisson solve, projection and pressure update (E3).  nu = 1/Re.
 * Uses the plan's workspace; the plan precision sets the field type. */
int ibm_substep(ibm_plan plan, ibm_state *st, int rk_stage, double dt, double nu,
                ibm_markers *mk, void *stream, ibm_info *info);

/* Wall data of the inflow-outflow configuration (Sec. 3): a uniform inflow
 * v = v_in through the y = 0 face (u = w = 0 on that wall) and an outlet at
 * y = Ly advected with d phi/dt + c_out d phi/dy = 0.  u_out, w_out hold u
 * and w on the outlet wall, v_out the wall-normal velocity on the outlet
 * face: device planes [nz][nx] of the plan precision, 16-byte aligned,
 * owned by the caller, updated in place every stage. */
typedef struct {
  double v_in;   /* inflow speed (finite)                                   */
  double c_out;  /* outlet advection speed (finite, >= 0)                   */
  void *u_out, *v_out, *w_out;
} ibm_inout;

/* One RK stage as ibm_substep, with the inflow-outflow walls of ibm_inout
 * in place of the no-slip walls.  The stage first advances the outlet
 * values over its step (alpha_n + beta_n) dt by first-order upwinding from
 * the last interior plane and shifts v_out by a constant so that its mean
 * equals v_in (outflow = inflow; the Poisson right-hand side keeps zero
 * mean), and stores v = v_in on plane 0 of v.  Those values are the wall
 * data of the whole stage: the explicit terms (Laplacian ghosts 2 g - u,
 * advective fluxes through the walls), the divergence and the projection
 * see them; the Helmholtz increment solves need none (the data are the
 * same at both ends of the increment).  The paper gives the outlet's
 * discretisation only by reference; the upwind form is the reading used
 * here.  Returns IBM_ERR_ARG for NULL io, NULL or misaligned planes, a
 * non-finite v_in or a negative or non-finite c_out; otherwise as
 * ibm_substep. */
int ibm_substep_inout(ibm_plan plan, ibm_state *st, const ibm_inout *io, int rk_stage, double dt,
                      double nu, ibm_markers *mk, void *stream, ibm_info *info);

/* ---------------------------------------------------------------------------
 * Batches: many independent grids solved in one CUDA-graph launch
 * ------------------------------------------------------------------------- */

/* Create a batch of `count` independent problems; dims = [count][3]
 * (nx, ny, nz), h = [count][3].  All share precision and refine_iters. */
int ibm_batch_create(int count, const int *dims, const double *h, int precision,
                     int refine_iters, ibm_batch *out);
int ibm_batch_destroy(ibm_batch batch);
/* Poisson-solve every problem: rhs[i], phi[i] are device fields of problem
 * i.  The whole batch is captured once into a CUDA graph per distinct
 * pointer set and replayed as a single graph launch on `stream`. */
int ibm_batch_poisson(ibm_batch batch, const void *const *rhs, void *const *phi,
                      void *stream);
/* One RK stage (as ibm_substep, Eq. 2a-2h with the immersed boundary of
 * Sec. 2.3.2) of every instance: states[i] is instance i's state and
 * markers[i] its marker set (n = 0, or markers == NULL, for none).  The
 * instances' stages run as concurrent branches of one CUDA graph launch on
 * `stream`.  When no instance's markers move (IBM_MOTION_STATIC) the graph
 * is kept per set of pointers, stage, dt and nu and replayed by later calls;
 * moving markers (whose positions are evaluated at the stage start time on
 * the host) are captured anew on every call.  The first call of a plan
 * allocates its stage buffers.  Every state's t is advanced as by
 * ibm_substep.  Errors as ibm_substep, per instance. */
int ibm_batch_substep(ibm_batch batch, ibm_state *states, ibm_markers *markers, int rk_stage,
                      double dt, double nu, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solve requests with HBM-based admission
 * ------------------------------------------------------------------------- */

enum { IBM_REQ_POISSON = 0, IBM_REQ_HELMHOLTZ = 1, IBM_REQ_SUBSTEP = 2 };

/* Where a request's data live (ibm_request.data). */
enum {
  IBM_DATA_HOST_FP64 = 0, /* host FP64 arrays: staged through pinned memory and
                             converted to the plan precision on the device    */
  IBM_DATA_DEVICE = 1     /* device arrays in the plan precision (float for
                             IBM_FP32_REFINED, double for IBM_FP64), 16-byte
                             aligned: no staging, no conversion                */
};

typedef struct {
  int kind;              /* IBM_REQ_*                                         */
  int nx, ny, nz;
  double h[3];
  int precision;         /* IBM_FP64 / IBM_FP32_REFINED                       */
  int refine_iters;
  double c;              /* Helmholtz coefficient                             */
  int field_bc;          /* Helmholtz wall rows                               */
  const void *in;        /* input: rhs [ny][nz][nx] (Poisson, Helmholtz) or
                            u,v,w,p packed [4][ny][nz][nx] (substep); host
                            FP64 or device, by `data`                         */
  void *out;             /* output, same shape as `in` (distinct from it)      */
  int n_markers;         /* substep: markers                                  */
  const void *X0;        /* substep: [n][3], host FP64 or device, by `data`   */
  const void *dV;        /* substep: [n], likewise                            */
  int motion;
  double params[4];
  double dt, nu;         /* substep                                           */
  int rk_stage;          /* substep                                           */
  int data;              /* IBM_DATA_*                                        */
} ibm_request;

typedef struct {
  int status;            /* IBM_OK, IBM_PENDING or an error code              */
  double queue_ms;       /* submit -> admission                               */
  double device_ms;      /* device time of the solve (events)                 */
  double total_ms;       /* submit -> completion seen by the server           */
  double removed_mean;
} ibm_result;

/* Create a server that admits requests while their device memory fits in
 * hbm_budget_bytes, keeps plans resident per shape and runs admitted work
 * on n_streams CUDA streams so that requests overlap on the device.
 * max_queue bounds the pending queue (ibm_submit returns IBM_ERR_BUSY when
 * full). */
int ibm_server_create(size_t hbm_budget_bytes, int n_streams, int max_queue,
                      ibm_server *out);
int ibm_server_destroy(ibm_server server);
/* Non-blocking: copies the request descriptor (not the data; `in`, `out`
 * and the marker arrays must stay valid and, for IBM_DATA_DEVICE, unchanged
 * until completion) and returns a ticket.  A substep request's `out` receives
 * the stage's u, v, w, p; with IBM_DATA_DEVICE the stage runs on `out`
 * itself after a device copy of `in`. */
int ibm_submit(ibm_server server, const ibm_request *req, uint64_t *ticket);
/* Non-blocking: IBM_PENDING while running; IBM_OK (result filled, `out`
 * written) once done; an error code for a failed request.  A finished
 * ticket is released by the poll that reports it. */
int ibm_poll(ibm_server server, uint64_t ticket, ibm_result *out);
/* Blocking variant of ibm_poll with a deadline (seconds). */
int ibm_wait(ibm_server server, uint64_t ticket, double timeout_s, ibm_result *out);
/* Cancel a request that has not been admitted yet. */
int ibm_cancel(ibm_server server, uint64_t ticket);

/* Thread-local description of the last error on this thread. */
const char *ibm_last_error(void);
/* Library version string. */
const char *ibm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H */
