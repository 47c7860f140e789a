/*
 * rmt.h -- C ABI of the GB300 (sm_103a) per-timestep grid update of the 3D reference map
 * technique for fluid-structure interaction (Lin, Derr & Rycroft, arXiv 2104.00095).
 *
 * One opaque grid holds one simulation: a fixed Cartesian grid (cell-centred velocity u,
 * density rho and per-body reference map xi; nodal pressure p) with any number of
 * immersed neo-Hookean bodies.  All state lives in device memory owned by the library.
 * Every call returns an rmt_status; errors are sticky per grid (after an error only
 * rmt_read_fields, rmt_last_error and rmt_destroy_grid are accepted).
 *
 * Layouts (all reads and writes are FP64, whatever the compute precision):
 *   cell field        [nz][ny][nx], x fastest
 *   vector cell field [3][nz][ny][nx]
 *   nodal field       [nnz][nny][nnx], nn_d = n_d + 1 on a walled axis, n_d on a periodic one
 *   face field, d     [nz][ny][nx+1] for d = x (and likewise for y, z): n_d + 1 faces along d;
 *                     on a periodic axis the first and last face are the same face
 * Per-body fields (XI, PHI, LAYER) cover the whole grid; cells outside the body's band
 * read NaN (XI, PHI) or -1 (LAYER).
 */
#ifndef RMT_H
#define RMT_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmt_grid rmt_grid;

typedef enum {
  RMT_OK = 0,
  RMT_EINVAL = 1,       /* bad argument or descriptor                                  */
  RMT_ENOMEM = 2,       /* device or host allocation failed                            */
  RMT_ECUDA = 3,        /* a CUDA call failed (message in rmt_last_error)              */
  RMT_ESTATE = 4,       /* call not allowed now (after an error, or add after a step)  */
  RMT_ENOCONVERGE = 5,  /* a multigrid solve missed its tolerance within its cycle cap */
  RMT_EDIVERGED = 6,    /* non-finite velocity detected                                */
  RMT_ETIMEOUT = 7,     /* reserved for bounded device-side waits (none in this build)  */
  RMT_EDEGENERATE = 8,  /* a least-squares extrapolation stayed degenerate at r_s = 4  */
  RMT_ERANGE = 9        /* FP32 form: a body's band came within 3 cells of the point half a
                           period from its centre on a periodic axis (the reference map is
                           stored relative to one periodic image of the grid around the body)*/
} rmt_status;

enum { RMT_BC_NOSLIP = 0, RMT_BC_PERIODIC = 1 };
enum { RMT_PREC_FP64 = 0, RMT_PREC_FP32_REFINE = 1 };
enum { RMT_SHAPE_SPHERE = 0, RMT_SHAPE_ELLIPSOID = 1 };

/* Simulation set-up: the parameters of the paper's Table "pars" plus the grid, the
 * boundary conditions and the solver controls (SI "Configuring a simulation"). */
typedef struct {
  int n[3];               /* cells per axis; the spacing must be isotropic (main text, Results) */
  double lo[3], hi[3];    /* domain corners                                                   */
  int bc[6];              /* RMT_BC_* for faces -x,+x,-y,+y,-z,+z; periodic in pairs          */
  double wall_u[6][3];    /* no-slip wall velocity (tangential only; a lid)                   */
  double rho_f, mu;       /* fluid density and viscosity                                      */
  double eps_h;           /* half blur-zone width epsilon, in cells                           */
  int band_layers;        /* extrapolation layers (1..8)                                      */
  double dt;              /* time step; <= 0: min(0.2h, 0.8 rho_min h^2/(6 mu_max),
                             0.5 h / sqrt(G_max/rho_min))                                     */
  double gravity[3];      /* body force is (rho - rho_f) g                                    */
  int precision;          /* RMT_PREC_FP64, or FP32 bulk: FP32 fields (reference maps stored as
                             displacements from the cell centres) and V-cycles, with the
                             projections' residuals, right-hand sides and solutions refined
                             in two-float arithmetic (hi + lo FP32 pairs)                    */
  double mg_rtol;         /* relative residual target of both Poisson solves (<=0: 1e-12)    */
  int mg_max_cycles;      /* cap on V-cycles per solve (<=0: 60)                              */
  int mg_fixed_cycles;    /* > 0: run exactly this many MAC cycles, no residual checks (no host
                             synchronisation inside rmt_step)                                 */
  int mg_fixed_cycles_fe; /* the same for the FE solve (<= 0: mg_fixed_cycles)                */
  void* cuda_stream;      /* cudaStream_t all work is ordered on (NULL: legacy stream)        */
  double wall_dw;         /* wall-repulsion threshold distance d_w (<= 0: one grid spacing;
                             SI "Contact with a wall")                                        */
} rmt_grid_desc;

/* One immersed body (main text "Hyperelastic formulation", "Swimming"). The reference
 * configuration is the body at t = 0: xi^0 = x inside phi_0 < 0. */
typedef struct {
  int shape;                          /* RMT_SHAPE_*                                         */
  double center[3], semi_axes[3];     /* sphere: semi_axes[0] is the radius                  */
  double rot[9];                      /* body -> world rotation, row-major                   */
  double rho_s, G, mu_a, gamma_t;     /* density, shear modulus, artificial viscosity, blur
                                         viscosity factor (Table pars)                       */
  double active_A, active_omega, active_len; /* active stress A sin(2 pi X/len - omega t)
                                         along the body x axis; A = 0: passive            */
  double rep_A;                       /* wall-repulsion acceleration A_rep (0: none): cells of
                                         the body nearer than d_w to a no-slip wall get
                                         A_rep times the transition factor of eq. wall_acc
                                         along the wall's inward normal (SI "Contact with a
                                         wall"); see rmt_wall_repulsion                   */
} rmt_solid_desc;

/* Creates a grid.  Validates the descriptor; allocates the device state lazily on the first
 * step/read/write.  out receives the handle (caller destroys it).  Errors: RMT_EINVAL, also
 * for (n_x + 1)(n_y + 1)(n_z + 1) >= 2^31 (cell, node and face indices are 32-bit; such a grid
 * would need more than 400 GB of device memory). */
rmt_status rmt_create_grid(const rmt_grid_desc* desc, rmt_grid** out);

/* Registers a body before the first step (SI "Initialization": xi^0 = x where
 * phi_0(x) < 0, then extrapolation, phi and rho).  solid_id receives its index. */
rmt_status rmt_add_solid(rmt_grid* g, const rmt_solid_desc* s, int* solid_id);

/* Advances nsteps timesteps of the 13-step algorithm (SI "Timestepping algorithm").
 * Work is enqueued on the grid's stream; with mg_fixed_cycles = 0 each Poisson solve reads
 * its residual norm back to the host once per cycle, and the call waits for its steps and
 * reports their failures.  With fixed cycle counts nothing waits: every step copies the grid's
 * device error words to pinned host memory as its last operation, and a later rmt_step (or
 * rmt_batch_sync, or the server's poll) reports a failure found there: RMT_EDIVERGED (a NaN or
 * infinity reached the mean or norm that every pressure solve takes of its right-hand side and
 * solution), RMT_EDEGENERATE, RMT_ERANGE.  Errors: those of the status list; RMT_ESTATE after a
 * sticky error. */
rmt_status rmt_step(rmt_grid* g, int nsteps);

/* Initial pressure iterations (SI "Initialization" item 2), before the first step: a timestep
 * from the initial state is run with the current estimate of p^{-1/2}; its p^{1/2} becomes
 * the next estimate and every other change is undone (velocity, density, reference maps,
 * time).  Stops once the estimate moves by at most tol relative (||p_k - p_{k-1}||_2 <=
 * tol ||p_k||_2; the paper names a tolerance on the divergence of u^0, which these iterations
 * do not change) or after max_iters iterations; iters_out receives the count.  Synchronous.
 * Errors: RMT_EINVAL, RMT_ESTATE (after the first step, or for a batch member), and those of
 * rmt_step. */
rmt_status rmt_init_pressure(rmt_grid* g, int max_iters, double tol, int* iters_out);

enum {
  RMT_F_U = 1, RMT_F_P = 2, RMT_F_RHO = 3, RMT_F_XI = 4, RMT_F_PHI = 5, RMT_F_LAYER = 6,
  /* intermediates of the last step (same meaning as the oracle's) */
  RMT_F_DIVTAU_N = 20, RMT_F_DIVTAU_H = 21, RMT_F_UFACE_X = 22, RMT_F_UFACE_Y = 23,
  RMT_F_UFACE_Z = 24, RMT_F_MAC_Q = 25, RMT_F_ADV_U = 26, RMT_F_USTAR = 27, RMT_F_PSI = 28,
  RMT_F_RHO_HALF = 29, RMT_F_XI_HALF = 30, RMT_F_UMAC_X = 31, RMT_F_UMAC_Y = 32,
  RMT_F_UMAC_Z = 33,
  RMT_F_REPULSION = 34 /* wall-repulsion acceleration that entered the last step's u* (3 N) */
};

/* Number of FP64 values of a field (see layouts above), or -1 for an unknown field. */
long rmt_field_len(rmt_grid* g, int field);

/* Copies a field as FP64 into dst (dst_bytes >= 8 * rmt_field_len).  dst is host memory
 * (dst_is_device = 0; pinned or pageable) or device memory on the grid's GPU.  Synchronises
 * the grid's stream.  solid_id selects the body for XI, PHI, LAYER, XI_HALF. */
rmt_status rmt_read_fields(rmt_grid* g, int field, int solid_id, void* dst, size_t dst_bytes,
                           int dst_is_device);

/* Overwrites U (3 N values), P (nodal) or XI of one body (3 N values, NaN = no primary value)
 * from FP64 src.  Writing XI re-classifies, re-marks the layers, re-extrapolates and re-blends
 * rho, exactly as initialisation does.  Asynchronous on the grid's stream for device src. */
rmt_status rmt_write_fields(rmt_grid* g, int field, int solid_id, const void* src,
                            size_t src_bytes, int src_is_device);

/* The same two calls with FP32 host or device buffers (dst_bytes / src_bytes >= 4 *
 * rmt_field_len): the FP64 values rounded to float, or converted from float.  For U and P of an
 * RMT_PREC_FP32_REFINE grid these are the stored values themselves, copied without conversion
 * (half the bytes of the FP64 calls, and no rounding either way).  Same synchronisation and
 * errors as rmt_read_fields / rmt_write_fields, except that writing U or P of such a grid from
 * page-locked host memory (cudaHostAlloc / cudaMallocHost / registered) leaves the copy
 * asynchronous on the grid's stream: the caller must not modify src until a call that
 * synchronises the grid (a read, for one) has returned. */
rmt_status rmt_read_fields_float(rmt_grid* g, int field, int solid_id, void* dst, size_t dst_bytes,
                                 int dst_is_device);
rmt_status rmt_write_fields_float(rmt_grid* g, int field, int solid_id, const void* src,
                                  size_t src_bytes, int src_is_device);

/* Multigrid cycles used by the last step's MAC (which = 0) and FE (which = 1) solves. */
int rmt_last_cycles(rmt_grid* g, int which);
/* The time step in use (after initialisation). */
double rmt_dt(rmt_grid* g);

/* Solver schedule options (any time): "mac_pre", "mac_post" (red-black Gauss-Seidel sweeps
 * before / after the coarse correction, 0..16, default 3), "fe_pre", "fe_post" (weighted Jacobi
 * sweeps, default 2), "fe_omega" (Jacobi weight in (0,2), default 0.9), "mac_omega" (relaxation
 * factor of the red-black sweeps in (0,2), default 1), "mac_inner", "fe_inner"
 * (V-cycles on the storage-precision correction equation per high-precision residual, 1..16,
 * default 1), "mac_block", "fe_block" (rows of 32 threads per block of the multigrid level
 * kernels: 1, 2, 4 or 8, default 4), "mac_cycles", "fe_cycles" (replace the descriptor's
 * mg_fixed_cycles / mg_fixed_cycles_fe), "mac_warm", "fe_warm" (nonzero: each solve starts from the
 * previous step's solution instead of zero; default 0; both projections solve for increments of
 * the pressure, which change quickly while the flow starts up, so this helps only once they vary
 * slowly from step to step), "mac_zchunk", "fe_zchunk" (planes a block
 * of the finest level's fused red-black sweep / FE tiles marches; 0, the default, picks the
 * length that fills whole waves of resident blocks), "mac_coarse_pre", "mac_coarse_post",
 * "fe_coarse_pre", "fe_coarse_post" (sweeps on the levels below the finest, 0..16; default: the
 * finest level's), "mac_sweep" (FP32 grids: 1, the default, runs each red-black sweep of a
 * level with n_x % 4 == 0, even periodic sides, n_x >= 64 and at least 2^20 cells as one fused
 * pass over both colours; 2 does so on every level with n_x % 4 == 0 and even periodic sides; 0
 * runs one pass per colour everywhere; all give the same sweep), "graph" (nonzero: with fixed
 * cycle counts, rmt_step replays a captured CUDA graph of the step instead of launching its
 * kernels one by one; the results are the same).  Cycle counts (mg_fixed_cycles,
 * rmt_last_cycles) count V-cycles.
 * Fault injection from the host, for testing failure handling (no device fault is involved):
 * "inject_nan_step" (k >= 0: before step k runs, one velocity value is overwritten with NaN, as
 * a diverging scheme would leave it; -1 turns it off), "inject_alloc" (k >= 0, before the first
 * step: the grid's k-th device allocation fails as cudaMalloc would, giving RMT_ENOMEM).
 * Errors: RMT_EINVAL, RMT_ESTATE for a batch member (and for inject_alloc after allocation). */
rmt_status rmt_set_option(rmt_grid* g, const char* name, double value);

/* A_rep of SI "Contact with a wall" for one body: the largest of U_safe^2/d_w (a safety
 * floor; the paper uses U_safe about 4.5), V U^2 / (2 d_w^2 L_min^2) (stops a body of volume V
 * approaching the wall at speed U within d_w, taking d_w L_min^2 as the breached volume, L_min
 * the body's smallest length) and |rho_s - rho_f| V g / (rho_s d_w L_min^2) (carries its net
 * weight when it rests on the wall).  Pure function; no grid needed. */
double rmt_wall_repulsion(double V, double U, double d_w, double L_min, double rho_s, double rho_f, double g,
                          double U_safe);

/* Diagnostics of body solid_id at the grid's current time (main text "Swimming"; SI "Swimming
 * statistics"; SI "Pre-stretched sphere", eq. elas), written to out[7] (host memory):
 *   out[0..3)  centroid velocity: sum w u / sum w over the cells that hold the body's reference
 *              map, w = 1 - H_eps(phi) its solid fraction (eq. heaviside);
 *   out[3]     active power: -sum w sigma_a : grad u h^3, sigma_a the active stress of the stress
 *              model at the cell centre and time t (main text "Swimming"), built from F =
 *              (grad xi)^-1 by centred differences of xi, grad u by centred differences of the
 *              cell velocities (periodic wrap, mirrored ghost at a wall);
 *   out[4]     volume: sum w h^3;
 *   out[5]     elastic energy: sum w G/2 (tr(F^T F) - 3 - 2 ln J) h^3, J = det F (eq. elas);
 *   out[6]     RMS of J - 1 over the body (weights w).
 * A cell whose grad xi lacks a neighbour value or has det <= 0 adds to out[0..5) only.  The
 * sums are taken in FP64 in a fixed order (deterministic).  A passive body (active_A = 0) gives
 * zero power.  Synchronous (a batch member waits for its batch's queued steps).
 * Errors: RMT_EINVAL (null, bad solid id), RMT_ECUDA. */
rmt_status rmt_body_stats(rmt_grid* g, int solid_id, double out[7]);

/* Autotuner of the two multigrid solves (no paper counterpart: the paper's multigrid library
 * is not described).  On the right-hand sides of the grid's last step (RMT_ESTATE before the
 * first step) it tries, per solver, smoother sweeps before/after the coarse correction (1..4
 * for the 7-point solve, 1..3 for the nodal one), the relaxation factor of the red-black sweeps
 * (1.0, 1.15), the Jacobi weight of the nodal smoother (0.8, 0.9, 1.0) and 1, 2 or 4 V-cycles per
 * high-precision residual: for each, it counts the V-cycles
 * needed to reach the relative residual rtol and times that many with CUDA events.  It then
 * times the block height of the level kernels (1, 2, 4, 8 rows of 32 threads) for the fastest
 * schedule, and the z-chunk length of the finest level's plane-marching stencil tiles (the fused
 * red-black sweep, the FE tiles: the wave-filling default, 8, 16, 32, 64, 128 planes).  The
 * winners are applied with rmt_set_option, including the cycle counts ("mac_cycles",
 * "fe_cycles") and the chunks ("mac_zchunk", "fe_zchunk"), so that later steps run fixed-cycle
 * without host synchronisation.  The solvers' solution buffers are overwritten (fields MAC_Q and PSI read
 * afterwards show a tuning solve); the simulation state is not changed.  Synchronous.
 * Errors: RMT_EINVAL (rtol outside (0,1)), RMT_ESTATE, RMT_ENOCONVERGE (no schedule reached rtol
 * within 40 cycles), RMT_ECUDA. */
typedef struct {
  int mac_pre, mac_post, mac_inner, mac_block, mac_cycles;
  int fe_pre, fe_post, fe_inner, fe_block, fe_cycles;
  double fe_omega;
  double mac_ms, fe_ms; /* time of one solve with the chosen settings */
  int trials;           /* schedules and shapes tried */
  int mac_zchunk, fe_zchunk; /* z-chunk of the finest level's plane-marching tiles (0: default) */
  double mac_omega;          /* relaxation factor of the red-black sweeps */
} rmt_tune_result;
rmt_status rmt_autotune(rmt_grid* g, double rtol, rmt_tune_result* out);

/* Extrapolates one body's reference map on caller-owned device buffers without allocating
 * anything (the paper has no counterpart: this serves callers that cannot allocate device
 * memory while they run, e.g. because their own pool owns the memory budget, or because
 * cudaMalloc may synchronise the device in the middle of their pipeline).  It runs the same
 * classification, layer marking and least-squares extrapolation as initialisation and
 * rmt_write_fields(RMT_F_XI), in FP64, on the grid and body that desc and s describe
 * (desc: n, lo, hi, bc, eps_h, band_layers are read).
 *   xi_in     device, 3 N doubles ([3][nz][ny][nx]); finite entries are candidate primary
 *             values, NaN marks "no value" (as rmt_write_fields).  Not modified.
 *   xi_out    device, 3 N doubles: the extrapolated map, NaN outside the band.
 *   phi_out   device, N doubles: phi_0(xi) in the band, NaN outside.
 *   layer_out device, N signed chars: layer labels, -1 outside the band.
 *   stream    cudaStream_t the work is ordered on; the call synchronises it before returning.
 * Scratch (band list, bounding box, counters) lives in one static device array sized for grids
 * of at most 2^21 cells (e.g. 128^3); larger grids return RMT_EINVAL before any work.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress), so make the
 * first call on each device outside any stream capture.  All calls in the process share the
 * array: calls that overlap on the GPU (other streams, other threads) race; serialise them.
 * Returns RMT_EDEGENERATE when a fit stayed degenerate, RMT_ECUDA on a CUDA error. */
rmt_status rmt_extrapolate_noalloc(const rmt_grid_desc* desc, const rmt_solid_desc* s, const double* xi_in,
                                   double* xi_out, double* phi_out, signed char* layer_out, void* stream);

/* Device bytes that a grid described by desc with nsolids bodies requests from cudaMalloc over
 * its lifetime: every field, scratch array and both multigrid hierarchies, each allocation
 * counted in 256-byte units.  0 for an invalid description.  The serving runtime admits jobs by
 * this number.  (The paper has no counterpart: its runs own whole MPI ranks.) */
size_t rmt_grid_footprint(const rmt_grid_desc* desc, int nsolids);
/* Device bytes the grid has requested so far; equals rmt_grid_footprint after initialisation. */
size_t rmt_grid_device_bytes(const rmt_grid* g);

/* ---- batched stepping (no paper counterpart: the paper runs one simulation per MPI job) ----
 * A batch advances several independent grids together, each step of all members being one
 * launch of an instantiated CUDA graph.  Every member's step is captured on its own branch of
 * the graph, so the kernels of different members run concurrently on the GPU; the graph is
 * captured once per membership (two graphs: the reference-map buffers alternate between two
 * parities) and replayed.  Members need fixed multigrid cycle counts (mg_fixed_cycles > 0 and
 * mg_fixed_cycles_fe > 0, so that a step never waits for the host) and profiling off.  While a
 * grid is a member, rmt_step, rmt_write_fields, rmt_set_option and rmt_destroy_grid on it return
 * RMT_ESTATE, and rmt_read_fields first waits for the batch's stream.  Members share no data, so
 * every member's result is the same as when it is stepped alone.
 *   rmt_batch_create: stream = cudaStream_t the step graphs are launched on (may be null).
 *   rmt_batch_add:    initialises the grid if needed; synchronous.  RMT_EINVAL for a grid
 *                     without fixed cycle counts or already a member.
 *   rmt_batch_remove: waits for the batch's work; the grid keeps its state and can step alone.
 *   rmt_batch_step:   asynchronous; nsteps launches of the step graph.
 *   rmt_batch_sync:   waits, then reads every member's error flag; the first error is returned
 *                     (the member's rmt_last_error has the message).
 *   rmt_batch_destroy: removes all members (they are not destroyed). */
typedef struct rmt_batch rmt_batch;
rmt_status rmt_batch_create(void* cuda_stream, rmt_batch** out);
rmt_status rmt_batch_add(rmt_batch* b, rmt_grid* g);
rmt_status rmt_batch_remove(rmt_batch* b, rmt_grid* g);
rmt_status rmt_batch_step(rmt_batch* b, int nsteps);
rmt_status rmt_batch_sync(rmt_batch* b);
int rmt_batch_size(const rmt_batch* b);
rmt_status rmt_batch_destroy(rmt_batch* b);
const char* rmt_batch_last_error(const rmt_batch* b);

/* ---- serving: continuous batching of simulation jobs (no paper counterpart) ----------------
 * rmt_server_submit queues a job (grid description with fixed cycle counts, bodies, number of
 * steps); its footprint (rmt_grid_footprint) must fit the budget.  Each rmt_server_poll
 *   1. evicts the running jobs whose error words (copied to the host by every step) report a
 *      failure: a diverged velocity (RMT_EDIVERGED), a degenerate extrapolation: the job is
 *      marked failed, its grid destroyed and its memory returned to the budget, and the others
 *      carry on; then retires the running jobs whose last step has been launched: completion
 *      time = when the GPU finished that step (CUDA event), then the job's error words are read;
 *   2. admits queued jobs in arrival order while their footprint fits next to the resident
 *      jobs (a job that does not fit waits; later, smaller jobs may pass it); an admitted job's
 *      grid is created, initialised and added to the server's batch;
 *   3. launches one batched step of all running jobs, with at most two steps in flight.
 * A job that fails (bad description, allocation, divergence, degenerate extrapolation) is
 * marked failed and the others carry on.  Finished jobs keep their fields on the device, readable through
 * rmt_server_job_grid, until rmt_server_release, and count against the budget until then.
 * Times are seconds since rmt_server_create (rmt_server_clock).  rmt_server_set_option applies
 * rmt_set_option(name, value) to every job grid at admission. */
typedef struct rmt_server rmt_server;
enum { RMT_JOB_QUEUED = 0, RMT_JOB_RUNNING = 1, RMT_JOB_DONE = 2, RMT_JOB_FAILED = 3 };
typedef struct {
  int state;           /* RMT_JOB_* */
  rmt_status status;   /* RMT_OK, or why the job failed */
  long steps_done, steps_total;
  double t_submit, t_admit, t_done;  /* seconds; -1 while not reached */
  size_t device_bytes; /* footprint charged against the budget */
} rmt_job_info;
rmt_status rmt_server_create(size_t budget_bytes, void* cuda_stream, rmt_server** out);
rmt_status rmt_server_set_option(rmt_server* s, const char* name, double value);
rmt_status rmt_server_submit(rmt_server* s, const rmt_grid_desc* desc, const rmt_solid_desc* solids, int nsolids,
                             long nsteps, int* job_id);
rmt_status rmt_server_poll(rmt_server* s, int* n_running, int* n_queued);
rmt_status rmt_server_job(rmt_server* s, int job_id, rmt_job_info* info);
rmt_grid* rmt_server_job_grid(rmt_server* s, int job_id);
rmt_status rmt_server_release(rmt_server* s, int job_id);
size_t rmt_server_resident_bytes(const rmt_server* s);
const char* rmt_server_last_error(const rmt_server* s);
typedef struct {
  long batched_steps;   /* batched steps launched */
  long graph_captures;  /* step graphs captured and instantiated (two per membership) */
  double capture_s;     /* host seconds spent capturing and instantiating them */
  double admit_s;       /* host seconds spent admitting jobs (grid creation and initialisation) */
  double retire_s;      /* host seconds spent retiring jobs (waiting for their last step, error check) */
  double cell_steps;    /* cells x steps launched for all jobs */
} rmt_server_stats_t;
rmt_status rmt_server_stats(const rmt_server* s, rmt_server_stats_t* out);
double rmt_server_clock(const rmt_server* s);
double rmt_server_cell_steps(const rmt_server* s); /* cells x steps launched for all jobs */
rmt_status rmt_server_destroy(rmt_server* s);

/* Total number of CUDA kernels this library has launched in this process (all grids).  A
 * replayed step graph counts its kernel nodes. */
long rmt_kernel_launches(void);

/* Timing of the step's stages and of the finest-level multigrid kernels with CUDA events on
 * the grid's stream.  rmt_profile(g, 1) clears and starts collecting, rmt_profile(g, 0) stops.
 * Entries: 0..12 are stages of the timestep (each a group of kernels), 13..17 single kernels
 * (7-point smoother colour, 7-point high-precision residual, 27-point smoother colour, 27-point
 * high-precision residual, fused red-black sweep; high precision is FP64 in the FP64 form and
 * two-float in the FP32 form).  rmt_profile_read synchronises the stream and returns the
 * accumulated time, the number of timed launches and, for 13..17, the algorithmic bytes of one
 * launch (0 else). */
rmt_status rmt_profile(rmt_grid* g, int enable);
int rmt_profile_entries(void);
const char* rmt_profile_name(int entry);
rmt_status rmt_profile_read(rmt_grid* g, int entry, double* total_ms, long* launches, double* bytes_per_launch);

rmt_status rmt_destroy_grid(rmt_grid* g);
const char* rmt_last_error(const rmt_grid* g);

#ifdef __cplusplus
}
#endif
#endif
