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
  RMT_ETIMEOUT = 7,     /* reserved for bounded device-side waits                      */
  RMT_EDEGENERATE = 8   /* a least-squares extrapolation stayed degenerate at r_s = 4  */
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
  int precision;          /* RMT_PREC_FP64, or FP32 bulk with FP64 multigrid refinement      */
  double mg_rtol;         /* relative residual target of both Poisson solves (<=0: 1e-12)    */
  int mg_max_cycles;      /* cap on V-cycles per solve (<=0: 60)                              */
  int mg_fixed_cycles;    /* > 0: run exactly this many MAC cycles, no residual checks (no host
                             synchronisation inside rmt_step)                                 */
  int mg_fixed_cycles_fe; /* the same for the FE solve (<= 0: mg_fixed_cycles)                */
  void* cuda_stream;      /* cudaStream_t all work is ordered on (NULL: legacy stream)        */
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
} rmt_solid_desc;

/* Creates a grid.  Validates the descriptor; allocates the device state lazily on the first
 * step/read/write.  out receives the handle (caller destroys it).  Errors: RMT_EINVAL. */
rmt_status rmt_create_grid(const rmt_grid_desc* desc, rmt_grid** out);

/* Registers a body before the first step (SI "Initialization": xi^0 = x where
 * phi_0(x) < 0, then extrapolation, phi and rho).  solid_id receives its index. */
rmt_status rmt_add_solid(rmt_grid* g, const rmt_solid_desc* s, int* solid_id);

/* Advances nsteps timesteps of the 13-step algorithm (SI "Timestepping algorithm").
 * Work is enqueued on the grid's stream; with mg_fixed_cycles = 0 each Poisson solve reads
 * its residual norm back to the host once per cycle. */
rmt_status rmt_step(rmt_grid* g, int nsteps);

enum {
  RMT_F_U = 1, RMT_F_P = 2, RMT_F_RHO = 3, RMT_F_XI = 4, RMT_F_PHI = 5, RMT_F_LAYER = 6,
  /* intermediates of the last step (same meaning as the oracle's) */
  RMT_F_DIVTAU_N = 20, RMT_F_DIVTAU_H = 21, RMT_F_UFACE_X = 22, RMT_F_UFACE_Y = 23,
  RMT_F_UFACE_Z = 24, RMT_F_MAC_Q = 25, RMT_F_ADV_U = 26, RMT_F_USTAR = 27, RMT_F_PSI = 28,
  RMT_F_RHO_HALF = 29, RMT_F_XI_HALF = 30, RMT_F_UMAC_X = 31, RMT_F_UMAC_Y = 32,
  RMT_F_UMAC_Z = 33
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

/* Multigrid cycles used by the last step's MAC (which = 0) and FE (which = 1) solves. */
int rmt_last_cycles(rmt_grid* g, int which);
/* The time step in use (after initialisation). */
double rmt_dt(rmt_grid* g);

/* Solver schedule options (any time): "mac_pre", "mac_post" (red-black Gauss-Seidel sweeps
 * before / after the coarse correction, 0..16, default 3), "fe_pre", "fe_post" (weighted Jacobi
 * sweeps, default 2), "fe_omega" (Jacobi weight in (0,2), default 0.9), "mac_inner", "fe_inner"
 * (V-cycles on the storage-precision correction equation per FP64 residual, 1..16, default 1).  Cycle
 * counts (mg_fixed_cycles, rmt_last_cycles) count V-cycles.  Errors: RMT_EINVAL. */
rmt_status rmt_set_option(rmt_grid* g, const char* name, double value);

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

/* Total number of CUDA kernels this library has launched in this process (all grids). */
long rmt_kernel_launches(void);

/* Timing of the step's stages and of the finest-level multigrid kernels with CUDA events on
 * the grid's stream.  rmt_profile(g, 1) clears and starts collecting, rmt_profile(g, 0) stops.
 * Entries: 0..12 are stages of the timestep (each a group of kernels), 13..16 single kernels
 * (7-point smoother colour, 7-point FP64 residual, 27-point smoother colour, 27-point FP64
 * residual).  rmt_profile_read synchronises the stream and returns the accumulated time, the
 * number of timed launches and, for 13..16, the algorithmic bytes of one launch (0 else). */
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
