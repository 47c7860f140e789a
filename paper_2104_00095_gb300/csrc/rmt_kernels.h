// Host-side launchers of the RMT kernels (explicitly instantiated for float and double).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rmt_common.cuh"

// streaming multiprocessors of the current device (its attribute, read once per device); launch
// widths are multiples of it
int sm_count();

// Planes per thread column of a column-marching kernel over `units` points (cap at most): one
// plane on small grids, where a column's planes would only follow one another, and more once
// the columns alone give every SM a full set of resident threads.
inline int column_chunk(long units, int cap) {
  const long c = units / ((long)sm_count() * 2048);
  return c < 1 ? 1 : (c > cap ? cap : (int)c);
}

// A multigrid right-hand side or solution as the step kernels see it.  FP64 mode: the FP64
// array d.  FP32 mode: two-float pairs, value = h + l (d is null), so that no FP64 arithmetic
// runs in the FP32 step.
struct MGVec {
  double* d;
  float* h;
  float* l;
};

// face-array bundle: vector value at every d-face (3 comps) for d = 0..2
template <typename T>
struct Faces3 {
  T* v[3][3];  // v[d][a]
};

// ---- flow (rmt_flow.cu) -------------------------------------------------------------
// bbs: band boxes of the bodies (6 ints each, stride ints apart) of the time level of views;
// list (N ints) and count: scratch for the cells a band reaches; rows: nine cell arrays of
// scratch for the face rows of those cells (the Godunov slope arrays, free at both stress passes)
// t: device pointer to the simulated time; the stress is evaluated at *t + toff
template <typename T>
cudaError_t launch_stress_div(const Geo& g, const T* u, const Body* bodies, const BodyView<T>* views, int nb,
                              const int* bbs, int bstride, const double* t, double toff, T* out, int* list,
                              int* count, T* const rows[9], cudaStream_t s);
void launch_tick(double* t, double dt, cudaStream_t s);
// slopes: nine cell arrays, written by launch_bar_states (limited slope of u_a along d at 3d+a)
// and read by launch_face_states
template <typename T>
void launch_bar_states(const Geo& g, const T* u, T* const slopes[9], T* const ubar[3][3], T* const vadv[3],
                       cudaStream_t s);
// wcell: nine cell arrays of scratch for the side-independent part of the face states
template <typename T>
// bodies / views / nb: the bodies at step n, for the wall-repulsion term of the forcing
void launch_face_states(const Geo& g, const T* u, const T* p, const T* rho, const T* divtau, const Body* bodies,
                        const BodyView<T>* views, int nb, T* const slopes[9], T* const wcell[9], T* const ubar[3][3],
                        T* const vadv[3], T* const uf[3][3], cudaStream_t s);
template <typename T>
void launch_mac_setup(const Geo& g, T* const uf[3][3], MGVec b, cudaStream_t s);
template <typename T>
void launch_mac_correct(const Geo& g, T* const uf[3][3], const T* rho, MGVec q, T* const umac[3],
                        cudaStream_t s);
template <typename T>
void launch_advect(const Geo& g, T* const uf[3][3], T* const umac[3], T* adv, cudaStream_t s);
// scratch_s, scratch_xb, scratch_ok: N-sized scratch (9 + 9 arrays of T, 3 of int8) reused by
// every body in turn
template <typename T>
void launch_xi_predict(const Geo& g, const T* u, T* const vadv[3], T* const uf[3][3], T* const umac[3],
                       const int* bb, int blocks, const T* x, const int8_t* lay, T* const scratch_s[9],
                       T* const scratch_xb[9], int8_t* const scratch_ok[3], T* xn, cudaStream_t s);
template <typename T>
void launch_density(const Geo& g, const Body* bodies, const BodyView<T>* views, int nb, const int* bbs, int bstride,
                    T* rho, cudaStream_t s);
template <typename T>
// bodies / views / nb: the bodies at step n+1/2, for the wall-repulsion term
void launch_ustar(const Geo& g, const T* u, const T* adv, const T* p, const T* rho_h, const T* divtau_h,
                  T* ustar, const Body* bodies, const BodyView<T>* views, int nb, cudaStream_t s);
// the wall-repulsion acceleration of every cell from the given bodies' phi, as FP64 (3 N)
template <typename T>
void launch_rep_field(const Geo& g, const Body* bodies, const BodyView<T>* views, int nb, double* out, cudaStream_t s);

// ---- swimmer diagnostics (rmt_diag.cu) ----------------------------------------------
// one body's sums [w u (3), w, w sigma_a : grad u, w Phi_elas, w over cells with F, w (J-1)^2]
// into scratch[0..8) (FP64); scratch holds body_stats_scratch_bytes(); t: device time
size_t body_stats_scratch_bytes();
template <typename T>
void launch_body_stats(const Geo& g, const T* u, const Body& b, const BodyView<T>& v, const double* t, double* scratch,
                       cudaStream_t s);
template <typename T>
void launch_fe_setup(const Geo& g, const T* u, const T* ustar, MGVec b, cudaStream_t s);
template <typename T>
void launch_fe_update(const Geo& g, const T* ustar, const T* rho_h, MGVec psi, T* u, T* p,
                      T* psi_out, cudaStream_t s);
template <typename T>
void launch_fill(T* a, T v, long n, cudaStream_t s);

// ---- extrapolation (rmt_extrap.cu) ------------------------------------------------
template <typename T>
void launch_init_xi(const Geo& g, const Body& b, T* x, cudaStream_t s);
// bb_in: band bounding box of the step (null: whole grid); bb_out receives the new band's box;
// blocks: launch width for the body's window (kernels stride over the whole window); list: the
// band's cells sorted by layer (capacity: the grid), written by the layer passes of
// launch_extrapolate and read by launch_corrector of the same step; cnt: BAND_COUNTERS ints,
// cnt[l] the cells of layer l (l = 1..8), cnt[0] and cnt[9] the lengths of the FP64 redo lists
// of the two fitting passes; redo: FP32 storage, a list of the grid's size for the cells whose
// FP32 fits were too ill-conditioned (null for FP64 storage); wls_blocks: launch width of the
// one-warp-per-cell fits.
// err[0] counts degenerate fits, err[1] (FP32 storage) band cells near the seam of the body's
// image window; returns the error of the one runtime call it makes besides launches
constexpr int BAND_COUNTERS = 10;
template <typename T>
cudaError_t launch_extrapolate(const Geo& g, const Body& b, const int* bb_in, int* bb_out, int blocks, int* list,
                               int* cnt, int* redo, int wls_blocks, T* x, T* phi, int8_t* lay, int* err,
                               cudaStream_t s);
template <typename T>
void launch_corrector(const Geo& g, const Body& b, const int* bb_in, int blocks, const int* list, int* cnt, int* redo,
                      int wls_blocks, const T* x, const int8_t* lay, const T* xn, const int8_t* layn, T* xh, T* phih,
                      int* err, cudaStream_t s);

// ---- multigrid (rmt_mg.cu) ----------------------------------------------------------
struct MGSolver;  // opaque
// kind 0: cell-centred 7-point (MAC), kind 1: nodal trilinear FE (27-point)
MGSolver* mg_create(const Geo& g, int kind, int prec_fp32, cudaError_t* err);
size_t mg_footprint(const Geo& g, int kind, int prec_fp32);  // device bytes mg_create would request
size_t mg_device_bytes(const MGSolver* m);                   // device bytes it did request
// device bytes charged for one allocation of `bytes` (allocations are 256-byte granular, at least 16 bytes asked)
inline size_t dev_bytes(size_t bytes) { return ((bytes < 16 ? 16 : bytes) + 255) / 256 * 256; }
void mg_destroy(MGSolver* m);
// Level-0 right-hand side (filled before a solve) and solution, as MGVec.
MGVec mg_rhs(MGSolver* m);
MGVec mg_solution(MGSolver* m);
// FP64 copy of the solution for read-back (FP32 mode: converted on s first)
const double* mg_solution64(MGSolver* m, cudaStream_t s);
// the cell density the operator is built from on the finest level (the caller's array, type T)
void mg_set_density(MGSolver* m, const void* rho);
// smoother sweeps before/after the coarse correction and the Jacobi weight (negative: keep)
void mg_set_smoother(MGSolver* m, int pre, int post, double omega);
// sweeps on the levels below the finest (negative: the finest level's counts)
void mg_set_coarse_smoother(MGSolver* m, int pre, int post);
// V-cycles on the correction equation between FP64 residual evaluations (>= 1)
void mg_set_inner(MGSolver* m, int inner);
// block height (1, 2, 4 or 8 rows of 32 threads) of the level kernels
void mg_set_block(MGSolver* m, int by);
// start each solve from the previous solution (zero before the first) instead of from zero
void mg_set_warm(MGSolver* m, int warm);
// device int set to 1 when a solve's right-hand-side mean, solution mean or residual norm is
// not finite (null: not checked)
void mg_set_nonfinite_flag(MGSolver* m, int* flag);
// z-chunk length (planes a block marches) of the finest level's stencil tiles: the fused
// red-black sweep (MAC; ignored where the level does not take it) or the FE tile kernels;
// 0 restores the wave-filling heuristic.  mg_zchunk returns the length in use.
void mg_set_zchunk(MGSolver* m, int zchunk);
int mg_zchunk(const MGSolver* m);
// MAC in FP32: one fused red-black pass per sweep (1: on the large levels that allow it, the
// default; 2: on every level that allows it; 0: never), else one pass per colour
void mg_set_sweep(MGSolver* m, int fused);
// Optional timing hook around the finest-level smoother and FP64-residual launches:
// hook(ctx, which, begin, stream) with which = 0 (smoother colour), 1 (FP64 residual) or 2 (fused
// red-black sweep).
typedef void (*mg_hook_fn)(void* ctx, int which, int begin, cudaStream_t s);
void mg_set_hook(MGSolver* m, mg_hook_fn fn, void* ctx);
// Solves to rtol (or a fixed cycle count); returns cycles used, -1 on non-convergence.
int mg_solve(MGSolver* m, double rtol, int max_cycles, int fixed_cycles, cudaStream_t s, cudaError_t* err);
