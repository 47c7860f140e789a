// Autotuner of the two multigrid solves (smoother schedule, cycle count, kernel block shapes
// and the z-extent of the finest level's stencil tiles).
//
// For each solver it tries the smoother schedules of a small grid (sweeps before / after the
// coarse correction, Jacobi weight for the nodal solve, 1, 2 or 4 V-cycles per high-precision
// residual) on the right-hand side of the grid's last step: it counts the V-cycles a schedule
// needs to reach the requested relative residual, times that many cycles with CUDA events, and
// keeps the fastest.  Then it times the block heights of the level kernels with that schedule,
// and the z-chunk length (planes one block marches) of the finest level's plane-marching tiles
// (the fused red-black sweep, the FE Jacobi / residual tiles): the wave-filling default against
// 8, 16, 32, 64 and 128 planes.  The winner becomes the grid's fixed-cycle configuration
// (rmt_set_option), so later steps take no host synchronisation.
#include <cstdio>

#include "rmt.h"
#include "rmt_internal.h"
#include "rmt_kernels.h"

namespace {

struct Sched {
  int pre, post, inner, block;
  double omega;
};

// time of one fixed-cycle solve (ms), after a warm-up solve; negative on a CUDA error
double time_solve(MGSolver* m, int cycles, cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  cudaError_t e = cudaSuccess;
  mg_solve(m, 0.0, 0, cycles, s, &e);
  if (e != cudaSuccess) return -1.0;
  constexpr int REPS = 2;
  cudaEventRecord(a, s);
  for (int r = 0; r < REPS; r++) mg_solve(m, 0.0, 0, cycles, s, &e);
  cudaEventRecord(b, s);
  if (cudaEventSynchronize(b) != cudaSuccess || e != cudaSuccess) return -1.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms / REPS;
}

void apply(MGSolver* m, const Sched& c) {
  mg_set_smoother(m, c.pre, c.post, c.omega);
  mg_set_inner(m, c.inner);
  mg_set_block(m, c.block);
}

// best schedule of one solver: returns its cycles (-1: nothing converged), fills best and ms
int tune_one(MGSolver* m, int kind, double rtol, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, Sched& best,
             double& best_ms, int& trials, int& zchunk) {
  const int nsw = kind == 0 ? 4 : 3;
  // relaxation factors: red-black sweeps (1 and an over-relaxed 1.15), Jacobi weights
  const double omegas[2][3] = {{1.0, 1.15, 0.0}, {0.8, 0.9, 1.0}};
  const int nom = kind == 0 ? 2 : 3;
  int best_cyc = -1;
  best_ms = 1e300;
  for (int pre = 1; pre <= nsw; pre++)
    for (int post = 1; post <= nsw; post++)
      for (int io = 0; io < nom; io++)
        for (int inner : {1, 2, 4}) {
          const Sched c{pre, post, inner, 4, omegas[kind][io]};
          apply(m, c);
          cudaError_t e = cudaSuccess;
          const int cyc = mg_solve(m, rtol, 40, 0, s, &e);
          trials++;
          if (e != cudaSuccess || cyc < 1) continue;
          const double ms = time_solve(m, cyc, s, a, b);
          if (ms > 0 && ms < best_ms) {
            best_ms = ms;
            best = c;
            best_cyc = cyc;
          }
        }
  if (best_cyc < 0) return -1;
  for (int by : {1, 2, 8}) {
    Sched c = best;
    c.block = by;
    apply(m, c);
    const double ms = time_solve(m, best_cyc, s, a, b);
    trials++;
    if (ms > 0 && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  apply(m, best);
  // z-chunk of the finest level's tiles (0: the wave-filling default)
  zchunk = 0;
  mg_set_zchunk(m, 0);
  const int def = mg_zchunk(m);
  for (int zc : {8, 16, 32, 64, 128}) {
    if (zc == def) continue;
    mg_set_zchunk(m, zc);
    if (mg_zchunk(m) != zc) continue;  // the level is shorter, or takes no plane-marching tile
    const double ms = time_solve(m, best_cyc, s, a, b);
    trials++;
    if (ms > 0 && ms < best_ms) {
      best_ms = ms;
      zchunk = zc;
    }
  }
  mg_set_zchunk(m, zchunk);
  return best_cyc;
}

}  // namespace

extern "C" rmt_status rmt_autotune(rmt_grid* g, double rtol, rmt_tune_result* out) {
  if (!g || !(rtol > 0.0 && rtol < 1.0)) return RMT_EINVAL;
  MGSolver *mac = nullptr, *fe = nullptr;
  cudaStream_t s = nullptr;
  double grid_rtol = 0.0;
  rmt_status st = grid_solvers(g, &mac, &fe, &s, &grid_rtol);
  if (st != RMT_OK) return st;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return grid_fail(g, RMT_ECUDA, "autotune: event creation failed");
  }
  Sched bm{}, bf{};
  double ms_mac = 0, ms_fe = 0;
  int trials = 0, zm = 0, zf = 0;
  const int cm = tune_one(mac, 0, rtol, s, a, b, bm, ms_mac, trials, zm);
  const int cf = tune_one(fe, 1, rtol, s, a, b, bf, ms_fe, trials, zf);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cm < 0 || cf < 0) return grid_fail(g, RMT_ENOCONVERGE, "autotune: no schedule reached the tolerance");
  // the grid's own options follow the winners (and make the step fixed-cycle)
  const struct {
    const char* name;
    double v;
  } opts[] = {{"mac_pre", (double)bm.pre}, {"mac_post", (double)bm.post}, {"mac_inner", (double)bm.inner},
              {"mac_block", (double)bm.block}, {"mac_cycles", (double)cm}, {"fe_pre", (double)bf.pre},
              {"fe_post", (double)bf.post}, {"fe_inner", (double)bf.inner}, {"fe_block", (double)bf.block},
              {"fe_omega", bf.omega}, {"fe_cycles", (double)cf}, {"mac_zchunk", (double)zm},
              {"fe_zchunk", (double)zf}, {"mac_omega", bm.omega}};
  for (const auto& o : opts)
    if ((st = rmt_set_option(g, o.name, o.v)) != RMT_OK) return st;
  if (out) {
    out->mac_pre = bm.pre;
    out->mac_post = bm.post;
    out->mac_inner = bm.inner;
    out->mac_block = bm.block;
    out->mac_cycles = cm;
    out->mac_ms = ms_mac;
    out->fe_pre = bf.pre;
    out->fe_post = bf.post;
    out->fe_inner = bf.inner;
    out->fe_block = bf.block;
    out->fe_cycles = cf;
    out->fe_omega = bf.omega;
    out->fe_ms = ms_fe;
    out->trials = trials;
    out->mac_zchunk = zm;
    out->fe_zchunk = zf;
    out->mac_omega = bm.omega;
  }
  return RMT_OK;
}
