// C ABI of the RMT per-step update (declared in include/rmt.h).  Owns the device state of
// one simulation and sequences the kernels of one timestep in the order of the paper's
// SI "Timestepping algorithm" (13 steps) on the grid's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>
#include <atomic>

#include "rmt.h"
#include "rmt_internal.h"
#include "rmt_kernels.h"

static std::atomic<long> g_launches{0};
void rmt_count_launches(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
  constexpr int MAXDEV = 64;
  static std::atomic<int> cached[MAXDEV];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) dev = 0;
  int n = cached[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cached[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {

struct BodyMem {
  int* bb = nullptr;  // band bounding boxes of the two parities (2 x 6 ints, device)
  int blocks = 1;     // launch width of the body's window kernels
  int* list = nullptr;   // compacted band cells of the current step (capacity N)
  int* count = nullptr;  // per-layer counts of the list and the redo lists' lengths (device)
  int* redo = nullptr;   // FP32: cells whose fits are redone in FP64 (device)
  void* X[2] = {nullptr, nullptr};
  void* PHI[2] = {nullptr, nullptr};
  int8_t* LAY[2] = {nullptr, nullptr};
  void* XH = nullptr;
  void* PHIH = nullptr;
};

}  // namespace

namespace {
enum {
  P_STRESS_N, P_GODUNOV, P_MAC_SETUP, P_MAC_SOLVE, P_MAC_CORR_ADV, P_XI_PRED, P_EXTRAP, P_CORR, P_STRESS_H,
  P_USTAR, P_FE_SETUP, P_FE_SOLVE, P_FE_UPDATE, P_MAC_SMOOTH, P_MAC_RESID, P_FE_SMOOTH, P_FE_RESID, P_MAC_SWEEP, P_NUM
};
const char* const kProfNames[P_NUM] = {
    "stress_n", "godunov_velocity", "mac_setup", "mac_solve", "mac_correct_advect", "xi_predict", "extrapolate_corrector",
    "corrector", "stress_half", "density_ustar", "fe_setup", "fe_solve", "fe_update_density",
    "k_rbgs(mac,level0,colour)", "k_resid64(mac)", "k_jacobi(fe,level0)", "k_resid64(fe)",
    "k_rbgs_sweep(mac,level0)"};
struct Prof {
  int on = 0;
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int e;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  cudaEvent_t open[P_NUM] = {};
  double ms[P_NUM] = {};
  long n[P_NUM] = {};
};
struct HookCtx {
  rmt_grid* g;
  int kind;
};
}  // namespace

struct rmt_grid {
  rmt_grid_desc desc;
  Geo g;
  int fp32 = 0;
  size_t esz = 8;
  cudaStream_t s = nullptr;
  int inited = 0;
  rmt_status init_st = RMT_OK;  // outcome of the initialisation (ensure_init)
  rmt_status sticky = RMT_OK;
  char msg[512] = {0};
  std::vector<rmt_solid_desc> solids;
  std::vector<Body> bodies;
  std::vector<BodyMem> bm;
  Body* bodies_d = nullptr;
  int* bb_all = nullptr;  // band boxes: body m, parity p at 12 m + 6 p
  int *slist = nullptr, *scount = nullptr;  // cells some band reaches (stress pass 2)
  double* t_d = nullptr;                      // simulated time (device copy of t)
  std::vector<cudaStream_t> body_s;           // one stream per body (re-extrapolation, corrector)
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  void* views_d = nullptr;  // BodyView<T>[2 parities][3 levels][nb]
  int par = 0;
  void *u = nullptr, *p = nullptr, *rho = nullptr, *rho_h = nullptr, *divn = nullptr, *divh = nullptr;
  void *adv = nullptr, *ustar = nullptr, *psi = nullptr;
  void* xscr_s[9] = {};
  void* xscr_b[9] = {};
  int8_t* xscr_ok[3] = {};
  int8_t* xscr_ok2[3] = {};  // the second predictor scratch set's flags (its arrays: slopes, wcell)
  void* vadv[3] = {};
  void* ub[3][3] = {};
  void* slopes[9] = {};
  void* wcell[9] = {};
  void* uf[3][3] = {};
  void* umac[3] = {};
  MGSolver* mac = nullptr;
  MGSolver* fe = nullptr;
  // device error words, copied to err_h (pinned) at the end of every step: [0] degenerate fits,
  // [1] FP32 band cells near the seam of their image window, [2] a non-finite mean or norm in a
  // projection (the velocity diverged)
  int* err_d = nullptr;
  int* err_h = nullptr;
  double* stage = nullptr;
  float* stage_f = nullptr;  // FP32 field I/O of fields without FP32 storage (first use)
  long stage_len = 0;
  int cycles[2] = {0, 0};
  double t = 0.0;
  long step = 0;
  std::vector<void*> allocs;
  Prof prof;
  HookCtx hctx[2];
  // smoother schedule (negative: solver default)
  int mac_pre = -1, mac_post = -1, fe_pre = -1, fe_post = -1, mac_inner = 1, fe_inner = 1;
  int mac_cpre = -1, mac_cpost = -1, fe_cpre = -1, fe_cpost = -1;  // coarse levels (negative: as level 0)
  int mac_block = 4, fe_block = 4;  // block height of the multigrid level kernels
  int mac_warm = 0, fe_warm = 0;    // warm-started solves
  int mac_sweep = 1;                // fused red-black sweeps (FP32 MAC)
  int mac_zchunk = 0, fe_zchunk = 0;  // finest-level stencil tile z-chunks (0: heuristic)
  double fe_omega = -1.0, mac_omega = -1.0;
  size_t bytes = 0;  // device bytes requested by dalloc
  int dry = 0;       // dalloc only counts (footprint model)
  // host-side fault injection (rmt_set_option): a NaN written into u before step
  // inject_nan_step, a failure of the grid's inject_alloc-th device allocation (-1: off)
  long inject_nan_step = -1, inject_alloc = -1, nalloc = 0;
  // captured step graphs (fixed-cycle mode): one per parity of the reference-map buffers
  int use_graph = 0;
  cudaStream_t cap_s = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long gnodes[2] = {0, 0};
  // set while the grid is a member of a batch: its work runs on that batch's stream
  cudaStream_t batch_s = nullptr;
  int in_batch = 0;
};

namespace {

// launch width of the one-warp-per-band-cell fits: 4 resident blocks of 128 threads per SM
inline int wls_blocks() { return sm_count() * 4; }

rmt_status fail(rmt_grid* g, rmt_status st, const char* fmt, ...) {
  if (g) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g->msg, sizeof g->msg, fmt, ap);
    va_end(ap);
    if (st != RMT_EINVAL) g->sticky = st;
  }
  return st;
}

// reads the grid's device error words after waiting for its stream (defined below)
rmt_status check_err(rmt_grid* g);

// a call refused in the grid's present state: message only, the grid stays usable
rmt_status refuse(rmt_grid* g, const char* why) {
  snprintf(g->msg, sizeof g->msg, "%s", why);
  return RMT_ESTATE;
}

#define CK(g, call)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(g, RMT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t prof_event(rmt_grid* g) {
  cudaEvent_t e = nullptr;
  if (!g->prof.pool.empty()) {
    e = g->prof.pool.back();
    g->prof.pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}
void pb(rmt_grid* g, int e) {
  if (!g->prof.on) return;
  g->prof.open[e] = prof_event(g);
  cudaEventRecord(g->prof.open[e], g->s);
}
void pe(rmt_grid* g, int e) {
  if (!g->prof.on || !g->prof.open[e]) return;
  cudaEvent_t b = prof_event(g);
  cudaEventRecord(b, g->s);
  g->prof.recs.push_back({e, g->prof.open[e], b});
  g->prof.open[e] = nullptr;
  g->prof.n[e]++;
}
void prof_flush(rmt_grid* g) {
  if (g->prof.recs.empty()) return;
  cudaStreamSynchronize(g->s);
  for (auto& r : g->prof.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) g->prof.ms[r.e] += ms;
    g->prof.pool.push_back(r.a);
    g->prof.pool.push_back(r.b);
  }
  g->prof.recs.clear();
}
void mg_hook(void* ctx, int which, int begin, cudaStream_t) {
  HookCtx* h = (HookCtx*)ctx;
  const int e = h->kind == 0 ? (which == 0 ? P_MAC_SMOOTH : (which == 2 ? P_MAC_SWEEP : P_MAC_RESID))
                             : (which == 0 ? P_FE_SMOOTH : P_FE_RESID);
  if (begin) pb(h->g, e);
  else pe(h->g, e);
}
// algorithmic bytes of one launch of the profiled multigrid kernels (w = bytes per word, N
// cells, NN nodes): red-black colour pass (7-point): x and rho read once, b read and x written
// for half the cells; Jacobi pass (27-point): x, b read and x written per node, rho per cell;
// FP64 residual: x and b 8 bytes each, rho, and the residual copy in the storage type; fused
// red-black sweep: x, rho and b read and x written once per cell.
double prof_bytes(const rmt_grid* g, int e) {
  const double w = (double)g->esz, N = (double)g->g.N, NN = (double)g->g.NN;
  switch (e) {
    case P_MAC_SMOOTH: return 3.0 * N * w;
    case P_MAC_RESID: return 16.0 * N + 2.0 * N * w;
    case P_FE_SMOOTH: return 3.0 * NN * w + N * w;
    case P_FE_RESID: return 16.0 * NN + N * w + NN * w;
    case P_MAC_SWEEP: return 4.0 * N * w;
  }
  return 0.0;
}

rmt_status dalloc(rmt_grid* g, void** p, size_t bytes) {
  g->bytes += dev_bytes(bytes);
  if (g->dry) {
    *p = nullptr;
    return RMT_OK;
  }
  if (g->inject_alloc >= 0 && g->nalloc++ == g->inject_alloc) {
    *p = nullptr;
    return fail(g, RMT_ENOMEM, "cudaMalloc(%zu): failure injected by the inject_alloc option", bytes);
  }
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) return fail(g, RMT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  g->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes < 16 ? 16 : bytes, g->s);
  if (e != cudaSuccess) return fail(g, RMT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  return RMT_OK;
}

// Reading of the time step when the caller gives none: explicit viscous and elastic-wave
// limits, dt = min(0.2 h, 0.8 rho_min h^2/(6 mu_max), 0.5 h/sqrt(G_max/rho_min)).
double pick_dt(const rmt_grid* g) {
  if (g->desc.dt > 0.0) return g->desc.dt;
  const double h = g->g.h;
  double rmin = g->desc.rho_f, mumax = g->desc.mu, gmax = 0.0;
  for (const auto& s : g->solids) {
    if (s.rho_s < rmin) rmin = s.rho_s;
    const double ma = s.mu_a * (1.0 + s.gamma_t);
    if (ma > mumax) mumax = ma;
    if (s.G > gmax) gmax = s.G;
  }
  double dt = 0.2 * h;
  const double dv = 0.8 * rmin * h * h / (6.0 * mumax);
  if (dv < dt) dt = dv;
  if (gmax > 0.0) {
    const double de = 0.5 * h / sqrt(gmax / rmin);
    if (de < dt) dt = de;
  }
  return dt;
}

template <typename T>
__global__ void k_cvt(const T* __restrict__ a, double* __restrict__ b, long n) {
  GRID_LOOP(i, n) b[i] = (double)a[i];
}
template <typename T>
__global__ void k_cvt_back(const double* __restrict__ a, T* __restrict__ b, long n) {
  GRID_LOOP(i, n) b[i] = (T)a[i];
}
__global__ void k_cvt_i8(const int8_t* __restrict__ a, double* __restrict__ b, long n) {
  GRID_LOOP(i, n) b[i] = (double)a[i];
}
// a reference map to FP64 xi (FP32 storage: the displacement plus the cell centre's image)
template <typename T>
__global__ void k_xi_out(Geo g, Body b, const T* __restrict__ x, double* __restrict__ out) {
  GRID_LOOP(q, 3 * g.N) {
    double v = (double)x[q];
    if constexpr (disp_storage<T>()) {
      const int a = (int)(q / g.N);
      const long c = q - a * g.N;
      const int ii[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long)g.n[0] * g.n[1]))};
      v += g.lo[a] + (img_u(g, b, a, ii[a]) + 0.5) * g.h;
    }
    out[q] = v;
  }
}
// FP64 xi to the stored form
template <typename T>
__global__ void k_xi_in(Geo g, Body b, const double* __restrict__ in, T* __restrict__ x) {
  GRID_LOOP(q, 3 * g.N) {
    double v = in[q];
    if constexpr (disp_storage<T>()) {
      const int a = (int)(q / g.N);
      const long c = q - a * g.N;
      const int ii[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long)g.n[0] * g.n[1]))};
      v -= g.lo[a] + (img_u(g, b, a, ii[a]) + 0.5) * g.h;
    }
    x[q] = (T)v;
  }
}
inline int nbk(long n) {
  long b = (n + 255) / 256;
  if (b > (long)sm_count() * 32) b = (long)sm_count() * 32;
  return (int)(b < 1 ? 1 : b);
}

template <typename T>
BodyView<T>* views(rmt_grid* g, int par, int level) {
  return (BodyView<T>*)g->views_d + ((size_t)(par * 3 + level) * g->bodies.size());
}

template <typename T>
rmt_status build_views(rmt_grid* g) {
  const int nb = (int)g->bodies.size();
  std::vector<BodyView<T>> hv((size_t)6 * (nb > 0 ? nb : 1));
  for (int par = 0; par < 2; par++)
    for (int m = 0; m < nb; m++) {
      BodyMem& b = g->bm[m];
      hv[(par * 3 + 0) * nb + m] = {(const T*)b.X[par], (const T*)b.PHI[par], b.LAY[par]};
      hv[(par * 3 + 1) * nb + m] = {(const T*)b.XH, (const T*)b.PHIH, b.LAY[1 - par]};
      hv[(par * 3 + 2) * nb + m] = {(const T*)b.X[1 - par], (const T*)b.PHI[1 - par], b.LAY[1 - par]};
    }
  if (nb > 0) {
    CK(g, cudaMemcpyAsync(g->views_d, hv.data(), hv.size() * sizeof(BodyView<T>), cudaMemcpyHostToDevice, g->s));
    CK(g, cudaMemcpyAsync(g->bodies_d, g->bodies.data(), nb * sizeof(Body), cudaMemcpyHostToDevice, g->s));
    CK(g, cudaStreamSynchronize(g->s));
  }
  return RMT_OK;
}

// launch width of each body's window kernels from its band box (the kernels stride over the
// whole window, so this only sizes the launch)
rmt_status size_windows(rmt_grid* g) {
  const Geo& G = g->g;
  for (auto& b : g->bm) {
    int h[6];
    CK(g, cudaMemcpy(h, b.bb, sizeof h, cudaMemcpyDeviceToHost));
    long vol = 1;
    for (int d = 0; d < 3; d++) {
      long e = h[d] <= h[3 + d] ? (long)(h[3 + d] - h[d] + 1) + 8 : 0;
      if (e > G.n[d]) e = G.n[d];
      vol *= e;
    }
    long blocks = (vol + 127) / 128;
    if (blocks < 1) blocks = 1;
    if (blocks > (long)sm_count() * 64) blocks = (long)sm_count() * 64;
    b.blocks = (int)blocks;
  }
  return RMT_OK;
}

// every device allocation of the grid (with g->dry set: only their sizes, into g->bytes)
template <typename T>
rmt_status alloc_t(rmt_grid* g) {
  const Geo& G = g->g;
  const long N = G.N;
  rmt_status st;
#define AL(ptr, bytes) \
  if ((st = dalloc(g, (void**)&(ptr), (bytes))) != RMT_OK) return st;
  const size_t e = sizeof(T);
  AL(g->u, 3 * N * e);
  AL(g->p, G.NN * e);
  AL(g->rho, N * e);
  AL(g->rho_h, N * e);
  AL(g->divn, 3 * N * e);
  AL(g->divh, 3 * N * e);
  AL(g->adv, 3 * N * e);
  AL(g->ustar, 3 * N * e);
  AL(g->psi, G.NN * e);
  for (int q = 0; q < 9; q++) AL(g->slopes[q], N * e);
  for (int q = 0; q < 9; q++) AL(g->wcell[q], N * e);
  if (!g->bodies.empty()) {
    for (int q = 0; q < 9; q++) {
      AL(g->xscr_s[q], N * e);
      AL(g->xscr_b[q], N * e);
    }
    for (int q = 0; q < 3; q++) AL(g->xscr_ok[q], N);
    if (g->bodies.size() > 1)
      for (int q = 0; q < 3; q++) AL(g->xscr_ok2[q], N);
  }
  for (int d = 0; d < 3; d++) {
    const long nf = nfaces(G, d);
    for (int a = 0; a < 3; a++) {
      AL(g->ub[d][a], nf * e);
      AL(g->uf[d][a], nf * e);
    }
    AL(g->vadv[d], nf * e);
    AL(g->umac[d], nf * e);
  }
  const int nb = (int)g->bodies.size();
  g->bm.assign(nb, BodyMem());
  for (int m = 0; m < nb; m++) {
    BodyMem& b = g->bm[m];
    for (int q = 0; q < 2; q++) {
      AL(b.X[q], 3 * N * e);
      AL(b.PHI[q], N * e);
      AL(b.LAY[q], N);
    }
    AL(b.XH, 3 * N * e);
    AL(b.PHIH, N * e);
    b.bb = nullptr;  // set below: all bodies' boxes are contiguous
    AL(b.list, N * sizeof(int));
    AL(b.count, BAND_COUNTERS * sizeof(int));
    if (e == 4) AL(b.redo, N * sizeof(int));
  }
  AL(g->bb_all, (nb > 0 ? nb : 1) * 12 * sizeof(int));
  AL(g->slist, (nb > 0 ? N : 1) * sizeof(int));
  AL(g->scount, 16);
  AL(g->t_d, 16);
  for (int m = 0; m < nb; m++) g->bm[m].bb = g->bb_all + 12 * m;
  AL(g->bodies_d, (nb > 0 ? nb : 1) * sizeof(Body));
  AL(g->views_d, (size_t)6 * (nb > 0 ? nb : 1) * sizeof(BodyView<T>));
  AL(g->err_d, 16);
  long sl = 3 * N;
  for (int d = 0; d < 3; d++)
    if (3 * nfaces(G, d) > sl) sl = 3 * nfaces(G, d);
  if (G.NN > sl) sl = G.NN;
  AL(g->stage, sl * sizeof(double));
  g->stage_len = sl;
#undef AL
  if (g->dry) {
    g->bytes += mg_footprint(G, 0, g->fp32) + mg_footprint(G, 1, g->fp32);
    return RMT_OK;
  }
  CK(g, cudaMallocHost((void**)&g->err_h, 16));
  // no step has copied its error words yet: a step polls them before its first copy lands, and
  // pinned memory may come back from an earlier grid with that grid's words in it
  memset(g->err_h, 0, 16);
  cudaError_t ce = cudaSuccess;
  g->mac = mg_create(G, 0, g->fp32, &ce);
  if (ce != cudaSuccess) return fail(g, RMT_ENOMEM, "multigrid (MAC) allocation: %s", cudaGetErrorString(ce));
  g->fe = mg_create(G, 1, g->fp32, &ce);
  if (ce != cudaSuccess) return fail(g, RMT_ENOMEM, "multigrid (FE) allocation: %s", cudaGetErrorString(ce));
  g->hctx[0] = {g, 0};
  g->hctx[1] = {g, 1};
  mg_set_hook(g->mac, mg_hook, &g->hctx[0]);
  mg_set_hook(g->fe, mg_hook, &g->hctx[1]);
  mg_set_smoother(g->mac, g->mac_pre, g->mac_post, g->mac_omega);
  mg_set_smoother(g->fe, g->fe_pre, g->fe_post, g->fe_omega);
  mg_set_coarse_smoother(g->mac, g->mac_cpre, g->mac_cpost);
  mg_set_coarse_smoother(g->fe, g->fe_cpre, g->fe_cpost);
  mg_set_inner(g->mac, g->mac_inner);
  mg_set_inner(g->fe, g->fe_inner);
  mg_set_block(g->mac, g->mac_block);
  mg_set_block(g->fe, g->fe_block);
  mg_set_warm(g->mac, g->mac_warm);
  mg_set_sweep(g->mac, g->mac_sweep);
  mg_set_warm(g->fe, g->fe_warm);
  mg_set_zchunk(g->mac, g->mac_zchunk);
  mg_set_zchunk(g->fe, g->fe_zchunk);
  mg_set_nonfinite_flag(g->mac, g->err_d + 2);
  mg_set_nonfinite_flag(g->fe, g->err_d + 2);
  g->bytes += mg_device_bytes(g->mac) + mg_device_bytes(g->fe);
  return RMT_OK;
}

template <typename T>
rmt_status init_t(rmt_grid* g) {
  const Geo& G = g->g;
  const long N = G.N;
  const int nb = (int)g->bodies.size();
  rmt_status st = alloc_t<T>(g);
  if (st != RMT_OK) return st;
  CK(g, cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
  g->body_s.assign(nb, nullptr);
  g->ev_join.assign(nb, nullptr);
  for (int m = 0; m < nb; m++) {
    CK(g, cudaStreamCreateWithFlags(&g->body_s[m], cudaStreamNonBlocking));
    CK(g, cudaEventCreateWithFlags(&g->ev_join[m], cudaEventDisableTiming));
  }
  // outside a body's band every per-body array reads "absent" (layer -1, NaN); the window
  // kernels rely on it, since they only ever touch the band's neighbourhood
  const T nanv = (T)NAN;
  for (int m = 0; m < nb; m++) {
    BodyMem& b = g->bm[m];
    launch_fill<int8_t>(b.LAY[1], (int8_t)-1, N, g->s);
    launch_fill<T>((T*)b.X[1], nanv, 3 * N, g->s);
    launch_fill<T>((T*)b.PHI[1], nanv, N, g->s);
    launch_fill<T>((T*)b.XH, nanv, 3 * N, g->s);
    launch_fill<T>((T*)b.PHIH, nanv, N, g->s);
  }
  if ((st = build_views<T>(g)) != RMT_OK) return st;
  // SI "Initialization": u^0 = 0, p = 0, xi^0 = x, extrapolation, phi, rho^0
  const int full_blocks = (int)std::min((G.N + 127) / 128, (long)sm_count() * 64);
  for (int m = 0; m < nb; m++) {
    BodyMem& b = g->bm[m];
    launch_init_xi<T>(G, g->bodies[m], (T*)b.X[0], g->s);
    CK(g, launch_extrapolate<T>(G, g->bodies[m], nullptr, b.bb, full_blocks, b.list, b.count, b.redo, wls_blocks(),
                                (T*)b.X[0], (T*)b.PHI[0], b.LAY[0], g->err_d, g->s));
  }
  launch_density<T>(G, g->bodies_d, views<T>(g, 0, 0), nb, g->bb_all, 12, (T*)g->rho, g->s);
  CK(g, cudaGetLastError());
  CK(g, cudaStreamSynchronize(g->s));
  return size_windows(g);
}

template <typename T>
rmt_status step_t(rmt_grid* g) {
  const Geo& G = g->g;
  cudaStream_t s = g->s;
  const int nb = (int)g->bodies.size();
  const int cur = g->par, nxt = 1 - g->par;
  T* ub[3][3];
  T* slopes[9];
  T* wcell[9];
  T* vadv[3];
  T* uf[3][3];
  T* umac[3];
  for (int d = 0; d < 3; d++) {
    for (int a = 0; a < 3; a++) {
      ub[d][a] = (T*)g->ub[d][a];
      uf[d][a] = (T*)g->uf[d][a];
    }
    vadv[d] = (T*)g->vadv[d];
    umac[d] = (T*)g->umac[d];
  }
  for (int q = 0; q < 9; q++) {
    slopes[q] = (T*)g->slopes[q];
    wcell[q] = (T*)g->wcell[q];
  }
  T* u = (T*)g->u;
  // 1. tau^n and its divergence
  pb(g, P_STRESS_N);
  CK(g, launch_stress_div<T>(G, u, g->bodies_d, views<T>(g, cur, 0), nb, g->bb_all + 6 * cur, 12, g->t_d, 0.0,
                              (T*)g->divn, g->slist, g->scount, slopes, s));
  pe(g, P_STRESS_N);
  // 2. Godunov face states of u (transverse bar states first)
  pb(g, P_GODUNOV);
  launch_bar_states<T>(G, u, slopes, ub, vadv, s);
  launch_face_states<T>(G, u, (const T*)g->p, (const T*)g->rho, (const T*)g->divn, g->bodies_d, views<T>(g, cur, 0),
                        nb, slopes, wcell, ub, vadv, uf, s);
  pe(g, P_GODUNOV);
  // 3. MAC projection of the normal face velocities
  pb(g, P_MAC_SETUP);
  launch_mac_setup<T>(G, uf, mg_rhs(g->mac), s);
  mg_set_density(g->mac, g->rho);
  pe(g, P_MAC_SETUP);
  cudaError_t ce = cudaSuccess;
  const double rtol = g->desc.mg_rtol > 0 ? g->desc.mg_rtol : 1e-12;
  const int maxc = g->desc.mg_max_cycles > 0 ? g->desc.mg_max_cycles : 60;
  pb(g, P_MAC_SOLVE);
  int cyc = mg_solve(g->mac, rtol, maxc, g->desc.mg_fixed_cycles, s, &ce);
  pe(g, P_MAC_SOLVE);
  if (ce != cudaSuccess) return fail(g, RMT_ECUDA, "MAC solve: %s", cudaGetErrorString(ce));
  if (cyc < 0) {
    const rmt_status es = check_err(g);  // a non-finite right-hand side stops a solve too
    if (es != RMT_OK) return es;
    return fail(g, RMT_ENOCONVERGE, "MAC multigrid missed rtol %.3g in %d cycles at step %ld", rtol, maxc, g->step);
  }
  g->cycles[0] = cyc;
  pb(g, P_MAC_CORR_ADV);
  launch_mac_correct<T>(G, uf, (const T*)g->rho, mg_solution(g->mac), umac, s);
  // 4. advective term
  launch_advect<T>(G, uf, umac, (T*)g->adv, s);
  pe(g, P_MAC_CORR_ADV);
  // 5. predictor of every body.  Two scratch sets: the predictor's own and the Godunov slope and
  // cell-state arrays (free from the Godunov stage until the half-step stress), so the even
  // bodies run one after another on the step's stream and the odd ones on a second stream
  pb(g, P_XI_PRED);
  cudaStream_t s2 = nb > 1 ? g->body_s[1] : s;
  if (nb > 1) {
    CK(g, cudaEventRecord(g->ev_fork, s));
    CK(g, cudaStreamWaitEvent(s2, g->ev_fork, 0));
  }
  for (int m = 0; m < nb; m++) {
    BodyMem& b = g->bm[m];
    const bool odd = (m & 1) != 0;
    launch_xi_predict<T>(G, u, vadv, uf, umac, b.bb + 6 * cur, b.blocks, (const T*)b.X[cur], b.LAY[cur],
                         odd ? slopes : (T* const*)g->xscr_s, odd ? wcell : (T* const*)g->xscr_b,
                         odd ? g->xscr_ok2 : g->xscr_ok, (T*)b.X[nxt], odd ? s2 : s);
  }
  if (nb > 1) {
    CK(g, cudaEventRecord(g->ev_join[1], s2));
    CK(g, cudaStreamWaitEvent(s, g->ev_join[1], 0));
  }
  pe(g, P_XI_PRED);
  // 6.-7. re-extrapolation and corrector: the bodies are independent, so each runs on its own
  // stream, forked from and joined back into the step's stream (parallel branches when the step
  // is captured as a graph)
  pb(g, P_EXTRAP);
  if (nb > 0) CK(g, cudaEventRecord(g->ev_fork, s));
  for (int m = 0; m < nb; m++) {
    BodyMem& b = g->bm[m];
    cudaStream_t bs = g->body_s[m];
    CK(g, cudaStreamWaitEvent(bs, g->ev_fork, 0));
    const int* bbc = b.bb + 6 * cur;
    CK(g, launch_extrapolate<T>(G, g->bodies[m], bbc, b.bb + 6 * nxt, b.blocks, b.list, b.count, b.redo, wls_blocks(),
                                (T*)b.X[nxt], (T*)b.PHI[nxt], b.LAY[nxt], g->err_d, bs));
    launch_corrector<T>(G, g->bodies[m], bbc, b.blocks, b.list, b.count, b.redo, wls_blocks(), (const T*)b.X[cur], b.LAY[cur],
                        (const T*)b.X[nxt], b.LAY[nxt], (T*)b.XH, (T*)b.PHIH, g->err_d, bs);
    CK(g, cudaEventRecord(g->ev_join[m], bs));
  }
  for (int m = 0; m < nb; m++) CK(g, cudaStreamWaitEvent(s, g->ev_join[m], 0));
  pe(g, P_EXTRAP);
  // 8. tau^{n+1/2}; 9. rho^{n+1/2}; 10. u*
  pb(g, P_STRESS_H);
  CK(g, launch_stress_div<T>(G, u, g->bodies_d, views<T>(g, cur, 1), nb, g->bb_all + 6 * nxt, 12, g->t_d,
                              0.5 * G.dt, (T*)g->divh, g->slist, g->scount, slopes, s));
  pe(g, P_STRESS_H);
  pb(g, P_USTAR);
  launch_density<T>(G, g->bodies_d, views<T>(g, cur, 1), nb, g->bb_all + 6 * nxt, 12, (T*)g->rho_h, s);
  launch_ustar<T>(G, u, (const T*)g->adv, (const T*)g->p, (const T*)g->rho_h, (const T*)g->divh, (T*)g->ustar,
                  g->bodies_d, views<T>(g, cur, 1), nb, s);
  pe(g, P_USTAR);
  // 11. approximate projection, u^{n+1}, p^{n+1/2}
  pb(g, P_FE_SETUP);
  launch_fe_setup<T>(G, u, (const T*)g->ustar, mg_rhs(g->fe), s);
  mg_set_density(g->fe, g->rho_h);
  pe(g, P_FE_SETUP);
  pb(g, P_FE_SOLVE);
  cyc = mg_solve(g->fe, rtol, maxc, g->desc.mg_fixed_cycles_fe > 0 ? g->desc.mg_fixed_cycles_fe : g->desc.mg_fixed_cycles,
               s, &ce);
  pe(g, P_FE_SOLVE);
  if (ce != cudaSuccess) return fail(g, RMT_ECUDA, "FE solve: %s", cudaGetErrorString(ce));
  if (cyc < 0) {
    const rmt_status es = check_err(g);
    if (es != RMT_OK) return es;
    return fail(g, RMT_ENOCONVERGE, "FE multigrid missed rtol %.3g in %d cycles at step %ld", rtol, maxc, g->step);
  }
  g->cycles[1] = cyc;
  pb(g, P_FE_UPDATE);
  launch_fe_update<T>(G, (const T*)g->ustar, (const T*)g->rho_h, mg_solution(g->fe), u, (T*)g->p, (T*)g->psi, s);
  // 12. xi <- xi^{n+1} (parity flip); 13. rho^{n+1}
  g->par = nxt;
  launch_density<T>(G, g->bodies_d, views<T>(g, nxt, 0), nb, g->bb_all + 6 * nxt, 12, (T*)g->rho, s);
  launch_tick(g->t_d, G.dt, s);
  pe(g, P_FE_UPDATE);
  // the error words reach the host with the step (no synchronisation; read by poll_err)
  CK(g, cudaMemcpyAsync(g->err_h, g->err_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(g, cudaGetLastError());
  g->t += G.dt;
  g->step++;
  return RMT_OK;
}

rmt_status ensure_init(rmt_grid* g) {
  if (g->inited) return g->init_st;
  g->g.dt = pick_dt(g);
  g->g.utol = 1e-12 * g->g.h / g->g.dt;
  geo_finish(g->g);
  g->bodies.clear();
  for (const auto& s : g->solids) {
    Body b;
    b.shape = s.shape;
    for (int d = 0; d < 3; d++) {
      b.c[d] = s.center[d];
      b.a[d] = s.semi_axes[d];
    }
    for (int q = 0; q < 9; q++) b.R[q] = s.rot[q];
    b.rho_s = s.rho_s;
    b.G = s.G;
    b.mu_a = s.mu_a;
    b.gamma_t = s.gamma_t;
    b.actA = s.active_A;
    b.actW = s.active_omega;
    b.actL = s.active_len;
    b.repA = s.rep_A;
    body_finish(b);
    body_image(b, g->g);
    g->bodies.push_back(b);
    if (s.rep_A != 0.0) g->g.any_rep = 1;
  }
  g->g.dw = g->desc.wall_dw > 0.0 ? g->desc.wall_dw : g->g.h;
  g->g.f.dw = (float)g->g.dw;
  g->inited = 1;
  // a failed initialisation (allocation, CUDA error) leaves the state unusable: every later call
  // that needs it gets the same status
  g->init_st = g->fp32 ? init_t<float>(g) : init_t<double>(g);
  return g->init_st;
}

// the status the error words e[0..2] report (RMT_OK when all clear), recorded on g
rmt_status err_words(rmt_grid* g, const volatile int* e) {
  if (e[2] != 0)
    return fail(g, RMT_EDIVERGED, "non-finite values reached a pressure projection by step %ld (the velocity "
                "diverged)", g->step);
  if (e[0] != 0)
    return fail(g, RMT_EDEGENERATE, "%d least-squares extrapolations stayed degenerate up to r_s = 4", e[0]);
  if (e[1] != 0)
    return fail(g, RMT_ERANGE,
                "%d band cells came within %d cells of the seam of their body's periodic image window (FP32 "
                "storage keeps the reference map relative to a fixed image; the body has drifted about half a "
                "period)", e[1], SEAM_MARGIN);
  return RMT_OK;
}

// Without waiting: the error words as of the last step whose copy has landed (fixed-cycle and
// graph steps never synchronise, so a failure surfaces at a later call).  Records the first
// error found as the grid's sticky status.
rmt_status poll_err(rmt_grid* g) {
  if (!g->err_h || g->sticky != RMT_OK) return RMT_OK;
  return err_words(g, (const volatile int*)g->err_h);
}

// host-side fault injection before the step that is about to run: one velocity value becomes
// NaN (written from the host, as a diverging scheme would leave it)
rmt_status inject(rmt_grid* g) {
  if (g->inject_nan_step < 0 || g->step != g->inject_nan_step) return RMT_OK;
  const long c = g->g.N / 2 + g->g.n[0] / 2;
  CK(g, cudaMemsetAsync((char*)g->u + c * g->esz, 0xff, g->esz, g->s));  // all-ones bits: a NaN
  return RMT_OK;
}

rmt_status check_err(rmt_grid* g) {
  CK(g, cudaMemcpyAsync(g->err_h, g->err_d, 4 * sizeof(int), cudaMemcpyDeviceToHost, g->s));
  CK(g, cudaStreamSynchronize(g->s));
  return err_words(g, g->err_h);
}

// ----------------------------------------------------------------------------- step graphs
bool fixed_cycles(const rmt_grid* g) { return g->desc.mg_fixed_cycles > 0 && g->desc.mg_fixed_cycles_fe > 0; }

void drop_graphs(rmt_grid* g) {
  for (int p = 0; p < 2; p++) {
    if (g->gexec[p]) cudaGraphExecDestroy(g->gexec[p]);
    g->gexec[p] = nullptr;
    g->gnodes[p] = 0;
  }
}

// host-side effect of one step, for a step that ran from a captured graph
void advance_host(rmt_grid* g) {
  g->par = 1 - g->par;
  g->t += g->g.dt;
  g->step++;
  g->cycles[0] = g->desc.mg_fixed_cycles;
  g->cycles[1] = g->desc.mg_fixed_cycles_fe;
}

// Records one step of g on stream cs, which is capturing; the host state (parity, time, step
// count) is left as it was, since nothing has run yet.
rmt_status capture_step(rmt_grid* g, cudaStream_t cs) {
  const int par = g->par, prof = g->prof.on;
  const double t = g->t;
  const long step = g->step;
  cudaStream_t s0 = g->s;
  g->s = cs;
  g->prof.on = 0;
  rmt_status st = g->fp32 ? step_t<float>(g) : step_t<double>(g);
  g->s = s0;
  g->prof.on = prof;
  g->par = par;
  g->t = t;
  g->step = step;
  return st;
}

// captures and instantiates the step graph of the grid's current parity
rmt_status build_graph(rmt_grid* g) {
  if (!g->cap_s) CK(g, cudaStreamCreateWithFlags(&g->cap_s, cudaStreamNonBlocking));
  const long c0 = rmt_kernel_launches();
  CK(g, cudaStreamBeginCapture(g->cap_s, cudaStreamCaptureModeRelaxed));
  rmt_status st = capture_step(g, g->cap_s);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->cap_s, &graph);
  const long nodes = rmt_kernel_launches() - c0;
  rmt_count_launches(-nodes);  // counted when the graph is launched
  if (st != RMT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(g, RMT_ECUDA, "step capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g->gexec[g->par], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(g, RMT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  g->gnodes[g->par] = nodes;
  return RMT_OK;
}

}  // namespace

namespace {
template <typename T>
rmt_status gather_t(rmt_grid* g, int field, int sid, double* out) {
  const Geo& G = g->g;
  const long N = G.N;
  cudaStream_t s = g->s;
  auto cvt = [&](const void* src, long n, long off) { k_cvt<T><<<nbk(n), 256, 0, s>>>((const T*)src, out + off, n); rmt_count_launches(1); };
  switch (field) {
    case RMT_F_U: cvt(g->u, 3 * N, 0); break;
    case RMT_F_P: cvt(g->p, G.NN, 0); break;
    case RMT_F_RHO: cvt(g->rho, N, 0); break;
    case RMT_F_XI:
      k_xi_out<T><<<nbk(3 * N), 256, 0, s>>>(G, g->bodies[sid], (const T*)g->bm[sid].X[g->par], out);
      rmt_count_launches(1);
      break;
    case RMT_F_PHI: cvt(g->bm[sid].PHI[g->par], N, 0); break;
    case RMT_F_LAYER: k_cvt_i8<<<nbk(N), 256, 0, s>>>(g->bm[sid].LAY[g->par], out, N); rmt_count_launches(1); break;
    case RMT_F_XI_HALF:
      k_xi_out<T><<<nbk(3 * N), 256, 0, s>>>(G, g->bodies[sid], (const T*)g->bm[sid].XH, out);
      rmt_count_launches(1);
      break;
    case RMT_F_DIVTAU_N: cvt(g->divn, 3 * N, 0); break;
    case RMT_F_DIVTAU_H: cvt(g->divh, 3 * N, 0); break;
    case RMT_F_ADV_U: cvt(g->adv, 3 * N, 0); break;
    case RMT_F_USTAR: cvt(g->ustar, 3 * N, 0); break;
    case RMT_F_RHO_HALF: cvt(g->rho_h, N, 0); break;
    case RMT_F_REPULSION:  // from the last step's half-level bodies
      launch_rep_field<T>(G, g->bodies_d, views<T>(g, 1 - g->par, 1), (int)g->bodies.size(), out, s);
      break;
    case RMT_F_MAC_Q:
      CK(g, cudaMemcpyAsync(out, mg_solution64(g->mac, s), N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      break;
    case RMT_F_PSI:
      CK(g, cudaMemcpyAsync(out, mg_solution64(g->fe, s), G.NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
      break;
    case RMT_F_UFACE_X: case RMT_F_UFACE_Y: case RMT_F_UFACE_Z: {
      const int d = field - RMT_F_UFACE_X;
      const long nf = nfaces(G, d);
      for (int a = 0; a < 3; a++) cvt(g->uf[d][a], nf, a * nf);
      break;
    }
    case RMT_F_UMAC_X: case RMT_F_UMAC_Y: case RMT_F_UMAC_Z: {
      const int d = field - RMT_F_UMAC_X;
      cvt(g->umac[d], nfaces(G, d), 0);
      break;
    }
    default: return fail(g, RMT_EINVAL, "unknown field %d", field);
  }
  CK(g, cudaGetLastError());
  return RMT_OK;
}

template <typename T>
rmt_status scatter_t(rmt_grid* g, int field, int sid) {
  const Geo& G = g->g;
  cudaStream_t s = g->s;
  if (field == RMT_F_U) {
    k_cvt_back<T><<<nbk(3 * G.N), 256, 0, s>>>(g->stage, (T*)g->u, 3 * G.N); rmt_count_launches(1);
  } else if (field == RMT_F_P) {
    k_cvt_back<T><<<nbk(G.NN), 256, 0, s>>>(g->stage, (T*)g->p, G.NN); rmt_count_launches(1);
  } else {
    BodyMem& b = g->bm[sid];
    k_xi_in<T><<<nbk(3 * G.N), 256, 0, s>>>(G, g->bodies[sid], g->stage, (T*)b.X[g->par]); rmt_count_launches(1);
    const int full_blocks = (int)std::min((G.N + 127) / 128, (long)sm_count() * 64);
    CK(g, launch_extrapolate<T>(G, g->bodies[sid], nullptr, b.bb + 6 * g->par, full_blocks, b.list, b.count, b.redo,
                                wls_blocks(), (T*)b.X[g->par], (T*)b.PHI[g->par], b.LAY[g->par], g->err_d, s));
    launch_density<T>(G, g->bodies_d, views<T>(g, g->par, 0), (int)g->bodies.size(), g->bb_all + 6 * g->par, 12,
                      (T*)g->rho, s);
  }
  CK(g, cudaGetLastError());
  return RMT_OK;
}
// the body of rmt_read_fields (FP64 dst) and rmt_read_fields_float (FP32 dst)
rmt_status read_field(rmt_grid* g, int field, int solid_id, void* dst, size_t dst_bytes, int dst_is_device, bool f32) {
  if (!g || !dst) return RMT_EINVAL;
  rmt_status st = ensure_init(g);
  if (st != RMT_OK) return st;
  const long n = rmt_field_len(g, field);
  if (n < 0) return fail(g, RMT_EINVAL, "unknown field %d", field);
  if (dst_bytes < (size_t)n * (f32 ? sizeof(float) : sizeof(double))) return fail(g, RMT_EINVAL, "destination too small");
  if ((field == RMT_F_XI || field == RMT_F_PHI || field == RMT_F_LAYER || field == RMT_F_XI_HALF) &&
      (solid_id < 0 || solid_id >= (int)g->bodies.size()))
    return fail(g, RMT_EINVAL, "bad solid id %d", solid_id);
  if (g->in_batch && g->batch_s != g->s) CK(g, cudaStreamSynchronize(g->batch_s));  // the batch's steps first
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f32 && g->fp32 && (field == RMT_F_U || field == RMT_F_P)) {
    // stored in this layout: one copy, no conversion
    CK(g, cudaMemcpyAsync(dst, field == RMT_F_U ? g->u : g->p, (size_t)n * sizeof(float), kind, g->s));
  } else if (f32) {
    st = g->fp32 ? gather_t<float>(g, field, solid_id, g->stage) : gather_t<double>(g, field, solid_id, g->stage);
    if (st != RMT_OK) return st;
    if (!g->stage_f) CK(g, cudaMalloc((void**)&g->stage_f, (size_t)g->stage_len * sizeof(float)));
    k_cvt_back<float><<<nbk(n), 256, 0, g->s>>>(g->stage, g->stage_f, n);
    rmt_count_launches(1);
    CK(g, cudaMemcpyAsync(dst, g->stage_f, (size_t)n * sizeof(float), kind, g->s));
  } else {
    double* out = dst_is_device ? (double*)dst : g->stage;
    st = g->fp32 ? gather_t<float>(g, field, solid_id, out) : gather_t<double>(g, field, solid_id, out);
    if (st != RMT_OK) return st;
    if (!dst_is_device) CK(g, cudaMemcpyAsync(dst, g->stage, (size_t)n * sizeof(double), kind, g->s));
  }
  CK(g, cudaStreamSynchronize(g->s));
  return RMT_OK;
}

// the body of rmt_write_fields (FP64 src) and rmt_write_fields_float (FP32 src)
rmt_status write_field(rmt_grid* g, int field, int solid_id, const void* src, size_t src_bytes, int src_is_device,
                       bool f32) {
  if (!g || !src) return RMT_EINVAL;
  if (g->sticky != RMT_OK) return RMT_ESTATE;
  rmt_status st = ensure_init(g);
  if (st != RMT_OK) return st;
  if (g->in_batch) return refuse(g, "the grid is stepped by its batch");
  if (field != RMT_F_U && field != RMT_F_P && field != RMT_F_XI) return fail(g, RMT_EINVAL, "field %d is not writable", field);
  if (field == RMT_F_XI && (solid_id < 0 || solid_id >= (int)g->bodies.size()))
    return fail(g, RMT_EINVAL, "bad solid id %d", solid_id);
  const long n = rmt_field_len(g, field);
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  if (src_bytes < (size_t)n * esz) return fail(g, RMT_EINVAL, "source too small");
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (f32 && g->fp32 && field != RMT_F_XI) {
    // U and P of an FP32 grid are stored in this layout: one copy, no conversion.  From
    // page-locked host memory the copy stays asynchronous (the host can launch the next step
    // while it runs; the caller keeps src until a synchronising call), from pageable memory the
    // call waits so that the caller may reuse src at once.
    CK(g, cudaMemcpyAsync(field == RMT_F_U ? g->u : g->p, src, (size_t)n * sizeof(float), kind, g->s));
    if (!src_is_device) {
      cudaPointerAttributes at;
      const cudaError_t pe = cudaPointerGetAttributes(&at, src);
      if (pe != cudaSuccess) cudaGetLastError();  // not a pointer the runtime knows: pageable
      const bool pinned = pe == cudaSuccess && at.type == cudaMemoryTypeHost;
      if (!pinned) CK(g, cudaStreamSynchronize(g->s));
    }
    return RMT_OK;
  }
  if (f32) {
    if (!g->stage_f) CK(g, cudaMalloc((void**)&g->stage_f, (size_t)g->stage_len * sizeof(float)));
    CK(g, cudaMemcpyAsync(g->stage_f, src, (size_t)n * sizeof(float), kind, g->s));
    k_cvt<float><<<nbk(n), 256, 0, g->s>>>(g->stage_f, g->stage, n);
    rmt_count_launches(1);
  } else {
    CK(g, cudaMemcpyAsync(g->stage, src, (size_t)n * sizeof(double), kind, g->s));
  }
  if (field == RMT_F_XI) drop_graphs(g);  // re-extrapolation resizes the body's launch windows
  st = g->fp32 ? scatter_t<float>(g, field, solid_id) : scatter_t<double>(g, field, solid_id);
  if (st != RMT_OK) return st;
  if (field == RMT_F_XI) {
    if ((st = check_err(g)) != RMT_OK) return st;
    return size_windows(g);
  }
  if (!src_is_device) CK(g, cudaStreamSynchronize(g->s));  // the caller may reuse src
  return RMT_OK;
}

}  // namespace

extern "C" {

rmt_status rmt_create_grid(const rmt_grid_desc* d, rmt_grid** out) {
  if (!d || !out) return RMT_EINVAL;
  *out = nullptr;
  for (int a = 0; a < 3; a++) {
    if (d->n[a] < 4 || !(d->hi[a] > d->lo[a])) return RMT_EINVAL;
    const int p0 = d->bc[2 * a] == RMT_BC_PERIODIC, p1 = d->bc[2 * a + 1] == RMT_BC_PERIODIC;
    if (p0 != p1) return RMT_EINVAL;
    if (!p0 && (d->bc[2 * a] != RMT_BC_NOSLIP || d->bc[2 * a + 1] != RMT_BC_NOSLIP)) return RMT_EINVAL;
    if (p0 && (d->n[a] & 1)) return RMT_EINVAL;  // red-black colouring needs an even period
    if (d->wall_u[2 * a][a] != 0.0 || d->wall_u[2 * a + 1][a] != 0.0) return RMT_EINVAL;
  }
  // cell, node and face indices are formed in 32-bit arithmetic
  if ((long)(d->n[0] + 1) * (d->n[1] + 1) * (d->n[2] + 1) >= (1L << 31)) return RMT_EINVAL;
  const double h = (d->hi[0] - d->lo[0]) / d->n[0];
  for (int a = 1; a < 3; a++)
    if (fabs((d->hi[a] - d->lo[a]) / d->n[a] - h) > 1e-12 * h) return RMT_EINVAL;
  if (!(d->rho_f > 0) || !(d->mu >= 0) || !(d->eps_h > 0) || d->band_layers < 1 || d->band_layers > 8)
    return RMT_EINVAL;
  if (d->precision != RMT_PREC_FP64 && d->precision != RMT_PREC_FP32_REFINE) return RMT_EINVAL;
  rmt_grid* g = new (std::nothrow) rmt_grid();
  if (!g) return RMT_ENOMEM;
  g->desc = *d;
  g->s = (cudaStream_t)d->cuda_stream;
  g->fp32 = d->precision == RMT_PREC_FP32_REFINE;
  g->esz = g->fp32 ? 4 : 8;
  Geo& G = g->g;
  for (int a = 0; a < 3; a++) {
    G.n[a] = d->n[a];
    G.per[a] = d->bc[2 * a] == RMT_BC_PERIODIC;
    G.nn[a] = G.per[a] ? G.n[a] : G.n[a] + 1;
    G.lo[a] = d->lo[a];
    G.len[a] = d->hi[a] - d->lo[a];
    G.grav[a] = d->gravity[a];
  }
  for (int f = 0; f < 6; f++)
    for (int a = 0; a < 3; a++) G.wall[f][a] = d->wall_u[f][a];
  G.N = (long)G.n[0] * G.n[1] * G.n[2];
  G.NN = (long)G.nn[0] * G.nn[1] * G.nn[2];
  G.h = h;
  G.eps = d->eps_h * h;
  G.rho_f = d->rho_f;
  G.mu = d->mu;
  G.layers = d->band_layers;
  G.dt = 0.0;
  *out = g;
  return RMT_OK;
}

rmt_status rmt_add_solid(rmt_grid* g, const rmt_solid_desc* s, int* solid_id) {
  if (!g || !s) return RMT_EINVAL;
  if (g->inited) return fail(g, RMT_ESTATE, "bodies must be added before the first step, read or write");
  if (g->solids.size() >= RMT_MAX_BODIES) return fail(g, RMT_EINVAL, "at most %d bodies", RMT_MAX_BODIES);
  if (s->shape != RMT_SHAPE_SPHERE && s->shape != RMT_SHAPE_ELLIPSOID) return fail(g, RMT_EINVAL, "unknown shape");
  for (int a = 0; a < 3; a++)
    if (!(s->semi_axes[a] > 0) && !(s->shape == RMT_SHAPE_SPHERE && a > 0)) return fail(g, RMT_EINVAL, "semi-axes must be positive");
  if (!(s->rho_s > 0) || !(s->G >= 0) || !(s->mu_a >= 0)) return fail(g, RMT_EINVAL, "bad material constants");
  if (s->active_A != 0.0 && !(s->active_len > 0)) return fail(g, RMT_EINVAL, "active_len must be positive");
  g->solids.push_back(*s);
  if (solid_id) *solid_id = (int)g->solids.size() - 1;
  return RMT_OK;
}

rmt_status rmt_step(rmt_grid* g, int nsteps) {
  if (!g || nsteps < 0) return RMT_EINVAL;
  rmt_status st = poll_err(g);  // a failure of an earlier, unsynchronised step
  if (st != RMT_OK) return st;
  if (g->sticky != RMT_OK) return RMT_ESTATE;
  if (g->in_batch) return refuse(g, "the grid is stepped by its batch");
  st = ensure_init(g);
  if (st != RMT_OK) return st;
  if (g->use_graph && fixed_cycles(g) && !g->prof.on) {
    for (int k = 0; k < nsteps; k++) {
      if ((st = inject(g)) != RMT_OK) return st;
      if (!g->gexec[g->par] && (st = build_graph(g)) != RMT_OK) return st;
      CK(g, cudaGraphLaunch(g->gexec[g->par], g->s));
      rmt_count_launches(g->gnodes[g->par]);
      advance_host(g);
    }
    return RMT_OK;
  }
  for (int k = 0; k < nsteps; k++) {
    if ((st = inject(g)) != RMT_OK) return st;
    st = g->fp32 ? step_t<float>(g) : step_t<double>(g);
    if (st != RMT_OK) return st;
  }
  if (g->desc.mg_fixed_cycles <= 0) return check_err(g);
  return RMT_OK;
}

rmt_status rmt_init_pressure(rmt_grid* g, int max_iters, double tol, int* iters_out) {
  if (!g || max_iters < 0 || !(tol >= 0.0)) return RMT_EINVAL;
  if (g->in_batch) return refuse(g, "the grid is stepped by its batch");
  if (g->sticky != RMT_OK) return RMT_ESTATE;
  rmt_status st = ensure_init(g);
  if (st != RMT_OK) return st;
  if (g->step != 0) return refuse(g, "initial pressure iterations run before the first step");
  const Geo& G = g->g;
  const size_t e = g->esz;
  void *u0 = nullptr, *rho0 = nullptr;
  CK(g, cudaMalloc(&u0, 3 * G.N * e));
  if (cudaMalloc(&rho0, G.N * e) != cudaSuccess) {
    cudaFree(u0);
    return fail(g, RMT_ENOMEM, "initial pressure iterations: no memory for the saved state");
  }
  std::vector<double> prev((size_t)G.NN), cur((size_t)G.NN);
  auto read_p = [&](std::vector<double>& dst) -> rmt_status {
    rmt_status s2 = g->fp32 ? gather_t<float>(g, RMT_F_P, 0, g->stage) : gather_t<double>(g, RMT_F_P, 0, g->stage);
    if (s2 != RMT_OK) return s2;
    CK(g, cudaMemcpyAsync(dst.data(), g->stage, G.NN * sizeof(double), cudaMemcpyDeviceToHost, g->s));
    CK(g, cudaStreamSynchronize(g->s));
    return RMT_OK;
  };
  int it = 0;
  st = RMT_OK;
  if (cudaMemcpyAsync(u0, g->u, 3 * G.N * e, cudaMemcpyDeviceToDevice, g->s) != cudaSuccess ||
      cudaMemcpyAsync(rho0, g->rho, G.N * e, cudaMemcpyDeviceToDevice, g->s) != cudaSuccess)
    st = fail(g, RMT_ECUDA, "initial pressure iterations: saving the state failed");
  if (st == RMT_OK) st = read_p(prev);
  while (st == RMT_OK && it < max_iters) {
    // a step from the initial state with the current estimate of p^{-1/2} ...
    const int prof = g->prof.on;
    g->prof.on = 0;
    st = g->fp32 ? step_t<float>(g) : step_t<double>(g);
    g->prof.on = prof;
    it++;
    // ... keeps only p^{1/2}: u, rho, the reference maps (their parity), time and step count
    // return to the initial state
    g->par = 1 - g->par;
    g->t = 0.0;
    g->step = 0;
    if (cudaMemcpyAsync(g->u, u0, 3 * G.N * e, cudaMemcpyDeviceToDevice, g->s) != cudaSuccess ||
        cudaMemcpyAsync(g->rho, rho0, G.N * e, cudaMemcpyDeviceToDevice, g->s) != cudaSuccess ||
        cudaMemsetAsync(g->t_d, 0, sizeof(double), g->s) != cudaSuccess) {
      st = fail(g, RMT_ECUDA, "initial pressure iterations: restoring the state failed");
      break;
    }
    if (st != RMT_OK) break;
    if ((st = read_p(cur)) != RMT_OK) break;
    double dn = 0.0, pn = 0.0;
    for (long q = 0; q < G.NN; q++) {
      const double dv = cur[q] - prev[q];
      dn += dv * dv;
      pn += cur[q] * cur[q];
    }
    if (dn <= tol * tol * pn) break;
    prev.swap(cur);
  }
  cudaStreamSynchronize(g->s);
  cudaFree(u0);
  cudaFree(rho0);
  if (iters_out) *iters_out = it;
  if (st != RMT_OK) return st;
  return check_err(g);
}

long rmt_field_len(rmt_grid* g, int field) {
  if (!g) return -1;
  const Geo& G = g->g;
  switch (field) {
    case RMT_F_U: case RMT_F_XI: case RMT_F_DIVTAU_N: case RMT_F_DIVTAU_H: case RMT_F_ADV_U:
    case RMT_F_USTAR: case RMT_F_XI_HALF: case RMT_F_REPULSION: return 3 * G.N;
    case RMT_F_P: case RMT_F_PSI: return G.NN;
    case RMT_F_RHO: case RMT_F_PHI: case RMT_F_LAYER: case RMT_F_MAC_Q: case RMT_F_RHO_HALF: return G.N;
    case RMT_F_UFACE_X: case RMT_F_UFACE_Y: case RMT_F_UFACE_Z: return 3 * nfaces(G, field - RMT_F_UFACE_X);
    case RMT_F_UMAC_X: case RMT_F_UMAC_Y: case RMT_F_UMAC_Z: return nfaces(G, field - RMT_F_UMAC_X);
  }
  return -1;
}


rmt_status rmt_read_fields(rmt_grid* g, int field, int solid_id, void* dst, size_t dst_bytes, int dst_is_device) {
  return read_field(g, field, solid_id, dst, dst_bytes, dst_is_device, false);
}

rmt_status rmt_read_fields_float(rmt_grid* g, int field, int solid_id, void* dst, size_t dst_bytes,
                                 int dst_is_device) {
  return read_field(g, field, solid_id, dst, dst_bytes, dst_is_device, true);
}

rmt_status rmt_body_stats(rmt_grid* g, int solid_id, double out[7]) {
  if (!g || !out) return RMT_EINVAL;
  rmt_status st = ensure_init(g);
  if (st != RMT_OK) return st;
  if (solid_id < 0 || solid_id >= (int)g->bodies.size()) return fail(g, RMT_EINVAL, "bad solid id %d", solid_id);
  if (g->in_batch && g->batch_s != g->s) CK(g, cudaStreamSynchronize(g->batch_s));
  const Geo& G = g->g;
  const size_t need = body_stats_scratch_bytes();
  double* scratch = g->stage;
  double* tmp = nullptr;
  if ((size_t)g->stage_len * sizeof(double) < need) {
    CK(g, cudaMalloc(&tmp, need));
    scratch = tmp;
  }
  const Body& b = g->bodies[solid_id];
  const BodyMem& m = g->bm[solid_id];
  const int par = g->par;
  if (g->fp32)
    launch_body_stats<float>(G, (const float*)g->u, b, BodyView<float>{(const float*)m.X[par], (const float*)m.PHI[par], m.LAY[par]},
                             g->t_d, scratch, g->s);
  else
    launch_body_stats<double>(G, (const double*)g->u, b,
                              BodyView<double>{(const double*)m.X[par], (const double*)m.PHI[par], m.LAY[par]}, g->t_d,
                              scratch, g->s);
  double sums[8];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums, scratch, sizeof sums, cudaMemcpyDeviceToHost, g->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(g, RMT_ECUDA, "body statistics: %s", cudaGetErrorString(e));
  const double dv = G.h * G.h * G.h;
  for (int a = 0; a < 3; a++) out[a] = sums[3] > 0.0 ? sums[a] / sums[3] : 0.0;
  out[3] = -sums[4] * dv;
  out[4] = sums[3] * dv;
  out[5] = sums[5] * dv;
  out[6] = sums[6] > 0.0 ? sqrt(sums[7] / sums[6]) : 0.0;
  return RMT_OK;
}

rmt_status rmt_write_fields(rmt_grid* g, int field, int solid_id, const void* src, size_t src_bytes, int src_is_device) {
  return write_field(g, field, solid_id, src, src_bytes, src_is_device, false);
}

rmt_status rmt_write_fields_float(rmt_grid* g, int field, int solid_id, const void* src, size_t src_bytes,
                                  int src_is_device) {
  return write_field(g, field, solid_id, src, src_bytes, src_is_device, true);
}

int rmt_last_cycles(rmt_grid* g, int which) { return g ? g->cycles[which ? 1 : 0] : -1; }
double rmt_dt(rmt_grid* g) { return g ? g->g.dt : 0.0; }

rmt_status rmt_destroy_grid(rmt_grid* g) {
  if (!g) return RMT_EINVAL;
  if (g->in_batch) return refuse(g, "remove the grid from its batch first");
  if (g->s) cudaStreamSynchronize(g->s);
  else cudaDeviceSynchronize();
  drop_graphs(g);
  if (g->cap_s) cudaStreamDestroy(g->cap_s);
  for (cudaStream_t b : g->body_s)
    if (b) cudaStreamDestroy(b);
  for (cudaEvent_t e : g->ev_join)
    if (e) cudaEventDestroy(e);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  for (void* p : g->allocs) cudaFree(p);
  if (g->stage_f) cudaFree(g->stage_f);
  if (g->err_h) cudaFreeHost(g->err_h);
  mg_destroy(g->mac);
  mg_destroy(g->fe);
  for (auto& r : g->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : g->prof.pool) cudaEventDestroy(e);
  delete g;
  return RMT_OK;
}

const char* rmt_last_error(const rmt_grid* g) { return g ? g->msg : "null grid"; }

long rmt_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rmt_status rmt_profile(rmt_grid* g, int enable) {
  if (!g) return RMT_EINVAL;
  prof_flush(g);
  if (enable) {
    for (int e = 0; e < P_NUM; e++) {
      g->prof.ms[e] = 0.0;
      g->prof.n[e] = 0;
    }
  }
  g->prof.on = enable ? 1 : 0;
  return RMT_OK;
}

int rmt_profile_entries(void) { return P_NUM; }

rmt_status rmt_set_option(rmt_grid* g, const char* name, double value) {
  if (!g || !name) return RMT_EINVAL;
  if (g->in_batch) return refuse(g, "the grid is stepped by its batch");
  int* ip = nullptr;
  if (!strcmp(name, "mac_pre")) ip = &g->mac_pre;
  else if (!strcmp(name, "mac_post")) ip = &g->mac_post;
  else if (!strcmp(name, "fe_pre")) ip = &g->fe_pre;
  else if (!strcmp(name, "fe_post")) ip = &g->fe_post;
  else if (!strcmp(name, "mac_inner")) ip = &g->mac_inner;
  else if (!strcmp(name, "fe_inner")) ip = &g->fe_inner;
  else if (!strcmp(name, "mac_warm")) ip = &g->mac_warm;
  else if (!strcmp(name, "mac_sweep")) ip = &g->mac_sweep;
  else if (!strcmp(name, "fe_warm")) ip = &g->fe_warm;
  else if (!strcmp(name, "mac_coarse_pre")) ip = &g->mac_cpre;
  else if (!strcmp(name, "mac_coarse_post")) ip = &g->mac_cpost;
  else if (!strcmp(name, "fe_coarse_pre")) ip = &g->fe_cpre;
  else if (!strcmp(name, "fe_coarse_post")) ip = &g->fe_cpost;
  if (ip) {
    if (value < 0 || value > 16) return fail(g, RMT_EINVAL, "%s out of range", name);
    *ip = (int)value;
  } else if (!strcmp(name, "mac_block") || !strcmp(name, "fe_block")) {
    const int v = (int)value;
    if (v != 1 && v != 2 && v != 4 && v != 8) return fail(g, RMT_EINVAL, "%s must be 1, 2, 4 or 8", name);
    (name[0] == 'm' ? g->mac_block : g->fe_block) = v;
  } else if (!strcmp(name, "mac_cycles") || !strcmp(name, "fe_cycles")) {
    if (value < 0 || value > 1000) return fail(g, RMT_EINVAL, "%s out of range", name);
    (name[0] == 'm' ? g->desc.mg_fixed_cycles : g->desc.mg_fixed_cycles_fe) = (int)value;
  } else if (!strcmp(name, "fe_omega") || !strcmp(name, "mac_omega")) {
    if (!(value > 0.0 && value < 2.0)) return fail(g, RMT_EINVAL, "%s out of range", name);
    (name[0] == 'f' ? g->fe_omega : g->mac_omega) = value;
  } else if (!strcmp(name, "mac_zchunk") || !strcmp(name, "fe_zchunk")) {
    if (value < 0 || value > 65536) return fail(g, RMT_EINVAL, "%s out of range", name);
    (name[0] == 'm' ? g->mac_zchunk : g->fe_zchunk) = (int)value;
  } else if (!strcmp(name, "graph")) {
    g->use_graph = value != 0.0;
  } else if (!strcmp(name, "inject_nan_step")) {
    g->inject_nan_step = value < 0 ? -1 : (long)value;
  } else if (!strcmp(name, "inject_alloc")) {
    if (g->inited) return refuse(g, "inject_alloc is set before the grid allocates");
    g->inject_alloc = value < 0 ? -1 : (long)value;
  } else {
    return fail(g, RMT_EINVAL, "unknown option %s", name);
  }
  drop_graphs(g);
  if (g->inited) {
    mg_set_smoother(g->mac, g->mac_pre, g->mac_post, g->mac_omega);
    mg_set_smoother(g->fe, g->fe_pre, g->fe_post, g->fe_omega);
    mg_set_coarse_smoother(g->mac, g->mac_cpre, g->mac_cpost);
    mg_set_coarse_smoother(g->fe, g->fe_cpre, g->fe_cpost);
    mg_set_inner(g->mac, g->mac_inner);
    mg_set_inner(g->fe, g->fe_inner);
    mg_set_block(g->mac, g->mac_block);
    mg_set_block(g->fe, g->fe_block);
    mg_set_warm(g->mac, g->mac_warm);
    mg_set_sweep(g->mac, g->mac_sweep);
    mg_set_warm(g->fe, g->fe_warm);
    mg_set_zchunk(g->mac, g->mac_zchunk);
    mg_set_zchunk(g->fe, g->fe_zchunk);
  }
  return RMT_OK;
}

size_t rmt_grid_footprint(const rmt_grid_desc* d, int nsolids) {
  if (nsolids < 0 || nsolids > RMT_MAX_BODIES) return 0;
  rmt_grid* g = nullptr;
  if (rmt_create_grid(d, &g) != RMT_OK) return 0;
  g->bodies.resize(nsolids);  // only the count matters to the allocation sizes
  g->dry = 1;
  const rmt_status st = g->fp32 ? alloc_t<float>(g) : alloc_t<double>(g);
  const size_t b = st == RMT_OK ? g->bytes : 0;
  delete g;  // nothing was allocated
  return b;
}

size_t rmt_grid_device_bytes(const rmt_grid* g) { return g ? g->bytes : 0; }

double rmt_wall_repulsion(double V, double U, double d_w, double L_min, double rho_s, double rho_f, double g,
                          double U_safe) {
  const double vrep = d_w * L_min * L_min;  // the breached volume the paper assumes
  double a = U_safe * U_safe / d_w;
  const double stop = V * U * U / (2.0 * d_w * vrep), hold = fabs(rho_s - rho_f) * V * g / (rho_s * vrep);
  if (stop > a) a = stop;
  if (hold > a) a = hold;
  return a;
}

const char* rmt_profile_name(int entry) { return (entry >= 0 && entry < P_NUM) ? kProfNames[entry] : ""; }

rmt_status rmt_profile_read(rmt_grid* g, int entry, double* total_ms, long* launches, double* bytes_per_launch) {
  if (!g || entry < 0 || entry >= P_NUM) return RMT_EINVAL;
  prof_flush(g);
  if (total_ms) *total_ms = g->prof.ms[entry];
  if (launches) *launches = g->prof.n[entry];
  if (bytes_per_launch) *bytes_per_launch = prof_bytes(g, entry);
  return RMT_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- batch hooks
rmt_status grid_join_batch(rmt_grid* g, cudaStream_t batch_stream) {
  if (!g) return RMT_EINVAL;
  if (g->in_batch) return refuse(g, "the grid already belongs to a batch");
  if (g->sticky != RMT_OK) return RMT_ESTATE;
  if (!fixed_cycles(g)) return fail(g, RMT_EINVAL, "batched grids need mg_fixed_cycles and mg_fixed_cycles_fe > 0");
  if (g->prof.on) return refuse(g, "profiling is on");
  rmt_status st = ensure_init(g);
  if (st != RMT_OK) return st;
  if ((st = check_err(g)) != RMT_OK) return st;  // also waits for the grid's own work
  g->in_batch = 1;
  g->batch_s = batch_stream;
  return RMT_OK;
}
void grid_leave_batch(rmt_grid* g) {
  g->in_batch = 0;
  g->batch_s = nullptr;
}
rmt_status grid_capture_step(rmt_grid* g, cudaStream_t s) { return capture_step(g, s); }
void grid_advance_host(rmt_grid* g) { advance_host(g); }
int grid_parity(const rmt_grid* g) { return g->par; }
rmt_status grid_check(rmt_grid* g) {
  if (g->sticky != RMT_OK) return g->sticky;
  return check_err(g);
}
rmt_status grid_fail(rmt_grid* g, rmt_status st, const char* msg) { return fail(g, st, "%s", msg); }
rmt_status grid_pre_step(rmt_grid* g, cudaStream_t s) {
  cudaStream_t s0 = g->s;
  g->s = s;
  const rmt_status st = inject(g);
  g->s = s0;
  return st;
}
rmt_status grid_poll(rmt_grid* g) {
  const rmt_status st = poll_err(g);
  return st != RMT_OK ? st : g->sticky;
}

// ----------------------------------------------------------------------------- autotuner hooks
rmt_status grid_solvers(rmt_grid* g, MGSolver** mac, MGSolver** fe, cudaStream_t* s, double* rtol) {
  if (!g->inited || g->step == 0) return refuse(g, "the autotuner needs a grid that has taken a step");
  *mac = g->mac;
  *fe = g->fe;
  *s = g->s;
  *rtol = g->desc.mg_rtol > 0 ? g->desc.mg_rtol : 1e-12;
  return RMT_OK;
}
