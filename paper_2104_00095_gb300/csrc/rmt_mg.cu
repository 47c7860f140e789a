// Geometric multigrid for the two projections of the RMT step (arXiv 2104.00095, SI
// "MAC projection" and "Approximate pressure-Poisson projection"; the paper solves both
// with its own multigrid library whose design it does not describe).
//
// kind 0 (MAC): cell-centred variable-coefficient 7-point operator
//     (A q)_c = h^-2 sum_faces beta_f (q_c - q_nb),  beta_f = 1/rho_face, 0 on walls.
// kind 1 (FE): nodal trilinear finite-element stiffness, beta = 1/rho per cell
//     (K psi)_i = (h/12) sum_{cells c at i} beta_c (4 psi_i - sum of the 4 corners of c that
//     differ from i in two or three coordinates).
// Both operators are symmetric positive semi-definite with the constants as null space
// (walls are Neumann, periodic axes wrap); right-hand sides and solutions are kept mean-free.
//
// Solve = iterative refinement: the residual of the FP64 iterate is formed in FP64 and a
// V(2,2)-cycle in the storage type T (double or float) approximately solves for the
// correction.  Smoothers: red-black Gauss-Seidel (7-point), 8-colour Gauss-Seidel
// (27-point).  Transfers: averaging / trilinear (cell-centred), full weighting / trilinear
// (nodal).  Coarse operators are re-discretised with averaged coefficients.  The coarsest
// level is solved by one thread block with many smoothing sweeps.  All norms use fixed-order
// two-stage reductions, so results are deterministic.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rmt_kernels.h"

namespace {

constexpr int TPB = 256;
constexpr int RED_BLOCKS = 1024;
inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > 152L * 32) b = 152L * 32;
  return (int)(b < 1 ? 1 : b);
}

struct Lv {
  int n[3], nn[3], per[3];
  long ncell, nnode, nunk;
  double h;
};

__device__ __forceinline__ void dec3(long c, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(c % nx);
  long r = c / nx;
  j = (int)(r % ny);
  k = (int)(r / ny);
}
__device__ __forceinline__ long cix(const Lv& L, int i, int j, int k) { return i + (long)L.n[0] * (j + (long)L.n[1] * k); }
__device__ __forceinline__ long nix(const Lv& L, int i, int j, int k) { return i + (long)L.nn[0] * (j + (long)L.nn[1] * k); }
__device__ __forceinline__ long fix(const Lv& L, int d, int i, int j, int k) {
  long e0 = L.n[0] + (d == 0), e1 = L.n[1] + (d == 1);
  return i + e0 * (j + e1 * (long)k);
}
// neighbour cell along d (s = +-1): wrap on periodic axes, clamp at walls (face beta is 0 there)
__device__ __forceinline__ int nbc(const Lv& L, int d, int i, int s) {
  int v = i + s;
  if (v < 0) return L.per[d] ? L.n[d] - 1 : 0;
  if (v >= L.n[d]) return L.per[d] ? 0 : L.n[d] - 1;
  return v;
}
// cell coordinate for the FE cell loop; false outside a wall
__device__ __forceinline__ bool cellc(const Lv& L, int d, int& i) {
  if (i >= 0 && i < L.n[d]) return true;
  if (!L.per[d]) return false;
  i = (i + L.n[d]) % L.n[d];
  return true;
}
__device__ __forceinline__ int nodec(const Lv& L, int d, int i) {
  if (L.per[d]) {
    if (i >= L.nn[d]) i -= L.nn[d];
    if (i < 0) i += L.nn[d];
  }
  return i;
}

// ----------------------------------------------------------------------------- operators
// MAC: returns (A x)_c and the diagonal; XT: type of x, CT: type of coefficients
template <typename XT, typename CT>
__device__ __forceinline__ double mac_apply(const Lv& L, const XT* __restrict__ x, const CT* __restrict__ bx,
                                            const CT* __restrict__ by, const CT* __restrict__ bz, int i, int j, int k,
                                            double& diag) {
  const long c = cix(L, i, j, k);
  const double b0 = bx[fix(L, 0, i, j, k)], b1 = bx[fix(L, 0, i + 1, j, k)];
  const double b2 = by[fix(L, 1, i, j, k)], b3 = by[fix(L, 1, i, j + 1, k)];
  const double b4 = bz[fix(L, 2, i, j, k)], b5 = bz[fix(L, 2, i, j, k + 1)];
  const double off = b0 * (double)x[cix(L, nbc(L, 0, i, -1), j, k)] + b1 * (double)x[cix(L, nbc(L, 0, i, 1), j, k)] +
                     b2 * (double)x[cix(L, i, nbc(L, 1, j, -1), k)] + b3 * (double)x[cix(L, i, nbc(L, 1, j, 1), k)] +
                     b4 * (double)x[cix(L, i, j, nbc(L, 2, k, -1))] + b5 * (double)x[cix(L, i, j, nbc(L, 2, k, 1))];
  diag = b0 + b1 + b2 + b3 + b4 + b5;
  const double ih2 = 1.0 / (L.h * L.h);
  diag *= ih2;
  return diag * (double)x[c] - off * ih2;
}

// FE: returns (K x)_i and the diagonal
template <typename XT, typename CT>
__device__ __forceinline__ double fe_apply(const Lv& L, const XT* __restrict__ x, const CT* __restrict__ beta, int i,
                                           int j, int k, double& diag) {
  const double xi = (double)x[nix(L, i, j, k)];
  double acc = 0.0, bs = 0.0;
#pragma unroll
  for (int s = 0; s < 8; s++) {
    const int sx = s & 1, sy = (s >> 1) & 1, sz = (s >> 2) & 1;
    int ci = i - 1 + sx, cj = j - 1 + sy, ck = k - 1 + sz;
    if (!cellc(L, 0, ci) || !cellc(L, 1, cj) || !cellc(L, 2, ck)) continue;
    const double b = (double)beta[cix(L, ci, cj, ck)];
    // node i sits at local corner (1-sx, 1-sy, 1-sz) of this cell; the corners differing in
    // two or three coordinates are the ones with at least two flipped bits
    const int qi = (1 - sx) | ((1 - sy) << 1) | ((1 - sz) << 2);
    double so = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (__popc(q ^ qi) < 2) continue;
      const int ni = nodec(L, 0, ci + (q & 1)), nj = nodec(L, 1, cj + ((q >> 1) & 1)), nk = nodec(L, 2, ck + ((q >> 2) & 1));
      so += (double)x[nix(L, ni, nj, nk)];
    }
    acc += b * (4.0 * xi - so);
    bs += b;
  }
  const double s12 = L.h / 12.0;
  diag = 4.0 * bs * s12;
  return acc * s12;
}

// ----------------------------------------------------------------------------- kernels
template <typename T>
__global__ void k_zero(T* a, long n) {
  GRID_LOOP(i, n) a[i] = T(0);
}

// FP64 residual r = b - A x of the FP64 iterate; writes the T copy for the V-cycle and
// per-block partial sums of r^2
template <typename CT>
__global__ void k_resid64(Lv L, int kind, const double* __restrict__ x, const double* __restrict__ b,
                          const CT* __restrict__ c0, const CT* __restrict__ c1, const CT* __restrict__ c2,
                          CT* __restrict__ rT, double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  double loc = 0.0;
  GRID_LOOP(u, L.nunk) {
    int i, j, k;
    double dg, ax;
    if (kind == 0) {
      dec3(u, L.n[0], L.n[1], i, j, k);
      ax = mac_apply(L, x, c0, c1, c2, i, j, k, dg);
    } else {
      dec3(u, L.nn[0], L.nn[1], i, j, k);
      ax = fe_apply(L, x, c0, i, j, k, dg);
    }
    const double r = b[u] - ax;
    rT[u] = (CT)r;
    loc += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < TPB / 32; w++) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// sum (mode 0) or sum of squares (mode 1) of a vector: per-block partials
template <typename XT>
__global__ void k_partial(const XT* __restrict__ a, long n, int mode, double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  double loc = 0.0;
  GRID_LOOP(i, n) {
    const double v = (double)a[i];
    loc += mode ? v * v : v;
  }
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < TPB / 32; w++) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// final fixed-order sum of the partials (one block); out = scale * sum
__global__ void k_final(const double* __restrict__ part, int np, double scale, double* __restrict__ out) {
  __shared__ double sh[1024];
  double loc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) loc += part[i];
  sh[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] * scale;
}

template <typename XT>
__global__ void k_sub_scalar(XT* __restrict__ a, long n, const double* __restrict__ s) {
  const double v = *s;
  GRID_LOOP(i, n) a[i] = (XT)((double)a[i] - v);
}

template <typename T>
__global__ void k_copy_to64(const T* __restrict__ a, double* __restrict__ b, long n, int add) {
  GRID_LOOP(i, n) b[i] = add ? b[i] + (double)a[i] : (double)a[i];
}

// one colour of the smoother: MAC red-black (colour = (i+j+k)&1); FE 8 colours
template <typename T>
__global__ void k_smooth(Lv L, int kind, int colour, T* __restrict__ x, const T* __restrict__ b,
                         const T* __restrict__ c0, const T* __restrict__ c1, const T* __restrict__ c2) {
  if (kind == 0) {
    GRID_LOOP(u, L.ncell) {
      int i, j, k;
      dec3(u, L.n[0], L.n[1], i, j, k);
      if (((i + j + k) & 1) != colour) continue;
      double dg;
      const double ax = mac_apply(L, x, c0, c1, c2, i, j, k, dg);
      if (dg > 0.0) x[u] = (T)((double)x[u] + ((double)b[u] - ax) / dg);
    }
  } else {
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = (colour >> 2) & 1;
    const int mx = (L.nn[0] - cx + 1) / 2, my = (L.nn[1] - cy + 1) / 2, mz = (L.nn[2] - cz + 1) / 2;
    GRID_LOOP(t, (long)mx * my * mz) {
      int a, bb, cc;
      dec3(t, mx, my, a, bb, cc);
      const int i = 2 * a + cx, j = 2 * bb + cy, k = 2 * cc + cz;
      double dg;
      const double ax = fe_apply(L, x, c0, i, j, k, dg);
      const long u = nix(L, i, j, k);
      if (dg > 0.0) x[u] = (T)((double)x[u] + ((double)b[u] - ax) / dg);
    }
  }
}

template <typename T>
__global__ void k_resid(Lv L, int kind, const T* __restrict__ x, const T* __restrict__ b, const T* __restrict__ c0,
                        const T* __restrict__ c1, const T* __restrict__ c2, T* __restrict__ r) {
  GRID_LOOP(u, L.nunk) {
    int i, j, k;
    double dg, ax;
    if (kind == 0) {
      dec3(u, L.n[0], L.n[1], i, j, k);
      ax = mac_apply(L, x, c0, c1, c2, i, j, k, dg);
    } else {
      dec3(u, L.nn[0], L.nn[1], i, j, k);
      ax = fe_apply(L, x, c0, i, j, k, dg);
    }
    r[u] = (T)((double)b[u] - ax);
  }
}

// restriction of the residual to the coarse right-hand side (coarse x zeroed)
template <typename T>
__global__ void k_restrict(Lv F, Lv C, int kind, const T* __restrict__ rf, T* __restrict__ bc, T* __restrict__ xc) {
  GRID_LOOP(u, C.nunk) {
    int I, J, K;
    double s = 0.0;
    if (kind == 0) {
      dec3(u, C.n[0], C.n[1], I, J, K);
#pragma unroll
      for (int q = 0; q < 8; q++) s += (double)rf[cix(F, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + ((q >> 2) & 1))];
      s *= 0.125;
    } else {
      dec3(u, C.nn[0], C.nn[1], I, J, K);
      for (int oz = -1; oz <= 1; oz++)
        for (int oy = -1; oy <= 1; oy++)
          for (int ox = -1; ox <= 1; ox++) {
            int fi = 2 * I + ox, fj = 2 * J + oy, fk = 2 * K + oz;
            bool in = true;
            int ff[3] = {fi, fj, fk};
#pragma unroll
            for (int d = 0; d < 3; d++) {
              if (F.per[d]) ff[d] = (ff[d] + F.nn[d]) % F.nn[d];
              else if (ff[d] < 0 || ff[d] >= F.nn[d]) in = false;
            }
            if (!in) continue;
            const double w = (ox ? 0.5 : 1.0) * (oy ? 0.5 : 1.0) * (oz ? 0.5 : 1.0);
            s += w * (double)rf[nix(F, ff[0], ff[1], ff[2])];
          }
    }
    bc[u] = (T)s;
    xc[u] = T(0);
  }
}

// trilinear prolongation of the coarse correction, added to the fine iterate
template <typename T>
__global__ void k_prolong(Lv F, Lv C, int kind, const T* __restrict__ xc, T* __restrict__ xf) {
  GRID_LOOP(u, F.nunk) {
    int i, j, k;
    double v = 0.0;
    if (kind == 0) {
      dec3(u, F.n[0], F.n[1], i, j, k);
      const int ff[3] = {i, j, k};
      int own[3], oth[3];
      double wo[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        own[d] = ff[d] >> 1;
        int o = own[d] + ((ff[d] & 1) ? 1 : -1);
        if (o < 0 || o >= C.n[d]) {
          if (C.per[d]) {
            o = (o + C.n[d]) % C.n[d];
            wo[d] = 0.75;
          } else {
            o = own[d];
            wo[d] = 1.0;  // Neumann: the mirror value equals the boundary cell
          }
        } else {
          wo[d] = 0.75;
        }
        oth[d] = o;
      }
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int sx = q & 1, sy = (q >> 1) & 1, sz = (q >> 2) & 1;
        const double w = (sx ? 1.0 - wo[0] : wo[0]) * (sy ? 1.0 - wo[1] : wo[1]) * (sz ? 1.0 - wo[2] : wo[2]);
        if (w == 0.0) continue;
        v += w * (double)xc[cix(C, sx ? oth[0] : own[0], sy ? oth[1] : own[1], sz ? oth[2] : own[2])];
      }
    } else {
      dec3(u, F.nn[0], F.nn[1], i, j, k);
      const int ff[3] = {i, j, k};
      int lo[3], hi[3];
      double wl[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        lo[d] = ff[d] >> 1;
        if (ff[d] & 1) {
          hi[d] = lo[d] + 1;
          if (C.per[d] && hi[d] >= C.nn[d]) hi[d] -= C.nn[d];
          wl[d] = 0.5;
        } else {
          hi[d] = lo[d];
          wl[d] = 1.0;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int sx = q & 1, sy = (q >> 1) & 1, sz = (q >> 2) & 1;
        const double w = (sx ? 1.0 - wl[0] : wl[0]) * (sy ? 1.0 - wl[1] : wl[1]) * (sz ? 1.0 - wl[2] : wl[2]);
        if (w == 0.0) continue;
        v += w * (double)xc[nix(C, sx ? hi[0] : lo[0], sy ? hi[1] : lo[1], sz ? hi[2] : lo[2])];
      }
    }
    xf[u] = (T)((double)xf[u] + v);
  }
}

// coarse coefficients: MAC face beta = mean of the 4 fine faces; FE cell beta = mean of 8
template <typename T>
__global__ void k_coarsen_mac(Lv F, Lv C, int d, const T* __restrict__ bf, T* __restrict__ bc) {
  const int ex = C.n[0] + (d == 0), ey = C.n[1] + (d == 1);
  const long nf = C.ncell / C.n[d] * (C.n[d] + 1);
  GRID_LOOP(f, nf) {
    int I, J, K;
    dec3(f, ex, ey, I, J, K);
    int base[3] = {2 * I, 2 * J, 2 * K};
    double s = 0.0;
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int c3[3] = {base[0], base[1], base[2]};
      c3[e1] += q & 1;
      c3[e2] += (q >> 1) & 1;
      s += (double)bf[fix(F, d, c3[0], c3[1], c3[2])];
    }
    bc[f] = (T)(0.25 * s);
  }
}
template <typename T>
__global__ void k_coarsen_fe(Lv F, Lv C, const T* __restrict__ bf, T* __restrict__ bc) {
  GRID_LOOP(u, C.ncell) {
    int I, J, K;
    dec3(u, C.n[0], C.n[1], I, J, K);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) s += (double)bf[cix(F, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + ((q >> 2) & 1))];
    bc[u] = (T)(0.125 * s);
  }
}

// coarsest level: one block, mean-free right-hand side, many smoothing sweeps, mean-free result
template <typename T>
__global__ void k_coarse_solve(Lv L, int kind, int sweeps, T* __restrict__ x, T* __restrict__ b, const T* __restrict__ c0,
                               const T* __restrict__ c1, const T* __restrict__ c2) {
  __shared__ double sh[1024];
  __shared__ double mean;
  // mean of b
  double loc = 0.0;
  for (long u = threadIdx.x; u < L.nunk; u += blockDim.x) loc += (double)b[u];
  sh[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) mean = sh[0] / (double)L.nunk;
  __syncthreads();
  for (long u = threadIdx.x; u < L.nunk; u += blockDim.x) {
    b[u] = (T)((double)b[u] - mean);
    x[u] = T(0);
  }
  __syncthreads();
  const int ncol = kind == 0 ? 2 : 8;
  for (int it = 0; it < sweeps; it++) {
    for (int col = 0; col < ncol; col++) {
      for (long u = threadIdx.x; u < L.nunk; u += blockDim.x) {
        int i, j, k;
        double dg, ax;
        if (kind == 0) {
          dec3(u, L.n[0], L.n[1], i, j, k);
          if (((i + j + k) & 1) != col) continue;
          ax = mac_apply(L, x, c0, c1, c2, i, j, k, dg);
        } else {
          dec3(u, L.nn[0], L.nn[1], i, j, k);
          if (((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) != col) continue;
          ax = fe_apply(L, x, c0, i, j, k, dg);
        }
        if (dg > 0.0) x[u] = (T)((double)x[u] + ((double)b[u] - ax) / dg);
      }
      __syncthreads();
    }
  }
  loc = 0.0;
  for (long u = threadIdx.x; u < L.nunk; u += blockDim.x) loc += (double)x[u];
  sh[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) mean = sh[0] / (double)L.nunk;
  __syncthreads();
  for (long u = threadIdx.x; u < L.nunk; u += blockDim.x) x[u] = (T)((double)x[u] - mean);
}

}  // namespace

// ------------------------------------------------------------------------------- solver
struct MGSolver {
  int kind = 0, fp32 = 0, nlev = 0;
  Lv lv[16];
  void* x[16] = {};
  void* b[16] = {};
  void* r[16] = {};
  void* c[16][3] = {};
  double *x64 = nullptr, *b64 = nullptr, *part = nullptr, *scal = nullptr;
  double* hpin = nullptr;
  size_t esz = 8;
  mg_hook_fn hook = nullptr;
  void* hook_ctx = nullptr;
};

void mg_set_hook(MGSolver* m, mg_hook_fn fn, void* ctx) {
  m->hook = fn;
  m->hook_ctx = ctx;
}

namespace {
inline void hk(MGSolver* m, int l, int which, int begin, cudaStream_t s) {
  if (m->hook && l == 0) m->hook(m->hook_ctx, which, begin, s);
}
}  // namespace

static cudaError_t dmalloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes < 16 ? 16 : bytes);
  return e;
}

MGSolver* mg_create(const Geo& g, int kind, int prec_fp32, cudaError_t* err) {
  MGSolver* m = new MGSolver();
  m->kind = kind;
  m->fp32 = prec_fp32;
  m->esz = prec_fp32 ? 4 : 8;
  Lv L;
  for (int d = 0; d < 3; d++) {
    L.n[d] = g.n[d];
    L.per[d] = g.per[d];
  }
  L.h = g.h;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 16; l++) {
    for (int d = 0; d < 3; d++) L.nn[d] = L.per[d] ? L.n[d] : L.n[d] + 1;
    L.ncell = (long)L.n[0] * L.n[1] * L.n[2];
    L.nnode = (long)L.nn[0] * L.nn[1] * L.nn[2];
    L.nunk = kind == 0 ? L.ncell : L.nnode;
    m->lv[l] = L;
    m->nlev = l + 1;
    const size_t vb = (size_t)L.nunk * m->esz;
    if (e == cudaSuccess) e = dmalloc(&m->x[l], vb);
    if (e == cudaSuccess) e = dmalloc(&m->b[l], vb);
    if (e == cudaSuccess) e = dmalloc(&m->r[l], vb);
    if (kind == 0) {
      for (int d = 0; d < 3 && e == cudaSuccess; d++)
        e = dmalloc(&m->c[l][d], (size_t)(L.ncell / L.n[d] * (L.n[d] + 1)) * m->esz);
    } else if (e == cudaSuccess) {
      e = dmalloc(&m->c[l][0], (size_t)L.ncell * m->esz);
    }
    // coarsen while every axis halves to an even-enough size
    bool can = true;
    for (int d = 0; d < 3; d++) {
      const int h2 = L.n[d] / 2;
      if ((L.n[d] & 1) || h2 < 3 || (L.per[d] && (h2 & 1))) can = false;
    }
    if (!can || l == 15) break;
    for (int d = 0; d < 3; d++) L.n[d] /= 2;
    L.h *= 2.0;
  }
  const Lv& L0 = m->lv[0];
  if (e == cudaSuccess) e = dmalloc((void**)&m->x64, L0.nunk * sizeof(double));
  if (e == cudaSuccess) e = dmalloc((void**)&m->b64, L0.nunk * sizeof(double));
  if (e == cudaSuccess) e = dmalloc((void**)&m->part, RED_BLOCKS * sizeof(double));
  if (e == cudaSuccess) e = dmalloc((void**)&m->scal, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->hpin, 8 * sizeof(double));
  if (err) *err = e;
  return m;
}

void mg_destroy(MGSolver* m) {
  if (!m) return;
  for (int l = 0; l < m->nlev; l++) {
    cudaFree(m->x[l]);
    cudaFree(m->b[l]);
    cudaFree(m->r[l]);
    for (int d = 0; d < 3; d++) cudaFree(m->c[l][d]);
  }
  cudaFree(m->x64);
  cudaFree(m->b64);
  cudaFree(m->part);
  cudaFree(m->scal);
  cudaFreeHost(m->hpin);
  delete m;
}

double* mg_rhs(MGSolver* m) { return m->b64; }
double* mg_solution(MGSolver* m) { return m->x64; }
void* mg_coef0(MGSolver* m, int d) { return m->c[0][d]; }

namespace {

template <typename T>
void sum_into(MGSolver* m, const T* a, long n, int mode, double scale, double* out, cudaStream_t s) {
  int nb = nblocks(n);
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  k_partial<T><<<nb, TPB, 0, s>>>(a, n, mode, m->part); rmt_count_launches(1);
  k_final<<<1, 1024, 0, s>>>(m->part, nb, scale, out); rmt_count_launches(1);
}

template <typename T>
void vcycle(MGSolver* m, int l, cudaStream_t s) {
  const Lv& L = m->lv[l];
  T* x = (T*)m->x[l];
  T* b = (T*)m->b[l];
  const T* c0 = (const T*)m->c[l][0];
  const T* c1 = (const T*)m->c[l][1];
  const T* c2 = (const T*)m->c[l][2];
  const int ncol = m->kind == 0 ? 2 : 8;
  if (l == m->nlev - 1) {
    int nmax = L.n[0];
    if (L.n[1] > nmax) nmax = L.n[1];
    if (L.n[2] > nmax) nmax = L.n[2];
    const int sweeps = 2 * nmax * nmax + 20;
    k_coarse_solve<T><<<1, 1024, 0, s>>>(L, m->kind, sweeps, x, b, c0, c1, c2); rmt_count_launches(1);
    return;
  }
  const int nb = nblocks(L.nunk);
  for (int it = 0; it < 2; it++)
    for (int col = 0; col < ncol; col++) {
      hk(m, l, 0, 1, s);
      k_smooth<T><<<nb, TPB, 0, s>>>(L, m->kind, col, x, b, c0, c1, c2);
      rmt_count_launches(1);
      hk(m, l, 0, 0, s);
    }
  k_resid<T><<<nb, TPB, 0, s>>>(L, m->kind, x, b, c0, c1, c2, (T*)m->r[l]); rmt_count_launches(1);
  const Lv& C = m->lv[l + 1];
  k_restrict<T><<<nblocks(C.nunk), TPB, 0, s>>>(L, C, m->kind, (const T*)m->r[l], (T*)m->b[l + 1], (T*)m->x[l + 1]); rmt_count_launches(1);
  vcycle<T>(m, l + 1, s);
  k_prolong<T><<<nb, TPB, 0, s>>>(L, C, m->kind, (const T*)m->x[l + 1], x); rmt_count_launches(1);
  for (int it = 0; it < 2; it++)
    for (int col = ncol - 1; col >= 0; col--) {
      hk(m, l, 0, 1, s);
      k_smooth<T><<<nb, TPB, 0, s>>>(L, m->kind, col, x, b, c0, c1, c2);
      rmt_count_launches(1);
      hk(m, l, 0, 0, s);
    }
}

template <typename T>
int solve_t(MGSolver* m, double rtol, int max_cycles, int fixed_cycles, cudaStream_t s, cudaError_t* err) {
  const Lv& L0 = m->lv[0];
  const long n = L0.nunk;
  // coarse-level coefficients from level 0
  for (int l = 1; l < m->nlev; l++) {
    const Lv& F = m->lv[l - 1];
    const Lv& C = m->lv[l];
    if (m->kind == 0) {
      for (int d = 0; d < 3; d++) {
        const long nf = C.ncell / C.n[d] * (C.n[d] + 1);
        k_coarsen_mac<T><<<nblocks(nf), TPB, 0, s>>>(F, C, d, (const T*)m->c[l - 1][d], (T*)m->c[l][d]); rmt_count_launches(1);
      }
    } else {
      k_coarsen_fe<T><<<nblocks(C.ncell), TPB, 0, s>>>(F, C, (const T*)m->c[l - 1][0], (T*)m->c[l][0]); rmt_count_launches(1);
    }
  }
  // mean-free right-hand side, zero start
  sum_into<double>(m, m->b64, n, 0, 1.0 / (double)n, m->scal, s);
  k_sub_scalar<double><<<nblocks(n), TPB, 0, s>>>(m->b64, n, m->scal); rmt_count_launches(1);
  double bn2 = 0.0;
  if (fixed_cycles <= 0) {
    sum_into<double>(m, m->b64, n, 1, 1.0, m->scal + 1, s);
    cudaMemcpyAsync(m->hpin, m->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((*err = cudaStreamSynchronize(s)) != cudaSuccess) return -1;
    bn2 = m->hpin[0];
  }
  k_zero<double><<<nblocks(n), TPB, 0, s>>>(m->x64, n); rmt_count_launches(1);
  const T* c0 = (const T*)m->c[0][0];
  const T* c1 = (const T*)m->c[0][1];
  const T* c2 = (const T*)m->c[0][2];
  int nbr = nblocks(n);
  if (nbr > RED_BLOCKS) nbr = RED_BLOCKS;
  int cycles = 0;
  int ok = 1;
  if (fixed_cycles <= 0 && bn2 == 0.0) {
    *err = cudaGetLastError();
    return 0;
  }
  const int cap = fixed_cycles > 0 ? fixed_cycles : max_cycles;
  for (;;) {
    hk(m, 0, 1, 1, s);
    k_resid64<T><<<nbr, TPB, 0, s>>>(L0, m->kind, m->x64, m->b64, c0, c1, c2, (T*)m->b[0], m->part);
    rmt_count_launches(1);
    hk(m, 0, 1, 0, s);
    if (fixed_cycles <= 0) {
      k_final<<<1, 1024, 0, s>>>(m->part, nbr, 1.0, m->scal + 2); rmt_count_launches(1);
      cudaMemcpyAsync(m->hpin + 1, m->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
      if ((*err = cudaStreamSynchronize(s)) != cudaSuccess) return -1;
      const double rn2 = m->hpin[1];
      if (!(rn2 == rn2)) { ok = 0; break; }  // NaN
      if (rn2 <= rtol * rtol * bn2) break;
    }
    if (cycles >= cap) {
      if (fixed_cycles <= 0) ok = 0;
      break;
    }
    k_zero<T><<<nblocks(n), TPB, 0, s>>>((T*)m->x[0], n); rmt_count_launches(1);
    vcycle<T>(m, 0, s);
    k_copy_to64<T><<<nblocks(n), TPB, 0, s>>>((const T*)m->x[0], m->x64, n, 1); rmt_count_launches(1);
    cycles++;
    if (fixed_cycles > 0 && cycles >= fixed_cycles) break;
  }
  sum_into<double>(m, m->x64, n, 0, 1.0 / (double)n, m->scal + 3, s);
  k_sub_scalar<double><<<nblocks(n), TPB, 0, s>>>(m->x64, n, m->scal + 3); rmt_count_launches(1);
  *err = cudaGetLastError();
  return ok ? cycles : -1;
}

}  // namespace

int mg_solve(MGSolver* m, double rtol, int max_cycles, int fixed_cycles, cudaStream_t s, cudaError_t* err) {
  cudaError_t e = cudaSuccess;
  int r = m->fp32 ? solve_t<float>(m, rtol, max_cycles, fixed_cycles, s, &e)
                  : solve_t<double>(m, rtol, max_cycles, fixed_cycles, s, &e);
  if (err) *err = e;
  return r;
}
