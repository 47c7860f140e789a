// Parallel layer-wise extrapolation of the reference map (arXiv 2104.00095, main text
// "Extrapolation of xi(x,t)"; SI "Weighting scheme for weighted least squares-based
// extrapolation"): classification of the interior (phi_0(xi) < 0), layer marking over
// face neighbours, and one weighted least-squares fit per band cell, layer after layer.
//
// This translation unit is compiled with --fmad=false: the fits are evaluated operation
// by operation in a fixed order, so that the integer outcomes (layer labels, which fits
// are degenerate, which weights are positive) are reproducible.  All fits run in FP64.
#include "rmt_kernels.h"

namespace {

constexpr int TPB = 128;
inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > 152L * 128) b = 152L * 128;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void decode(long c, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(c % nx);
  long r = c / nx;
  j = (int)(r % ny);
  k = (int)(r / ny);
}

// xi^0 = x at every cell; on a periodic axis the image of x nearest the body centre
template <typename T>
__global__ void k_init_xi(Geo g, Body b, T* __restrict__ x) {
  GRID_LOOP(c, g.N) {
    int ii[3];
    decode(c, g.n[0], g.n[1], ii[0], ii[1], ii[2]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      double v = g.lo[d] + (ii[d] + 0.5) * g.h;
      if (g.per[d]) v += g.len[d] * floor((b.c[d] - v) / g.len[d] + 0.5);
      x[d * g.N + c] = (T)v;
    }
  }
}

// layer 0 = candidates (finite xi) with phi_0(xi) < 0; everything else unmarked
template <typename T>
__global__ void k_classify(Geo g, Body b, const T* __restrict__ x, int8_t* __restrict__ lay) {
  GRID_LOOP(c, g.N) {
    const T x0 = x[c], x1 = x[g.N + c], x2 = x[2 * g.N + c];
    int8_t l = -1;
    if (isfinite(x0) && isfinite(x1) && isfinite(x2) && phi0(b, x0, x1, x2) < T(0)) l = 0;
    lay[c] = l;
  }
}

// unmarked face neighbours of layer l-1 become layer l (walls stop, periodic axes wrap);
// in place is race-free: only -1 -> l writes, and only l-1 is tested
__global__ void k_bfs(Geo g, int l, int8_t* __restrict__ lay) {
  GRID_LOOP(c, g.N) {
    if (lay[c] != -1) continue;
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int f = 0; f < 6; f++) {
      long nb;
      if (!cell_at(g, i + off[f][0], j + off[f][1], k + off[f][2], nb)) continue;
      if (lay[nb] == l - 1) {
        lay[c] = (int8_t)l;
        break;
      }
    }
  }
}

// LDL^T solve of the 4x4 normal equations, three right-hand sides; degenerate when a
// pivot is not above 1e-12 trace(A)/4
__device__ bool solve4(double A[4][4], double B[4][3], double X[4][3]) {
  double L[4][4], D[4];
  for (int r = 0; r < 4; r++)
    for (int q = 0; q < 4; q++) L[r][q] = 0.0;
  const double tr = A[0][0] + A[1][1] + A[2][2] + A[3][3];
  const double tol = 1e-12 * tr / 4.0;
  for (int k = 0; k < 4; k++) {
    double s = A[k][k];
    for (int j = 0; j < k; j++) s -= L[k][j] * L[k][j] * D[j];
    D[k] = s;
    if (!(s > tol)) return false;
    L[k][k] = 1.0;
    for (int i = k + 1; i < 4; i++) {
      double t = A[i][k];
      for (int j = 0; j < k; j++) t -= L[i][j] * L[k][j] * D[j];
      L[i][k] = t / D[k];
    }
  }
  for (int c = 0; c < 3; c++) {
    double y[4];
    for (int i = 0; i < 4; i++) {
      double t = B[i][c];
      for (int j = 0; j < i; j++) t -= L[i][j] * y[j];
      y[i] = t;
    }
    for (int i = 0; i < 4; i++) y[i] /= D[i];
    for (int i = 3; i >= 0; i--) {
      double t = y[i];
      for (int j = i + 1; j < 4; j++) t -= L[j][i] * X[j][c];
      X[i][c] = t;
    }
  }
  return true;
}

// One affine WLS fit centred at cell (i,j,k) of layer le with search radius rs.
// mode 0: kernel 2^-(|di|+|dj|+|dk|); mode 1: times max(0, cos) against the normal n_e.
template <typename T>
__device__ bool wls_fit(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int i, int j, int k,
                        int le, int rs, int mode, const double nrm[3], double sol[4][3]) {
  double A[4][4], B[4][3];
  for (int r = 0; r < 4; r++) {
    for (int q = 0; q < 4; q++) A[r][q] = 0.0;
    for (int a = 0; a < 3; a++) B[r][a] = 0.0;
  }
  int npos = 0;
  for (int dk = -rs; dk <= rs; dk++)
    for (int dj = -rs; dj <= rs; dj++)
      for (int di = -rs; di <= rs; di++) {
        long c;
        if (!cell_at(g, i + di, j + dj, k + dk, c)) continue;
        const int ld = lay[c];
        if (ld < 0 || ld >= le) continue;
        const int s = abs(di) + abs(dj) + abs(dk);
        double w = ldexp(1.0, -s);
        if (mode == 1) {
          const double len = sqrt((double)(di * di + dj * dj + dk * dk));
          const double cs = -((double)di * nrm[0] + (double)dj * nrm[1] + (double)dk * nrm[2]) / len;
          w = cs * w;
          if (!(w > 0.0)) continue;
        }
        const double v[4] = {1.0, (double)di, (double)dj, (double)dk};
        const double xv[3] = {(double)x[c], (double)x[g.N + c], (double)x[2 * g.N + c]};
        for (int r = 0; r < 4; r++) {
          for (int q = 0; q < 4; q++) A[r][q] += w * v[r] * v[q];
          for (int a = 0; a < 3; a++) B[r][a] += w * v[r] * xv[a];
        }
        npos++;
      }
  if (npos < 4) return false;
  return solve4(A, B, sol);
}

// Extrapolates one cell: kernel-only fit, then (layers 1 and 2) the fit weighted by the
// normal n_e = normalised (grad xi)^T grad_X phi_0(xi_e) of that first fit; the search
// radius grows up to 4 while the system stays degenerate.
template <typename T>
__device__ bool wls_cell(const Geo& g, const Body& b, const T* __restrict__ x, const int8_t* __restrict__ lay, int i,
                         int j, int k, int le, double out[3]) {
  for (int rs = 2; rs <= 4; rs++) {
    double s1[4][3];
    if (!wls_fit(g, x, lay, i, j, k, le, rs, 0, nullptr, s1)) continue;
    if (le <= 2) {
      const double c0[3] = {s1[0][0], s1[0][1], s1[0][2]};
      double gX[3], v[3];
      phi0_dir<double>(b, c0, gX);
      for (int q = 0; q < 3; q++) v[q] = s1[1 + q][0] * gX[0] + s1[1 + q][1] * gX[1] + s1[1 + q][2] * gX[2];
      const double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (!(nv > 0.0)) continue;
      const double nrm[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
      double s2[4][3];
      if (!wls_fit(g, x, lay, i, j, k, le, rs, 1, nrm, s2)) continue;
      out[0] = s2[0][0]; out[1] = s2[0][1]; out[2] = s2[0][2];
      return true;
    }
    out[0] = s1[0][0]; out[1] = s1[0][1]; out[2] = s1[0][2];
    return true;
  }
  return false;
}

template <typename T>
__global__ void k_wls(Geo g, Body b, int l, T* __restrict__ x, int8_t* __restrict__ lay, int* __restrict__ err) {
  GRID_LOOP(c, g.N) {
    if (lay[c] != l) continue;
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    double out[3];
    if (wls_cell(g, b, x, lay, i, j, k, l, out)) {
      x[c] = (T)out[0];
      x[g.N + c] = (T)out[1];
      x[2 * g.N + c] = (T)out[2];
    } else {
      lay[c] = -1;
      atomicAdd(err, 1);
    }
  }
}

template <typename T>
__global__ void k_finalize(Geo g, Body b, T* __restrict__ x, T* __restrict__ phi, const int8_t* __restrict__ lay) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  GRID_LOOP(c, g.N) {
    if (lay[c] >= 0) {
      phi[c] = phi0(b, x[c], x[g.N + c], x[2 * g.N + c]);
    } else {
      x[c] = x[g.N + c] = x[2 * g.N + c] = nanv;
      phi[c] = nanv;
    }
  }
}

// corrector xi^{n+1/2} = (xi^n + xi^{n+1})/2 where both exist
template <typename T>
__global__ void k_corr(Geo g, const T* __restrict__ x, const int8_t* __restrict__ lay, const T* __restrict__ xn,
                       const int8_t* __restrict__ layn, T* __restrict__ xh) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  GRID_LOOP(c, g.N) {
    if (layn[c] < 0 || lay[c] < 0) {
      xh[c] = xh[g.N + c] = xh[2 * g.N + c] = nanv;
      continue;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) xh[a * g.N + c] = T(0.5) * (x[a * g.N + c] + xn[a * g.N + c]);
  }
}

// cells new to the band: xi^{n+1/2} by the same WLS from the corrected lower layers
template <typename T>
__global__ void k_wls_half(Geo g, Body b, int l, const int8_t* __restrict__ lay, const int8_t* __restrict__ layn,
                           const T* __restrict__ xn, T* __restrict__ xh, int* __restrict__ err) {
  GRID_LOOP(c, g.N) {
    if (layn[c] != l || lay[c] >= 0) continue;
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    double out[3];
    if (wls_cell(g, b, xh, layn, i, j, k, l, out)) {
      xh[c] = (T)out[0];
      xh[g.N + c] = (T)out[1];
      xh[2 * g.N + c] = (T)out[2];
    } else {
      xh[c] = xn[c];
      xh[g.N + c] = xn[g.N + c];
      xh[2 * g.N + c] = xn[2 * g.N + c];
      atomicAdd(err, 1);
    }
  }
}

template <typename T>
__global__ void k_phi_half(Geo g, Body b, const T* __restrict__ xh, const int8_t* __restrict__ layn, T* __restrict__ phih) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  GRID_LOOP(c, g.N) {
    phih[c] = layn[c] >= 0 ? phi0(b, xh[c], xh[g.N + c], xh[2 * g.N + c]) : nanv;
  }
}

}  // namespace

template <typename T>
void launch_init_xi(const Geo& g, const Body& b, T* x, cudaStream_t s) {
  k_init_xi<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, x); rmt_count_launches(1);
}

template <typename T>
void launch_extrapolate(const Geo& g, const Body* /*bdev*/, const Body& b, T* x, T* phi, int8_t* lay, int* err,
                        cudaStream_t s) {
  k_classify<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, x, lay); rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) { k_bfs<<<nblocks(g.N), TPB, 0, s>>>(g, l, lay); rmt_count_launches(1); }
  for (int l = 1; l <= g.layers; l++) { k_wls<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, l, x, lay, err); rmt_count_launches(1); }
  k_finalize<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, x, phi, lay); rmt_count_launches(1);
}

template <typename T>
void launch_corrector(const Geo& g, const Body* /*bdev*/, const Body& b, const T* x, const int8_t* lay, const T* xn,
                      const int8_t* layn, T* xh, T* phih, int* err, cudaStream_t s) {
  k_corr<T><<<nblocks(g.N), TPB, 0, s>>>(g, x, lay, xn, layn, xh); rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) { k_wls_half<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, l, lay, layn, xn, xh, err); rmt_count_launches(1); }
  k_phi_half<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, xh, layn, phih); rmt_count_launches(1);
}

#define INST(T)                                                                                               \
  template void launch_init_xi<T>(const Geo&, const Body&, T*, cudaStream_t);                                  \
  template void launch_extrapolate<T>(const Geo&, const Body*, const Body&, T*, T*, int8_t*, int*, cudaStream_t); \
  template void launch_corrector<T>(const Geo&, const Body*, const Body&, const T*, const int8_t*, const T*,    \
                                    const int8_t*, T*, T*, int*, cudaStream_t);
INST(float)
INST(double)
