// Parallel layer-wise extrapolation of the reference map (arXiv 2104.00095, main text
// "Extrapolation of xi(x,t)"; SI "Weighting scheme for weighted least squares-based
// extrapolation"): classification of the interior (phi_0(xi) < 0), layer marking over
// face neighbours, and one weighted least-squares fit per band cell, layer after layer.
//
// This translation unit is compiled with --fmad=false: the fits are evaluated operation
// by operation in a fixed order, so that the integer outcomes (layer labels, which fits
// are degenerate, which weights are positive) are reproducible.  FP64 storage fits in FP64;
// FP32 storage holds displacements S = xi - x0 (rmt_common.cuh) and fits them in FP32, redone
// in FP64 when ill-conditioned.
#include "rmt_kernels.h"

namespace {

constexpr int TPB = 128;
inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > (long)sm_count() * 128) b = (long)sm_count() * 128;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void decode(long c, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(c % nx);
  long r = c / nx;
  j = (int)(r % ny);
  k = (int)(r / ny);
}

// xi^0 = x at every cell; on a periodic axis the image of x nearest the body centre (FP32
// storage: the displacement from the cell's image, zero)
template <typename T>
__global__ void k_init_xi(Geo g, Body b, T* __restrict__ x) {
  GRID_LOOP(c, g.N) {
    if constexpr (disp_storage<T>()) {
      x[c] = x[g.N + c] = x[2 * g.N + c] = T(0);
      continue;
    }
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
__global__ void k_classify(Geo g, Body b, const int* __restrict__ bb, const T* __restrict__ x,
                           int8_t* __restrict__ lay) {
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
    const T x0 = x[c], x1 = x[g.N + c], x2 = x[2 * g.N + c];
    int8_t l = -1;
    if (isfinite(x0) && isfinite(x1) && isfinite(x2) && phi_stored(g, b, i, j, k, x0, x1, x2) < T(0)) l = 0;
    lay[c] = l;
  }
}

// unmarked face neighbours of layer l-1 become layer l (walls stop, periodic axes wrap);
// in place is race-free: only -1 -> l writes, and only l-1 is tested
__global__ void k_bfs(Geo g, const int* __restrict__ bb, int l, int8_t* __restrict__ lay) {
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
    if (lay[c] != -1) continue;
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

// LDL^T solve of the 4x4 normal equations, three right-hand sides, in AT; fails (degenerate)
// when a pivot is not above tolfac * trace(A)/4 (tolfac = 1e-12 in FP64)
template <typename AT>
__device__ bool solve4(AT A[4][4], AT B[4][3], AT X[4][3], AT tolfac) {
  AT L[4][4], D[4];
  for (int r = 0; r < 4; r++)
    for (int q = 0; q < 4; q++) L[r][q] = AT(0);
  const AT tr = A[0][0] + A[1][1] + A[2][2] + A[3][3];
  const AT tol = tolfac * tr / AT(4);
  for (int k = 0; k < 4; k++) {
    AT s = A[k][k];
    for (int j = 0; j < k; j++) s -= L[k][j] * L[k][j] * D[j];
    D[k] = s;
    if (!(s > tol)) return false;
    L[k][k] = AT(1);
    for (int i = k + 1; i < 4; i++) {
      AT t = A[i][k];
      for (int j = 0; j < k; j++) t -= L[i][j] * L[k][j] * D[j];
      L[i][k] = t / D[k];
    }
  }
  for (int c = 0; c < 3; c++) {
    AT y[4];
    for (int i = 0; i < 4; i++) {
      AT t = B[i][c];
      for (int j = 0; j < i; j++) t -= L[i][j] * y[j];
      y[i] = t;
    }
    for (int i = 0; i < 4; i++) y[i] /= D[i];
    for (int i = 3; i >= 0; i--) {
      AT t = y[i];
      for (int j = i + 1; j < 4; j++) t -= L[j][i] * X[j][c];
      X[i][c] = t;
    }
  }
  return true;
}

// One affine WLS fit centred at cell (i,j,k) of layer le with search radius rs, computed by a
// whole warp: the lanes split the (2 rs + 1)^3 candidate cells and the normal-equation sums are
// combined by a butterfly (every lane ends with the same totals, in a fixed order).
// mode 0: kernel 2^-(|di|+|dj|+|dk|); mode 1: times max(0, cos) against the normal n_e.
// The data are the stored values: xi_d (FP64 storage), or the displacements S_d (FP32 storage),
// which the affine model fits exactly as it fits xi (the identity is affine): the fitted values
// are then small, so the solve's error, which scales with the data, carries no O(1) positions
// into the extrapolated maps.
template <typename AT, typename T>
__device__ bool wls_fit_warp(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int i, int j,
                             int k, int le, int rs, int mode, const AT nrm[3], AT tolfac, AT sol[4][3]) {
  const int lane = threadIdx.x & 31;
  AT a[10], bsum[12];
#pragma unroll
  for (int q = 0; q < 10; q++) a[q] = AT(0);
#pragma unroll
  for (int q = 0; q < 12; q++) bsum[q] = AT(0);
  int npos = 0;
  const int w = 2 * rs + 1, nc = w * w * w;
  for (int t = lane; t < nc; t += 32) {
    const int di = t % w - rs, dj = (t / w) % w - rs, dk = t / (w * w) - rs;
    long c;
    if (!cell_at(g, i + di, j + dj, k + dk, c)) continue;
    const int ld = lay[c];
    if (ld < 0 || ld >= le) continue;
    const int sr = abs(di) + abs(dj) + abs(dk);
    AT wt = sizeof(AT) == 4 ? (AT)ldexpf(1.0f, -sr) : (AT)ldexp(1.0, -sr);
    if (mode == 1) {
      const AT len = sqrt((AT)(di * di + dj * dj + dk * dk));
      const AT cs = -((AT)di * nrm[0] + (AT)dj * nrm[1] + (AT)dk * nrm[2]) / len;
      wt = cs * wt;
      if (!(wt > AT(0))) continue;
    }
    const AT v[4] = {AT(1), (AT)di, (AT)dj, (AT)dk};
    const AT xv[3] = {(AT)x[c], (AT)x[g.N + c], (AT)x[2 * g.N + c]};
    int q = 0;
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int cc = r; cc < 4; cc++) a[q++] += wt * v[r] * v[cc];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int d = 0; d < 3; d++) bsum[3 * r + d] += wt * v[r] * xv[d];
    npos++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 10; q++) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
#pragma unroll
    for (int q = 0; q < 12; q++) bsum[q] += __shfl_xor_sync(0xffffffffu, bsum[q], o);
    npos += __shfl_xor_sync(0xffffffffu, npos, o);
  }
  if (npos < 4) return false;
  AT A[4][4], B[4][3];
  int q = 0;
  for (int r = 0; r < 4; r++)
    for (int cc = r; cc < 4; cc++) {
      A[r][cc] = a[q];
      A[cc][r] = a[q];
      q++;
    }
  for (int r = 0; r < 4; r++)
    for (int d = 0; d < 3; d++) B[r][d] = bsum[3 * r + d];
  return solve4<AT>(A, B, sol, tolfac);
}

// Extrapolates one cell (whole warp) with fits accumulated in AT: kernel-only fit, then (layers
// 1 and 2) the fit weighted by the normal n_e = normalised (grad xi)^T grad_X phi_0(xi_e) of that
// first fit; the search radius grows up to 4 while the system stays degenerate.  Returns 1 on
// success, 0 when degenerate, -1 when an FP32 attempt was too ill-conditioned to trust.
template <typename AT, typename T>
__device__ int wls_cell_try(const Geo& g, const Body& b, const T* __restrict__ x, const int8_t* __restrict__ lay,
                            int i, int j, int k, int le, double out[3]) {
  // FP64: the degeneracy threshold; FP32: also the point below which the fit is redone in FP64
  const AT tolfac = sizeof(AT) == 8 ? AT(1e-12) : AT(1e-4);
  // FP32 storage fits displacements: the identity's slope per cell offset is added back to the
  // fitted gradient, and the cell's x0 - c to the fitted value, where the normal needs xi
  const AT hid = disp_storage<T>() ? (sizeof(AT) == 4 ? (AT)g.f.h : (AT)g.h) : AT(0);
  for (int rs = 2; rs <= 4; rs++) {
    AT s1[4][3];
    if (!wls_fit_warp<AT>(g, x, lay, i, j, k, le, rs, 0, (const AT*)nullptr, tolfac, s1)) {
      if (sizeof(AT) == 4) return -1;
      continue;
    }
    if (le <= 2) {
      AT gX[3], v[3];
      if constexpr (disp_storage<T>()) {
        const AT r0[3] = {cell_rel<AT>(g, b, 0, i) + s1[0][0], cell_rel<AT>(g, b, 1, j) + s1[0][1],
                          cell_rel<AT>(g, b, 2, k) + s1[0][2]};
        phi0_dir_r<AT>(b, r0, gX);
      } else {
        const AT c0[3] = {s1[0][0], s1[0][1], s1[0][2]};
        phi0_dir<AT>(b, c0, gX);
      }
      for (int q = 0; q < 3; q++)
        v[q] = (s1[1 + q][0] + (q == 0 ? hid : AT(0))) * gX[0] + (s1[1 + q][1] + (q == 1 ? hid : AT(0))) * gX[1] +
               (s1[1 + q][2] + (q == 2 ? hid : AT(0))) * gX[2];
      const AT nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (!(nv > AT(0))) {
        if (sizeof(AT) == 4) return -1;
        continue;
      }
      const AT nrm[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
      AT s2[4][3];
      if (!wls_fit_warp<AT>(g, x, lay, i, j, k, le, rs, 1, nrm, tolfac, s2)) {
        if (sizeof(AT) == 4) return -1;
        continue;
      }
      for (int d = 0; d < 3; d++) out[d] = (double)s2[0][d];
      return 1;
    }
    for (int d = 0; d < 3; d++) out[d] = (double)s1[0][d];
    return 1;
  }
  return 0;
}

// FP64 storage: FP64 fits.  FP32 storage: FP32 fits, redone in FP64 when ill-conditioned.
template <typename T>
__device__ bool wls_cell_warp(const Geo& g, const Body& b, const T* __restrict__ x, const int8_t* __restrict__ lay,
                              int i, int j, int k, int le, double out[3]) {
  if (sizeof(T) == 4) {
    const int r = wls_cell_try<float>(g, b, x, lay, i, j, k, le, out);
    if (r >= 0) return r == 1;
  }
  return wls_cell_try<double>(g, b, x, lay, i, j, k, le, out) == 1;
}

// compacted list of the band cells (layers 1..L) of a body's window
__global__ void k_band_list(Geo g, const int* __restrict__ bb, const int8_t* __restrict__ lay, int* __restrict__ list,
                            int* __restrict__ count) {
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
    const int l = lay[c];
    if (l >= 1) list[atomicAdd(count, 1)] = (int)c;
  }
}

// one warp per listed cell of layer l
template <typename T>
__global__ void k_wls(Geo g, Body b, int l, T* __restrict__ x, int8_t* __restrict__ lay, const int* __restrict__ list,
                      const int* __restrict__ count, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int n = *count;
  for (int e = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < n; e += (gridDim.x * blockDim.x) >> 5) {
    const long c = list[e];
    if (lay[c] != l) continue;
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((long)g.n[0] * g.n[1]));
    double out[3];
    const bool ok = wls_cell_warp(g, b, x, lay, i, j, k, l, out);
    __syncwarp();
    if (lane == 0) {
      if (ok) {
        x[c] = (T)out[0];
        x[g.N + c] = (T)out[1];
        x[2 * g.N + c] = (T)out[2];
      } else {
        lay[c] = -1;
        atomicAdd(err, 1);
      }
    }
  }
}

// phi of the band cells, NaN elsewhere, the band's box; FP32 storage: band cells near the seam of
// the body's image window are counted in *seam
template <typename T>
__global__ void k_finalize(Geo g, Body b, const int* __restrict__ bb, T* __restrict__ x, T* __restrict__ phi,
                           const int8_t* __restrict__ lay, int* __restrict__ bb_out, int* __restrict__ seam) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
    if (lay[c] >= 0) {
#pragma unroll
      for (int d = 0; d < 3; d++) {
        atomicMin(&bb_out[d], u[d]);
        atomicMax(&bb_out[3 + d], u[d]);
      }
    }
    if (lay[c] >= 0) {
      phi[c] = phi_stored(g, b, i, j, k, x[c], x[g.N + c], x[2 * g.N + c]);
      if (disp_storage<T>() && near_seam(g, b, i, j, k)) atomicAdd(seam, 1);
    } else {
      x[c] = x[g.N + c] = x[2 * g.N + c] = nanv;
      phi[c] = nanv;
    }
  }
}

// corrector xi^{n+1/2} = (xi^n + xi^{n+1})/2 where both exist
template <typename T>
__global__ void k_corr(Geo g, const int* __restrict__ bb, const T* __restrict__ x, const int8_t* __restrict__ lay,
                       const T* __restrict__ xn, const int8_t* __restrict__ layn, T* __restrict__ xh) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
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
                           const T* __restrict__ xn, T* __restrict__ xh, const int* __restrict__ list,
                           const int* __restrict__ count, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int n = *count;
  for (int e = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < n; e += (gridDim.x * blockDim.x) >> 5) {
    const long c = list[e];
    if (layn[c] != l || lay[c] >= 0) continue;
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((long)g.n[0] * g.n[1]));
    double out[3];
    const bool ok = wls_cell_warp(g, b, xh, layn, i, j, k, l, out);
    __syncwarp();
    if (lane == 0) {
      if (ok) {
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
}

template <typename T>
__global__ void k_phi_half(Geo g, Body b, const int* __restrict__ bb, const T* __restrict__ xh,
                           const int8_t* __restrict__ layn, T* __restrict__ phih) {
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int u[3], i, j, k;
    long c;
    win_cell(g, w, t, u, i, j, k, c);
    phih[c] = layn[c] >= 0 ? phi_stored(g, b, i, j, k, xh[c], xh[g.N + c], xh[2 * g.N + c]) : nanv;
  }
}

// empty bounding box (min above max)
__global__ void k_bb_reset(int* bb) {
  if (threadIdx.x == 0) {
    bb[0] = bb[1] = bb[2] = 0x7fffffff;
    bb[3] = bb[4] = bb[5] = -0x7fffffff;
  }
}
// shift the box of a periodic axis so that its minimum lies in [0, n)
__global__ void k_bb_normalise(Geo g, int* bb) {
  if (threadIdx.x != 0) return;
  for (int d = 0; d < 3; d++) {
    if (!g.per[d] || bb[d] > bb[3 + d]) continue;
    int q = bb[d] / g.n[d];
    if (bb[d] < 0 && bb[d] % g.n[d]) q -= 1;
    bb[d] -= q * g.n[d];
    bb[3 + d] -= q * g.n[d];
  }
}

}  // namespace

template <typename T>
void launch_init_xi(const Geo& g, const Body& b, T* x, cudaStream_t s) {
  k_init_xi<T><<<nblocks(g.N), TPB, 0, s>>>(g, b, x); rmt_count_launches(1);
}

template <typename T>
cudaError_t launch_extrapolate(const Geo& g, const Body& b, const int* bb_in, int* bb_out, int blocks, int* list,
                               int* count, int wls_blocks, T* x, T* phi, int8_t* lay, int* err, cudaStream_t s) {
  k_classify<T><<<blocks, TPB, 0, s>>>(g, b, bb_in, x, lay);
  rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) {
    k_bfs<<<blocks, TPB, 0, s>>>(g, bb_in, l, lay);
    rmt_count_launches(1);
  }
  const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_band_list<<<blocks, TPB, 0, s>>>(g, bb_in, lay, list, count);
  rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) {
    k_wls<T><<<wls_blocks, TPB, 0, s>>>(g, b, l, x, lay, list, count, err);
    rmt_count_launches(1);
  }
  k_bb_reset<<<1, 32, 0, s>>>(bb_out);
  rmt_count_launches(1);
  k_finalize<T><<<blocks, TPB, 0, s>>>(g, b, bb_in, x, phi, lay, bb_out, err + 1);
  rmt_count_launches(1);
  k_bb_normalise<<<1, 32, 0, s>>>(g, bb_out);
  rmt_count_launches(1);
  return cudaSuccess;
}

template <typename T>
void launch_corrector(const Geo& g, const Body& b, const int* bb_in, int blocks, const int* list, const int* count,
                      int wls_blocks, const T* x, const int8_t* lay, const T* xn, const int8_t* layn, T* xh, T* phih,
                      int* err, cudaStream_t s) {
  k_corr<T><<<blocks, TPB, 0, s>>>(g, bb_in, x, lay, xn, layn, xh);
  rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) {
    k_wls_half<T><<<wls_blocks, TPB, 0, s>>>(g, b, l, lay, layn, xn, xh, list, count, err);
    rmt_count_launches(1);
  }
  k_phi_half<T><<<blocks, TPB, 0, s>>>(g, b, bb_in, xh, layn, phih);
  rmt_count_launches(1);
}

#define INST(T)                                                                                                \
  template void launch_init_xi<T>(const Geo&, const Body&, T*, cudaStream_t);                                   \
  template cudaError_t launch_extrapolate<T>(const Geo&, const Body&, const int*, int*, int, int*, int*, int, T*, \
                                             T*, int8_t*, int*, cudaStream_t);                                  \
  template void launch_corrector<T>(const Geo&, const Body&, const int*, int, const int*, const int*, int,        \
                                    const T*, const int8_t*, const T*, const int8_t*, T*, T*, int*, cudaStream_t);
INST(float)
INST(double)
