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
#include <type_traits>

#include "rmt_kernels.h"

namespace {

constexpr int TPB = 128;
inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > (long)sm_count() * 128) b = (long)sm_count() * 128;
  return (int)(b < 1 ? 1 : b);
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

// The band list is sorted by layer: cnt[l] (l = 1..L) counts the cells of layer l, and they sit
// at list[base_l ...], base_l = cnt[1] + ... + cnt[l-1] (the earlier passes have finished).
__device__ __forceinline__ int layer_base(const int* __restrict__ cnt, int l) {
  int b = 0;
  for (int q = 1; q < l; q++) b += cnt[q];
  return b;
}

// unmarked face neighbours of layer l-1 become layer l (walls stop, periodic axes wrap) and are
// appended to layer l's segment of the band list; in place is race-free: only -1 -> l writes,
// and only l-1 is tested
__global__ void k_bfs(Geo g, const int* __restrict__ bb, int l, int8_t* __restrict__ lay, int* __restrict__ list,
                      int* __restrict__ cnt) {
  const Win w = make_win(g, bb, 2);
  const int base = layer_base(cnt, l);
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
        list[base + atomicAdd(&cnt[l], 1)] = (int)c;
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

// The candidate cells of the radius-2 search box around one cell, loaded once per cell for
// every fit that uses that box (the kernel-only fit, the normal-weighted fit and an FP64 redo):
// lane L holds the candidates t = L + 32 q (q < 4) of the 5^3 box, a bit per slot that says
// whether the candidate is a cell of a lower layer, and its stored values.  The layer bytes of
// the four slots are read first and the values of the usable ones after them, so a cell costs
// two dependent memory round trips instead of two per slot and fit.
constexpr int RS0 = 2, NC0 = (2 * RS0 + 1) * (2 * RS0 + 1) * (2 * RS0 + 1), NQ0 = (NC0 + 31) / 32;
template <typename T>
struct Cand {
  unsigned ok;
  T v[NQ0][3];
};

template <typename T>
__device__ __forceinline__ void load_cand(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay,
                                          int i, int j, int k, int le, Cand<T>& cd) {
  const int lane = threadIdx.x & 31;
  long cc[NQ0];
  int ld[NQ0];
#pragma unroll
  for (int q = 0; q < NQ0; q++) {
    const int t = lane + 32 * q, w = 2 * RS0 + 1;
    ld[q] = -1;
    cc[q] = 0;
    long c;
    if (t < NC0 && cell_at(g, i + t % w - RS0, j + (t / w) % w - RS0, k + t / (w * w) - RS0, c)) {
      cc[q] = c;
      ld[q] = lay[c];
    }
  }
  cd.ok = 0u;
#pragma unroll
  for (int q = 0; q < NQ0; q++) {
    cd.v[q][0] = cd.v[q][1] = cd.v[q][2] = T(0);
    if (ld[q] >= 0 && ld[q] < le) {
      cd.ok |= 1u << q;
      cd.v[q][0] = x[cc[q]];
      cd.v[q][1] = x[g.N + cc[q]];
      cd.v[q][2] = x[2 * g.N + cc[q]];
    }
  }
}

// One affine WLS fit centred at cell (i,j,k) of layer le with search radius rs, computed by a
// whole warp: the lanes split the (2 rs + 1)^3 candidate cells and the normal-equation sums are
// combined by a butterfly (every lane ends with the same totals, in a fixed order).
// mode 0: kernel 2^-(|di|+|dj|+|dk|); mode 1: times max(0, cos) against the normal n_e.
// The data are the stored values: xi_d (FP64 storage), or the displacements S_d (FP32 storage),
// which the affine model fits exactly as it fits xi (the identity is affine): the fitted values
// are then small, so the solve's error, which scales with the data, carries no O(1) positions
// into the extrapolated maps.  With cd (rs = 2 only) the candidates come from the registers that
// load_cand filled, in the same order, so the sums are the same to the last bit.
template <typename AT, typename T>
__device__ bool wls_fit_warp(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int i, int j,
                             int k, int le, int rs, int mode, const AT nrm[3], AT tolfac, AT sol[4][3],
                             const Cand<T>* cd = nullptr) {
  const int lane = threadIdx.x & 31;
  AT a[10], bsum[12];
#pragma unroll
  for (int q = 0; q < 10; q++) a[q] = AT(0);
#pragma unroll
  for (int q = 0; q < 12; q++) bsum[q] = AT(0);
  int npos = 0;
  const int w = 2 * rs + 1, nc = w * w * w;
  // one candidate's contribution; false when its weight is not positive
  auto add = [&](int di, int dj, int dk, T x0, T x1, T x2) {
    const int sr = abs(di) + abs(dj) + abs(dk);
    AT wt = sizeof(AT) == 4 ? (AT)ldexpf(1.0f, -sr) : (AT)ldexp(1.0, -sr);
    if (mode == 1) {
      const AT len = sqrt((AT)(di * di + dj * dj + dk * dk));
      const AT cs = -((AT)di * nrm[0] + (AT)dj * nrm[1] + (AT)dk * nrm[2]) / len;
      wt = cs * wt;
      if (!(wt > AT(0))) return;
    }
    const AT v[4] = {AT(1), (AT)di, (AT)dj, (AT)dk};
    const AT xv[3] = {(AT)x0, (AT)x1, (AT)x2};
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
  };
  if (cd) {
#pragma unroll
    for (int q = 0; q < NQ0; q++) {
      if (!(cd->ok >> q & 1u)) continue;
      const int t = lane + 32 * q;
      add(t % w - rs, (t / w) % w - rs, t / (w * w) - rs, cd->v[q][0], cd->v[q][1], cd->v[q][2]);
    }
  } else {
    for (int t = lane; t < nc; t += 32) {
      const int di = t % w - rs, dj = (t / w) % w - rs, dk = t / (w * w) - rs;
      long c;
      if (!cell_at(g, i + di, j + dj, k + dk, c)) continue;
      const int ld = lay[c];
      if (ld < 0 || ld >= le) continue;
      add(di, dj, dk, x[c], x[g.N + c], x[2 * g.N + c]);
    }
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
// success, 0 when degenerate, -1 when an FP32 attempt was too ill-conditioned to trust.  cd: the
// preloaded candidates of the radius-2 box.
template <typename AT, typename T>
__device__ int wls_cell_try(const Geo& g, const Body& b, const T* __restrict__ x, const int8_t* __restrict__ lay,
                            int i, int j, int k, int le, const Cand<T>& cd, double out[3]) {
  // FP64: the degeneracy threshold; FP32: also the point below which the fit is redone in FP64
  const AT tolfac = sizeof(AT) == 8 ? AT(1e-12) : AT(1e-4);
  // FP32 storage fits displacements: the identity's slope per cell offset is added back to the
  // fitted gradient, and the cell's x0 - c to the fitted value, where the normal needs xi
  const AT hid = disp_storage<T>() ? (sizeof(AT) == 4 ? (AT)g.f.h : (AT)g.h) : AT(0);
  for (int rs = RS0; rs <= 4; rs++) {
    const Cand<T>* cp = rs == RS0 ? &cd : nullptr;
    AT s1[4][3];
    if (!wls_fit_warp<AT>(g, x, lay, i, j, k, le, rs, 0, (const AT*)nullptr, tolfac, s1, cp)) {
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
      if (!wls_fit_warp<AT>(g, x, lay, i, j, k, le, rs, 1, nrm, tolfac, s2, cp)) {
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

// One cell's fits in the accumulation type of the storage: FP64 storage fits in FP64 (1:
// extrapolated, 0: degenerate); FP32 storage fits in FP32 and returns -1 when the system was too
// ill-conditioned to trust, for the FP64 redo kernel (a separate kernel, so that the FP32 one
// keeps the register budget of FP32 fits).  FP64: the redo itself.
template <typename AT, typename T>
__device__ int wls_cell_warp(const Geo& g, const Body& b, const T* __restrict__ x, const int8_t* __restrict__ lay,
                             int i, int j, int k, int le, double out[3]) {
  Cand<T> cd;
  load_cand(g, x, lay, i, j, k, le, cd);
  return wls_cell_try<AT>(g, b, x, lay, i, j, k, le, cd, out);
}

// FP32 fits run at six blocks per SM (80 registers a thread, 8 bytes spilled); FP64 fits take what
// they need
#define WLS_MINB(T, REDO) ((sizeof(T) == 4 && !(REDO)) ? 6 : 1)

// one warp per cell of layer l (its segment of the band list).  REDO: the FP64 pass over the
// cells whose FP32 fits were too ill-conditioned (redo[0 .. cnt[0]), filtered by layer);
// otherwise the storage type's pass, which lists such cells in redo (FP32 storage).
template <typename T, bool REDO>
__global__ void __launch_bounds__(TPB, WLS_MINB(T, REDO)) k_wls(Geo g, Body b, int l, T* __restrict__ x, int8_t* __restrict__ lay, const int* __restrict__ list,
                      int* __restrict__ cnt, int* __restrict__ redo, int* __restrict__ err) {
  using AT = typename std::conditional<REDO || sizeof(T) == 8, double, float>::type;
  const int lane = threadIdx.x & 31;
  const int base = REDO ? 0 : layer_base(cnt, l), n = REDO ? cnt[0] : cnt[l];
  const int* src = REDO ? redo : list + base;
  for (int e = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < n; e += (gridDim.x * blockDim.x) >> 5) {
    const long c = src[e];
    if (REDO && lay[c] != l) continue;  // listed by an earlier layer's pass
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    double out[3];
    const int r = wls_cell_warp<AT>(g, b, x, lay, i, j, k, l, out);
    __syncwarp();
    if (lane == 0) {
      if (r == 1) {
        x[c] = (T)out[0];
        x[g.N + c] = (T)out[1];
        x[2 * g.N + c] = (T)out[2];
      } else if (r == 0) {
        lay[c] = -1;
        atomicAdd(err, 1);
      } else {
        redo[atomicAdd(&cnt[0], 1)] = (int)c;
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

// cells new to the band: xi^{n+1/2} by the same WLS from the corrected lower layers (layer l's
// segment of the new band's list; REDO as for k_wls, with its own redo count cnt[9])
template <typename T, bool REDO>
__global__ void __launch_bounds__(TPB, WLS_MINB(T, REDO)) k_wls_half(Geo g, Body b, int l, const int8_t* __restrict__ lay, const int8_t* __restrict__ layn,
                           const T* __restrict__ xn, T* __restrict__ xh, const int* __restrict__ list,
                           int* __restrict__ cnt, int* __restrict__ redo, int* __restrict__ err) {
  using AT = typename std::conditional<REDO || sizeof(T) == 8, double, float>::type;
  const int lane = threadIdx.x & 31;
  const int base = REDO ? 0 : layer_base(cnt, l), n = REDO ? cnt[9] : cnt[l];
  const int* src = REDO ? redo : list + base;
  for (int e = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < n; e += (gridDim.x * blockDim.x) >> 5) {
    const long c = src[e];
    if (layn[c] != l || lay[c] >= 0) continue;
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    double out[3];
    const int r = wls_cell_warp<AT>(g, b, xh, layn, i, j, k, l, out);
    __syncwarp();
    if (lane == 0) {
      if (r < 0) {
        redo[atomicAdd(&cnt[9], 1)] = (int)c;
      } else if (r == 1) {
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

// cnt: BAND_COUNTERS ints (see rmt_kernels.h); redo: FP32 storage, a list of the grid's size
template <typename T>
cudaError_t launch_extrapolate(const Geo& g, const Body& b, const int* bb_in, int* bb_out, int blocks, int* list,
                               int* cnt, int* redo, int wls_blocks, T* x, T* phi, int8_t* lay, int* err,
                               cudaStream_t s) {
  const cudaError_t e = cudaMemsetAsync(cnt, 0, BAND_COUNTERS * sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_classify<T><<<blocks, TPB, 0, s>>>(g, b, bb_in, x, lay);
  rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) {
    k_bfs<<<blocks, TPB, 0, s>>>(g, bb_in, l, lay, list, cnt);
    rmt_count_launches(1);
  }
  for (int l = 1; l <= g.layers; l++) {
    k_wls<T, false><<<wls_blocks, TPB, 0, s>>>(g, b, l, x, lay, list, cnt, redo, err);
    rmt_count_launches(1);
    if (sizeof(T) == 4) {
      k_wls<T, true><<<sm_count(), TPB, 0, s>>>(g, b, l, x, lay, list, cnt, redo, err);
      rmt_count_launches(1);
    }
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
void launch_corrector(const Geo& g, const Body& b, const int* bb_in, int blocks, const int* list, int* cnt, int* redo,
                      int wls_blocks, const T* x, const int8_t* lay, const T* xn, const int8_t* layn, T* xh, T* phih,
                      int* err, cudaStream_t s) {
  k_corr<T><<<blocks, TPB, 0, s>>>(g, bb_in, x, lay, xn, layn, xh);
  rmt_count_launches(1);
  for (int l = 1; l <= g.layers; l++) {
    k_wls_half<T, false><<<wls_blocks, TPB, 0, s>>>(g, b, l, lay, layn, xn, xh, list, cnt, redo, err);
    rmt_count_launches(1);
    if (sizeof(T) == 4) {
      k_wls_half<T, true><<<sm_count(), TPB, 0, s>>>(g, b, l, lay, layn, xn, xh, list, cnt, redo, err);
      rmt_count_launches(1);
    }
  }
  k_phi_half<T><<<blocks, TPB, 0, s>>>(g, b, bb_in, xh, layn, phih);
  rmt_count_launches(1);
}

#define INST(T)                                                                                                \
  template void launch_init_xi<T>(const Geo&, const Body&, T*, cudaStream_t);                                   \
  template cudaError_t launch_extrapolate<T>(const Geo&, const Body&, const int*, int*, int, int*, int*, int*, int, \
                                             T*, T*, int8_t*, int*, cudaStream_t);                              \
  template void launch_corrector<T>(const Geo&, const Body&, const int*, int, const int*, int*, int*, int,        \
                                    const T*, const int8_t*, const T*, const int8_t*, T*, T*, int*, cudaStream_t);
INST(float)
INST(double)
