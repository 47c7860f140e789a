// Predictor of the reference map (arXiv 2104.00095, eq. dis_xi_adv with the Godunov face
// states of eq. xi_taylor_final and the tangential terms of SI "Tangential derivatives").
// One thread per cell of layers 0 and 1 rebuilds the xi states at its six faces.
#include "rmt_kernels.h"

namespace {

constexpr int TPB = 256;

inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > 152L * 64) b = 152L * 64;  // grid-stride beyond 64 blocks per SM
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void decode(long c, int nx, int ny, int& i, int& j, int& k) {
  i = (int)(c % nx);
  long r = c / nx;
  j = (int)(r % ny);
  k = (int)(r / ny);
}


template <typename T>
__device__ __forceinline__ void cell_faces(const Geo& g, int e, int i, int j, int k, long& lo, long& hi) {
  lo = fidx(g, e, i, j, k);
  int ii[3] = {i, j, k};
  ii[e] += 1;
  hi = fidx(g, e, ii[0], ii[1], ii[2]);
}
// ---------------------------------------------------------------------------------
// predictor of the reference map at the cells of layers 0 and 1 (eq. dis_xi_adv)

struct XiPredPtrs {
  const void* vadv[3];
  const void* unpre[3];
  const void* umac[3];
};

template <typename T>
__device__ __forceinline__ bool xi3(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int i,
                                    int j, int k, T v[3]) {
  long c;
  if (!cell_at(g, i, j, k, c) || lay[c] < 0) return false;
  v[0] = x[c];
  v[1] = x[g.N + c];
  v[2] = x[2 * g.N + c];
  return true;
}

template <typename T>
__device__ __noinline__ void slope_xi(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int d, int i, int j,
                         int k, T s[3]) {
  T q[3][5];
  unsigned ok = 0;
#pragma unroll
  for (int t = -2; t <= 2; t++) {
    int ii[3] = {i, j, k};
    ii[d] += t;
    T v[3];
    if (xi3(g, x, lay, ii[0], ii[1], ii[2], v)) {
      ok |= 1u << (t + 2);
      q[0][t + 2] = v[0]; q[1][t + 2] = v[1]; q[2][t + 2] = v[2];
    } else {
      q[0][t + 2] = q[1][t + 2] = q[2][t + 2] = T(0);
    }
  }
  const T ih = cv<T>(g.ih, g.f.ih);
#pragma unroll
  for (int a = 0; a < 3; a++) s[a] = lim_slope(q[a], ok, ih);
}

// xi bar state at the e-face below cell (i,j,k); false when unavailable
template <typename T>
__device__ __noinline__ bool xbar(const Geo& g, const T* __restrict__ u, const T* __restrict__ x, const int8_t* __restrict__ lay,
                     const T* __restrict__ vadv_e, int e, int i, int j, int k, T out[3]) {
  int fc = e == 0 ? i : (e == 1 ? j : k);
  if (!g.per[e] && (fc <= 0 || fc >= g.n[e])) return false;  // wall face
  int lo[3] = {i, j, k};
  lo[e] -= 1;
  T xD[3], xU[3];
  if (!xi3(g, x, lay, lo[0], lo[1], lo[2], xD) || !xi3(g, x, lay, i, j, k, xU)) return false;
  T sD[3], sU[3];
  slope_xi(g, x, lay, e, lo[0], lo[1], lo[2], sD);
  slope_xi(g, x, lay, e, i, j, k, sU);
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt);
  const T uD = uval(g, u, e, lo[0], lo[1], lo[2]), uU = uval(g, u, e, i, j, k);
  int hi[3] = {i, j, k};
  wrap_axis(g, 0, hi[0]);
  wrap_axis(g, 1, hi[1]);
  wrap_axis(g, 2, hi[2]);
  const T va = vadv_e[fidx(g, e, hi[0], hi[1], hi[2])];
#pragma unroll
  for (int a = 0; a < 3; a++)
    out[a] = upwind(xD[a] + (T(0.5) * h - T(0.5) * dt * uD) * sD[a], xU[a] - (T(0.5) * h + T(0.5) * dt * uU) * sU[a], va,
                    cv<T>(g.utol, g.f.utol));
  return true;
}

// Taylor state of xi from cell c toward its d-face; side 0: the face above c (L state),
// side 1: the face below c (R state)
template <typename T>
__device__ __noinline__ void xi_state(const Geo& g, const T* __restrict__ u, const T* __restrict__ x,
                         const int8_t* __restrict__ lay, const XiPredPtrs& pp, int d, int side, int i, int j, int k,
                         T out[3]) {
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt), ih = cv<T>(g.ih, g.f.ih);
  T xc[3], s[3];
  xi3(g, x, lay, i, j, k, xc);
  slope_xi(g, x, lay, d, i, j, k, s);
  const T ud = uval(g, u, d, i, j, k);
  const T coef = side == 0 ? (T(0.5) * h - T(0.5) * dt * ud) : -(T(0.5) * h + T(0.5) * dt * ud);
  T tr[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int e = 0; e < 3; e++) {
    if (e == d) continue;
    int up[3] = {i, j, k};
    up[e] += 1;
    T bl[3], bh[3];
    if (!xbar(g, u, x, lay, (const T*)pp.vadv[e], e, i, j, k, bl)) continue;
    if (!xbar(g, u, x, lay, (const T*)pp.vadv[e], e, up[0], up[1], up[2], bh)) continue;
    int cw[3] = {i, j, k};
    wrap_axis(g, 0, cw[0]);
    wrap_axis(g, 1, cw[1]);
    wrap_axis(g, 2, cw[2]);
    long lo, hi;
    cell_faces<T>(g, e, cw[0], cw[1], cw[2], lo, hi);
    const T* va = (const T*)pp.vadv[e];
    const T vav = T(0.5) * (va[lo] + va[hi]);
#pragma unroll
    for (int a = 0; a < 3; a++) tr[a] += vav * (bh[a] - bl[a]) * ih;
  }
#pragma unroll
  for (int a = 0; a < 3; a++) out[a] = xc[a] + coef * s[a] - T(0.5) * dt * tr[a];
}

template <typename T>
__global__ void k_xi_predict(Geo g, const T* __restrict__ u, XiPredPtrs pp, const int* __restrict__ bb,
                             const T* __restrict__ x, const int8_t* __restrict__ lay, T* __restrict__ xn) {
  const T ih = cv<T>(g.ih, g.f.ih), dt = cv<T>(g.dt, g.f.dt);
  const T nanv = T(__longlong_as_double(0x7ff8000000000000ll));
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int uu[3], i, j, k;
    long c;
    win_cell(g, w, t, uu, i, j, k, c);
    const int l = lay[c];
    if (l < 0 || l > 1) {
      xn[c] = nanv; xn[g.N + c] = nanv; xn[2 * g.N + c] = nanv;
      continue;
    }
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      T xf[2][3];
#pragma unroll
      for (int fs = 0; fs < 2; fs++) {
        // fs = 0: face below c (a = c - e_d, b = c); fs = 1: face above (a = c, b = c + e_d)
        int ca[3] = {i, j, k}, cb[3] = {i, j, k};
        if (fs == 0) ca[d] -= 1; else cb[d] += 1;
        T t0[3];
        const bool okA = xi3(g, x, lay, ca[0], ca[1], ca[2], t0);
        const bool okB = xi3(g, x, lay, cb[0], cb[1], cb[2], t0);
        int fw[3] = {cb[0], cb[1], cb[2]};
        // face index: the d-index of cell b before wrapping (n_d allowed)
        if (fw[d] > g.n[d]) fw[d] -= g.n[d];
        const long f = fidx(g, d, fw[0], fw[1], fw[2]);
        const T un = ((const T*)pp.unpre[d])[f];
        T L[3], R[3];
        if (okA) xi_state(g, u, x, lay, pp, d, 0, ca[0], ca[1], ca[2], L);
        if (okB) xi_state(g, u, x, lay, pp, d, 1, cb[0], cb[1], cb[2], R);
#pragma unroll
        for (int a = 0; a < 3; a++) xf[fs][a] = (okA && okB) ? upwind(L[a], R[a], un, cv<T>(g.utol, g.f.utol)) : (okA ? L[a] : R[a]);
      }
      long lo, hi;
      cell_faces<T>(g, d, i, j, k, lo, hi);
      const T* U = (const T*)pp.umac[d];
      const T va = T(0.5) * (U[lo] + U[hi]);
#pragma unroll
      for (int a = 0; a < 3; a++) acc[a] += va * (xf[1][a] - xf[0][a]) * ih;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) xn[a * g.N + c] = x[a * g.N + c] - dt * acc[a];
  }
}

}  // namespace

template <typename T>
void launch_xi_predict(const Geo& g, const T* u, T* const vadv[3], T* const uf[3][3], T* const umac[3], const int* bb,
                       int blocks, const T* x, const int8_t* lay, T* xn, cudaStream_t s) {
  XiPredPtrs pp;
  for (int d = 0; d < 3; d++) {
    pp.vadv[d] = vadv[d];
    pp.unpre[d] = uf[d][d];
    pp.umac[d] = umac[d];
  }
  k_xi_predict<T><<<blocks, TPB, 0, s>>>(g, u, pp, bb, x, lay, xn);
  rmt_count_launches(1);
}

template void launch_xi_predict<float>(const Geo&, const float*, float* const[3], float* const[3][3], float* const[3],
                                       const int*, int, const float*, const int8_t*, float*, cudaStream_t);
template void launch_xi_predict<double>(const Geo&, const double*, double* const[3], double* const[3][3],
                                        double* const[3], const int*, int, const double*, const int8_t*, double*,
                                        cudaStream_t);
