// Predictor of the reference map (arXiv 2104.00095, eq. dis_xi_adv with the Godunov face
// states of eq. xi_taylor_final and the tangential terms of SI "Tangential derivatives").
// Three passes over a body's window: limited slopes of xi, transverse bar states on faces,
// then the predictor at the cells of layers 0 and 1.
//
// FP32 storage holds S = xi - x0 (rmt_common.cuh).  The slopes are those of xi (the limiter sees
// differences of xi: h + dS along the component's own axis, dS across it); every face state
// is stored as the displacement from the face centre's image, so where the FP64 form adds a
// Taylor term (h/2) s to xi, the FP32 form adds (h/2)(s - 1) for the component along the
// face's axis, and a difference of face states across a cell gains h on that component.
#include "rmt_kernels.h"

namespace {

constexpr int TPB = 256;

inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > (long)sm_count() * 64) b = (long)sm_count() * 64;  // grid-stride beyond 64 blocks per SM
  return (int)(b < 1 ? 1 : b);
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
__device__ __forceinline__ void slope_xi(const Geo& g, const T* __restrict__ x, const int8_t* __restrict__ lay, int d,
                                         int i, int j, int k, T s[3]) {
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
      // FP32 storage: the identity's part of xi_d along axis d, relative to the centre cell (the
      // band never pairs cells across the seam of the body's image window)
      if constexpr (disp_storage<T>()) q[d][t + 2] += T(t) * g.f.h;
    } else {
      q[0][t + 2] = q[1][t + 2] = q[2][t + 2] = T(0);
    }
  }
  const T ih = cv<T>(g.ih, g.f.ih);
#pragma unroll
  for (int a = 0; a < 3; a++) s[a] = lim_slope(q[a], ok, ih);
}

// Per-body scratch shared by the three passes (N-sized arrays, reused body after body):
// s[3d+a] limited slope of xi_a along d at a cell; xb[3e+a] the upwinded bar state of xi_a
// on the e-face below a cell, ok[e] its availability.
struct XiScratch {
  void* s[9];
  void* xb[9];
  int8_t* ok[3];
};

// pass 1: limited slopes of xi at every band cell of the window
template <typename T>
__global__ void k_xi_slopes(Geo g, const int* __restrict__ bb, const T* __restrict__ x, const int8_t* __restrict__ lay,
                            XiScratch sc) {
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int uu[3], i, j, k;
    long c;
    win_cell(g, w, t, uu, i, j, k, c);
    if (lay[c] < 0) continue;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      T s3[3];
      slope_xi(g, x, lay, d, i, j, k, s3);
#pragma unroll
      for (int a = 0; a < 3; a++) ((T*)sc.s[3 * d + a])[c] = s3[a];
    }
  }
}

// pass 2: transverse bar states of xi on the e-face below every window cell (SI "Tangential
// derivatives"), upwinded with the velocity's advecting bar velocity; unavailable on walls
// and where either cell lacks xi
template <typename T>
__global__ void k_xi_bar(Geo g, const int* __restrict__ bb, const T* __restrict__ u, XiPredPtrs pp,
                         const T* __restrict__ x, const int8_t* __restrict__ lay, XiScratch sc) {
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt);
  const Win w = make_win(g, bb, 2);
  WIN_LOOP(t, w) {
    int uu[3], i, j, k;
    long c;
    win_cell(g, w, t, uu, i, j, k, c);
    const int cc[3] = {i, j, k};
#pragma unroll
    for (int e = 0; e < 3; e++) {
      int8_t ok = 0;
      if ((g.per[e] || cc[e] > 0) && lay[c] >= 0) {
        int lo[3] = {i, j, k};
        lo[e] = cc[e] > 0 ? cc[e] - 1 : g.n[e] - 1;
        const long cD = cidx(g, lo[0], lo[1], lo[2]);
        if (lay[cD] >= 0) {
          ok = 1;
          const T uD = u[e * g.N + cD], uU = u[e * g.N + c];
          const T va = ((const T*)pp.vadv[e])[fidx(g, e, i, j, k)];
#pragma unroll
          for (int a = 0; a < 3; a++) {
            const T sD = ((const T*)sc.s[3 * e + a])[cD], sU = ((const T*)sc.s[3 * e + a])[c];
            T L, R;
            if constexpr (disp_storage<T>()) {
              // displacements from the face centre's image x0_D + (h/2) e_e = x0_U - (h/2) e_e
              const T id = a == e ? T(1) : T(0);
              L = x[a * g.N + cD] + T(0.5) * h * (sD - id) - T(0.5) * dt * uD * sD;
              R = x[a * g.N + c] - T(0.5) * h * (sU - id) - T(0.5) * dt * uU * sU;
            } else {
              L = x[a * g.N + cD] + (T(0.5) * h - T(0.5) * dt * uD) * sD;
              R = x[a * g.N + c] - (T(0.5) * h + T(0.5) * dt * uU) * sU;
            }
            ((T*)sc.xb[3 * e + a])[c] = upwind(L, R, va, cv<T>(g.utol, g.f.utol));
          }
        }
      }
      sc.ok[e][c] = ok;
    }
  }
}

// Taylor state of xi from cell (i,j,k) (inside the grid) toward its d-face (eq. xi_taylor_final):
// side 0 the face above the cell (L state), side 1 the face below (R state)
template <typename T>
__device__ __forceinline__ void xi_state(const Geo& g, const T* __restrict__ u, const T* __restrict__ x,
                                         const XiPredPtrs& pp, const XiScratch& sc, int d, int side, int i, int j,
                                         int k, T out[3]) {
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt), ih = cv<T>(g.ih, g.f.ih);
  const long c = cidx(g, i, j, k);
  const T ud = u[d * g.N + c];
  const T coef = side == 0 ? (T(0.5) * h - T(0.5) * dt * ud) : -(T(0.5) * h + T(0.5) * dt * ud);
  T tr[3] = {T(0), T(0), T(0)};
  const int cc[3] = {i, j, k};
#pragma unroll
  for (int e = 0; e < 3; e++) {
    if (e == d) continue;
    // bar states on the e-faces below and above the cell; the one above is owned by the next
    // cell along e (none past a wall)
    if (!sc.ok[e][c]) continue;
    if (!g.per[e] && cc[e] == g.n[e] - 1) continue;
    int up[3] = {i, j, k};
    up[e] = cc[e] + 1 < g.n[e] ? cc[e] + 1 : 0;
    const long cu = cidx(g, up[0], up[1], up[2]);
    if (!sc.ok[e][cu]) continue;
    long lo, hi;
    cell_faces<T>(g, e, i, j, k, lo, hi);
    const T* va = (const T*)pp.vadv[e];
    const T vav = T(0.5) * (va[lo] + va[hi]);
#pragma unroll
    for (int a = 0; a < 3; a++)
      tr[a] += vav * (((const T*)sc.xb[3 * e + a])[cu] - ((const T*)sc.xb[3 * e + a])[c]) * ih;
    // FP32 storage: the two bar states are displacements from face centres h apart along e
    if constexpr (disp_storage<T>()) tr[e] += vav;
  }
  if constexpr (disp_storage<T>()) {
    // displacement from the face centre's image x0_c +- (h/2) e_d
    const T sg = side == 0 ? T(0.5) * h : -T(0.5) * h;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const T s = ((const T*)sc.s[3 * d + a])[c];
      out[a] = x[a * g.N + c] + sg * (s - (a == d ? T(1) : T(0))) - T(0.5) * dt * ud * s - T(0.5) * dt * tr[a];
    }
    return;
  }
#pragma unroll
  for (int a = 0; a < 3; a++)
    out[a] = x[a * g.N + c] + coef * ((const T*)sc.s[3 * d + a])[c] - T(0.5) * dt * tr[a];
}

// pass 3: xi^{n+1} = xi^n - dt [(u.grad) xi]^{n+1/2} at the cells of layers 0 and 1 whose six faces
// carry xi^{n+1/2}; NaN at every other window cell
template <typename T>
__global__ void k_xi_predict(Geo g, const T* __restrict__ u, XiPredPtrs pp, const int* __restrict__ bb,
                             const T* __restrict__ x, const int8_t* __restrict__ lay, XiScratch sc,
                             T* __restrict__ xn) {
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
        const long f = fidx(g, d, cb[0], cb[1], cb[2]);  // face index: d-index of b, up to n_d
        long la, lb;
        const bool okA = cell_at(g, ca[0], ca[1], ca[2], la) && lay[la] >= 0;
        const bool okB = cell_at(g, cb[0], cb[1], cb[2], lb) && lay[lb] >= 0;
        wrap_axis(g, d, ca[d]);
        wrap_axis(g, d, cb[d]);
        const T un = ((const T*)pp.unpre[d])[f];
        T L[3], R[3];
        if (okA) xi_state(g, u, x, pp, sc, d, 0, ca[0], ca[1], ca[2], L);
        if (okB) xi_state(g, u, x, pp, sc, d, 1, cb[0], cb[1], cb[2], R);
#pragma unroll
        for (int a = 0; a < 3; a++)
          xf[fs][a] = (okA && okB) ? upwind(L[a], R[a], un, cv<T>(g.utol, g.f.utol)) : (okA ? L[a] : R[a]);
      }
      long lo, hi;
      cell_faces<T>(g, d, i, j, k, lo, hi);
      const T* U = (const T*)pp.umac[d];
      const T va = T(0.5) * (U[lo] + U[hi]);
#pragma unroll
      for (int a = 0; a < 3; a++) acc[a] += va * (xf[1][a] - xf[0][a]) * ih;
      // FP32 storage: the face states are displacements from face centres h apart along d
      if constexpr (disp_storage<T>()) acc[d] += va;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) xn[a * g.N + c] = x[a * g.N + c] - dt * acc[a];
  }
}

}  // namespace

template <typename T>
void launch_xi_predict(const Geo& g, const T* u, T* const vadv[3], T* const uf[3][3], T* const umac[3], const int* bb,
                       int blocks, const T* x, const int8_t* lay, T* const scratch_s[9], T* const scratch_xb[9],
                       int8_t* const scratch_ok[3], T* xn, cudaStream_t s) {
  XiPredPtrs pp;
  XiScratch sc;
  for (int d = 0; d < 3; d++) {
    pp.vadv[d] = vadv[d];
    pp.unpre[d] = uf[d][d];
    pp.umac[d] = umac[d];
    sc.ok[d] = scratch_ok[d];
  }
  for (int q = 0; q < 9; q++) {
    sc.s[q] = scratch_s[q];
    sc.xb[q] = scratch_xb[q];
  }
  k_xi_slopes<T><<<blocks, TPB, 0, s>>>(g, bb, x, lay, sc);
  rmt_count_launches(1);
  k_xi_bar<T><<<blocks, TPB, 0, s>>>(g, bb, u, pp, x, lay, sc);
  rmt_count_launches(1);
  k_xi_predict<T><<<blocks, TPB, 0, s>>>(g, u, pp, bb, x, lay, sc, xn);
  rmt_count_launches(1);
}

template void launch_xi_predict<float>(const Geo&, const float*, float* const[3], float* const[3][3], float* const[3],
                                       const int*, int, const float*, const int8_t*, float* const[9], float* const[9],
                                       int8_t* const[3], float*, cudaStream_t);
template void launch_xi_predict<double>(const Geo&, const double*, double* const[3], double* const[3][3],
                                        double* const[3], const int*, int, const double*, const int8_t*,
                                        double* const[9], double* const[9], int8_t* const[3], double*, cudaStream_t);
