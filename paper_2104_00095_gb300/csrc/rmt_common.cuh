// Device-side building blocks of the RMT per-step update (arXiv 2104.00095).
// Everything here is templated on the compute type T (double: FP64 path; float: FP32 bulk).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RMT_MAX_BODIES 64

// process-wide count of kernels launched by this library (defined in rmt_api.cu)
void rmt_count_launches(long n);
#define RMT_PI 3.14159265358979323846

// Grid geometry and the fluid constants, passed by value to every kernel.
struct Geo {
  int n[3];        // cells per axis
  int per[3];      // 1 on a periodic axis
  int nn[3];       // nodes per axis (n+1 walled, n periodic)
  long N, NN;      // cells, nodes
  double h, dt, eps, rho_f, mu;
  double utol;     // |v| <= utol counts as zero in the upwind decisions (1e-12 h/dt)
  double lo[3], len[3];
  double wall[6][3];
  double grav[3];
  int layers;      // extrapolation layers
  double dw;       // wall-repulsion threshold distance
  int any_rep;     // some body has a wall-repulsion acceleration
  // derived constants (host-computed by geo_finish) and float mirrors of everything a kernel
  // reads, so that FP32 kernels never convert or divide in FP64
  double ih, q4, hdt_h, two_dt, fe_rhs;  // 1/h, 0.25/h, dt/(2h), 2/dt, h^2/(4 dt)
  struct {
    float h, ih, q4, hdt_h, dt, eps, rho_f, mu, utol, wall[6][3], grav[3];
    float two_dt, two_dt_lo, fe_rhs, fe_rhs_lo;  // two-float pairs (value = hi + lo)
    float dw;
  } f;
};

// One body's constants (Table pars + shape + active stress), with float mirrors.
struct Body {
  int shape;
  double c[3], a[3], R[9];
  double rho_s, G, mu_a, gamma_t, actA, actW, actL;
  double repA;         // wall-repulsion acceleration (0: none)
  double a2[3], mina;  // squared semi-axes, smallest semi-axis (body_finish)
  // FP32 storage keeps the reference map as the displacement S = xi - x0 from x0, the cell
  // centre's image in a fixed window of periodic images around the body centre: unwrapped cell
  // coordinates wlo[d] .. wlo[d] + n_d - 1 on a periodic axis (the cell itself on a walled one).
  // cu: the cell coordinate nearest the centre; off = lo + (cu + 1/2) h - c, so that x0 - c =
  // (u - cu) h + off holds small numbers only (body_image)
  int wlo[3], cu[3];
  double off[3];
  struct {
    float c[3], a[3], R[9], a2[3], mina, rho_s, G, mu_a, gamma_t, actA, actW, actL, repA, off[3];
  } f;
};

// the value of a constant in the compute type: its float mirror for float, itself for double
template <typename T>
__host__ __device__ __forceinline__ T cv(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// fills the derived constants and float mirrors of a grid (host)
inline void geo_finish(Geo& g) {
  g.ih = 1.0 / g.h;
  g.q4 = 0.25 / g.h;
  g.hdt_h = 0.5 * g.dt / g.h;
  g.two_dt = g.dt > 0 ? 2.0 / g.dt : 0.0;
  g.fe_rhs = g.dt > 0 ? g.h * g.h / 4.0 / g.dt : 0.0;
  g.f.h = (float)g.h;
  g.f.ih = (float)g.ih;
  g.f.q4 = (float)g.q4;
  g.f.hdt_h = (float)g.hdt_h;
  g.f.dt = (float)g.dt;
  g.f.eps = (float)g.eps;
  g.f.rho_f = (float)g.rho_f;
  g.f.mu = (float)g.mu;
  g.f.utol = (float)g.utol;
  for (int q = 0; q < 6; q++)
    for (int a = 0; a < 3; a++) g.f.wall[q][a] = (float)g.wall[q][a];
  for (int a = 0; a < 3; a++) g.f.grav[a] = (float)g.grav[a];
  g.f.two_dt = (float)g.two_dt;
  g.f.two_dt_lo = (float)(g.two_dt - (double)g.f.two_dt);
  g.f.fe_rhs = (float)g.fe_rhs;
  g.f.fe_rhs_lo = (float)(g.fe_rhs - (double)g.f.fe_rhs);
  g.f.dw = (float)g.dw;
}
// fills the derived constants and float mirrors of a body (host)
inline void body_finish(Body& b) {
  b.mina = b.a[0];
  if (b.a[1] < b.mina) b.mina = b.a[1];
  if (b.a[2] < b.mina) b.mina = b.a[2];
  for (int a = 0; a < 3; a++) {
    b.a2[a] = b.a[a] * b.a[a];
    b.f.c[a] = (float)b.c[a];
    b.f.a[a] = (float)b.a[a];
    b.f.a2[a] = (float)b.a2[a];
  }
  for (int q = 0; q < 9; q++) b.f.R[q] = (float)b.R[q];
  b.f.mina = (float)b.mina;
  b.f.rho_s = (float)b.rho_s;
  b.f.G = (float)b.G;
  b.f.mu_a = (float)b.mu_a;
  b.f.gamma_t = (float)b.gamma_t;
  b.f.actA = (float)b.actA;
  b.f.actW = (float)b.actW;
  b.f.actL = (float)b.actL;
  b.f.repA = (float)b.repA;
}
// the image window of a body on grid g (host; after body_finish and geo_finish)
inline void body_image(Body& b, const Geo& g) {
  for (int d = 0; d < 3; d++) {
    const double ci = (b.c[d] - g.lo[d]) / g.h - 0.5;
    b.cu[d] = (int)floor(ci + 0.5);
    b.off[d] = g.lo[d] + (b.cu[d] + 0.5) * g.h - b.c[d];
    b.f.off[d] = (float)b.off[d];
    b.wlo[d] = g.per[d] ? b.cu[d] - g.n[d] / 2 : 0;
  }
}

// The reference-map fields of one body at one time level.
template <typename T>
struct BodyView {
  const T* x;        // [3][N]
  const T* phi;      // [N]
  const int8_t* lay; // [N], -1 = absent
};

// Linear indices of cells, nodes and faces are formed in 32-bit arithmetic (a 64-bit product is
// several instructions on the GPU): grid creation refuses grids of 2^31 or more nodes, so none of
// them overflows an int.
__host__ __device__ __forceinline__ long cidx(const Geo& g, int i, int j, int k) {
  return (long)(i + g.n[0] * (j + g.n[1] * k));
}
__host__ __device__ __forceinline__ long nidx(const Geo& g, int i, int j, int k) {
  return (long)(i + g.nn[0] * (j + g.nn[1] * k));
}
// d-face whose d-index is the face index f in [0, n_d] (between cells f-1 and f)
__host__ __device__ __forceinline__ long fidx(const Geo& g, int d, int i, int j, int k) {
  const int e0 = g.n[0] + (d == 0), e1 = g.n[1] + (d == 1);
  return (long)(i + e0 * (j + e1 * k));
}
__host__ __device__ __forceinline__ long nfaces(const Geo& g, int d) {
  return g.N / g.n[d] * (g.n[d] + 1);
}

// wraps a cell coordinate on a periodic axis; false outside a wall
__device__ __forceinline__ bool wrap_axis(const Geo& g, int d, int& i) {
  const int n = g.n[d];
  if (i >= 0 && i < n) return true;
  if (!g.per[d]) return false;
  i %= n;
  if (i < 0) i += n;
  return true;
}
__device__ __forceinline__ bool cell_at(const Geo& g, int i, int j, int k, long& c) {
  if (!wrap_axis(g, 0, i) || !wrap_axis(g, 1, j) || !wrap_axis(g, 2, k)) return false;
  c = cidx(g, i, j, k);
  return true;
}
__device__ __forceinline__ long node_at(const Geo& g, int i, int j, int k) {
  if (g.per[0] && i >= g.nn[0]) i -= g.nn[0];
  if (g.per[1] && j >= g.nn[1]) j -= g.nn[1];
  if (g.per[2] && k >= g.nn[2]) k -= g.nn[2];
  return nidx(g, i, j, k);
}

// Velocity component a at any cell coordinate: periodic wrap, or the mirrored ghost
// 2 u_wall - u_mirror across a no-slip wall (applied axis by axis).
template <typename T>
__device__ __forceinline__ T uval(const Geo& g, const T* __restrict__ u, int a, int i, int j, int k) {
  T add = T(0), s = T(1);
  int ii[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const int n = g.n[d];
    if (ii[d] < 0 || ii[d] >= n) {
      if (g.per[d]) {
        ii[d] %= n;
        if (ii[d] < 0) ii[d] += n;
      } else {
        const int f = ii[d] < 0 ? 2 * d : 2 * d + 1;
        add += s * (T(2) * cv<T>(g.wall[f][a], g.f.wall[f][a]));
        s = -s;
        ii[d] = ii[d] < 0 ? -1 - ii[d] : 2 * n - 1 - ii[d];
      }
    }
  }
  return add + s * u[a * g.N + cidx(g, ii[0], ii[1], ii[2])];
}

// u component a at (i,j,k) along with its +-r neighbours on axis d: direct loads when the whole
// stencil lies inside the grid (the common case), the boundary rules otherwise
template <typename T>
__device__ __forceinline__ bool inside(const Geo& g, int d, int i, int j, int k, int r) {
  const int ii[3] = {i, j, k};
  if (ii[0] < 0 || ii[0] >= g.n[0] || ii[1] < 0 || ii[1] >= g.n[1] || ii[2] < 0 || ii[2] >= g.n[2]) return false;
  return ii[d] - r >= 0 && ii[d] + r < g.n[d];
}

// 3-D launch geometry for cell/face/node kernels: 32 x 4 threads per block in x and y, one
// block layer per z index
#define TILE_X 32
#define TILE_Y 4
#define THREAD_XYZ(i, j, k)                     \
  const int i = blockIdx.x * TILE_X + threadIdx.x; \
  const int j = blockIdx.y * TILE_Y + threadIdx.y; \
  const int k = blockIdx.z

// -------------------------------------------------------------------------------------
// explicitly rounded arithmetic (no contraction), used where a sign decides an integer
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }

// Level set phi_0 of a body's reference shape (main text "Blurred interface method").
// Sphere: exact signed distance.  Ellipsoid: (g-1)/|grad g| with g = |D^-1 R^T (X-c)|.
// phi0_r takes the position relative to the centre, r = X - c.
template <typename T>
__device__ T phi0_r(const Body& b, T r0, T r1, T r2) {
#define BC(x) cv<T>(b.x, b.f.x)
  if (b.shape == 0)
    return sub_rn(sqrt_rn(add_rn(add_rn(mul_rn(r0, r0), mul_rn(r1, r1)), mul_rn(r2, r2))), BC(a[0]));
  const T z0 = add_rn(add_rn(mul_rn(BC(R[0]), r0), mul_rn(BC(R[3]), r1)), mul_rn(BC(R[6]), r2));
  const T z1 = add_rn(add_rn(mul_rn(BC(R[1]), r0), mul_rn(BC(R[4]), r1)), mul_rn(BC(R[7]), r2));
  const T z2 = add_rn(add_rn(mul_rn(BC(R[2]), r0), mul_rn(BC(R[5]), r1)), mul_rn(BC(R[8]), r2));
  const T y0 = div_rn(z0, BC(a[0])), y1 = div_rn(z1, BC(a[1])), y2 = div_rn(z2, BC(a[2]));
  const T gg = sqrt_rn(add_rn(add_rn(mul_rn(y0, y0), mul_rn(y1, y1)), mul_rn(y2, y2)));
  if (gg < T(1e-12)) return -BC(mina);
  const T w0 = div_rn(y0, BC(a[0])), w1 = div_rn(y1, BC(a[1])), w2 = div_rn(y2, BC(a[2]));
  const T wn = sqrt_rn(add_rn(add_rn(mul_rn(w0, w0), mul_rn(w1, w1)), mul_rn(w2, w2)));
  return div_rn(mul_rn(sub_rn(gg, T(1)), gg), wn);
}
template <typename T>
__device__ T phi0(const Body& b, T X0, T X1, T X2) {
  return phi0_r(b, sub_rn(X0, BC(c[0])), sub_rn(X1, BC(c[1])), sub_rn(X2, BC(c[2])));
}

// direction of grad_X phi_0 at X = c + r (the WLS weights use its direction only)
template <typename T>
__device__ void phi0_dir_r(const Body& b, const T r[3], T gd[3]) {
  if (b.shape == 0) {
    gd[0] = r[0]; gd[1] = r[1]; gd[2] = r[2];
    return;
  }
  T w[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const T z = BC(R[a]) * r[0] + BC(R[3 + a]) * r[1] + BC(R[6 + a]) * r[2];
    w[a] = z / BC(a2[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) gd[a] = BC(R[3 * a]) * w[0] + BC(R[3 * a + 1]) * w[1] + BC(R[3 * a + 2]) * w[2];
}
template <typename T>
__device__ void phi0_dir(const Body& b, const T X[3], T gd[3]) {
  const T r[3] = {X[0] - BC(c[0]), X[1] - BC(c[1]), X[2] - BC(c[2])};
  phi0_dir_r(b, r, gd);
}
#undef BC

// ---- stored reference maps --------------------------------------------------------
// FP64 storage holds xi itself; FP32 storage holds S = xi - x0 (see Body), so that FP32
// rounding applies to the displacement rather than to O(1) positions: a difference of
// neighbouring values is (x0 difference, a multiple of h) + (S difference).
template <typename T>
__host__ __device__ __forceinline__ constexpr bool disp_storage() { return sizeof(T) == 4; }

// unwrapped image coordinate of cell index i (in [0, n)) on axis d
__host__ __device__ __forceinline__ int img_u(const Geo& g, const Body& b, int d, int i) {
  if (!g.per[d]) return i;
  int t = (i - b.wlo[d]) % g.n[d];
  if (t < 0) t += g.n[d];
  return b.wlo[d] + t;
}
// x0 - c of cell index i on axis d (x0: the image of the cell centre)
template <typename T>
__device__ __forceinline__ T cell_rel(const Geo& g, const Body& b, int d, int i) {
  return T(img_u(g, b, d, i) - b.cu[d]) * cv<T>(g.h, g.f.h) + cv<T>(b.off[d], b.f.off[d]);
}
// xi - c at cell (i,j,k) from its stored value v
template <typename T>
__device__ __forceinline__ void xi_rel(const Geo& g, const Body& b, int i, int j, int k, const T v[3], T r[3]) {
  if constexpr (disp_storage<T>()) {
    r[0] = cell_rel<T>(g, b, 0, i) + v[0];
    r[1] = cell_rel<T>(g, b, 1, j) + v[1];
    r[2] = cell_rel<T>(g, b, 2, k) + v[2];
  } else {
    r[0] = sub_rn(v[0], (T)b.c[0]);
    r[1] = sub_rn(v[1], (T)b.c[1]);
    r[2] = sub_rn(v[2], (T)b.c[2]);
  }
}
// phi_0(xi) at cell (i,j,k) from its stored value (FP64: exactly phi0 of the value)
template <typename T>
__device__ __forceinline__ T phi_stored(const Geo& g, const Body& b, int i, int j, int k, T v0, T v1, T v2) {
  const T v[3] = {v0, v1, v2};
  T r[3];
  xi_rel<T>(g, b, i, j, k, v, r);
  return phi0_r(b, r[0], r[1], r[2]);
}
// FP32 storage: a band cell closer than this many cells to the edge of its body's image window
// on a periodic axis is reported (the stencils then never pair cells across the window's seam)
constexpr int SEAM_MARGIN = 3;
__device__ __forceinline__ bool near_seam(const Geo& g, const Body& b, int i, int j, int k) {
  const int ii[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (!g.per[d]) continue;
    const int t = img_u(g, b, d, ii[d]) - b.wlo[d];
    if (t < SEAM_MARGIN || t > g.n[d] - 1 - SEAM_MARGIN) return true;
  }
  return false;
}

// smoothed Heaviside (eq. sm_heavi) and its derivative
template <typename T>
__device__ __forceinline__ T heavi(T phi, T eps) {
  if (phi <= -eps) return T(0);
  if (phi >= eps) return T(1);
  return T(0.5) * (T(1) + phi / eps + sin(T(RMT_PI) * phi / eps) / T(RMT_PI));
}
template <typename T>
__device__ __forceinline__ T dheavi(T phi, T eps) {
  if (phi <= -eps || phi >= eps) return T(0);
  return T(0.5) / eps * (T(1) + cos(T(RMT_PI) * phi / eps));
}

// Fourth-order monotonicity-limited slope (after Colella 1990); q[0..4] = q_{i-2..i+2}.
// Missing outer values fall back to the second-order limited slope, a missing inner
// neighbour gives zero.
template <typename T>
__device__ __forceinline__ T mc_lim(T qm, T q0, T qp) {
  const T a = qp - q0, b = q0 - qm;
  return (a * b > T(0)) ? T(2) * fmin(fabs(a), fabs(b)) : T(0);
}
// sgn(s) min(|x|, y) for y >= 0, written as copysign(min(|x|, y), s): equal to the product form
// for every s (s = 0 makes the limiters' y vanish, so both give zero, up to the sign of zero)
template <typename T>
__device__ __forceinline__ T sgn_min(T s, T x, T y) { return copysign(fmin(fabs(x), y), s); }
template <typename T>
__device__ __forceinline__ T dflim(T qm, T q0, T qp) {
  const T dc = T(0.5) * (qp - qm);
  return sgn_min(dc, dc, mc_lim(qm, q0, qp));
}
template <typename T>
__device__ __forceinline__ T lim_slope(const T q[5], unsigned okmask, T inv_h) {
  // okmask bit s set when q[s] is present
  if ((okmask & 0xE) != 0xE) return T(0);
  const T dc = T(0.5) * (q[3] - q[1]);
  const T dl = mc_lim(q[1], q[2], q[3]);
  if ((okmask & 0x11) != 0x11) return sgn_min(dc, dc, dl) * inv_h;
  const T dfp = dflim(q[2], q[3], q[4]);
  const T dfm = dflim(q[0], q[1], q[2]);
  // FP32: the sixth as a product (a division per slope would dominate the kernel)
  T d4;
  if constexpr (sizeof(T) == 4) d4 = T(4.0 / 3.0) * dc - (dfp + dfm) * T(1.0 / 6.0);
  else d4 = T(4.0 / 3.0) * dc - (dfp + dfm) / T(6);
  return sgn_min(dc, d4, dl) * inv_h;
}

// Godunov choice of the normal velocity and upwinding of other quantities
// (SI "Godunov-type upwinding scheme")
// (SI "Godunov-type upwinding scheme"); the "= 0" cases hold for |v| <= tol so that a velocity
// that vanishes in exact arithmetic does not choose its side from rounding noise
template <typename T>
__device__ __forceinline__ T god_normal(T L, T R, T tol) {
  if (L > tol && L + R > tol) return L;
  if (R < -tol && L + R < -tol) return R;
  return T(0);
}
template <typename T>
__device__ __forceinline__ T upwind(T L, T R, T un, T tol) {
  return un > tol ? L : (un < -tol ? R : T(0.5) * (L + R));
}

// Multi-body mixing (SI eq. mod_heaviside): in place, w[m] = 1 - H_m on entry, the
// (normalised) solid weights on exit; returns the fluid fraction.
template <typename T>
__device__ __forceinline__ T mix_weights(int cnt, T* w) {
  T sum = T(0);
  for (int m = 0; m < cnt; m++) sum += w[m];
  if (sum > T(1))
    for (int m = 0; m < cnt; m++) w[m] = w[m] / sum;
  const T H = T(1) - sum;
  return H > T(0) ? H : T(0);
}

// 3x3 inverse by the adjugate; false when singular
template <typename T>
__device__ __forceinline__ bool inv3(const T A[9], T F[9]) {
  const T det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (det == T(0) || !isfinite(det)) return false;
  F[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  F[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  F[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  F[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  F[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  F[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  F[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  F[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  F[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return true;
}

// Work window of one body: the bounding box of its band (unwrapped cell coordinates,
// inclusive min in bb[0..2], max in bb[3..5]) dilated by dil cells, clamped at walls; a null
// box means the whole grid.  The band moves less than a cell per step, so a window dilated by
// two cells covers every cell a step can add to or remove from the band.
struct Win {
  int lo[3], ext[3];
  long vol;
};
__device__ __forceinline__ Win make_win(const Geo& g, const int* bb, int dil) {
  Win w;
  w.vol = 1;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int lo = 0, hi = g.n[d];
    if (bb) {
      if (bb[d] > bb[3 + d]) {
        lo = 0;
        hi = 0;
      } else {
        lo = bb[d] - dil;
        hi = bb[3 + d] + dil + 1;
        if (!g.per[d]) {
          if (lo < 0) lo = 0;
          if (hi > g.n[d]) hi = g.n[d];
        } else if (hi - lo > g.n[d]) {
          lo = 0;
          hi = g.n[d];
        }
      }
    }
    w.lo[d] = lo;
    w.ext[d] = hi > lo ? hi - lo : 0;
    w.vol *= w.ext[d];
  }
  return w;
}
// (a, b, c) of the linear index t on an n0 x n1 x .. box, a fastest.  32-bit arithmetic while t
// fits: a 64-bit integer division is a long emulated instruction sequence on the GPU, which
// dominated the grid-stride kernels that decoded every index with it.
__device__ __forceinline__ void split3(long t, int n0, int n1, int& a, int& b, int& c) {
  if (t <= 0x7fffffffL) {
    const unsigned tu = (unsigned)t, r = tu / (unsigned)n0, q = r / (unsigned)n1;
    a = (int)(tu - r * (unsigned)n0);
    b = (int)(r - q * (unsigned)n1);
    c = (int)q;
  } else {
    const long r = t / n0, q = r / n1;
    a = (int)(t - r * n0);
    b = (int)(r - q * n1);
    c = (int)q;
  }
}
// cell or node coordinates of a linear index on an nx x ny x .. grid
__device__ __forceinline__ void decode(long c, int nx, int ny, int& i, int& j, int& k) { split3(c, nx, ny, i, j, k); }

// t-th cell of a window: unwrapped coordinates u[] and the wrapped cell index c
__device__ __forceinline__ void win_cell(const Geo& g, const Win& w, long t, int u[3], int& i, int& j, int& k,
                                         long& c) {
  int a, b, cc;
  split3(t, w.ext[0], w.ext[1], a, b, cc);
  u[0] = w.lo[0] + a;
  u[1] = w.lo[1] + b;
  u[2] = w.lo[2] + cc;
  int v[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    v[d] = u[d] % g.n[d];
    if (v[d] < 0) v[d] += g.n[d];
  }
  i = v[0];
  j = v[1];
  k = v[2];
  c = cidx(g, i, j, k);
}
#define WIN_LOOP(t, w) \
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < (w).vol; t += (long)gridDim.x * blockDim.x)

// Band boxes of all bodies staged in shared memory (6 ints per body: inclusive min, max; min
// above max for an empty band), so that a cell reads a body's layer byte only inside its box.
__device__ __forceinline__ void stage_boxes(const int* __restrict__ bbs, int stride, int nb, int* sbb) {
  for (int q = threadIdx.x + blockDim.x * threadIdx.y; q < 6 * nb; q += blockDim.x * blockDim.y)
    sbb[q] = bbs[(q / 6) * stride + q % 6];
  __syncthreads();
}
__device__ __forceinline__ bool in_box_axis(int v, int lo, int hi, int per, int n) {
  int t = v - lo;
  if (per && t < 0) t += n;
  return lo <= hi && t >= 0 && t <= hi - lo;
}
// does the cell range [a, b] of axis d (0 <= a <= b < n) meet the box's range on that axis?
__device__ __forceinline__ bool tile_meets_box(const Geo& g, const int* bb, int d, int a, int b) {
  const int lo = bb[d], hi = bb[3 + d];
  if (lo > hi) return false;
  if (!g.per[d]) return lo <= b && hi >= a;
  const int n = g.n[d];
  if (hi - lo + 1 >= n) return true;
  // the box starts inside the range, or the range starts inside the box
  int s = lo % n;
  if (s < 0) s += n;
  return (s >= a && s <= b) || in_box_axis(a, lo, hi, 1, n);
}
__device__ __forceinline__ bool in_box(const Geo& g, const int* bb, int i, int j, int k) {
  return in_box_axis(i, bb[0], bb[3], g.per[0], g.n[0]) && in_box_axis(j, bb[1], bb[4], g.per[1], g.n[1]) &&
         in_box_axis(k, bb[2], bb[5], g.per[2], g.n[2]);
}

// Wall-repulsion acceleration at cell (i,j,k), index c (SI "Contact with a wall", eq.
// wall_acc): for every no-slip wall whose distance to the cell centre is below d_w, each body
// present at the cell with a repulsion adds A_rep times the transition factor of its phi
// (1 for phi <= -h, 1/2 - phi/(2h) for |phi| < h, 0 beyond) along the wall's inward normal.
// Returns false (out untouched) for cells that no wall reaches.
template <typename T>
__device__ __forceinline__ bool rep_accel(const Geo& g, const Body* __restrict__ bodies,
                                          const BodyView<T>* __restrict__ views, int nb, int i, int j, int k, long c,
                                          T out[3]) {
  const T h = cv<T>(g.h, g.f.h), dw = cv<T>(g.dw, g.f.dw);
  const int ii[3] = {i, j, k};
  T ns[3] = {T(0), T(0), T(0)};
  bool near = false;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (g.per[d]) continue;
    if ((T(ii[d]) + T(0.5)) * h < dw) {
      ns[d] += T(1);
      near = true;
    }
    if ((T(g.n[d] - ii[d]) - T(0.5)) * h < dw) {
      ns[d] -= T(1);
      near = true;
    }
  }
  if (!near) return false;
  out[0] = out[1] = out[2] = T(0);
  for (int m = 0; m < nb; m++) {
    const Body& B = bodies[m];
    if (B.repA == 0.0) continue;
    if (views[m].lay[c] < 0) continue;
    const T ph = views[m].phi[c];
    const T f = ph <= -h ? T(1) : (ph < h ? T(0.5) - ph / (T(2) * h) : T(0));
    const T fa = f * cv<T>(B.repA, B.f.repA);
#pragma unroll
    for (int a = 0; a < 3; a++) out[a] += fa * ns[a];
  }
  return true;
}

// Bodies whose band box meets the block's tile (TILE_X x TILE_Y cells of planes k0..k1): only
// they need a per-cell test.  All threads of the block call it; warp 0 writes the mask to *slot.
__device__ __forceinline__ unsigned long long tile_body_mask(const Geo& g, const int* sbb, int nb, int k0, int k1,
                                                             unsigned long long* slot) {
  if (threadIdx.y == 0) {
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * TILE_Y;
    const int i1 = min(i0 + TILE_X, g.n[0]) - 1, j1 = min(j0 + TILE_Y, g.n[1]) - 1;
    unsigned long long mk = 0;
    for (int base = 0; base < nb; base += 32) {
      const int m = base + threadIdx.x;
      bool hit = false;
      if (m < nb) {
        const int* b = sbb + 6 * m;
        hit = tile_meets_box(g, b, 0, i0, i1) && tile_meets_box(g, b, 1, j0, j1) && tile_meets_box(g, b, 2, k0, k1);
      }
      mk |= (unsigned long long)__ballot_sync(0xffffffffu, hit) << base;
    }
    if (threadIdx.x == 0) *slot = mk;
  }
  __syncthreads();
  return *slot;
}

// grid-stride helper
#define GRID_LOOP(idx, total) \
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < (total); idx += (long)gridDim.x * blockDim.x)
