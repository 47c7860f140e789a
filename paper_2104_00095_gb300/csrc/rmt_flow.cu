// Flow kernels of the RMT per-step update (arXiv 2104.00095, SI sections "Evaluating the
// advective term", "MAC projection", "Approximate pressure-Poisson projection"): Godunov
// velocity states, projection glue, advective term, density mixing and u*.  One thread per
// cell, face or node; templated on T.
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
// Godunov predictor

template <typename T>
__device__ __forceinline__ T slope_u(const Geo& g, const T* __restrict__ u, int a, int d, int i, int j, int k) {
  T q[5];
  if (d == 0 && g.per[0]) {
    // periodic x: wrap by selects, one path for the whole row (no divergence at its ends)
    const T* row = u + (long)a * g.N + cidx(g, 0, j, k);
    const int n0 = g.n[0];
#pragma unroll
    for (int s = -2; s <= 2; s++) {
      int ii = i + s;
      ii += ii < 0 ? n0 : 0;
      ii -= ii >= n0 ? n0 : 0;
      q[s + 2] = row[ii];
    }
  } else if (inside<T>(g, d, i, j, k, 2)) {
    const long c = (long)a * g.N + cidx(g, i, j, k);
    const long st = d == 0 ? 1 : (d == 1 ? (long)g.n[0] : (long)g.n[0] * g.n[1]);
#pragma unroll
    for (int s = -2; s <= 2; s++) q[s + 2] = u[c + s * st];
  } else {
#pragma unroll
    for (int s = -2; s <= 2; s++) {
      int ii[3] = {i, j, k};
      ii[d] += s;
      q[s + 2] = uval(g, u, a, ii[0], ii[1], ii[2]);
    }
  }
  return lim_slope(q, 0x1Fu, cv<T>(g.ih, g.f.ih));
}

// limited slopes of the three velocity components along the three axes at every cell
// (SI "Normal derivatives"); S[3 * d + a] = d u_a / d x_d
struct Slopes9 {
  void* s[9];
};
// A cell whose five-point stencils reach no wall ghost (all points inside, or wrapped across
// periodic sides: every cell of a periodic box) takes the offsets of its +-1, +-2 neighbours
// along each axis once and reads the three components through them; the others go through
// slope_u's boundary rules.  The same values reach the same limiter either way.
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_slopes(Geo g, const T* __restrict__ u, Slopes9 S) {
  THREAD_XYZ(i, j, k);
  if (i >= g.n[0] || j >= g.n[1]) return;
  const long c = cidx(g, i, j, k);
  const int ii[3] = {i, j, k};
  const long st[3] = {1, (long)g.n[0], (long)g.n[0] * g.n[1]};
  long off[3][4];  // neighbours -2, -1, +1, +2 along each axis
  bool fast = true;
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int sft = q < 2 ? q - 2 : q - 1;
      int v = ii[d] + sft;
      if (v < 0 || v >= g.n[d]) {
        fast = fast && g.per[d];
        v += v < 0 ? g.n[d] : -g.n[d];
      }
      off[d][q] = (long)(v - ii[d]) * st[d];
    }
  if (fast) {
    const T ih = cv<T>(g.ih, g.f.ih);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const T* pc = u + (long)a * g.N + c;
      const T x0 = pc[0];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        const T q[5] = {pc[off[d][0]], pc[off[d][1]], x0, pc[off[d][2]], pc[off[d][3]]};
        ((T*)S.s[3 * d + a])[c] = lim_slope(q, 0x1Fu, ih);
      }
    }
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int a = 0; a < 3; a++) ((T*)S.s[3 * d + a])[c] = slope_u(g, u, a, d, i, j, k);
}

__device__ __forceinline__ bool is_wall_face(const Geo& g, int d, int f) {
  return !g.per[d] && (f == 0 || f == g.n[d]);
}

// transverse bar states at every e-face (SI "Tangential derivatives")
template <typename T, int e>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_bar(Geo g, const T* __restrict__ u, Slopes9 S,
                                                         T* __restrict__ ub0, T* __restrict__ ub1, T* __restrict__ ub2,
                                                         T* __restrict__ vadv) {
  const int ex = g.n[0] + (e == 0), ey = g.n[1] + (e == 1), ez = g.n[2] + (e == 2);
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt);
  T* ub[3] = {ub0, ub1, ub2};
  THREAD_XYZ(i, j, k);
  if (i >= ex || j >= ey || k >= ez) return;
  const long f = (long)(i + ex * (j + ey * k));
  const int fi = e == 0 ? i : (e == 1 ? j : k);
  if (is_wall_face(g, e, fi)) {
    const int face = fi == 0 ? 2 * e : 2 * e + 1;
#pragma unroll
    for (int a = 0; a < 3; a++) ub[a][f] = cv<T>(g.wall[face][a], g.f.wall[face][a]);
    vadv[f] = cv<T>(g.wall[face][e], g.f.wall[face][e]);
    return;
  }
  // the two cells of an interior (or periodic) face: D below, U above
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  lo[e] -= 1;
  if (lo[e] < 0) lo[e] += g.n[e];
  if (hi[e] >= g.n[e]) hi[e] -= g.n[e];
  const long cD = cidx(g, lo[0], lo[1], lo[2]), cU = cidx(g, hi[0], hi[1], hi[2]);
  const T uD = u[e * g.N + cD], uU = u[e * g.N + cU];
  T qD[3], qU[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const T* Sa = (const T*)S.s[3 * e + a];
    qD[a] = u[a * g.N + cD] + (T(0.5) * h - T(0.5) * dt * uD) * Sa[cD];
    qU[a] = u[a * g.N + cU] - (T(0.5) * h + T(0.5) * dt * uU) * Sa[cU];
  }
  const T va = god_normal(qD[e], qU[e], cv<T>(g.utol, g.f.utol));
  vadv[f] = va;
#pragma unroll
  for (int a = 0; a < 3; a++) ub[a][f] = upwind(qD[a], qU[a], va, cv<T>(g.utol, g.f.utol));
}

struct BarPtrs {
  const void* ub[3][3];
  const void* vadv[3];
  void* uf[3];
};

// Side-independent part of the face states of every cell (eqs. left_final, right_final):
// W[3d+a] = u_a - (dt/2) T_d(u_a) + dt/(2 rho) F_a, with T_d the tangential terms along the two
// axes other than d (SI "Tangential derivatives") and F = -grad p^{n-1/2} + div tau^n + b^n,
// b = (rho - rho_f) g.  A face state is then W + (+-h/2 - dt/2 u_d) * slope.
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_cellw(Geo g, const T* __restrict__ u, const T* __restrict__ p,
                                                           const T* __restrict__ rho, const T* __restrict__ divtau,
                                                           BarPtrs bp, Slopes9 W, const Body* __restrict__ bodies,
                                                           const BodyView<T>* __restrict__ views, int nb) {
  THREAD_XYZ(i, j, k);
  if (i >= g.n[0] || j >= g.n[1]) return;
  const T dt = cv<T>(g.dt, g.f.dt), ih = cv<T>(g.ih, g.f.ih);
  const long c = cidx(g, i, j, k);
  T gp[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int sa = q & 1, sb = (q >> 1) & 1, sc = (q >> 2) & 1;
    const T pv = p[node_at(g, i + sa, j + sb, k + sc)];
    gp[0] += sa ? pv : -pv;
    gp[1] += sb ? pv : -pv;
    gp[2] += sc ? pv : -pv;
  }
  const T r = rho[c];
  // wall repulsion joins b (SI "Contact with a wall"), from phi^n
  T rep[3];
  const bool has_rep = g.any_rep && rep_accel(g, bodies, views, nb, i, j, k, c, rep);
  T vavg[3];
  long lo[3], hi[3];
#pragma unroll
  for (int e = 0; e < 3; e++) {
    cell_faces<T>(g, e, i, j, k, lo[e], hi[e]);
    const T* vad = (const T*)bp.vadv[e];
    vavg[e] = T(0.5) * (vad[lo[e]] + vad[hi[e]]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    T F = -gp[a] * (T(0.25) * ih) + divtau[a * g.N + c] + (r - cv<T>(g.rho_f, g.f.rho_f)) * cv<T>(g.grav[a], g.f.grav[a]);
    if (has_rep) F = F + r * rep[a];
    T term[3];
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const T* ube = (const T*)bp.ub[e][a];
      term[e] = vavg[e] * (ube[hi[e]] - ube[lo[e]]) * ih;
    }
    const T base = u[a * g.N + c] + T(0.5) * dt / r * F;
    ((T*)W.s[a])[c] = base - T(0.5) * dt * (term[1] + term[2]);
    ((T*)W.s[3 + a])[c] = base - T(0.5) * dt * (term[0] + term[2]);
    ((T*)W.s[6 + a])[c] = base - T(0.5) * dt * (term[0] + term[1]);
  }
}

// normal-face states of the velocity and the Godunov choice (SI "Godunov-type upwinding")
template <typename T, int d>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_face(Geo g, const T* __restrict__ u, Slopes9 S, Slopes9 W,
                                                          BarPtrs bp) {
  const int ex = g.n[0] + (d == 0), ey = g.n[1] + (d == 1), ez = g.n[2] + (d == 2);
  const T h = cv<T>(g.h, g.f.h), dt = cv<T>(g.dt, g.f.dt);
  T* uf[3] = {(T*)bp.uf[0], (T*)bp.uf[1], (T*)bp.uf[2]};
  THREAD_XYZ(i, j, k);
  if (i >= ex || j >= ey || k >= ez) return;
  const long f = (long)(i + ex * (j + ey * k));
  const int fi = d == 0 ? i : (d == 1 ? j : k);
  if (is_wall_face(g, d, fi)) {
    const int face = fi == 0 ? 2 * d : 2 * d + 1;
#pragma unroll
    for (int a = 0; a < 3; a++) uf[a][f] = cv<T>(g.wall[face][a], g.f.wall[face][a]);
    return;
  }
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  lo[d] -= 1;
  if (lo[d] < 0) lo[d] += g.n[d];
  if (hi[d] >= g.n[d]) hi[d] -= g.n[d];
  const long cc[2] = {cidx(g, lo[0], lo[1], lo[2]), cidx(g, hi[0], hi[1], hi[2])};
  T st[2][3];
#pragma unroll
  for (int side = 0; side < 2; side++) {
    const long c = cc[side];
    const T ud = u[d * g.N + c];
    const T coef = side == 0 ? (T(0.5) * h - T(0.5) * dt * ud) : -(T(0.5) * h + T(0.5) * dt * ud);
#pragma unroll
    for (int a = 0; a < 3; a++) st[side][a] = ((const T*)W.s[3 * d + a])[c] + coef * ((const T*)S.s[3 * d + a])[c];
  }
  const T un = god_normal(st[0][d], st[1][d], cv<T>(g.utol, g.f.utol));
#pragma unroll
  for (int a = 0; a < 3; a++) uf[a][f] = (a == d) ? un : upwind(st[0][a], st[1][a], un, cv<T>(g.utol, g.f.utol));
}

// ---------------------------------------------------------------------------------
// MAC projection glue: right-hand side, face coefficients, correction

struct FacePtrs3 {
  void* p[3];
};

// Two-float helpers (FP32 mode hands the multigrid right-hand side and solution over as
// value = hi + lo pairs): Knuth's two-sum and the FMA product, with explicit rounding so that
// no contraction changes them.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// a - b for two-float a = (ah, al), b = (bh, bl), rounded to float (the leading difference is exact)
__device__ __forceinline__ float ff_diff(float ah, float al, float bh, float bl) {
  float s, e;
  two_sum_f(ah, -bh, s, e);
  return __fadd_rn(s, __fadd_rn(e, __fsub_rn(al, bl)));
}
// writes the exact product x * (ch + cl) (x float, c a two-float constant) as a two-float pair
__device__ __forceinline__ void store_prod(MGVec b, long i, float x, float ch, float cl) {
  const float p = __fmul_rn(x, ch);
  const float e = __fmaf_rn(x, cl, __fmaf_rn(x, ch, -p));
  float s, t;
  two_sum_f(p, e, s, t);
  b.h[i] = s;
  b.l[i] = t;
}

template <typename T>
__global__ void k_mac_rhs(Geo g, FacePtrs3 un, MGVec b) {
  const T ih = cv<T>(g.ih, g.f.ih);
  GRID_LOOP(c, g.N) {
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    T dv = T(0);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      long lo, hi;
      cell_faces<T>(g, d, i, j, k, lo, hi);
      const T* U = (const T*)un.p[d];
      dv += (U[hi] - U[lo]) * ih;
    }
    // positive operator A = -div(beta grad): A q = -div(u)/(dt/2)
    if constexpr (sizeof(T) == 8)
      b.d[c] = -(double)dv * g.two_dt;
    else
      store_prod(b, c, -dv, g.f.two_dt, g.f.two_dt_lo);
  }
}

// The three directions' corrections in one pass: one thread per point (i, j, k) of the
// (n0+1) x (n1+1) x (n2+1) lattice of face corners handles the x-, y- and z-faces with that
// index (those that exist), so the cell above the three faces, (i, j, k), has its q and rho read
// once for all of them.  Face coefficient 1/rho_face with rho_face the mean of the two cells.
struct Umac3 {
  const void* un[3];
  void* um[3];
};
// A thread marches up to MCZ lattice points of its (i, j) column: the cell below a z-face is the
// cell above the previous point's faces, so its q and rho come from registers; the column's
// neighbour columns and wall tests are set up once.
constexpr int MCZ = 8;
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_mac_correct3(Geo g, Umac3 F, const T* __restrict__ rho, MGVec q,
                                                                 int zc) {
  const int i = blockIdx.x * TILE_X + threadIdx.x, j = blockIdx.y * TILE_Y + threadIdx.y;
  if (i > g.n[0] || j > g.n[1]) return;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, g.n[2] + 1);
  const T fac = cv<T>(g.hdt_h, g.f.hdt_h);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long plane = (long)n0 * n1;
  const bool cij = i < n0 && j < n1;  // (i, j) is a cell column
  // per direction d < 2: the face (i, j, k) exists (other index a cell), is a wall face, and the
  // columns of its lower and upper cells (the upper one wraps at the periodic end)
  bool has[2], wall[2];
  int colA[2], colB[2];
#pragma unroll
  for (int d = 0; d < 2; d++) {
    const int fi = d == 0 ? i : j;
    has[d] = d == 0 ? j < n1 : i < n0;
    wall[d] = is_wall_face(g, d, fi);
    int lo = fi - 1, up = fi;  // both exist (wrapped) unless the face is a wall face
    wrap_axis(g, d, lo);
    wrap_axis(g, d, up);
    colA[d] = d == 0 ? lo + n0 * j : i + n0 * lo;
    colB[d] = d == 0 ? up + n0 * j : i + n0 * up;
  }
  const int col = i + n0 * j;
  T pr = T(0), ph = T(0), pl = T(0);  // rho and q of cell (i, j, k-1), once loaded
  bool have_prev = false;
  for (int k = k0; k < k1; k++) {
    const bool kin = k < n2;
    const bool bin = cij && kin;  // the cell above the faces exists
    const long cb = col + plane * k;
    T rb = T(0), qbh = T(0), qbl = T(0);
    if (bin) {
      rb = rho[cb];
      if constexpr (sizeof(T) == 8)
        qbh = q.d[cb];
      else {
        qbh = q.h[cb];
        qbl = q.l[cb];
      }
    }
    if (kin) {
#pragma unroll
      for (int d = 0; d < 2; d++) {
        if (!has[d]) continue;
        const long f = fidx(g, d, i, j, k);
        const T* un = (const T*)F.un[d];
        T* um = (T*)F.um[d];
        if (wall[d]) {
          um[f] = un[f];
          continue;
        }
        const long ca = colA[d] + plane * k;
        const long cbb = bin ? cb : colB[d] + plane * k;
        const T ra = rho[ca], rbb = bin ? rb : rho[cbb];
        const T beta = T(2) / (ra + rbb);
        T dq;
        if constexpr (sizeof(T) == 8)
          dq = (bin ? qbh : q.d[cbb]) - q.d[ca];
        else
          dq = bin ? ff_diff(qbh, qbl, q.h[ca], q.l[ca]) : ff_diff(q.h[cbb], q.l[cbb], q.h[ca], q.l[ca]);
        um[f] = un[f] - fac * beta * dq;
      }
    }
    if (cij) {
      // the z-face (i, j, k)
      const long f = fidx(g, 2, i, j, k);
      const T* un = (const T*)F.un[2];
      T* um = (T*)F.um[2];
      if (is_wall_face(g, 2, k)) {
        um[f] = un[f];
      } else {
        if (!have_prev) {  // cell (i, j, k-1), wrapped at the periodic start
          const long ca = col + plane * (k > 0 ? k - 1 : n2 - 1);
          pr = rho[ca];
          if constexpr (sizeof(T) == 8)
            ph = q.d[ca];
          else {
            ph = q.h[ca];
            pl = q.l[ca];
          }
        }
        const long cbb = bin ? cb : col;  // the periodic end: cell (i, j, 0)
        const T rbb = bin ? rb : rho[cbb];
        const T beta = T(2) / (pr + rbb);
        T dq;
        if constexpr (sizeof(T) == 8)
          dq = (bin ? qbh : q.d[cbb]) - ph;
        else
          dq = bin ? ff_diff(qbh, qbl, ph, pl) : ff_diff(q.h[cbb], q.l[cbb], ph, pl);
        um[f] = un[f] - fac * beta * dq;
      }
    }
    pr = rb;
    ph = qbh;
    pl = qbl;
    have_prev = bin;
  }
}

// advective term (eq. adv_terms) with the MAC-corrected normal velocities
struct AdvPtrs {
  const void* uf[3][3];
  const void* umac[3];
};

template <typename T>
__global__ void k_adv(Geo g, AdvPtrs ap, T* __restrict__ adv) {
  const T ih = cv<T>(g.ih, g.f.ih);
  GRID_LOOP(c, g.N) {
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      long lo, hi;
      cell_faces<T>(g, d, i, j, k, lo, hi);
      const T* U = (const T*)ap.umac[d];
      const T va = T(0.5) * (U[lo] + U[hi]);
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const T* Q = (a == d) ? U : (const T*)ap.uf[d][a];
        acc[a] += va * (Q[hi] - Q[lo]) * ih;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) adv[a * g.N + c] = acc[a];
  }
}

// ---------------------------------------------------------------------------------
// density by mixing (eq. mod_heaviside) and u*

// A block marches over up to DZ planes of a TILE_X x TILE_Y column, so the body boxes and the
// tile's body mask are set up once per column.
constexpr int DZ = 8;
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_density(Geo g, const Body* __restrict__ bodies,
                                                             const BodyView<T>* __restrict__ views, int nb,
                                                             const int* __restrict__ bbs, int bstride,
                                                             T* __restrict__ rho, int zc) {
  __shared__ int sbb[6 * RMT_MAX_BODIES];
  __shared__ unsigned long long tile_mask;
  stage_boxes(bbs, bstride, nb, sbb);
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, g.n[2]);
  const unsigned long long tm = tile_body_mask(g, sbb, nb, k0, k1 - 1, &tile_mask);
  const T eps = cv<T>(g.eps, g.f.eps);
  const int i = blockIdx.x * TILE_X + threadIdx.x, j = blockIdx.y * TILE_Y + threadIdx.y;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const T rf = cv<T>(g.rho_f, g.f.rho_f);
  for (int k = k0; k < k1; k++) {
    const long c = cidx(g, i, j, k);
    T wsum = T(0), acc = T(0);
    for (unsigned long long r = tm; r; r &= r - 1) {
      const int m = __ffsll((long long)r) - 1;
      if (!in_box(g, sbb + 6 * m, i, j, k) || views[m].lay[c] < 0) continue;
      const T w = T(1) - heavi(views[m].phi[c], eps);
      acc += w * cv<T>(bodies[m].rho_s, bodies[m].f.rho_s);
      wsum += w;
    }
    const T Hf = wsum < T(1) ? T(1) - wsum : T(0);
    const T sc = wsum > T(1) ? T(1) / wsum : T(1);
    rho[c] = Hf * rf + acc * sc;
  }
}

template <typename T>
__global__ void k_ustar(Geo g, const T* __restrict__ u, const T* __restrict__ adv, const T* __restrict__ p,
                        const T* __restrict__ rho_h, const T* __restrict__ divtau_h, T* __restrict__ ustar,
                        const Body* __restrict__ bodies, const BodyView<T>* __restrict__ views, int nb) {
  const T dt = cv<T>(g.dt, g.f.dt), q4 = cv<T>(g.q4, g.f.q4);
  GRID_LOOP(c, g.N) {
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    T gp[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int sa = q & 1, sb = (q >> 1) & 1, sc = (q >> 2) & 1;
      const T pv = p[node_at(g, i + sa, j + sb, k + sc)];
      gp[0] += sa ? pv : -pv;
      gp[1] += sb ? pv : -pv;
      gp[2] += sc ? pv : -pv;
    }
    const T r = rho_h[c];
    // wall repulsion joins b^{n+1/2} (SI "Contact with a wall"), from phi^{n+1/2}
    T rep[3];
    const bool has_rep = g.any_rep && rep_accel(g, bodies, views, nb, i, j, k, c, rep);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T f = divtau_h[a * g.N + c] - gp[a] * q4 + (r - cv<T>(g.rho_f, g.f.rho_f)) * cv<T>(g.grav[a], g.f.grav[a]);
      if (has_rep) f = f + r * rep[a];
      ustar[a * g.N + c] = u[a * g.N + c] - dt * adv[a * g.N + c] + dt / r * f;
    }
  }
}

// ---------------------------------------------------------------------------------
// approximate FE projection glue

// weak divergence of V = (u* - u^n)/dt at every node: sum over adjacent cells of
// (h^2/4) sum_d sigma_d V_d, sigma_d = +1 when the node is the cell's high corner along d.
// A thread marches up a column of up to FEZ nodes; the four cells of the plane below a node are
// the ones above the previous node, so each cell plane is loaded once per column (the eight cells'
// contributions are still summed in the order sx, sy, sz).
constexpr int FEZ = 16;
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_fe_rhs(Geo g, const T* __restrict__ u,
                                                           const T* __restrict__ ustar, MGVec b, int zc) {
  const int i = blockIdx.x * TILE_X + threadIdx.x, j = blockIdx.y * TILE_Y + threadIdx.y;
  if (i >= g.nn[0] || j >= g.nn[1]) return;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, g.nn[2]);
  // the 2 x 2 cell columns around the node column (sx + 2 sy), -1 outside a wall
  int col[4];
  {
    int cx[2] = {i - 1, i}, cy[2] = {j - 1, j};
    const bool okx0 = wrap_axis(g, 0, cx[0]), okx1 = wrap_axis(g, 0, cx[1]);
    const bool oky0 = wrap_axis(g, 1, cy[0]), oky1 = wrap_axis(g, 1, cy[1]);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int sx = q & 1, sy = q >> 1;
      const bool ok = (sx ? okx1 : okx0) && (sy ? oky1 : oky0);
      col[q] = ok ? cx[sx] + g.n[0] * cy[sy] : -1;
    }
  }
  const int plane = g.n[0] * g.n[1];
  const T* const u1 = u + g.N;
  const T* const u2 = u + 2 * g.N;
  const T* const s1 = ustar + g.N;
  const T* const s2 = ustar + 2 * g.N;
  // V of the four cells of cell plane kc (wrapped; skipped outside a wall)
  auto load = [&](int kc, T (&V)[4][3], bool (&ok)[4]) {
    const bool okz = wrap_axis(g, 2, kc);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      ok[q] = okz && col[q] >= 0;
      const int c = ok[q] ? col[q] + plane * kc : 0;
      V[q][0] = ustar[c] - u[c];
      V[q][1] = s1[c] - u1[c];
      V[q][2] = s2[c] - u2[c];
    }
  };
  T lo[4][3], hi[4][3];
  bool oklo[4], okhi[4];
  load(k0 - 1, lo, oklo);
  for (int k = k0; k < k1; k++) {
    load(k, hi, okhi);
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int sx = q & 1, sy = (q >> 1) & 1, sz = (q >> 2) & 1;
      if (!(sz ? okhi[q & 3] : oklo[q & 3])) continue;
      const T v0 = sz ? hi[q & 3][0] : lo[q & 3][0], v1 = sz ? hi[q & 3][1] : lo[q & 3][1],
              v2 = sz ? hi[q & 3][2] : lo[q & 3][2];
      acc += (sx ? -v0 : v0) + (sy ? -v1 : v1) + (sz ? -v2 : v2);
    }
    const long nd = nidx(g, i, j, k);
    if constexpr (sizeof(T) == 8)
      b.d[nd] = (double)acc * g.fe_rhs;
    else
      store_prod(b, nd, acc, g.f.fe_rhs, g.f.fe_rhs_lo);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      oklo[q] = okhi[q];
#pragma unroll
      for (int a = 0; a < 3; a++) lo[q][a] = hi[q][a];
    }
  }
}

// u^{n+1} = u* - dt/rho grad psi with the cell gradient of the nodal psi.  A thread marches up
// a column of up to FEZ cells; the four nodes below a cell are the ones above the previous cell, so
// each node plane is loaded once per column.
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y) k_fe_update_u(Geo g, const T* __restrict__ ustar,
                                                                const T* __restrict__ rho_h, MGVec psi,
                                                                T* __restrict__ u, int zc) {
  const int i = blockIdx.x * TILE_X + threadIdx.x, j = blockIdx.y * TILE_Y + threadIdx.y;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, g.n[2]);
  const T dt = cv<T>(g.dt, g.f.dt);
  // the 2 x 2 node columns of the cell column (sx + 2 sy), wrapped on a periodic axis
  int col[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    int x = i + (q & 1), y = j + (q >> 1);
    if (g.per[0] && x >= g.nn[0]) x -= g.nn[0];
    if (g.per[1] && y >= g.nn[1]) y -= g.nn[1];
    col[q] = x + g.nn[0] * y;
  }
  const int plane = g.nn[0] * g.nn[1];
  auto node_plane = [&](int kn) { return g.per[2] && kn >= g.nn[2] ? kn - g.nn[2] : kn; };
  // psi at the four nodes of node plane kn (FP64: v[q][0]; FP32: the pair h, l)
  auto load = [&](int kn, T (&v)[4][2]) {
    const int base = plane * node_plane(kn);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if constexpr (sizeof(T) == 8) {
        v[q][0] = psi.d[col[q] + base];
        v[q][1] = 0.0;
      } else {
        v[q][0] = psi.h[col[q] + base];
        v[q][1] = psi.l[col[q] + base];
      }
    }
  };
  T lo[4][2], hi[4][2];
  load(k0, lo);
  for (int k = k0; k < k1; k++) {
    load(k + 1, hi);
    T gp[3];
    if constexpr (sizeof(T) == 8) {
      double s[3] = {0, 0, 0};
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const double pv = q & 4 ? hi[q & 3][0] : lo[q & 3][0];
        s[0] += (q & 1) ? pv : -pv;
        s[1] += ((q >> 1) & 1) ? pv : -pv;
        s[2] += ((q >> 2) & 1) ? pv : -pv;
      }
      for (int a = 0; a < 3; a++) gp[a] = s[a] * g.q4;
    } else {
      // each component: four differences across the cell, each exact to float rounding
      float v[8][2];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        v[q][0] = q & 4 ? hi[q & 3][0] : lo[q & 3][0];
        v[q][1] = q & 4 ? hi[q & 3][1] : lo[q & 3][1];
      }
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const int bit = 1 << a;
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; q++)
          if (q & bit) s += ff_diff(v[q][0], v[q][1], v[q ^ bit][0], v[q ^ bit][1]);
        gp[a] = s * g.f.q4;
      }
    }
    const long c = cidx(g, i, j, k);
    const T r = rho_h[c];
#pragma unroll
    for (int a = 0; a < 3; a++) u[a * g.N + c] = ustar[a * g.N + c] - dt / r * gp[a];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      lo[q][0] = hi[q][0];
      lo[q][1] = hi[q][1];
    }
  }
}

template <typename T>
__global__ void k_fe_update_p(long nn, MGVec psi, T* __restrict__ p, T* __restrict__ psi_out) {
  GRID_LOOP(i, nn) {
    T v;
    if constexpr (sizeof(T) == 8)
      v = psi.d[i];
    else
      v = __fadd_rn(psi.h[i], psi.l[i]);
    p[i] += v;
    psi_out[i] = v;
  }
}

// the wall-repulsion acceleration of every cell as FP64 (read-back of RMT_F_REPULSION)
template <typename T>
__global__ void k_rep_field(Geo g, const Body* __restrict__ bodies, const BodyView<T>* __restrict__ views, int nb,
                            double* __restrict__ out) {
  GRID_LOOP(c, g.N) {
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    T rep[3];
    const bool has = g.any_rep && rep_accel(g, bodies, views, nb, i, j, k, c, rep);
#pragma unroll
    for (int a = 0; a < 3; a++) out[a * g.N + c] = has ? (double)rep[a] : 0.0;
  }
}

template <typename T>
__global__ void k_fill(T* a, T v, long n) {
  GRID_LOOP(i, n) a[i] = v;
}

}  // namespace

template <typename T>
void launch_bar_states(const Geo& g, const T* u, T* const slopes[9], T* const ubar[3][3], T* const vadv[3],
                       cudaStream_t s) {
  Slopes9 S;
  for (int q = 0; q < 9; q++) S.s[q] = slopes[q];
  const dim3 gc((g.n[0] + TILE_X - 1) / TILE_X, (g.n[1] + TILE_Y - 1) / TILE_Y, g.n[2]);
  k_slopes<T><<<gc, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, S);
  rmt_count_launches(1);
  for (int e = 0; e < 3; e++) {
    const dim3 gr((g.n[0] + (e == 0) + TILE_X - 1) / TILE_X, (g.n[1] + (e == 1) + TILE_Y - 1) / TILE_Y, g.n[2] + (e == 2));
    // the direction is a template argument: a runtime index into the pointer bundles would
    // copy them to local memory in every thread
    auto kb = e == 0 ? k_bar<T, 0> : (e == 1 ? k_bar<T, 1> : k_bar<T, 2>);
    kb<<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, S, ubar[e][0], ubar[e][1], ubar[e][2], vadv[e]);
    rmt_count_launches(1);
  }
}
template <typename T>
void launch_face_states(const Geo& g, const T* u, const T* p, const T* rho, const T* divtau, const Body* bodies,
                        const BodyView<T>* views, int nb, T* const slopes[9],
                        T* const wcell[9], T* const ubar[3][3], T* const vadv[3], T* const uf[3][3], cudaStream_t s) {
  BarPtrs bp;
  Slopes9 S, W;
  for (int q = 0; q < 9; q++) {
    S.s[q] = slopes[q];
    W.s[q] = wcell[q];
  }
  for (int e = 0; e < 3; e++) {
    for (int a = 0; a < 3; a++) bp.ub[e][a] = ubar[e][a];
    bp.vadv[e] = vadv[e];
  }
  const dim3 gc((g.n[0] + TILE_X - 1) / TILE_X, (g.n[1] + TILE_Y - 1) / TILE_Y, g.n[2]);
  k_cellw<T><<<gc, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, p, rho, divtau, bp, W, bodies, views, nb);
  rmt_count_launches(1);
  for (int d = 0; d < 3; d++) {
    for (int a = 0; a < 3; a++) bp.uf[a] = uf[d][a];
    const dim3 gr((g.n[0] + (d == 0) + TILE_X - 1) / TILE_X, (g.n[1] + (d == 1) + TILE_Y - 1) / TILE_Y, g.n[2] + (d == 2));
    auto kf = d == 0 ? k_face<T, 0> : (d == 1 ? k_face<T, 1> : k_face<T, 2>);
    kf<<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, S, W, bp);
    rmt_count_launches(1);
  }
}
template <typename T>
void launch_mac_setup(const Geo& g, T* const uf[3][3], MGVec b64, cudaStream_t s) {
  FacePtrs3 un;
  for (int d = 0; d < 3; d++) un.p[d] = uf[d][d];
  k_mac_rhs<T><<<nblocks(g.N), TPB, 0, s>>>(g, un, b64);
  rmt_count_launches(1);
}
template <typename T>
void launch_mac_correct(const Geo& g, T* const uf[3][3], const T* rho, MGVec q, T* const umac[3],
                        cudaStream_t s) {
  Umac3 F;
  for (int d = 0; d < 3; d++) {
    F.un[d] = uf[d][d];
    F.um[d] = umac[d];
  }
  const int zc = column_chunk(g.N, MCZ);
  const dim3 gr((g.n[0] + 1 + TILE_X - 1) / TILE_X, (g.n[1] + 1 + TILE_Y - 1) / TILE_Y, (g.n[2] + 1 + zc - 1) / zc);
  k_mac_correct3<T><<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, F, rho, q, zc);
  rmt_count_launches(1);
}
template <typename T>
void launch_advect(const Geo& g, T* const uf[3][3], T* const umac[3], T* adv, cudaStream_t s) {
  AdvPtrs ap;
  for (int d = 0; d < 3; d++) {
    ap.umac[d] = umac[d];
    for (int a = 0; a < 3; a++) ap.uf[d][a] = uf[d][a];
  }
  k_adv<T><<<nblocks(g.N), TPB, 0, s>>>(g, ap, adv); rmt_count_launches(1);
}
template <typename T>
void launch_density(const Geo& g, const Body* bodies, const BodyView<T>* views, int nb, const int* bbs, int bstride,
                    T* rho, cudaStream_t s) {
  const int zc = column_chunk(g.N, DZ);
  const dim3 gr((g.n[0] + TILE_X - 1) / TILE_X, (g.n[1] + TILE_Y - 1) / TILE_Y, (g.n[2] + zc - 1) / zc);
  k_density<T><<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, bodies, views, nb, bbs, bstride, rho, zc);
  rmt_count_launches(1);
}
template <typename T>
void launch_rep_field(const Geo& g, const Body* bodies, const BodyView<T>* views, int nb, double* out, cudaStream_t s) {
  k_rep_field<T><<<nblocks(g.N), TPB, 0, s>>>(g, bodies, views, nb, out);
  rmt_count_launches(1);
}
template <typename T>
void launch_ustar(const Geo& g, const T* u, const T* adv, const T* p, const T* rho_h, const T* divtau_h, T* ustar,
                  const Body* bodies, const BodyView<T>* views, int nb, cudaStream_t s) {
  k_ustar<T><<<nblocks(g.N), TPB, 0, s>>>(g, u, adv, p, rho_h, divtau_h, ustar, bodies, views, nb);
  rmt_count_launches(1);
}
template <typename T>
void launch_fe_setup(const Geo& g, const T* u, const T* ustar, MGVec b64, cudaStream_t s) {
  const int zc = column_chunk(g.NN, FEZ);
  const dim3 gr((g.nn[0] + TILE_X - 1) / TILE_X, (g.nn[1] + TILE_Y - 1) / TILE_Y, (g.nn[2] + zc - 1) / zc);
  k_fe_rhs<T><<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, ustar, b64, zc);
  rmt_count_launches(1);
}
template <typename T>
void launch_fe_update(const Geo& g, const T* ustar, const T* rho_h, MGVec psi, T* u, T* p, T* psi_out,
                      cudaStream_t s) {
  const int zc = column_chunk(g.N, FEZ);
  const dim3 gr((g.n[0] + TILE_X - 1) / TILE_X, (g.n[1] + TILE_Y - 1) / TILE_Y, (g.n[2] + zc - 1) / zc);
  k_fe_update_u<T><<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, ustar, rho_h, psi, u, zc); rmt_count_launches(1);
  k_fe_update_p<T><<<nblocks(g.NN), TPB, 0, s>>>(g.NN, psi, p, psi_out); rmt_count_launches(1);
}
template <typename T>
void launch_fill(T* a, T v, long n, cudaStream_t s) {
  k_fill<T><<<nblocks(n), TPB, 0, s>>>(a, v, n); rmt_count_launches(1);
}

#define INST(T)                                                                                                   \
  template void launch_bar_states<T>(const Geo&, const T*, T* const[9], T* const[3][3], T* const[3], cudaStream_t); \
  template void launch_face_states<T>(const Geo&, const T*, const T*, const T*, const T*, const Body*,          \
                                      const BodyView<T>*, int, T* const[9],                                   \
                                      T* const[9], T* const[3][3], T* const[3], T* const[3][3], cudaStream_t);   \
  template void launch_mac_setup<T>(const Geo&, T* const[3][3], MGVec, cudaStream_t);                            \
  template void launch_mac_correct<T>(const Geo&, T* const[3][3], const T*, MGVec, T* const[3],                 \
                                      cudaStream_t);                                                             \
  template void launch_advect<T>(const Geo&, T* const[3][3], T* const[3], T*, cudaStream_t);                      \
  template void launch_density<T>(const Geo&, const Body*, const BodyView<T>*, int, const int*, int, T*,        \
                                  cudaStream_t);                                                                \
  template void launch_ustar<T>(const Geo&, const T*, const T*, const T*, const T*, const T*, T*, const Body*,  \
                                const BodyView<T>*, int, cudaStream_t);                                       \
  template void launch_rep_field<T>(const Geo&, const Body*, const BodyView<T>*, int, double*, cudaStream_t);   \
  template void launch_fe_setup<T>(const Geo&, const T*, const T*, MGVec, cudaStream_t);                        \
  template void launch_fe_update<T>(const Geo&, const T*, const T*, MGVec, T*, T*, T*, cudaStream_t);          \
  template void launch_fill<T>(T*, T, long, cudaStream_t);

INST(float)
INST(double)
template void launch_fill<int8_t>(int8_t*, int8_t, long, cudaStream_t);
