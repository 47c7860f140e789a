// Geometric multigrid for the two projections of the RMT step (arXiv 2104.00095, SI
// "MAC projection" and "Approximate pressure-Poisson projection"; the paper solves both
// with its own multigrid library whose design it does not describe).
//
// kind 0 (MAC): cell-centred variable-coefficient 7-point operator
//     (A q)_c = h^-2 sum_faces beta_f (q_c - q_nb),  beta_f = 2/(rho_a + rho_b), 0 on walls.
// kind 1 (FE): nodal trilinear finite-element stiffness with beta_c = 1/rho_c per cell
//     (K psi)_i = (h/12) sum_{cells c at i} beta_c (4 psi_i - the 4 corners of c that differ
//     from i in two or three coordinates).
// Both are symmetric positive semi-definite with the constants as null space (walls are
// Neumann, periodic axes wrap); right-hand sides and solutions are kept mean-free.  The MAC
// operator reads the cell density rho (the caller's array on the finest level); the FE operator
// reads beta = 1/rho per cell, formed once per solve.  Coefficients are evaluated in the
// storage type; the FP64 residual only accumulates in FP64, so it needs no FP64 division.
//
// Solve = iterative refinement: the residual of a high-precision iterate is formed in high
// precision and V-cycles in the storage type T (double or float) compute the correction.  With
// T = double the iterate and its residual are FP64.  With T = float they are two-float numbers
// (hi + lo, about 48 significant bits; Knuth's two-sum and the FMA two-product), so the
// residual runs on the FP32 pipe: GB300 issues FP64 at 1/64 of the FP32 rate, and an FP64
// residual of the 27-point operator costs several times a V-cycle.  Smoothers:
// red-black Gauss-Seidel (7-point; one thread per same-colour cell pair along x) and weighted
// Jacobi (27-point; one fused pass per sweep).  Transfers: 8-cell average / trilinear
// (cell-centred), full weighting / trilinear (nodal).  Coarse densities are 8-cell means.
// The coarsest level is solved by one block with conjugate gradients.  Norms use fixed-order
// two-stage reductions, so results are deterministic.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "rmt_kernels.h"

namespace {

constexpr int TPB = 256;
constexpr int RED_BLOCKS = 1024;
// Level kernels run on blocks of BX x by threads: BX = one warp along x, by (1, 2, 4 or 8) a
// per-solver setting that the autotuner picks.
constexpr int BX = 32, BYMAX = 8;

inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > (long)sm_count() * 32) b = (long)sm_count() * 32;
  return (int)(b < 1 ? 1 : b);
}

struct Lv {
  int n[3], nn[3], per[3];
  long ncell, nnode, nunk;
  double h, ih2, s12;  // spacing, 1/h^2 (MAC), h/12 (FE)
  float f_ih2, f_s12;
  float f_ih2_lo, f_s12_lo;  // ih2 - f_ih2, s12 - f_s12: the two-float constants
};

inline dim3 grid3(int nx, int ny, int nz, int by) { return dim3((nx + BX - 1) / BX, (ny + by - 1) / by, nz); }

// 32-bit index arithmetic: every level is at most the finest grid, below 2^31 nodes
__device__ __forceinline__ long cix(const Lv& L, int i, int j, int k) { return (long)(i + L.n[0] * (j + L.n[1] * k)); }
__device__ __forceinline__ long nix(const Lv& L, int i, int j, int k) { return (long)(i + L.nn[0] * (j + L.nn[1] * k)); }
// neighbour cell index along d: wrap on periodic axes; -1 outside a wall
__device__ __forceinline__ int cnb(const Lv& L, int d, int v) {
  if (v < 0) return L.per[d] ? L.n[d] - 1 : -1;
  if (v >= L.n[d]) return L.per[d] ? 0 : -1;
  return v;
}
// neighbour node index along d: wrap on periodic axes; clamped on walls (its weight is 0 there)
__device__ __forceinline__ int nnb(const Lv& L, int d, int v) {
  if (v < 0) return L.per[d] ? L.nn[d] - 1 : 0;
  if (v >= L.nn[d]) return L.per[d] ? 0 : L.nn[d] - 1;
  return v;
}

// ----------------------------------------------------------------------------- operators
// approximate FP32 reciprocal: the hardware's reciprocal instruction alone (PTX rcp.approx.ftz)
__device__ __forceinline__ float rcp_approx(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}
// MAC face coefficient 2/(rho_a + rho_b) in the coefficient type; FAST: approximate reciprocal
// (smoothers and the V-cycle residual only)
template <bool FAST, typename CT>
__device__ __forceinline__ CT face_beta(CT ra, CT rb) {
  if constexpr (FAST && sizeof(CT) == 4) return 2.0f * rcp_approx(ra + rb);
  return CT(2) / (ra + rb);
}

// MAC at cell (i,j,k): returns (A x)_c (in AT) and its diagonal.  Rows away from the y and z
// boundaries share one path: the two x neighbours come from selects (periodic wrap, or a zero
// weight at a wall), so a warp whose row reaches i = 0 or n-1 does not diverge.
template <typename AT, bool FAST = false, typename XT, typename CT>
__device__ __forceinline__ AT mac_op(const Lv& L, const XT* __restrict__ x, const CT* __restrict__ rho, int i, int j,
                                     int k, AT& diag) {
  const long c = cix(L, i, j, k);
  const CT rc = rho[c];
  AT off = AT(0), dg = AT(0);
  if (j > 0 && j + 1 < L.n[1] && k > 0 && k + 1 < L.n[2]) {
    // 32-bit offsets from the cell (a level holds fewer than 2^31 cells); a missing x neighbour
    // reads the cell itself with weight 0
    const int sy = L.n[0], sz = L.n[0] * L.n[1];
    const bool lo = i > 0, hi = i + 1 < L.n[0];
    const bool hasl = lo || L.per[0], hash = hi || L.per[0];
    const int off6[6] = {lo ? -1 : (L.per[0] ? L.n[0] - 1 : 0), hi ? 1 : (L.per[0] ? 1 - L.n[0] : 0), -sy, sy, -sz, sz};
    const CT* rp = rho + c;
    const XT* xp = x + c;
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const bool has = f == 0 ? hasl : (f == 1 ? hash : true);
      const AT beta = has ? (AT)face_beta<FAST>(rc, rp[off6[f]]) : AT(0);
      off += beta * (AT)xp[off6[f]];
      dg += beta;
    }
    const AT ih2 = cv<AT>(L.ih2, L.f_ih2);
    diag = dg * ih2;
    return (dg * (AT)x[c] - off) * ih2;
  }
  const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const int d = f >> 1;
    const int v = cnb(L, d, nb[f][d]);
    if (v < 0) continue;
    int q[3] = {i, j, k};
    q[d] = v;
    const long cn = cix(L, q[0], q[1], q[2]);
    const AT beta = (AT)face_beta<FAST>(rc, rho[cn]);
    off += beta * (AT)x[cn];
    dg += beta;
  }
  const AT ih2 = cv<AT>(L.ih2, L.f_ih2);
  diag = dg * ih2;
  return (dg * (AT)x[c] - off) * ih2;
}

// FE at node (i,j,k): returns (K x)_i and its diagonal
template <typename AT, typename XT, typename CT>
__device__ __forceinline__ AT fe_op_interior(const Lv& L, const XT* __restrict__ x, const CT* __restrict__ beta, int i,
                                             int j, int k, AT& diag) {
  // node away from every boundary: its 8 cells and 26 neighbours at fixed offsets
  const long sx = 1, sy = L.nn[0], sz = (long)L.nn[0] * L.nn[1];
  const long cy = L.n[0], cz = (long)L.n[0] * L.n[1];
  const long c0 = cix(L, i - 1, j - 1, k - 1);
  AT b[2][2][2];
  AT bs = AT(0);
#pragma unroll
  for (int qz = 0; qz < 2; qz++)
#pragma unroll
    for (int qy = 0; qy < 2; qy++)
#pragma unroll
      for (int qx = 0; qx < 2; qx++) {
        b[qx][qy][qz] = (AT)beta[c0 + qx + qy * cy + qz * cz];
        bs += b[qx][qy][qz];
      }
  const long n0 = nix(L, i, j, k);
  AT s = AT(0);
#pragma unroll
  for (int qz = 0; qz < 2; qz++)
#pragma unroll
    for (int qy = 0; qy < 2; qy++)
#pragma unroll
      for (int qx = 0; qx < 2; qx++)
        s += b[qx][qy][qz] * (AT)x[n0 + (2 * qx - 1) * sx + (2 * qy - 1) * sy + (2 * qz - 1) * sz];
#pragma unroll
  for (int qy = 0; qy < 2; qy++)
#pragma unroll
    for (int qx = 0; qx < 2; qx++) s += (b[qx][qy][0] + b[qx][qy][1]) * (AT)x[n0 + (2 * qx - 1) * sx + (2 * qy - 1) * sy];
#pragma unroll
  for (int qz = 0; qz < 2; qz++)
#pragma unroll
    for (int qx = 0; qx < 2; qx++) s += (b[qx][0][qz] + b[qx][1][qz]) * (AT)x[n0 + (2 * qx - 1) * sx + (2 * qz - 1) * sz];
#pragma unroll
  for (int qz = 0; qz < 2; qz++)
#pragma unroll
    for (int qy = 0; qy < 2; qy++) s += (b[0][qy][qz] + b[1][qy][qz]) * (AT)x[n0 + (2 * qy - 1) * sy + (2 * qz - 1) * sz];
  const AT s12 = cv<AT>(L.s12, L.f_s12);
  diag = AT(4) * bs * s12;
  return (AT(4) * bs * (AT)x[n0] - s) * s12;
}

template <typename AT, typename XT, typename CT>
__device__ __forceinline__ AT fe_op(const Lv& L, const XT* __restrict__ x, const CT* __restrict__ beta, int i, int j,
                                    int k, AT& diag) {
  if (i > 0 && i + 1 < L.nn[0] && j > 0 && j + 1 < L.nn[1] && k > 0 && k + 1 < L.nn[2] && i <= L.n[0] &&
      j <= L.n[1] && k <= L.n[2])
    return fe_op_interior<AT>(L, x, beta, i, j, k, diag);
  AT b[2][2][2];
  AT bs = AT(0);
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++)
#pragma unroll
      for (int sx = 0; sx < 2; sx++) {
        const int ci = cnb(L, 0, i - 1 + sx), cj = cnb(L, 1, j - 1 + sy), ck = cnb(L, 2, k - 1 + sz);
        AT v = AT(0);
        if (ci >= 0 && cj >= 0 && ck >= 0) v = (AT)beta[cix(L, ci, cj, ck)];
        b[sx][sy][sz] = v;
        bs += v;
      }
  const int X[2] = {nnb(L, 0, i - 1), nnb(L, 0, i + 1)};
  const int Y[2] = {nnb(L, 1, j - 1), nnb(L, 1, j + 1)};
  const int Z[2] = {nnb(L, 2, k - 1), nnb(L, 2, k + 1)};
  AT s = AT(0);
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++)
#pragma unroll
      for (int sx = 0; sx < 2; sx++) s += b[sx][sy][sz] * (AT)x[nix(L, X[sx], Y[sy], Z[sz])];  // body diagonals
#pragma unroll
  for (int sy = 0; sy < 2; sy++)
#pragma unroll
    for (int sx = 0; sx < 2; sx++) s += (b[sx][sy][0] + b[sx][sy][1]) * (AT)x[nix(L, X[sx], Y[sy], k)];  // xy
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sx = 0; sx < 2; sx++) s += (b[sx][0][sz] + b[sx][1][sz]) * (AT)x[nix(L, X[sx], j, Z[sz])];  // xz
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++) s += (b[0][sy][sz] + b[1][sy][sz]) * (AT)x[nix(L, i, Y[sy], Z[sz])];  // yz
  const AT s12 = cv<AT>(L.s12, L.f_s12);
  diag = AT(4) * bs * s12;
  return (AT(4) * bs * (AT)x[nix(L, i, j, k)] - s) * s12;
}

// ----------------------------------------------------------------------------- two-float residual
// A two-float number is an unevaluated sum hi + lo of floats.  Every rounding step is spelled
// with an _rn intrinsic so that no multiply-add contraction can change it.
struct F2 {
  float h, l;
};
// Knuth's two-sum: s + e == a + b exactly
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// product of two two-float numbers (the FMA gives the rounding error of the leading product)
__device__ __forceinline__ F2 ff_mul(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  return two_sum(p, e);
}
// (sh, sl) += w (a - b) with a = ah + al, b = bh + bl and a float weight w: the difference of
// the leading parts is exact (two-sum), the product's leading rounding error is kept (FMA)
__device__ __forceinline__ void acc_wdiff(float w, float ah, float al, float bh, float bl, float& sh, float& sl) {
  const F2 d = two_sum(ah, -bh);
  const float dlo = __fadd_rn(d.l, __fsub_rn(al, bl));
  const float ph = __fmul_rn(w, d.h);
  const float pl = __fmaf_rn(w, dlo, __fmaf_rn(w, d.h, -ph));
  const F2 t = two_sum(sh, ph);
  sh = t.h;
  sl = __fadd_rn(sl, __fadd_rn(t.l, pl));
}

// (h, l) -= m, m a two-float pair (m[0] + m[1])
__device__ __forceinline__ void ff_sub_pair(float& h, float& l, const float* m) {
  const F2 t = two_sum(h, -m[0]);
  const F2 r = two_sum(t.h, __fadd_rn(t.l, __fsub_rn(l, m[1])));
  h = r.h;
  l = r.l;
}

// MAC operator on a two-float iterate: h^-2 sum_faces beta_f (x_c - x_nb), beta_f the same
// float coefficient the smoothers and the velocity correction use
__device__ __forceinline__ F2 mac_op_ff(const Lv& L, const float* __restrict__ xh, const float* __restrict__ xl,
                                        const float* __restrict__ rho, int i, int j, int k) {
  const long c = cix(L, i, j, k);
  const float rc = rho[c], ch = xh[c], cl = xl[c];
  float sh = 0.0f, sl = 0.0f;
  if (i > 0 && i + 1 < L.n[0] && j > 0 && j + 1 < L.n[1] && k > 0 && k + 1 < L.n[2]) {
    // interior: six neighbours at fixed offsets (2/(ra+rb) = 2 x the correctly rounded
    // reciprocal, the same float as the division)
    const int st[3] = {1, L.n[0], L.n[0] * L.n[1]};
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const long cn = c + ((f & 1) ? st[f >> 1] : -st[f >> 1]);
      acc_wdiff(2.0f * __frcp_rn(rc + rho[cn]), ch, cl, xh[cn], xl[cn], sh, sl);
    }
    return ff_mul(sh, sl, L.f_ih2, L.f_ih2_lo);
  }
  const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const int d = f >> 1;
    const int v = cnb(L, d, nb[f][d]);
    if (v < 0) continue;
    int q[3] = {i, j, k};
    q[d] = v;
    const long cn = cix(L, q[0], q[1], q[2]);
    acc_wdiff(2.0f * __frcp_rn(rc + rho[cn]), ch, cl, xh[cn], xl[cn], sh, sl);
  }
  return ff_mul(sh, sl, L.f_ih2, L.f_ih2_lo);
}

// FE operator on a two-float iterate: (h/12) sum_{cells c at the node} beta_c sum_{the 4 corners
// of c that differ from the node in two or three coordinates} (x_node - x_corner)
__device__ __forceinline__ F2 fe_op_ff(const Lv& L, const float* __restrict__ xh, const float* __restrict__ xl,
                                       const float* __restrict__ beta, int i, int j, int k) {
  if (i > 0 && i + 1 < L.nn[0] && j > 0 && j + 1 < L.nn[1] && k > 0 && k + 1 < L.nn[2] && i <= L.n[0] &&
      j <= L.n[1] && k <= L.n[2]) {
    // interior: the 8 cells and 26 neighbours at fixed offsets; a corner shared by two cells of
    // the node (the 12 face diagonals) takes the sum of their coefficients, so 20 weighted
    // differences instead of 32
    const int sx = 1, sy = L.nn[0], sz = L.nn[0] * L.nn[1];
    const int cy = L.n[0], cz = L.n[0] * L.n[1];
    const float* bp = beta + cix(L, i - 1, j - 1, k - 1);
    float b[2][2][2];
#pragma unroll
    for (int qz = 0; qz < 2; qz++)
#pragma unroll
      for (int qy = 0; qy < 2; qy++)
#pragma unroll
        for (int qx = 0; qx < 2; qx++) b[qx][qy][qz] = bp[qx + qy * cy + qz * cz];
    const long n0 = nix(L, i, j, k);
    const float* ph = xh + n0;
    const float* pl = xl + n0;
    const float ch = ph[0], cl = pl[0];
    float sh = 0.0f, sl = 0.0f;
#pragma unroll
    for (int qz = 0; qz < 2; qz++)
#pragma unroll
      for (int qy = 0; qy < 2; qy++)
#pragma unroll
        for (int qx = 0; qx < 2; qx++) {
          const int o = (2 * qx - 1) * sx + (2 * qy - 1) * sy + (2 * qz - 1) * sz;
          acc_wdiff(b[qx][qy][qz], ch, cl, ph[o], pl[o], sh, sl);  // body diagonals
        }
#pragma unroll
    for (int qy = 0; qy < 2; qy++)
#pragma unroll
      for (int qx = 0; qx < 2; qx++) {
        const int o = (2 * qx - 1) * sx + (2 * qy - 1) * sy;
        acc_wdiff(__fadd_rn(b[qx][qy][0], b[qx][qy][1]), ch, cl, ph[o], pl[o], sh, sl);  // xy
      }
#pragma unroll
    for (int qz = 0; qz < 2; qz++)
#pragma unroll
      for (int qx = 0; qx < 2; qx++) {
        const int o = (2 * qx - 1) * sx + (2 * qz - 1) * sz;
        acc_wdiff(__fadd_rn(b[qx][0][qz], b[qx][1][qz]), ch, cl, ph[o], pl[o], sh, sl);  // xz
      }
#pragma unroll
    for (int qz = 0; qz < 2; qz++)
#pragma unroll
      for (int qy = 0; qy < 2; qy++) {
        const int o = (2 * qy - 1) * sy + (2 * qz - 1) * sz;
        acc_wdiff(__fadd_rn(b[0][qy][qz], b[1][qy][qz]), ch, cl, ph[o], pl[o], sh, sl);  // yz
      }
    return ff_mul(sh, sl, L.f_s12, L.f_s12_lo);
  }
  const int X[2] = {nnb(L, 0, i - 1), nnb(L, 0, i + 1)};
  const int Y[2] = {nnb(L, 1, j - 1), nnb(L, 1, j + 1)};
  const int Z[2] = {nnb(L, 2, k - 1), nnb(L, 2, k + 1)};
  const long n0 = nix(L, i, j, k);
  const float ch = xh[n0], cl = xl[n0];
  float sh = 0.0f, sl = 0.0f;
#pragma unroll
  for (int sz = 0; sz < 2; sz++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++)
#pragma unroll
      for (int sx = 0; sx < 2; sx++) {
        const int ci = cnb(L, 0, i - 1 + sx), cj = cnb(L, 1, j - 1 + sy), ck = cnb(L, 2, k - 1 + sz);
        if (ci < 0 || cj < 0 || ck < 0) continue;
        const float bc = beta[cix(L, ci, cj, ck)];
        const long q[4] = {nix(L, X[sx], Y[sy], Z[sz]), nix(L, X[sx], Y[sy], k), nix(L, X[sx], j, Z[sz]),
                           nix(L, i, Y[sy], Z[sz])};
#pragma unroll
        for (int t = 0; t < 4; t++) acc_wdiff(bc, ch, cl, xh[q[t]], xl[q[t]], sh, sl);
      }
  return ff_mul(sh, sl, L.f_s12, L.f_s12_lo);
}

// ----------------------------------------------------------------------------- kernels
template <typename T>
__global__ void k_zero(T* a, long n) {
  GRID_LOOP(i, n) a[i] = T(0);
}

__device__ __forceinline__ bool thread_cell(const int ext[3], int& i, int& j, int& k) {
  i = blockIdx.x * BX + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  k = blockIdx.z;
  return i < ext[0] && j < ext[1];
}

__device__ __forceinline__ void block_partial(double loc, double* part) {
  __shared__ double sh[BX * BYMAX / 32];
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) sh[t >> 5] = loc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)blockDim.y; w++) s += sh[w];
    part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
  }
}

// FP64 residual r = b - A x of the FP64 iterate (T = double); writes r for the V-cycle and
// per-block partial sums of r^2
__global__ void __launch_bounds__(BX* BYMAX) k_resid64(Lv L, int kind, const double* __restrict__ x,
                                                     const double* __restrict__ b, const double* __restrict__ rho,
                                                     double* __restrict__ rT, double* __restrict__ part) {
  const int ext[3] = {kind == 0 ? L.n[0] : L.nn[0], kind == 0 ? L.n[1] : L.nn[1], kind == 0 ? L.n[2] : L.nn[2]};
  int i, j, k;
  double loc = 0.0;
  if (thread_cell(ext, i, j, k)) {
    double dg;
    const double ax = kind == 0 ? mac_op<double>(L, x, rho, i, j, k, dg) : fe_op<double>(L, x, rho, i, j, k, dg);
    const long u = (long)(i + ext[0] * (j + ext[1] * k));
    const double r = b[u] - ax;
    rT[u] = r;
    loc = r * r;
  }
  block_partial(loc, part);
}

// per-block partial sum of a float per thread: warp sums in float, block sum in FP64
__device__ __forceinline__ void block_partial_f(float loc, double* part) {
  __shared__ double sh[BX * BYMAX / 32];
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) sh[t >> 5] = (double)loc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)blockDim.y; w++) s += sh[w];
    part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
  }
}

// first residual of the zero iterate, r = b (FP64 mode): removes the mean (*mean) from b, writes
// r and per-block partial sums of r^2
__global__ void __launch_bounds__(BX* BYMAX) k_first_resid64(Lv L, int kind, double* __restrict__ b,
                                                           const double* __restrict__ mean, double* __restrict__ rT,
                                                           double* __restrict__ part) {
  const int ext[3] = {kind == 0 ? L.n[0] : L.nn[0], kind == 0 ? L.n[1] : L.nn[1], kind == 0 ? L.n[2] : L.nn[2]};
  int i, j, k;
  double loc = 0.0;
  if (thread_cell(ext, i, j, k)) {
    const long u = (long)(i + ext[0] * (j + ext[1] * k));
    const double v = b[u] - *mean;
    b[u] = v;
    rT[u] = v;
    loc = v * v;
  }
  block_partial(loc, part);
}

// the same for the two-float right-hand side (FP32 mode; mean given as a two-float pair).
// once: the solve is a single pass from zero (fixed cycles, no later residual), so the
// mean-free right-hand side is not stored back, no norm is needed, and the storage-precision
// iterate x is zeroed here instead of by a separate launch.
__global__ void __launch_bounds__(BX* BYMAX) k_first_resid_ff(Lv L, int kind, float* __restrict__ bh,
                                                            float* __restrict__ bl, const float* __restrict__ mean,
                                                            float* __restrict__ rT, double* __restrict__ part,
                                                            int once, float* __restrict__ x) {
  const int ext[3] = {kind == 0 ? L.n[0] : L.nn[0], kind == 0 ? L.n[1] : L.nn[1], kind == 0 ? L.n[2] : L.nn[2]};
  int i, j, k;
  float loc = 0.0f;
  if (thread_cell(ext, i, j, k)) {
    const long u = (long)(i + ext[0] * (j + ext[1] * k));
    float h = bh[u], l = bl[u];
    ff_sub_pair(h, l, mean);
    const float r = __fadd_rn(h, l);
    rT[u] = r;
    if (once) {
      x[u] = 0.0f;
    } else {
      bh[u] = h;
      bl[u] = l;
      loc = r * r;
    }
  }
  if (!once) block_partial_f(loc, part);
}

// residual r = b - A x of the two-float iterate (xh + xl) against the two-float right-hand
// side (bh + bl); writes the float r for the V-cycle and per-block partial sums of r^2
__global__ void __launch_bounds__(BX* BYMAX) k_resid_ff(Lv L, int kind, const float* __restrict__ xh,
                                                      const float* __restrict__ xl, const float* __restrict__ bh,
                                                      const float* __restrict__ bl, const float* __restrict__ rho,
                                                      float* __restrict__ rT, double* __restrict__ part) {
  const int ext[3] = {kind == 0 ? L.n[0] : L.nn[0], kind == 0 ? L.n[1] : L.nn[1], kind == 0 ? L.n[2] : L.nn[2]};
  int i, j, k;
  float loc = 0.0f;
  if (thread_cell(ext, i, j, k)) {
    const F2 ax = kind == 0 ? mac_op_ff(L, xh, xl, rho, i, j, k) : fe_op_ff(L, xh, xl, rho, i, j, k);
    const long u = (long)(i + ext[0] * (j + ext[1] * k));
    const F2 t = two_sum(bh[u], -ax.h);
    const float r = __fadd_rn(t.h, __fadd_rn(t.l, __fsub_rn(bl[u], ax.l)));
    rT[u] = r;
    loc = r * r;
  }
  block_partial_f(loc, part);
}

// two-float iterate update (xh + xl) += e; set: (xh, xl) = (e, 0)
__global__ void k_add_ff(const float* __restrict__ e, float* __restrict__ xh, float* __restrict__ xl, long n,
                         int set) {
  GRID_LOOP(i, n) {
    if (set) {
      xh[i] = e[i];
      xl[i] = 0.0f;
    } else {
      const F2 s = two_sum(xh[i], e[i]);
      const F2 r = two_sum(s.h, __fadd_rn(s.l, xl[i]));
      xh[i] = r.h;
      xl[i] = r.l;
    }
  }
}

// FP64 value of a two-float array (read-back only)
__global__ void k_ff_to64(const float* __restrict__ xh, const float* __restrict__ xl, double* __restrict__ x, long n) {
  GRID_LOOP(i, n) x[i] = (double)xh[i] + (double)xl[i];
}

// red-black Gauss-Seidel update (7-point) of the cell of this colour among x = 2p and 2p+1 of
// row (j, k); the increment scales the residual, so an approximate FP32 quotient moves the sweep,
// not its fixed point
template <typename T>
__device__ __forceinline__ void rbgs_at(const Lv& L, int colour, T w, T* __restrict__ x, const T* __restrict__ b,
                                        const T* __restrict__ rho, int p, int j, int k) {
  const int i = 2 * p + ((j + k + colour) & 1);
  if (i >= L.n[0]) return;
  T dg;
  const T ax = mac_op<T, true>(L, x, rho, i, j, k, dg);
  const long c = cix(L, i, j, k);
  if (dg > T(0)) {
    if constexpr (sizeof(T) == 4) x[c] = x[c] + w * ((b[c] - ax) * rcp_approx(dg));
    else x[c] = x[c] + w * ((b[c] - ax) / dg);
  }
}
// one colour pass: one thread per cell pair along x
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_rbgs(Lv L, int colour, T w, T* __restrict__ x, const T* __restrict__ b,
                                                  const T* __restrict__ rho) {
  const int p = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= L.n[1]) return;
  rbgs_at(L, colour, w, x, b, rho, p, j, (int)blockIdx.z);
}

// weighted Jacobi sweep of the 7-point operator, out of place (x -> xo): the smoother of MAC
// levels with an odd periodic side, where a red-black colouring is not consistent across the wrap
// (two neighbours of one colour would update in the same pass)
constexpr double MAC_JACOBI_W = 6.0 / 7.0;
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_jacobi_mac(Lv L, T w, const T* __restrict__ x, T* __restrict__ xo,
                                                        const T* __restrict__ b, const T* __restrict__ rho) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  T dg;
  const T ax = mac_op<T, true>(L, x, rho, i, j, k, dg);
  const long c = cix(L, i, j, k);
  T v = x[c];
  if (dg > T(0)) {
    if constexpr (sizeof(T) == 4) v = v + w * ((b[c] - ax) * rcp_approx(dg));
    else v = v + w * ((b[c] - ax) / dg);
  }
  xo[c] = v;
}

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes; size 0 fills zeros), so that
// several planes of a stencil tile are in flight while one is computed.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Full red-black sweep in one pass (FP32): both colours of a Gauss-Seidel sweep, out of place
// (x_in -> x_out), marching up a z-chunk of a GX x GY tile.  At plane q the block updates the
// first colour c0 on the tile and a one-cell ring around it (from x_in only), then the second
// colour on the tile at plane q-1 (from the new c0 values of planes q-2..q, kept in shared
// memory).  The ring is recomputed by the neighbouring block with the same arithmetic, so no
// block reads another block's output, and each value equals that of two in-place colour
// passes.  Per sweep, x, rho and b are read once and x written once (4 words per cell instead of
// 6 for two colour passes).  Planes of x, rho and b (with a halo of 4 cells along x, for 16-byte
// cp.async rows, and 2 rows along y) arrive through a ring of GR slots two planes ahead of use.
// The second colour's cell at plane q-1 is the cell of the thread's first colour at plane q (the
// colour alternates along z), so that update's own values stay in registers.  Warps cover 16 cell pairs of two adjacent rows: the cells of one colour then fall in opposite
// bank parities in the two half-warps, so the stencil's shared-memory reads are conflict-free.
// Cells outside a wall are staged as x = 0, rho = 0, and a face whose far density is 0 gets
// coefficient 0 (the wall's Neumann condition).  Requires n_x % 4 == 0 and even periodic sides.
constexpr int GX = 64, GY = 8;           // tile: cells along x, rows along y
constexpr int GW = GX + 8, GH = GY + 4;  // staged plane: 4 halo cells each side along x, 2 rows along y
constexpr int GP = GW * GH;              // floats per staged plane
constexpr int GR = 6;                    // ring slots per staged array (planes q-2 .. q+3)
constexpr int GCH = GW / 4;              // 16-byte chunks per staged row
constexpr int GNCH = 3 * GH * GCH;       // chunks per plane over x, rho and b
constexpr int GT = 256;                  // threads per block
constexpr size_t SWEEP_SMEM = (size_t)(3 * GR + 3) * GP * sizeof(float);
static_assert((GX / 2) * GY == GT, "one thread per cell pair of the tile");
static_assert(GW % 4 == 0 && GNCH <= 3 * GT, "staging layout");

// wrapped index along an axis of n cells (periodic), or -1 outside a wall
__device__ __forceinline__ int sweep_wrap(int v, int n, int per) {
  if (per) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return (v >= 0 && v < n) ? v : -1;
}

// Gauss-Seidel update of one cell: rc, xc, bc its rho, x and b; rn, xn the rho and x of its six
// face neighbours (-x, +x, -y, +y, -z, +z).  The face coefficient 2/(rho_c + rho_n) is carried as
// r = 1/(rho_c + rho_n) with the 2 moved into ih2x2 = 2/h^2 (a power-of-two scaling, so every
// rounding is that of the colour-pass kernel); WALLS: a staged rho of 0 (outside a wall) gives
// the face weight 0.
template <bool WALLS>
__device__ __forceinline__ float sweep_update(float rc, const float (&rn)[6], const float (&xn)[6], float xc, float bc,
                                              float ih2x2, float w) {
  float off = 0.f, dg = 0.f;
#pragma unroll
  for (int f = 0; f < 6; f++) {
    float r = rcp_approx(rc + rn[f]);
    if constexpr (WALLS) r = rn[f] > 0.f ? r : 0.f;
    off += r * xn[f];
    dg += r;
  }
  const float ax = (dg * xc - off) * ih2x2;
  const float diag = dg * ih2x2;
  return diag > 0.f ? xc + w * ((bc - ax) * rcp_approx(diag)) : xc;
}

template <bool WALLS>
__global__ void __launch_bounds__(GT, 3) k_rbgs_sweep(Lv L, int c0, float w, const float* __restrict__ xin,
                                                      float* __restrict__ xout, const float* __restrict__ b,
                                                      const float* __restrict__ rho, int zc) {
  extern __shared__ float4 sweep_sm4[];
  float* const sm = reinterpret_cast<float*>(sweep_sm4);  // all shared reads index this base
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int i0 = blockIdx.x * GX, j0 = blockIdx.y * GY;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, nz);
  const long pst = (long)nx * ny;
  const float ih2x2 = 2.0f * L.f_ih2;
  const int perx = L.per[0], pery = L.per[1], perz = L.per[2];
  // staging: this thread's chunks (up to 3 of the GNCH per plane): shared address in slot 0, and
  // the source row in plane 0 (null outside a wall)
  const unsigned sm_base = (unsigned)__cvta_generic_to_shared(sm);
  const float* c_src[3];
  unsigned c_sa[3];
  bool c_on[3];
#pragma unroll
  for (int s = 0; s < 3; s++) {
    const int c = t + GT * s;
    c_src[s] = nullptr;
    c_sa[s] = 0;
    c_on[s] = c < GNCH;
    if (c < GNCH) {
      const int a = c / (GH * GCH), rc = c % (GH * GCH), r = rc / GCH, cc = rc % GCH;
      const int gy = sweep_wrap(j0 - 2 + r, ny, pery);
      const int gx = sweep_wrap(i0 - 4 + 4 * cc, nx, perx);
      const float* base = a == 0 ? xin : (a == 1 ? rho : b);
      c_sa[s] = sm_base + 4u * (unsigned)(a * GR * GP + r * GW + 4 * cc);
      if (gy >= 0 && gx >= 0) c_src[s] = base + (long)gy * nx + gx;
    }
  }
  // plane p of the staged arrays sits in ring slot (p - k0 + 2) % GR, its RED plane in slot
  // (p - k0 + 3) % 3; the loop keeps both for plane q and derives the others by one add
  auto adv = [](int s, int d, int m) { return s + d >= m ? s + d - m : s + d; };
  auto issue = [&](int p, int slot) {
    // p lies in [k0-2, k1+1], within two planes of the grid
    const int pz = p < 0 ? (perz ? p + nz : -1) : (p >= nz ? (perz ? p - nz : -1) : p);
#pragma unroll
    for (int s = 0; s < 3; s++) {
      if (!c_on[s]) continue;
      const bool ok = pz >= 0 && c_src[s] != nullptr;
      const float* g = ok ? c_src[s] + (long)pz * pst : xin;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(c_sa[s] + 4u * (unsigned)(slot * GP)),
                   "l"(g), "r"(ok ? 16 : 0));
    }
  };
  // the thread's cell pair of the tile: 16 pairs of two adjacent rows per warp
  const int pp = 16 * (wp & 1) + (lane & 15), jj = 2 * (wp >> 1) + (lane >> 4);
  // its ring pair (first 80 threads): rows -1 and GY across pairs 0..31, then pairs -1 and 32
  // for rows 0..GY-1 (the corners are not needed)
  constexpr int NRING = GX + 2 * GY;
  int hp = 0, hj = 0;
  const bool has_ring = t < NRING;
  if (t < GX) {
    hp = 16 * (t >> 5) + (t & 15);
    hj = (t & 16) ? GY : -1;
  } else if (has_ring) {
    const int r = t - GX;
    hp = r < GY ? -1 : GX / 2;
    hj = r < GY ? r : r - GY;
  }
  const bool tile_row = j0 + jj < ny;  // the thread's tile row lies in the grid
  const int orow = (jj + 2) * GW + 4, hrow = (hj + 2) * GW + 4;
  // prologue: planes k0-2 .. k0 in one group, k0+1 in the next
  issue(k0 - 2, 0);
  issue(k0 - 1, 1);
  issue(k0, 2);
  cp_async_commit();
  issue(k0 + 1, 3);
  cp_async_commit();
  int sq = 1, rq = 2;  // slots of plane q = k0-1
  for (int q = k0 - 1; q <= k1; q++, sq = adv(sq, 1, GR), rq = adv(rq, 1, 3)) {
    cp_async_wait<1>();  // plane q+1 has landed (q+2 may still fly)
    __syncthreads();     // ... for every thread; slot of plane q-3 and RED of q-2's store are free
    if (q + 3 <= k1 + 1) issue(q + 3, adv(sq, 3, GR));
    cp_async_commit();
    const int sm1 = adv(sq, GR - 1, GR), sm2 = adv(sq, GR - 2, GR), sp1 = adv(sq, 1, GR);
    // plane bases (float offsets into sm): x, rho, b of planes q-2..q+1; RED of q-2..q
    const int X0 = sq * GP, Xm1 = sm1 * GP, Xp1 = sp1 * GP;
    const int R0 = (GR + sq) * GP, Rm1 = (GR + sm1) * GP, Rm2 = (GR + sm2) * GP, Rp1 = (GR + sp1) * GP;
    const int B0 = (2 * GR + sq) * GP, Bm1 = (2 * GR + sm1) * GP;
    const int N0 = (3 * GR + rq) * GP, Nm1 = (3 * GR + adv(rq, 2, 3)) * GP, Nm2 = (3 * GR + adv(rq, 1, 3)) * GP;
    // plane q-2's tile (both colours) to x_out: one 16-byte store per thread
    if (q - 2 >= k0 && t < GX * GY / 4) {
      const int r = t / (GX / 4), cc = t % (GX / 4);
      const int gj = j0 + r, gi = i0 + 4 * cc;
      if (gj < ny && gi < nx) {
        const float4 v = *reinterpret_cast<const float4*>(sm + Nm2 + (r + 2) * GW + 4 + 4 * cc);
        *reinterpret_cast<float4*>(xout + (long)(q - 2) * pst + (long)gj * nx + gi) = v;
      }
    }
    const bool zin = !WALLS || perz || (q >= 0 && q < nz);
    // first colour at plane q: the thread's tile pair (its cell o is also the second colour's
    // cell at plane q-1, so the values below are reused there)
    const int e = (c0 + j0 + jj + q) & 1;
    const int o = orow + 2 * pp + e;
    const float rc = sm[R0 + o], rlo = sm[Rm1 + o], xlo = sm[Xm1 + o];
    float vq;
    {
      const float rn[6] = {sm[R0 + o - 1], sm[R0 + o + 1], sm[R0 + o - GW], sm[R0 + o + GW], rlo, sm[Rp1 + o]};
      const float xn[6] = {sm[X0 + o - 1], sm[X0 + o + 1], sm[X0 + o - GW], sm[X0 + o + GW], xlo, sm[Xp1 + o]};
      vq = sweep_update<WALLS>(rc, rn, xn, sm[X0 + o], sm[B0 + o], ih2x2, w);
      if constexpr (WALLS) {
        const bool real = zin && (pery || tile_row) && (perx || (unsigned)(i0 + o - orow) < (unsigned)nx);
        vq = real ? vq : 0.f;
      }
      sm[N0 + o] = vq;
    }
    if (has_ring) {
      const int eh = (c0 + j0 + hj + q) & 1;
      const int oh = hrow + 2 * hp + eh;
      const float rn[6] = {sm[R0 + oh - 1], sm[R0 + oh + 1], sm[R0 + oh - GW], sm[R0 + oh + GW], sm[Rm1 + oh],
                           sm[Rp1 + oh]};
      const float xn[6] = {sm[X0 + oh - 1], sm[X0 + oh + 1], sm[X0 + oh - GW], sm[X0 + oh + GW], sm[Xm1 + oh],
                           sm[Xp1 + oh]};
      float v = sweep_update<WALLS>(sm[R0 + oh], rn, xn, sm[X0 + oh], sm[B0 + oh], ih2x2, w);
      if constexpr (WALLS) {
        const bool real = zin && (pery || (unsigned)(j0 + hj) < (unsigned)ny) &&
                          (perx || (unsigned)(i0 + oh - hrow) < (unsigned)nx);
        v = real ? v : 0.f;
      }
      sm[N0 + oh] = v;
    }
    __syncthreads();
    // second colour on the tile at plane q-1, cell o (RED planes q-2..q hold the new first colour)
    if (q - 1 >= k0 && tile_row && i0 + o - orow < nx) {
      const float rn[6] = {sm[Rm1 + o - 1], sm[Rm1 + o + 1], sm[Rm1 + o - GW], sm[Rm1 + o + GW], sm[Rm2 + o], rc};
      const float xn[6] = {sm[Nm1 + o - 1], sm[Nm1 + o + 1], sm[Nm1 + o - GW], sm[Nm1 + o + GW], sm[Nm2 + o], vq};
      sm[Nm1 + o] = sweep_update<WALLS>(rlo, rn, xn, xlo, sm[Bm1 + o], ih2x2, w);
    }
  }
  // plane k1-1's tile (the last iteration's second colour)
  cp_async_wait<0>();
  __syncthreads();
  if (k1 - 1 >= k0 && t < GX * GY / 4) {
    const int Nl = (3 * GR + adv(rq, 1, 3)) * GP;  // rq is now the slot of k1+1
    const int r = t / (GX / 4), cc = t % (GX / 4);
    const int gj = j0 + r, gi = i0 + 4 * cc;
    if (gj < ny && gi < nx) {
      const float4 v = *reinterpret_cast<const float4*>(sm + Nl + (r + 2) * GW + 4 + 4 * cc);
      *reinterpret_cast<float4*>(xout + (long)(k1 - 1) * pst + (long)gj * nx + gi) = v;
    }
  }
}

// 27-point FE sweeps on a plane-marching tile: a block owns FX x FY nodes of every plane of a
// z-chunk (FZ planes, fewer on small levels; the grid's z extent sets it) and keeps a ring of
// RING planes of x and of beta (with a one-point halo) in shared memory, and each thread a
// register window of its column (below); the next planes arrive by cp.async while one is
// computed.
// Each value is read from global memory about once instead of up to 27 times.  Cells outside a
// wall carry beta = 0, which makes the stencil uniform (the clamped x of an outside node always
// meets a zero weight).  MODE 0: weighted Jacobi, out = x + w (b - K x) / diag (x where
// diag = 0); MODE 1: residual, out = b - K x.
// VEC (FP32, periodic x with n_x % 4 == 0): planes arrive as 16-byte rows, one copy per thread
// per plane (x rows widened to 4 halo nodes on each side, beta rows to 4 halo cells on the left)
// instead of one 4-byte copy per element.
constexpr int FX = 32, FY = 8, FZ = 32, RING = 5;
constexpr int XH = (FX + 2) * (FY + 2) - FX * FY;  // halo nodes of an x plane (84)
constexpr int BH = (FX + 1) * (FY + 1) - FX * FY;  // halo cells of a beta plane (41)
constexpr int VXC = (FX + 8) / 4, VBC = (FX + 4) / 4, VRC = FX / 4;  // 16-byte chunks per staged row (VEC)
constexpr int VNX = (FY + 2) * VXC, VNR = FY * VRC, VNB = (FY + 1) * VBC;  // chunks per plane (VEC)
static_assert(VNX + VNR + VNB <= FX * FY, "one staged chunk per thread and plane");
template <typename T, int MODE, bool VEC = false>
__global__ void __launch_bounds__(FX* FY) k_fe_tile(Lv L, T w, const T* __restrict__ x, T* __restrict__ out,
                                                    const T* __restrict__ b, const T* __restrict__ beta) {
  static_assert(!VEC || sizeof(T) == 4, "16-byte rows of floats");
  constexpr int XW = VEC ? FX + 8 : FX + 2, BW = VEC ? FX + 4 : FX + 1;  // staged row lengths
  constexpr int XO = VEC ? 3 : 0, BO = VEC ? 3 : 0;  // column of node i0-1 / cell i0-1
  __shared__ __align__(16) T xs[RING][FY + 2][XW];
  __shared__ __align__(16) T bs[RING][FY + 1][BW];
  __shared__ __align__(16) T rs[RING][FY][FX];  // right-hand side b of the tile's nodes
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * FX + tx;
  const int i0 = blockIdx.x * FX, j0 = blockIdx.y * FY;
  const int fz = (L.nn[2] + (int)gridDim.z - 1) / (int)gridDim.z;  // planes per block (FZ, or fewer on small levels)
  const int k0 = blockIdx.z * fz, k1 = min(k0 + fz, L.nn[2]);
  const long sy = L.nn[0], sz = (long)L.nn[0] * L.nn[1];
  const long cy = L.n[0], cz = (long)L.n[0] * L.n[1];
  // this thread's elements of a plane: its own node (tx+1, ty+1) and, for the first XH threads,
  // one halo node; likewise its own cell (i0+tx, j0+ty) and one halo cell for the first BH
  int hxa = 0, hxc = 0, hba = 0, hbc = 0;
  if (t < XH) {
    // halo ring of the (FX+2) x (FY+2) plane: row 0, row FY+1, then columns 0 and FX+1
    if (t < FX + 2) {
      hxa = t;
      hxc = 0;
    } else if (t < 2 * (FX + 2)) {
      hxa = t - (FX + 2);
      hxc = FY + 1;
    } else {
      const int r = t - 2 * (FX + 2);
      hxa = (r & 1) ? FX + 1 : 0;
      hxc = 1 + (r >> 1);
    }
  }
  if (t < BH) {
    // row 0 of the (FX+1) x (FY+1) cell plane, then column 0
    if (t < FX + 1) {
      hba = t;
      hbc = 0;
    } else {
      hba = 0;
      hbc = t - FX;
    }
  }
  const long xo_own = nnb(L, 0, i0 + tx) + nnb(L, 1, j0 + ty) * sy;
  const long xo_halo = nnb(L, 0, i0 - 1 + hxa) + nnb(L, 1, j0 - 1 + hxc) * sy;
  const int ci_own = cnb(L, 0, i0 + tx), cj_own = cnb(L, 1, j0 + ty);
  const int ci_halo = cnb(L, 0, i0 - 1 + hba), cj_halo = cnb(L, 1, j0 - 1 + hbc);
  const bool b_own_ok = ci_own >= 0 && cj_own >= 0, b_halo_ok = ci_halo >= 0 && cj_halo >= 0;
  const long bo_own = b_own_ok ? ci_own + cj_own * cy : 0, bo_halo = b_halo_ok ? ci_halo + cj_halo * cy : 0;
  // VEC: this thread's chunk of a plane (kind 0: an x row chunk, 1: a b row chunk, 2: a beta row
  // chunk, -1: none), its in-plane source offset and its shared slot-0 address
  int vk = -1;
  long voff = 0;
  bool vok = true;
  T* vdst = nullptr;
  size_t vslot = 0;  // elements between ring slots of the chunk's array
  if constexpr (VEC) {
    const int nx0 = L.n[0];  // = nn[0] on a periodic x axis
    auto wx = [&](int v) { return ((v % nx0) + nx0) % nx0; };
    if (t < VNX) {
      const int r = t / VXC, cc = t % VXC;
      vk = 0;
      voff = nnb(L, 1, j0 - 1 + r) * sy + wx(i0 - 4 + 4 * cc);
      vdst = &xs[0][r][4 * cc];
      vslot = (size_t)(FY + 2) * XW;
    } else if (t < VNX + VNR) {
      const int u = t - VNX, r = u / VRC, cc = u % VRC;
      vk = 1;
      voff = (long)min(j0 + r, L.nn[1] - 1) * sy + wx(i0 + 4 * cc);
      vdst = &rs[0][r][4 * cc];
      vslot = (size_t)FY * FX;
    } else if (t < VNX + VNR + VNB) {
      const int u = t - VNX - VNR, r = u / VBC, cc = u % VBC;
      const int cyv = cnb(L, 1, j0 - 1 + r);
      vk = 2;
      vok = cyv >= 0;
      voff = vok ? (long)cyv * cy + wx(i0 - 4 + 4 * cc) : 0;
      vdst = &bs[0][r][4 * cc];
      vslot = (size_t)(FY + 1) * BW;
    }
  }
  auto cp16 = [&](T* dst, const T* src, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 16 : 0));
  };
  // x plane p lives in ring slot (p - k0 + 1) % RING, beta cell plane c in (c - k0 + 1) % RING
  auto issue_x = [&](int p) {  // x plane p with its halo, and b of the tile's nodes on it
    const int slot = (p - k0 + 1 + RING) % RING;
    const long base = nnb(L, 2, p) * sz;
    if constexpr (VEC) {
      if (vk == 0 || vk == 1) cp16(vdst + slot * vslot, (vk == 0 ? x : b) + base + voff, true);
    } else {
      cp_async_elem(&xs[slot][ty + 1][tx + 1], x + xo_own + base, true);
      if (t < XH) cp_async_elem(&xs[slot][hxc][hxa], x + xo_halo + base, true);
      cp_async_elem(&rs[slot][ty][tx], b + xo_own + base, true);
    }
  };
  auto issue_b = [&](int c) {
    const int slot = (c - k0 + 1 + RING) % RING;
    const int ck = cnb(L, 2, c);
    const long base = ck >= 0 ? ck * cz : 0;
    if constexpr (VEC) {
      if (vk == 2) cp16(vdst + slot * vslot, beta + base + voff, vok && ck >= 0);
    } else {
      cp_async_elem(&bs[slot][ty + 1][tx + 1], beta + bo_own + base, b_own_ok && ck >= 0);
      if (t < BH) cp_async_elem(&bs[slot][hbc][hba], beta + bo_halo + base, b_halo_ok && ck >= 0);
    }
  };
  // group 0: x planes k0-1 .. k0+1, cell planes k0-1, k0; then one group per further plane
  issue_x(k0 - 1);
  issue_x(k0);
  issue_x(k0 + 1);
  issue_b(k0 - 1);
  issue_b(k0);
  cp_async_commit();
  issue_x(k0 + 2);
  issue_b(k0 + 1);
  cp_async_commit();
  issue_x(k0 + 3);
  issue_b(k0 + 2);
  cp_async_commit();
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < L.nn[0] && j < L.nn[1];
  const T s12 = cv<T>(L.s12, L.f_s12);
  // Register window of the thread's column: three x planes (i-1..i+1, j-1..j+1) and two beta
  // cell planes (the cells around the node below / above it).  The window moves up one plane
  // per iteration by reading only the new plane from shared memory (shared-memory bandwidth,
  // not DRAM, is the next limit of this kernel); the loop is unrolled so that the arrays change
  // roles instead of being copied.
  T Xa[3][3], Xb[3][3], Xc[3][3], Ba[2][2], Bb[2][2];
  auto rd_x = [&](T (&P)[3][3], int slot) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int a = 0; a < 3; a++) P[c][a] = xs[slot][ty + c][tx + XO + a];
  };
  auto rd_b = [&](T (&P)[2][2], int slot) {
#pragma unroll
    for (int c = 0; c < 2; c++)
#pragma unroll
      for (int a = 0; a < 2; a++) P[c][a] = bs[slot][ty + c][tx + BO + a];
  };
  const long ubase = (long)i + (long)j * sy;
  int k = k0;
  int sxp = 2, sbc = 1;  // ring slots of x plane k+1 and of cell plane k
  // one plane: M, C, P = x planes k-1, k, k+1 (P is filled here), Bl, Bu = cell planes k-1, k
  // (Bu is filled here)
  auto plane = [&](T (&M)[3][3], T (&C)[3][3], T (&P)[3][3], T (&Bl)[2][2], T (&Bu)[2][2]) {
    cp_async_wait<2>();  // x plane k+1 and cell plane k have landed (two newer groups may fly)
    __syncthreads();     // ... for every thread; the slots refilled below were last read at
                         // least one iteration ago, before this barrier
    rd_x(P, sxp);
    rd_b(Bu, sbc);
    const T bcur = rs[sxp == 0 ? RING - 1 : sxp - 1][ty][tx];  // b of plane k (slot before k+1)
    issue_x(k + 4);
    issue_b(k + 3);
    cp_async_commit();
    sxp = sxp + 1 == RING ? 0 : sxp + 1;
    sbc = sbc + 1 == RING ? 0 : sbc + 1;
    if (own) {
      const T bsum = (Bl[0][0] + Bl[0][1]) + (Bl[1][0] + Bl[1][1]) + ((Bu[0][0] + Bu[0][1]) + (Bu[1][0] + Bu[1][1]));
      T acc = T(0);
#pragma unroll
      for (int qy = 0; qy < 2; qy++)
#pragma unroll
        for (int qx = 0; qx < 2; qx++) acc += Bl[qy][qx] * M[2 * qy][2 * qx];
#pragma unroll
      for (int qy = 0; qy < 2; qy++)
#pragma unroll
        for (int qx = 0; qx < 2; qx++) acc += Bu[qy][qx] * P[2 * qy][2 * qx];
#pragma unroll
      for (int qy = 0; qy < 2; qy++)
#pragma unroll
        for (int qx = 0; qx < 2; qx++) acc += (Bl[qy][qx] + Bu[qy][qx]) * C[2 * qy][2 * qx];
#pragma unroll
      for (int qx = 0; qx < 2; qx++) acc += (Bl[0][qx] + Bl[1][qx]) * M[1][2 * qx];
#pragma unroll
      for (int qx = 0; qx < 2; qx++) acc += (Bu[0][qx] + Bu[1][qx]) * P[1][2 * qx];
#pragma unroll
      for (int qy = 0; qy < 2; qy++) acc += (Bl[qy][0] + Bl[qy][1]) * M[2 * qy][1];
#pragma unroll
      for (int qy = 0; qy < 2; qy++) acc += (Bu[qy][0] + Bu[qy][1]) * P[2 * qy][1];
      const T xc = C[1][1];
      const T diag = T(4) * bsum * s12;
      const T ax = (T(4) * bsum * xc - acc) * s12;
      const long u = ubase + (long)k * sz;
      if constexpr (MODE == 0 && sizeof(T) == 4)
        out[u] = diag > T(0) ? xc + w * __fdividef(bcur - ax, diag) : xc;  // increment only (see k_rbgs)
      else if constexpr (MODE == 0)
        out[u] = diag > T(0) ? xc + w * (bcur - ax) / diag : xc;
      else
        out[u] = bcur - ax;
    }
    k++;
  };
  // planes k0-1, k0 and cell plane k0-1 start the window
  cp_async_wait<2>();
  __syncthreads();
  rd_x(Xa, 0);
  rd_x(Xb, 1);
  rd_b(Ba, 0);
  while (k < k1) {
    plane(Xa, Xb, Xc, Ba, Bb);
    if (k >= k1) break;
    plane(Xb, Xc, Xa, Bb, Ba);
    if (k >= k1) break;
    plane(Xc, Xa, Xb, Ba, Bb);
    if (k >= k1) break;
    plane(Xa, Xb, Xc, Bb, Ba);
    if (k >= k1) break;
    plane(Xb, Xc, Xa, Ba, Bb);
    if (k >= k1) break;
    plane(Xc, Xa, Xb, Bb, Ba);
  }
  cp_async_wait<0>();
}

// MAC: residual of the V-cycle's operator and its restriction in one pass: one thread per coarse
// cell forms r = b - A x at its 8 fine cells and writes their mean (the 8-cell average of the
// restriction), and zeroes the coarse iterate.  The operator is the smoothers' (approximate
// coefficient quotient); the high-precision residual outside the V-cycle uses the exactly
// rounded one.
// The 8 fine cells' stencils share their values: x and rho of the 2 x 2 x 2 block and of the 24
// cells beyond its faces are read once (32 of each instead of 8 x 7), and each fine cell's
// operator is accumulated from registers face by face in mac_op's order.
template <typename T>
__device__ __forceinline__ void resid_restrict_mac_at(const Lv& F, const Lv& C, const T* __restrict__ x,
                                                      const T* __restrict__ b, const T* __restrict__ rho,
                                                      T* __restrict__ bc, T* __restrict__ xc, int I, int J, int K) {
  const int base[3] = {2 * I, 2 * J, 2 * K};
  T xb[8], rb[8];  // the block, q = a + 2 b + 4 c
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const long c = cix(F, base[0] + (q & 1), base[1] + ((q >> 1) & 1), base[2] + (q >> 2));
    xb[q] = x[c];
    rb[q] = rho[c];
  }
  // beyond the face of axis d on side sd (0: below the block, 1: above): cell t of the face, t =
  // the offsets along the other two axes in increasing axis order; missing outside a wall
  T xo[3][2][4], ro[3][2][4];
  bool ho[3][2][4];
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const int v = cnb(F, d, sd ? base[d] + 2 : base[d] - 1);
      const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
#pragma unroll
      for (int t = 0; t < 4; t++) {
        int p[3];
        p[d] = v;
        p[e1] = base[e1] + (t & 1);
        p[e2] = base[e2] + (t >> 1);
        ho[d][sd][t] = v >= 0;
        xo[d][sd][t] = T(0);
        ro[d][sd][t] = T(0);
        if (v >= 0) {
          const long c = cix(F, p[0], p[1], p[2]);
          xo[d][sd][t] = x[c];
          ro[d][sd][t] = rho[c];
        }
      }
    }
  const T ih2 = cv<T>(F.ih2, F.f_ih2);
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int pq[3] = {q & 1, (q >> 1) & 1, q >> 2};
    const T rc = rb[q];
    T off = T(0), dg = T(0);
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const int d = f >> 1, up = f & 1;
      const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
      T rn, xn;
      bool has = true;
      if (pq[d] != up) {  // the neighbour is the block cell across the block's middle
        const int qn = q + (up ? 1 : -1) * (1 << d);
        rn = rb[qn];
        xn = xb[qn];
      } else {
        const int t = pq[e1] + 2 * pq[e2];
        rn = ro[d][up][t];
        xn = xo[d][up][t];
        has = ho[d][up][t];
      }
      if (has) {
        const T beta = face_beta<true>(rc, rn);
        off += beta * xn;
        dg += beta;
      }
    }
    const T ax = (dg * xb[q] - off) * ih2;
    s += b[cix(F, base[0] + pq[0], base[1] + pq[1], base[2] + pq[2])] - ax;
  }
  const long u = cix(C, I, J, K);
  bc[u] = s * T(0.125);
  xc[u] = T(0);
}
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_resid_restrict_mac(Lv F, Lv C, const T* __restrict__ x,
                                                                const T* __restrict__ b, const T* __restrict__ rho,
                                                                T* __restrict__ bc, T* __restrict__ xc) {
  int I, J, K;
  if (!thread_cell(C.n, I, J, K)) return;
  resid_restrict_mac_at(F, C, x, b, rho, bc, xc, I, J, K);
}

// restriction of the residual to the coarse right-hand side at coarse unknown (I, J, K) (coarse
// x zeroed): MAC the 8-cell mean, FE full weighting
// Restriction of the fine residual to the coarse right-hand side (and a zero coarse iterate).
// Cell-centred: the mean of the 8 children.  Nodal: full weighting, weight 1/2 per axis on which
// the fine node lies between coarse nodes, summed plane by plane (fine planes 2K-1, 2K, 2K+1).
// One thread marches up to RZ coarse unknowns of its (I, J) column; in the nodal case the fine
// plane 2K+1 is kept in registers as the next unknown's plane 2K'-1.
constexpr int RZ = 8;
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_restrict(Lv F, Lv C, int kind, const T* __restrict__ rf,
                                                      T* __restrict__ bc, T* __restrict__ xc, int zc) {
  const int ext[3] = {kind == 0 ? C.n[0] : C.nn[0], kind == 0 ? C.n[1] : C.nn[1], kind == 0 ? C.n[2] : C.nn[2]};
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= ext[0] || J >= ext[1]) return;
  const int K0 = blockIdx.z * zc, K1 = min(K0 + zc, ext[2]);
  if (kind == 0) {
    for (int K = K0; K < K1; K++) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < 8; q++) s += rf[cix(F, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + ((q >> 2) & 1))];
      s *= T(0.125);
      const long u = cix(C, I, J, K);
      bc[u] = s;
      xc[u] = T(0);
    }
    return;
  }
  // the fine x and y node indices 2I-1, 2I, 2I+1 (wrapped; -1 outside a wall) and the columns
  int fx[3], fy[3];
#pragma unroll
  for (int o = 0; o < 3; o++) {
    int v = 2 * I + o - 1, w = 2 * J + o - 1;
    if (v < 0 || v >= F.nn[0]) v = F.per[0] ? (v < 0 ? v + F.nn[0] : v - F.nn[0]) : -1;
    if (w < 0 || w >= F.nn[1]) w = F.per[1] ? (w < 0 ? w + F.nn[1] : w - F.nn[1]) : -1;
    fx[o] = v;
    fy[o] = w;
  }
  const int fplane = F.nn[0] * F.nn[1];
  // the 3 x 3 values of fine plane p (zero where a node lies outside a wall: skipped in the sum)
  auto load = [&](int p, T (&v)[3][3]) {
    if (p < 0 || p >= F.nn[2]) p = F.per[2] ? (p < 0 ? p + F.nn[2] : p - F.nn[2]) : -1;
#pragma unroll
    for (int oy = 0; oy < 3; oy++)
#pragma unroll
      for (int ox = 0; ox < 3; ox++) {
        const bool in = p >= 0 && fy[oy] >= 0 && fx[ox] >= 0;
        v[oy][ox] = in ? rf[fx[ox] + F.nn[0] * fy[oy] + (long)fplane * p] : T(0);
      }
  };
  // whether each fine plane and row/column exists (a node outside a wall adds nothing)
  auto zin = [&](int p) { return F.per[2] || (p >= 0 && p < F.nn[2]); };
  T lo[3][3], mid[3][3], hi[3][3];
  load(2 * K0 - 1, lo);
  for (int K = K0; K < K1; K++) {
    load(2 * K, mid);
    load(2 * K + 1, hi);
    T s = T(0);
#pragma unroll
    for (int oz = 0; oz < 3; oz++) {
      if (!zin(2 * K + oz - 1)) continue;
#pragma unroll
      for (int oy = 0; oy < 3; oy++) {
        if (fy[oy] < 0) continue;
#pragma unroll
        for (int ox = 0; ox < 3; ox++) {
          if (fx[ox] < 0) continue;
          const T w = (ox != 1 ? T(0.5) : T(1)) * (oy != 1 ? T(0.5) : T(1)) * (oz != 1 ? T(0.5) : T(1));
          const T v = oz == 0 ? lo[oy][ox] : (oz == 1 ? mid[oy][ox] : hi[oy][ox]);
          s += w * v;
        }
      }
    }
    const long u = nix(C, I, J, K);
    bc[u] = s;
    xc[u] = T(0);
#pragma unroll
    for (int oy = 0; oy < 3; oy++)
#pragma unroll
      for (int ox = 0; ox < 3; ox++) lo[oy][ox] = hi[oy][ox];
  }
}

// Trilinear prolongation of the coarse correction, added to the fine iterate; a thread marches up
// to PZ coarse cells of its (I, J) column and writes each one's 2 x 2 x 2 fine children.
// Cell-centred: along each axis a child takes 3/4 of its parent and 1/4 of the parent's
// neighbour on the child's side (the parent itself beyond a wall: Neumann mirror), applied
// axis by axis; the x- and y-interpolated coarse planes below and above stay in registers.
constexpr int PZ = 8;  // coarse planes per thread column
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_prolong_mac(Lv F, Lv C, const T* __restrict__ xc, T* __restrict__ xf,
                                                         int zc) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.n[0] || J >= C.n[1]) return;
  const int K0 = blockIdx.z * zc, K1 = min(K0 + zc, C.n[2]);
  int nx[3], ny[3];  // coarse indices of I-1, I, I+1 and J-1, J, J+1
#pragma unroll
  for (int q = 0; q < 3; q++) {
    int a = I + q - 1, b = J + q - 1;
    if (a < 0 || a >= C.n[0]) a = C.per[0] ? (a < 0 ? a + C.n[0] : a - C.n[0]) : I;
    if (b < 0 || b >= C.n[1]) b = C.per[1] ? (b < 0 ? b + C.n[1] : b - C.n[1]) : J;
    nx[q] = a;
    ny[q] = b;
  }
  const T w0 = T(0.75), w1 = T(0.25);
  // coarse plane of K + dk (wrapped, or K itself beyond a wall)
  auto zp = [&](int K, int dk) {
    const int c = K + dk;
    if (c >= 0 && c < C.n[2]) return c;
    return C.per[2] ? (c < 0 ? c + C.n[2] : c - C.n[2]) : K;
  };
  // one coarse plane interpolated along x (child side cx), then along y (child side cy): Y[cy][cx]
  auto plane_y = [&](int Kp, T (&Y)[2][2]) {
    T rx[3][2];
#pragma unroll
    for (int qy = 0; qy < 3; qy++) {
      const long row = (long)(C.n[0] * (ny[qy] + C.n[1] * Kp));
      const T xm = xc[row + nx[0]], x0 = xc[row + nx[1]], xp = xc[row + nx[2]];
      rx[qy][0] = w0 * x0 + w1 * xm;
      rx[qy][1] = w0 * x0 + w1 * xp;
    }
#pragma unroll
    for (int cy = 0; cy < 2; cy++)
#pragma unroll
      for (int cx = 0; cx < 2; cx++) Y[cy][cx] = w0 * rx[1][cx] + w1 * rx[2 * cy][cx];
  };
  T Ym[2][2], Y0[2][2], Yp[2][2];
  plane_y(zp(K0, -1), Ym);
  plane_y(K0, Y0);
  for (int K = K0; K < K1; K++) {
    plane_y(zp(K, 1), Yp);
#pragma unroll
    for (int cz = 0; cz < 2; cz++)
#pragma unroll
      for (int cy = 0; cy < 2; cy++) {
        const long base = (long)(2 * I + (2 * J + cy) * F.n[0] + (2 * K + cz) * (F.n[0] * F.n[1]));
#pragma unroll
        for (int cx = 0; cx < 2; cx++) xf[base + cx] += w0 * Y0[cy][cx] + w1 * (cz ? Yp[cy][cx] : Ym[cy][cx]);
      }
#pragma unroll
    for (int cy = 0; cy < 2; cy++)
#pragma unroll
      for (int cx = 0; cx < 2; cx++) {
        Ym[cy][cx] = Y0[cy][cx];
        Y0[cy][cx] = Yp[cy][cx];
      }
  }
}

// Nodal: a fine node on a coarse node takes its value, one between two coarse nodes their mean
// (per axis).
template <typename T>
__device__ __forceinline__ void prolong_fe_at(const Lv& F, const Lv& C, const T* __restrict__ xc, T* __restrict__ xf,
                                              int I, int J, int K) {
  const int I1 = I + 1 < C.nn[0] ? I + 1 : (C.per[0] ? 0 : I);
  const int J1 = J + 1 < C.nn[1] ? J + 1 : (C.per[1] ? 0 : J);
  const int K1 = K + 1 < C.nn[2] ? K + 1 : (C.per[2] ? 0 : K);
  const T c000 = xc[nix(C, I, J, K)], c100 = xc[nix(C, I1, J, K)], c010 = xc[nix(C, I, J1, K)],
          c110 = xc[nix(C, I1, J1, K)], c001 = xc[nix(C, I, J, K1)], c101 = xc[nix(C, I1, J, K1)],
          c011 = xc[nix(C, I, J1, K1)], c111 = xc[nix(C, I1, J1, K1)];
  const T h = T(0.5);
#pragma unroll
  for (int cz = 0; cz < 2; cz++) {
    const int fk = 2 * K + cz;
    if (fk >= F.nn[2]) continue;
#pragma unroll
    for (int cy = 0; cy < 2; cy++) {
      const int fj = 2 * J + cy;
      if (fj >= F.nn[1]) continue;
#pragma unroll
      for (int cx = 0; cx < 2; cx++) {
        const int fi = 2 * I + cx;
        if (fi >= F.nn[0]) continue;
        // mean along each odd axis
        T a0 = cx ? h * (c000 + c100) : c000, a1 = cx ? h * (c010 + c110) : c010;
        T a2 = cx ? h * (c001 + c101) : c001, a3 = cx ? h * (c011 + c111) : c011;
        T b0 = cy ? h * (a0 + a1) : a0, b1 = cy ? h * (a2 + a3) : a2;
        const T v = cz ? h * (b0 + b1) : b0;
        xf[nix(F, fi, fj, fk)] += v;
      }
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_prolong_fe(Lv F, Lv C, const T* __restrict__ xc, T* __restrict__ xf) {
  int I, J, K;
  if (!thread_cell(C.nn, I, J, K)) return;
  prolong_fe_at(F, C, xc, xf, I, J, K);
}

// FE coefficient beta = 1/rho per cell (finest level)
template <typename T>
__global__ void k_inv(long n, const T* __restrict__ rho, T* __restrict__ beta) {
  GRID_LOOP(i, n) beta[i] = T(1) / rho[i];
}

// coarse coefficient (MAC: density, FE: beta) = mean of the 8 fine cells
template <typename T>
__global__ void __launch_bounds__(BX* BYMAX) k_coarsen(Lv F, Lv C, const T* __restrict__ rf, T* __restrict__ rc) {
  int I, J, K;
  if (!thread_cell(C.n, I, J, K)) return;
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; q++) s += rf[cix(F, 2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + ((q >> 2) & 1))];
  rc[cix(C, I, J, K)] = T(0.125) * s;
}

// sum (mode 0) or sum of squares (mode 1): per-block partials
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

// final fixed-order sum of the partials (one block); out = scale * sum; a non-finite result
// sets *nonfinite (when given): every solve takes the mean of its right-hand side and of its
// solution, so a NaN or infinity anywhere in the velocity that feeds them is caught here
__global__ void __launch_bounds__(1024) k_final(const double* __restrict__ part, int np, double scale,
                                                double* __restrict__ out, float* __restrict__ out_ff = nullptr,
                                                int* __restrict__ nonfinite = nullptr) {
  __shared__ double sh[1024];
  double loc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) loc += part[i];
  sh[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = sh[0] * scale;
    *out = v;
    if (nonfinite && !isfinite(v)) *nonfinite = 1;
    if (out_ff) {  // the same value as a two-float pair
      out_ff[0] = (float)v;
      out_ff[1] = (float)(v - (double)out_ff[0]);
    }
  }
}

// per-block partial sums of the two-float array h + l (l null: all zero): two-float
// accumulation per thread, FP64 across threads
__global__ void k_partial_ff(const float* __restrict__ h, const float* __restrict__ l, long n,
                             double* __restrict__ part) {
  __shared__ double sh[TPB / 32];
  float ah = 0.0f, al = 0.0f;
  GRID_LOOP(i, n) {
    const F2 t = two_sum(ah, h[i]);
    ah = t.h;
    al = __fadd_rn(al, __fadd_rn(t.l, l ? l[i] : 0.0f));
  }
  double loc = (double)ah + (double)al;
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < TPB / 32; w++) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// (h, l) = (e, 0) - m: the two-float solution from a single FP32 solve, mean-free
__global__ void k_set_ff_sub_mean(const float* __restrict__ e, float* __restrict__ h, float* __restrict__ l, long n,
                                  const float* __restrict__ m) {
  GRID_LOOP(i, n) {
    float a = e[i], b = 0.0f;
    ff_sub_pair(a, b, m);
    h[i] = a;
    l[i] = b;
  }
}

__global__ void k_ff_sub_mean(float* __restrict__ h, float* __restrict__ l, long n, const float* __restrict__ m) {
  GRID_LOOP(i, n) {
    float a = h[i], b = l[i];
    ff_sub_pair(a, b, m);
    h[i] = a;
    l[i] = b;
  }
}

template <typename XT>
__global__ void k_sub_scalar(XT* __restrict__ a, long n, const double* __restrict__ s) {
  const double v = *s;
  GRID_LOOP(i, n) a[i] = (XT)((double)a[i] - v);
}

// b += a (set: b = a)
template <typename T>
__global__ void k_add_to64(const T* __restrict__ a, double* __restrict__ b, long n, int set) {
  GRID_LOOP(i, n) b[i] = set ? (double)a[i] : b[i] + (double)a[i];
}

// coarsest level: one block solves it by conjugate gradients (the operator is symmetric
// positive semi-definite with the constants as null space; the right-hand side is made
// mean-free and so is the result)
constexpr int COARSE_TPB = 512;
// relative tolerance of the coarsest solve: FP64 solves to 1e-10; an FP32 V-cycle needs its
// coarse correction to well below its own convergence factor (about 0.1), and FP32 CG on the
// periodic coarsest levels stalls on rounding near 1e-5 (it then ran to its iteration cap), so
// FP32 stops at 1e-3
template <typename T>
constexpr double coarse_tol() { return sizeof(T) == 4 ? 1e-3 : 1e-10; }
// dynamic shared memory of the coarse solve: x, r, p, q = A p and the coefficient of the level,
// or 0 when they do not fit next to the kernel's static shared memory (it then works on global
// memory)
inline size_t coarse_smem(const Lv& L, size_t esz) {
  const size_t need = (4 * (size_t)L.nunk + (size_t)L.ncell) * esz;
  constexpr size_t avail = 227 * 1024 - (COARSE_TPB / 32 + 2) * sizeof(double);
  return need <= avail ? need : 0;
}

// Reductions and scalars of the coarsest solve run in the storage type: FP32 levels sum and divide
// in FP32 (the solve is a correction inside an FP32 V-cycle; FP64 shuffles and divisions on
// GB300's narrow FP64 pipe made each iteration a long latency chain), FP64 levels in FP64.
// sum over the block (every thread gets it), in R; red: COARSE_TPB / 32 values of shared memory
template <typename R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read by the previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  R t = R(0);
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
  return t;
}

// Conjugate gradients on one level by the whole block: r holds the right-hand side on entry (it
// is made mean-free), x receives the mean-free solution, p and q are scratch; every thread of the
// block calls it.  red: COARSE_TPB / 32 doubles of shared memory.
template <typename T>
__device__ void cg_block(const Lv& L, int kind, int max_it, double rtol, T* x, T* r, T* p, T* q, const T* rho,
                         double* redd) {
  const long n = L.nunk;
  T* red = reinterpret_cast<T*>(redd);
  T loc = T(0);
  for (long u = threadIdx.x; u < n; u += blockDim.x) loc += r[u];
  const T mean = block_sum(loc, red) / T(n);
  loc = T(0);
  for (long u = threadIdx.x; u < n; u += blockDim.x) {
    const T v = r[u] - mean;
    r[u] = v;
    p[u] = v;
    x[u] = T(0);
    loc += v * v;
  }
  T rr = block_sum(loc, red);
  const T stop = T(rtol * rtol) * rr;
  const int ex = kind == 0 ? L.n[0] : L.nn[0], ey = kind == 0 ? L.n[1] : L.nn[1];
  for (int it = 0; it < max_it && rr > stop; it++) {
    __syncthreads();  // p complete
    loc = T(0);
    for (long u = threadIdx.x; u < n; u += blockDim.x) {
      int i, j, k;
      decode(u, ex, ey, i, j, k);
      T dg;
      const T ap = kind == 0 ? mac_op<T>(L, p, rho, i, j, k, dg) : fe_op<T>(L, p, rho, i, j, k, dg);
      q[u] = ap;
      loc += p[u] * ap;
    }
    const T pq = block_sum(loc, red);
    if (!(pq > T(0))) break;
    const T a = rr / pq;
    loc = T(0);
    for (long u = threadIdx.x; u < n; u += blockDim.x) {
      x[u] += a * p[u];
      const T v = r[u] - a * q[u];
      r[u] = v;
      loc += v * v;
    }
    const T rr2 = block_sum(loc, red);
    const T beta = rr2 / rr;
    rr = rr2;
    for (long u = threadIdx.x; u < n; u += blockDim.x) p[u] = r[u] + beta * p[u];
  }
  __syncthreads();
  loc = T(0);
  for (long u = threadIdx.x; u < n; u += blockDim.x) loc += x[u];
  const T xm = block_sum(loc, red) / T(n);
  for (long u = threadIdx.x; u < n; u += blockDim.x) x[u] = x[u] - xm;
  __syncthreads();
}

// The same iteration run by one warp (the calling warp; small levels, where the block's barriers
// would dominate): reductions by shuffles only.
template <typename T>
__device__ void cg_warp(const Lv& L, int kind, int max_it, double rtol, T* x, T* r, T* p, T* q, const T* rho) {
  const int lane = threadIdx.x & 31;
  const int n = (int)L.nunk;
  auto wsum = [](T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  T loc = T(0);
  for (int u = lane; u < n; u += 32) loc += r[u];
  const T mean = wsum(loc) / T(n);
  loc = T(0);
  for (int u = lane; u < n; u += 32) {
    const T v = r[u] - mean;
    r[u] = v;
    p[u] = v;
    x[u] = T(0);
    loc += v * v;
  }
  T rr = wsum(loc);
  const T stop = T(rtol * rtol) * rr;
  const int ex = kind == 0 ? L.n[0] : L.nn[0], ey = kind == 0 ? L.n[1] : L.nn[1];
  for (int it = 0; it < max_it && rr > stop; it++) {
    __syncwarp();  // p complete
    loc = T(0);
    for (int u = lane; u < n; u += 32) {
      const int rw = u / ex;
      const int i = u - rw * ex, j = rw % ey, k = rw / ey;
      T dg;
      const T ap = kind == 0 ? mac_op<T>(L, p, rho, i, j, k, dg) : fe_op<T>(L, p, rho, i, j, k, dg);
      q[u] = ap;
      loc += p[u] * ap;
    }
    const T pq = wsum(loc);
    if (!(pq > T(0))) break;
    const T a = rr / pq;
    loc = T(0);
    for (int u = lane; u < n; u += 32) {
      x[u] += a * p[u];
      const T v = r[u] - a * q[u];
      r[u] = v;
      loc += v * v;
    }
    const T rr2 = wsum(loc);
    const T beta = rr2 / rr;
    rr = rr2;
    __syncwarp();  // every lane has read p for its q before p changes
    for (int u = lane; u < n; u += 32) p[u] = r[u] + beta * p[u];
  }
  __syncwarp();
  loc = T(0);
  for (int u = lane; u < n; u += 32) loc += x[u];
  const T xm = wsum(loc) / T(n);
  for (int u = lane; u < n; u += 32) x[u] = x[u] - xm;
  __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(COARSE_TPB) k_coarse_cg(Lv L, int kind, int max_it, double rtol, T* __restrict__ gx,
                                                         T* __restrict__ gp, T* __restrict__ gb,
                                                         T* __restrict__ gq, const T* __restrict__ grho,
                                                         int in_smem) {
  __shared__ double red[COARSE_TPB / 32];
  extern __shared__ unsigned char smem[];
  const long n = L.nunk;
  T *x = gx, *r = gb, *p = gp, *q = gq;
  const T* rho = grho;
  if (in_smem) {
    x = (T*)smem;
    r = x + n;
    p = r + n;
    q = p + n;
    T* c = q + n;
    for (long u = threadIdx.x; u < n; u += blockDim.x) r[u] = gb[u];
    for (long u = threadIdx.x; u < L.ncell; u += blockDim.x) c[u] = grho[u];
    rho = c;
    __syncthreads();
  }
  if (blockDim.x == 32)
    cg_warp(L, kind, max_it, rtol, x, r, p, q, rho);
  else
    cg_block(L, kind, max_it, rtol, x, r, p, q, rho, red);
  if (in_smem)
    for (long u = threadIdx.x; u < n; u += blockDim.x) gx[u] = x[u];
}

}  // namespace

// ------------------------------------------------------------------------------- solver
struct MGSolver {
  int kind = 0, fp32 = 0, nlev = 0;
  Lv lv[16];
  void* x[16] = {};
  void* xt[16] = {};
  void* b[16] = {};
  void* r[16] = {};
  void* rho[16] = {};  // per-level coefficient: MAC density (level 0: the caller's array), FE beta
  const void* rho_in = nullptr;
  double *x64 = nullptr, *b64 = nullptr, *part = nullptr, *scal = nullptr;
  float *xh = nullptr, *xl = nullptr, *bh = nullptr, *bl = nullptr;  // two-float iterate and rhs (T = float)
  double* hpin = nullptr;
  size_t esz = 8;
  int pre = 2, post = 2;
  int cpre = -1, cpost = -1;  // levels below the finest (negative: pre, post)
  int inner = 1;  // V-cycles on the storage-precision correction equation per high-precision residual
  int by = 4;     // block height of the level kernels
  int warm = 0;   // start from the last solution instead of zero
  // MAC (FP32): fused red-black sweeps (k_rbgs_sweep): 0 never, 1 on the large levels that allow
  // them, 2 on every level that allows them
  int sweep = 1;
  int zc[16] = {};      // z-chunk of k_rbgs_sweep per level (0: the level's layout does not allow it)
  bool big[16] = {};    // level large enough for the fused sweep to pay
  bool jac[16] = {};    // MAC level with an odd periodic side: Jacobi sweeps instead of red-black
  double omega = 0.9;
  mg_hook_fn hook = nullptr;
  void* hook_ctx = nullptr;
  int* nonfinite = nullptr;  // device flag set when a mean or norm of a solve is not finite
  int zc0_auto = 0;          // z-chunk of the finest level's fused sweep from the wave heuristic
  int fe_zc0 = 0;            // z-chunk of the finest level's FE tiles (0: the heuristic)
  size_t bytes = 0;          // device bytes requested
};

void mg_set_hook(MGSolver* m, mg_hook_fn fn, void* ctx) {
  m->hook = fn;
  m->hook_ctx = ctx;
}
void mg_set_smoother(MGSolver* m, int pre, int post, double omega) {
  if (pre >= 0) m->pre = pre;
  if (post >= 0) m->post = post;
  if (omega > 0) m->omega = omega;
}
void mg_set_coarse_smoother(MGSolver* m, int pre, int post) {
  m->cpre = pre;
  m->cpost = post;
}
void mg_set_inner(MGSolver* m, int inner) {
  if (inner >= 1) m->inner = inner;
}
void mg_set_warm(MGSolver* m, int warm) { m->warm = warm != 0; }
void mg_set_nonfinite_flag(MGSolver* m, int* flag) { m->nonfinite = flag; }
void mg_set_sweep(MGSolver* m, int fused) { m->sweep = fused < 0 ? 0 : (fused > 2 ? 2 : fused); }
void mg_set_block(MGSolver* m, int by) {
  if (by == 1 || by == 2 || by == 4 || by == 8) m->by = by;
}

// z-chunk of the fused sweep on level Q with `resident` blocks on the GPU at once: the chunk
// count that best fills whole waves, discounted by the two extra first-colour planes a chunk
// recomputes
static int sweep_chunk(const Lv& Q, int resident) {
  const long tiles = (long)((Q.n[0] + GX - 1) / GX) * ((Q.n[1] + GY - 1) / GY);
  int best = Q.n[2];
  double best_eff = -1.0;
  for (int c = 1; c <= Q.n[2]; c++) {
    const int zc = (Q.n[2] + c - 1) / c;
    const long blocks = tiles * ((Q.n[2] + zc - 1) / zc);
    const long waves = (blocks + resident - 1) / resident;
    const double eff = (double)blocks / (double)(waves * resident) * (double)zc / (double)(zc + 2);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = zc;
    }
  }
  return best;
}

static cudaError_t dmalloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes < 16 ? 16 : bytes);
  return e;
}

namespace {
// Builds the level hierarchy; with dry set it only adds up the device bytes it would allocate.
MGSolver* mg_build(const Geo& g, int kind, int prec_fp32, bool dry, cudaError_t* err) {
  MGSolver* m = new MGSolver();
  m->kind = kind;
  m->fp32 = prec_fp32;
  m->esz = prec_fp32 ? 4 : 8;
  m->omega = kind == 0 ? 1.0 : 0.9;
  m->pre = m->post = kind == 0 ? 3 : 2;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    m->bytes += dev_bytes(bytes);
    if (dry || e != cudaSuccess) return;
    e = dmalloc(p, bytes);
  };
  Lv L;
  for (int d = 0; d < 3; d++) {
    L.n[d] = g.n[d];
    L.per[d] = g.per[d];
  }
  L.h = g.h;
  for (int l = 0; l < 16; l++) {
    for (int d = 0; d < 3; d++) L.nn[d] = L.per[d] ? L.n[d] : L.n[d] + 1;
    L.ncell = (long)L.n[0] * L.n[1] * L.n[2];
    L.nnode = (long)L.nn[0] * L.nn[1] * L.nn[2];
    L.nunk = kind == 0 ? L.ncell : L.nnode;
    L.ih2 = 1.0 / (L.h * L.h);
    L.s12 = L.h / 12.0;
    L.f_ih2 = (float)L.ih2;
    L.f_s12 = (float)L.s12;
    L.f_ih2_lo = (float)(L.ih2 - (double)L.f_ih2);
    L.f_s12_lo = (float)(L.s12 - (double)L.f_s12);
    m->lv[l] = L;
    m->nlev = l + 1;
    for (int d = 0; d < 3; d++)
      if (kind == 0 && L.per[d] && (L.n[d] & 1)) m->jac[l] = true;
    const size_t vb = (size_t)L.nunk * m->esz;
    alloc(&m->x[l], vb);
    alloc(&m->xt[l], vb);
    alloc(&m->b[l], vb);
    alloc(&m->r[l], vb);
    if (l > 0 || kind == 1) alloc(&m->rho[l], (size_t)L.ncell * m->esz);
    // coarsen while every axis is even and halves to at least 3 (a MAC level with an odd periodic
    // side is smoothed by Jacobi sweeps, see jac)
    bool can = true;
    for (int d = 0; d < 3; d++) {
      const int h2 = L.n[d] / 2;
      if ((L.n[d] & 1) || h2 < 3) can = false;
    }
    if (!can || l == 15) break;
    for (int d = 0; d < 3; d++) L.n[d] /= 2;
    L.h *= 2.0;
  }
  const Lv& L0 = m->lv[0];
  const long nbr = (long)((L0.nn[0] + BX - 1) / BX) * L0.nn[1] * L0.nn[2];  // partials at by = 1
  alloc((void**)&m->x64, L0.nunk * sizeof(double));
  if (!prec_fp32) alloc((void**)&m->b64, L0.nunk * sizeof(double));
  if (prec_fp32) {
    alloc((void**)&m->xh, L0.nunk * sizeof(float));
    alloc((void**)&m->xl, L0.nunk * sizeof(float));
    alloc((void**)&m->bh, L0.nunk * sizeof(float));
    alloc((void**)&m->bl, L0.nunk * sizeof(float));
  }
  alloc((void**)&m->part, (size_t)(nbr > RED_BLOCKS ? nbr : RED_BLOCKS) * sizeof(double));
  alloc((void**)&m->scal, 8 * sizeof(double));
  if (!dry) {
    if (e == cudaSuccess) e = cudaMallocHost((void**)&m->hpin, 8 * sizeof(double));
    // the coarsest level lives in shared memory during its solve (when it fits): opt in to its
    // size once, outside any stream capture
    const size_t smem = coarse_smem(m->lv[m->nlev - 1], m->esz);
    // the attribute belongs to the kernel, shared by every solver: it only ever grows
    static std::mutex mu;
    static size_t opted[2] = {0, 0};
    std::lock_guard<std::mutex> lock(mu);
    if (e == cudaSuccess && smem > opted[prec_fp32 ? 1 : 0]) {
      if (prec_fp32)
        e = cudaFuncSetAttribute(k_coarse_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      else
        e = cudaFuncSetAttribute(k_coarse_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) opted[prec_fp32 ? 1 : 0] = smem;
    }

    // the fused sweep's staging ring (beyond the 48 KB default) with the largest shared-memory
    // carveout, so that three blocks fit on an SM; once per process
    static bool sweep_opted = false;
    if (e == cudaSuccess && kind == 0 && prec_fp32 && !sweep_opted) {
      for (int v = 0; v < 2 && e == cudaSuccess; v++) {
        const void* fn = v ? (const void*)k_rbgs_sweep<true> : (const void*)k_rbgs_sweep<false>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
      }
      if (e == cudaSuccess) sweep_opted = true;
    }
    if (e == cudaSuccess && kind == 0 && prec_fp32) {
      // levels that take the fused sweep: rows of whole 16-byte chunks and even periodic sides (a
      // consistent two-colouring across the wrap); z-chunks sized to the blocks resident at once
      const int nsm = sm_count();
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbgs_sweep<true>, GT, SWEEP_SMEM) != cudaSuccess ||
          per_sm < 1)
        per_sm = 1;
      for (int l = 0; l < m->nlev; l++) {
        const Lv& Q = m->lv[l];
        bool ok = Q.n[0] % 4 == 0;
        for (int d = 0; d < 3; d++)
          if (Q.per[d] && (Q.n[d] & 1)) ok = false;
        m->zc[l] = ok ? sweep_chunk(Q, per_sm * nsm) : 0;
        if (l == 0) m->zc0_auto = m->zc[0];
        m->big[l] = Q.n[0] >= 64 && Q.ncell >= (1L << 20);
      }
    }
  }
  if (err) *err = e;
  return m;
}
}  // namespace

MGSolver* mg_create(const Geo& g, int kind, int prec_fp32, cudaError_t* err) {
  return mg_build(g, kind, prec_fp32, false, err);
}

size_t mg_footprint(const Geo& g, int kind, int prec_fp32) {
  MGSolver* m = mg_build(g, kind, prec_fp32, true, nullptr);
  const size_t b = m->bytes;
  delete m;
  return b;
}
size_t mg_device_bytes(const MGSolver* m) { return m ? m->bytes : 0; }

void mg_destroy(MGSolver* m) {
  if (!m) return;
  for (int l = 0; l < m->nlev; l++) {
    cudaFree(m->x[l]);
    cudaFree(m->xt[l]);
    cudaFree(m->b[l]);
    cudaFree(m->r[l]);
    if (l > 0 || m->kind == 1) cudaFree(m->rho[l]);
  }
  cudaFree(m->x64);
  cudaFree(m->b64);
  cudaFree(m->xh);
  cudaFree(m->xl);
  cudaFree(m->bh);
  cudaFree(m->bl);
  cudaFree(m->part);
  cudaFree(m->scal);
  cudaFreeHost(m->hpin);
  delete m;
}

MGVec mg_rhs(MGSolver* m) { return m->fp32 ? MGVec{nullptr, m->bh, m->bl} : MGVec{m->b64, nullptr, nullptr}; }
MGVec mg_solution(MGSolver* m) { return m->fp32 ? MGVec{nullptr, m->xh, m->xl} : MGVec{m->x64, nullptr, nullptr}; }
const double* mg_solution64(MGSolver* m, cudaStream_t s) {
  if (m->fp32) {
    const long n = m->lv[0].nunk;
    k_ff_to64<<<nblocks(n), TPB, 0, s>>>(m->xh, m->xl, m->x64, n);
    rmt_count_launches(1);
  }
  return m->x64;
}
void mg_set_density(MGSolver* m, const void* rho) {
  m->rho_in = rho;
  if (m->kind == 0) m->rho[0] = (void*)rho;
}

namespace {

inline void hk(MGSolver* m, int l, int which, int begin, cudaStream_t s) {
  if (m->hook && l == 0) m->hook(m->hook_ctx, which, begin, s);
}

template <typename T>
void sum_into(MGSolver* m, const T* a, long n, int mode, double scale, double* out, cudaStream_t s) {
  int nb = nblocks(n);
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  k_partial<T><<<nb, TPB, 0, s>>>(a, n, mode, m->part);
  rmt_count_launches(1);
  k_final<<<1, 1024, 0, s>>>(m->part, nb, scale, out, nullptr, m->nonfinite);
  rmt_count_launches(1);
}

// out = scale * sum(h + l); out_ff receives the same value as a two-float pair
void sum_ff(MGSolver* m, const float* h, const float* l, long n, double scale, double* out, float* out_ff,
            cudaStream_t s) {
  int nb = nblocks(n);
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  k_partial_ff<<<nb, TPB, 0, s>>>(h, l, n, m->part);
  rmt_count_launches(1);
  k_final<<<1, 1024, 0, s>>>(m->part, nb, scale, out, out_ff, m->nonfinite);
  rmt_count_launches(1);
}

// the FE tile kernel stages 16-byte rows on FP32 levels with a periodic x axis of n_x % 4 == 0
template <typename T>
inline bool fe_vec(const Lv& L) {
  return sizeof(T) == 4 && L.per[0] && L.n[0] % 4 == 0;
}
inline dim3 fe_grid(const Lv& L, int zchunk = 0) {
  // z-chunks of FZ planes, or more and shorter chunks on small levels, so that at least two
  // blocks per SM march concurrently (a block's planes follow one another); zchunk > 0 sets the
  // chunk length instead (the autotuner's choice); the kernel takes its chunk from the grid
  const int tx = (L.nn[0] + FX - 1) / FX, ty = (L.nn[1] + FY - 1) / FY;
  int nch = (L.nn[2] + FZ - 1) / FZ;
  const int want = (2 * sm_count() + tx * ty - 1) / (tx * ty);
  if (want > nch) nch = want < L.nn[2] ? want : L.nn[2];
  if (zchunk > 0) nch = (L.nn[2] + zchunk - 1) / zchunk;
  const int fz = (L.nn[2] + nch - 1) / nch;
  return dim3(tx, ty, (L.nn[2] + fz - 1) / fz);
}

template <typename T>
void smooth(MGSolver* m, int l, int sweeps, bool forward, cudaStream_t s) {
  const Lv& L = m->lv[l];
  const T* b = (const T*)m->b[l];
  const T* rho = (const T*)m->rho[l];
  for (int it = 0; it < sweeps; it++) {
    if constexpr (sizeof(T) == 4) {
      if (m->kind == 0 && m->zc[l] > 0 && (m->sweep == 2 || (m->sweep == 1 && m->big[l]))) {
        // both colours in one out-of-place pass: x[l] -> xt[l], then the two swap roles
        const dim3 gr((L.n[0] + GX - 1) / GX, (L.n[1] + GY - 1) / GY, (L.n[2] + m->zc[l] - 1) / m->zc[l]);
        hk(m, l, 2, 1, s);
        if (L.per[0] && L.per[1] && L.per[2])
          k_rbgs_sweep<false><<<gr, GT, SWEEP_SMEM, s>>>(L, forward ? 0 : 1, (float)m->omega, (const float*)m->x[l],
                                                         (float*)m->xt[l], b, rho, m->zc[l]);
        else
          k_rbgs_sweep<true><<<gr, GT, SWEEP_SMEM, s>>>(L, forward ? 0 : 1, (float)m->omega, (const float*)m->x[l],
                                                        (float*)m->xt[l], b, rho, m->zc[l]);
        rmt_count_launches(1);
        hk(m, l, 2, 0, s);
        void* t = m->x[l];
        m->x[l] = m->xt[l];
        m->xt[l] = t;
        continue;
      }
    }
    if (m->kind == 0 && m->jac[l]) {
      hk(m, l, 0, 1, s);
      k_jacobi_mac<T><<<grid3(L.n[0], L.n[1], L.n[2], m->by), dim3(BX, m->by), 0, s>>>(
          L, T(MAC_JACOBI_W), (const T*)m->x[l], (T*)m->xt[l], b, rho);
      rmt_count_launches(1);
      hk(m, l, 0, 0, s);
      void* t = m->x[l];
      m->x[l] = m->xt[l];
      m->xt[l] = t;
    } else if (m->kind == 0) {
      const dim3 gr(((L.n[0] + 1) / 2 + BX - 1) / BX, (L.n[1] + m->by - 1) / m->by, L.n[2]);
      for (int q = 0; q < 2; q++) {
        const int col = forward ? q : 1 - q;
        hk(m, l, 0, 1, s);
        k_rbgs<T><<<gr, dim3(BX, m->by), 0, s>>>(L, col, T(m->omega), (T*)m->x[l], b, rho);
        rmt_count_launches(1);
        hk(m, l, 0, 0, s);
      }
    } else {
      hk(m, l, 0, 1, s);
      const dim3 fg = fe_grid(L, l == 0 ? m->fe_zc0 : 0);
      if (fe_vec<T>(L))
        k_fe_tile<float, 0, true><<<fg, dim3(FX, FY), 0, s>>>(L, (float)m->omega, (const float*)m->x[l],
                                                                      (float*)m->xt[l], (const float*)b,
                                                                      (const float*)rho);
      else
        k_fe_tile<T, 0><<<fg, dim3(FX, FY), 0, s>>>(L, T(m->omega), (const T*)m->x[l], (T*)m->xt[l], b, rho);
      rmt_count_launches(1);
      hk(m, l, 0, 0, s);
      void* t = m->x[l];
      m->x[l] = m->xt[l];
      m->xt[l] = t;
    }
  }
}

template <typename T>
void vcycle(MGSolver* m, int l, cudaStream_t s) {
  const Lv& L = m->lv[l];
  if (l == m->nlev - 1) {
    int nmax = L.n[0];
    if (L.n[1] > nmax) nmax = L.n[1];
    if (L.n[2] > nmax) nmax = L.n[2];
    // conjugate gradients converge in O(nmax) iterations on this level; the cap only bounds
    // the launch, the tolerance ends it
    const int max_it = 8 * nmax + 64;
    const double tol = coarse_tol<T>();
    const size_t smem = coarse_smem(L, sizeof(T));  // opted in at creation
    // as many warps as the level has unknowns for, and a single warp (reductions by shuffles, no
    // block barriers) up to 512 unknowns: a small level's iterations are bound by the reductions
    const long want = (L.nunk + 31) / 32 * 32;
    const int tpb = L.nunk <= 512 ? 32 : (want < COARSE_TPB ? (int)want : COARSE_TPB);
    k_coarse_cg<T><<<1, tpb, smem, s>>>(L, m->kind, max_it, tol, (T*)m->x[l], (T*)m->xt[l], (T*)m->b[l],
                                               (T*)m->r[l], (const T*)m->rho[l], smem > 0);
    rmt_count_launches(1);
    return;
  }
  const int npre = l > 0 && m->cpre >= 0 ? m->cpre : m->pre, npost = l > 0 && m->cpost >= 0 ? m->cpost : m->post;
  smooth<T>(m, l, npre, true, s);
  const Lv& C = m->lv[l + 1];
  if (m->kind == 0) {
    k_resid_restrict_mac<T><<<grid3(C.n[0], C.n[1], C.n[2], m->by), dim3(BX, m->by), 0, s>>>(
        L, C, (const T*)m->x[l], (const T*)m->b[l], (const T*)m->rho[l], (T*)m->b[l + 1], (T*)m->x[l + 1]);
    rmt_count_launches(1);
  } else {
    const dim3 fg = fe_grid(L, l == 0 ? m->fe_zc0 : 0);
    if (fe_vec<T>(L))
      k_fe_tile<float, 1, true><<<fg, dim3(FX, FY), 0, s>>>(L, 0.f, (const float*)m->x[l], (float*)m->r[l],
                                                                    (const float*)m->b[l], (const float*)m->rho[l]);
    else
      k_fe_tile<T, 1><<<fg, dim3(FX, FY), 0, s>>>(L, T(0), (const T*)m->x[l], (T*)m->r[l], (const T*)m->b[l],
                                                         (const T*)m->rho[l]);
    rmt_count_launches(1);
    const int zc = column_chunk(C.nnode, RZ);
    k_restrict<T><<<grid3(C.nn[0], C.nn[1], (C.nn[2] + zc - 1) / zc, m->by), dim3(BX, m->by), 0, s>>>(
        L, C, m->kind, (const T*)m->r[l], (T*)m->b[l + 1], (T*)m->x[l + 1], zc);
    rmt_count_launches(1);
  }
  vcycle<T>(m, l + 1, s);
  if (m->kind == 0) {
    const int zc = column_chunk(C.ncell, PZ);
    k_prolong_mac<T><<<grid3(C.n[0], C.n[1], (C.n[2] + zc - 1) / zc, m->by), dim3(BX, m->by), 0, s>>>(
        L, C, (const T*)m->x[l + 1], (T*)m->x[l], zc);
  } else
    k_prolong_fe<T><<<grid3(C.nn[0], C.nn[1], C.nn[2], m->by), dim3(BX, m->by), 0, s>>>(L, C, (const T*)m->x[l + 1],
                                                                                        (T*)m->x[l]);
  rmt_count_launches(1);
  smooth<T>(m, l, npost, false, s);
}

template <typename T>
int solve_t(MGSolver* m, double rtol, int max_cycles, int fixed_cycles, cudaStream_t s, cudaError_t* err) {
  const Lv& L0 = m->lv[0];
  const long n = L0.nunk;
  // coefficients of every level
  if (m->kind == 1) {
    k_inv<T><<<nblocks(L0.ncell), TPB, 0, s>>>(L0.ncell, (const T*)m->rho_in, (T*)m->rho[0]);
    rmt_count_launches(1);
  }
  for (int l = 1; l < m->nlev; l++) {
    const Lv& F = m->lv[l - 1];
    const Lv& C = m->lv[l];
    k_coarsen<T><<<grid3(C.n[0], C.n[1], C.n[2], m->by), dim3(BX, m->by), 0, s>>>(F, C, (const T*)m->rho[l - 1], (T*)m->rho[l]);
    rmt_count_launches(1);
  }
  // scal: [0] mean of b, [2] |r|^2, [3] mean of x (FP64); fm: the two means as two-float pairs
  float* fm = (float*)(m->scal + 6);
  constexpr bool ff = sizeof(T) == 4;  // two-float right-hand side and iterate
  if constexpr (ff)
    sum_ff(m, m->bh, m->bl, n, 1.0 / (double)n, m->scal, fm, s);
  else
    sum_into<double>(m, m->b64, n, 0, 1.0 / (double)n, m->scal, s);
  const int ex = m->kind == 0 ? L0.n[0] : L0.nn[0], ey = m->kind == 0 ? L0.n[1] : L0.nn[1],
            ez = m->kind == 0 ? L0.n[2] : L0.nn[2];
  const dim3 g0 = grid3(ex, ey, ez, m->by);
  const int nbr = (int)((long)g0.x * g0.y * g0.z);
  const int cap = fixed_cycles > 0 ? fixed_cycles : max_cycles;
  int cycles = 0;
  int ok = 1;
  bool have_x = false;  // false: the iterate is still zero
  bool single = false;  // FP32: one solve from zero, its result still in x[0]
  double bn2 = -1.0;
  if (m->warm) {
    // warm start from the last solution (mean-free; zero before the first solve): remove the
    // mean of b here, since the first residual is a full one
    have_x = true;
    if constexpr (ff) {
      k_ff_sub_mean<<<nblocks(n), TPB, 0, s>>>(m->bh, m->bl, n, fm);
    } else {
      k_sub_scalar<double><<<nblocks(n), TPB, 0, s>>>(m->b64, n, m->scal);
    }
    rmt_count_launches(1);
    if (fixed_cycles <= 0) {
      if constexpr (ff)
        sum_into<float>(m, m->bh, n, 1, 1.0, m->scal + 1, s);
      else
        sum_into<double>(m, m->b64, n, 1, 1.0, m->scal + 1, s);
      cudaMemcpyAsync(m->hpin, m->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
      if ((*err = cudaStreamSynchronize(s)) != cudaSuccess) return -1;
      bn2 = m->hpin[0];
    }
  }
  // a single FP32 pass from zero: fixed cycles that one round of inner V-cycles covers
  const bool once = ff && !have_x && fixed_cycles > 0 && m->inner >= fixed_cycles;
  bool x_zeroed = false;
  for (;;) {
    if (!have_x) {
      // the residual of the zero iterate is b itself: remove its mean, no operator
      if constexpr (ff) {
        k_first_resid_ff<<<g0, dim3(BX, m->by), 0, s>>>(L0, m->kind, m->bh, m->bl, fm, (float*)m->b[0], m->part,
                                                        once ? 1 : 0, (float*)m->x[0]);
        x_zeroed = once;
      } else
        k_first_resid64<<<g0, dim3(BX, m->by), 0, s>>>(L0, m->kind, m->b64, m->scal, (double*)m->b[0], m->part);
      rmt_count_launches(1);
    } else {
      hk(m, 0, 1, 1, s);
      if constexpr (ff)
        k_resid_ff<<<g0, dim3(BX, m->by), 0, s>>>(L0, m->kind, m->xh, m->xl, m->bh, m->bl, (const float*)m->rho[0],
                                               (float*)m->b[0], m->part);
      else
        k_resid64<<<g0, dim3(BX, m->by), 0, s>>>(L0, m->kind, m->x64, m->b64, (const double*)m->rho[0],
                                              (double*)m->b[0], m->part);
      rmt_count_launches(1);
      hk(m, 0, 1, 0, s);
    }
    if (fixed_cycles <= 0) {
      k_final<<<1, 1024, 0, s>>>(m->part, nbr, 1.0, m->scal + 2, nullptr, m->nonfinite);
      rmt_count_launches(1);
      cudaMemcpyAsync(m->hpin + 1, m->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
      if ((*err = cudaStreamSynchronize(s)) != cudaSuccess) return -1;
      const double rn2 = m->hpin[1];
      if (!(rn2 == rn2)) {
        ok = 0;
        break;
      }
      if (bn2 < 0.0) bn2 = rn2;  // |b|^2 of the mean-free right-hand side (zero start)
      if (bn2 == 0.0) break;
      if (rn2 <= rtol * rtol * bn2) break;
    }
    if (cycles >= cap) {
      if (fixed_cycles <= 0) ok = 0;
      break;
    }
    if (!x_zeroed) {
      k_zero<T><<<nblocks(n), TPB, 0, s>>>((T*)m->x[0], n);
      rmt_count_launches(1);
    }
    x_zeroed = false;
    // inner V-cycles on A e = r in the storage type (the high-precision residual is re-formed after them)
    for (int q = 0; q < m->inner && cycles < cap; q++) {
      vcycle<T>(m, 0, s);
      cycles++;
    }
    if (ff && !have_x && fixed_cycles > 0 && cycles >= fixed_cycles) {
      single = true;  // x[0] is the whole solution: converted below with its mean removed
      have_x = true;
      break;
    }
    if constexpr (ff)
      k_add_ff<<<nblocks(n), TPB, 0, s>>>((const float*)m->x[0], m->xh, m->xl, n, have_x ? 0 : 1);
    else
      k_add_to64<<<nblocks(n), TPB, 0, s>>>((const double*)m->x[0], m->x64, n, have_x ? 0 : 1);
    rmt_count_launches(1);
    have_x = true;
    if (fixed_cycles > 0 && cycles >= fixed_cycles) break;
  }
  // mean-free solution
  if constexpr (ff) {
    if (!have_x) {
      k_zero<float><<<nblocks(n), TPB, 0, s>>>(m->xh, n);
      k_zero<float><<<nblocks(n), TPB, 0, s>>>(m->xl, n);
      rmt_count_launches(2);
    } else if (single) {
      // the same values as setting (x, 0) and removing the two-float mean, in one pass
      sum_ff(m, (const float*)m->x[0], nullptr, n, 1.0 / (double)n, m->scal + 3, fm + 2, s);
      k_set_ff_sub_mean<<<nblocks(n), TPB, 0, s>>>((const float*)m->x[0], m->xh, m->xl, n, fm + 2);
      rmt_count_launches(1);
    } else {
      sum_ff(m, m->xh, m->xl, n, 1.0 / (double)n, m->scal + 3, fm + 2, s);
      k_ff_sub_mean<<<nblocks(n), TPB, 0, s>>>(m->xh, m->xl, n, fm + 2);
      rmt_count_launches(1);
    }
  } else {
    if (!have_x) {
      k_zero<double><<<nblocks(n), TPB, 0, s>>>(m->x64, n);
      rmt_count_launches(1);
    } else {
      sum_into<double>(m, m->x64, n, 0, 1.0 / (double)n, m->scal + 3, s);
      k_sub_scalar<double><<<nblocks(n), TPB, 0, s>>>(m->x64, n, m->scal + 3);
      rmt_count_launches(1);
    }
  }
  *err = cudaGetLastError();
  return ok ? cycles : -1;
}

}  // namespace

// does the finest MAC level run the fused red-black sweep?
static bool mac_fused0(const MGSolver* m) {
  return m->fp32 && m->zc[0] > 0 && (m->sweep == 2 || (m->sweep == 1 && m->big[0]));
}
void mg_set_zchunk(MGSolver* m, int zchunk) {
  const Lv& L = m->lv[0];
  if (m->kind == 0) {
    if (!mac_fused0(m)) return;  // the finest level does not take the fused sweep
    m->zc[0] = zchunk > 0 ? (zchunk < L.n[2] ? zchunk : L.n[2]) : m->zc0_auto;
  } else {
    m->fe_zc0 = zchunk > 0 ? (zchunk < L.nn[2] ? zchunk : L.nn[2]) : 0;
  }
}
int mg_zchunk(const MGSolver* m) {
  if (m->kind == 0) return mac_fused0(m) ? m->zc[0] : 0;
  const Lv& L = m->lv[0];
  const dim3 g = fe_grid(L, m->fe_zc0);
  return (L.nn[2] + (int)g.z - 1) / (int)g.z;
}

int mg_solve(MGSolver* m, double rtol, int max_cycles, int fixed_cycles, cudaStream_t s, cudaError_t* err) {
  cudaError_t e = cudaSuccess;
  int r = m->fp32 ? solve_t<float>(m, rtol, max_cycles, fixed_cycles, s, &e)
                  : solve_t<double>(m, rtol, max_cycles, fixed_cycles, s, &e);
  if (err) *err = e;
  return r;
}
