// Stress kernel of the RMT per-step update (arXiv 2104.00095, SI "Stress calculations",
// eq. mixed_stresses and the multi-body rule; main text "Swimming" for the active stress).
// Three passes: every cell that no body's band reaches takes the pure-fluid divergence at once
// and the rest are listed; then one thread per listed cell computes the face-normal rows of the
// blended stress at its three lower faces, and one per listed cell their divergence.  Templated
// on T.
//
// FP32 storage holds S = xi - x0 (rmt_common.cuh): the stencil differences give grad S =
// grad xi - I, and the neo-Hookean stress is formed from it without cancellation: with
// E = F - I = -F grad S, B - I = E + E^T + E E^T, so the deviator of B keeps the relative
// accuracy of the small strain instead of the absolute accuracy of entries near 1.
#include "rmt_kernels.h"

namespace {

constexpr int TPB = 256;

inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > (long)sm_count() * 64) b = (long)sm_count() * 64;  // grid-stride beyond 64 blocks per SM
  return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------------
// stress: face-normal row of the blended deviatoric stress, then its divergence

template <typename T>
__device__ __forceinline__ bool xget(const Geo& g, const BodyView<T>& v, int i, int j, int k, T x[3]) {
  long c;
  if (!cell_at(g, i, j, k, c)) return false;
  if (v.lay[c] < 0) return false;
  x[0] = v.x[c];
  x[1] = v.x[g.N + c];
  x[2] = v.x[2 * g.N + c];
  return true;
}

// Row tau . e_d at the d-face below cell (i,j,k) (cell a = (i,j,k) - e_d, b = (i,j,k)).
// bmask: bodies that may have xi at a or b.
template <typename T>
__device__ __noinline__ void face_row(const Geo& g, const T* __restrict__ u, const Body* __restrict__ bodies,
                         const BodyView<T>* __restrict__ views, uint64_t bmask, int d, int i, int j, int k,
                         T tt, T row[3]) {
  const T ih = cv<T>(g.ih, g.f.ih);
  int ia[3] = {i, j, k};
  ia[d] -= 1;
  T du[3];
#pragma unroll
  for (int a = 0; a < 3; a++) du[a] = (uval(g, u, a, i, j, k) - uval(g, u, a, ia[0], ia[1], ia[2])) * ih;
  T acc[3] = {T(0), T(0), T(0)};
  T wsum = T(0);
  const T eps = cv<T>(g.eps, g.f.eps);
  while (bmask) {
    const int m = __ffsll((long long)bmask) - 1;
    bmask &= bmask - 1;
    const BodyView<T> v = views[m];
    T xa[3], xb[3];
    if (!xget(g, v, ia[0], ia[1], ia[2], xa) || !xget(g, v, i, j, k, xb)) continue;
    T A[9];
#pragma unroll
    for (int a = 0; a < 3; a++) A[3 * a + d] = (xb[a] - xa[a]) * ih;
    bool ok = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == d) continue;
      int ap[3] = {ia[0], ia[1], ia[2]}, am[3] = {ia[0], ia[1], ia[2]};
      int bp[3] = {i, j, k}, bm[3] = {i, j, k};
      ap[e]++; am[e]--; bp[e]++; bm[e]--;
      T v1[3], v2[3], v3[3], v4[3];
      if (!xget(g, v, ap[0], ap[1], ap[2], v1) || !xget(g, v, bp[0], bp[1], bp[2], v2) ||
          !xget(g, v, am[0], am[1], am[2], v3) || !xget(g, v, bm[0], bm[1], bm[2], v4)) {
        ok = false;
        break;
      }
#pragma unroll
      for (int a = 0; a < 3; a++) A[3 * a + e] = (v1[a] + v2[a] - v3[a] - v4[a]) * (T(0.25) * ih);
    }
    if (!ok) continue;
    const Body& B = bodies[m];
    // xi at the face, relative to the body centre
    T r[3];
    if constexpr (disp_storage<T>()) {
      const int ib[3] = {i, j, k};
#pragma unroll
      for (int a = 0; a < 3; a++)
        r[a] = cell_rel<T>(g, B, a, ib[a]) + T(0.5) * (xa[a] + xb[a]) - (a == d ? T(0.5) * g.f.h : T(0));
    } else {
      const T xf[3] = {T(0.5) * (xa[0] + xb[0]), T(0.5) * (xa[1] + xb[1]), T(0.5) * (xa[2] + xb[2])};
#pragma unroll
      for (int a = 0; a < 3; a++) r[a] = xf[a] - cv<T>(B.c[a], B.f.c[a]);
    }
    const T ph = disp_storage<T>() ? phi0_r(B, r[0], r[1], r[2]) : phi0(B, T(0.5) * (xa[0] + xb[0]),
                                                                         T(0.5) * (xa[1] + xb[1]),
                                                                         T(0.5) * (xa[2] + xb[2]));
    const T w = T(1) - heavi(ph, eps);
    if (!(w > T(0))) continue;
    T F[9];
    const T G = cv<T>(B.G, B.f.G);
    T tau[3];
    if constexpr (disp_storage<T>()) {
      // A = grad S; F = (I + A)^-1, E = F - I = -F A; row d of dev(B) from B - I = E + E^T + E E^T
      T M[9];
#pragma unroll
      for (int q = 0; q < 9; q++) M[q] = A[q] + ((q == 0 || q == 4 || q == 8) ? T(1) : T(0));
      if (!inv3(M, F)) continue;
      T E[9];
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) E[3 * a + b] = -(F[3 * a] * A[b] + F[3 * a + 1] * A[3 + b] + F[3 * a + 2] * A[6 + b]);
      T Kd[3];
#pragma unroll
      for (int a = 0; a < 3; a++)
        Kd[a] = E[3 * a + d] + E[3 * d + a] + E[3 * a] * E[3 * d] + E[3 * a + 1] * E[3 * d + 1] +
                E[3 * a + 2] * E[3 * d + 2];
      T ee = T(0);
#pragma unroll
      for (int q = 0; q < 9; q++) ee += E[q] * E[q];
      const T tr3 = (T(2) * (E[0] + E[4] + E[8]) + ee) * T(1.0 / 3.0);
#pragma unroll
      for (int a = 0; a < 3; a++) tau[a] = G * (Kd[a] - (a == d ? tr3 : T(0)));
    } else {
      if (!inv3(A, F)) continue;
      // neo-Hookean: tau = G (F F^T - tr/3 I); only row d is needed (tau is symmetric)
      T Bd[3];
#pragma unroll
      for (int a = 0; a < 3; a++) Bd[a] = F[3 * a] * F[3 * d] + F[3 * a + 1] * F[3 * d + 1] + F[3 * a + 2] * F[3 * d + 2];
      const T tr3 = (F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3] + F[4] * F[4] + F[5] * F[5] +
                     F[6] * F[6] + F[7] * F[7] + F[8] * F[8]) / T(3);
#pragma unroll
      for (int a = 0; a < 3; a++) tau[a] = G * (Bd[a] - (a == d ? tr3 : T(0)));
    }
    if (B.actA != 0.0) {
      // active stress (3 Z s0 / 2)(e e^T - I/3), e = F E_X / |F E_X|, s0 = A sin(2 pi X/l - w t)
      const T Xb = cv<T>(B.R[0], B.f.R[0]) * r[0] + cv<T>(B.R[3], B.f.R[3]) * r[1] + cv<T>(B.R[6], B.f.R[6]) * r[2];
      const T Zb = cv<T>(B.R[2], B.f.R[2]) * r[0] + cv<T>(B.R[5], B.f.R[5]) * r[1] + cv<T>(B.R[8], B.f.R[8]) * r[2];
      const T s0 = cv<T>(B.actA, B.f.actA) * sin(T(2.0 * RMT_PI) * Xb / cv<T>(B.actL, B.f.actL) - cv<T>(B.actW, B.f.actW) * tt);
      const T EX[3] = {cv<T>(B.R[0], B.f.R[0]), cv<T>(B.R[3], B.f.R[3]), cv<T>(B.R[6], B.f.R[6])};
      T f[3];
#pragma unroll
      for (int a = 0; a < 3; a++) f[a] = F[3 * a] * EX[0] + F[3 * a + 1] * EX[1] + F[3 * a + 2] * EX[2];
      const T fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
      const T amp = T(1.5) * Zb * s0;
      const T ed = f[d] / fn;
#pragma unroll
      for (int a = 0; a < 3; a++) tau[a] += amp * ((f[a] / fn) * ed - (a == d ? T(1.0 / 3.0) : T(0)));
    }
    const T visc = cv<T>(B.mu_a, B.f.mu_a) * (T(1) + cv<T>(B.gamma_t, B.f.gamma_t) * eps * dheavi(ph, eps));
#pragma unroll
    for (int a = 0; a < 3; a++) acc[a] += w * (tau[a] + visc * du[a]);
    wsum += w;
  }
  const T Hf = wsum < T(1) ? T(1) - wsum : T(0);
  const T sc = wsum > T(1) ? T(1) / wsum : T(1);
  const T mu = cv<T>(g.mu, g.f.mu);
#pragma unroll
  for (int a = 0; a < 3; a++) row[a] = Hf * mu * du[a] + acc[a] * sc;
}

// bodies whose band holds cell (i,j,k): only they can contribute at its six faces
template <typename T>
__device__ __forceinline__ uint64_t cell_bodies(const Geo& g, const BodyView<T>* __restrict__ views, int nb,
                                                const int* sbb, int i, int j, int k, long c) {
  uint64_t bm = 0;
  for (int m = 0; m < nb; m++)
    if (in_box(g, sbb + 6 * m, i, j, k) && views[m].lay[c] >= 0) bm |= (1ull << m);
  return bm;
}

// Pass 1, every cell: cells no body reaches take the pure-fluid divergence mu lap(u) here; the
// others are appended to a list (one atomic per warp and plane) for pass 2.  A block marches
// over SFZ planes of a TILE_X x TILE_Y column, so the body boxes and the tile's body mask are
// set up once per column, and keeps u of the planes below and above in registers.  Every
// neighbour comes from selects (periodic wrap, or the mirrored ghost 2 u_wall - u at a no-slip
// wall), so no warp takes a separate path at the domain's edges.
constexpr int SFZ = 8;
template <typename T>
__global__ void __launch_bounds__(TILE_X* TILE_Y, 8) k_stress_fluid(Geo g, const T* __restrict__ u,
                                                                  const BodyView<T>* __restrict__ views, int nb,
                                                                  const int* __restrict__ bbs, int bstride,
                                                                  T* __restrict__ out, int* __restrict__ list,
                                                                  int* __restrict__ count) {
  __shared__ int sbb[6 * RMT_MAX_BODIES];
  __shared__ unsigned long long tile_mask;
  stage_boxes(bbs, bstride, nb, sbb);
  const int k0 = blockIdx.z * SFZ, k1 = min(k0 + SFZ, g.n[2]);
  if (threadIdx.y == 0) {
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * TILE_Y;
    const int i1 = min(i0 + TILE_X, g.n[0]) - 1, j1 = min(j0 + TILE_Y, g.n[1]) - 1;
    unsigned long long mk = 0;
    for (int base = 0; base < nb; base += 32) {
      const int m = base + threadIdx.x;
      bool hit = false;
      if (m < nb) {
        const int* b = sbb + 6 * m;
        hit = tile_meets_box(g, b, 0, i0, i1) && tile_meets_box(g, b, 1, j0, j1) && tile_meets_box(g, b, 2, k0, k1 - 1);
      }
      mk |= (unsigned long long)__ballot_sync(0xffffffffu, hit) << base;
    }
    if (threadIdx.x == 0) tile_mask = mk;
  }
  __syncthreads();
  const unsigned long long tm = tile_mask;
  const int i = blockIdx.x * TILE_X + threadIdx.x, j = blockIdx.y * TILE_Y + threadIdx.y;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const T ih = cv<T>(g.ih, g.f.ih);
  const T mu = cv<T>(g.mu, g.f.mu);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long sy = n0, sz = (long)n0 * n1;
  // x and y neighbours: offsets from the cell (the cell itself where a wall ghost is used)
  const bool xl = i > 0, xh = i + 1 < n0, yl = j > 0, yh = j + 1 < n1;
  const long oxl = xl ? -1 : (g.per[0] ? n0 - 1 : 0), oxh = xh ? 1 : (g.per[0] ? 1 - n0 : 0);
  const long oyl = yl ? -sy : (g.per[1] ? (n1 - 1) * sy : 0), oyh = yh ? sy : (g.per[1] ? (1 - n1) * sy : 0);
  const bool gxl = !xl && !g.per[0], gxh = !xh && !g.per[0], gyl = !yl && !g.per[1], gyh = !yh && !g.per[1];
  // the plane below the first one and the first one
  auto zoff = [&](int kk) -> long {  // plane index kk in [-1, n2] -> offset of (i, j, kk) (own plane at a wall)
    if (kk < 0) return g.per[2] ? (long)(n2 - 1) * sz : -1;
    if (kk >= n2) return g.per[2] ? 0 : -1;
    return (long)kk * sz;
  };
  const long cij = i + (long)j * sy;
  // win[a][0..2] = u_a at planes k-1, k, k+1; pre[a] = the value stored at plane k+2 (the cell's
  // own plane beyond a wall), loaded one iteration ahead so that two planes of loads are in flight
  T win[3][3], pre[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const T* ua = u + (long)a * g.N + cij;
    const T uk = ua[(long)k0 * sz];
    const long ol = zoff(k0 - 1);
    const T vl = ua[ol >= 0 ? ol : (long)k0 * sz];
    win[a][0] = ol >= 0 ? vl : T(2) * cv<T>(g.wall[4][a], g.f.wall[4][a]) - uk;
    win[a][1] = uk;
    const long o1 = zoff(k0 + 1);
    pre[a] = ua[o1 >= 0 ? o1 : (long)k0 * sz];
  }
  for (int k = k0; k < k1; k++) {
    const long c = cij + (long)k * sz;
    const long oh = zoff(k + 1);
#pragma unroll
    for (int a = 0; a < 3; a++) win[a][2] = oh >= 0 ? pre[a] : T(2) * cv<T>(g.wall[5][a], g.f.wall[5][a]) - win[a][1];
    if (k + 1 < k1) {
      const long o2 = zoff(k + 2);
#pragma unroll
      for (int a = 0; a < 3; a++) pre[a] = u[(long)a * g.N + cij + (o2 >= 0 ? o2 : (long)(k + 1) * sz)];
    }
    uint64_t bm = 0;
    for (unsigned long long r = tm; r; r &= r - 1) {
      const int m = __ffsll((long long)r) - 1;
      if (in_box(g, sbb + 6 * m, i, j, k) && views[m].lay[c] >= 0) bm |= (1ull << m);
    }
    const unsigned act = __activemask();
    const unsigned want = __ballot_sync(act, bm != 0);
    if (bm != 0) {
      const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
      const int leader = __ffs(want) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(count, __popc(want));
      base = __shfl_sync(want, base, leader);
      list[base + __popc(want & ((1u << lane) - 1u))] = (int)c;
    } else {
      // pure fluid around this cell: every face row is mu (u_b - u_a)/h
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const T* ua = u + (long)a * g.N + c;
        const T uc = win[a][1];
        const T wxl = T(2) * cv<T>(g.wall[0][a], g.f.wall[0][a]) - uc, wxh = T(2) * cv<T>(g.wall[1][a], g.f.wall[1][a]) - uc;
        const T wyl = T(2) * cv<T>(g.wall[2][a], g.f.wall[2][a]) - uc, wyh = T(2) * cv<T>(g.wall[3][a], g.f.wall[3][a]) - uc;
        const T vxl = ua[oxl], vxh = ua[oxh], vyl = ua[oyl], vyh = ua[oyh];
        const T nb6[6] = {gxl ? wxl : vxl, gxh ? wxh : vxh, gyl ? wyl : vyl, gyh ? wyh : vyh, win[a][0], win[a][2]};
        T acc = T(0);
#pragma unroll
        for (int d = 0; d < 3; d++)
          acc += (mu * ((nb6[2 * d + 1] - uc) * ih) - mu * ((uc - nb6[2 * d]) * ih)) * ih;
        out[a * g.N + c] = acc;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      win[a][0] = win[a][1];
      win[a][1] = win[a][2];
    }
  }
}

// Pass 2, the listed cells (a body's band reaches them): the blended face row of each listed
// cell's three lower faces (the face below the cell along d), one thread per cell, into rows
// (nine cell arrays, row component a of the d-face at 3d+a).  A face row depends only on the face:
// a body contributes where it holds both cells of the face, and every such body is in the mask of
// either cell, so each face is computed once.
struct Rows9 {
  void* r[9];
};
template <typename T>
__global__ void __launch_bounds__(128) k_stress_rows(Geo g, const T* __restrict__ u, const Body* __restrict__ bodies,
                                                      const BodyView<T>* __restrict__ views, int nb,
                                                      const int* __restrict__ bbs, int bstride,
                                                      const double* __restrict__ t, double toff,
                                                      const int* __restrict__ list, const int* __restrict__ count,
                                                      Rows9 R) {
  __shared__ int sbb[6 * RMT_MAX_BODIES];
  stage_boxes(bbs, bstride, nb, sbb);
  const int n = *count;
  const T tt = (T)(*t + toff);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long c = list[e];
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    const uint64_t bm = cell_bodies(g, views, nb, sbb, i, j, k, c);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      T rm[3];
      face_row(g, u, bodies, views, bm, d, i, j, k, tt, rm);
#pragma unroll
      for (int a = 0; a < 3; a++) ((T*)R.r[3 * d + a])[c] = rm[a];
    }
  }
}

// Pass 3, the listed cells: divergence of the face rows.  The upper face along d is the lower
// face of the neighbour above: its row is read from rows where that neighbour is listed, and
// computed here otherwise (the band region's outer faces and the faces on a wall).
template <typename T>
__global__ void __launch_bounds__(128) k_stress_band(Geo g, const T* __restrict__ u, const Body* __restrict__ bodies,
                                                      const BodyView<T>* __restrict__ views, int nb,
                                                      const int* __restrict__ bbs, int bstride,
                                                      const double* __restrict__ t, double toff,
                                                      const int* __restrict__ list, const int* __restrict__ count,
                                                      Rows9 R, T* __restrict__ out) {
  __shared__ int sbb[6 * RMT_MAX_BODIES];
  stage_boxes(bbs, bstride, nb, sbb);
  const int n = *count;
  const T tt = (T)(*t + toff);
  const T ih = cv<T>(g.ih, g.f.ih);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const long c = list[e];
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    uint64_t bm = 0;
    bool have_bm = false;
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      int ip[3] = {i, j, k};
      ip[d] += 1;
      T rp[3];
      long cn;
      if (cell_at(g, ip[0], ip[1], ip[2], cn) && cell_bodies(g, views, nb, sbb, ip[0], ip[1], ip[2], cn) != 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) rp[a] = ((const T*)R.r[3 * d + a])[cn];
      } else {
        if (!have_bm) {
          bm = cell_bodies(g, views, nb, sbb, i, j, k, c);
          have_bm = true;
        }
        face_row(g, u, bodies, views, bm, d, ip[0], ip[1], ip[2], tt, rp);
      }
#pragma unroll
      for (int a = 0; a < 3; a++) acc[a] += (rp[a] - ((const T*)R.r[3 * d + a])[c]) * ih;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) out[a * g.N + c] = acc[a];
  }
}

}  // namespace

template <typename T>
cudaError_t launch_stress_div(const Geo& g, const T* u, const Body* bodies, const BodyView<T>* views, int nb,
                              const int* bbs, int bstride, const double* t, double toff, T* out, int* list,
                              int* count, T* const rows[9], cudaStream_t s) {
  const dim3 gr((g.n[0] + TILE_X - 1) / TILE_X, (g.n[1] + TILE_Y - 1) / TILE_Y, (g.n[2] + SFZ - 1) / SFZ);
  const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_stress_fluid<T><<<gr, dim3(TILE_X, TILE_Y), 0, s>>>(g, u, views, nb, bbs, bstride, out, list, count);
  rmt_count_launches(1);
  if (nb == 0) return cudaSuccess;
  Rows9 R;
  for (int q = 0; q < 9; q++) R.r[q] = rows[q];
  k_stress_rows<T><<<sm_count() * 8, 128, 0, s>>>(g, u, bodies, views, nb, bbs, bstride, t, toff, list, count, R);
  rmt_count_launches(1);
  k_stress_band<T><<<sm_count() * 8, 128, 0, s>>>(g, u, bodies, views, nb, bbs, bstride, t, toff, list, count, R,
                                                  out);
  rmt_count_launches(1);
  return cudaSuccess;
}

template cudaError_t launch_stress_div<float>(const Geo&, const float*, const Body*, const BodyView<float>*, int,
                                              const int*, int, const double*, double, float*, int*, int*,
                                              float* const[9], cudaStream_t);
template cudaError_t launch_stress_div<double>(const Geo&, const double*, const Body*, const BodyView<double>*, int,
                                               const int*, int, const double*, double, double*, int*, int*,
                                               double* const[9], cudaStream_t);

// simulated time on the device: t += dt after each step (read by the stress kernels, so that a
// captured step graph needs no per-step parameter)
__global__ void k_tick(double* t, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) t[0] = t[0] + dt;
}
void launch_tick(double* t, double dt, cudaStream_t s) {
  k_tick<<<1, 32, 0, s>>>(t, dt);
  rmt_count_launches(1);
}
