// Diagnostics of one body (main text "Swimming"; SI "Swimming statistics"; SI "Pre-stretched
// sphere", eq. elas): the centroid velocity, the active power P = -int sigma_a : grad u dV, the
// volume, the elastic energy int G/2 (tr(F^T F) - 3 - 2 ln J) dV and the RMS of J - 1, every
// sum weighted by the body's solid fraction 1 - H_eps(phi) over the cells that hold its
// reference map.  Cell-centred centred differences for grad xi and grad u; F = (grad xi)^-1;
// the active stress of the stress calculation at the cell centre, at the current time.  A
// cell with a missing neighbour value of xi or det(grad xi) <= 0 adds to the centroid
// velocity and the volume only.  Accumulated in FP64 with a fixed-order two-stage reduction,
// so repeated calls agree bit for bit.  FP32 storage holds S = xi - x0 (rmt_common.cuh):
// grad xi = I + grad S, and xi - c = (x0 - c) + S, both formed in FP64.
#include "rmt_kernels.h"

namespace {

constexpr int DTPB = 256;
constexpr int DBLOCKS = 608;  // fixed width: the same summation order on every GPU
constexpr int NS = 8;  // partial sums per block

template <typename T>
__device__ __forceinline__ bool xi_at(const Geo& g, const BodyView<T>& v, int i, int j, int k, double x[3]) {
  long c;
  if (!cell_at(g, i, j, k, c) || v.lay[c] < 0) return false;
  x[0] = (double)v.x[c];
  x[1] = (double)v.x[g.N + c];
  x[2] = (double)v.x[2 * g.N + c];
  return true;
}

// per block: sums of w u (3), w, w sigma_a : grad u, w Phi_elas, w (over cells with F), w (J-1)^2.
// The per-cell arithmetic is FP64 for both storage types: the energy density is a small
// difference of O(1) terms at small strain, and only the body's cells take this branch.
template <typename T>
__global__ void __launch_bounds__(DTPB) k_body_stats(Geo g, const T* __restrict__ u, Body B, BodyView<T> v,
                                                     const double* __restrict__ tptr, double* __restrict__ part) {
  const double h = g.h, t = *tptr;
  double acc[NS] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  GRID_LOOP(c, g.N) {
    if (v.lay[c] < 0) continue;
    const double w = 1.0 - heavi((double)v.phi[c], g.eps);
    if (!(w > 0.0)) continue;
    for (int a = 0; a < 3; a++) acc[a] += w * (double)u[a * g.N + c];
    acc[3] += w;
    int i, j, k;
    decode(c, g.n[0], g.n[1], i, j, k);
    const int ii[3] = {i, j, k};
    double A[9];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      int p[3] = {i, j, k}, m[3] = {i, j, k};
      p[d]++;
      m[d]--;
      double xp[3], xm[3];
      if (!xi_at(g, v, p[0], p[1], p[2], xp) || !xi_at(g, v, m[0], m[1], m[2], xm)) {
        ok = false;
        break;
      }
#pragma unroll
      for (int a = 0; a < 3; a++) A[3 * a + d] = (xp[a] - xm[a]) / (2.0 * h) + (disp_storage<T>() && a == d ? 1.0 : 0.0);
    }
    if (!ok) continue;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(det > 0.0)) continue;
    double F[9];
    if (!inv3(A, F)) continue;
    double trC = 0.0;
#pragma unroll
    for (int q = 0; q < 9; q++) trC += F[q] * F[q];
    const double J = 1.0 / det;
    acc[5] += w * (0.5 * B.G * (trC - 3.0 - 2.0 * log(J)));
    acc[6] += w;
    acc[7] += w * (J - 1.0) * (J - 1.0);
    if (B.actA == 0.0) continue;
    double r[3] = {(double)v.x[c] - B.c[0], (double)v.x[g.N + c] - B.c[1], (double)v.x[2 * g.N + c] - B.c[2]};
    if constexpr (disp_storage<T>()) {
      for (int a = 0; a < 3; a++) r[a] = cell_rel<double>(g, B, a, ii[a]) + (double)v.x[a * g.N + c];
    }
    const double Xb = B.R[0] * r[0] + B.R[3] * r[1] + B.R[6] * r[2];
    const double Zb = B.R[2] * r[0] + B.R[5] * r[1] + B.R[8] * r[2];
    const double s0 = B.actA * sin(2.0 * RMT_PI * Xb / B.actL - B.actW * t);
    const double EX[3] = {B.R[0], B.R[3], B.R[6]};
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) f[a] = F[3 * a] * EX[0] + F[3 * a + 1] * EX[1] + F[3 * a + 2] * EX[2];
    const double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    const double amp = 1.5 * Zb * s0;
    double sg = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int d = 0; d < 3; d++) {
        int p[3] = {ii[0], ii[1], ii[2]}, m[3] = {ii[0], ii[1], ii[2]};
        p[d]++;
        m[d]--;
        const double gu =
            ((double)uval(g, u, a, p[0], p[1], p[2]) - (double)uval(g, u, a, m[0], m[1], m[2])) / (2.0 * h);
        const double sig = amp * ((f[a] / fn) * (f[d] / fn) - (a == d ? 1.0 / 3.0 : 0.0));
        sg += sig * gu;
      }
    acc[4] += w * sg;
  }
  __shared__ double sh[NS][DTPB / 32];
#pragma unroll
  for (int q = 0; q < NS; q++) {
    double x = acc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double s = 0.0;
    for (int w2 = 0; w2 < DTPB / 32; w2++) s += sh[threadIdx.x][w2];
    part[NS * blockIdx.x + threadIdx.x] = s;
  }
}

__global__ void k_body_stats_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x < NS) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[NS * b + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

}  // namespace

size_t body_stats_scratch_bytes() { return (size_t)(NS * DBLOCKS + NS) * sizeof(double); }

template <typename T>
void launch_body_stats(const Geo& g, const T* u, const Body& b, const BodyView<T>& v, const double* t, double* scratch,
                       cudaStream_t s) {
  k_body_stats<T><<<DBLOCKS, DTPB, 0, s>>>(g, u, b, v, t, scratch + NS);
  rmt_count_launches(1);
  k_body_stats_final<<<1, 32, 0, s>>>(scratch + NS, DBLOCKS, scratch);
  rmt_count_launches(1);
}

template void launch_body_stats<float>(const Geo&, const float*, const Body&, const BodyView<float>&, const double*,
                                       double*, cudaStream_t);
template void launch_body_stats<double>(const Geo&, const double*, const Body&, const BodyView<double>&,
                                        const double*, double*, cudaStream_t);
