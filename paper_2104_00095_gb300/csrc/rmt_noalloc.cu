// rmt_extrapolate_noalloc: the reference-map extrapolation of one body (classification,
// layer marking, least-squares fits) on buffers the caller owns, without any allocation.
//
// Some callers cannot allocate device memory while they run this step: a host application
// that has handed its whole memory budget to its own pool, code that runs while another
// component holds the allocator, or a pipeline that must not call cudaMalloc (it may
// synchronise the device).  The grid API (rmt_create_grid ...) allocates its own state, so
// those callers use this entry point instead.  The scratch the pipeline needs (the compacted
// list of band cells, its length, the band's bounding box and the count of degenerate fits)
// lives in one file-scope __device__ array of fixed size; every GPU that loads the library
// holds it until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "rmt.h"
#include "rmt_kernels.h"

namespace {

// largest grid (cells) the static scratch serves: every band cell needs one list entry and a
// band never holds more cells than the grid
constexpr long NOALLOC_MAX_CELLS = 1L << 21;  // 2,097,152 cells, e.g. 128^3
// layout of the scratch (ints): [0, 16) the band list's counters (BAND_COUNTERS of them),
// [16, 22) bounding box, [22] degenerate-fit counter; [64, 64 + NOALLOC_MAX_CELLS) the band list
constexpr long SCR_COUNT = 0, SCR_BB = 16, SCR_ERR = 22, SCR_LIST = 64;
static_assert(BAND_COUNTERS <= SCR_BB && SCR_ERR < SCR_LIST, "scratch layout");
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) int g_noalloc_scratch[SCR_LIST + NOALLOC_MAX_CELLS];

std::mutex g_setup_mutex;
int* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch on the current device; resolved once per device (the host
// symbol itself is not a device address).
cudaError_t scratch_for_current_device(int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (int*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

rmt_status rmt_extrapolate_noalloc(const rmt_grid_desc* d, const rmt_solid_desc* s, const double* xi_in,
                                   double* xi_out, double* phi_out, signed char* layer_out, void* stream) {
  if (!d || !s || !xi_in || !xi_out || !phi_out || !layer_out) return RMT_EINVAL;
  Geo G;
  memset(&G, 0, sizeof G);
  for (int a = 0; a < 3; a++) {
    if (d->n[a] < 4 || !(d->hi[a] > d->lo[a])) return RMT_EINVAL;
    const int p0 = d->bc[2 * a] == RMT_BC_PERIODIC, p1 = d->bc[2 * a + 1] == RMT_BC_PERIODIC;
    if (p0 != p1) return RMT_EINVAL;
    G.n[a] = d->n[a];
    G.per[a] = p0;
    G.nn[a] = p0 ? d->n[a] : d->n[a] + 1;
    G.lo[a] = d->lo[a];
    G.len[a] = d->hi[a] - d->lo[a];
  }
  G.h = (d->hi[0] - d->lo[0]) / d->n[0];
  for (int a = 1; a < 3; a++)
    if (fabs((d->hi[a] - d->lo[a]) / d->n[a] - G.h) > 1e-12 * G.h) return RMT_EINVAL;
  if (d->band_layers < 1 || d->band_layers > 8) return RMT_EINVAL;
  G.N = (long)G.n[0] * G.n[1] * G.n[2];
  G.NN = (long)G.nn[0] * G.nn[1] * G.nn[2];
  G.layers = d->band_layers;
  G.eps = d->eps_h * G.h;
  if (G.N > NOALLOC_MAX_CELLS) return RMT_EINVAL;  // the band list could outgrow the static scratch
  if (s->shape != RMT_SHAPE_SPHERE && s->shape != RMT_SHAPE_ELLIPSOID) return RMT_EINVAL;
  Body b;
  b.shape = s->shape;
  for (int a = 0; a < 3; a++) {
    b.c[a] = s->center[a];
    b.a[a] = s->semi_axes[a];
  }
  for (int q = 0; q < 9; q++) b.R[q] = s->rot[q];
  b.rho_s = s->rho_s;
  b.G = s->G;
  b.mu_a = s->mu_a;
  b.gamma_t = s->gamma_t;
  b.actA = s->active_A;
  b.actW = s->active_omega;
  b.actL = s->active_len;
  b.repA = s->rep_A;
  body_finish(b);
  geo_finish(G);
  body_image(b, G);

  cudaStream_t st = (cudaStream_t)stream;
  int* scr = nullptr;
  cudaError_t e = scratch_for_current_device(&scr);
  if (e != cudaSuccess) return RMT_ECUDA;
  // the degenerate-fit counter must start at zero (the count is cleared by the pipeline itself)
  e = cudaMemsetAsync(scr + SCR_ERR, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xi_out, xi_in, 3 * G.N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return RMT_ECUDA;
  const long wide = (long)sm_count() * 64;
  const int blocks = (int)((G.N + 127) / 128 < wide ? (G.N + 127) / 128 : wide);
  e = launch_extrapolate<double>(G, b, nullptr, scr + SCR_BB, blocks, scr + SCR_LIST, scr + SCR_COUNT, nullptr,
                                 sm_count() * 4,
                                 xi_out, phi_out, (int8_t*)layer_out, scr + SCR_ERR, st);
  int nbad = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, scr + SCR_ERR, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return RMT_ECUDA;
  if (nbad) return RMT_EDEGENERATE;
  return RMT_OK;
}

}  // extern "C"
