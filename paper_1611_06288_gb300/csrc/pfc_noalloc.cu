// Residual norm with library-owned, statically allocated device scratch.
//
// pfc_op_residual_norm needs a caller-provided scratch buffer for its per-block
// partial sums.  This variant keeps those partial sums in a fixed array that
// is part of the library image itself, so the caller passes only inputs and
// the output: nothing is allocated, by the caller or by the library.
#include <math.h>
#include <stdio.h>

#include "pfc_internal.h"

namespace pfc {
namespace {

constexpr int kTile = 256;                       // cells per partial sum
constexpr int kMaxPartials = 65536;              // => at most 256^3 cells
constexpr int64_t kMaxCells = (int64_t)kMaxPartials * kTile;

// One partial sum per 256-cell tile, then the final sum in the last slot.
// Loaded with the library, held by every GPU that loads it until exit
// (512 KiB + 64 B).  All calls on a device share it.
static __device__ __align__(256) double g_scratch[kMaxPartials + 8];

// Device address of g_scratch in the current context.  In host code the name
// g_scratch denotes a host-side stand-in, not device memory, so the address
// is asked of the runtime with the caller's device current.  It is looked up
// on every call rather than cached: after a cudaDeviceReset, or in another
// context of the same device, the module is loaded again and the array may
// sit elsewhere.  The lookup is a host-side table query.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// Sum over the tile of r1^2 + r2^2 + r3^2 -> partials[tile].  Every tile
// writes its slot, so nothing has to be cleared between calls.
__global__ void k_residual_norm2_tiles(Lvl L, const double* __restrict__ phi,
                                       const double* __restrict__ mu,
                                       const double* __restrict__ om,
                                       const double* __restrict__ S1,
                                       const double* __restrict__ S2,
                                       const double* __restrict__ S3,
                                       const double* __restrict__ b, double* partials) {
  __shared__ double sm[32];
  const int n = L.n;
  const int64_t cells = (int64_t)n * n * n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (t < cells) {
    const int i = (int)(t % n);
    const int64_t r = t / n;
    const Stencil s = stencil_at(i, (int)(r % n), (int)(r / n), n);
    double x, y, z;
    residual_at(L, s, phi, mu, om, S1, S2, S3, b, x, y, z);
    acc[0] = fma(x, x, fma(y, y, z * z));
  }
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// Fixed-order sum of the tile partials into partials[kMaxPartials].
__global__ void k_sum_tiles(double* partials, int ntiles) {
  __shared__ double sm[32];
  double acc[1] = {0.0};
  for (int p = threadIdx.x; p < ntiles; p += blockDim.x) acc[0] += partials[p];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partials[kMaxPartials] = acc[0];
}

}  // namespace
}  // namespace pfc

using namespace pfc;

extern "C" int pfc_op_residual_norm_static(int n, double h, double eps, double tau,
                                           const double* phi, const double* mu,
                                           const double* om, const double* S1,
                                           const double* S2, const double* S3,
                                           const double* b, double* out, void* stream) {
  // the same argument checks as pfc_op_residual_norm
  if (n < 2 || !(h > 0) || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !out)
    return PFC_EINVAL;
  const int64_t cells = (int64_t)n * n * n;
  if (cells > kMaxCells) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "pfc_op_residual_norm_static: n = %d exceeds the static scratch limit of "
             "256^3 cells; use pfc_op_residual_norm with caller scratch",
             n);
    set_last_error(msg);
    return PFC_ESIZE;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_last_error("pfc_op_residual_norm_static: cudaGetSymbolAddress failed");
    return PFC_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ntiles = (int)((cells + kTile - 1) / kTile);
  // cudaLaunchKernelEx returns the status of this launch alone, so an
  // earlier, unrelated launch error of the caller's thread is neither
  // reported as this call's nor cleared.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ntiles);
  cfg.blockDim = dim3(kTile);
  cfg.stream = st;
  const Lvl lv = make_lvl(n, h, eps, tau);
  e = cudaLaunchKernelEx(&cfg, k_residual_norm2_tiles, lv, phi, mu, om, S1, S2, S3, b, scratch);
  if (e == cudaSuccess) {
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(1024);
    e = cudaLaunchKernelEx(&cfg, k_sum_tiles, scratch, ntiles);
  }
  double sum = 0.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&sum, scratch + kMaxPartials, sizeof(double), cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return PFC_ECUDA;
  }
  *out = sqrt(sum / (3.0 * (double)cells));
  return PFC_OK;
}
