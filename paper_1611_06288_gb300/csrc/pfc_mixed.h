// Mixed-precision time-step solve: FP64 defect correction around an FP32
// multigrid solve of the linearised split system.
//
// Outer loop (FP64): r = S - N(u) with the FP64 operator of Eqs. 5.4-5.6, the
// RMS of r checked against the tolerance, and q = f'(phi) + (1-eps)/2 (the
// Jacobian of the cubic term of Eq. 5.2 at the current phi) formed in FP64.
// Inner solve (FP32): J d = r with
//   J1 d = d_phi - tau Lap d_mu
//   J2 d = d_mu - q d_phi - Lap d_om
//   J3 d = d_om - Lap d_phi / 2
// by V-cycles of red-black Gauss-Seidel with the same pointwise 3x3 system as
// the FP64 smoother (q frozen), 8-cell restriction of the residual and of q,
// and trilinear prolongation of the correction.  Then u += d in FP64.
// The fixed point is the FP64 solution of N(u) = S: the FP32 part only
// computes corrections.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "pfc.h"
#include "pfc_device.cuh"
#include "pfc_internal.h"

namespace pfc {

constexpr int kMaxLevelsMixed = 24;

struct MixedBufs {
  float* d[kMaxLevelsMixed][3];   // correction (d_phi, d_mu, d_om) per level
  float* t[kMaxLevelsMixed][3];   // Jacobi ping-pong partner of d
  float* r[kMaxLevelsMixed][3];   // right-hand side per level
  float* q[kMaxLevelsMixed];      // frozen cubic-term Jacobian + (1-eps)/2
};

template <class Take>
void mixed_carve(MixedBufs* mx, int n, int nl, const int* sizes, Take take) {
  (void)n;
  for (int l = 0; l < nl; ++l) {
    const size_t m3 = (size_t)sizes[l] * sizes[l] * sizes[l];
    for (int c = 0; c < 3; ++c) mx->d[l][c] = take(m3);
    for (int c = 0; c < 3; ++c) mx->t[l][c] = take(m3);
    for (int c = 0; c < 3; ++c) mx->r[l][c] = take(m3);
    mx->q[l] = take(m3);
  }
}

// FP64 defect r = S - N(u) -> FP32 r and q on level 0, and the sum of |r|^2 at
// dout[0] (two launches).
cudaError_t mixed_enqueue_defect(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                 double* const S[3], const double* b, double* partials,
                                 double* dout, cudaStream_t st, Prof* pr);

// One defect correction after mixed_enqueue_defect: q restricted to every
// level, p.inner_cycles FP32 V-cycles on J d = r from d = 0, then u += d.
cudaError_t mixed_enqueue_correction(MixedBufs& mx, const pfc_params& p, int nl,
                                     const int* sizes, double* const u[3], cudaStream_t st,
                                     Prof* pr);

// Primitive launches of the FP32 kernels (for the C ABI checks).
cudaError_t launch_residual64_to32(const Lvl& L, const double* phi, const double* mu,
                                   const double* om, const double* S1, const double* S2,
                                   const double* S3, const double* b, float* r1, float* r2,
                                   float* r3, float* q, double* partials, double* out,
                                   cudaStream_t st);
cudaError_t launch_lin_smooth32(const Lvl& L, int sweeps, bool zero_init, float* d1,
                                float* d2, float* d3, const float* r1, const float* r2,
                                const float* r3, const float* q, cudaStream_t st);
cudaError_t launch_lin_jacobi32(const Lvl& L, int sweeps, float w, bool zero_init,
                                float* d1, float* d2, float* d3, float* t1, float* t2,
                                float* t3, const float* r1, const float* r2, const float* r3,
                                const float* q, cudaStream_t st);
cudaError_t launch_correct64(int n, double* u1, double* u2, double* u3, const float* d1,
                             const float* d2, const float* d3, cudaStream_t st);

}  // namespace pfc
