// Mixed-precision time-step solves: a defect correction around an FP32
// multigrid solve of the linearised split system.
//
// Outer loop: r = S - N(u) with the operator of Eqs. 5.4-5.6, the RMS of r
// checked against the tolerance, and q = f'(phi) + (1-eps)/2 (the Jacobian of
// the cubic term of Eq. 5.2 at the current phi).  PFC_MIXED keeps phi, mu,
// omega, S2, S3, r, q and the sums in FP64; PFC_MIXED_DF keeps the state in
// double-float (hi, lo) FP32 pairs with a 48-bit significand (pfc_df.cuh) and
// forms q in FP32.
// Inner solve (FP32): J d = r with
//   J1 d = d_phi - tau Lap d_mu
//   J2 d = d_mu - q d_phi - Lap d_om
//   J3 d = d_om - Lap d_phi / 2
// by V-cycles of red-black Gauss-Seidel or damped collective Jacobi with the
// same pointwise 3x3 system as the FP64 smoother (q frozen), 8-cell
// restriction of the residual and of q, and trilinear prolongation of the
// correction.  Then u += d in the outer precision.
// The fixed point is the solution of N(u) = S to the rounding of the outer
// residual: the FP32 part only computes corrections.
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

// The FP32 hierarchy of `members` ensemble members: each level's fields hold
// the members one after another.
template <class Take>
void mixed_carve(MixedBufs* mx, int n, int nl, const int* sizes, Take take, int members = 1) {
  (void)n;
  for (int l = 0; l < nl; ++l) {
    const size_t m3 = (size_t)sizes[l] * sizes[l] * sizes[l] * members;
    for (int c = 0; c < 3; ++c) mx->d[l][c] = take(m3);
    for (int c = 0; c < 3; ++c) mx->t[l][c] = take(m3);
    for (int c = 0; c < 3; ++c) mx->r[l][c] = take(m3);
    mx->q[l] = take(m3);
  }
}

// Defect r = S - N(u) of the FP64 state (PFC_MIXED) -> FP32 r and q on
// level 0, and the FP64 sum of |r|^2 at dout[0] (two launches).
// With `members` > 1 the fields hold an ensemble member after member, each
// member's (1-eps)/2 at c1m[m] and its sum at dout[m].
cudaError_t mixed_enqueue_defect(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                 double* const S[3], const double* b, double* partials,
                                 double* dout, cudaStream_t st, Prof* pr, double* lap,
                                 int members = 1, const double* c1m = nullptr,
                                 double* const M[3] = nullptr, double* lapmu = nullptr,
                                 double* lapom = nullptr, int planes = 0,
                                 const DecideArgs* da = nullptr, bool* decided = nullptr);

// The first defect of a step that starts from the previous step's solution
// (phi := b, mu and omega kept), pointwise from the Laplacians of b, mu and
// omega that the previous step's last defect stored; writes lapb to lap.
cudaError_t mixed_enqueue_defect_point(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                       double* const S[3], const double* b,
                                       const double* lapb, const double* lapmu,
                                       const double* lapom, double* lap, double* partials,
                                       double* dout, cudaStream_t st, Prof* pr, int members,
                                       const double* c1m, const DecideArgs* da = nullptr,
                                       bool* decided = nullptr);

// Start of a warm PFC_MIXED step in one launch (plus its reduction): S2, S3
// into S[1], S[2], phi^{k+1} := b into u[0], and the pointwise first defect
// (as mixed_enqueue_defect_point with those S2, S3); lapc is the stored
// Laplacian of phi^{k-1}.
//
// With da (the step's decision arguments) and a single member, each of
// these three takes the convergence decision in its final reduction kernel
// and sets *decided; otherwise *decided is false and the caller launches the
// decision.
cudaError_t mixed_enqueue_start_point(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                      double* const S[3], const double* b,
                                      const double* lapb, const double* lapc,
                                      const double* lapmu, const double* lapom, double* lap,
                                      double* partials, double* dout, cudaStream_t st, Prof* pr,
                                      int members, const double* c1m,
                                      const DecideArgs* da = nullptr, bool* decided = nullptr);

// Start of a step from u^{k+1} := 2 u^k - u^{k-1} in all three fields
// (u[1], u[2] and lapmu1, lapom1 hold step k-1's mu, omega and their
// Laplacians on entry, the iterate's on exit; u[0] receives phi): S2, S3,
// the iterate, its Laplacians and the first defect in one pointwise pass
// from the stored Laplacians, then the reduction (and decision, as above).
cudaError_t mixed_enqueue_start_extrap(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                       double* const S[3], const double* b, const double* c,
                                       const double* lapb, const double* lapc,
                                       const double* mu0, const double* om0,
                                       const double* lapmu0, const double* lapom0,
                                       double* lapmu1, double* lapom1, double* lap,
                                       double* partials, double* dout, cudaStream_t st,
                                       Prof* pr, int members, const double* c1m,
                                       const DecideArgs* da = nullptr, bool* decided = nullptr);

// Defect r = S - N(u) of the df state -> FP32 r and q on level 0, and the
// sum of |r|^2 at dout[0] (two launches).  S[0] is S1 (= b in a time step).
cudaError_t mixed_enqueue_defect(MixedBufs& mx, const Lvl& L0, float2* const u[3],
                                 float2* const S[3], const float2* b, double* partials,
                                 double* dout, cudaStream_t st, Prof* pr, float2* lap);

// One defect correction after mixed_enqueue_defect: q restricted to every
// level, p.inner_cycles FP32 V-cycles on J d = r from d = 0, then u += d in
// FP64 (PFC_MIXED) or double-float (PFC_MIXED_DF).
cudaError_t mixed_enqueue_correction(MixedBufs& mx, const pfc_params& p, int nl,
                                     const int* sizes, double* const u[3], cudaStream_t st,
                                     Prof* pr, int members = 1, double tau_scale = 1.0);
cudaError_t mixed_enqueue_correction(MixedBufs& mx, const pfc_params& p, int nl,
                                     const int* sizes, float2* const u[3], cudaStream_t st,
                                     Prof* pr);

// S2, S3 of Eqs. 5.9-5.10 from df fields b = phi^k, c = phi^{k-1}.
cudaError_t launch_source_df(const Lvl& L, const float2* b, const float2* c, float2* S2,
                             float2* S3, cudaStream_t st);

// launch_guess on df fields (double-float arithmetic).
cudaError_t launch_guess_df(const Lvl& L, const float2* b, const float2* c, float2* S2,
                            float2* S3, float2* phig, float2* mug, float2* omg,
                            cudaStream_t st);

// The raw sums of launch_diagnostics (out[0..5]) from df fields a = phi^k,
// b = phi^{k-1}, in double-float; partials: kReduceBlocks * 6 float2 slots
// (the FP64 path's partial-sum buffer).
cudaError_t launch_diagnostics_df(int n, const float2* a, const float2* b, double* partials,
                                  double* out, cudaStream_t st);

// The FP64 -> FP32 rounding (nearest, ties to even) and exact FP32 -> FP64
// widening that the FP64 outer loop performs on the integer pipe, on arrays.
cudaError_t launch_round_f32(int64_t count, const double* x, float* y, cudaStream_t st);
cudaError_t launch_widen_f64(int64_t count, const float* x, double* y, cudaStream_t st);

// df counterparts of launch_laplacian, launch_source_cached and
// launch_diagnostics_cached.
cudaError_t launch_laplacian_df(int n, const float2* v, float2* lap, cudaStream_t st);
cudaError_t launch_source_cached_df(const Lvl& L, const float2* b, const float2* lapb,
                                    const float2* lapc, float2* S2, float2* S3, cudaStream_t st);
cudaError_t launch_diagnostics_cached_df(int n, const float2* a, const float2* b,
                                         const float2* lapa, const float2* lapb,
                                         double* partials, double* out, cudaStream_t st);

// Whole-field conversions FP64 <-> df (count cells; in place allowed).
cudaError_t launch_df_from_f64(int64_t count, const double* x, float2* y, cudaStream_t st);
cudaError_t launch_df_to_f64(int64_t count, const float2* y, double* x, cudaStream_t st);

// Adjoint step: J^T psi = (g, 0, 0) is solved as J z = (0, g, 0), psi =
// (z2, z1, 2 z3).  launch_adj_defect64: r = (0, g, 0) - J z in FP64 with q
// at (a, b), to FP32 r, q on level 0, |r|^2 at out[0].  launch_adj_accumulate:
// gk += -(dF/db)^T psi, gkm1 += -(dF/dc)^T psi (gkm1 may equal gk), out[0] =
// -(dF/deps)^T psi.
cudaError_t launch_adj_defect64(const Lvl& L, const double* z1, const double* z2,
                                const double* z3, const double* g, const double* a,
                                const double* b, float* r1, float* r2, float* r3, float* q,
                                double* partials, double* out, cudaStream_t st);
cudaError_t launch_adj_accumulate(const Lvl& L, const double* z1, const double* z2,
                                  const double* z3, const double* a, const double* b,
                                  double* gk, double* gkm1, double* partials, double* out,
                                  cudaStream_t st);

// Primitive launches of the FP32 kernels (for the C ABI checks).
cudaError_t launch_defect64(const Lvl& L, const double* phi, const double* mu,
                            const double* om, const double* S1, const double* S2,
                            const double* S3, const double* b, float* r1, float* r2, float* r3,
                            float* q, double* partials, double* out, cudaStream_t st,
                            double* lap = nullptr, int members = 1,
                            const double* c1m = nullptr, const double* Mx = nullptr,
                            const double* My = nullptr, const double* Mz = nullptr,
                            double* lapmu = nullptr, double* lapom = nullptr,
                            bool pdl = false, int planes = 0, const DecideArgs* da = nullptr,
                            bool* decided = nullptr);
// The pointwise start from u^{k+1} := 2 u^k - u^{k-1} (k_start64_extrap) and
// its reduction to out[member] (for the C ABI checks and the step).
cudaError_t launch_start64_extrap(const Lvl& L, const double* b, const double* c,
                                  const double* lapb, const double* lapc, const double* mu0,
                                  const double* om0, const double* lapmu0,
                                  const double* lapom0, double* mu1, double* om1,
                                  double* lapmu1, double* lapom1, double* S2, double* S3,
                                  double* phi, float* r1, float* r2, float* r3, float* q,
                                  double* partials, double* out, double* lap, cudaStream_t st,
                                  int members = 1, const double* c1m = nullptr,
                                  bool pdl = false, const DecideArgs* da = nullptr,
                                  bool* decided = nullptr);
// Face mobilities M(A phi_*), phi_* = 3/2 b - 1/2 c, M(phi) = m0 + m2 phi^2,
// face i+1/2 of each axis stored at cell i (FP64).
cudaError_t launch_face_mobility(int n, double m0, double m2, const double* b, const double* c,
                                 double* Mx, double* My, double* Mz, cudaStream_t st);
cudaError_t launch_correct64(int n, double* u1, double* u2, double* u3, const float* d1,
                             const float* d2, const float* d3, cudaStream_t st,
                             bool pdl = true, int members = 1);
cudaError_t launch_defect_df(const Lvl& L, const float2* phi, const float2* mu,
                             const float2* om, const float2* S1, const float2* S2,
                             const float2* S3, const float2* b, float* r1, float* r2, float* r3,
                             float* q, double* partials, double* out, cudaStream_t st,
                             float2* lap = nullptr);
cudaError_t launch_lin_residual_restrict32(const Lvl& L, bool zero, const float* d1,
                                          const float* d2, const float* d3, const float* r1,
                                          const float* r2, const float* r3, const float* q,
                                          float* c1, float* c2, float* c3, cudaStream_t st);
// The restriction of launch_lin_residual_restrict32 to c and, in the same
// launch, `extra` (1 or 2) further 8-cell averages to e and g (n/2 a
// multiple of 16).
// q (colour-split, n^3) averaged down 1 + extra levels (extra 0..2; extra > 0
// needs n/2 a multiple of 16); c, e, g the levels produced.
cudaError_t launch_restrict_q(int n, int extra, const float* q, float* c, float* e, float* g,
                              cudaStream_t st);
cudaError_t launch_lin_restrict_chain32(const Lvl& L, bool zero, int extra, const float* d1,
                                       const float* d2, const float* d3, const float* r1,
                                       const float* r2, const float* r3, const float* q,
                                       float* const c[3], float* const e[3], float* const g[3],
                                       cudaStream_t st);
// skip0: the colour-0 cells of d are left untouched (a red-black pass of
// colour 0 recomputes them next).
cudaError_t launch_prolong32(int n, bool assign, bool skip0, const float* e1, const float* e2,
                             const float* e3, float* d1, float* d2, float* d3, cudaStream_t st);
cudaError_t launch_lin_smooth32(const Lvl& L, int sweeps, bool zero_init, float* d1,
                                float* d2, float* d3, const float* r1, const float* r2,
                                const float* r3, const float* q, cudaStream_t st);
// `sweeps` (>= 1) FP32 red-black sweeps whose last colour-1 pass adds d to
// the FP64 state u instead of storing d's colour-1 cells; n % 4 == 0.
cudaError_t launch_lin_smooth_correct32(const Lvl& L, int sweeps, float* d1, float* d2,
                                       float* d3, const float* r1, const float* r2,
                                       const float* r3, const float* q, double* u1, double* u2,
                                       double* u3, cudaStream_t st);

// d (+)= P e (e of (n/2)^3 cells) and one post-smoothing sweep of `kind`
// (PFC_SWEEP_RB or PFC_SWEEP_JACOBI, weight w; t is Jacobi scratch) in one
// fused launch plus the rest of the sweep; n a multiple of 32.
cudaError_t launch_lin_prolong_smooth32(const Lvl& L, int kind, bool assign, float w,
                                       const float* e1, const float* e2, const float* e3,
                                       float* d1, float* d2, float* d3, float* t1, float* t2,
                                       float* t3, const float* r1, const float* r2,
                                       const float* r3, const float* q, cudaStream_t st);
cudaError_t launch_lin_jacobi32(const Lvl& L, int sweeps, float w, bool zero_init,
                                float* d1, float* d2, float* d3, float* t1, float* t2,
                                float* t3, const float* r1, const float* r2, const float* r3,
                                const float* q, cudaStream_t st);
cudaError_t launch_correct_df(int n, float2* u1, float2* u2, float2* u3, const float* d1,
                              const float* d2, const float* d3, cudaStream_t st,
                              bool pdl = true);

}  // namespace pfc
