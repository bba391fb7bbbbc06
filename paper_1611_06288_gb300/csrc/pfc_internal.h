// Host-side launchers shared by the C ABI (pfc_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pfc.h"
#include "pfc_device.cuh"

namespace pfc {

// Largest number of partial sums a reduction writes (one per block).
constexpr int kReduceBlocks = 1216;   // 8 * 152 SMs
constexpr int kReduceThreads = 256;
constexpr int kReduceComps = 8;       // doubles per block partial

// Event timing of kernel launches per (class, level); see pfc_profile_enable.
struct Prof {
  static constexpr int kPool = 1024;
  unsigned mask = 0;
  bool created = false;
  int pending = 0;
  cudaEvent_t ev[2 * kPool];
  int cls[kPool], lev[kPool], nlaunch[kPool];
  double ms[PFC_K_COUNT][PFC_PROFILE_LEVELS];
  long long cnt[PFC_K_COUNT][PFC_PROFILE_LEVELS];
  long long launches = 0;   // every kernel launch of the context, timed or not
};
// Convergence state of one time step, kept in device memory and read back
// once per step (graph mode) or once per cycle (timed mode).
struct StepState {
  double rms0;   // RMS residual of the initial guess
  double rms;    // latest RMS residual
  int iters;     // V-cycles (FP64) or defect corrections (mixed) done
  int status;    // kStepRunning, kStepConverged, kStepNaN, kStepNoConv
};
constexpr int kStepRunning = 0, kStepConverged = 1, kStepNaN = 2, kStepNoConv = 3;

// One member's convergence decision from its sum of squared residuals: the
// RMS residual against the tolerance, NaN, the cycle budget; a member that
// has converged stays converged.  running / failed report the new status.
__device__ __forceinline__ void decide_member(StepState& st, double sum, double inv_3n3,
                                              double tol, int max_iter, int first, int& running,
                                              int& failed) {
  const double rms = sqrt(sum * inv_3n3);
  if (first) {
    st.iters = 0;
    st.rms0 = rms;
    st.status = kStepRunning;
  }
  if (first || st.status == kStepRunning) {
    if (!first) st.iters += 1;
    st.rms = rms;
    int status;
    if (rms <= tol)
      status = kStepConverged;
    else if (!isfinite(rms))
      status = kStepNaN;
    else if (st.iters >= max_iter)
      status = kStepNoConv;
    else
      status = kStepRunning;
    st.status = status;
  } else if (st.status == kStepConverged) {
    st.rms = rms;
  }
  running = st.status == kStepRunning;
  failed = st.status == kStepNaN || st.status == kStepNoConv;
}

// The decision of a single-member step taken by the kernel that reduces its
// residual (one launch instead of two): the arguments of launch_decide.
struct DecideArgs {
  cudaGraphConditionalHandle handle;
  int use_handle;
  StepState* state;
  double inv_3n3, tol;
  int max_iter, first;
};

// From the reduced sums of squared residuals sum[m] of `members` ensemble
// members (1 for a single problem): update state[m] (a converged member stays
// converged) and, if use_handle, set the WHILE condition of the step graph to
// "keep going" while some member runs and none has failed.
cudaError_t launch_decide(cudaGraphConditionalHandle handle, int use_handle,
                          const double* sum, StepState* state, double inv_3n3, double tol,
                          int max_iter, int first, cudaStream_t st, int members = 1,
                          bool pdl = false);

// Convergence states of the contexts of a group (pfc_group_*), passed to the
// group decision by value: no device memory beyond the contexts' own.
constexpr int kMaxGroup = PFC_MAX_GROUP;
struct GroupStates {
  const StepState* s[kMaxGroup];
  int members[kMaxGroup];
  int count;
};

// Set, per context of a group, the IF condition of its loop body: the
// context still has a running member (and no member of any context failed).
struct GroupHandles {
  cudaGraphConditionalHandle h[kMaxGroup];
};
cudaError_t launch_group_select(const GroupHandles& hs, const GroupStates& g,
                                cudaStream_t st);

// Set the WHILE condition of a group's step graph: "keep going" while some
// member of some context runs and no member of any context has failed (the
// per-context states are those the contexts' own decisions wrote).
cudaError_t launch_group_decide(cudaGraphConditionalHandle handle, const GroupStates& g,
                                cudaStream_t st);

// Detail string returned by pfc_last_error() on this host thread.
void set_last_error(const char* msg);

// No-ops unless pr is non-null and the class is enabled.
void prof_begin(Prof* pr, int cls, cudaStream_t st);
void prof_end(Prof* pr, int cls, int level, int nlaunch, cudaStream_t st);
// Accumulate the completed brackets (call after the stream has synchronised).
void prof_harvest(Prof* pr);

// FP64 kernels (pfc_fp64.cu).  All enqueue on `st` and return the launch error.
// S2, S3 and the extrapolated initial iterate (phi_g, mu_g, omega_g) of a
// step from b = phi^k, c = phi^{k-1} (two launches).
// PFC_GUESS_EXTRAPOLATE_ALL's initial iterate (k_guess_all): phi = 2b - c,
// m1 = 2 m0 - m1, o1 = 2 o0 - o1 (extrap), else phi = b, m1 = m0, o1 = o0.
cudaError_t launch_guess_all(int64_t cells, bool extrap, const double* b, const double* c,
                             const double* m0, const double* o0, double* m1, double* o1,
                             double* phi, cudaStream_t st, bool pdl);
cudaError_t launch_guess(const Lvl& L, const double* b, const double* c, double* S2,
                         double* S3, double* phig, double* mug, double* omg, cudaStream_t st);
cudaError_t launch_source(const Lvl& L, const double* b, const double* c, double* S2,
                          double* S3, cudaStream_t st);
cudaError_t launch_smooth(const Lvl& L, int lin, int sweeps, double* phi, double* mu,
                          double* om, const double* S1, const double* S2,
                          const double* S3, const double* b, cudaStream_t st);
// `sweeps` damped collective Jacobi sweeps ping-ponging through t1..3; the
// result is left in phi, mu, om.
cudaError_t launch_jacobi(const Lvl& L, int lin, int sweeps, double w, double* phi,
                          double* mu, double* om, double* t1, double* t2, double* t3,
                          const double* S1, const double* S2, const double* S3,
                          const double* b, cudaStream_t st);
cudaError_t launch_residual(const Lvl& L, const double* phi, const double* mu,
                            const double* om, const double* S1, const double* S2,
                            const double* S3, const double* b, double* r1, double* r2,
                            double* r3, cudaStream_t st);
cudaError_t launch_residual_restrict(const Lvl& L, const double* phi, const double* mu,
                                     const double* om, const double* S1,
                                     const double* S2, const double* S3, const double* b,
                                     double* rc1, double* rc2, double* rc3, double* uc1,
                                     double* uc2, double* uc3, double* wc1, double* wc2,
                                     double* wc3, cudaStream_t st);
cudaError_t launch_restrict(int n, const double* fine, double* coarse, cudaStream_t st);
cudaError_t launch_coarse_source(const Lvl& Lc, const double* uc1, const double* uc2,
                                 const double* uc3, const double* bc, double* r1,
                                 double* r2, double* r3, cudaStream_t st);
// e_c = v_c - w_c in place over w_c (three coarse fields of size nc^3).
cudaError_t launch_coarse_diff(int nc, const double* v1, const double* v2,
                               const double* v3, double* w1, double* w2, double* w3,
                               cudaStream_t st);
// u += P e_c for a fine level of size n (e_c on n/2).
cudaError_t launch_prolong_add(int n, const double* e1, const double* e2,
                               const double* e3, double* u1, double* u2, double* u3,
                               cudaStream_t st);
cudaError_t launch_coarse_solve(const Lvl& L, int lin, int kind, double w, int max_sweeps,
                                double* phi, double* mu, double* om, double* t1, double* t2,
                                double* t3, const double* S1, const double* S2,
                                const double* S3, const double* b, cudaStream_t st);

// Smoother kind of a level of spacing h under the parameters' policy.
inline int level_kind(const pfc_params* p, double h) {
  if (p->policy == PFC_POLICY_RB) return PFC_SWEEP_RB;
  const double s = 108.0 * p->dt / (h * h * h * h * h * h);
  return (s > p->stiff_lo && s < p->stiff_hi) ? PFC_SWEEP_JACOBI : PFC_SWEEP_RB;
}
// Sum over cells of r1^2 + r2^2 + r3^2 -> partials (one per block), then the
// fixed-order final sum into out[0] (device).
// lap (may be null) receives the unscaled Laplacian of phi.
cudaError_t launch_residual_norm2(const Lvl& L, const double* phi, const double* mu,
                                  const double* om, const double* S1, const double* S2,
                                  const double* S3, const double* b, double* partials,
                                  double* out, cudaStream_t st, double* lap = nullptr);
// Unscaled 7-point Laplacian (neighbour sum - 6 centre) of a field.
cudaError_t launch_laplacian(int n, const double* v, double* lap, cudaStream_t st,
                             int members = 1);
// S2, S3 from b and the stored unscaled Laplacians of b and c.
cudaError_t launch_source_cached(const Lvl& L, const double* b, const double* lapb,
                                 const double* lapc, double* S2, double* S3, cudaStream_t st,
                                 int members = 1, const double* c1m = nullptr, bool pdl = false);
// launch_diagnostics from the stored unscaled Laplacians of a and b.
// state_out (optional, with state): the final reduction also copies the
// members' step states there; out and state_out may be mapped host memory.
cudaError_t launch_diagnostics_cached(int n, const double* a, const double* b,
                                      const double* lapa, const double* lapb, double* partials,
                                      double* out, cudaStream_t st, int members = 1,
                                      bool pdl = false, const StepState* state = nullptr,
                                      StepState* state_out = nullptr);
// out[0..5] = sum a^4, sum a^2, sum |D a|^2 (faces), sum (Lap a)^2 (times h^4
// removed: raw stencil sums), sum |D(a-b)|^2, sum a.  Raw sums; the host scales.
cudaError_t launch_diagnostics(int n, const double* a, const double* b, double* partials,
                               double* out, cudaStream_t st);

}  // namespace pfc
