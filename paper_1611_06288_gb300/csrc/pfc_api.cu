// C ABI of libpfc (include/pfc.h): the solver context, the workspace carving,
// the FAS V-cycle driver of Algorithm 1 and the primitive operations.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "pfc_internal.h"
#include "pfc_mixed.h"

namespace pfc {
namespace {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  return PFC_ECUDA;
}

#define PFC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Enqueue `call` bracketed by the profiler's events for (cls, level).
#define PFC_TIMED(pr, cls, level, nlaunch, st, call) \
  do {                                                \
    prof_begin(pr, cls, st);                          \
    PFC_CUDA(call);                                   \
    prof_end(pr, cls, level, nlaunch, st);            \
  } while (0)

constexpr int kMaxLevels = 24;
constexpr int kMaxMembers = 1024;   // ensemble members of one context (one decide block)
constexpr size_t kAlign = 256;
constexpr int kVariants = 6;        // step graphs per ring position (pfc_ctx::variant)

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The mixed path stores phi, mu, omega, S2 and S3 as (hi, lo) FP32 pairs in
// the same 8-byte slots the FP64 path uses for doubles.
inline float2* as_df(double* p) { return reinterpret_cast<float2*>(p); }
inline const float2* as_df(const double* p) { return reinterpret_cast<const float2*>(p); }

// Whether M(phi) = m0 + m2 phi^2 differs from M == 1.
inline bool variable_mobility(const pfc_params* p) {
  return p->mobility_m0 != 1.0 || p->mobility_m2 != 0.0;
}

// The mixed paths (FP32 correction solves) and the one whose state is df.
inline bool is_mixed(const pfc_params* p) { return p->precision != PFC_FP64; }
inline bool df_state(const pfc_params* p) { return p->precision == PFC_MIXED_DF; }

// Level sizes: halve while the size is even and larger than `coarsest`; the
// mixed path also stops at the first coarse level of at most 16^3 cells whose
// stiffness 108 tau/h^6 is at most coarse_stiffness (its coarsest solve runs
// in FP32 in one block; the FP64 path keeps coarsening because one SM's FP64
// rate makes a large single-block FP64 solve slow).
int level_sizes(const pfc_params* p, int* sizes) {
  int n = p->n, nl = 0;
  double h = p->L / p->n;
  sizes[nl++] = n;
  while (n % 2 == 0 && n > p->coarsest && nl < kMaxLevels) {
    n /= 2;
    h *= 2.0;
    sizes[nl++] = n;
    const double s = 108.0 * p->dt / (h * h * h * h * h * h);
    if (p->precision != PFC_FP64 && n <= 16 && s <= p->coarse_stiffness) break;
  }
  return nl;
}

int validate(const pfc_params* p) {
  if (!p) return PFC_EINVAL;
  if (p->n < 4 || (p->n & 1)) return PFC_ESIZE;
  if (!(p->L > 0) || !(p->eps >= 0 && p->eps < 1) || !(p->dt > 0)) return PFC_EINVAL;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1) return PFC_EINVAL;
  if (!(p->tol > 0) || p->max_cycles < 1 || p->coarsest < 2) return PFC_EINVAL;
  if (p->precision != PFC_FP64 && p->precision != PFC_MIXED && p->precision != PFC_MIXED_DF)
    return PFC_EINVAL;
  if (p->smoother != PFC_NEWTON && p->smoother != PFC_PICARD) return PFC_EINVAL;
  if (p->precision != PFC_FP64 && p->inner_cycles < 1) return PFC_EINVAL;
  if (p->policy != PFC_POLICY_HYBRID && p->policy != PFC_POLICY_RB) return PFC_EINVAL;
  if (!(p->jacobi_weight > 0 && p->jacobi_weight <= 1) || p->jacobi_factor < 1 ||
      p->jacobi_factor0 < 1)
    return PFC_EINVAL;
  if (!(p->stiff_lo >= 0) || !(p->stiff_hi >= p->stiff_lo)) return PFC_EINVAL;
  if (!(p->coarse_stiffness >= 0) || p->coarse_sweeps < 1) return PFC_EINVAL;
  if (p->guess != PFC_GUESS_PREVIOUS && p->guess != PFC_GUESS_EXTRAPOLATE &&
      p->guess != PFC_GUESS_EXTRAPOLATE_ALL)
    return PFC_EINVAL;
  if (p->guess == PFC_GUESS_EXTRAPOLATE_ALL && p->precision == PFC_MIXED_DF) return PFC_EINVAL;
  if (!(p->mobility_m0 > 0) || !(p->mobility_m2 >= 0)) return PFC_EINVAL;
  if (variable_mobility(p) && p->precision != PFC_MIXED) return PFC_EINVAL;
  if (p->cluster_tail < 0 || p->cluster_tail > 2) return PFC_EINVAL;
  if (p->step_diagnostics != 0 && p->step_diagnostics != 1) return PFC_EINVAL;
  if (p->defect_planes < 0) return PFC_EINVAL;
  int sizes[kMaxLevels];
  const int nl = level_sizes(p, sizes);
  const int nc = sizes[nl - 1];
  if (nc % 2 != 0 || nc > 16 || nl < 2) return PFC_ESIZE;
  return PFC_OK;
}

struct Carver {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align_up(count * sizeof(T));
    return p;
  }
};

}  // namespace

struct Level64 {
  int n;
  int kind;          // PFC_SWEEP_RB or PFC_SWEEP_JACOBI
  Lvl L;
  double *u[3], *w[3], *S[3], *b;   // level 0 uses only the ring/context fields
  double* t[3];      // Jacobi ping-pong partner of u (and coarse-solve scratch)
};

}  // namespace pfc

struct pfc_ctx {
  pfc_params p;
  cudaStream_t st;
  int nl;
  int sizes[pfc::kMaxLevels];
  pfc::Level64 lev[pfc::kMaxLevels];
  double* ring[3];   // phi^{k-1}, phi^k, phi^{k+1} rotate through these
  int ic, ib, ia;
  double *mu, *om, *S2, *S3;  // ring, mu .. S3: doubles (FP64) or df pairs (mixed)
  double* lap[3];    // unscaled Laplacian of ring[r], written by the residual
                     // kernels on the iterate and by pfc_set_state (same format)
  int nb;            // ensemble members (1: a single problem); every field holds
                     // the members one after another
  double* c1m;       // (1 - eps_m)/2 per member on the device (null when nb == 1)
  double* eps_host;  // eps per member on the host (nb entries)
  double* M[3];      // face mobilities of the current step (variable mobility only)
  double *lmu, *lom; // unscaled Laplacians of mu and omega at the last defect's
                     // iterate (PFC_MIXED with M == 1)
  int warm;          // the state is the last step's solution and lmu, lom are
                     // its Laplacians: the next first defect is pointwise
  double tau_scale;  // reference mobility of the FP32 correction solve (1 for M == 1)
  double* t0[3];     // level-0 Jacobi scratch
  double* partials;  // reduction partial sums
  double* dout;      // 8 device doubles of reduction results
  double* hout;      // 8 pinned host doubles
  double* hdiag;     // pinned: the raw diagnostics sums formed by the last step
                     // (step_diagnostics), valid while diag_valid
  int diag_valid;
  pfc::MixedBufs mx; // FP32 hierarchy of the mixed path
  int step;
  pfc::Prof prof;    // optional event timing of launches
  pfc::StepState* dstate;  // device convergence state of the current step
  pfc::StepState* hstate;  // pinned host copy
  pfc::StepState* hstate_dev;  // its device address (mapped): written by a step graph's last kernel
  double* hdiag_dev;       // device address of hdiag (mapped)
  int use_graphs;    // run each step as one graph launch (default on)
  int graph_gen;     // bumped whenever the step graphs are rebuilt (groups key on it)
  cudaStream_t cap_st;  // private stream the step graphs are captured on
  struct Graph {
    cudaGraphExec_t exec;
    long long launches_pre, launches_body;
  } graph[pfc::kVariants][3];  // [step variant][position of the phi ring]
  int variant;       // of the step in flight: 0 full first defect, 1 pointwise,
                     // 2 + 2 slot + extrap for PFC_GUESS_EXTRAPOLATE_ALL
  double* mslot[2];  // PFC_GUESS_EXTRAPOLATE_ALL: mu of the last two converged
  double* oslot[2];  // steps (and omega); mu, om point at the current one
  double* lmslot[2]; // their Laplacians (lmu, lom point at the current step's;
  double* loslot[2]; // null without lmu, lom)
  int mcur;          // slot of the last converged step's mu, omega
  int nconv;         // converged steps in a row whose mu, omega the slots hold (<= 2)
};

namespace pfc {
namespace {

size_t carve(pfc_ctx* c, const pfc_params* p, char* base, int members) {
  Carver cv{base, 0};
  const int64_t n3 = (int64_t)p->n * p->n * p->n * members;
  int sizes[kMaxLevels];
  const int nl = level_sizes(p, sizes);
  for (int r = 0; r < 3; ++r) {
    double* f = cv.take<double>(n3);
    if (c) c->ring[r] = f;
  }
  for (int r = 0; r < 3; ++r) {
    double* f = cv.take<double>(n3);
    if (c) c->lap[r] = f;
  }
  for (int q = 0; q < 3; ++q) {
    double* f = variable_mobility(p) ? cv.take<double>(n3) : nullptr;
    if (c) c->M[q] = f;
  }
  {
    const bool keep = p->precision == PFC_MIXED && !variable_mobility(p);
    const bool two = keep && p->guess == PFC_GUESS_EXTRAPOLATE_ALL;
    double* a = keep ? cv.take<double>(n3) : nullptr;
    double* b = keep ? cv.take<double>(n3) : nullptr;
    double* a2 = two ? cv.take<double>(n3) : nullptr;
    double* b2 = two ? cv.take<double>(n3) : nullptr;
    if (c) {
      c->lmu = a;
      c->lom = b;
      c->lmslot[0] = a;
      c->lmslot[1] = a2;
      c->loslot[0] = b;
      c->loslot[1] = b2;
    }
  }
  double* mu = cv.take<double>(n3);
  double* om = cv.take<double>(n3);
  const bool all = p->guess == PFC_GUESS_EXTRAPOLATE_ALL;
  double* mu2 = all ? cv.take<double>(n3) : nullptr;
  double* om2 = all ? cv.take<double>(n3) : nullptr;
  double* S2 = cv.take<double>(n3);
  double* S3 = cv.take<double>(n3);
  const bool fp64 = p->precision == PFC_FP64;
  for (int q = 0; q < 3; ++q) {
    double* f = fp64 ? cv.take<double>(n3) : nullptr;
    if (c) c->t0[q] = f;
  }
  if (c) {
    c->mu = mu;
    c->om = om;
    c->mslot[0] = mu;
    c->mslot[1] = mu2;
    c->oslot[0] = om;
    c->oslot[1] = om2;
    c->mcur = 0;
    c->nconv = 0;
    c->S2 = S2;
    c->S3 = S3;
    c->nl = nl;
    for (int l = 0; l < nl; ++l) c->sizes[l] = sizes[l];
  }
  // the FP64 coarse hierarchy is used by the FAS path only
  for (int l = 1; l < nl && fp64; ++l) {
    const int64_t m3 = (int64_t)sizes[l] * sizes[l] * sizes[l];
    Level64 lv;
    for (int q = 0; q < 3; ++q) lv.u[q] = cv.take<double>(m3);
    for (int q = 0; q < 3; ++q) lv.w[q] = cv.take<double>(m3);
    for (int q = 0; q < 3; ++q) lv.S[q] = cv.take<double>(m3);
    lv.b = cv.take<double>(m3);
    for (int q = 0; q < 3; ++q) lv.t[q] = cv.take<double>(m3);
    if (c) c->lev[l] = lv;
  }
  double* partials = cv.take<double>((size_t)kReduceBlocks * kReduceComps);
  double* dout = cv.take<double>((size_t)kReduceComps * members);
  StepState* dstate = cv.take<StepState>(members);
  double* c1m = members > 1 ? cv.take<double>(members) : nullptr;
  if (c) {
    c->partials = partials;
    c->dout = dout;
    c->dstate = dstate;
    c->c1m = c1m;
    c->nb = members;
  }
  if (is_mixed(p)) {
    MixedBufs mx;
    mixed_carve(
        &mx, p->n, nl, sizes, [&](size_t count) { return cv.take<float>(count); }, members);
    if (c) c->mx = mx;
  }
  return cv.off;
}

// Views of level 0 for the current ring position.
void level0(pfc_ctx* c, Level64* lv) {
  lv->n = c->p.n;
  lv->L = c->lev[0].L;
  lv->u[0] = c->ring[c->ia];
  lv->u[1] = c->mu;
  lv->u[2] = c->om;
  lv->S[0] = c->ring[c->ib];
  lv->S[1] = c->S2;
  lv->S[2] = c->S3;
  lv->b = c->ring[c->ib];
  lv->kind = c->lev[0].kind;
  for (int q = 0; q < 3; ++q) lv->t[q] = c->t0[q];
}

// Pre- or post-smoothing of one level under the level's smoother kind.
int smooth_level(pfc_ctx* c, int l, const Level64& lv, int sweeps) {
  if (sweeps <= 0) return PFC_OK;
  cudaStream_t st = c->st;
  Prof* pr = &c->prof;
  if (lv.kind == PFC_SWEEP_JACOBI) {
    const int js = sweeps * (l == 0 ? c->p.jacobi_factor0 : c->p.jacobi_factor);
    PFC_TIMED(pr, PFC_K_SMOOTH, l, js, st,
              launch_jacobi(lv.L, c->p.smoother, js, c->p.jacobi_weight, lv.u[0], lv.u[1],
                            lv.u[2], lv.t[0], lv.t[1], lv.t[2], lv.S[0], lv.S[1], lv.S[2],
                            lv.b, st));
  } else {
    PFC_TIMED(pr, PFC_K_SMOOTH, l, 2 * sweeps, st,
              launch_smooth(lv.L, c->p.smoother, sweeps, lv.u[0], lv.u[1], lv.u[2], lv.S[0],
                            lv.S[1], lv.S[2], lv.b, st));
  }
  return PFC_OK;
}

int vcycle64(pfc_ctx* c, int l, const Level64& lv) {
  const int lin = c->p.smoother;
  cudaStream_t st = c->st;
  Prof* pr = &c->prof;
  if (l == c->nl - 1) {
    PFC_TIMED(pr, PFC_K_COARSE_SOLVE, l, 1, st,
              launch_coarse_solve(lv.L, lin, lv.kind, c->p.jacobi_weight, 400, lv.u[0],
                                  lv.u[1], lv.u[2], lv.t[0], lv.t[1], lv.t[2], lv.S[0],
                                  lv.S[1], lv.S[2], lv.b, st));
    return PFC_OK;
  }
  Level64& cl = c->lev[l + 1];
  int rc0 = smooth_level(c, l, lv, c->p.nu1);
  if (rc0) return rc0;
  PFC_TIMED(pr, PFC_K_RESIDUAL_RESTRICT, l, 1, st,
            launch_residual_restrict(lv.L, lv.u[0], lv.u[1], lv.u[2], lv.S[0], lv.S[1],
                                     lv.S[2], lv.b, cl.S[0], cl.S[1], cl.S[2], cl.u[0],
                                     cl.u[1], cl.u[2], cl.w[0], cl.w[1], cl.w[2], st));
  PFC_TIMED(pr, PFC_K_COARSE_SOURCE, l + 1, 1, st,
            launch_coarse_source(cl.L, cl.u[0], cl.u[1], cl.u[2], cl.b, cl.S[0], cl.S[1],
                                 cl.S[2], st));
  int rc = vcycle64(c, l + 1, cl);
  if (rc) return rc;
  prof_begin(pr, PFC_K_PROLONG, st);
  PFC_CUDA(launch_coarse_diff(cl.n, cl.u[0], cl.u[1], cl.u[2], cl.w[0], cl.w[1], cl.w[2],
                              st));
  PFC_CUDA(launch_prolong_add(lv.n, cl.w[0], cl.w[1], cl.w[2], lv.u[0], lv.u[1], lv.u[2],
                              st));
  prof_end(pr, PFC_K_PROLONG, l, 2, st);
  return smooth_level(c, l, lv, c->p.nu2);
}

// F_h, the modified energy, the mass and ||grad phi||^2 of every member from
// the six raw sums of the diagnostics kernel.
void diagnostics_finish(int n, double h, const double* eps, int members,
                               const double* hout, double* res) {
  (void)n;
  const double h3 = h * h * h;
  for (int m = 0; m < members; ++m) {
    const double* o = hout + (size_t)m * kReduceComps;
    const double F = 0.25 * h3 * o[0] + 0.5 * (1.0 - eps[m]) * h3 * o[1] - h * o[2] +
                     0.5 * o[3] / h;
    res[4 * m] = F;
    res[4 * m + 1] = F + 0.5 * h * o[4];
    res[4 * m + 2] = h3 * o[5];
    res[4 * m + 3] = h * o[2];
  }
}

// Diagnostics kernels of the state (a, b) and their raw sums copied to hout
// (asynchronous).
// direct (FP64 fields with stored Laplacians only): the final reduction
// writes the sums to direct_out (hout's device mapping) and copies the step
// states state -> state_out itself, so no copy follows.
cudaError_t enqueue_diagnostics(int n, int members, const double* a, const double* b,
                                const double* lapa, const double* lapb, bool df_fields,
                                double* partials, double* dout, double* hout, cudaStream_t st,
                                bool pdl = false, double* direct_out = nullptr,
                                const StepState* state = nullptr,
                                StepState* state_out = nullptr) {
  if (direct_out && !df_fields && lapa)
    return launch_diagnostics_cached(n, a, b, lapa, lapb, partials, direct_out, st, members, pdl,
                                     state, state_out);
  cudaError_t e;
  if (df_fields && lapa)
    e = launch_diagnostics_cached_df(n, as_df(a), as_df(b), as_df(lapa), as_df(lapb), partials,
                                     dout, st);
  else if (df_fields)
    e = launch_diagnostics_df(n, as_df(a), as_df(b), partials, dout, st);
  else if (lapa)
    e = launch_diagnostics_cached(n, a, b, lapa, lapb, partials, dout, st, members, pdl);
  else
    e = launch_diagnostics(n, a, b, partials, dout, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(hout, dout, kReduceComps * members * sizeof(double),
                         cudaMemcpyDeviceToHost, st);
}

// The convergence decision from the sum of squared residuals in dout.
int enqueue_decide(pfc_ctx* c, cudaGraphConditionalHandle h, int use_handle, int first) {
  const double n3 = (double)c->p.n * c->p.n * c->p.n;
  PFC_CUDA(launch_decide(h, use_handle, c->dout, c->dstate, 1.0 / (3.0 * n3), c->p.tol,
                         c->p.max_cycles, first, c->st, c->nb, c->prof.mask == 0));
  c->prof.launches += 1;
  return PFC_OK;
}

// The arguments of the step's convergence decision, for residual kernels
// that take it in their final reduction (single-member contexts).
DecideArgs decide_args(const pfc_ctx* c, cudaGraphConditionalHandle h, int use_handle,
                       int first) {
  const double n3 = (double)c->p.n * c->p.n * c->p.n;
  DecideArgs a;
  a.handle = h;
  a.use_handle = use_handle;
  a.state = c->dstate;
  a.inv_3n3 = 1.0 / (3.0 * n3);
  a.tol = c->p.tol;
  a.max_iter = c->p.max_cycles;
  a.first = first;
  return a;
}

// Sum of squared residuals of the level-0 iterate (to dout[0]) and the
// convergence decision into dstate.
int enqueue_residual_decide(pfc_ctx* c, const Level64& lv, cudaGraphConditionalHandle h,
                            int use_handle, int first, bool point = false) {
  cudaStream_t st = c->st;
  const DecideArgs da = decide_args(c, h, use_handle, first);
  bool decided = false;
  if (df_state(&c->p)) {
    float2* u[3];
    float2* S[3];
    for (int q = 0; q < 3; ++q) {
      u[q] = as_df(lv.u[q]);
      S[q] = as_df(lv.S[q]);
    }
    PFC_CUDA(mixed_enqueue_defect(c->mx, lv.L, u, S, as_df(lv.b), c->partials, c->dout, st,
                                  &c->prof, as_df(c->lap[c->ia])));
  } else if (point) {
    PFC_CUDA(mixed_enqueue_defect_point(c->mx, lv.L, lv.u, lv.S, lv.b, c->lap[c->ib], c->lmu,
                                        c->lom, c->lap[c->ia], c->partials, c->dout, st,
                                        &c->prof, c->nb, c->c1m, &da, &decided));
  } else if (is_mixed(&c->p)) {
    PFC_CUDA(mixed_enqueue_defect(c->mx, lv.L, lv.u, lv.S, lv.b, c->partials, c->dout, st,
                                  &c->prof, c->lap[c->ia], c->nb, c->c1m,
                                  c->M[0] ? c->M : nullptr, c->lmu, c->lom,
                                  c->p.defect_planes, &da, &decided));
  } else {
    PFC_TIMED(&c->prof, PFC_K_RESIDUAL_NORM, 0, 2, st,
              launch_residual_norm2(lv.L, lv.u[0], lv.u[1], lv.u[2], lv.S[0], lv.S[1],
                                    lv.S[2], lv.b, c->partials, c->dout, st,
                                    c->lap[c->ia]));
  }
  // a residual that took the decision in its reduction needs no launch of it
  return decided ? PFC_OK : enqueue_decide(c, h, use_handle, first);
}

// Work of a step before its convergence loop: S2, S3 (Eqs. 5.9-5.10), phi^k on
// the coarse levels (FAS path), the initial guess phi^{k+1} := phi^k, and the
// first residual and decision (warm: pointwise, from the Laplacians the last
// step's final defect stored).
int enqueue_pre(pfc_ctx* c, const Level64& lv, cudaGraphConditionalHandle h, int use_handle,
                bool warm) {
  const double* cprev = c->ring[c->ic];
  const int64_t n3 = (int64_t)c->p.n * c->p.n * c->p.n * c->nb;
  Prof* pr = &c->prof;
  const bool extrapolate = c->p.guess == PFC_GUESS_EXTRAPOLATE;
  if (warm) {
    // the last step's solution is the initial iterate and its Laplacians are
    // stored (PFC_MIXED, M == 1): S2, S3, the iterate and the first defect
    // in one pass
    const DecideArgs da = decide_args(c, h, use_handle, 1);
    bool decided = false;
    PFC_CUDA(mixed_enqueue_start_point(c->mx, lv.L, lv.u, lv.S, lv.b, c->lap[c->ib],
                                       c->lap[c->ic], c->lmu, c->lom, c->lap[c->ia],
                                       c->partials, c->dout, c->st, pr, c->nb, c->c1m, &da,
                                       &decided));
    return decided ? PFC_OK : enqueue_decide(c, h, use_handle, 1);
  }
  if (c->p.guess == PFC_GUESS_EXTRAPOLATE_ALL && c->nconv >= 2 && c->lmu) {
    // the two last steps' mu, omega and all their Laplacians are stored:
    // S2, S3, the extrapolated iterate and the first defect in one pass
    const int x = c->mcur;
    const DecideArgs da = decide_args(c, h, use_handle, 1);
    bool decided = false;
    PFC_CUDA(mixed_enqueue_start_extrap(c->mx, lv.L, lv.u, lv.S, lv.b, cprev, c->lap[c->ib],
                                        c->lap[c->ic], c->mslot[x], c->oslot[x],
                                        c->lmslot[x], c->loslot[x], c->lmu, c->lom,
                                        c->lap[c->ia], c->partials, c->dout, c->st, pr, c->nb,
                                        c->c1m, &da, &decided));
    return decided ? PFC_OK : enqueue_decide(c, h, use_handle, 1);
  }
  if (extrapolate && df_state(&c->p)) {
    PFC_TIMED(pr, PFC_K_SOURCE, 0, 2, c->st,
              launch_guess_df(lv.L, as_df(lv.b), as_df(cprev), as_df(c->S2), as_df(c->S3),
                              as_df(lv.u[0]), as_df(lv.u[1]), as_df(lv.u[2]), c->st));
  } else if (extrapolate) {
    PFC_TIMED(pr, PFC_K_SOURCE, 0, 2, c->st,
              launch_guess(lv.L, lv.b, cprev, c->S2, c->S3, lv.u[0], lv.u[1], lv.u[2],
                           c->st));
  } else if (df_state(&c->p)) {
    PFC_TIMED(pr, PFC_K_SOURCE, 0, 1, c->st,
              launch_source_cached_df(lv.L, as_df(lv.b), as_df(c->lap[c->ib]),
                                      as_df(c->lap[c->ic]), as_df(c->S2), as_df(c->S3),
                                      c->st));
  } else {
    PFC_TIMED(pr, PFC_K_SOURCE, 0, 1, c->st,
              launch_source_cached(lv.L, lv.b, c->lap[c->ib], c->lap[c->ic], c->S2, c->S3,
                                   c->st, c->nb, c->c1m, c->prof.mask == 0));
  }
  if (c->p.precision == PFC_FP64) {
    const double* fine = lv.b;
    for (int l = 1; l < c->nl; ++l) {
      PFC_TIMED(pr, PFC_K_RESTRICT, l - 1, 1, c->st,
                launch_restrict(c->sizes[l - 1], fine, c->lev[l].b, c->st));
      fine = c->lev[l].b;
    }
  }
  if (c->p.guess == PFC_GUESS_EXTRAPOLATE_ALL) {
    // the new iterate goes to the slots of mu^{k-1}, omega^{k-1} (lv.u[1], lv.u[2])
    PFC_TIMED(pr, PFC_K_SOURCE, 0, 1, c->st,
              launch_guess_all(n3, c->nconv >= 2, lv.b, cprev, c->mslot[c->mcur],
                               c->oslot[c->mcur], lv.u[1], lv.u[2], lv.u[0], c->st,
                               c->prof.mask == 0));
  } else if (!extrapolate) {
    PFC_CUDA(cudaMemcpyAsync(lv.u[0], lv.b, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->st));
  }
  if (c->M[0]) {
    // M(A phi_*) of this step (Section 5: phi_* = 3/2 phi^k - 1/2 phi^{k-1})
    PFC_CUDA(launch_face_mobility(c->p.n, c->p.mobility_m0, c->p.mobility_m2, lv.b, cprev,
                                  c->M[0], c->M[1], c->M[2], c->st));
    c->prof.launches += 1;
  }
  return enqueue_residual_decide(c, lv, h, use_handle, 1, warm);
}

// One iteration of the convergence loop: a V-cycle (FP64 FAS) or a defect
// correction (mixed), then the residual and decision.
int enqueue_body(pfc_ctx* c, const Level64& lv, cudaGraphConditionalHandle h,
                 int use_handle) {
  if (df_state(&c->p)) {
    float2* u[3] = {as_df(lv.u[0]), as_df(lv.u[1]), as_df(lv.u[2])};
    PFC_CUDA(mixed_enqueue_correction(c->mx, c->p, c->nl, c->sizes, u, c->st, &c->prof));
  } else if (is_mixed(&c->p)) {
    PFC_CUDA(mixed_enqueue_correction(c->mx, c->p, c->nl, c->sizes, lv.u, c->st, &c->prof,
                                      c->nb, c->tau_scale));
  } else {
    int rc = vcycle64(c, 0, lv);
    if (rc) return rc;
  }
  return enqueue_residual_decide(c, lv, h, use_handle, 0);
}

int read_state(pfc_ctx* c) {
  PFC_CUDA(cudaMemcpyAsync(c->hstate, c->dstate, sizeof(StepState) * c->nb,
                           cudaMemcpyDeviceToHost, c->st));
  PFC_CUDA(cudaStreamSynchronize(c->st));
  prof_harvest(&c->prof);
  return PFC_OK;
}

// Build the graph of one step for the current ring position: pre-loop work,
// then a WHILE node whose body is one loop iteration; k_decide sets the
// condition on the device, so a step needs one launch and one readback.
int build_graph_on(pfc_ctx* c, const Level64& lv, pfc_ctx::Graph* g, bool warm);

// Capture on the context's private stream (the caller's stream may be the
// legacy default stream, which cannot be captured); the graph is launched on
// the caller's stream.
int build_graph(pfc_ctx* c, const Level64& lv, pfc_ctx::Graph* g, bool warm) {
  if (!c->cap_st) PFC_CUDA(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  cudaStream_t user = c->st;
  c->st = c->cap_st;
  int rc = build_graph_on(c, lv, g, warm);
  c->st = user;
  return rc;
}

int build_graph_on(pfc_ctx* c, const Level64& lv, pfc_ctx::Graph* g, bool warm) {
  cudaGraph_t G = nullptr;
  PFC_CUDA(cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(c->st, G, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(G);
    return cuda_fail(e, "graph setup");
  }
  long long l0 = c->prof.launches;
  int rc = enqueue_pre(c, lv, h, 1, warm);
  g->launches_pre = c->prof.launches - l0;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNode_t cnode;
  if (rc == PFC_OK) {
    e = cudaStreamGetCaptureInfo(c->st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, G, deps, nullptr, ndeps, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(c->st, &cnode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    // the new state's energy/mass sums in the same graph launch; with FP64
    // fields their final reduction also copies the step state to the mapped
    // host copy (a copy node costs a few microseconds of the step)
    const bool direct = c->p.step_diagnostics && !df_state(&c->p) && c->lap[c->ia] != nullptr;
    if (e == cudaSuccess && !direct)
      e = cudaMemcpyAsync(c->hstate, c->dstate, sizeof(StepState) * c->nb,
                          cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && c->p.step_diagnostics) {
      e = enqueue_diagnostics(c->p.n, c->nb, c->ring[c->ia], c->ring[c->ib], c->lap[c->ia],
                              c->lap[c->ib], df_state(&c->p), c->partials, c->dout, c->hdiag,
                              c->st, c->prof.mask == 0, direct ? c->hdiag_dev : nullptr,
                              c->dstate, c->hstate_dev);
      g->launches_pre += 2;
    }
  }
  cudaGraph_t cap = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->st, &cap);
  if (rc == PFC_OK && e == cudaSuccess) e = e2;
  if (rc == PFC_OK && e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      l0 = c->prof.launches;
      rc = enqueue_body(c, lv, h, 1);
      g->launches_body = c->prof.launches - l0;
      cudaGraph_t bcap = nullptr;
      e2 = cudaStreamEndCapture(c->st, &bcap);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (rc == PFC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, G, 0);
  cudaGraphDestroy(G);
  if (rc) return rc;
  if (e != cudaSuccess) {
    g->exec = nullptr;
    return cuda_fail(e, "graph build");
  }
  return PFC_OK;
}

// The step's outcome over all ensemble members: the worst status, the most
// cycles and the largest residuals.
StepState combined_state(const pfc_ctx* c) {
  StepState s = c->hstate[0];
  for (int m = 1; m < c->nb; ++m) {
    const StepState& t = c->hstate[m];
    if (t.iters > s.iters) s.iters = t.iters;
    if (!(t.rms <= s.rms)) s.rms = t.rms;
    if (!(t.rms0 <= s.rms0)) s.rms0 = t.rms0;
    // NaN over no-convergence over running over converged
    const int rank_t = t.status == kStepNaN ? 3 : t.status == kStepNoConv ? 2
                       : t.status == kStepRunning ? 1 : 0;
    const int rank_s = s.status == kStepNaN ? 3 : s.status == kStepNoConv ? 2
                       : s.status == kStepRunning ? 1 : 0;
    if (rank_t > rank_s) s.status = t.status;
  }
  return s;
}

// Start of a step: level-0 views of the current ring position; returns
// whether the first defect is pointwise (the state is the last step's
// solution, guess phi^{k+1} := phi^k, and lmu, lom hold its Laplacians).
bool step_prepare(pfc_ctx* c, Level64* lv) {
  const bool warm = c->warm && c->lmu && c->p.guess == PFC_GUESS_PREVIOUS;
  c->variant = warm ? 1 : 0;
  if (c->p.guess == PFC_GUESS_EXTRAPOLATE_ALL) {
    // the step's iterate takes the other slot; mcur keeps the last solution's
    const int y = 1 - c->mcur;
    c->mu = c->mslot[y];
    c->om = c->oslot[y];
    c->lmu = c->lmslot[y];
    c->lom = c->loslot[y];
    c->variant = 2 + 2 * y + (c->nconv >= 2 ? 1 : 0);
  }
  level0(c, lv);
  c->warm = 0;                       // until this step has converged
  c->diag_valid = 0;
  return warm;
}

// A step stopped before its end (another member of its group failed): the
// state stays the last solution.
void step_abandon(pfc_ctx* c) {
  if (c->p.guess != PFC_GUESS_EXTRAPOLATE_ALL) return;
  c->mu = c->mslot[c->mcur];
  c->om = c->oslot[c->mcur];
  c->lmu = c->lmslot[c->mcur];
  c->lom = c->loslot[c->mcur];
  c->nconv = 0;
}

// End of a step whose device state (hstate) has been read back: the step's
// outcome, stats, and on success the ring rotation.
int step_finish(pfc_ctx* c, pfc_step_stats* stats) {
  const int64_t n3 = (int64_t)c->p.n * c->p.n * c->p.n * c->nb;
  int rc = PFC_OK;
  const StepState s = combined_state(c);
  if (s.status == kStepNaN) rc = PFC_ENAN;
  else if (s.status == kStepNoConv) rc = PFC_ENOCONV;
  else if (s.status != kStepConverged) rc = PFC_ECUDA;
  if (stats) {
    stats->cycles_last = s.iters;
    stats->cycles_total += s.iters;
    stats->residual = s.rms;
    stats->residual0 = s.rms0;
  }
  if (c->p.guess == PFC_GUESS_EXTRAPOLATE_ALL) {
    if (rc) {
      // back to the last solution's mu, omega (the failed iterate's slot held
      // mu^{k-1}, which is gone)
      c->mu = c->mslot[c->mcur];
      c->om = c->oslot[c->mcur];
      c->lmu = c->lmslot[c->mcur];
      c->lom = c->loslot[c->mcur];
      c->nconv = 0;
    } else {
      c->mcur = 1 - c->mcur;
      if (c->nconv < 2) c->nconv += 1;
    }
  }
  if (rc == PFC_ENAN && c->p.guess != PFC_GUESS_EXTRAPOLATE_ALL) {
    cudaMemsetAsync(c->mu, 0, n3 * sizeof(double), c->st);
    cudaMemsetAsync(c->om, 0, n3 * sizeof(double), c->st);
  }
  if (rc) return rc;
  const int old_c = c->ic;
  c->ic = c->ib;
  c->ib = c->ia;
  c->ia = old_c;
  c->step += 1;
  c->warm = c->lmu != nullptr;
  c->diag_valid = c->p.step_diagnostics;
  if (stats) stats->steps += 1;
  return PFC_OK;
}

int step_once(pfc_ctx* c, pfc_step_stats* stats) {
  Level64 lv;
  const bool warm = step_prepare(c, &lv);
  int rc = PFC_OK;
  if (c->use_graphs && c->prof.mask == 0) {
    pfc_ctx::Graph* g = &c->graph[c->variant][c->ia];
    if (!g->exec) {
      rc = build_graph(c, lv, g, warm);
      if (rc) return rc;
    }
    PFC_CUDA(cudaGraphLaunch(g->exec, c->st));
    PFC_CUDA(cudaStreamSynchronize(c->st));
    c->prof.launches +=
        g->launches_pre + g->launches_body * (long long)combined_state(c).iters;
  } else {
    rc = enqueue_pre(c, lv, 0, 0, warm);
    if (rc == PFC_OK) rc = read_state(c);
    while (rc == PFC_OK && combined_state(c).status == kStepRunning) {
      rc = enqueue_body(c, lv, 0, 0);
      if (rc == PFC_OK) rc = read_state(c);
    }
    if (rc == PFC_OK && c->p.step_diagnostics) {
      PFC_CUDA(enqueue_diagnostics(c->p.n, c->nb, c->ring[c->ia], c->ring[c->ib], c->lap[c->ia],
                                   c->lap[c->ib], df_state(&c->p), c->partials, c->dout,
                                   c->hdiag, c->st));
      PFC_CUDA(cudaStreamSynchronize(c->st));
      c->prof.launches += 2;
    }
    if (rc) return rc;
  }
  return step_finish(c, stats);
}

}  // namespace

void set_last_error(const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

void prof_begin(Prof* pr, int cls, cudaStream_t st) {
  if (!pr || !((pr->mask >> cls) & 1u)) return;
  if (pr->pending == Prof::kPool) {
    cudaEventSynchronize(pr->ev[2 * Prof::kPool - 1]);
    prof_harvest(pr);
  }
  cudaEventRecord(pr->ev[2 * pr->pending], st);
}

void prof_end(Prof* pr, int cls, int level, int nlaunch, cudaStream_t st) {
  if (!pr) return;
  pr->launches += nlaunch;
  if (!((pr->mask >> cls) & 1u)) return;
  const int i = pr->pending;
  cudaEventRecord(pr->ev[2 * i + 1], st);
  pr->cls[i] = cls;
  pr->lev[i] = level < PFC_PROFILE_LEVELS ? level : PFC_PROFILE_LEVELS - 1;
  pr->nlaunch[i] = nlaunch;
  pr->pending = i + 1;
}

void prof_harvest(Prof* pr) {
  if (!pr) return;
  for (int i = 0; i < pr->pending; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pr->ev[2 * i], pr->ev[2 * i + 1]) == cudaSuccess) {
      pr->ms[pr->cls[i]][pr->lev[i]] += t;
      pr->cnt[pr->cls[i]][pr->lev[i]] += pr->nlaunch[i];
    }
  }
  pr->pending = 0;
}

}  // namespace pfc

using namespace pfc;

extern "C" {

void pfc_default_params(pfc_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nu1 = 2;
  p->nu2 = 2;
  p->tol = 1e-9;
  p->max_cycles = 50;
  p->precision = PFC_FP64;
  p->smoother = PFC_NEWTON;
  p->coarsest = 2;
  p->inner_cycles = 1;
  p->policy = PFC_POLICY_HYBRID;
  p->jacobi_weight = 0.7;
  p->jacobi_factor = 4;
  p->jacobi_factor0 = 2;
  p->stiff_hi = 1000.0;
  p->stiff_lo = 0.25;
  p->coarse_stiffness = 0.05;
  p->coarse_sweeps = 4;
  p->guess = PFC_GUESS_PREVIOUS;
  p->mobility_m0 = 1.0;
  p->mobility_m2 = 0.0;
  p->cluster_tail = 0;
  p->step_diagnostics = 0;
  p->defect_planes = 0;
}

int pfc_level_info(const pfc_params* p, int level, int* n, double* h, int* kind) {
  if (validate(p) != PFC_OK || level < 0) return PFC_EINVAL;
  int sizes[kMaxLevels];
  const int nl = level_sizes(p, sizes);
  if (level >= nl) return PFC_EINVAL;
  const double hl = p->L / p->n * (double)(1 << level);
  if (n) *n = sizes[level];
  if (h) *h = hl;
  if (kind) *kind = level_kind(p, hl);
  return PFC_OK;
}

size_t pfc_workspace_bytes(const pfc_params* p) {
  if (validate(p) != PFC_OK) return 0;
  return carve(nullptr, p, nullptr, 1);
}

// Ensemble sizes the launch grids can cover: the kernels put planes x members
// (x 3 components in the transfers, 3 n/2 planes per member) on the grid's
// z extent, which CUDA bounds by 65535.
static bool members_fit(const pfc_params* p, int members) {
  return members >= 1 && members <= kMaxMembers && 3LL * p->n * members / 2 <= 65535;
}

size_t pfc_batch_workspace_bytes(const pfc_params* p, int members) {
  if (validate(p) != PFC_OK || !members_fit(p, members)) return 0;
  if (members > 1 && p->precision != PFC_MIXED) return 0;
  return carve(nullptr, p, nullptr, members);
}

const char* pfc_last_error(void) { return g_last_error; }

// Context of `members` independent runs (one for pfc_init) sharing n, L, tau
// and the solver settings, member m with eps[m] and its initial fields at
// offset m n^3 of any_phi0 / any_phi1.
static int init_members(pfc_ctx** out, const pfc_params* p, int members, const double* eps,
                        void* d_workspace, size_t workspace_bytes, const double* any_phi0,
                        const double* any_phi1, void* stream) {
  if (!out || !d_workspace || !any_phi0) return PFC_EINVAL;
  *out = nullptr;
  int v = validate(p);
  if (v) return v;
  if (!members_fit(p, members)) return PFC_EINVAL;
  if (members > 1 && p->precision != PFC_MIXED) return PFC_EINVAL;
  if (members > 1 && variable_mobility(p)) return PFC_EINVAL;
  for (int m = 0; m < members; ++m)
    if (!(eps[m] >= 0 && eps[m] < 1)) return PFC_EINVAL;
  if (((uintptr_t)d_workspace) % kAlign) return PFC_EINVAL;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, d_workspace);
  if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes(workspace)");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return PFC_EINVAL;
  const size_t need = carve(nullptr, p, nullptr, members);
  if (workspace_bytes < need) return PFC_ESIZE;
  pfc_ctx* c = (pfc_ctx*)calloc(1, sizeof(pfc_ctx));
  if (!c) return PFC_EINVAL;
  c->p = *p;
  c->st = (cudaStream_t)stream;
  carve(c, p, (char*)d_workspace, members);
  double h = p->L / p->n;
  for (int l = 0; l < c->nl; ++l) {
    c->lev[l].n = c->sizes[l];
    c->lev[l].L = make_lvl(c->sizes[l], h, p->eps, p->dt);
    c->lev[l].kind = level_kind(p, h);
    h *= 2.0;
  }
  c->eps_host = (double*)malloc(sizeof(double) * members);
  if (!c->eps_host) {
    free(c);
    return PFC_EINVAL;
  }
  memcpy(c->eps_host, eps, sizeof(double) * members);
  e = cudaHostAlloc((void**)&c->hout, kReduceComps * sizeof(double) * members,
                    cudaHostAllocDefault);
  // the step state and the diagnostics sums are mapped: a step graph's last
  // kernel writes them, with no copy node
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&c->hstate, sizeof(StepState) * members, cudaHostAllocMapped);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&c->hdiag, kReduceComps * sizeof(double) * members,
                      cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->hstate_dev, c->hstate, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->hdiag_dev, c->hdiag, 0);
  if (e != cudaSuccess) {
    if (c->hout) cudaFreeHost(c->hout);
    if (c->hstate) cudaFreeHost(c->hstate);
    if (c->hdiag) cudaFreeHost(c->hdiag);
    free(c->eps_host);
    free(c);
    return cuda_fail(e, "cudaHostAlloc");
  }
  memset(c->hstate, 0, sizeof(StepState) * members);
  c->use_graphs = 1;
  c->ic = 0;
  c->ib = 1;
  c->ia = 2;
  c->tau_scale = 1.0;
  int rc = PFC_OK;
  if (c->c1m) {
    for (int m = 0; m < members; ++m) c->hout[m] = 0.5 * (1.0 - eps[m]);
    e = cudaMemcpyAsync(c->c1m, c->hout, sizeof(double) * members, cudaMemcpyHostToDevice,
                        c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(eps)");
  }
  const size_t bytes = (size_t)p->n * p->n * p->n * members * sizeof(double);
  if (rc == PFC_OK)
    rc = pfc_set_state(c, any_phi1 ? any_phi1 : any_phi0, any_phi1 ? any_phi0 : nullptr);
  if (rc == PFC_OK) {
    e = cudaMemsetAsync(c->mu, 0, bytes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->om, 0, bytes, c->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
  }
  if (rc) {
    pfc_destroy(c);
    return rc;
  }
  c->step = any_phi1 ? 1 : 0;
  *out = c;
  return PFC_OK;
}

int pfc_init(pfc_ctx** out, const pfc_params* p, void* d_workspace,
             size_t workspace_bytes, const double* any_phi0, const double* any_phi1,
             void* stream) {
  if (!p) return PFC_EINVAL;
  return init_members(out, p, 1, &p->eps, d_workspace, workspace_bytes, any_phi0, any_phi1,
                      stream);
}

int pfc_batch_init(pfc_ctx** out, const pfc_params* p, int members, const double* eps,
                   void* d_workspace, size_t workspace_bytes, const double* any_phi0,
                   void* stream) {
  if (!p || !eps) return PFC_EINVAL;
  return init_members(out, p, members, eps, d_workspace, workspace_bytes, any_phi0, nullptr,
                      stream);
}

int pfc_set_state(pfc_ctx* c, const double* any_phi, const double* any_phi_prev) {
  if (!c || !any_phi) return PFC_EINVAL;
  c->warm = 0;                       // mu, omega are no longer the state's own
  c->nconv = 0;
  c->diag_valid = 0;
  const int64_t n3 = (int64_t)c->p.n * c->p.n * c->p.n * c->nb;
  const size_t bytes = (size_t)n3 * sizeof(double);
  PFC_CUDA(cudaMemcpyAsync(c->ring[c->ib], any_phi, bytes, cudaMemcpyDefault, c->st));
  PFC_CUDA(cudaMemcpyAsync(c->ring[c->ic], any_phi_prev ? any_phi_prev : any_phi, bytes,
                           cudaMemcpyDefault, c->st));
  if (df_state(&c->p)) {
    // PFC_MIXED_DF keeps phi as df pairs: convert in place
    PFC_CUDA(launch_df_from_f64(n3, c->ring[c->ib], as_df(c->ring[c->ib]), c->st));
    PFC_CUDA(launch_df_from_f64(n3, c->ring[c->ic], as_df(c->ring[c->ic]), c->st));
    PFC_CUDA(launch_laplacian_df(c->p.n, as_df(c->ring[c->ib]), as_df(c->lap[c->ib]), c->st));
    PFC_CUDA(launch_laplacian_df(c->p.n, as_df(c->ring[c->ic]), as_df(c->lap[c->ic]), c->st));
    c->prof.launches += 4;
  } else {
    PFC_CUDA(launch_laplacian(c->p.n, c->ring[c->ib], c->lap[c->ib], c->st, c->nb));
    PFC_CUDA(launch_laplacian(c->p.n, c->ring[c->ic], c->lap[c->ic], c->st, c->nb));
    c->prof.launches += 2;
  }
  if (variable_mobility(&c->p)) {
    // reference mobility of the FP32 correction solve: m0 + m2 mean(phi^2)
    // of the state (sum phi^2 is the diagnostics' second raw sum)
    PFC_CUDA(launch_diagnostics_cached(c->p.n, c->ring[c->ib], c->ring[c->ic], c->lap[c->ib],
                                       c->lap[c->ic], c->partials, c->dout, c->st));
    PFC_CUDA(cudaMemcpyAsync(c->hout, c->dout, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                             c->st));
    PFC_CUDA(cudaStreamSynchronize(c->st));
    c->prof.launches += 2;
    const double scale = c->p.mobility_m0 + c->p.mobility_m2 * c->hout[1] / (double)n3;
    if (scale != c->tau_scale) {
      // the step graphs hold the FP32 level constants: rebuild them
      c->graph_gen += 1;
      for (int v = 0; v < kVariants; ++v)
        for (int r = 0; r < 3; ++r)
          if (c->graph[v][r].exec) {
            cudaGraphExecDestroy(c->graph[v][r].exec);
            c->graph[v][r].exec = nullptr;
          }
      c->tau_scale = scale;
    }
  }
  return PFC_OK;
}

int pfc_step(pfc_ctx* c, int nsteps, pfc_step_stats* stats) {
  if (!c || nsteps < 0) return PFC_EINVAL;
  if (stats) memset(stats, 0, sizeof(*stats));
  for (int s = 0; s < nsteps; ++s) {
    int rc = step_once(c, stats);
    if (rc) return rc;
  }
  return PFC_OK;
}

// Copy a state field out as FP64.  PFC_MIXED_DF's df fields are converted
// first into ring[ia], the slot of phi^{k+1}, which holds nothing between
// steps (each step starts by overwriting it with phi^k).
static int copy_field(pfc_ctx* c, const double* src, double* dst) {
  if (!c || !dst) return PFC_EINVAL;
  const int64_t n3 = (int64_t)c->p.n * c->p.n * c->p.n * c->nb;
  const size_t bytes = (size_t)n3 * sizeof(double);
  if (df_state(&c->p)) {
    double* stage = c->ring[c->ia];
    PFC_CUDA(launch_df_to_f64(n3, as_df(src), stage, c->st));
    c->prof.launches += 1;
    src = stage;
  }
  PFC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->st));
  return PFC_OK;
}

int pfc_get_phi(pfc_ctx* c, double* any_dst) {
  return c ? copy_field(c, c->ring[c->ib], any_dst) : PFC_EINVAL;
}
int pfc_get_mu(pfc_ctx* c, double* any_dst) {
  return c ? copy_field(c, c->mu, any_dst) : PFC_EINVAL;
}
int pfc_get_omega(pfc_ctx* c, double* any_dst) {
  return c ? copy_field(c, c->om, any_dst) : PFC_EINVAL;
}

// Energy, modified energy, mass and |grad a|^2 of a = phi^k, b = phi^{k-1}
// for `members` ensemble members (eps[m] each, res[4 m .. 4 m + 3]); with
// lapa, lapb (their stored unscaled Laplacians) the kernels skip the
// stencils.
static int diagnostics(int n, double h, const double* eps, int members, const double* a,
                       const double* b, const double* lapa, const double* lapb,
                       bool df_fields, double* partials, double* dout, double* hout,
                       cudaStream_t st, double* res) {
  PFC_CUDA(enqueue_diagnostics(n, members, a, b, lapa, lapb, df_fields, partials, dout, hout,
                               st));
  PFC_CUDA(cudaStreamSynchronize(st));
  diagnostics_finish(n, h, eps, members, hout, res);
  return PFC_OK;
}

int pfc_batch_diagnostics(pfc_ctx* c, double* out) {
  if (!c || !out) return PFC_EINVAL;
  if (c->diag_valid) {
    // formed by the last step (step_diagnostics): no further GPU work
    diagnostics_finish(c->p.n, c->p.L / c->p.n, c->eps_host, c->nb, c->hdiag, out);
    return PFC_OK;
  }
  c->prof.launches += 2;
  return diagnostics(c->p.n, c->p.L / c->p.n, c->eps_host, c->nb, c->ring[c->ib],
                     c->ring[c->ic], c->lap[c->ib], c->lap[c->ic], df_state(&c->p),
                     c->partials, c->dout, c->hout, c->st, out);
}

int pfc_diagnostics(pfc_ctx* c, double out[4]) {
  if (!c || !out) return PFC_EINVAL;
  if (c->nb == 1) return pfc_batch_diagnostics(c, out);
  double* all = (double*)malloc(sizeof(double) * 4 * c->nb);
  if (!all) return PFC_EINVAL;
  const int rc = pfc_batch_diagnostics(c, all);
  if (rc == PFC_OK) memcpy(out, all, 4 * sizeof(double));
  free(all);
  return rc;
}

int pfc_adjoint_step(pfc_ctx* c, const double* phi_next, const double* phi_k,
                     const double* gnext, double* gk, double* gkm1, double* z, double rtol,
                     int max_cycles, double* eps_bar, int* cycles) {
  if (!c || !phi_next || !phi_k || !gnext || !gk || !gkm1 || !z || !eps_bar ||
      !(rtol > 0) || max_cycles < 1)
    return PFC_EINVAL;
  if (c->p.precision != PFC_MIXED || c->nb != 1 || variable_mobility(&c->p))
    return PFC_EINVAL;
  const int64_t n3 = (int64_t)c->p.n * c->p.n * c->p.n;
  cudaStream_t st = c->st;
  double* z1 = z;
  double* z2 = z + n3;
  double* z3 = z + 2 * n3;
  PFC_CUDA(cudaMemsetAsync(z, 0, 3 * n3 * sizeof(double), st));
  const Lvl& L0 = c->lev[0].L;
  double* u[3] = {z1, z2, z3};
  double rms0 = 0.0;
  int it = 0;
  for (;; ++it) {
    // FP64 defect of J z = (0, g, 0): the linear outer loop
    PFC_CUDA(launch_adj_defect64(L0, z1, z2, z3, gnext, phi_next, phi_k, c->mx.r[0][0],
                                 c->mx.r[0][1], c->mx.r[0][2], c->mx.q[0], c->partials,
                                 c->dout, st));
    PFC_CUDA(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, st));
    PFC_CUDA(cudaStreamSynchronize(st));
    c->prof.launches += 2;
    const double rms = sqrt(c->hout[0] / (3.0 * (double)n3));
    if (!std::isfinite(rms)) return PFC_ENAN;
    if (it == 0) rms0 = rms;
    if (rms <= rtol * rms0 || rms == 0.0) break;
    if (it >= max_cycles) {
      if (cycles) *cycles = it;
      return PFC_ENOCONV;
    }
    // FP32 V-cycles on J d = r (q frozen at the step's solution), z += d
    PFC_CUDA(mixed_enqueue_correction(c->mx, c->p, c->nl, c->sizes, u, st, nullptr, 1));
  }
  PFC_CUDA(launch_adj_accumulate(L0, z1, z2, z3, phi_next, phi_k, gk, gkm1, c->partials,
                                 c->dout, st));
  PFC_CUDA(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFC_CUDA(cudaStreamSynchronize(st));
  c->prof.launches += 2;
  *eps_bar += c->hout[0];
  if (cycles) *cycles = it;
  return PFC_OK;
}

int pfc_batch_status(const pfc_ctx* c, int* iters, double* residual, double* residual0) {
  if (!c) return PFC_EINVAL;
  for (int m = 0; m < c->nb; ++m) {
    if (iters) iters[m] = c->hstate[m].iters;
    if (residual) residual[m] = c->hstate[m].rms;
    if (residual0) residual0[m] = c->hstate[m].rms0;
  }
  return PFC_OK;
}

int pfc_batch_members(const pfc_ctx* c) { return c ? c->nb : -1; }

int pfc_energy(pfc_ctx* c, double* F, double* F_modified) {
  double r[4];
  int rc = pfc_diagnostics(c, r);
  if (rc) return rc;
  if (F) *F = r[0];
  if (F_modified) *F_modified = r[1];
  return PFC_OK;
}

int pfc_mass(pfc_ctx* c, double* mass) {
  if (!mass) return PFC_EINVAL;
  double r[4];
  int rc = pfc_diagnostics(c, r);
  if (rc) return rc;
  *mass = r[2];
  return PFC_OK;
}

long long pfc_launch_count(const pfc_ctx* c) { return c ? c->prof.launches : -1; }

int pfc_use_graphs(pfc_ctx* c, int on) {
  if (!c) return PFC_EINVAL;
  c->use_graphs = on ? 1 : 0;
  return PFC_OK;
}

int pfc_step_index(const pfc_ctx* c) { return c ? c->step : -1; }

int pfc_profile_enable(pfc_ctx* c, unsigned mask) {
  if (!c) return PFC_EINVAL;
  Prof& pr = c->prof;
  PFC_CUDA(cudaStreamSynchronize(c->st));
  prof_harvest(&pr);
  if (mask && !pr.created) {
    for (int i = 0; i < 2 * Prof::kPool; ++i) PFC_CUDA(cudaEventCreate(&pr.ev[i]));
    pr.created = true;
  }
  pr.mask = mask;
  memset(pr.ms, 0, sizeof(pr.ms));
  memset(pr.cnt, 0, sizeof(pr.cnt));
  return PFC_OK;
}

int pfc_profile_read(pfc_ctx* c, int kclass, int level, long long* launches, double* ms) {
  if (!c || kclass < 0 || kclass >= PFC_K_COUNT || level < 0 || level >= PFC_PROFILE_LEVELS)
    return PFC_EINVAL;
  PFC_CUDA(cudaStreamSynchronize(c->st));
  prof_harvest(&c->prof);
  if (launches) *launches = c->prof.cnt[kclass][level];
  if (ms) *ms = c->prof.ms[kclass][level];
  return PFC_OK;
}

void pfc_destroy(pfc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  for (int v = 0; v < kVariants; ++v)
    for (int r = 0; r < 3; ++r)
      if (c->graph[v][r].exec) cudaGraphExecDestroy(c->graph[v][r].exec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->hout) cudaFreeHost(c->hout);
  if (c->hstate) cudaFreeHost(c->hstate);
  if (c->hdiag) cudaFreeHost(c->hdiag);
  free(c->eps_host);
  if (c->prof.created)
    for (int i = 0; i < 2 * Prof::kPool; ++i) cudaEventDestroy(c->prof.ev[i]);
  free(c);
}

// ---------------------------------------------------------------------------
// Groups of contexts (ensembles of different grid sizes): one graph per step
// ---------------------------------------------------------------------------

struct pfc_group {
  int count;
  pfc_ctx* ctx[pfc::kMaxGroup];
  cudaStream_t st;       // launch stream (the caller's)
  cudaStream_t cap_st;   // private stream the step graphs are captured on
  cudaEvent_t fork;
  cudaEvent_t join[pfc::kMaxGroup];
  cudaEvent_t ready[pfc::kMaxGroup];
  struct Graph {
    // (first defect pointwise, ring position, graph generation) per context
    int key[3 * pfc::kMaxGroup];
    cudaGraphExec_t exec;
    long long pre[pfc::kMaxGroup], body[pfc::kMaxGroup];
  };
  std::vector<Graph> graphs;
  long long graph_launches;
};

namespace pfc {
namespace {

// Fork: every context's capture stream takes the group capture stream's
// current dependencies.  Join: the group stream waits for all of them.
cudaError_t group_fork(pfc_group* g) {
  cudaError_t e = cudaEventRecord(g->fork, g->cap_st);
  for (int i = 0; i < g->count && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(g->ctx[i]->cap_st, g->fork, 0);
  return e;
}

cudaError_t group_join(pfc_group* g) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < g->count && e == cudaSuccess; ++i) {
    e = cudaEventRecord(g->join[i], g->ctx[i]->cap_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cap_st, g->join[i], 0);
  }
  return e;
}

// The graph of one group step: every context's pre-loop work side by side,
// the group decision, a WHILE node whose body sets one IF condition per
// context (it still has a running member), runs each context's loop body
// under its IF node side by side and then the group decision, and after the
// loop every context's state readback (and diagnostics).  Each context's own
// decision keeps its members' states; only the group kernels set
// conditions.  A converged context takes no further correction, so every
// context ends the step exactly as if it had been stepped alone.
int group_build(pfc_group* g, const bool* warm, const Level64* lv, pfc_group::Graph* gr) {
  cudaGraph_t G = nullptr;
  PFC_CUDA(cudaGraphCreate(&G, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(g->cap_st, G, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(G);
    return cuda_fail(e, "group graph setup");
  }
  GroupStates gs = {};
  gs.count = g->count;
  cudaStream_t saved[kMaxGroup];
  for (int i = 0; i < g->count; ++i) {
    gs.s[i] = g->ctx[i]->dstate;
    gs.members[i] = g->ctx[i]->nb;
    saved[i] = g->ctx[i]->st;
    g->ctx[i]->st = g->ctx[i]->cap_st;
  }
  int rc = PFC_OK;
  e = group_fork(g);
  for (int i = 0; i < g->count && rc == PFC_OK && e == cudaSuccess; ++i) {
    pfc_ctx* c = g->ctx[i];
    const long long l0 = c->prof.launches;
    rc = enqueue_pre(c, lv[i], h, 0, warm[i]);
    gr->pre[i] = c->prof.launches - l0;
  }
  if (rc == PFC_OK && e == cudaSuccess) e = group_join(g);
  if (rc == PFC_OK && e == cudaSuccess) e = launch_group_decide(h, gs, g->cap_st);
  cudaGraphNodeParams cp = {};
  if (rc == PFC_OK && e == cudaSuccess) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraphNode_t cnode;
    e = cudaStreamGetCaptureInfo(g->cap_st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, G, deps, nullptr, ndeps, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(g->cap_st, &cnode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) e = group_fork(g);
    for (int i = 0; i < g->count && e == cudaSuccess; ++i) {
      pfc_ctx* c = g->ctx[i];
      e = cudaMemcpyAsync(c->hstate, c->dstate, sizeof(StepState) * c->nb,
                          cudaMemcpyDeviceToHost, c->st);
      if (e == cudaSuccess && c->p.step_diagnostics) {
        e = enqueue_diagnostics(c->p.n, c->nb, c->ring[c->ia], c->ring[c->ib], c->lap[c->ia],
                                c->lap[c->ib], df_state(&c->p), c->partials, c->dout,
                                c->hdiag, c->st, c->prof.mask == 0);
        gr->pre[i] += 2;
      }
    }
    if (e == cudaSuccess) e = group_join(g);
  }
  cudaGraph_t cap = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->cap_st, &cap);
  if (rc == PFC_OK && e == cudaSuccess) e = e2;
  if (rc == PFC_OK && e == cudaSuccess) {
    // loop body: the IF conditions, then per context an IF node holding its
    // loop body (captured on the context's stream into the node's graph),
    // then the group decision after all of them
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    GroupHandles hs = {};
    for (int i = 0; i < g->count && e == cudaSuccess; ++i)
      e = cudaGraphConditionalHandleCreate(&hs.h[i], body, 0, 0);
    cudaGraphNode_t sel = nullptr;
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(g->cap_st, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = launch_group_select(hs, gs, g->cap_st);
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      if (e == cudaSuccess)
        e = cudaStreamGetCaptureInfo(g->cap_st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
      if (e == cudaSuccess && ndeps == 1) sel = deps[0];
      cudaGraph_t scap = nullptr;
      e2 = cudaStreamEndCapture(g->cap_st, &scap);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess && !sel) e = cudaErrorStreamCaptureInvalidated;
    }
    cudaGraphNode_t ifs[kMaxGroup];
    for (int i = 0; i < g->count && rc == PFC_OK && e == cudaSuccess; ++i) {
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hs.h[i];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      e = cudaGraphAddNode(&ifs[i], body, &sel, nullptr, 1, &ip);
      pfc_ctx* c = g->ctx[i];
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(c->st, ip.conditional.phGraph_out[0], nullptr,
                                          nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const long long l0 = c->prof.launches;
        rc = enqueue_body(c, lv[i], h, 0);
        gr->body[i] = c->prof.launches - l0;
        cudaGraph_t icap = nullptr;
        e2 = cudaStreamEndCapture(c->st, &icap);
        if (e == cudaSuccess) e = e2;
      }
    }
    if (rc == PFC_OK && e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(g->cap_st, body, ifs, nullptr, g->count,
                                        cudaStreamCaptureModeThreadLocal);
    if (rc == PFC_OK && e == cudaSuccess) {
      e = launch_group_decide(h, gs, g->cap_st);
      cudaGraph_t dcap = nullptr;
      e2 = cudaStreamEndCapture(g->cap_st, &dcap);
      if (e == cudaSuccess) e = e2;
    }
  }
  for (int i = 0; i < g->count; ++i) g->ctx[i]->st = saved[i];
  if (rc == PFC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gr->exec, G, 0);
  cudaGraphDestroy(G);
  if (rc) return rc;
  if (e != cudaSuccess) {
    gr->exec = nullptr;
    return cuda_fail(e, "group graph build");
  }
  return PFC_OK;
}

int group_step_once(pfc_group* g, pfc_step_stats* stats) {
  bool graphs = true;
  for (int i = 0; i < g->count; ++i)
    if (!g->ctx[i]->use_graphs || g->ctx[i]->prof.mask != 0) graphs = false;
  if (!graphs) {
    // host-driven or timed contexts: one after another
    int first = PFC_OK;
    for (int i = 0; i < g->count; ++i) {
      const int rc = step_once(g->ctx[i], stats ? &stats[i] : nullptr);
      if (rc && first == PFC_OK) first = rc;
    }
    return first;
  }
  Level64 lv[kMaxGroup];
  bool warm[kMaxGroup];
  int key[3 * kMaxGroup] = {0};
  for (int i = 0; i < g->count; ++i) {
    warm[i] = step_prepare(g->ctx[i], &lv[i]);
    key[3 * i] = g->ctx[i]->variant;
    key[3 * i + 1] = g->ctx[i]->ia;
    key[3 * i + 2] = g->ctx[i]->graph_gen;
  }
  pfc_group::Graph* gr = nullptr;
  for (auto& x : g->graphs)
    if (memcmp(x.key, key, sizeof(key)) == 0) gr = &x;
  if (!gr) {
    pfc_group::Graph ng = {};
    memcpy(ng.key, key, sizeof(key));
    const int rc = group_build(g, warm, lv, &ng);
    if (rc) return rc;
    g->graphs.push_back(ng);
    gr = &g->graphs.back();
  }
  // after the work already enqueued on the contexts' own streams
  for (int i = 0; i < g->count; ++i) {
    PFC_CUDA(cudaEventRecord(g->ready[i], g->ctx[i]->st));
    PFC_CUDA(cudaStreamWaitEvent(g->st, g->ready[i], 0));
  }
  PFC_CUDA(cudaGraphLaunch(gr->exec, g->st));
  g->graph_launches += 1;
  PFC_CUDA(cudaStreamSynchronize(g->st));
  // the loop ran as many iterations as the slowest context needed
  int loop = 0;
  bool failed = false;
  for (int i = 0; i < g->count; ++i) {
    const StepState s = combined_state(g->ctx[i]);
    if (s.iters > loop) loop = s.iters;
    failed = failed || s.status == kStepNaN || s.status == kStepNoConv;
  }
  g->ctx[0]->prof.launches += 1 + 2 * loop;  // the group decisions and IF selections
  int first = PFC_OK;
  for (int i = 0; i < g->count; ++i) {
    pfc_ctx* c = g->ctx[i];
    // a context's body ran while it had a running member
    c->prof.launches += gr->pre[i] + gr->body[i] * (long long)combined_state(c).iters;
    // a context still running when another failed takes no step
    if (failed && combined_state(c).status == kStepRunning) {
      step_abandon(c);
      continue;
    }
    const int rc = step_finish(c, stats ? &stats[i] : nullptr);
    if (rc && first == PFC_OK) first = rc;
  }
  return first;
}

}  // namespace
}  // namespace pfc

int pfc_group_init(pfc_group** out, pfc_ctx* const* ctxs, int count, void* stream) {
  if (!out || !ctxs || count < 1 || count > kMaxGroup) return PFC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return PFC_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return PFC_EINVAL;
  }
  pfc_group* g = new pfc_group();
  g->count = count;
  g->st = (cudaStream_t)stream;
  g->graph_launches = 0;
  for (int i = 0; i < count; ++i) g->ctx[i] = ctxs[i];
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess && !ctxs[i]->cap_st)
      e = cudaStreamCreateWithFlags(&ctxs[i]->cap_st, cudaStreamNonBlocking);
  }
  if (e != cudaSuccess) {
    pfc_group_destroy(g);
    return cuda_fail(e, "pfc_group_init");
  }
  *out = g;
  return PFC_OK;
}

int pfc_group_step(pfc_group* g, int nsteps, pfc_step_stats* stats) {
  if (!g || nsteps < 0) return PFC_EINVAL;
  if (stats) memset(stats, 0, sizeof(*stats) * g->count);
  for (int s = 0; s < nsteps; ++s) {
    const int rc = group_step_once(g, stats);
    if (rc) return rc;
  }
  return PFC_OK;
}

long long pfc_group_graph_launches(const pfc_group* g) { return g ? g->graph_launches : -1; }

void pfc_group_destroy(pfc_group* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  for (auto& x : g->graphs)
    if (x.exec) cudaGraphExecDestroy(x.exec);
  if (g->cap_st) cudaStreamDestroy(g->cap_st);
  if (g->fork) cudaEventDestroy(g->fork);
  for (int i = 0; i < g->count; ++i) {
    if (g->join[i]) cudaEventDestroy(g->join[i]);
    if (g->ready[i]) cudaEventDestroy(g->ready[i]);
  }
  delete g;
}

const char* pfc_strerror(int code) {
  switch (code) {
    case PFC_OK: return "ok";
    case PFC_EINVAL: return "invalid argument";
    case PFC_ESIZE: return "grid size not supported or workspace too small";
    case PFC_ENOCONV: return "multigrid did not reach the tolerance within max_cycles";
    case PFC_ENAN: return "residual is NaN or Inf";
    case PFC_ECUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// Primitive operations
// ---------------------------------------------------------------------------

int pfc_op_source(int n, double h, double eps, const double* b, const double* c,
                  double* S2, double* S3, void* stream) {
  if (n < 2 || !b || !c || !S2 || !S3 || !(h > 0)) return PFC_EINVAL;
  PFC_CUDA(launch_source(make_lvl(n, h, eps, 0.0), b, c, S2, S3, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_smooth(int n, double h, double eps, double tau, int smoother, int sweeps,
                  double* phi, double* mu, double* om, const double* S1, const double* S2,
                  const double* S3, const double* b, void* stream) {
  if (n < 2 || (n & 1) || sweeps < 0 || !phi || !mu || !om || !S1 || !S2 || !S3 || !b)
    return PFC_EINVAL;
  if (smoother != PFC_NEWTON && smoother != PFC_PICARD) return PFC_EINVAL;
  PFC_CUDA(launch_smooth(make_lvl(n, h, eps, tau), smoother, sweeps, phi, mu, om, S1, S2,
                         S3, b, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_residual(int n, double h, double eps, double tau, const double* phi,
                    const double* mu, const double* om, const double* S1, const double* S2,
                    const double* S3, const double* b, double* r1, double* r2, double* r3,
                    void* stream) {
  if (n < 2 || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !r1 || !r2 || !r3)
    return PFC_EINVAL;
  PFC_CUDA(launch_residual(make_lvl(n, h, eps, tau), phi, mu, om, S1, S2, S3, b, r1, r2, r3,
                           (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_residual_restrict(int n, double h, double eps, double tau, const double* phi,
                             const double* mu, const double* om, const double* S1,
                             const double* S2, const double* S3, const double* b,
                             double* rc1, double* rc2, double* rc3, double* uc1,
                             double* uc2, double* uc3, void* stream) {
  if (n < 2 || (n & 1) || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !rc1 || !rc2 ||
      !rc3 || !uc1 || !uc2 || !uc3)
    return PFC_EINVAL;
  PFC_CUDA(launch_residual_restrict(make_lvl(n, h, eps, tau), phi, mu, om, S1, S2, S3, b,
                                    rc1, rc2, rc3, uc1, uc2, uc3, nullptr, nullptr,
                                    nullptr, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_restrict(int n, const double* fine, double* coarse, void* stream) {
  if (n < 2 || (n & 1) || !fine || !coarse) return PFC_EINVAL;
  PFC_CUDA(launch_restrict(n, fine, coarse, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_coarse_source(int n, double h, double eps, double tau, const double* uc1,
                         const double* uc2, const double* uc3, const double* bc,
                         double* r1, double* r2, double* r3, void* stream) {
  if (n < 1 || !uc1 || !uc2 || !uc3 || !bc || !r1 || !r2 || !r3) return PFC_EINVAL;
  PFC_CUDA(launch_coarse_source(make_lvl(n, h, eps, tau), uc1, uc2, uc3, bc, r1, r2, r3,
                                (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_prolong_correct(int n, const double* vc1, const double* vc2, const double* vc3,
                           const double* wc1, const double* wc2, const double* wc3,
                           double* u1, double* u2, double* u3, void* stream) {
  if (n < 2 || (n & 1) || !vc1 || !vc2 || !vc3 || !wc1 || !wc2 || !wc3 || !u1 || !u2 || !u3)
    return PFC_EINVAL;
  // e = v - w is formed in place over w, then interpolated and added.
  cudaStream_t st = (cudaStream_t)stream;
  PFC_CUDA(launch_coarse_diff(n / 2, vc1, vc2, vc3, (double*)wc1, (double*)wc2,
                              (double*)wc3, st));
  PFC_CUDA(launch_prolong_add(n, wc1, wc2, wc3, u1, u2, u3, st));
  return PFC_OK;
}

int pfc_op_coarse_solve(int n, double h, double eps, double tau, int smoother, int kind,
                        double weight, int max_sweeps, double* phi, double* mu, double* om,
                        double* t1, double* t2, double* t3, const double* S1,
                        const double* S2, const double* S3, const double* b,
                        void* stream) {
  if (n < 2 || (n & 1) || n > 16 || max_sweeps < 1 || !phi || !mu || !om || !S1 || !S2 ||
      !S3 || !b)
    return PFC_EINVAL;
  if (smoother != PFC_NEWTON && smoother != PFC_PICARD) return PFC_EINVAL;
  if (kind != PFC_SWEEP_RB && kind != PFC_SWEEP_JACOBI) return PFC_EINVAL;
  if (kind == PFC_SWEEP_JACOBI && (!t1 || !t2 || !t3 || !(weight > 0 && weight <= 1)))
    return PFC_EINVAL;
  PFC_CUDA(launch_coarse_solve(make_lvl(n, h, eps, tau), smoother, kind, weight, max_sweeps,
                               phi, mu, om, t1, t2, t3, S1, S2, S3, b,
                               (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_jacobi(int n, double h, double eps, double tau, int smoother, int sweeps,
                  double weight, double* phi, double* mu, double* om, double* t1, double* t2,
                  double* t3, const double* S1, const double* S2, const double* S3,
                  const double* b, void* stream) {
  if (n < 1 || sweeps < 0 || !phi || !mu || !om || !t1 || !t2 || !t3 || !S1 || !S2 || !S3 ||
      !b || !(weight > 0 && weight <= 1))
    return PFC_EINVAL;
  if (smoother != PFC_NEWTON && smoother != PFC_PICARD) return PFC_EINVAL;
  PFC_CUDA(launch_jacobi(make_lvl(n, h, eps, tau), smoother, sweeps, weight, phi, mu, om, t1,
                         t2, t3, S1, S2, S3, b, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_jacobi(int n, double h, double eps, double tau, int sweeps, double weight,
                      int zero_init, float* d1, float* d2, float* d3, float* t1, float* t2,
                      float* t3, const float* r1, const float* r2, const float* r3,
                      const float* q, void* stream) {
  if (n < 1 || sweeps < 0 || !d1 || !d2 || !d3 || !t1 || !t2 || !t3 || !r1 || !r2 || !r3 ||
      !q || !(weight > 0 && weight <= 1))
    return PFC_EINVAL;
  PFC_CUDA(launch_lin_jacobi32(make_lvl(n, h, eps, tau), sweeps, (float)weight,
                               zero_init != 0, d1, d2, d3, t1, t2, t3, r1, r2, r3, q,
                               (cudaStream_t)stream));
  return PFC_OK;
}

size_t pfc_reduce_scratch_bytes(int n) {
  (void)n;
  return ((size_t)kReduceBlocks * kReduceComps + kReduceComps) * sizeof(double);
}

static int op_diagnostics(int n, double h, double eps, const double* a, const double* b,
                          bool df_fields, void* scratch, double* out, void* stream) {
  if (n < 2 || !a || !b || !scratch || !out || !(h > 0)) return PFC_EINVAL;
  double* partials = (double*)scratch;
  double* dout = partials + (size_t)kReduceBlocks * kReduceComps;
  double hout[8];
  return diagnostics(n, h, &eps, 1, a, b, nullptr, nullptr, df_fields, partials, dout, hout,
                     (cudaStream_t)stream, out);
}

int pfc_op_diagnostics(int n, double h, double eps, const double* a, const double* b,
                       void* scratch, double* out, void* stream) {
  return op_diagnostics(n, h, eps, a, b, false, scratch, out, stream);
}

int pfc_op_diagnostics_df(int n, double h, double eps, const float* a, const float* b,
                          void* scratch, double* out, void* stream) {
  return op_diagnostics(n, h, eps, reinterpret_cast<const double*>(a),
                        reinterpret_cast<const double*>(b), true, scratch, out, stream);
}

int pfc_op_residual_norm(int n, double h, double eps, double tau, const double* phi,
                         const double* mu, const double* om, const double* S1,
                         const double* S2, const double* S3, const double* b,
                         void* scratch, double* out, void* stream) {
  if (n < 2 || !(h > 0) || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !scratch || !out)
    return PFC_EINVAL;
  double* partials = (double*)scratch;
  double* dout = partials + (size_t)kReduceBlocks * kReduceComps;
  double hv = 0;
  cudaStream_t st = (cudaStream_t)stream;
  PFC_CUDA(launch_residual_norm2(make_lvl(n, h, eps, tau), phi, mu, om, S1, S2, S3, b,
                                 partials, dout, st));
  PFC_CUDA(cudaMemcpyAsync(&hv, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFC_CUDA(cudaStreamSynchronize(st));
  *out = sqrt(hv / (3.0 * (double)n * n * n));
  return PFC_OK;
}

int pfc_op_guess(int n, double h, double eps, const double* b, const double* c, double* S2,
                 double* S3, double* phi, double* mu, double* om, void* stream) {
  if (n < 1 || !(h > 0) || !b || !c || !S2 || !S3 || !phi || !mu || !om) return PFC_EINVAL;
  PFC_CUDA(launch_guess(make_lvl(n, h, eps, 1.0), b, c, S2, S3, phi, mu, om,
                        (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_guess_df(int n, double h, double eps, const float* b, const float* c, float* S2,
                    float* S3, float* phi, float* mu, float* om, void* stream) {
  if (n < 1 || !(h > 0) || !b || !c || !S2 || !S3 || !phi || !mu || !om) return PFC_EINVAL;
  auto D = [](float* p) { return reinterpret_cast<float2*>(p); };
  PFC_CUDA(launch_guess_df(make_lvl(n, h, eps, 1.0), reinterpret_cast<const float2*>(b),
                           reinterpret_cast<const float2*>(c), D(S2), D(S3), D(phi), D(mu),
                           D(om), (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_round_f32(long long count, const double* x, float* y, void* stream) {
  if (count < 0 || (count > 0 && (!x || !y))) return PFC_EINVAL;
  PFC_CUDA(launch_round_f32(count, x, y, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_widen_f64(long long count, const float* x, double* y, void* stream) {
  if (count < 0 || (count > 0 && (!x || !y))) return PFC_EINVAL;
  PFC_CUDA(launch_widen_f64(count, x, y, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_df_from_f64(long long count, const double* x, float* y, void* stream) {
  if (count < 0 || (count > 0 && (!x || !y))) return PFC_EINVAL;
  PFC_CUDA(launch_df_from_f64(count, x, reinterpret_cast<float2*>(y), (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_df_to_f64(long long count, const float* y, double* x, void* stream) {
  if (count < 0 || (count > 0 && (!x || !y))) return PFC_EINVAL;
  PFC_CUDA(launch_df_to_f64(count, reinterpret_cast<const float2*>(y), x,
                            (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_source_df(int n, double h, double eps, const float* b, const float* c, float* S2,
                     float* S3, void* stream) {
  if (n < 1 || !(h > 0) || !b || !c || !S2 || !S3) return PFC_EINVAL;
  PFC_CUDA(launch_source_df(make_lvl(n, h, eps, 1.0), reinterpret_cast<const float2*>(b),
                            reinterpret_cast<const float2*>(c), reinterpret_cast<float2*>(S2),
                            reinterpret_cast<float2*>(S3), (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_defect(int n, double h, double eps, double tau, const double* phi,
                  const double* mu, const double* om, const double* S1, const double* S2,
                  const double* S3, const double* b, float* r1, float* r2, float* r3,
                  float* q, void* scratch, double* out, double* lap, void* stream) {
  if (n < 2 || (n & 1) || !(h > 0) || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !r1 ||
      !r2 || !r3 || !q || !scratch || !out)
    return PFC_EINVAL;
  double* partials = (double*)scratch;
  double* dout = partials + (size_t)kReduceBlocks * kReduceComps;
  double hv = 0;
  cudaStream_t st = (cudaStream_t)stream;
  PFC_CUDA(launch_defect64(make_lvl(n, h, eps, tau), phi, mu, om, S1, S2, S3, b, r1, r2, r3, q,
                           partials, dout, st, lap));
  PFC_CUDA(cudaMemcpyAsync(&hv, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFC_CUDA(cudaStreamSynchronize(st));
  *out = sqrt(hv / (3.0 * (double)n * n * n));
  return PFC_OK;
}

int pfc_op_start_extrap(int n, double h, double eps, double tau, const double* b,
                        const double* c, const double* lapb, const double* lapc,
                        const double* mu0, const double* om0, const double* lapmu0,
                        const double* lapom0, double* mu1, double* om1, double* lapmu1,
                        double* lapom1, double* S2, double* S3, double* phi, double* lap,
                        float* r1, float* r2, float* r3, float* q, void* scratch, double* out,
                        void* stream) {
  if (n < 2 || (n & 1) || !(h > 0) || !b || !c || !lapb || !lapc || !mu0 || !om0 || !lapmu0 ||
      !lapom0 || !mu1 || !om1 || !lapmu1 || !lapom1 || !S2 || !S3 || !phi || !lap || !r1 ||
      !r2 || !r3 || !q || !scratch || !out)
    return PFC_EINVAL;
  double* partials = (double*)scratch;
  double* dout = partials + (size_t)kReduceBlocks * kReduceComps;
  double hv = 0;
  cudaStream_t st = (cudaStream_t)stream;
  PFC_CUDA(launch_start64_extrap(make_lvl(n, h, eps, tau), b, c, lapb, lapc, mu0, om0, lapmu0,
                                 lapom0, mu1, om1, lapmu1, lapom1, S2, S3, phi, r1, r2, r3, q,
                                 partials, dout, lap, st));
  PFC_CUDA(cudaMemcpyAsync(&hv, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFC_CUDA(cudaStreamSynchronize(st));
  *out = sqrt(hv / (3.0 * (double)n * n * n));
  return PFC_OK;
}

int pfc_op_defect_df(int n, double h, double eps, double tau, const float* phi, const float* mu,
                  const float* om, const float* S1, const float* S2, const float* S3,
                  const float* b, float* r1, float* r2, float* r3, float* q, void* scratch,
                  double* out, float* lap, void* stream) {
  if (n < 2 || (n & 1) || !(h > 0) || !phi || !mu || !om || !S1 || !S2 || !S3 || !b || !r1 ||
      !r2 || !r3 || !q || !scratch || !out)
    return PFC_EINVAL;
  double* partials = (double*)scratch;
  double* dout = partials + (size_t)kReduceBlocks * kReduceComps;
  double hv = 0;
  cudaStream_t st = (cudaStream_t)stream;
  auto D = [](const float* p) { return reinterpret_cast<const float2*>(p); };
  PFC_CUDA(launch_defect_df(make_lvl(n, h, eps, tau), D(phi), D(mu), D(om), D(S1), D(S2),
                            D(S3), D(b), r1, r2, r3, q, partials, dout, st,
                            reinterpret_cast<float2*>(lap)));
  PFC_CUDA(cudaMemcpyAsync(&hv, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFC_CUDA(cudaStreamSynchronize(st));
  *out = sqrt(hv / (3.0 * (double)n * n * n));
  return PFC_OK;
}

int pfc_op_lin_smooth(int n, double h, double eps, double tau, int sweeps, int zero_init,
                      float* d1, float* d2, float* d3, const float* r1, const float* r2,
                      const float* r3, const float* q, void* stream) {
  if (n < 2 || (n & 1) || sweeps < 0 || !d1 || !d2 || !d3 || !r1 || !r2 || !r3 || !q)
    return PFC_EINVAL;
  PFC_CUDA(launch_lin_smooth32(make_lvl(n, h, eps, tau), sweeps, zero_init != 0, d1, d2, d3,
                               r1, r2, r3, q, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_residual_restrict(int n, double h, double eps, double tau, int zero_init,
                                 const float* d1, const float* d2, const float* d3,
                                 const float* r1, const float* r2, const float* r3,
                                 const float* q, float* c1, float* c2, float* c3,
                                 void* stream) {
  if (n < 2 || (n & 3) || !(h > 0) || !r1 || !r2 || !r3 || !c1 || !c2 || !c3 ||
      (!zero_init && (!d1 || !d2 || !d3 || !q)))
    return PFC_EINVAL;
  PFC_CUDA(launch_lin_residual_restrict32(make_lvl(n, h, eps, tau), zero_init != 0, d1, d2, d3,
                                          r1, r2, r3, q, c1, c2, c3, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_restrict_chain(int n, double h, double eps, double tau, int zero_init,
                              int levels, const float* d1, const float* d2, const float* d3,
                              const float* r1, const float* r2, const float* r3,
                              const float* q, float* c1, float* c2, float* c3, float* e1,
                              float* e2, float* e3, float* g1, float* g2, float* g3,
                              void* stream) {
  if (n < 32 || (n % 32) != 0 || !(h > 0) || levels < 2 || levels > 3 || !r1 || !r2 || !r3 ||
      !c1 || !c2 || !c3 || !e1 || !e2 || !e3 ||
      (levels == 3 && (!g1 || !g2 || !g3)) || (!zero_init && (!d1 || !d2 || !d3 || !q)))
    return PFC_EINVAL;
  float* const c[3] = {c1, c2, c3};
  float* const e[3] = {e1, e2, e3};
  float* const g[3] = {g1, g2, g3};
  PFC_CUDA(launch_lin_restrict_chain32(make_lvl(n, h, eps, tau), zero_init != 0, levels - 1, d1,
                                       d2, d3, r1, r2, r3, q, c, e, g, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_restrict_q(int n, int levels, const float* q, float* c, float* e, float* g,
                      void* stream) {
  if (n < 2 || (n & 1) || levels < 1 || levels > 3 || !q || !c || (levels >= 2 && !e) ||
      (levels == 3 && !g) || (levels >= 2 && (n % 32) != 0))
    return PFC_EINVAL;
  PFC_CUDA(launch_restrict_q(n, levels - 1, q, c, e, g, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_prolong(int n, int assign, const float* e1, const float* e2, const float* e3,
                       float* d1, float* d2, float* d3, void* stream) {
  if (n < 2 || (n & 3) || !e1 || !e2 || !e3 || !d1 || !d2 || !d3) return PFC_EINVAL;
  if (assign < 0 || assign > (PFC_PROLONG_ASSIGN | PFC_PROLONG_SKIP_COLOUR0)) return PFC_EINVAL;
  PFC_CUDA(launch_prolong32(n, (assign & PFC_PROLONG_ASSIGN) != 0,
                            (assign & PFC_PROLONG_SKIP_COLOUR0) != 0, e1, e2, e3, d1, d2, d3,
                            (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_smooth_correct(int n, double h, double eps, double tau, int sweeps, float* d1,
                              float* d2, float* d3, const float* r1, const float* r2,
                              const float* r3, const float* q, double* u1, double* u2,
                              double* u3, void* stream) {
  if (n < 4 || n % 4 != 0 || !(h > 0) || sweeps < 1 || !d1 || !d2 || !d3 || !r1 || !r2 || !r3 ||
      !q || !u1 || !u2 || !u3 || ((uintptr_t)u1 | (uintptr_t)u2 | (uintptr_t)u3) % 16 != 0)
    return PFC_EINVAL;
  PFC_CUDA(launch_lin_smooth_correct32(make_lvl(n, h, eps, tau), sweeps, d1, d2, d3, r1, r2, r3,
                                       q, u1, u2, u3, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_lin_prolong_smooth(int n, double h, double eps, double tau, int kind, int assign,
                              double weight, const float* e1, const float* e2, const float* e3,
                              float* d1, float* d2, float* d3, float* t1, float* t2, float* t3,
                              const float* r1, const float* r2, const float* r3, const float* q,
                              void* stream) {
  if (n < 32 || n % 32 != 0 || !(h > 0) || (kind != PFC_SWEEP_RB && kind != PFC_SWEEP_JACOBI) ||
      (assign != 0 && assign != PFC_PROLONG_ASSIGN) || !e1 || !e2 || !e3 || !d1 || !d2 || !d3 ||
      !t1 || !t2 || !t3 || !r1 || !r2 || !r3 || !q ||
      (kind == PFC_SWEEP_JACOBI && !(weight > 0 && weight <= 1)))
    return PFC_EINVAL;
  PFC_CUDA(launch_lin_prolong_smooth32(make_lvl(n, h, eps, tau), kind, assign != 0, (float)weight,
                                       e1, e2, e3, d1, d2, d3, t1, t2, t3, r1, r2, r3, q,
                                       (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_correct(int n, double* u1, double* u2, double* u3, const float* d1,
                   const float* d2, const float* d3, void* stream) {
  if (n < 2 || (n & 1) || !u1 || !u2 || !u3 || !d1 || !d2 || !d3) return PFC_EINVAL;
  PFC_CUDA(launch_correct64(n, u1, u2, u3, d1, d2, d3, (cudaStream_t)stream));
  return PFC_OK;
}

int pfc_op_correct_df(int n, float* u1, float* u2, float* u3, const float* d1,
                      const float* d2, const float* d3, void* stream) {
  if (n < 2 || (n & 1) || !u1 || !u2 || !u3 || !d1 || !d2 || !d3) return PFC_EINVAL;
  PFC_CUDA(launch_correct_df(n, reinterpret_cast<float2*>(u1), reinterpret_cast<float2*>(u2),
                             reinterpret_cast<float2*>(u3), d1, d2, d3, (cudaStream_t)stream));
  return PFC_OK;
}

}  // extern "C"
