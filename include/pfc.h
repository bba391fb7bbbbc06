/*
 * pfc.h - C ABI of libpfc, the GB300 (sm_103a) solver for the second-order
 * convex-splitting finite-difference scheme of the periodic 3D phase field
 * crystal (PFC) equation, each time step solved by a nonlinear FAS multigrid
 * V-cycle (Dong, Feng, Wang, Wise, Zhang, arXiv:1611.06288).
 *
 * Model (Section 3, Eq. 1.10, in the split form of Section 5, Eqs. 5.1-5.10,
 * mobility M = 1): given phi^k = b and phi^{k-1} = c on the periodic
 * cell-centred grid of n^3 cells, h = L/n, find u = (phi^{k+1}, mu, omega) with
 *   N1 = phi - tau Lap_h mu                                    = S1 = b
 *   N2 = mu - (phi+b)(phi^2+b^2)/4 - (1-eps)/2 phi - Lap_h omega
 *                                      = S2 = (1-eps)/2 b + 3 Lap_h b - Lap_h c
 *   N3 = omega - Lap_h phi / 2                                 = S3 = Lap_h b / 2
 * where Lap_h is the 7-point Laplacian of Section 2.
 *
 * Conventions for every entry point:
 *  - A "field" is n*n*n doubles (or floats where stated), x fastest: cell
 *    (i, j, k) is element i + n*(j + n*k).  Fields must not overlap unless
 *    stated.
 *  - Pointers named d_* are device pointers on the current CUDA device.
 *    Pointers named any_* may be device or host memory (copied with
 *    cudaMemcpyDefault; pinned host memory keeps the copy asynchronous).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls return before it completes
 *    unless stated as blocking.
 *  - The library never frees caller memory.  It allocates no device memory:
 *    the caller passes a workspace of pfc_workspace_bytes() bytes.  The only
 *    host allocation is the context itself and a small pinned readback slot.
 *  - Return value: PFC_OK (0) or a negative PFC_E* code; nothing is printed
 *    and nothing aborts.  pfc_strerror() gives a message.
 */
#ifndef PFC_H
#define PFC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFC_OK       0
#define PFC_EINVAL  -1  /* bad argument (null pointer, eps >= 1, tau <= 0 ...) */
#define PFC_ESIZE   -2  /* n not coarsenable to an even coarsest size, or workspace too small */
#define PFC_ENOCONV -3  /* max_cycles reached before the residual tolerance */
#define PFC_ENAN    -4  /* residual became NaN or Inf */
#define PFC_ECUDA   -5  /* a CUDA runtime call failed */

#define PFC_FP64  0     /* FAS V-cycles entirely in FP64 (Algorithm 1) */
#define PFC_MIXED 1     /* FP64 defect correction around FP32 multigrid */
#define PFC_MIXED_DF 2  /* the same with the outer state, residual, update and
                           energy/mass sums in double-float (FP32 pairs) */

#define PFC_NEWTON 0    /* pointwise Newton linearisation of the cubic term */
#define PFC_PICARD 1    /* the paper's local Picard linearisation (Section 5) */

#define PFC_POLICY_HYBRID 0  /* red-black sweeps where the level stiffness
                                s = 108 tau / h^6 is >= stiff_hi or <= stiff_lo,
                                damped collective Jacobi sweeps in between */
#define PFC_POLICY_RB     1  /* the paper's red-black sweep on every level */

#define PFC_SWEEP_RB     0   /* level smoother kinds (pfc_level_info) */
#define PFC_SWEEP_JACOBI 1

typedef struct pfc_ctx pfc_ctx;   /* opaque; owns no device memory */

typedef struct pfc_params {
  int    n;            /* cells per side (cube only, Section 2); n >= 4, even */
  double L;            /* side of the periodic box; h = L / n */
  double eps;          /* model epsilon, 0 <= eps < 1 */
  double dt;           /* time step tau > 0 */
  int    nu1, nu2;     /* pre/post smoothing sweeps (Algorithm 1); >= 0 */
  double tol;          /* absolute tolerance on the fine-grid residual (FP64;
                          double-float for PFC_MIXED_DF), RMS over the three
                          components */
  int    max_cycles;   /* V-cycles (or defect corrections) per step */
  int    precision;    /* PFC_FP64, PFC_MIXED or PFC_MIXED_DF */
  int    smoother;     /* PFC_NEWTON or PFC_PICARD (FP64 path) */
  int    coarsest;     /* coarsen while the level size is even and larger
                          than this; the last level is solved by sweeping to
                          convergence.  >= 2 */
  int    inner_cycles; /* mixed paths: FP32 V-cycles per defect correction */
  int    policy;       /* PFC_POLICY_HYBRID or PFC_POLICY_RB */
  double jacobi_weight;/* damping of the collective Jacobi sweep, (0, 1] */
  int    jacobi_factor;/* Jacobi sweeps per requested sweep on coarse Jacobi levels */
  int    jacobi_factor0;/* the same on the finest level */
  double stiff_hi, stiff_lo; /* thresholds of the hybrid policy */
  double coarse_stiffness;   /* mixed paths: also stop coarsening at the first
                                level (below the finest, of at most 16^3
                                cells) whose stiffness 108 tau/h^6 is <= this:
                                there the system is nearly pointwise and FP32
                                sweeps solve it */
  int    coarse_sweeps;      /* mixed paths: most FP32 sweeps on the coarsest
                                level (stopping earlier once the largest change
                                is below 1e-6 of the largest value) */
  int    guess;              /* initial iterate of a step: PFC_GUESS_PREVIOUS,
                                PFC_GUESS_EXTRAPOLATE or
                                PFC_GUESS_EXTRAPOLATE_ALL */
  double mobility_m0, mobility_m2;
                             /* mobility M(phi) = m0 + m2 phi^2 (m0 > 0,
                                m2 >= 0), evaluated on every face at
                                A phi_*, phi_* = 3/2 phi^k - 1/2 phi^{k-1}
                                (Section 5): N1 = phi - tau d(M D mu).
                                m0 = 1, m2 = 0 (the default) is M == 1.
                                Any other M needs PFC_MIXED and one member:
                                the FP64 defect uses the face mobilities,
                                the FP32 correction solve the reference
                                mobility m0 + m2 mean(phi^2) measured at
                                pfc_set_state (an approximate Jacobian: the
                                converged state is exact) */
  int    cluster_tail;       /* mixed paths: 1 runs the coarse part of each
                                FP32 V-cycle from the first level of at most
                                32^3 cells whose size is a multiple of 8 and
                                at least 16 as one launch of an 8-CTA
                                thread-block cluster per member (levels in z
                                slabs over the CTAs, neighbour planes through
                                distributed shared memory) where the device
                                can run such a cluster; 2 uses the cluster
                                only where the single-block tail would start
                                (levels of at most 16^3 cells), the levels
                                above keeping their full-GPU launches (1464
                                against 1425 steps/s on the 128^3 smooth-mode
                                workload); 0 (default) keeps separate
                                launches down to 16^3 and one block below,
                                faster for ensembles.  Same arithmetic up to
                                summation order and the approximate division
                                of the pointwise solve */
  int    step_diagnostics;   /* 1: every step also forms the energy/mass sums
                                of its new state in the same graph launch
                                (no further launch or synchronisation), and
                                pfc_diagnostics, pfc_batch_diagnostics,
                                pfc_energy and pfc_mass return them until the
                                state changes; 0 (default): they are formed
                                on request */
  int    defect_planes;      /* PFC_MIXED: planes per thread block of the FP64
                                defect (its tiles are 32 x 8 cells x this many
                                planes); 0 (default) chooses them from the SM
                                count (fewest waves), a value > 0 fixes them
                                (an autotuner's choice; larger than n means
                                n) */
} pfc_params;

#define PFC_GUESS_PREVIOUS    0  /* phi^{k+1} := phi^k; mu, omega from the last
                                    step */
#define PFC_GUESS_EXTRAPOLATE 1  /* phi^{k+1} := 2 phi^k - phi^{k-1} (second
                                    order in tau), then the omega and mu that
                                    satisfy rows 3 and 2 of N(u) = S exactly:
                                    omega = Lap(phi + phi^k)/2, mu = S2 +
                                    f(phi, phi^k) + (1-eps)/2 phi + Lap omega.
                                    The step converges to the same solution
                                    (Prop. 3.1) from a residual O(tau^2) in
                                    the first row only. */
#define PFC_GUESS_EXTRAPOLATE_ALL 2  /* phi, mu and omega of step k+1 :=
                                    2 u^k - u^{k-1} from the two last
                                    converged steps (u^k alone after a start,
                                    pfc_set_state or a failed step); the
                                    first defect is O(tau^2) in all three rows
                                    and a smooth step converges in one
                                    correction.  Holds a second mu and omega
                                    (16 n^3 bytes per member more; 32 n^3 on
                                    PFC_MIXED with M == 1, which also keeps
                                    their Laplacians and then forms the
                                    iterate and its first defect pointwise
                                    from them); not with PFC_MIXED_DF
                                    (EINVAL). */

typedef struct pfc_step_stats {
  int    steps;        /* steps completed by the call */
  int    cycles_last;  /* V-cycles (FP64) or corrections (mixed) in the last step */
  int    cycles_total; /* summed over the call */
  double residual;     /* final RMS residual of the last step */
  double residual0;    /* RMS residual of the initial guess of the last step */
} pfc_step_stats;

/* Fill *p with defaults: V(2,2), Newton smoother, tol 1e-9, max_cycles 50,
 * FP64, coarsest 2, inner_cycles 1, hybrid policy with Jacobi weight 0.7,
 * factor 4 (2 on the finest level), stiff_hi 1000, stiff_lo 0.25,
 * coarse_stiffness 0.05, coarse_sweeps 4, guess PFC_GUESS_PREVIOUS, mobility
 * m0 = 1, m2 = 0, cluster_tail 0, step_diagnostics 0, defect_planes 0.  n, L,
 * eps, dt are set to 0.
 *
 * Why the hybrid policy: on the split system the red-black pointwise sweep
 * of Section 5 amplifies the error pair made of the constant mode and the
 * checkerboard mode by more than 1 per sweep once 108 tau/h^6 (the product
 * of the tau/h^2, 6/h^2 and 3/h^2 couplings) is of order 1 to 1000, and its
 * V-cycles then stall or diverge.  The damped collective Jacobi sweep does not
 * couple the two modes. */
void pfc_default_params(pfc_params* p);

/* Size, spacing and smoother kind (PFC_SWEEP_*) of multigrid level `level`
 * (0 = finest) for *p; PFC_EINVAL past the coarsest level.  Host only. */
int pfc_level_info(const pfc_params* p, int level, int* n, double* h, int* kind);

/* Bytes of device workspace pfc_init needs for *p (0 if *p is invalid). */
size_t pfc_workspace_bytes(const pfc_params* p);

/* Create a solver context.
 * d_workspace: >= pfc_workspace_bytes(p) bytes of device memory, 256-byte
 *   aligned, owned by the caller and kept alive until pfc_destroy.
 * any_phi0: phi^0 (a field).  any_phi1: phi^1, or NULL to start with the
 *   rule phi^{-1} := phi^0 (the first step then uses c = b).
 * Copies the initial fields into the workspace and returns after they are
 * enqueued on `stream`.  Errors: PFC_EINVAL, PFC_ESIZE, PFC_ECUDA. */
int pfc_init(pfc_ctx** out, const pfc_params* p, void* d_workspace,
             size_t workspace_bytes, const double* any_phi0,
             const double* any_phi1, void* stream);

/* Advance nsteps time steps of Eq. 1.10.  Each step forms S (Eqs. 5.8-5.10)
 * and runs V-cycles (or defect corrections) until the RMS residual <= tol.
 * By default a step is one CUDA graph launch whose convergence loop is a
 * device-side WHILE node (the graph of each of the three positions of the
 * phi ring is built on first use); with graphs off, or while kernel timing is
 * enabled, the loop runs on the host with one readback per iteration.
 * Blocking.  On PFC_ENOCONV / PFC_ENAN phi is not advanced (mu and omega are
 * reset to zero after a NaN).  stats may be NULL. */
int pfc_step(pfc_ctx* ctx, int nsteps, pfc_step_stats* stats);

/* Switch the graph execution of pfc_step on (default) or off. */
int pfc_use_graphs(pfc_ctx* ctx, int on);

/* Replace the state by (phi^k, phi^{k-1}) = (any_phi, any_phi_prev);
 * any_phi_prev NULL means phi^{k-1} := phi^k.  mu and omega are kept as warm
 * starts.  Enqueued on the context stream. */
int pfc_set_state(pfc_ctx* ctx, const double* any_phi, const double* any_phi_prev);

/* Copy phi^k (the newest level) / mu^{k-1/2} / omega^{k-1/2} to any_dst.
 * Enqueued on the context stream (synchronise before reading host memory). */
int pfc_get_phi(pfc_ctx* ctx, double* any_dst);
int pfc_get_mu(pfc_ctx* ctx, double* any_dst);
int pfc_get_omega(pfc_ctx* ctx, double* any_dst);

/* Discrete energy F_h(phi^k) (Eq. 2.1) and the modified energy
 * F_h(phi^k) + 1/2 ||grad_h(phi^k - phi^{k-1})||^2 (Prop. 3.1); either
 * output may be NULL.  Blocking.  Deterministic (fixed summation order). */
int pfc_energy(pfc_ctx* ctx, double* F, double* F_modified);

/* Mass (phi^k, 1)_2 = h^3 sum phi^k (Section 2).  Blocking, deterministic. */
int pfc_mass(pfc_ctx* ctx, double* mass);

/* All diagnostics of phi^k in one pass (blocking, deterministic):
 * out[0] = F_h(phi^k), out[1] = modified energy, out[2] = mass,
 * out[3] = ||grad_h phi^k||^2. */
int pfc_diagnostics(pfc_ctx* ctx, double out[4]);

/* Steps taken since pfc_init (counting phi^1 when it was given). */
int pfc_step_index(const pfc_ctx* ctx);

/* Kernel launches enqueued by pfc_step / pfc_energy / pfc_mass /
 * pfc_diagnostics since pfc_init (a host-side counter). */
long long pfc_launch_count(const pfc_ctx* ctx);

void pfc_destroy(pfc_ctx* ctx);
const char* pfc_strerror(int code);

/* Detail of the last PFC_ECUDA returned on this host thread ("" if none). */
const char* pfc_last_error(void);

/* ------------------------------------------------------------------------
 * Kernel timing (tracing).  When enabled for a set of kernel classes, every
 * launch of those classes made by pfc_step is bracketed by CUDA events on the
 * context stream and its device time is accumulated per (class, level);
 * level 0 is the finest grid.  Timing adds two event records per bracketed
 * launch group and nothing else.
 * --------------------------------------------------------------------- */
#define PFC_K_SOURCE            0   /* S2, S3 (Eqs. 5.9-5.10) */
#define PFC_K_RESTRICT          1   /* 8-cell average of phi^k or q per level */
#define PFC_K_SMOOTH            2   /* FP64 red-black half-sweeps */
#define PFC_K_RESIDUAL_RESTRICT 3   /* FP64 residual + restriction */
#define PFC_K_COARSE_SOURCE     4   /* FAS coarse right-hand side */
#define PFC_K_PROLONG           5   /* FP64 correction e = v - w, u += P e */
#define PFC_K_COARSE_SOLVE      6   /* FP64 coarsest-level solve */
#define PFC_K_RESIDUAL_NORM     7   /* FP64 residual norm (convergence test) */
#define PFC_K_DEFECT            8   /* mixed: FP64 or df residual -> FP32, q */
#define PFC_K_LIN_SMOOTH        9   /* mixed: FP32 red-black half-sweeps */
#define PFC_K_LIN_RESTRICT     10   /* mixed: FP32 residual + restriction */
#define PFC_K_LIN_PROLONG      11   /* mixed: FP32 d += P d_c */
#define PFC_K_LIN_COARSE       12   /* mixed: FP32 coarsest-level solve */
#define PFC_K_CORRECT          13   /* mixed: u += d in FP64 or double-float */
#define PFC_K_START            14   /* mixed: pointwise start of a step (S2, S3,
                                       the iterate and its first defect from
                                       stored Laplacians) */
#define PFC_K_COUNT            15
#define PFC_PROFILE_LEVELS     24

/* Enable timing for the classes whose bit (1 << PFC_K_*) is set in mask
 * (0 disables) and clear the accumulators.  Creates CUDA events on first use. */
int pfc_profile_enable(pfc_ctx* ctx, unsigned mask);

/* Accumulated kernel launches and device milliseconds of one class on one
 * level since pfc_profile_enable.  Synchronises the context stream. */
int pfc_profile_read(pfc_ctx* ctx, int kclass, int level, long long* launches,
                     double* ms);

/* ------------------------------------------------------------------------
 * Primitive operations: one per stage of the V-cycle, on caller device
 * buffers, enqueued on `stream`.  n is the level size (cells per side), h its
 * spacing.  They exist so that every stage can be checked on its own; the
 * solver above calls the same kernels.
 * --------------------------------------------------------------------- */

/* S2 = (1-eps)/2 b + 3 Lap_h b - Lap_h c and S3 = Lap_h b / 2
 * (Eqs. 5.9-5.10); S1 is b itself (Eq. 5.8). */
int pfc_op_source(int n, double h, double eps, const double* d_b,
                  const double* d_c, double* d_S2, double* d_S3, void* stream);

/* `sweeps` red-black nonlinear Gauss-Seidel sweeps on u = (phi, mu, om) in
 * place (Section 5): red cells ((i+j+k) even) first, each solving the
 * pointwise 3x3 system with its neighbours fixed; `smoother` selects the
 * Newton or the paper's Picard linearisation.  n even. */
int pfc_op_smooth(int n, double h, double eps, double tau, int smoother,
                  int sweeps, double* d_phi, double* d_mu, double* d_om,
                  const double* d_S1, const double* d_S2, const double* d_S3,
                  const double* d_b, void* stream);

/* `sweeps` damped collective Jacobi sweeps on u = (phi, mu, om): every cell
 * solves the same pointwise 3x3 system as pfc_op_smooth with the neighbours
 * of the previous sweep and moves by `weight` of the change.  d_t1..3 are
 * three scratch fields; the result is in d_phi, d_mu, d_om. */
int pfc_op_jacobi(int n, double h, double eps, double tau, int smoother,
                  int sweeps, double weight, double* d_phi, double* d_mu,
                  double* d_om, double* d_t1, double* d_t2, double* d_t3,
                  const double* d_S1, const double* d_S2, const double* d_S3,
                  const double* d_b, void* stream);

/* r = S - N(u) (Algorithm 1 "Residual"), full fine-grid fields. */
int pfc_op_residual(int n, double h, double eps, double tau,
                    const double* d_phi, const double* d_mu, const double* d_om,
                    const double* d_S1, const double* d_S2, const double* d_S3,
                    const double* d_b, double* d_r1, double* d_r2, double* d_r3,
                    void* stream);

/* Fused residual + restriction (Algorithm 1 "Residual", "Coarsening"): for
 * every coarse cell, the 8-cell averages of r = S - N(u) and of u are written
 * to d_rc* and d_uc* (fields of (n/2)^3).  n even. */
int pfc_op_residual_restrict(int n, double h, double eps, double tau,
                             const double* d_phi, const double* d_mu,
                             const double* d_om, const double* d_S1,
                             const double* d_S2, const double* d_S3,
                             const double* d_b, double* d_rc1, double* d_rc2,
                             double* d_rc3, double* d_uc1, double* d_uc2,
                             double* d_uc3, void* stream);

/* 8-cell average of one field onto the grid of size n/2. */
int pfc_op_restrict(int n, const double* d_fine, double* d_coarse, void* stream);

/* FAS coarse source S_c = N_c(u_c) + r_c on a level of size n, spacing h,
 * with b_c the restricted phi^k (in place over d_r*: on return d_r* hold
 * S_c).  Algorithm 1 "Solve"/"Recursion" right-hand side. */
int pfc_op_coarse_source(int n, double h, double eps, double tau,
                         const double* d_uc1, const double* d_uc2,
                         const double* d_uc3, const double* d_bc,
                         double* d_r1, double* d_r2, double* d_r3, void* stream);

/* Correction u += P(v_c - w_c) for the three components (Algorithm 1
 * "Correction"): P is trilinear cell-centred interpolation from the level of
 * size n/2; v_c the coarse solution, w_c the restricted u it started from. */
int pfc_op_prolong_correct(int n, const double* d_vc1, const double* d_vc2,
                           const double* d_vc3, const double* d_wc1,
                           const double* d_wc2, const double* d_wc3,
                           double* d_u1, double* d_u2, double* d_u3,
                           void* stream);

/* Coarsest-level solve of N(u) = S by sweeps until the largest relative
 * change is below 1e-14 or max_sweeps; one thread block.  kind = PFC_SWEEP_RB
 * or PFC_SWEEP_JACOBI (weight `weight`, scratch d_t1..3).  n even, n <= 16. */
int pfc_op_coarse_solve(int n, double h, double eps, double tau, int smoother,
                        int kind, double weight, int max_sweeps, double* d_phi,
                        double* d_mu, double* d_om, double* d_t1, double* d_t2,
                        double* d_t3, const double* d_S1, const double* d_S2,
                        const double* d_S3, const double* d_b, void* stream);

/* Diagnostics of one field pair (Section 2 norms, Eq. 2.1), blocking:
 * out[0] = F_h(a), out[1] = F_h(a) + 1/2 ||grad_h(a - b)||^2, out[2] = mass
 * h^3 sum a, out[3] = ||grad_h a||^2.  d_scratch: pfc_reduce_scratch_bytes(n)
 * bytes of device memory. */
size_t pfc_reduce_scratch_bytes(int n);
int pfc_op_diagnostics(int n, double h, double eps, const double* d_a,
                       const double* d_b, void* d_scratch, double* out,
                       void* stream);

/* The same diagnostics of df fields d_a, d_b (2*n^3 floats each, see the df
 * layout below), with the per-cell terms and all sums in double-float. */
int pfc_op_diagnostics_df(int n, double h, double eps, const float* d_a,
                          const float* d_b, void* d_scratch, double* out,
                          void* stream);

/* RMS residual sqrt(sum_c sum r_c^2 / (3 n^3)) of u (blocking).  n >= 2,
 * h > 0 and non-null pointers, else PFC_EINVAL. */
int pfc_op_residual_norm(int n, double h, double eps, double tau,
                         const double* d_phi, const double* d_mu,
                         const double* d_om, const double* d_S1,
                         const double* d_S2, const double* d_S3,
                         const double* d_b, void* d_scratch, double* out,
                         void* stream);

/* Same result as pfc_op_residual_norm, but the caller passes no scratch and
 * nothing is allocated: the per-tile partial sums live in a fixed device
 * array inside the library (512 KiB, loaded with the library and kept by
 * every GPU that loads it until the process exits).  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * themselves, e.g. a host application whose device memory is reserved up
 * front by its own pool allocator, or a latency-critical loop that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * Limit: n^3 <= 256^3 cells; larger grids return PFC_ESIZE (with a message in
 * pfc_last_error) and must use pfc_op_residual_norm.
 * Every call looks up the array's device address with the caller's device
 * current (cudaGetSymbolAddress).  Every tile slot a call reads is rewritten
 * by that call, so no state carries over that needs clearing; all calls on a
 * device share the array, so calls that overlap on the GPU (concurrent
 * streams, threads) race and must be serialised by the caller.  The call is
 * blocking (it reads the sum back and synchronises `stream`), so it cannot be
 * made on a stream that is being captured.  Arguments are checked as in
 * pfc_op_residual_norm: n >= 2, h > 0, non-null pointers, else PFC_EINVAL. */
int pfc_op_residual_norm_static(int n, double h, double eps, double tau,
                                const double* d_phi, const double* d_mu,
                                const double* d_om, const double* d_S1,
                                const double* d_S2, const double* d_S3,
                                const double* d_b, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Ensembles: `members` independent runs (1 <= members <= 1024) of one grid
 * size n, box L, tau and solver settings (PFC_MIXED only), each with its own
 * eps and initial field, advanced together: every kernel of a step covers
 * all members, so the small grids of an ensemble share each launch and one
 * CUDA graph runs the step of the whole ensemble.  Every field holds the
 * members one after another (member m at offset m*n^3 of the n^3*members
 * doubles passed to pfc_batch_init, pfc_set_state and pfc_get_*).  pfc_step
 * ends a step when every member has converged (a converged member stays
 * converged while the others continue; its further corrections only lower
 * its residual) and returns PFC_ENOCONV or PFC_ENAN if any member fails;
 * stats then report the most corrections and the largest residuals.
 * pfc_energy, pfc_mass and pfc_diagnostics report member 0.
 * --------------------------------------------------------------------- */

/* Workspace bytes of an ensemble (0 if invalid: as pfc_workspace_bytes;
 * 1 <= members <= 1024 with 3 n members / 2 <= 65535, the launch grids'
 * z extent; members > 1 requires PFC_MIXED). */
size_t pfc_batch_workspace_bytes(const pfc_params* p, int members);

/* As pfc_init for `members` runs: eps[m] (host array) replaces p->eps for
 * member m; any_phi0 holds the members' initial fields one after another;
 * each member starts with phi^{-1} := phi^0. */
int pfc_batch_init(pfc_ctx** out, const pfc_params* p, int members, const double* eps,
                   void* d_workspace, size_t workspace_bytes, const double* any_phi0,
                   void* stream);

/* Members of the context (1 for pfc_init), or -1 for NULL. */
int pfc_batch_members(const pfc_ctx* c);

/* out[4m .. 4m+3] = pfc_diagnostics of member m (host array of 4*members). */
int pfc_batch_diagnostics(pfc_ctx* c, double* out);

/* Per member, of the last step: corrections, final and initial RMS
 * residuals (host arrays of `members`; any may be NULL). */
int pfc_batch_status(const pfc_ctx* c, int* iters, double* residual, double* residual0);

/* ------------------------------------------------------------------------
 * Groups of ensembles of different grid sizes.  The paper runs one grid at a
 * time and has no counterpart; this serves ensembles whose runs have uneven
 * grid sizes (and eps).  A group holds 1 .. PFC_MAX_GROUP contexts made by
 * pfc_init or pfc_batch_init (typically one ensemble per grid size) and
 * advances them together: one CUDA graph per time step forks into every
 * context's pre-loop work (source, initial iterate, first residual), then
 * one device-side WHILE loop runs, per iteration, the loop body (a V-cycle
 * or a defect correction with its residual) of every context that still has
 * a running member, side by side under one conditional (IF) node per
 * context, until every member of every context has converged or one has
 * failed.  A context whose members have all converged takes no further
 * loop body, so each context ends the step exactly (bit for bit) as when
 * stepped alone with pfc_step.  The group owns
 * no device memory (the contexts' workspaces hold all state; its loop
 * decision takes the contexts' state addresses as a kernel argument) and
 * does not own the contexts: destroy the group before them.  Contexts must
 * be on the current device; a context may belong to one group at a time.
 * --------------------------------------------------------------------- */
#define PFC_MAX_GROUP 16

typedef struct pfc_group pfc_group;

/* Make a group of `count` distinct contexts (host array ctxs) launching on
 * `stream` (cudaStream_t, may be NULL).  PFC_EINVAL for count outside
 * 1..PFC_MAX_GROUP, a NULL or repeated context. */
int pfc_group_init(pfc_group** out, pfc_ctx* const* ctxs, int count, void* stream);

/* Advance every context `nsteps` steps, one graph launch per step (the
 * step graphs are built on first use for each combination of the contexts'
 * ring positions).  Waits for work already enqueued on the contexts' own
 * streams first; blocking.  stats (may be NULL): host array of `count`
 * entries, as pfc_step's for each context.  If a context sets
 * pfc_use_graphs(c, 0) or kernel timing, the contexts are stepped one after
 * another instead (same results).  On PFC_ENOCONV or PFC_ENAN the step is
 * kept for the contexts that converged and repeated by none: the contexts
 * may then stand at different step indices (pfc_step_index). */
int pfc_group_step(pfc_group* g, int nsteps, pfc_step_stats* stats);

/* Graph launches made by pfc_group_step so far (one per group step). */
long long pfc_group_graph_launches(const pfc_group* g);

void pfc_group_destroy(pfc_group* g);

/* ------------------------------------------------------------------------
 * Discrete adjoint of one time step (gradients through the scheme).  Step k
 * solves F(u; b, c, eps) = N(u; b) - S(b, c) = 0 for u = (phi^{k+1}, mu,
 * omega) (Eqs. 5.4-5.10); given dL/dphi^{k+1} = d_gnext, the implicit
 * function theorem gives psi from J^T psi = (d_gnext, 0, 0), J = dF/du at
 * the solution, and
 *   d_gk    += -(dF/db)^T psi = psi1 + (df/db + (1-eps)/2) psi2 + 3 Lap psi2
 *              + Lap psi3 / 2,   df/db = (a^2 + 2ab + 3b^2)/4
 *   d_gkm1  += -(dF/dc)^T psi = -Lap psi2
 *   *eps_bar += -(dF/deps)^T psi = -sum psi2 (a + b) / 2
 * with a = phi^{k+1} (d_phi_next) and b = phi^k (d_phi_k).  d_gkm1 may equal
 * d_gk (the first step, phi^{-1} := phi^0).  Because J^T = S P J P S^-1 (P
 * swaps the phi and mu components, S = diag(1, 1, 2)), the transposed system
 * is solved as J z = (0, d_gnext, 0), psi = (z2, z1, 2 z3), by the context's
 * own FP64 defect correction around FP32 V-cycles with q = f'(a, b) +
 * (1-eps)/2, until the RMS residual is <= rtol times its initial value
 * (PFC_ENOCONV after max_cycles corrections).  Needs a PFC_MIXED context of
 * one member (its FP32 hierarchy and reduction scratch are used, its state
 * is not touched); d_z: 3 n^3 doubles of scratch.  Blocking; *cycles (may be
 * NULL) receives the corrections used. */
int pfc_adjoint_step(pfc_ctx* c, const double* d_phi_next, const double* d_phi_k,
                     const double* d_gnext, double* d_gk, double* d_gkm1, double* d_z,
                     double rtol, int max_cycles, double* eps_bar, int* cycles);

/* ------------------------------------------------------------------------
 * Primitive operations of the mixed-precision paths.  The outer loop is a
 * defect correction: r = S - N(u), then an FP32 multigrid solve of J d = r,
 * with J the Jacobian of N at u (Eqs. 5.4-5.6 differentiated in phi: only the
 * cubic term's coefficient q = f'(phi) + (1-eps)/2, f(a) = (a+b)(a^2+b^2)/4,
 * depends on u), then u += d.  PFC_MIXED keeps u, r, q and the energy/mass
 * sums in FP64; PFC_MIXED_DF keeps them in double-float.  The paper computes
 * in FP64 and has no mixed-precision form; this is a solver strategy whose
 * fixed point is the solution of N(u) = S up to the rounding of the outer
 * residual.
 *
 * A df field ("double-float") is 2*n^3 floats in natural cell order: cell c
 * holds hi at [2c] and lo at [2c+1], value hi + lo with |lo| <= ulp(hi)/2,
 * a 48-bit significand (unit roundoff 2^-48 ~ 3.6e-15).  PFC_MIXED_DF keeps
 * phi, mu, omega, S2 and S3 in this form because GB300 issues FP32 at about
 * 60 times its FP64 rate; pfc_get_* and pfc_set_state convert at the
 * boundary, so callers of the context API see FP64 fields only.
 *
 * Every FP32 field (float*, not df) below is stored colour-split: within each
 * x-row (j, k) the n/2 cells with (i+j+k) even come first, ordered by i/2,
 * then the n/2 cells with (i+j+k) odd; cell (i, j, k) is element
 * (k*n + j)*n + ((i+j+k) & 1)*(n/2) + i/2.  A red-black half-sweep then reads
 * and writes contiguous runs of one colour.  n must be even.
 * --------------------------------------------------------------------- */

/* FP64 residual r = S - N(u) rounded to FP32 into d_r1..3, the coefficient
 * q = f'(phi) + (1-eps)/2 formed in FP64 and rounded to FP32 into d_q, and
 * *out = RMS of the residual (its FP32-rounded components, summed in FP32
 * within a thread block; blocking).  d_lap (may be NULL) receives the
 * unscaled 7-point Laplacian of phi (neighbour sum - 6 centre) the residual
 * uses: the time step keeps it for the next steps' sources and diagnostics.
 * d_scratch: pfc_reduce_scratch_bytes(n) bytes.  n even. */
int pfc_op_defect(int n, double h, double eps, double tau, const double* d_phi,
                  const double* d_mu, const double* d_om, const double* d_S1,
                  const double* d_S2, const double* d_S3, const double* d_b,
                  float* d_r1, float* d_r2, float* d_r3, float* d_q,
                  void* d_scratch, double* out, double* d_lap, void* stream);

/* The start of a time step from u^{k+1} := 2 u^k - u^{k-1} in phi, mu and
 * omega (PFC_GUESS_EXTRAPOLATE_ALL on PFC_MIXED) in one pointwise pass.
 * Inputs: phi^k = d_b, phi^{k-1} = d_c, mu^k = d_mu0, omega^k = d_om0 and
 * the unscaled 7-point Laplacians (neighbour sum - 6 centre) d_lapb,
 * d_lapc, d_lapmu0, d_lapom0 of those four fields; d_mu1, d_om1 hold
 * mu^{k-1}, omega^{k-1} and d_lapmu1, d_lapom1 their Laplacians on entry,
 * and receive the iterate's mu, omega and Laplacians.  Outputs: S2, S3 of
 * Eqs. 5.9-5.10, the iterate phi = 2 phi^k - phi^{k-1} (d_phi) and its
 * Laplacian (d_lap), formed as 2 Lap u^k - Lap u^{k-1} (the Laplacian is
 * linear); the residual r = S - N(u) of the iterate (Eqs. 5.4-5.6, with
 * S1 = phi^k) rounded to FP32 into d_r1..3 and q as in pfc_op_defect
 * (colour-split); *out = RMS of r (blocking).  The combinations of phi^k,
 * phi^{k-1} and their Laplacians are exact in 64-bit fixed point (inputs
 * quantised to 2^-54, |v| < 32; larger values take FP64), those of mu and
 * omega FP64, so results differ from FP64 arithmetic by about 1e-16
 * absolute.  d_scratch: pfc_reduce_scratch_bytes(n) bytes.  Device
 * pointers, caller-owned, n^3 doubles (floats for r, q) each; n even;
 * PFC_EINVAL on a null pointer or a bad size. */
int pfc_op_start_extrap(int n, double h, double eps, double tau, const double* d_b,
                        const double* d_c, const double* d_lapb, const double* d_lapc,
                        const double* d_mu0, const double* d_om0, const double* d_lapmu0,
                        const double* d_lapom0, double* d_mu1, double* d_om1,
                        double* d_lapmu1, double* d_lapom1, double* d_S2, double* d_S3,
                        double* d_phi, double* d_lap, float* d_r1, float* d_r2,
                        float* d_r3, float* d_q, void* d_scratch, double* out,
                        void* stream);

/* u += d (FP64 += FP32) for the three components; d colour-split.  n even. */
int pfc_op_correct(int n, double* d_u1, double* d_u2, double* d_u3,
                   const float* d_d1, const float* d_d2, const float* d_d3,
                   void* stream);

/* The conversions of the FP64 outer loop, done on the integer pipe from the
 * IEEE 754 bit layouts (GB300 converts FP64<->FP32 only at its FP64 rate):
 * d_y[i] = d_x[i] rounded to FP32, to nearest with ties to even (overflow
 * to infinity, results below the normal range, zeros, infinities and NaNs as
 * the hardware conversion), and the exact widening of FP32 to FP64. */
int pfc_op_round_f32(long long count, const double* d_x, float* d_y, void* stream);
int pfc_op_widen_f64(long long count, const float* d_x, double* d_y, void* stream);

/* The PFC_GUESS_EXTRAPOLATE initial iterate from b = phi^k, c = phi^{k-1}:
 * S2, S3 of Eqs. 5.9-5.10 into d_S2, d_S3, and phi_g = 2b - c,
 * omega_g = (3 Lap b - Lap c)/2, mu_g = S2 + f(phi_g, b) + (1-eps)/2 phi_g
 * + Lap omega_g into d_phi, d_om, d_mu (two launches), all FP64. */
int pfc_op_guess(int n, double h, double eps, const double* d_b, const double* d_c,
                 double* d_S2, double* d_S3, double* d_phi, double* d_mu,
                 double* d_om, void* stream);

/* d_y = df(d_x) for `count` values: hi = FP32 rounding of x, lo = FP32
 * rounding of x - hi.  d_y may equal d_x (in-place conversion of 8-byte
 * slots); otherwise the arrays must not overlap. */
int pfc_op_df_from_f64(long long count, const double* d_x, float* d_y, void* stream);

/* d_x = hi + lo (exact in FP64) for `count` df values; in place allowed. */
int pfc_op_df_to_f64(long long count, const float* d_y, double* d_x, void* stream);

/* S2 and S3 of Eqs. 5.9-5.10 from df fields b = phi^k and c = phi^{k-1},
 * written as df fields, computed in double-float (pfc_op_source in FP64). */
int pfc_op_source_df(int n, double h, double eps, const float* d_b,
                     const float* d_c, float* d_S2, float* d_S3, void* stream);

/* pfc_op_guess on df fields (all arithmetic in double-float). */
int pfc_op_guess_df(int n, double h, double eps, const float* d_b, const float* d_c,
                    float* d_S2, float* d_S3, float* d_phi, float* d_mu,
                    float* d_om, void* stream);

/* Residual r = S - N(u) of the df fields (phi, mu, om), sources S1..S3 and
 * b, evaluated in double-float and rounded to FP32 into d_r1..3; the
 * coefficient q = f'(phi) + (1-eps)/2 in FP32 from the hi parts of phi and b
 * into d_q; *out = RMS of the residual (blocking); d_lap (may be NULL) the
 * unscaled Laplacian of phi as a df field.  d_scratch:
 * pfc_reduce_scratch_bytes(n) bytes.  n even. */
int pfc_op_defect_df(int n, double h, double eps, double tau, const float* d_phi,
                  const float* d_mu, const float* d_om, const float* d_S1,
                  const float* d_S2, const float* d_S3, const float* d_b,
                  float* d_r1, float* d_r2, float* d_r3, float* d_q,
                  void* d_scratch, double* out, float* d_lap, void* stream);

/* `sweeps` red-black Gauss-Seidel sweeps in FP32 on J d = r with q frozen
 * (the same pointwise 3x3 system as pfc_op_smooth with q given).  zero_init
 * != 0 declares d = 0 on entry (d need not be initialised).  n even. */
int pfc_op_lin_smooth(int n, double h, double eps, double tau, int sweeps,
                      int zero_init, float* d_d1, float* d_d2, float* d_d3,
                      const float* d_r1, const float* d_r2, const float* d_r3,
                      const float* d_q, void* stream);

/* `sweeps` damped collective Jacobi sweeps in FP32 on J d = r (q frozen),
 * scratch d_t1..3, result in d_d1..3; zero_init as for pfc_op_lin_smooth. */
int pfc_op_lin_jacobi(int n, double h, double eps, double tau, int sweeps,
                      double weight, int zero_init, float* d_d1, float* d_d2,
                      float* d_d3, float* d_t1, float* d_t2, float* d_t3,
                      const float* d_r1, const float* d_r2, const float* d_r3,
                      const float* d_q, void* stream);

/* Restricted residual of the linear system, rho_c = I (r - J d): the 8-cell
 * average of r - J d with (J d)1 = d_phi - tau Lap d_mu, (J d)2 = d_mu -
 * q d_phi - Lap d_om, (J d)3 = d_om - Lap d_phi / 2 (Eqs. 5.4-5.6
 * differentiated in phi), from the level of n^3 cells (n divisible by 4) to
 * the colour-split d_c1..3 of (n/2)^3.  zero_init != 0 declares d = 0 (d
 * and q are then not read and may be NULL). */
int pfc_op_lin_residual_restrict(int n, double h, double eps, double tau,
                                 int zero_init, const float* d_d1,
                                 const float* d_d2, const float* d_d3,
                                 const float* d_r1, const float* d_r2,
                                 const float* d_r3, const float* d_q,
                                 float* d_c1, float* d_c2, float* d_c3,
                                 void* stream);

/* The restriction of pfc_op_lin_residual_restrict to d_c1..3 ((n/2)^3)
 * followed, in the same launch, by `levels` - 1 (1 or 2) plain 8-cell
 * averages: d_e1..3 ((n/4)^3) = I c, and with levels = 3 d_g1..3 ((n/8)^3)
 * = I e, all colour-split.  This is the V-cycle's descent without
 * pre-smoothing, where every coarser level starts from d = 0; the results
 * equal those of the separate restrictions bit for bit.  n a multiple of
 * 32; d_g1..3 may be NULL when levels = 2; zero_init as for
 * pfc_op_lin_residual_restrict. */
int pfc_op_lin_restrict_chain(int n, double h, double eps, double tau, int zero_init,
                              int levels, const float* d_d1, const float* d_d2,
                              const float* d_d3, const float* d_r1, const float* d_r2,
                              const float* d_r3, const float* d_q, float* d_c1, float* d_c2,
                              float* d_c3, float* d_e1, float* d_e2, float* d_e3,
                              float* d_g1, float* d_g2, float* d_g3, void* stream);

/* The FP32 Newton coefficient q (colour-split, n^3) averaged over 8 children
 * (the coarse-level operators of the correction solve, Section 5 transfers
 * of the FAS reading) down `levels` (1..3) levels in one launch: d_c =
 * (n/2)^3, d_e = (n/4)^3, d_g = (n/8)^3, colour-split; each average sums the
 * children in the order (x, then y, then z fastest-first) of the single-level
 * restriction, so every level equals the separate restrictions bit for bit.
 * n a multiple of 32 for levels >= 2 (n even for levels = 1); d_e, d_g may be
 * NULL when not produced. */
int pfc_op_restrict_q(int n, int levels, const float* d_q, float* d_c, float* d_e,
                      float* d_g, void* stream);

/* d += P e, P the trilinear cell-centred prolongation (weights 27, 9, 3, 1
 * over 64) from the colour-split (n/2)^3 fields d_e1..3 to the colour-split
 * n^3 fields d_d1..3; n divisible by 4.  `assign` holds flags:
 * PFC_PROLONG_ASSIGN: d = P e (d not read); PFC_PROLONG_SKIP_COLOUR0: the
 * colour-0 cells (the first half of each colour-split row) are neither read
 * nor written, as inside the V-cycle when a red-black pass of colour 0
 * follows (it recomputes those cells without reading them).  Other bits:
 * PFC_EINVAL. */
#define PFC_PROLONG_ASSIGN        1
#define PFC_PROLONG_SKIP_COLOUR0  2
int pfc_op_lin_prolong(int n, int assign, const float* d_e1, const float* d_e2,
                       const float* d_e3, float* d_d1, float* d_d2, float* d_d3,
                       void* stream);

/* `sweeps` (>= 1) FP32 red-black sweeps on J d = r as pfc_op_lin_smooth
 * (d != 0 on entry) with the defect correction folded into the last
 * colour-1 pass: instead of storing its colour-1 values that pass adds them,
 * and the colour-0 values, to the FP64 state (natural layout): u += d, as
 * pfc_op_correct after pfc_op_lin_smooth, bit for bit.  d's colour-1 cells
 * keep the values of the sweep before.  n a multiple of 4, d_u1..3 16-byte
 * aligned (PFC_EINVAL otherwise). */
int pfc_op_lin_smooth_correct(int n, double h, double eps, double tau, int sweeps,
                              float* d_d1, float* d_d2, float* d_d3, const float* d_r1,
                              const float* d_r2, const float* d_r3, const float* d_q,
                              double* d_u1, double* d_u2, double* d_u3, void* stream);

/* The V-cycle's way up on one level: d (+)= P e, exactly as
 * pfc_op_lin_prolong (PFC_PROLONG_ASSIGN in `assign`: d = P e, d not read),
 * followed by one post-smoothing sweep of `kind` on J d = r (q frozen):
 * PFC_SWEEP_RB, one red-black sweep as pfc_op_lin_smooth with sweeps = 1;
 * PFC_SWEEP_JACOBI, one damped collective Jacobi sweep of `weight` as
 * pfc_op_lin_jacobi with sweeps = 1 (d_t1..3 scratch).  The prolongation is
 * fused into the first pass (the colour-0 pass, or the Jacobi sweep), which
 * forms d_old + P e in shared memory instead of memory; the result in
 * d_d1..3 equals the separate entry points bit for bit.  n a multiple of 32
 * (PFC_EINVAL otherwise); d_e1..3 colour-split of (n/2)^3 cells. */
int pfc_op_lin_prolong_smooth(int n, double h, double eps, double tau, int kind,
                              int assign, double weight, const float* d_e1,
                              const float* d_e2, const float* d_e3, float* d_d1,
                              float* d_d2, float* d_d3, float* d_t1, float* d_t2,
                              float* d_t3, const float* d_r1, const float* d_r2,
                              const float* d_r3, const float* d_q, void* stream);

/* u += d for the three components: df fields d_u1..3 plus the colour-split
 * FP32 corrections d_d1..3, in double-float.  n even. */
int pfc_op_correct_df(int n, float* d_u1, float* d_u2, float* d_u3,
                   const float* d_d1, const float* d_d2, const float* d_d3,
                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PFC_H */
