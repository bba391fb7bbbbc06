// FP64 kernels of one FAS V-cycle (Algorithm 1) for the split PFC system
// (Eqs. 5.4-5.10, M = 1) and the Section 2 diagnostics.
//
// Layout: every field is n^3 doubles, x fastest (cell (i,j,k) at i + n(j + nk)),
// one array per component (phi, mu, omega), so warps load contiguous x-runs.
#include "pfc_fixed.cuh"
#include "pfc_internal.h"

namespace pfc {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t work, int threads = kThreads) {
  return (unsigned)((work + threads - 1) / threads);
}

__device__ __forceinline__ void cell_of(int64_t t, int n, int& i, int& j, int& k) {
  i = (int)(t % n);
  const int64_t r = t / n;
  j = (int)(r % n);
  k = (int)(r / n);
}

// ---------------------------------------------------------------------------
// a1: source S2 = (1-eps)/2 b + 3 Lap b - Lap c, S3 = Lap b / 2 (Eqs. 5.9-5.10)
// ---------------------------------------------------------------------------
__global__ void k_source(Lvl L, const double* __restrict__ b, const double* __restrict__ c,
                         double* __restrict__ S2, double* __restrict__ S3) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  const double bb = __ldg(b + s.c);
  const double lb = L.g * fma(-6.0, bb, nbsum(b, s));
  const double lc = L.g * fma(-6.0, __ldg(c + s.c), nbsum(c, s));
  S2[s.c] = fma(3.0, lb, fma(L.c1, bb, -lc));
  S3[s.c] = 0.5 * lb;
}

// S2, S3 as k_source, plus the first part of the extrapolated initial
// iterate: phi_g = 2 b - c and omega_g = (3 Lap b - Lap c)/2 = Lap(phi_g + b)/2,
// which satisfies row 3 of N(u) = S (Eq. 5.6) for phi_g.
__global__ void k_source_guess(Lvl L, const double* __restrict__ b,
                               const double* __restrict__ c, double* __restrict__ S2,
                               double* __restrict__ S3, double* __restrict__ phig,
                               double* __restrict__ omg) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  const double bb = __ldg(b + s.c), cc = __ldg(c + s.c);
  const double lb = L.g * fma(-6.0, bb, nbsum(b, s));
  const double lc = L.g * fma(-6.0, cc, nbsum(c, s));
  S2[s.c] = fma(3.0, lb, fma(L.c1, bb, -lc));
  S3[s.c] = 0.5 * lb;
  phig[s.c] = fma(2.0, bb, -cc);
  omg[s.c] = 0.5 * fma(3.0, lb, -lc);
}

// Initial iterate of PFC_GUESS_EXTRAPOLATE_ALL: every unknown extrapolated
// linearly from the two last converged steps, phi = 2 b - c (b = phi^k,
// c = phi^{k-1}), mu = 2 mu^k - mu^{k-1}, omega = 2 omega^k - omega^{k-1}
// (extrap), or the last step's values (phi = b; mu, omega copied) while
// fewer than two converged steps are at hand.  mu^{k-1}, omega^{k-1} live in
// the slots that receive the new iterate (m1, o1, in place).
__global__ void k_guess_all(int64_t cells, int extrap, const double* __restrict__ b,
                            const double* __restrict__ c, const double* __restrict__ m0,
                            const double* __restrict__ o0, double* m1, double* o1,
                            double* __restrict__ phi) {
  pdl_wait();
  pdl_trigger();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double bb = __ldg(b + t), mm = __ldg(m0 + t), oo = __ldg(o0 + t);
    if (extrap) {
      phi[t] = fma(2.0, bb, -__ldg(c + t));
      m1[t] = fma(2.0, mm, -m1[t]);
      o1[t] = fma(2.0, oo, -o1[t]);
    } else {
      phi[t] = bb;
      m1[t] = mm;
      o1[t] = oo;
    }
  }
}

// mu_g = S2 + f(phi_g, b) + (1-eps)/2 phi_g + Lap omega_g: row 2 of
// N(u) = S (Eq. 5.5) solved for mu at the extrapolated phi_g, omega_g.
__global__ void k_mu_guess(Lvl L, const double* __restrict__ phig,
                           const double* __restrict__ omg, const double* __restrict__ b,
                           const double* __restrict__ S2, double* __restrict__ mug) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  const double p = __ldg(phig + s.c);
  const double lw = fma(-6.0, __ldg(omg + s.c), nbsum(omg, s));
  mug[s.c] = fma(L.g, lw, fma(L.c1, p, __ldg(S2 + s.c) + cubic_f(p, __ldg(b + s.c))));
}

// Unscaled 7-point Laplacian of a field (neighbour sum - 6 centre), the
// quantity the residual kernels store for later reuse.
__global__ void k_laplacian(int n, int members, const double* __restrict__ v,
                            double* __restrict__ lap) {
  const int64_t cells = (int64_t)n * n * n;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells * members) return;
  const int64_t off = (t / cells) * cells;     // member after member
  t -= off;
  v += off;
  lap += off;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  lap[t] = fma(-6.0, __ldg(v + s.c), nbsum(v, s));
}

// S2, S3 of Eqs. 5.9-5.10 from the stored unscaled Laplacians of b = phi^k
// and c = phi^{k-1}: the arithmetic of k_source without its two stencils.
// Ensembles: `members` fields one after another, member m with (1-eps)/2 at
// c1m[m] (c1m null: L.c1).
__global__ void k_source_cached(Lvl L, int members, const double* __restrict__ c1m,
                                const double* __restrict__ b,
                                const double* __restrict__ lapb, const double* __restrict__ lapc,
                                double* __restrict__ S2, double* __restrict__ S3) {
  pdl_wait();
  pdl_trigger();
  const int64_t cells = (int64_t)L.n * L.n * L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells * members) return;
  const double c1 = c1m ? c1m[t / cells] : L.c1;
  const double lb = L.g * __ldg(lapb + t);
  const double lc = L.g * __ldg(lapc + t);
  S2[t] = fma(3.0, lb, fma(c1, __ldg(b + t), -lc));
  S3[t] = 0.5 * lb;
}

// ---------------------------------------------------------------------------
// a2/a7: one colour of the red-black nonlinear Gauss-Seidel sweep (Section 5).
// Thread t owns the t-th cell of the colour: i = 2p + ((j+k+colour) & 1).
// Its six neighbours have the other colour and are not written here.
// ---------------------------------------------------------------------------
template <int LIN>
__global__ void k_smooth_colour(Lvl L, int colour, double* phi, double* mu, double* om,
                                const double* __restrict__ S1,
                                const double* __restrict__ S2,
                                const double* __restrict__ S3,
                                const double* __restrict__ b) {
  const int n = L.n, half = n >> 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)half * n * n) return;
  const int p = (int)(t % half);
  const int64_t r = t / half;
  const int j = (int)(r % n), k = (int)(r / n);
  const int i = 2 * p + ((j + k + colour) & 1);
  const Stencil s = stencil_at(i, j, k, n);
  double np, nm, nw;
  point_solve<LIN>(L, nbsum(phi, s), nbsum(mu, s), nbsum(om, s), phi[s.c], __ldg(b + s.c),
                   __ldg(S1 + s.c), __ldg(S2 + s.c), __ldg(S3 + s.c), np, nm, nw);
  phi[s.c] = np;
  mu[s.c] = nm;
  om[s.c] = nw;
}

// ---------------------------------------------------------------------------
// a2/a7 on levels of intermediate stiffness: one damped collective Jacobi
// sweep, (phi, mu, om) -> (tp, tm, tw).  Every cell solves the same pointwise
// system with the neighbours of the previous sweep and moves by w of the
// change.
// ---------------------------------------------------------------------------
template <int LIN>
__global__ void k_jacobi64(Lvl L, double w, const double* __restrict__ phi,
                           const double* __restrict__ mu, const double* __restrict__ om,
                           double* __restrict__ tp, double* __restrict__ tm,
                           double* __restrict__ tw, const double* __restrict__ S1,
                           const double* __restrict__ S2, const double* __restrict__ S3,
                           const double* __restrict__ b) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  const double p0 = __ldg(phi + s.c), m0 = __ldg(mu + s.c), w0 = __ldg(om + s.c);
  double np, nm, nw;
  point_solve<LIN>(L, nbsum(phi, s), nbsum(mu, s), nbsum(om, s), p0, __ldg(b + s.c),
                   __ldg(S1 + s.c), __ldg(S2 + s.c), __ldg(S3 + s.c), np, nm, nw);
  tp[s.c] = fma(w, np - p0, p0);
  tm[s.c] = fma(w, nm - m0, m0);
  tw[s.c] = fma(w, nw - w0, w0);
}

// ---------------------------------------------------------------------------
// a3: residual r = S - N(u), full fields (used by the primitive op)
// ---------------------------------------------------------------------------
__global__ void k_residual(Lvl L, const double* __restrict__ phi,
                           const double* __restrict__ mu, const double* __restrict__ om,
                           const double* __restrict__ S1, const double* __restrict__ S2,
                           const double* __restrict__ S3, const double* __restrict__ b,
                           double* __restrict__ r1, double* __restrict__ r2,
                           double* __restrict__ r3) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  double a, c, d;
  residual_at(L, s, phi, mu, om, S1, S2, S3, b, a, c, d);
  r1[s.c] = a;
  r2[s.c] = c;
  r3[s.c] = d;
}

// ---------------------------------------------------------------------------
// a3: fused residual + 8-cell restriction of r and u; one thread per coarse
// cell.  Optionally also stores the restricted u a second time (wc), which the
// correction step needs after the coarse level has overwritten uc.
// ---------------------------------------------------------------------------
__global__ void k_residual_restrict(Lvl L, const double* __restrict__ phi,
                                    const double* __restrict__ mu,
                                    const double* __restrict__ om,
                                    const double* __restrict__ S1,
                                    const double* __restrict__ S2,
                                    const double* __restrict__ S3,
                                    const double* __restrict__ b, double* __restrict__ rc1,
                                    double* __restrict__ rc2, double* __restrict__ rc3,
                                    double* __restrict__ uc1, double* __restrict__ uc2,
                                    double* __restrict__ uc3, double* __restrict__ wc1,
                                    double* __restrict__ wc2, double* __restrict__ wc3) {
  const int n = L.n, nc = n >> 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nc * nc * nc) return;
  int I, J, K;
  cell_of(t, nc, I, J, K);
  double a1 = 0, a2 = 0, a3 = 0, v1 = 0, v2 = 0, v3 = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    const Stencil s = stencil_at(i, j, k, n);
    double x, y, z;
    residual_at(L, s, phi, mu, om, S1, S2, S3, b, x, y, z);
    a1 += x;
    a2 += y;
    a3 += z;
    v1 += __ldg(phi + s.c);
    v2 += __ldg(mu + s.c);
    v3 += __ldg(om + s.c);
  }
  rc1[t] = 0.125 * a1;
  rc2[t] = 0.125 * a2;
  rc3[t] = 0.125 * a3;
  uc1[t] = 0.125 * v1;
  uc2[t] = 0.125 * v2;
  uc3[t] = 0.125 * v3;
  if (wc1) {
    wc1[t] = 0.125 * v1;
    wc2[t] = 0.125 * v2;
    wc3[t] = 0.125 * v3;
  }
}

__global__ void k_restrict(int n, const double* __restrict__ f, double* __restrict__ c) {
  const int nc = n >> 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nc * nc * nc) return;
  int I, J, K;
  cell_of(t, nc, I, J, K);
  double acc = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
    acc += __ldg(f + i + n * (j + (int64_t)n * k));
  }
  c[t] = 0.125 * acc;
}

// ---------------------------------------------------------------------------
// a4: FAS coarse source S_c = N_c(u_c) + r_c, in place over r_c
// ---------------------------------------------------------------------------
__global__ void k_coarse_source(Lvl L, const double* __restrict__ u1,
                                const double* __restrict__ u2,
                                const double* __restrict__ u3,
                                const double* __restrict__ bc, double* r1, double* r2,
                                double* r3) {
  const int n = L.n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const Stencil s = stencil_at(i, j, k, n);
  double x, y, z;
  operator_at(L, s, u1, u2, u3, bc, x, y, z);
  r1[s.c] += x;
  r2[s.c] += y;
  r3[s.c] += z;
}

__global__ void k_coarse_diff(int64_t cells, const double* __restrict__ v1,
                              const double* __restrict__ v2,
                              const double* __restrict__ v3, double* w1, double* w2,
                              double* w3) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  w1[t] = v1[t] - w1[t];
  w2[t] = v2[t] - w2[t];
  w3[t] = v3[t] - w3[t];
}

// ---------------------------------------------------------------------------
// a6: u += P e, P trilinear cell-centred: fine cell 2I+a takes 3/4 of coarse I
// and 1/4 of coarse I+(a ? 1 : -1) per axis, i.e. weights 27, 9, 3, 1 (/64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double interp8(const double* __restrict__ e, int64_t o000,
                                          int64_t o100, int64_t o010, int64_t o001,
                                          int64_t o110, int64_t o101, int64_t o011,
                                          int64_t o111) {
  const double g2 = (__ldg(e + o100) + __ldg(e + o010)) + __ldg(e + o001);
  const double g3 = (__ldg(e + o110) + __ldg(e + o101)) + __ldg(e + o011);
  double acc = fma(3.0, g3, __ldg(e + o111));
  acc = fma(9.0, g2, acc);
  acc = fma(27.0, __ldg(e + o000), acc);
  return acc;
}

__global__ void k_prolong_add(int n, const double* __restrict__ e1,
                              const double* __restrict__ e2,
                              const double* __restrict__ e3, double* __restrict__ u1,
                              double* __restrict__ u2, double* __restrict__ u3) {
  const int nc = n >> 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n * n) return;
  int i, j, k;
  cell_of(t, n, i, j, k);
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  int I2 = (i & 1) ? I + 1 : I - 1;
  int J2 = (j & 1) ? J + 1 : J - 1;
  int K2 = (k & 1) ? K + 1 : K - 1;
  I2 = (I2 + nc) % nc;
  J2 = (J2 + nc) % nc;
  K2 = (K2 + nc) % nc;
  const int64_t nn = (int64_t)nc * nc;
  const int64_t zK = K * nn, zK2 = K2 * nn, yJ = (int64_t)J * nc, yJ2 = (int64_t)J2 * nc;
  const int64_t o000 = I + yJ + zK, o100 = I2 + yJ + zK, o010 = I + yJ2 + zK,
                o001 = I + yJ + zK2, o110 = I2 + yJ2 + zK, o101 = I2 + yJ + zK2,
                o011 = I + yJ2 + zK2, o111 = I2 + yJ2 + zK2;
  const double w = 1.0 / 64.0;
  u1[t] = fma(w, interp8(e1, o000, o100, o010, o001, o110, o101, o011, o111), u1[t]);
  u2[t] = fma(w, interp8(e2, o000, o100, o010, o001, o110, o101, o011, o111), u2[t]);
  u3[t] = fma(w, interp8(e3, o000, o100, o010, o001, o110, o101, o011, o111), u3[t]);
}

// ---------------------------------------------------------------------------
// a5: coarsest level: sweeps in one thread block until the largest relative
// change falls below 1e-14 or max_sweeps.  Red-black (kind 0) updates in
// place; damped Jacobi (kind 1) computes every cell into t and copies back.
// Neighbours are read with coherent loads because this block wrote them in
// the previous half-sweep.
// ---------------------------------------------------------------------------
template <int LIN>
__global__ void k_coarse_solve(Lvl L, int kind, double w, int max_sweeps, double* phi,
                               double* mu, double* om, double* t1, double* t2, double* t3,
                               const double* S1, const double* S2, const double* S3,
                               const double* b) {
  __shared__ double red[32];
  __shared__ int done;
  const int n = L.n, half = n >> 1;
  const int ncell = n * n * n;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double change = 0.0;
    if (kind == PFC_SWEEP_JACOBI) {
      for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, k = t / (n * n);
        const Stencil s = stencil_at(i, j, k, n);
        const double p0 = phi[s.c], m0 = mu[s.c], w0 = om[s.c];
        double np, nm, nw;
        point_solve<LIN>(L, nbsum_coherent(phi, s), nbsum_coherent(mu, s),
                         nbsum_coherent(om, s), p0, b[s.c], S1[s.c], S2[s.c], S3[s.c], np,
                         nm, nw);
        t1[s.c] = fma(w, np - p0, p0);
        t2[s.c] = fma(w, nm - m0, m0);
        t3[s.c] = fma(w, nw - w0, w0);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        change = fmax(change, fabs(t1[t] - phi[t]) / (1.0 + fabs(t1[t])));
        change = fmax(change, fabs(t2[t] - mu[t]) / (1.0 + fabs(t2[t])));
        change = fmax(change, fabs(t3[t] - om[t]) / (1.0 + fabs(t3[t])));
        phi[t] = t1[t];
        mu[t] = t2[t];
        om[t] = t3[t];
      }
      __syncthreads();
    } else {
      const int cells = half * n * n;
      for (int colour = 0; colour < 2; ++colour) {
        for (int t = threadIdx.x; t < cells; t += blockDim.x) {
          const int p = t % half, r = t / half;
          const int j = r % n, k = r / n;
          const int i = 2 * p + ((j + k + colour) & 1);
          const Stencil s = stencil_at(i, j, k, n);
          const double op = phi[s.c], om_ = mu[s.c], ow = om[s.c];
          double np, nm, nw;
          point_solve<LIN>(L, nbsum_coherent(phi, s), nbsum_coherent(mu, s),
                           nbsum_coherent(om, s), op, b[s.c], S1[s.c], S2[s.c], S3[s.c],
                           np, nm, nw);
          phi[s.c] = np;
          mu[s.c] = nm;
          om[s.c] = nw;
          change = fmax(change, fabs(np - op) / (1.0 + fabs(np)));
          change = fmax(change, fabs(nm - om_) / (1.0 + fabs(nm)));
          change = fmax(change, fabs(nw - ow) / (1.0 + fabs(nw)));
        }
        __syncthreads();
      }
    }
    // block max of the change
    for (int o = 16; o > 0; o >>= 1) change = fmax(change, __shfl_down_sync(0xffffffffu, change, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = change;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int q = 0; q < (int)((blockDim.x + 31) >> 5); ++q) m = fmax(m, red[q]);
      done = (m < 1e-14);
    }
    __syncthreads();
    if (done) break;
  }
}

// ---------------------------------------------------------------------------
// Reductions (deterministic: fixed grid, fixed per-thread order, fixed tree)
// ---------------------------------------------------------------------------
__global__ void k_residual_norm2(Lvl L, const double* __restrict__ phi,
                                 const double* __restrict__ mu,
                                 const double* __restrict__ om,
                                 const double* __restrict__ S1,
                                 const double* __restrict__ S2,
                                 const double* __restrict__ S3,
                                 const double* __restrict__ b, double* partials,
                                 double* __restrict__ lap) {
  __shared__ double sm[32];
  const int n = L.n;
  const int64_t cells = (int64_t)n * n * n;
  double acc[1] = {0.0};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(t, n, i, j, k);
    const Stencil s = stencil_at(i, j, k, n);
    double x, y, z, lp;
    residual_at(L, s, phi, mu, om, S1, S2, S3, b, x, y, z, lp);
    acc[0] = fma(x, x, fma(y, y, fma(z, z, acc[0])));
    if (lap) lap[t] = lp;
  }
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// Fixed-order sum of NV-component block partials; one block per ensemble
// member, member m's sums at out[m * kReduceComps + c].
template <int NV>
__global__ void k_reduce_final(const double* __restrict__ partials, int nparts,
                               double* out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[32 * NV];
  partials += (size_t)blockIdx.x * nparts * NV;
  out += (size_t)blockIdx.x * kReduceComps;
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] += partials[(int64_t)p * NV + c];
  }
  block_sum<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) out[c] = acc[c];
  }
}

// Raw per-cell sums for F_h (Eq. 2.1), the modified energy and the mass.
// ||grad_h a||^2 is taken as -(a, Delta_h a) (summation by parts, Lemma 2.1),
// reusing the Laplacian that ||Delta_h a||^2 needs.
__global__ void k_diagnostics(int n, const double* __restrict__ a,
                              const double* __restrict__ b, double* partials) {
  __shared__ double sm[32 * 6];
  const int cells = n * n * n;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Stencil s = stencil_at(i, j, k, n);
    const double x = __ldg(a + s.c);
    const double lap = fma(-6.0, x, nbsum(a, s));
    const double y = x - __ldg(b + s.c);
    const double ex = (__ldg(a + s.xp) - __ldg(b + s.xp)) - y;
    const double ey = (__ldg(a + s.yp) - __ldg(b + s.yp)) - y;
    const double ez = (__ldg(a + s.zp) - __ldg(b + s.zp)) - y;
    const double x2 = x * x;
    acc[0] = fma(x2, x2, acc[0]);
    acc[1] += x2;
    acc[2] = fma(-x, lap, acc[2]);
    acc[3] = fma(lap, lap, acc[3]);
    acc[4] = fma(ex, ex, fma(ey, ey, fma(ez, ez, acc[4])));
    acc[5] += x;
  }
  block_sum<6>(acc, sm);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 6; ++c) partials[(int64_t)blockIdx.x * 6 + c] = acc[c];
  }
}

// The raw sums of k_diagnostics from the stored unscaled Laplacians of a and
// b: -(a, Lap a) and (Lap a)^2 directly, and the forward-face sum of
// |D(a-b)|^2 by summation by parts as -(a-b, Lap a - Lap b) (Lemma 2.1).
// The kernel is bound by GB300's FP64 pipe, so the two plain sums, sum a^2
// and sum a, run on the integer pipe: each value of magnitude below 1 enters
// as its fixed-point image (2^-54 quantum, pfc_fixed.cuh) into an exact int64
// sum, which is rounded to FP64 and added every 256 cells (at most 2^8 values
// below 2^54 each: no overflow); larger values take the FP64 adds.  The two
// differences a - b and Lap a - Lap b are formed from the same images (exact,
// one rounding each), which leaves 5 FP64 operations per cell.
__global__ void k_diagnostics_cached(int n, const double* __restrict__ a,
                                     const double* __restrict__ b,
                                     const double* __restrict__ lapa,
                                     const double* __restrict__ lapb, double* partials) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[32 * 6];
  const int cells = n * n * n;
  const size_t off = (size_t)blockIdx.y * cells;     // member of an ensemble
  a += off, b += off, lapa += off, lapb += off;
  partials += (size_t)blockIdx.y * gridDim.x * 6;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int64_t s1 = 0, s2 = 0;       // fixed-point sums of a and a^2 since the last flush
  int count = 0;
  auto cell = [&](double x, double la, double vb, double lb) {
    const double x2 = x * x;
    acc[0] = fma(x2, x2, acc[0]);
    acc[2] = fma(-x, la, acc[2]);
    acc[3] = fma(la, la, acc[3]);
    bool ok = ((fix_bits_of(x) >> 52) & 0x7FFu) <= 1022u;   // |x| < 1, so x^2 < 1
    const int64_t X = fix_of(x, ok), B = fix_of(vb, ok);
    const int64_t LA = fix_of(la, ok), LB = fix_of(lb, ok);
    if (ok) {
      // a - b and Lap a - Lap b exact in fixed point, each rounded once
      acc[4] = fma(-fix_to_double(X - B), fix_to_double(LA - LB), acc[4]);
      s1 += X;
      s2 += fix_of(x2, ok);
    } else {
      acc[4] = fma(-(x - vb), la - lb, acc[4]);
      acc[5] += x;
      acc[1] += x2;
    }
    if (++count == 256) {
      acc[5] += fix_to_double(s1);
      acc[1] += fix_to_double(s2);
      s1 = s2 = 0;
      count = 0;
    }
  };
  // four cells a thread in flight: their 16 loads are issued before the
  // arithmetic of the first (the kernel is latency bound with one)
  const int stride = gridDim.x * blockDim.x;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (; t + 3 * stride < cells; t += 4 * stride) {
    double x[4], la[4], vb[4], lb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[u] = __ldg(a + t + u * stride);
      la[u] = __ldg(lapa + t + u * stride);
      vb[u] = __ldg(b + t + u * stride);
      lb[u] = __ldg(lapb + t + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) cell(x[u], la[u], vb[u], lb[u]);
  }
  for (; t < cells; t += stride) cell(__ldg(a + t), __ldg(lapa + t), __ldg(b + t), __ldg(lapb + t));
  acc[5] += fix_to_double(s1);
  acc[1] += fix_to_double(s2);
  block_sum<6>(acc, sm);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 6; ++c) partials[(int64_t)blockIdx.x * 6 + c] = acc[c];
  }
}

// Convergence test of Algorithm 1's loop (RMS residual against the tolerance,
// NaN, cycle budget) on the device.
__global__ void k_decide(cudaGraphConditionalHandle handle, int use_handle,
                         const double* sum, StepState* s, int members, double inv_3n3,
                         double tol, int max_iter, int first) {
  pdl_wait();
  pdl_trigger();
  // one thread per ensemble member (sum[m] its sum of squared residuals);
  // a member that has converged stays converged, and the loop runs while
  // some member is still running and none has failed
  const int m = threadIdx.x;
  int running = 0, failed = 0;
  if (m < members)
    decide_member(s[m], sum[m], inv_3n3, tol, max_iter, first, running, failed);
  running = __syncthreads_or(running);
  failed = __syncthreads_or(failed);
  if (use_handle && threadIdx.x == 0)
    cudaGraphSetConditional(handle, (running && !failed) ? 1u : 0u);
}

// The loop condition of a group of contexts: every member of every context
// (states written by the contexts' own k_decide) is read once.
__global__ void k_group_decide(cudaGraphConditionalHandle handle, GroupStates g) {
  int running = 0, failed = 0;
  for (int c = 0; c < g.count; ++c)
    for (int m = threadIdx.x; m < g.members[c]; m += blockDim.x) {
      const int status = g.s[c][m].status;
      running |= status == kStepRunning;
      failed |= status == kStepNaN || status == kStepNoConv;
    }
  running = __syncthreads_or(running);
  failed = __syncthreads_or(failed);
  if (threadIdx.x == 0) cudaGraphSetConditional(handle, (running && !failed) ? 1u : 0u);
}

// The loop body of each context of a group runs only while that context
// has a running member: one warp per context sets its IF condition.
__global__ void k_group_select(GroupHandles hs, GroupStates g) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= g.count) return;
  int running = 0;
  for (int m = lane; m < g.members[c]; m += 32) running |= g.s[c][m].status == kStepRunning;
  running = __any_sync(0xffffffffu, running);
  if (lane == 0) cudaGraphSetConditional(hs.h[c], running ? 1u : 0u);
}

inline int reduce_blocks(int64_t cells) {
  const int64_t nb = (cells + kReduceThreads - 1) / kReduceThreads;
  return (int)(nb < kReduceBlocks ? nb : kReduceBlocks);
}

}  // namespace

cudaError_t launch_guess_all(int64_t cells, bool extrap, const double* b, const double* c,
                             const double* m0, const double* o0, double* m1, double* o1,
                             double* phi, cudaStream_t st, bool pdl) {
  return launch_ex(pdl, k_guess_all, dim3(grid_for(cells)), dim3(kThreads), 0, st, cells,
                   extrap ? 1 : 0, b, c, m0, o0, m1, o1, phi);
}

cudaError_t launch_guess(const Lvl& L, const double* b, const double* c, double* S2,
                         double* S3, double* phig, double* mug, double* omg, cudaStream_t st) {
  const int64_t cells = (int64_t)L.n * L.n * L.n;
  k_source_guess<<<grid_for(cells), kThreads, 0, st>>>(L, b, c, S2, S3, phig, omg);
  k_mu_guess<<<grid_for(cells), kThreads, 0, st>>>(L, phig, omg, b, S2, mug);
  return cudaGetLastError();
}

cudaError_t launch_laplacian(int n, const double* v, double* lap, cudaStream_t st,
                             int members) {
  k_laplacian<<<grid_for((int64_t)n * n * n * members), kThreads, 0, st>>>(n, members, v, lap);
  return cudaGetLastError();
}

cudaError_t launch_source_cached(const Lvl& L, const double* b, const double* lapb,
                                 const double* lapc, double* S2, double* S3, cudaStream_t st,
                                 int members, const double* c1m, bool pdl) {
  return launch_ex(pdl, k_source_cached, dim3(grid_for((int64_t)L.n * L.n * L.n * members)),
                   dim3(kThreads), 0, st, L, members, c1m, b, lapb, lapc, S2, S3);
}

// k_reduce_final<6> that also copies each member's step state (the step's
// end inside a step graph: out and state_out may be mapped host memory, so
// the graph needs no copy nodes).
__global__ void k_reduce_final_state(const double* __restrict__ partials, int nparts,
                                     double* out, const StepState* __restrict__ state,
                                     StepState* state_out) {
  pdl_wait();
  pdl_trigger();
  constexpr int NV = 6;
  __shared__ double sm[32 * NV];
  partials += (size_t)blockIdx.x * nparts * NV;
  out += (size_t)blockIdx.x * kReduceComps;
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] += partials[(int64_t)p * NV + c];
  }
  block_sum<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) out[c] = acc[c];
    state_out[blockIdx.x] = state[blockIdx.x];
  }
}

// Blocks of k_diagnostics_cached over all members: two per SM.  Its six
// FP64 block sums cost 5 lanes of FP64 adds per thread in the warp
// shuffles, as much as its per-cell work when a thread has only 7 cells
// (1216 blocks at 128^3), so each thread takes about 27.
constexpr int kDiagBlocks = 2 * 152;

cudaError_t launch_diagnostics_cached(int n, const double* a, const double* b,
                                      const double* lapa, const double* lapb, double* partials,
                                      double* out, cudaStream_t st, int members, bool pdl,
                                      const StepState* state, StepState* state_out) {
  const int64_t cells = (int64_t)n * n * n;
  int nb = kDiagBlocks / members;
  if (nb > (cells + kReduceThreads - 1) / kReduceThreads)
    nb = (int)((cells + kReduceThreads - 1) / kReduceThreads);
  if (nb < 1) nb = 1;
  cudaError_t e = launch_ex(pdl, k_diagnostics_cached, dim3(nb, members), dim3(kReduceThreads), 0,
                            st, n, a, b, lapa, lapb, partials);
  if (e == cudaSuccess && state_out)
    e = launch_ex(pdl, k_reduce_final_state, dim3(members), dim3(kReduceThreads), 0, st,
                  (const double*)partials, nb, out, state, state_out);
  else if (e == cudaSuccess)
    e = launch_ex(pdl, k_reduce_final<6>, dim3(members), dim3(kReduceThreads), 0, st,
                  (const double*)partials, nb, out);
  return e;
}

cudaError_t launch_source(const Lvl& L, const double* b, const double* c, double* S2,
                          double* S3, cudaStream_t st) {
  const int64_t cells = (int64_t)L.n * L.n * L.n;
  k_source<<<grid_for(cells), kThreads, 0, st>>>(L, b, c, S2, S3);
  return cudaGetLastError();
}

cudaError_t launch_smooth(const Lvl& L, int lin, int sweeps, double* phi, double* mu,
                          double* om, const double* S1, const double* S2,
                          const double* S3, const double* b, cudaStream_t st) {
  const int64_t work = (int64_t)(L.n / 2) * L.n * L.n;
  for (int s = 0; s < sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      if (lin == PFC_NEWTON)
        k_smooth_colour<PFC_NEWTON><<<grid_for(work), kThreads, 0, st>>>(
            L, colour, phi, mu, om, S1, S2, S3, b);
      else
        k_smooth_colour<PFC_PICARD><<<grid_for(work), kThreads, 0, st>>>(
            L, colour, phi, mu, om, S1, S2, S3, b);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const Lvl& L, int lin, int sweeps, double w, double* phi,
                          double* mu, double* om, double* t1, double* t2, double* t3,
                          const double* S1, const double* S2, const double* S3,
                          const double* b, cudaStream_t st) {
  const int64_t cells = (int64_t)L.n * L.n * L.n;
  double* src[3] = {phi, mu, om};
  double* dst[3] = {t1, t2, t3};
  for (int s = 0; s < sweeps; ++s) {
    if (lin == PFC_NEWTON)
      k_jacobi64<PFC_NEWTON><<<grid_for(cells), kThreads, 0, st>>>(
          L, w, src[0], src[1], src[2], dst[0], dst[1], dst[2], S1, S2, S3, b);
    else
      k_jacobi64<PFC_PICARD><<<grid_for(cells), kThreads, 0, st>>>(
          L, w, src[0], src[1], src[2], dst[0], dst[1], dst[2], S1, S2, S3, b);
    for (int q = 0; q < 3; ++q) {
      double* x = src[q];
      src[q] = dst[q];
      dst[q] = x;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && (sweeps & 1)) {
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
      e = cudaMemcpyAsync(q == 0 ? phi : q == 1 ? mu : om, src[q], cells * sizeof(double),
                          cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

cudaError_t launch_residual(const Lvl& L, const double* phi, const double* mu,
                            const double* om, const double* S1, const double* S2,
                            const double* S3, const double* b, double* r1, double* r2,
                            double* r3, cudaStream_t st) {
  const int64_t cells = (int64_t)L.n * L.n * L.n;
  k_residual<<<grid_for(cells), kThreads, 0, st>>>(L, phi, mu, om, S1, S2, S3, b, r1, r2,
                                                  r3);
  return cudaGetLastError();
}

cudaError_t launch_residual_restrict(const Lvl& L, const double* phi, const double* mu,
                                     const double* om, const double* S1,
                                     const double* S2, const double* S3, const double* b,
                                     double* rc1, double* rc2, double* rc3, double* uc1,
                                     double* uc2, double* uc3, double* wc1, double* wc2,
                                     double* wc3, cudaStream_t st) {
  const int nc = L.n / 2;
  const int64_t work = (int64_t)nc * nc * nc;
  k_residual_restrict<<<grid_for(work), kThreads, 0, st>>>(
      L, phi, mu, om, S1, S2, S3, b, rc1, rc2, rc3, uc1, uc2, uc3, wc1, wc2, wc3);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int n, const double* fine, double* coarse, cudaStream_t st) {
  const int nc = n / 2;
  const int64_t work = (int64_t)nc * nc * nc;
  k_restrict<<<grid_for(work), kThreads, 0, st>>>(n, fine, coarse);
  return cudaGetLastError();
}

cudaError_t launch_coarse_source(const Lvl& Lc, const double* uc1, const double* uc2,
                                 const double* uc3, const double* bc, double* r1,
                                 double* r2, double* r3, cudaStream_t st) {
  const int64_t cells = (int64_t)Lc.n * Lc.n * Lc.n;
  k_coarse_source<<<grid_for(cells), kThreads, 0, st>>>(Lc, uc1, uc2, uc3, bc, r1, r2, r3);
  return cudaGetLastError();
}

cudaError_t launch_coarse_diff(int nc, const double* v1, const double* v2,
                               const double* v3, double* w1, double* w2, double* w3,
                               cudaStream_t st) {
  const int64_t cells = (int64_t)nc * nc * nc;
  k_coarse_diff<<<grid_for(cells), kThreads, 0, st>>>(cells, v1, v2, v3, w1, w2, w3);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(int n, const double* e1, const double* e2,
                               const double* e3, double* u1, double* u2, double* u3,
                               cudaStream_t st) {
  const int64_t cells = (int64_t)n * n * n;
  k_prolong_add<<<grid_for(cells), kThreads, 0, st>>>(n, e1, e2, e3, u1, u2, u3);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const Lvl& L, int lin, int kind, double w, int max_sweeps,
                                double* phi, double* mu, double* om, double* t1, double* t2,
                                double* t3, const double* S1, const double* S2,
                                const double* S3, const double* b, cudaStream_t st) {
  const int work = L.n * L.n * L.n;
  int threads = ((work + 31) / 32) * 32;
  if (threads > 1024) threads = 1024;
  if (lin == PFC_NEWTON)
    k_coarse_solve<PFC_NEWTON><<<1, threads, 0, st>>>(L, kind, w, max_sweeps, phi, mu, om,
                                                       t1, t2, t3, S1, S2, S3, b);
  else
    k_coarse_solve<PFC_PICARD><<<1, threads, 0, st>>>(L, kind, w, max_sweeps, phi, mu, om,
                                                       t1, t2, t3, S1, S2, S3, b);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm2(const Lvl& L, const double* phi, const double* mu,
                                  const double* om, const double* S1, const double* S2,
                                  const double* S3, const double* b, double* partials,
                                  double* out, cudaStream_t st, double* lap) {
  const int nb = reduce_blocks((int64_t)L.n * L.n * L.n);
  k_residual_norm2<<<nb, kReduceThreads, 0, st>>>(L, phi, mu, om, S1, S2, S3, b, partials,
                                                  lap);
  k_reduce_final<1><<<1, kReduceThreads, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_decide(cudaGraphConditionalHandle handle, int use_handle,
                          const double* sum, StepState* state, double inv_3n3, double tol,
                          int max_iter, int first, cudaStream_t st, int members, bool pdl) {
  const int threads = ((members + 31) / 32) * 32;
  return launch_ex(pdl, k_decide, dim3(1), dim3(threads), 0, st, handle, use_handle, sum, state,
                   members, inv_3n3, tol, max_iter, first);
}

cudaError_t launch_group_select(const GroupHandles& hs, const GroupStates& g,
                                cudaStream_t st) {
  k_group_select<<<1, 32 * kMaxGroup, 0, st>>>(hs, g);
  return cudaGetLastError();
}

cudaError_t launch_group_decide(cudaGraphConditionalHandle handle, const GroupStates& g,
                                cudaStream_t st) {
  k_group_decide<<<1, 256, 0, st>>>(handle, g);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(int n, const double* a, const double* b, double* partials,
                               double* out, cudaStream_t st) {
  const int nb = reduce_blocks((int64_t)n * n * n);
  k_diagnostics<<<nb, kReduceThreads, 0, st>>>(n, a, b, partials);
  k_reduce_final<6><<<1, kReduceThreads, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

}  // namespace pfc
