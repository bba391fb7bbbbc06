// Device-side building blocks of the PFC multigrid kernels: level constants,
// periodic 7-point stencil addressing, the pointwise 3x3 solve of the
// red-black smoother (Section 5) and the residual r = S - N(u) of Eqs. 5.4-5.10.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pfc.h"

namespace pfc {

// Constants of one multigrid level (spacing h, shared eps and tau).
struct Lvl {
  int n;        // cells per side
  double g;     // 1/h^2
  double tg;    // tau/h^2
  double kap;   // 6 tau/h^2   (tau/h^2 times the six unit face mobilities)
  double g6;    // 6/h^2
  double g3;    // 3/h^2
  double gh;    // 1/(2 h^2)
  double Q0;    // 18/h^4      (the 6/h^2 * 3/h^2 coupling of rows 2 and 3)
  double c1;    // (1 - eps)/2
};

inline Lvl make_lvl(int n, double h, double eps, double tau) {
  Lvl L;
  double g = 1.0 / (h * h);
  L.n = n;
  L.g = g;
  L.tg = tau * g;
  L.kap = 6.0 * tau * g;
  L.g6 = 6.0 * g;
  L.g3 = 3.0 * g;
  L.gh = 0.5 * g;
  L.Q0 = 18.0 * g * g;
  L.c1 = 0.5 * (1.0 - eps);
  return L;
}

// Linear indices of a cell and its six periodic face neighbours.
struct Stencil {
  int64_t c, xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Stencil stencil_at(int i, int j, int k, int n) {
  const int im = (i == 0) ? n - 1 : i - 1, ip = (i + 1 == n) ? 0 : i + 1;
  const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
  const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
  const int64_t nn = (int64_t)n * n;
  const int64_t row = (int64_t)j * n + (int64_t)k * nn;
  Stencil s;
  s.c = row + i;
  s.xm = row + im;
  s.xp = row + ip;
  s.ym = (int64_t)jm * n + (int64_t)k * nn + i;
  s.yp = (int64_t)jp * n + (int64_t)k * nn + i;
  s.zm = (int64_t)j * n + (int64_t)km * nn + i;
  s.zp = (int64_t)j * n + (int64_t)kp * nn + i;
  return s;
}

template <class T>
__device__ __forceinline__ T nbsum(const T* __restrict__ v, const Stencil& s) {
  return ((__ldg(v + s.xm) + __ldg(v + s.xp)) + (__ldg(v + s.ym) + __ldg(v + s.yp))) +
         (__ldg(v + s.zm) + __ldg(v + s.zp));
}

// Neighbour sum through plain (coherent) loads, for arrays written earlier in
// the same kernel by other threads of the block.
template <class T>
__device__ __forceinline__ T nbsum_coherent(const T* v, const Stencil& s) {
  return ((v[s.xm] + v[s.xp]) + (v[s.ym] + v[s.yp])) + (v[s.zm] + v[s.zp]);
}

// Cubic term f(a) = (a+b)(a^2+b^2)/4 of Eq. 5.2 and its derivative in a.
__device__ __forceinline__ double cubic_f(double a, double b) {
  return 0.25 * (a + b) * fma(a, a, b * b);
}
__device__ __forceinline__ double cubic_fp(double a, double b) {
  return fma(0.75 * a, a, fma(0.5 * a, b, 0.25 * b * b));
}

// Pointwise solve of the smoother's 3x3 system (Section 5)
//   [ 1      kap   0   ] [phi]   [st1 = S1 + tau/h^2 sum mu_nb   ]
//   [ -q     1     6g  ] [mu ] = [st2 = S2 + extra + g sum om_nb ]
//   [ 3g     0     1   ] [om ]   [st3 = S3 + g/2 sum phi_nb      ]
// by eliminating phi and om: mu = (st2 - 6g st3 + (q + 18 g^2) st1) / det,
// det = 1 + kap (q + 18 g^2) >= 1 because q > 0.  The Newton variant uses
// q = f'(phi_n) + (1-eps)/2, extra = f(phi_n) - f'(phi_n) phi_n; the paper's
// Picard variant q = (phi_n^2 + b^2)/4 + (1-eps)/2, extra = (phi_n^2+b^2) b/4.
template <int LIN>
__device__ __forceinline__ void point_solve(const Lvl& L, double sphi, double smu,
                                            double som, double phin, double b,
                                            double s1, double s2, double s3,
                                            double& phi, double& mu, double& om) {
  const double st1 = fma(L.tg, smu, s1);
  const double st3 = fma(L.gh, sphi, s3);
  double q, extra;
  if (LIN == PFC_NEWTON) {
    const double fp = cubic_fp(phin, b);
    q = fp + L.c1;
    extra = fma(-fp, phin, cubic_f(phin, b));
  } else {
    const double p = 0.25 * fma(phin, phin, b * b);
    q = p + L.c1;
    extra = p * b;
  }
  const double st2 = fma(L.g, som, s2 + extra);
  const double Q = q + L.Q0;
  const double det = fma(L.kap, Q, 1.0);
  mu = fma(Q, st1, fma(-L.g6, st3, st2)) / det;
  phi = fma(-L.kap, mu, st1);
  om = fma(-L.g3, phi, st3);
}

// r = S - N(u) at one cell (Eqs. 5.4-5.6 with M = 1); lap receives the
// unscaled 7-point Laplacian of phi (neighbour sum - 6 centre) it computes.
__device__ __forceinline__ void residual_at(const Lvl& L, const Stencil& s,
                                            const double* __restrict__ phi,
                                            const double* __restrict__ mu,
                                            const double* __restrict__ om,
                                            const double* __restrict__ S1,
                                            const double* __restrict__ S2,
                                            const double* __restrict__ S3,
                                            const double* __restrict__ b,
                                            double& r1, double& r2, double& r3, double& lap) {
  const double p = __ldg(phi + s.c), m = __ldg(mu + s.c), w = __ldg(om + s.c);
  const double bb = __ldg(b + s.c);
  const double lmu = fma(-6.0, m, nbsum(mu, s));
  const double lom = fma(-6.0, w, nbsum(om, s));
  const double lphi = fma(-6.0, p, nbsum(phi, s));
  // N1 = phi - tau Lap mu ; N2 = mu - f - c1 phi - Lap om ; N3 = om - Lap phi / 2
  r1 = __ldg(S1 + s.c) - fma(-L.tg, lmu, p);
  r2 = __ldg(S2 + s.c) - (fma(-L.c1, p, m - cubic_f(p, bb)) - L.g * lom);
  r3 = __ldg(S3 + s.c) - fma(-L.gh, lphi, w);
  lap = lphi;
}

__device__ __forceinline__ void residual_at(const Lvl& L, const Stencil& s,
                                            const double* __restrict__ phi,
                                            const double* __restrict__ mu,
                                            const double* __restrict__ om,
                                            const double* __restrict__ S1,
                                            const double* __restrict__ S2,
                                            const double* __restrict__ S3,
                                            const double* __restrict__ b,
                                            double& r1, double& r2, double& r3) {
  double lap;
  residual_at(L, s, phi, mu, om, S1, S2, S3, b, r1, r2, r3, lap);
}

// N(u) at one cell (no source), coherent loads.
__device__ __forceinline__ void operator_at(const Lvl& L, const Stencil& s,
                                            const double* phi, const double* mu,
                                            const double* om, const double* b,
                                            double& n1, double& n2, double& n3) {
  const double p = phi[s.c], m = mu[s.c], w = om[s.c], bb = b[s.c];
  const double lmu = fma(-6.0, m, nbsum_coherent(mu, s));
  const double lom = fma(-6.0, w, nbsum_coherent(om, s));
  const double lphi = fma(-6.0, p, nbsum_coherent(phi, s));
  n1 = fma(-L.tg, lmu, p);
  n2 = fma(-L.c1, p, m - cubic_f(p, bb)) - L.g * lom;
  n3 = fma(-L.gh, lphi, w);
}

// FP64 <-> FP32 conversions on the integer pipe.  GB300 issues FP64<->FP32
// conversions at its FP64 rate (about 2 per SM per clock, like a DFMA), so
// the hot kernels form the bit patterns themselves from the IEEE 754 binary64
// and binary32 layouts (sign | biased exponent | fraction; biases 1023 and
// 127, fractions of 52 and 23 bits).  The rare cases (results that are zero
// or subnormal, overflow, infinities, NaN) are also integer code, kept out of
// line: a hardware conversion there would be evaluated predicated on every
// call and occupy the FP64 pipe (measured: the pointwise defect 29 % and the
// full defect 15 % slower with it).
//
// binary64 -> binary32, round to nearest, ties to even: the exponent is
// rebiased (e - 896), the top 23 fraction bits are kept and the 29 dropped
// ones decide the rounding (above half up; exactly half up when the kept bits
// are odd).  A carry out of the fraction increments the exponent, and past
// the largest finite float it yields the infinity IEEE 754 prescribes.
//
// The rare cases of d2f_rn from the bit fields (hi, lo) of x: NaN gives the
// quiet NaN 0x7FFFFFFF; |x| >= 2^128 or infinite gives the signed infinity;
// |x| < 2^-126 gives a subnormal or zero float, the 53-bit significand M
// (x = M 2^(e-1075)) shifted right by s = 926 - e >= 30 to units of 2^-149
// and rounded to nearest, ties to even (a carry into bit 23 is the smallest
// normal float, the same bit pattern); double subnormals and zeros give a
// signed zero.
static __device__ __noinline__ float d2f_rn_special(unsigned hi, unsigned lo) {
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e == 0x7FFu && ((hi & 0xFFFFFu) | lo)) return __uint_as_float(0x7FFFFFFFu);
  if (e > 1150u) return __uint_as_float(sign | 0x7F800000u);
  if (e == 0u) return __uint_as_float(sign);
  const int sh = 926 - (int)e;                        // >= 30 here (e < 897)
  if (sh >= 54) return __uint_as_float(sign);         // below half of 2^-149
  const unsigned long long M =
      ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const unsigned long long q = M >> sh;
  const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  const unsigned m = (unsigned)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
  return __uint_as_float(sign | m);
}

__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u > 253u) return d2f_rn_special(hi, lo);   // e outside [897, 1150]
  const unsigned kept = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  unsigned bits = ((e - 896u) << 23) | kept;
  bits += (rest > 0x10000000u || (rest == 0x10000000u && (kept & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | bits);
}

// binary32 -> binary64, exact: the exponent is rebiased (e + 896) and the 23
// fraction bits become the top of the 52.  Rare cases out of line: signed
// zeros, infinities, NaN (the quiet NaN 0x7FF80000 00000000 with the sign),
// and subnormal floats m 2^-149 (m < 2^23), normalised at the top set bit p
// of m: biased exponent p + 874, the bits below it the fraction.
static __device__ __noinline__ double f2d_special(unsigned u) {
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 255u)
    return __hiloint2double((int)(sign | (m ? 0x7FF80000u : 0x7FF00000u)), 0);
  if (m == 0u) return __hiloint2double((int)sign, 0);
  const int p = 31 - __clz(m);                        // 0 .. 22
  const unsigned long long f =
      ((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull;
  const unsigned hi = sign | ((unsigned)(p + 874) << 20) | (unsigned)(f >> 32);
  return __hiloint2double((int)hi, (int)(unsigned)f);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u > 253u) return f2d_special(u);             // e == 0 or e == 255
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled while its predecessor drains; pdl_wait()
// blocks until the predecessor has completed and its writes are visible (a
// no-op for a normal launch), pdl_trigger() lets the successor be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Launch with programmatic stream serialization when `pdl` is set (the
// kernel must call pdl_wait() before it reads what its predecessor wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Block-wide sum of NV doubles into thread 0 (fixed order: deterministic).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* 32*NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) smem[c * 32 + wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double x = (lane < nw) ? smem[c * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[c] = x;
    }
  }
  __syncthreads();
}

}  // namespace pfc
