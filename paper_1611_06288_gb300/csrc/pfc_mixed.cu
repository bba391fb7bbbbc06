// Mixed-precision defect correction: double-float residual, source and
// update, FP32 linear multigrid for the correction (see pfc_mixed.h).
#include <math.h>

#include <cooperative_groups.h>

#include "pfc_df.cuh"
#include "pfc_fixed.cuh"
#include "pfc_internal.h"
#include "pfc_mixed.h"

namespace pfc {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t work) { return (unsigned)((work + kThreads - 1) / kThreads); }

// Kernel launch that, when `pdl` is set, carries programmatic stream
// serialization (PDL): the kernel may be scheduled while its predecessor
// drains and must call pdl_wait() before it touches memory.  Profiled runs
// launch without it so that the events around each kernel time it alone.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
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

// 3-D launch over an nx * ny * nz index box: x is the fastest (contiguous)
// index, 256 threads per block; kernels read (x, y, z) from the grid and
// never divide.
struct Launch3 {
  dim3 grid, block;
};
inline Launch3 launch3(int nx, int ny, int nz) {
  int bx = 1;
  while (bx < nx && bx < 128) bx <<= 1;
  int by = 256 / bx;
  if (by > ny) by = ny;
  Launch3 l;
  l.block = dim3(bx, by, 1);
  l.grid = dim3((nx + bx - 1) / bx, (ny + by - 1) / by, nz);
  return l;
}

// FP32 constants of one level of the linearised system.
struct LvlF {
  int n;
  float g, tg, kap, g6, g3, gh, Q0;
};

inline LvlF to_f32(const Lvl& L) {
  LvlF f;
  f.n = L.n;
  f.g = (float)L.g;
  f.tg = (float)L.tg;
  f.kap = (float)L.kap;
  f.g6 = (float)L.g6;
  f.g3 = (float)L.g3;
  f.gh = (float)L.gh;
  f.Q0 = (float)L.Q0;
  return f;
}

// ---------------------------------------------------------------------------
// Colour-split layout of the FP32 fields.  Within every x-row (j, k) of an
// even-sized level the n/2 cells of colour 0 ((i+j+k) even) come first,
// ordered by i/2, then the n/2 cells of colour 1.  A red-black half-sweep then
// reads and writes contiguous runs of one colour only, and every neighbour of
// a cell lies in the other colour's half of its row or of the adjacent rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int split_index(int i, int j, int k, int n) {
  return (k * n + j) * n + ((i + j + k) & 1) * (n >> 1) + (i >> 1);
}

// Batched launches (ensembles of independent members of one grid size, stored
// member after member): the grid's z extent covers members x planes.  Returns
// the member of this block and reduces z to its plane; a single-member
// launch has member 0.
__device__ __forceinline__ int member_of(int& z, int planes) {
  const int m = z / planes;
  z -= m * planes;
  return m;
}

// The cell (p, j, k) of colour `colour` (i = 2p + ((j+k+colour) & 1)) and its six
// neighbours, as split-layout indices (32-bit arithmetic: n^3 < 2^31).
__device__ __forceinline__ Stencil split_stencil(int p, int j, int k, int colour, int n) {
  const int half = n >> 1;
  const int sigma = (j + k + colour) & 1;
  const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
  const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
  int pm = p - 1 + sigma;
  if (pm < 0) pm += half;
  int pp = p + sigma;
  if (pp >= half) pp -= half;
  const int oc = (1 - colour) * half;
  const int row = (k * n + j) * n;
  Stencil s;
  s.c = row + colour * half + p;
  s.xm = row + oc + pm;
  s.xp = row + oc + pp;
  s.ym = (k * n + jm) * n + oc + p;
  s.yp = (k * n + jp) * n + oc + p;
  s.zm = (km * n + j) * n + oc + p;
  s.zp = (kp * n + j) * n + oc + p;
  return s;
}

// Split-order thread index t -> (p, j, k, colour).
__device__ __forceinline__ void split_cell(int64_t t, int n, int& p, int& j, int& k,
                                           int& colour) {
  const int half = n >> 1;
  const int x = (int)(t % n);
  const int64_t r = t / n;
  j = (int)(r % n);
  k = (int)(r / n);
  colour = x >= half;
  p = x - colour * half;
}

// Constants of the double-float operator on one level.
struct LvlD {
  int n;
  df tg;     // tau/h^2
  df g;      // 1/h^2
  df gh;     // 1/(2 h^2)
  df c1;     // (1 - eps)/2
  float c1f;
};

LvlD to_df(const Lvl& L) {
  LvlD d;
  d.n = L.n;
  d.tg = df_const(L.tg);
  d.g = df_const(L.g);
  d.gh = df_const(L.gh);
  d.c1 = df_const(L.c1);
  d.c1f = (float)L.c1;
  return d;
}

// Natural-order indices of a cell's six periodic neighbours (32-bit: n^3 < 2^31).
struct Nb6 {
  int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nb6 nb6_at(int t, int i, int j, int k, int n) {
  const int nn = n * n;
  Nb6 s;
  s.xm = (i == 0) ? t + n - 1 : t - 1;
  s.xp = (i + 1 == n) ? t - (n - 1) : t + 1;
  s.ym = (j == 0) ? t + nn - n : t - n;
  s.yp = (j + 1 == n) ? t - (nn - n) : t + n;
  s.zm = (k == 0) ? t + n * nn - nn : t - nn;
  s.zp = (k + 1 == n) ? t - (n * nn - nn) : t + nn;
  return s;
}

// Unscaled 7-point Laplacian (neighbour sum - 6 centre) of a df field.
__device__ __forceinline__ df df_lap(const float2* __restrict__ v, const Nb6& s, df c) {
  const df sum = df_sum6(df_ld(v, s.xm), df_ld(v, s.xp), df_ld(v, s.ym), df_ld(v, s.yp),
                         df_ld(v, s.zm), df_ld(v, s.zp));
  return df_sub(sum, df_mul_f(c, 6.f));
}

// Block-wide FP32 sum into thread 0 (fixed order: deterministic).
__device__ __forceinline__ float block_sum_f(float v, float* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < nw) ? sm[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Neighbour sum of an FP64 field at the six indices of s (fixed order).
__device__ __forceinline__ double nbsum64(const double* __restrict__ v, const Nb6& s) {
  return ((__ldg(v + s.xm) + __ldg(v + s.xp)) + (__ldg(v + s.ym) + __ldg(v + s.yp))) +
         (__ldg(v + s.zm) + __ldg(v + s.zp));
}

// Defect of the FP64 outer loop (PFC_MIXED): r = S - N(u) in FP64 (Eqs.
// 5.4-5.6, M = 1) rounded to FP32 into the colour-split r1..r3, the Newton
// coefficient q = f'(phi) + (1-eps)/2 of the cubic term in FP64 rounded to
// FP32, and per-block sums of |r|^2 (of the FP32-rounded r, accumulated in
// FP32 within a block: the sum only decides convergence).  f and f' share
// phi^2, b^2 and phi b; the roundings to FP32 use the integer pipe.  lap
// (may be null) receives the unscaled Laplacian of phi for later reuse.
template <bool MOB>
__global__ void __launch_bounds__(256) k_defect64(Lvl L, const double* __restrict__ phi,
                                                  const double* __restrict__ mu,
                                                  const double* __restrict__ om,
                                                  const double* __restrict__ S1,
                                                  const double* __restrict__ S2,
                                                  const double* __restrict__ S3,
                                                  const double* __restrict__ b,
                                                  float* __restrict__ r1, float* __restrict__ r2,
                                                  float* __restrict__ r3, float* __restrict__ q,
                                                  double* partials, double* __restrict__ lap,
                                                  const double* __restrict__ c1m,
                                                  const double* __restrict__ Mx,
                                                  const double* __restrict__ My,
                                                  const double* __restrict__ Mz) {
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  const int m = blockIdx.y;                  // member of a batched launch
  const size_t off = (size_t)m * cells;
  phi += off, mu += off, om += off, S1 += off, S2 += off, S3 += off, b += off;
  r1 += off, r2 += off, r3 += off, q += off;
  if (lap) lap += off;
  partials += (size_t)m * gridDim.x;
  const double c1 = c1m ? c1m[m] : L.c1;
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Nb6 s = nb6_at(t, i, j, k, n);
    const double p = __ldg(phi + t), mm = __ldg(mu + t), w = __ldg(om + t);
    const double bb = __ldg(b + t);
    // row 1: d(M D mu) with the face mobilities (MOB), else the Laplacian;
    // M^x at t is the face i+1/2, at s.xm the face i-1/2
    double lmu;
    if (MOB) {
      lmu = fma(__ldg(Mx + t), __ldg(mu + s.xp) - mm, __ldg(Mx + s.xm) * (__ldg(mu + s.xm) - mm));
      lmu = fma(__ldg(My + t), __ldg(mu + s.yp) - mm,
                fma(__ldg(My + s.ym), __ldg(mu + s.ym) - mm, lmu));
      lmu = fma(__ldg(Mz + t), __ldg(mu + s.zp) - mm,
                fma(__ldg(Mz + s.zm), __ldg(mu + s.zm) - mm, lmu));
    } else {
      lmu = fma(-6.0, mm, nbsum64(mu, s));
    }
    const double lom = fma(-6.0, w, nbsum64(om, s));
    const double lphi = fma(-6.0, p, nbsum64(phi, s));
    const double p2 = p * p, b2 = bb * bb, pb = p * bb;
    const double f = 0.25 * ((p + bb) * (p2 + b2));          // f(phi, b), Eq. 5.2
    const double fp = fma(0.75, p2, fma(0.5, pb, 0.25 * b2));  // df/dphi
    const double x = __ldg(S1 + t) - fma(-L.tg, lmu, p);
    const double y = __ldg(S2 + t) - (fma(-c1, p, mm - f) - L.g * lom);
    const double z = __ldg(S3 + t) - fma(-L.gh, lphi, w);
    const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(z);
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    q[o] = d2f_rn(fp + c1);
    if (lap) lap[t] = lphi;
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// The FP64 defect with the three Laplacians' neighbour sums formed exactly in
// 64-bit fixed point on the integer pipe (pfc_fixed.cuh) and the rows in 12
// FP64 operations (defect_rows); M = 1.  r and the norm are those of the
// FP64 residual up to rounding order (the Laplacians: exact sums of the
// quantised inputs and one rounding, instead of five FP64 roundings).
//
// Tiling: a block of kFxTX x kFxTY threads owns that column of cells over
// `zc` planes starting at plane k0 and marches upwards in z.  Each thread
// keeps the fixed-point images of its cell in the planes k-1, k, k+1 in
// registers; the images of plane k, with a one-cell halo in x and y (wrapped
// periodically), sit in shared memory for the four in-plane neighbours.  So
// every value is loaded and converted once per block (plus the halo), not
// once per neighbour, and the raw values of the next plane are loaded one
// plane ahead.  Threads past the grid edge (n < kFxTX or n < kFxTY) load
// wrapped cells to fill the tile and write nothing.
//
// lap (may be null) receives the unscaled Laplacian of phi, lapmu and lapom
// (null, or both set) those of mu and omega, for the first defect of the next
// step (k_defect64_point).
//
// Range: inputs with |v| >= 32, Inf or NaN have no fixed-point image.  From
// the first plane whose tile holds such a value the block evaluates its
// Laplacians in FP64 from global memory (a block vote per plane); a cell
// whose own value in the plane above is out of range does so alone.  Same
// outputs either way.  Per-block partial sums of |r|^2 as k_defect64.
constexpr int kFxTX = 32, kFxTY = 8;
// Shared-memory ring of the fixed-point images of planes k-1, k, k+1 (own
// cells, and the halo of plane k): four slots, so one barrier per plane
// orders every write after the reads of the slot's previous plane.
constexpr int kFxRing = 4;
constexpr size_t kFxSmem = (size_t)kFxRing * 3 * (kFxTY + 2) * (kFxTX + 2) * sizeof(int64_t);

// The three rows at one cell from the unscaled Laplacians, in 12 FP64
// operations: x = S1 - phi + tau/h^2 Lap mu, y = S2 - mu + f + c1 phi +
// 1/h^2 Lap om with f = (phi + b)(phi^2 + b^2)/4 (Eq. 5.2), z = S3 - om +
// 1/(2h^2) Lap phi, each rounded to FP32 on the integer pipe.  The Newton
// coefficient q = f'(phi) + c1 only feeds the FP32 preconditioner: it is
// formed in FP32 from phi and b rounded to FP32 (a few FP32 roundings).
__device__ __forceinline__ void defect_rows(const Lvl& L, double c1, float c1f, double p,
                                            double mm, double w, double bb, double lmu,
                                            double lom, double lphi, double s1, double s2,
                                            double s3, float& xf, float& yf, float& zf,
                                            float& qf) {
  const double t = p + bb;
  const double sq = fma(p, p, bb * bb);
  const double x = fma(L.tg, lmu, s1 - p);
  const double y = fma(L.g, lom, fma(c1, p, fma(0.25 * t, sq, s2 - mm)));
  const double z = fma(L.gh, lphi, s3 - w);
  xf = d2f_rn(x);
  yf = d2f_rn(y);
  zf = d2f_rn(z);
  const float pf = d2f_rn(p), bf = d2f_rn(bb);
  qf = fmaf(0.75f * pf, pf, fmaf(0.5f * pf, bf, fmaf(0.25f * bf, bf, c1f)));
}

__global__ void __launch_bounds__(kFxTX * kFxTY, 4) k_defect64_fx(
    Lvl L, int zc, const double* __restrict__ phi, const double* __restrict__ mu,
    const double* __restrict__ om, const double* __restrict__ S1, const double* __restrict__ S2,
    const double* __restrict__ S3, const double* __restrict__ b, float* __restrict__ r1,
    float* __restrict__ r2, float* __restrict__ r3, float* __restrict__ q, double* partials,
    double* __restrict__ lap, const double* __restrict__ c1m, double* __restrict__ lapmu,
    double* __restrict__ lapom) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ int64_t ring[];   // [kFxRing][3][kFxTY + 2][kFxTX + 2]
  __shared__ float sm[32];
  constexpr int TW = kFxTX + 2, TP = (kFxTY + 2) * TW, TS = 3 * TP;
  const int n = L.n, nn = n * n;
  const int chunks = (n + zc - 1) / zc;
  int zb = blockIdx.z;
  const int m = member_of(zb, chunks);
  // the member's offset rides in the indices: the field pointers stay
  // kernel parameters instead of occupying registers
  const int64_t off = (int64_t)m * nn * n;
  const bool s1_is_b = S1 == b;
  const double c1 = c1m ? c1m[m] : L.c1;
  const float c1f = d2f_rn(c1);
  const int tid = threadIdx.x, tx = tid % kFxTX, ty = tid / kFxTX;   // 1-D block
  const int i0 = blockIdx.x * kFxTX, j0 = blockIdx.y * kFxTY;
  const int k0 = zb * zc, k1 = min(n, k0 + zc);
  const bool active = i0 + tx < n && j0 + ty < n;
  const int iw = (i0 + tx) % n, jw = (j0 + ty) % n;     // wrapped own column
  const int own = jw * n + iw;
  const int ocell = (ty + 1) * TW + tx + 1;              // own cell in a tile plane
  // halo cell of this thread (tid < 2 kFxTY + 2 kFxTX): in-plane index and
  // tile position
  int hidx = -1, hcell = 0;
  if (tid < 2 * kFxTY) {
    const int r = tid % kFxTY, side = tid / kFxTY;        // x = i0 - 1 or i0 + kFxTX
    hcell = (r + 1) * TW + (side ? kFxTX + 1 : 0);
    hidx = ((j0 + r) % n) * n + (side ? (i0 + kFxTX) % n : (i0 - 1 + n) % n);
  } else if (tid < 2 * kFxTY + 2 * kFxTX) {
    const int h = tid - 2 * kFxTY, c = h % kFxTX, side = h / kFxTX;   // y = j0 - 1 or j0 + kFxTY
    hcell = (side ? kFxTY + 1 : 0) * TW + c + 1;
    hidx = (side ? (j0 + kFxTY) % n : (j0 - 1 + n) % n) * n + (i0 + c) % n;
  }
#define PFC_FX_FLD(f) ((f) == 0 ? phi : (f) == 1 ? mu : om)
  // Software pipeline over the planes: the images of plane k+1 (own cells)
  // are formed from raw values loaded during plane k-1 and stored in the
  // ring slot of plane k+1; the halo of plane k arrives during plane k-1.
  // ok: the own images this thread formed so far are in range (they enter
  // the block vote of the next plane); okn: the own image of plane k+1,
  // checked per cell.
  bool ok = true;
  double dn[3], hraw[3];
  {
    const int km = (k0 - 1 + n) % n, kp = (k0 + 1) % n;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      ring[((k0 + kFxRing - 1) % kFxRing) * TS + f * TP + ocell] =
          fix_of(__ldg(PFC_FX_FLD(f) + off + km * nn + own), ok);
      ring[(k0 % kFxRing) * TS + f * TP + ocell] =
          fix_of(__ldg(PFC_FX_FLD(f) + off + k0 * nn + own), ok);
      dn[f] = __ldg(PFC_FX_FLD(f) + off + kp * nn + own);
      hraw[f] = hidx >= 0 ? __ldg(PFC_FX_FLD(f) + off + k0 * nn + hidx) : 0.0;
    }
  }
  bool fx_path = true;
  float acc = 0.f;
  for (int k = k0; k < k1; ++k) {
    const int kp = (k + 1 == n) ? 0 : k + 1;
    const int kp2 = (kp + 1 == n) ? 0 : kp + 1;
    const int t = k * nn + own;
    const bool more = k + 1 < k1;
    // kFxRing slots: the one written here (plane k+1) was last read two
    // planes ago, so the barrier of the previous plane orders the accesses
    int64_t* const cur = ring + (k % kFxRing) * TS;
    int64_t* const nxt = ring + ((k + 1) % kFxRing) * TS;
    const int64_t* const prv = ring + ((k + kFxRing - 1) % kFxRing) * TS;
    bool okn = true;
#pragma unroll
    for (int f = 0; f < 3; ++f) nxt[f * TP + ocell] = fix_of(dn[f], okn);
#pragma unroll
    for (int f = 0; f < 3; ++f)
      dn[f] = more ? __ldg(PFC_FX_FLD(f) + off + kp2 * nn + own) : 0.0;
    bool okt = ok;
    if (hidx >= 0) {
#pragma unroll
      for (int f = 0; f < 3; ++f) cur[f * TP + hcell] = fix_of(hraw[f], okt);
    }
    fx_path = __syncthreads_and(fx_path && okt) != 0;
    ok = okn;
    if (hidx >= 0 && more) {
#pragma unroll
      for (int f = 0; f < 3; ++f) hraw[f] = __ldg(PFC_FX_FLD(f) + off + kp * nn + hidx);
    }
    double lap3[3];
    if (fx_path && okn) {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const int64_t* const c = cur + f * TP;
        lap3[f] = fix_to_double(fix_lap(c[ocell - 1], c[ocell + 1], c[ocell - TW], c[ocell + TW],
                                        prv[f * TP + ocell], nxt[f * TP + ocell], c[ocell]));
      }
    } else {
      const Nb6 sn = nb6_at(t, iw, jw, k, n);
#pragma unroll
      for (int f = 0; f < 3; ++f)
        lap3[f] = fma(-6.0, __ldg(PFC_FX_FLD(f) + off + t), nbsum64(PFC_FX_FLD(f) + off, sn));
    }
    if (active) {
      const double bb = __ldg(b + off + t), s2 = __ldg(S2 + off + t), s3 = __ldg(S3 + off + t);
      const double s1 = s1_is_b ? bb : __ldg(S1 + off + t);
      float xf, yf, zf, qf;
      // the centre values of plane k, loaded two planes ago, come from L1
      defect_rows(L, c1, c1f, __ldg(phi + off + t), __ldg(mu + off + t), __ldg(om + off + t),
                  bb, lap3[1], lap3[2], lap3[0], s1, s2, s3, xf, yf, zf, qf);
      acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
      const int64_t o = off + split_index(iw, jw, k, n);
      r1[o] = xf;
      r2[o] = yf;
      r3[o] = zf;
      q[o] = qf;
      if (lap) lap[off + t] = lap3[0];
      if (lapmu) {
        lapmu[off + t] = lap3[1];
        lapom[off + t] = lap3[2];
      }
    }
  }
#undef PFC_FX_FLD
  acc = block_sum_f(acc, sm);
  if (tid == 0)
    partials[(size_t)m * (gridDim.x * gridDim.y * chunks) +
             ((size_t)zb * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = (double)acc;
}

// First defect of a step that starts from the previous step's solution
// (phi^{k+1} := phi^k = b bit for bit, mu and omega kept): r = S - N(u) from
// the Laplacians the previous step's last defect stored (lapb of phi^k = b,
// lapmu, lapom), with no stencil.  With phi = b = S1 the rows reduce to
//   x = tau/h^2 Lap mu,  y = S2 - mu + phi^3 + c1 phi + 1/h^2 Lap om
//   (f(phi, phi) = phi^3, Eq. 5.2),  z = S3 - om + 1/(2h^2) Lap phi,
// 8 FP64 operations, each rounded to FP32 on the integer pipe, and
// q = f'(phi, phi) + c1 = 3/2 phi^2 + c1 in FP32.  lap (the iterate's
// Laplacian slot) receives lapb.  Grid: blockIdx.y the member, a grid-stride
// loop over its cells; per-block sums of |r|^2 as k_defect64.
__global__ void __launch_bounds__(256) k_defect64_point(
    Lvl L, const double* __restrict__ b, const double* __restrict__ mu,
    const double* __restrict__ om, const double* __restrict__ S2,
    const double* __restrict__ S3, const double* __restrict__ lapb,
    const double* __restrict__ lapmu, const double* __restrict__ lapom, float* __restrict__ r1,
    float* __restrict__ r2, float* __restrict__ r3, float* __restrict__ q, double* partials,
    double* __restrict__ lap, const double* __restrict__ c1m) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  const int m = blockIdx.y;
  const size_t off = (size_t)m * cells;
  b += off, mu += off, om += off, S2 += off, S3 += off;
  lapb += off, lapmu += off, lapom += off, lap += off;
  r1 += off, r2 += off, r3 += off, q += off;
  partials += (size_t)m * gridDim.x;
  const double c1 = c1m ? c1m[m] : L.c1;
  const float c1f = d2f_rn(c1);
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const double p = __ldg(b + t), lb = __ldg(lapb + t);
    const double x = L.tg * __ldg(lapmu + t);
    const double y =
        fma(L.g, __ldg(lapom + t), fma(c1, p, fma(p * p, p, __ldg(S2 + t) - __ldg(mu + t))));
    const double z = fma(L.gh, lb, __ldg(S3 + t) - __ldg(om + t));
    const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(z);
    const float pf = d2f_rn(p);
    const float qf = fmaf(1.5f * pf, pf, c1f);
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    q[o] = qf;
    lap[t] = lb;
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// Start of a warm step in one pass: S2, S3 of Eqs. 5.9-5.10 from the stored
// unscaled Laplacians of phi^k (lapb) and phi^{k-1} (lapc), with the
// operations of k_source_cached; the initial iterate phi^{k+1} := phi^k
// (phi_next); and the pointwise first defect of k_defect64_point from those
// S2, S3 (the same values it would read back).  Bit-identical to the three
// separate steps; one read of b and lapb for all of them.
__global__ void __launch_bounds__(256) k_start64_point(
    Lvl L, const double* __restrict__ b, const double* __restrict__ mu,
    const double* __restrict__ om, const double* __restrict__ lapb,
    const double* __restrict__ lapc, const double* __restrict__ lapmu,
    const double* __restrict__ lapom, double* __restrict__ S2, double* __restrict__ S3,
    double* __restrict__ phi_next, float* __restrict__ r1, float* __restrict__ r2,
    float* __restrict__ r3, float* __restrict__ q, double* partials, double* __restrict__ lap,
    const double* __restrict__ c1m) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  const int m = blockIdx.y;
  const size_t off = (size_t)m * cells;
  b += off, mu += off, om += off, lapb += off, lapc += off, lapmu += off, lapom += off;
  S2 += off, S3 += off, phi_next += off, lap += off;
  r1 += off, r2 += off, r3 += off, q += off;
  partials += (size_t)m * gridDim.x;
  const double c1 = c1m ? c1m[m] : L.c1;
  const float c1f = d2f_rn(c1);
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const double p = __ldg(b + t), lbr = __ldg(lapb + t);
    const double lb = L.g * lbr;
    const double lc = L.g * __ldg(lapc + t);
    const double s2 = fma(3.0, lb, fma(c1, p, -lc));
    const double s3 = 0.5 * lb;
    S2[t] = s2;
    S3[t] = s3;
    phi_next[t] = p;
    const double x = L.tg * __ldg(lapmu + t);
    const double y = fma(L.g, __ldg(lapom + t), fma(c1, p, fma(p * p, p, s2 - __ldg(mu + t))));
    const double z = fma(L.gh, lbr, s3 - __ldg(om + t));
    const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(z);
    const float pf = d2f_rn(p);
    const float qf = fmaf(1.5f * pf, pf, c1f);
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    q[o] = qf;
    lap[t] = lbr;
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// Start of a step from the extrapolated iterate u^{k+1} := 2 u^k - u^{k-1}
// of all three fields, in one pass with no stencil: the Laplacian is linear,
// so the iterate's Laplacians are 2 Lap u^k - Lap u^{k-1} of the ones the two
// last steps' final defects stored (lapb, lapc of phi^k = b, phi^{k-1} = c;
// lapmu0, lapom0 of mu^k, omega^k; lapmu1, lapom1 of mu^{k-1}, omega^{k-1}).
// The rows of the first defect are then linear combinations of the twelve
// stored values with small integer weights plus the cubic f (Eq. 5.2):
//   x = (c - b) + tau/h^2 Lap mu,
//   z = (3 Lap b - Lap c)/(2h^2) - omega,
//   y = (3 Lap b - Lap c + Lap omega)/h^2 + c1 (3b - c) + f(phi, b) - mu,
// with S2 = (3 Lap b - Lap c)/h^2 + c1 b and S3 = Lap b/(2h^2) (Eqs. 5.9-5.10)
// and phi = 2b - c, mu, omega the iterate.  GB300's FP64 pipe is the limit of
// this pass (23 FP64 operations per cell in plain FP64), so the five
// combinations of b, c and their Laplacians (2b - c, c - b, 3b - c,
// 2 Lap b - Lap c, 3 Lap b - Lap c) are formed exactly on the integer pipe
// from the fixed-point images of pfc_fixed.cuh (each rounded once to
// binary64), leaving 16 FP64 operations and about as much integer work:
// converting every input instead moves the limit to the integer pipe (a
// conversion costs about 30 instructions).  A cell with b, c or a Laplacian
// outside the fixed-point range (|v| >= 32, Inf, NaN) takes the same
// formulas in FP64.  The results differ from FP64 arithmetic by the 2^-55
// quantisation of the inputs, far below the FP32 rounding of the rows.
// mu1, om1, lapmu1, lapom1 hold step k-1's fields on entry and the iterate's
// on exit: each cell is read, then written, by the same thread.  lap receives
// the iterate's Laplacian of phi.  Grid: blockIdx.y the member, a grid-stride
// loop over its cells; per-block sums of |r|^2.
__global__ void __launch_bounds__(256, 4) k_start64_extrap(
    Lvl L, const double* __restrict__ b, const double* __restrict__ c,
    const double* __restrict__ lapb, const double* __restrict__ lapc,
    const double* __restrict__ mu0, const double* __restrict__ om0,
    const double* __restrict__ lapmu0, const double* __restrict__ lapom0,
    double* __restrict__ mu1, double* __restrict__ om1, double* __restrict__ lapmu1,
    double* __restrict__ lapom1, double* __restrict__ S2, double* __restrict__ S3,
    double* __restrict__ phi, float* __restrict__ r1, float* __restrict__ r2,
    float* __restrict__ r3, float* __restrict__ q, double* partials,
    double* __restrict__ lap, const double* __restrict__ c1m) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  const int m = blockIdx.y;
  const size_t off = (size_t)m * cells;
  b += off, c += off, lapb += off, lapc += off, mu0 += off, om0 += off;
  lapmu0 += off, lapom0 += off, mu1 += off, om1 += off, lapmu1 += off, lapom1 += off;
  S2 += off, S3 += off, phi += off, lap += off;
  r1 += off, r2 += off, r3 += off, q += off;
  partials += (size_t)m * gridDim.x;
  const double c1 = c1m ? c1m[m] : L.c1;
  const float c1f = d2f_rn(c1);
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const double vb = __ldg(b + t), vc = __ldg(c + t);
    const double vlb = __ldg(lapb + t), vlc = __ldg(lapc + t);
    const double vm0 = __ldg(mu0 + t), vm1 = mu1[t];
    const double vo0 = __ldg(om0 + t), vo1 = om1[t];
    const double vlm0 = __ldg(lapmu0 + t), vlm1 = lapmu1[t];
    const double vlo0 = __ldg(lapom0 + t), vlo1 = lapom1[t];
    // the iterate, its Laplacians and the linear parts of the rows: the
    // combinations of phi^k, phi^{k-1} and their Laplacians in fixed point,
    // those of mu, omega in FP64 (the split that balances the two pipes)
    const double mm = fma(2.0, vm0, -vm1);
    const double w = fma(2.0, vo0, -vo1);
    const double lm = fma(2.0, vlm0, -vlm1);
    const double lo = fma(2.0, vlo0, -vlo1);
    double p, lp, cmb, k3, bs;
    bool ok = true;
    const int64_t B = fix_of(vb, ok), C = fix_of(vc, ok);
    const int64_t LB = fix_of(vlb, ok), LC = fix_of(vlc, ok);
    if (ok) {                       // |images| < 2^59: no overflow
      p = fix_to_double(2 * B - C);
      cmb = fix_to_double(C - B);
      bs = fix_to_double(3 * B - C);
      lp = fix_to_double(2 * LB - LC);
      k3 = fix_to_double(3 * LB - LC);
    } else {
      p = fma(2.0, vb, -vc);
      cmb = vc - vb;
      bs = vb + p;
      lp = fma(2.0, vlb, -vlc);
      k3 = fma(3.0, vlb, -vlc);
    }
    const double a = k3 + lo;
    const double s2 = fma(L.g, k3, c1 * vb);
    const double s3 = L.gh * vlb;
    S2[t] = s2;
    S3[t] = s3;
    phi[t] = p;
    mu1[t] = mm;
    om1[t] = w;
    lap[t] = lp;
    lapmu1[t] = lm;
    lapom1[t] = lo;
    const double sq = fma(p, p, vb * vb);
    const double x = fma(L.tg, lm, cmb);
    const double y = fma(L.g, a, fma(c1, bs, fma(0.25 * bs, sq, -mm)));
    const double z = fma(L.gh, k3, -w);
    const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(z);
    const float pf = d2f_rn(p), bf = d2f_rn(vb);
    const float qf = fmaf(0.75f * pf, pf, fmaf(0.5f * pf, bf, fmaf(0.25f * bf, bf, c1f)));
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    q[o] = qf;
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// Face mobilities of a step: M(A phi_*) on the faces i+1/2 of each axis for
// M(phi) = m0 + m2 phi^2, phi_* = 3/2 b - 1/2 c (b = phi^k, c = phi^{k-1});
// the face i+1/2 of an axis is stored at cell i.
__global__ void k_face_mobility(int n, double m0, double m2, const double* __restrict__ b,
                                const double* __restrict__ c, double* __restrict__ Mx,
                                double* __restrict__ My, double* __restrict__ Mz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const Nb6 s = nb6_at(t, i, j, k, n);
  const double ps = fma(1.5, __ldg(b + t), -0.5 * __ldg(c + t));
  const double px = fma(1.5, __ldg(b + s.xp), -0.5 * __ldg(c + s.xp));
  const double py = fma(1.5, __ldg(b + s.yp), -0.5 * __ldg(c + s.yp));
  const double pz = fma(1.5, __ldg(b + s.zp), -0.5 * __ldg(c + s.zp));
  const double ax = 0.5 * (ps + px), ay = 0.5 * (ps + py), az = 0.5 * (ps + pz);
  Mx[t] = fma(m2 * ax, ax, m0);
  My[t] = fma(m2 * ay, ay, m0);
  Mz[t] = fma(m2 * az, az, m0);
}

// Adjoint of a time step (the transposed linearised system).  With P the
// swap of the phi and mu components and S = diag(1, 1, 2), J^T = S P J P S^-1
// for J = [[I, -tau Lap, 0], [-diag(q), I, -Lap], [-Lap/2, 0, I]] (Eqs.
// 5.4-5.6 differentiated in u), so J^T psi = (g, 0, 0) is solved as
// J z = (0, g, 0) with psi = (z2, z1, 2 z3), by the forward correction
// machinery.  This kernel is its FP64 defect r = (0, g, 0) - J z with
// q = f'(a, b) + (1-eps)/2 at the step's solution a = phi^{k+1}, b = phi^k,
// r and q rounded to FP32 (colour-split), per-block sums of |r|^2.
__global__ void __launch_bounds__(256) k_adj_defect64(
    Lvl L, const double* __restrict__ z1, const double* __restrict__ z2,
    const double* __restrict__ z3, const double* __restrict__ g, const double* __restrict__ a,
    const double* __restrict__ b, float* __restrict__ r1, float* __restrict__ r2,
    float* __restrict__ r3, float* __restrict__ q, double* partials) {
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Nb6 s = nb6_at(t, i, j, k, n);
    const double x1 = __ldg(z1 + t), x2 = __ldg(z2 + t), x3 = __ldg(z3 + t);
    const double l1 = fma(-6.0, x1, nbsum64(z1, s));
    const double l2 = fma(-6.0, x2, nbsum64(z2, s));
    const double l3 = fma(-6.0, x3, nbsum64(z3, s));
    const double p = __ldg(a + t), bb = __ldg(b + t);
    const double qq = fma(0.75 * p, p, fma(0.5 * p, bb, 0.25 * bb * bb)) + L.c1;
    const double x = fma(L.tg, l2, -x1);                         // 0 - (z1 - tau Lap z2)
    const double y = __ldg(g + t) - (fma(-qq, x1, x2) - L.g * l3);
    const double zz = fma(L.gh, l1, -x3);                        // 0 - (z3 - Lap z1 / 2)
    const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(zz);
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    q[o] = d2f_rn(qq);
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// Gradient propagation of one adjoint step from psi = (z2, z1, 2 z3):
//   dL/dphi^k     += psi1 + (df/db + (1-eps)/2) psi2 + 3 Lap psi2 + Lap psi3 / 2
//   dL/dphi^{k-1} += -Lap psi2
//   dL/deps       += -sum psi2 (a + b) / 2         (per-block partials)
// (df/db = (a^2 + 2ab + 3b^2)/4 for f(a, b) = (a+b)(a^2+b^2)/4); when gkm1 ==
// gk (the first step, phi^{-1} = phi^0) both terms go to gk.
__global__ void __launch_bounds__(256) k_adj_accumulate(
    Lvl L, const double* __restrict__ z1, const double* __restrict__ z2,
    const double* __restrict__ z3, const double* __restrict__ a, const double* __restrict__ b,
    double* gk, double* gkm1, double* partials) {
  __shared__ double sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  const bool same = gk == gkm1;
  double acc[1] = {0.0};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Nb6 s = nb6_at(t, i, j, k, n);
    const double x1 = __ldg(z1 + t), x2 = __ldg(z2 + t), x3 = __ldg(z3 + t);
    const double lp2 = L.g * fma(-6.0, x1, nbsum64(z1, s));        // Lap psi2
    const double lp3 = 2.0 * L.g * fma(-6.0, x3, nbsum64(z3, s));  // Lap psi3
    const double p = __ldg(a + t), bb = __ldg(b + t);
    const double dfb = 0.25 * fma(p, p, fma(2.0 * p, bb, 3.0 * bb * bb));
    const double dk = fma(dfb + L.c1, x1, x2) + fma(3.0, lp2, 0.5 * lp3);
    if (same) {
      gk[t] += dk - lp2;
    } else {
      gk[t] += dk;
      gkm1[t] -= lp2;
    }
    acc[0] = fma(-0.5 * x1, p + bb, acc[0]);
  }
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}



// Unscaled 7-point Laplacian (neighbour sum - 6 centre) of a df field as an
// unnormalised pair: -6 c split exactly by one FMA, then the six neighbours.
__device__ __forceinline__ dacc dacc_lap(const float2* __restrict__ v, const Nb6& s, df c) {
  dacc L;
  L.hi = __fmul_rn(-6.f, c.hi);
  L.lo = __fmaf_rn(-6.f, c.lo, __fmaf_rn(-6.f, c.hi, -L.hi));
  dacc_add(L, df_ld(v, s.xm));
  dacc_add(L, df_ld(v, s.xp));
  dacc_add(L, df_ld(v, s.ym));
  dacc_add(L, df_ld(v, s.yp));
  dacc_add(L, df_ld(v, s.zm));
  dacc_add(L, df_ld(v, s.zp));
  return L;
}

// f(p, b) = (p+b)(p^2+b^2)/4 (Eq. 5.2) from df operands as an unnormalised
// pair: each factor is formed exactly in its hi part plus an FP32 correction.
__device__ __forceinline__ dacc dacc_cubic(df p, df b) {
  dacc s;                                     // p + b
  two_sum(p.hi, b.hi, s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, __fadd_rn(p.lo, b.lo));
  const float p2 = __fmul_rn(p.hi, p.hi), b2 = __fmul_rn(b.hi, b.hi);
  const float p2e = __fmaf_rn(__fadd_rn(p.hi, p.hi), p.lo, __fmaf_rn(p.hi, p.hi, -p2));
  const float b2e = __fmaf_rn(__fadd_rn(b.hi, b.hi), b.lo, __fmaf_rn(b.hi, b.hi, -b2));
  dacc t;                                     // p^2 + b^2
  two_sum(p2, b2, t.hi, t.lo);
  t.lo = __fadd_rn(t.lo, __fadd_rn(p2e, b2e));
  dacc f;                                     // s t / 4 (the 1/4 is exact)
  const float hi = __fmul_rn(s.hi, t.hi);
  const float lo =
      __fmaf_rn(s.lo, t.hi, __fmaf_rn(s.hi, t.lo, __fmaf_rn(s.hi, t.hi, -hi)));
  f.hi = __fmul_rn(0.25f, hi);
  f.lo = __fmul_rn(0.25f, lo);
  return f;
}

// Defect of the outer loop: r = S - N(u) (Eqs. 5.4-5.6, M = 1) evaluated in
// double-float from df fields, every component one unnormalised sum of its
// terms rounded to FP32 into the colour-split r1..r3;
// q = f'(phi) + (1-eps)/2 (Jacobian of the cubic term of Eq. 5.2) in FP32
// from the hi parts of phi and b, colour-split; per-block partial sums of
// |r|^2 (FP32 within a block, one double per block); lap (may be null)
// receives the unscaled Laplacian of phi as a df field.
__global__ void __launch_bounds__(256, 5) k_defect_df(
    LvlD L, const float2* __restrict__ phi, const float2* __restrict__ mu,
    const float2* __restrict__ om, const float2* __restrict__ S1,
    const float2* __restrict__ S2, const float2* __restrict__ S3,
    const float2* __restrict__ b, float* __restrict__ r1, float* __restrict__ r2,
    float* __restrict__ r3, float* __restrict__ q, double* partials, float2* __restrict__ lap) {
  __shared__ float sm[32];
  const int n = L.n;
  const int cells = n * n * n;
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Nb6 s = nb6_at(t, i, j, k, n);
    const df p = df_ld(phi, t), bb = df_ld(b, t);
    // r1 = S1 - phi + tau/h^2 Lap mu
    dacc x = dacc_of(df_ld(S1, t));
    dacc_sub(x, p);
    const dacc tl = dacc_mul(L.tg, dacc_lap(mu, s, df_ld(mu, t)));
    dacc_add(x, tl.hi, tl.lo);
    // r2 = S2 - mu + f(phi, b) + (1-eps)/2 phi + 1/h^2 Lap om
    dacc y = dacc_of(df_ld(S2, t));
    dacc_sub(y, df_ld(mu, t));
    const dacc f = dacc_cubic(p, bb);
    dacc_add(y, f.hi, f.lo);
    const dacc cp = dacc_mul(L.c1, dacc_of(p));
    dacc_add(y, cp.hi, cp.lo);
    const dacc gl = dacc_mul(L.g, dacc_lap(om, s, df_ld(om, t)));
    dacc_add(y, gl.hi, gl.lo);
    // r3 = S3 - omega + 1/(2h^2) Lap phi
    dacc z = dacc_of(df_ld(S3, t));
    dacc_sub(z, df_ld(om, t));
    const dacc lphi = dacc_lap(phi, s, p);
    const dacc hl = dacc_mul(L.gh, lphi);
    dacc_add(z, hl.hi, hl.lo);
    if (lap) {
      df v;
      two_sum(lphi.hi, lphi.lo, v.hi, v.lo);
      df_st(lap, t, v);
    }
    const float xf = dacc_round(x), yf = dacc_round(y), zf = dacc_round(z);
    acc = fmaf(xf, xf, fmaf(yf, yf, fmaf(zf, zf, acc)));
    const int o = split_index(i, j, k, n);
    r1[o] = xf;
    r2[o] = yf;
    r3[o] = zf;
    const float pf = p.hi, bf = bb.hi;
    q[o] = fmaf(0.75f * pf, pf, fmaf(0.5f * pf, bf, fmaf(0.25f * bf, bf, L.c1f)));
  }
  acc = block_sum_f(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = (double)acc;
}

// S2 = (1-eps)/2 b + 3 Lap b - Lap c and S3 = Lap b / 2 (Eqs. 5.9-5.10) in
// double-float (S1 = b needs no work).
__global__ void k_source_df(LvlD L, const float2* __restrict__ b, const float2* __restrict__ c,
                            float2* __restrict__ S2, float2* __restrict__ S3) {
  const int n = L.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const Nb6 s = nb6_at(t, i, j, k, n);
  const df bb = df_ld(b, t);
  const df lb = df_mul(L.g, df_lap(b, s, bb));
  const df lc = df_mul(L.g, df_lap(c, s, df_ld(c, t)));
  df_st(S2, t, df_add(df_mul_f(lb, 3.f), df_sub(df_mul(L.c1, bb), lc)));
  df_st(S3, t, df_scale2(lb, 0.5f));
}

// Block-wide df sums of NV values into thread 0 (fixed order: deterministic).
template <int NV>
__device__ __forceinline__ void block_sum_df(df (&v)[NV], float2* sm /* 32 * NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    df x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df y;
      y.hi = __shfl_down_sync(0xffffffffu, x.hi, o);
      y.lo = __shfl_down_sync(0xffffffffu, x.lo, o);
      x = df_add(x, y);
    }
    if (lane == 0) sm[c * 32 + wid] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const float2 w = (lane < nw) ? sm[c * 32 + lane] : make_float2(0.f, 0.f);
      df x;
      x.hi = w.x;
      x.lo = w.y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        df y;
        y.hi = __shfl_down_sync(0xffffffffu, x.hi, o);
        y.lo = __shfl_down_sync(0xffffffffu, x.lo, o);
        x = df_add(x, y);
      }
      v[c] = x;
    }
  }
  __syncthreads();
}

// Raw per-cell sums of the energy F_h (Eq. 2.1), the modified energy and the
// mass of the df fields a = phi^k, b = phi^{k-1}, in double-float:
// sum a^4, sum a^2, sum |D a|^2 (as -(a, Lap a), summation by parts, Lemma
// 2.1), sum (Lap a)^2, sum |D(a-b)|^2 (forward faces), sum a.  One df partial
// per block and component.
__global__ void k_diagnostics_df(int n, const float2* __restrict__ a,
                                 const float2* __restrict__ b, float2* partials) {
  __shared__ float2 sm[32 * 6];
  const int cells = n * n * n;
  df acc[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) acc[c] = df{0.f, 0.f};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const int i = t % n, rr = t / n, j = rr % n, k = rr / n;
    const Nb6 s = nb6_at(t, i, j, k, n);
    const df x = df_ld(a, t);
    const df axp = df_ld(a, s.xp), ayp = df_ld(a, s.yp), azp = df_ld(a, s.zp);
    const df lap = df_sub(df_sum6(df_ld(a, s.xm), axp, df_ld(a, s.ym), ayp, df_ld(a, s.zm), azp),
                          df_mul_f(x, 6.f));
    const df y = df_sub(x, df_ld(b, t));
    const df ex = df_sub(df_sub(axp, df_ld(b, s.xp)), y);
    const df ey = df_sub(df_sub(ayp, df_ld(b, s.yp)), y);
    const df ez = df_sub(df_sub(azp, df_ld(b, s.zp)), y);
    const df x2 = df_sqr(x);
    acc[0] = df_add(acc[0], df_sqr(x2));
    acc[1] = df_add(acc[1], x2);
    acc[2] = df_sub(acc[2], df_mul(x, lap));
    acc[3] = df_add(acc[3], df_sqr(lap));
    acc[4] = df_add(acc[4], df_add(df_add(df_sqr(ex), df_sqr(ey)), df_sqr(ez)));
    acc[5] = df_add(acc[5], x);
  }
  block_sum_df<6>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) partials[blockIdx.x * 6 + c] = make_float2(acc[c].hi, acc[c].lo);
  }
}

// Fixed-order df sum of the block partials -> out[0..5] as doubles.
__global__ void k_reduce_df6(const float2* __restrict__ partials, int nparts, double* out) {
  __shared__ float2 sm[32 * 6];
  df acc[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) acc[c] = df{0.f, 0.f};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] = df_add(acc[c], df_ld(partials, p * 6 + c));
  }
  block_sum_df<6>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) out[c] = (double)acc[c].hi + (double)acc[c].lo;
  }
}

// k_source_df plus phi_g = 2 b - c and omega_g = (3 Lap b - Lap c)/2 of the
// extrapolated initial iterate, in double-float.
__global__ void k_source_guess_df(LvlD L, const float2* __restrict__ b,
                                  const float2* __restrict__ c, float2* __restrict__ S2,
                                  float2* __restrict__ S3, float2* __restrict__ phig,
                                  float2* __restrict__ omg) {
  const int n = L.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const Nb6 s = nb6_at(t, i, j, k, n);
  const df bb = df_ld(b, t), cc = df_ld(c, t);
  const df lb = df_mul(L.g, df_lap(b, s, bb));
  const df lc = df_mul(L.g, df_lap(c, s, cc));
  df_st(S2, t, df_add(df_mul_f(lb, 3.f), df_sub(df_mul(L.c1, bb), lc)));
  df_st(S3, t, df_scale2(lb, 0.5f));
  df_st(phig, t, df_sub(df_scale2(bb, 2.f), cc));
  df_st(omg, t, df_scale2(df_sub(df_mul_f(lb, 3.f), lc), 0.5f));
}

// mu_g = S2 + f(phi_g, b) + (1-eps)/2 phi_g + Lap omega_g in double-float.
__global__ void k_mu_guess_df(LvlD L, const float2* __restrict__ phig,
                              const float2* __restrict__ omg, const float2* __restrict__ b,
                              const float2* __restrict__ S2, float2* __restrict__ mug) {
  const int n = L.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const Nb6 s = nb6_at(t, i, j, k, n);
  const df p = df_ld(phig, t);
  dacc m = dacc_of(df_ld(S2, t));
  const dacc f = dacc_cubic(p, df_ld(b, t));
  dacc_add(m, f.hi, f.lo);
  const dacc cp = dacc_mul(L.c1, dacc_of(p));
  dacc_add(m, cp.hi, cp.lo);
  const dacc gl = dacc_mul(L.g, dacc_lap(omg, s, df_ld(omg, t)));
  dacc_add(m, gl.hi, gl.lo);
  df r;
  two_sum(m.hi, m.lo, r.hi, r.lo);
  df_st(mug, t, r);
}

// Unscaled 7-point Laplacian of a df field, as a df field.
__global__ void k_laplacian_df(int n, const float2* __restrict__ v, float2* __restrict__ lap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const dacc L = dacc_lap(v, nb6_at(t, i, j, k, n), df_ld(v, t));
  df r;
  two_sum(L.hi, L.lo, r.hi, r.lo);
  df_st(lap, t, r);
}

// k_source_df from the stored df Laplacians of b and c.
__global__ void k_source_cached_df(LvlD L, const float2* __restrict__ b,
                                   const float2* __restrict__ lapb,
                                   const float2* __restrict__ lapc, float2* __restrict__ S2,
                                   float2* __restrict__ S3) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)L.n * L.n * L.n) return;
  const int u = (int)t;
  const df lb = df_mul(L.g, df_ld(lapb, u));
  const df lc = df_mul(L.g, df_ld(lapc, u));
  df_st(S2, u, df_add(df_mul_f(lb, 3.f), df_sub(df_mul(L.c1, df_ld(b, u)), lc)));
  df_st(S3, u, df_scale2(lb, 0.5f));
}

// k_diagnostics_df from the stored df Laplacians of a and b (the face sum of
// |D(a-b)|^2 by summation by parts, Lemma 2.1).
__global__ void k_diagnostics_cached_df(int n, const float2* __restrict__ a,
                                        const float2* __restrict__ b,
                                        const float2* __restrict__ lapa,
                                        const float2* __restrict__ lapb, float2* partials) {
  __shared__ float2 sm[32 * 6];
  const int cells = n * n * n;
  df acc[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) acc[c] = df{0.f, 0.f};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += gridDim.x * blockDim.x) {
    const df x = df_ld(a, t), la = df_ld(lapa, t);
    const df y = df_sub(x, df_ld(b, t));
    const df x2 = df_sqr(x);
    acc[0] = df_add(acc[0], df_sqr(x2));
    acc[1] = df_add(acc[1], x2);
    acc[2] = df_sub(acc[2], df_mul(x, la));
    acc[3] = df_add(acc[3], df_sqr(la));
    acc[4] = df_sub(acc[4], df_mul(y, df_sub(la, df_ld(lapb, t))));
    acc[5] = df_add(acc[5], x);
  }
  block_sum_df<6>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) partials[blockIdx.x * 6 + c] = make_float2(acc[c].hi, acc[c].lo);
  }
}

// The integer-pipe conversions of the FP64 outer loop on whole arrays.
__global__ void k_round_f32(int64_t count, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) y[t] = d2f_rn(x[t]);
}

__global__ void k_widen_f64(int64_t count, const float* __restrict__ x, double* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) y[t] = f2d(x[t]);
}

// FP64 <-> df conversions of whole fields; in place allowed (each thread
// reads its 8 bytes before writing them).
__global__ void k_df_from_f64(int64_t count, const double* x, float2* y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const df v = df_from_double(x[t]);
  y[t] = make_float2(v.hi, v.lo);
}

__global__ void k_df_to_f64(int64_t count, const float2* y, double* x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  x[t] = df_to_double(y[t]);
}

// Fixed-order sum of each member's partials (one block per member): out[m].
__global__ void k_reduce1(const double* __restrict__ partials, int nparts, double* out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[32];
  const int m = blockIdx.x;
  partials += (size_t)m * nparts;
  double acc[1] = {0.0};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) acc[0] += partials[p];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) out[m] = acc[0];
}

// k_reduce1 for a single member followed by its convergence decision (the
// work of k_decide) in the same block: the sum in the same order, one launch
// fewer per residual.
__global__ void k_reduce1_decide(const double* __restrict__ partials, int nparts, double* out,
                                 DecideArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sm[32];
  double acc[1] = {0.0};
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) acc[0] += partials[p];
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) {
    out[0] = acc[0];
    int running = 0, failed = 0;
    decide_member(a.state[0], acc[0], a.inv_3n3, a.tol, a.max_iter, a.first, running, failed);
    if (a.use_handle) cudaGraphSetConditional(a.handle, (running && !failed) ? 1u : 0u);
  }
}

// The final reduction of a residual's block sums: with a decision to take
// (single member) the fused kernel, else k_reduce1.
cudaError_t launch_reduce1(bool pdl, const double* partials, int nparts, double* out,
                           int members, cudaStream_t st, const DecideArgs* da, bool* decided) {
  if (da && members == 1) {
    if (decided) *decided = true;
    return launch_ex(pdl, k_reduce1_decide, dim3(1), dim3(kReduceThreads), 0, st, partials,
                     nparts, out, *da);
  }
  if (decided) *decided = false;
  return launch_ex(pdl, k_reduce1, dim3(members), dim3(kReduceThreads), 0, st, partials, nparts,
                   out);
}

// 8-cell average of a split-layout field onto the (split-layout) level n/2.
__global__ void k_restrict32(int n, const float* __restrict__ f, float* __restrict__ c) {
  pdl_wait();
  pdl_trigger();
  const int nc = n >> 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  int K = blockIdx.z;
  const int m = member_of(K, nc);
  if (I >= nc || J >= nc) return;
  f += (size_t)m * n * n * n;
  c += (size_t)m * nc * nc * nc;
  float acc = 0.f;
#pragma unroll
  for (int s = 0; s < 8; ++s)
    acc += __ldg(f + split_index(2 * I + (s & 1), 2 * J + ((s >> 1) & 1), 2 * K + (s >> 2), n));
  c[split_index(I, J, K, nc)] = 0.125f * acc;
}

// Pointwise solve of the linearised 3x3 system (q frozen):
//   [ 1   kap  0  ] [dp]   [r1 + tau/h^2 sum d_mu]
//   [ -q  1    6g ] [dm] = [r2 + g sum d_om      ]
//   [ 3g  0    1  ] [dw]   [r3 + g/2 sum d_phi   ]
__device__ __forceinline__ void lin_point(const LvlF& L, float sp, float sm_, float sw,
                                          float q, float r1, float r2, float r3,
                                          float& dp, float& dm, float& dw) {
  const float st1 = fmaf(L.tg, sm_, r1);
  const float st2 = fmaf(L.g, sw, r2);
  const float st3 = fmaf(L.gh, sp, r3);
  const float Q = q + L.Q0;
  const float det = fmaf(L.kap, Q, 1.0f);
  // the division by the 2x2 determinant within 2 ulp (__fdividef): an FP32
  // preconditioner step, and the IEEE division was a fifth of the sweep's
  // instructions
  dm = __fdividef(fmaf(Q, st1, fmaf(-L.g6, st3, st2)), det);
  dp = fmaf(-L.kap, dm, st1);
  dw = fmaf(-L.g3, dp, st3);
}

// One colour of a linear red-black sweep on split-layout fields: thread t
// owns the t-th cell of the colour, so the colour's cells are read and
// written as contiguous runs.  ZERO: d = 0 everywhere before this half-sweep
// (first red pass from d = 0), so no neighbour is read.
template <bool ZERO>
__global__ void k_lin_smooth32(LvlF L, int colour, float* d1, float* d2, float* d3,
                               const float* __restrict__ r1, const float* __restrict__ r2,
                               const float* __restrict__ r3, const float* __restrict__ q) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, half = n >> 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (p >= half || j >= n) return;
  d1 += off, d2 += off, d3 += off, r1 += off, r2 += off, r3 += off, q += off;
  const Stencil s = split_stencil(p, j, k, colour, n);
  float sp = 0.f, sm_ = 0.f, sw = 0.f;
  if (!ZERO) {
    sp = nbsum(d1, s);
    sm_ = nbsum(d2, s);
    sw = nbsum(d3, s);
  }
  float dp, dm, dw;
  lin_point(L, sp, sm_, sw, __ldg(q + s.c), __ldg(r1 + s.c), __ldg(r2 + s.c),
            __ldg(r3 + s.c), dp, dm, dw);
  d1[s.c] = dp;
  d2[s.c] = dm;
  d3[s.c] = dw;
}

// The same colour pass with two adjacent cells of the colour's half-row per
// thread (positions p0 = 2t and p0 + 1; n a multiple of 4, so every pair is
// 8-byte aligned): own r, q, the y and z neighbours and the results move as
// float2, and the pair's x neighbours in the other half are that half's
// pair (p0, p0 + 1) plus one cell on the side the colour's offset sigma =
// (j + k + colour) & 1 points to.  Same sums in the same order as above.
template <bool ZERO>
__global__ void k_lin_smooth32x2(LvlF L, int colour, float* d1, float* d2, float* d3,
                                 const float* __restrict__ r1, const float* __restrict__ r2,
                                 const float* __restrict__ r3, const float* __restrict__ q) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, half = n >> 1;
  const int p0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (p0 >= half || j >= n) return;
  d1 += off, d2 += off, d3 += off, r1 += off, r2 += off, r3 += off, q += off;
  const int sigma = (j + k + colour) & 1;
  const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
  const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
  const int oc = (1 - colour) * half;
  const int row = (k * n + j) * n;
  const int c = row + colour * half + p0;                // own pair
  const int xo = row + oc + p0;                          // other half, same positions
  int xe = sigma ? p0 + 2 : p0 - 1;                      // the extra x neighbour
  if (xe < 0) xe += half;
  if (xe >= half) xe -= half;
  xe += row + oc;
  const int ym = (k * n + jm) * n + oc + p0, yp = (k * n + jp) * n + oc + p0;
  const int zm = (km * n + j) * n + oc + p0, zp = (kp * n + j) * n + oc + p0;
  float s0[2] = {0.f, 0.f}, s1[2] = {0.f, 0.f}, s2[2] = {0.f, 0.f};
  if (!ZERO) {
    const float* f[3] = {d1, d2, d3};
    float* acc[3] = {s0, s1, s2};
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3) {
      const float* v = f[q3];
      const float2 a = __ldg(reinterpret_cast<const float2*>(v + xo));
      const float e = __ldg(v + xe);
      const float2 y0 = __ldg(reinterpret_cast<const float2*>(v + ym));
      const float2 y1 = __ldg(reinterpret_cast<const float2*>(v + yp));
      const float2 z0 = __ldg(reinterpret_cast<const float2*>(v + zm));
      const float2 z1 = __ldg(reinterpret_cast<const float2*>(v + zp));
      // cell p0: (xm, xp) = sigma ? (a.x, a.y) : (e, a.x); cell p0+1: sigma ? (a.y, e) : (a.x, a.y)
      const float xm0 = sigma ? a.x : e, xp0 = sigma ? a.y : a.x;
      const float xm1 = sigma ? a.y : a.x, xp1 = sigma ? e : a.y;
      acc[q3][0] = ((xm0 + xp0) + (y0.x + y1.x)) + (z0.x + z1.x);
      acc[q3][1] = ((xm1 + xp1) + (y0.y + y1.y)) + (z0.y + z1.y);
    }
  }
  const float2 qq = __ldg(reinterpret_cast<const float2*>(q + c));
  const float2 ra = __ldg(reinterpret_cast<const float2*>(r1 + c));
  const float2 rb = __ldg(reinterpret_cast<const float2*>(r2 + c));
  const float2 rc = __ldg(reinterpret_cast<const float2*>(r3 + c));
  float2 dp, dm, dw;
  lin_point(L, s0[0], s1[0], s2[0], qq.x, ra.x, rb.x, rc.x, dp.x, dm.x, dw.x);
  lin_point(L, s0[1], s1[1], s2[1], qq.y, ra.y, rb.y, rc.y, dp.y, dm.y, dw.y);
  *reinterpret_cast<float2*>(d1 + c) = dp;
  *reinterpret_cast<float2*>(d2 + c) = dm;
  *reinterpret_cast<float2*>(d3 + c) = dw;
}

// One damped collective Jacobi sweep on J d = r, d -> t (split layout).
// ZERO: d = 0 on entry (nothing is read from d).
template <bool ZERO>
__global__ void k_lin_jacobi32(LvlF L, float w, const float* __restrict__ d1,
                               const float* __restrict__ d2, const float* __restrict__ d3,
                               float* __restrict__ t1, float* __restrict__ t2,
                               float* __restrict__ t3, const float* __restrict__ r1,
                               const float* __restrict__ r2, const float* __restrict__ r3,
                               const float* __restrict__ q) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, half = n >> 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (x >= n || j >= n) return;
  d1 += off, d2 += off, d3 += off, t1 += off, t2 += off, t3 += off;
  r1 += off, r2 += off, r3 += off, q += off;
  const int colour = x >= half;
  const Stencil s = split_stencil(x - colour * half, j, k, colour, n);
  float sp = 0.f, sm_ = 0.f, sw = 0.f, p0 = 0.f, m0 = 0.f, w0 = 0.f;
  if (!ZERO) {
    sp = nbsum(d1, s);
    sm_ = nbsum(d2, s);
    sw = nbsum(d3, s);
    p0 = __ldg(d1 + s.c);
    m0 = __ldg(d2 + s.c);
    w0 = __ldg(d3 + s.c);
  }
  float dp, dm, dw;
  lin_point(L, sp, sm_, sw, __ldg(q + s.c), __ldg(r1 + s.c), __ldg(r2 + s.c),
            __ldg(r3 + s.c), dp, dm, dw);
  t1[s.c] = fmaf(w, dp - p0, p0);
  t2[s.c] = fmaf(w, dm - m0, m0);
  t3[s.c] = fmaf(w, dw - w0, w0);
}


// The same sweep with two adjacent cells of one half-row per thread (n a
// multiple of 4): the neighbour pattern of k_lin_smooth32x2 for the pair's
// colour, own d, r, q and the results as float2.
template <bool ZERO>
__global__ void k_lin_jacobi32x2(LvlF L, float w, const float* __restrict__ d1,
                                 const float* __restrict__ d2, const float* __restrict__ d3,
                                 float* __restrict__ t1, float* __restrict__ t2,
                                 float* __restrict__ t3, const float* __restrict__ r1,
                                 const float* __restrict__ r2, const float* __restrict__ r3,
                                 const float* __restrict__ q) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, half = n >> 1;
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (x >= n || j >= n) return;
  d1 += off, d2 += off, d3 += off, t1 += off, t2 += off, t3 += off;
  r1 += off, r2 += off, r3 += off, q += off;
  const int colour = x >= half, p0 = x - colour * half;
  const int sigma = (j + k + colour) & 1;
  const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
  const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
  const int oc = (1 - colour) * half;
  const int row = (k * n + j) * n;
  const int c = row + colour * half + p0;
  const int xo = row + oc + p0;
  int xe = sigma ? p0 + 2 : p0 - 1;
  if (xe < 0) xe += half;
  if (xe >= half) xe -= half;
  xe += row + oc;
  const int ym = (k * n + jm) * n + oc + p0, yp = (k * n + jp) * n + oc + p0;
  const int zm = (km * n + j) * n + oc + p0, zp = (kp * n + j) * n + oc + p0;
  float s0[2] = {0.f, 0.f}, s1[2] = {0.f, 0.f}, s2[2] = {0.f, 0.f};
  float2 o0 = make_float2(0.f, 0.f), o1 = o0, o2 = o0;
  if (!ZERO) {
    const float* f[3] = {d1, d2, d3};
    float* acc[3] = {s0, s1, s2};
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3) {
      const float* v = f[q3];
      const float2 a = __ldg(reinterpret_cast<const float2*>(v + xo));
      const float e = __ldg(v + xe);
      const float2 y0 = __ldg(reinterpret_cast<const float2*>(v + ym));
      const float2 y1 = __ldg(reinterpret_cast<const float2*>(v + yp));
      const float2 z0 = __ldg(reinterpret_cast<const float2*>(v + zm));
      const float2 z1 = __ldg(reinterpret_cast<const float2*>(v + zp));
      const float xm0 = sigma ? a.x : e, xp0 = sigma ? a.y : a.x;
      const float xm1 = sigma ? a.y : a.x, xp1 = sigma ? e : a.y;
      acc[q3][0] = ((xm0 + xp0) + (y0.x + y1.x)) + (z0.x + z1.x);
      acc[q3][1] = ((xm1 + xp1) + (y0.y + y1.y)) + (z0.y + z1.y);
    }
    o0 = __ldg(reinterpret_cast<const float2*>(d1 + c));
    o1 = __ldg(reinterpret_cast<const float2*>(d2 + c));
    o2 = __ldg(reinterpret_cast<const float2*>(d3 + c));
  }
  const float2 qq = __ldg(reinterpret_cast<const float2*>(q + c));
  const float2 ra = __ldg(reinterpret_cast<const float2*>(r1 + c));
  const float2 rb = __ldg(reinterpret_cast<const float2*>(r2 + c));
  const float2 rc = __ldg(reinterpret_cast<const float2*>(r3 + c));
  float2 dp, dm, dw;
  lin_point(L, s0[0], s1[0], s2[0], qq.x, ra.x, rb.x, rc.x, dp.x, dm.x, dw.x);
  lin_point(L, s0[1], s1[1], s2[1], qq.y, ra.y, rb.y, rc.y, dp.y, dm.y, dw.y);
  *reinterpret_cast<float2*>(t1 + c) =
      make_float2(fmaf(w, dp.x - o0.x, o0.x), fmaf(w, dp.y - o0.y, o0.y));
  *reinterpret_cast<float2*>(t2 + c) =
      make_float2(fmaf(w, dm.x - o1.x, o1.x), fmaf(w, dm.y - o1.y, o1.y));
  *reinterpret_cast<float2*>(t3 + c) =
      make_float2(fmaf(w, dw.x - o2.x, o2.x), fmaf(w, dw.y - o2.y, o2.y));
}

// The colour-1 pass of k_lin_smooth32x2 with the defect correction u += d
// folded in, for the last pass of a correction's last V-cycle on the finest
// level: d is not needed after it, so the pass adds its new colour-1 values
// and the colour-0 values it reads as x neighbours to the FP64 state instead
// of storing them.  A thread's pair of colour-1 cells and the two colour-0
// cells at the same positions of the other half are the four consecutive
// natural cells 2 p0 .. 2 p0 + 3 of the row (which of each pair comes first
// depends on the row's colour offset), so u moves as two 16-byte vectors per
// component.  Same sums and solve as the pass, same u + f2d(d) as
// k_correct64: u equals the two launches bit for bit.  d's colour-1 cells
// are left as they were.
__global__ void k_lin_smooth32x2_correct(LvlF L, const float* __restrict__ d1,
                                         const float* __restrict__ d2,
                                         const float* __restrict__ d3,
                                         const float* __restrict__ r1,
                                         const float* __restrict__ r2,
                                         const float* __restrict__ r3,
                                         const float* __restrict__ q, double* __restrict__ u1,
                                         double* __restrict__ u2, double* __restrict__ u3) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, half = n >> 1;
  const int p0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (p0 >= half || j >= n) return;
  d1 += off, d2 += off, d3 += off, r1 += off, r2 += off, r3 += off, q += off;
  u1 += off, u2 += off, u3 += off;
  const int sigma = (j + k + 1) & 1;                     // colour 1
  const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
  const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
  const int row = (k * n + j) * n;
  const int c = row + half + p0;                         // own pair
  const int xo = row + p0;                               // colour 0, same positions
  int xe = sigma ? p0 + 2 : p0 - 1;
  if (xe < 0) xe += half;
  if (xe >= half) xe -= half;
  xe += row;
  const int ym = (k * n + jm) * n + p0, yp = (k * n + jp) * n + p0;
  const int zm = (km * n + j) * n + p0, zp = (kp * n + j) * n + p0;
  float s[3][2];
  float2 a[3];
  const float* const f[3] = {d1, d2, d3};
#pragma unroll
  for (int q3 = 0; q3 < 3; ++q3) {
    const float* v = f[q3];
    a[q3] = __ldg(reinterpret_cast<const float2*>(v + xo));
    const float e = __ldg(v + xe);
    const float2 y0 = __ldg(reinterpret_cast<const float2*>(v + ym));
    const float2 y1 = __ldg(reinterpret_cast<const float2*>(v + yp));
    const float2 z0 = __ldg(reinterpret_cast<const float2*>(v + zm));
    const float2 z1 = __ldg(reinterpret_cast<const float2*>(v + zp));
    const float xm0 = sigma ? a[q3].x : e, xp0 = sigma ? a[q3].y : a[q3].x;
    const float xm1 = sigma ? a[q3].y : a[q3].x, xp1 = sigma ? e : a[q3].y;
    s[q3][0] = ((xm0 + xp0) + (y0.x + y1.x)) + (z0.x + z1.x);
    s[q3][1] = ((xm1 + xp1) + (y0.y + y1.y)) + (z0.y + z1.y);
  }
  const float2 qq = __ldg(reinterpret_cast<const float2*>(q + c));
  const float2 ra = __ldg(reinterpret_cast<const float2*>(r1 + c));
  const float2 rb = __ldg(reinterpret_cast<const float2*>(r2 + c));
  const float2 rc = __ldg(reinterpret_cast<const float2*>(r3 + c));
  float2 nd[3];
  lin_point(L, s[0][0], s[1][0], s[2][0], qq.x, ra.x, rb.x, rc.x, nd[0].x, nd[1].x, nd[2].x);
  lin_point(L, s[0][1], s[1][1], s[2][1], qq.y, ra.y, rb.y, rc.y, nd[0].y, nd[1].y, nd[2].y);
  double* const u[3] = {u1, u2, u3};
#pragma unroll
  for (int q3 = 0; q3 < 3; ++q3) {
    // natural order 2 p0 .. 2 p0 + 3: colour 1 first when sigma = 0
    const float v0 = sigma ? a[q3].x : nd[q3].x, v1 = sigma ? nd[q3].x : a[q3].x;
    const float v2 = sigma ? a[q3].y : nd[q3].y, v3 = sigma ? nd[q3].y : a[q3].y;
    double2* const up = reinterpret_cast<double2*>(u[q3] + row + 2 * p0);
    double2 lo = up[0], hi = up[1];
    lo.x += f2d(v0);
    lo.y += f2d(v1);
    hi.x += f2d(v2);
    hi.y += f2d(v3);
    up[0] = lo;
    up[1] = hi;
  }
}

__global__ void k_copy3(int cells, const float* __restrict__ a1, const float* __restrict__ a2,
                        const float* __restrict__ a3, float* __restrict__ b1,
                        float* __restrict__ b2, float* __restrict__ b3) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cells) return;
  b1[t] = a1[t];
  b2[t] = a2[t];
  b3[t] = a3[t];
}

// rho = r - J d at the 8 children of each coarse cell, averaged (split layout
// on both levels).
// Fine split-layout indices of the eight children of coarse cell (I, J, K)
// (in[8]: per fine row of the 2x2x2 block, the two cells at position I of
// the two colour halves) and of the 24 face neighbours of the block outside
// it (out[24]).  Cell (i, j, k) of the split layout sits in the half of
// colour (i+j+k)&1 at position i/2 of its row; n even.
__device__ __forceinline__ void block_indices(int I, int J, int K, int n, int (&in)[8],
                                              int (&out)[24]) {
  const int half = n >> 1;
  const int j0 = 2 * J, k0 = 2 * K;
  const int jm = (j0 == 0) ? n - 1 : j0 - 1, jp = (j0 + 2 == n) ? 0 : j0 + 2;
  const int km = (k0 == 0) ? n - 1 : k0 - 1, kp = (k0 + 2 == n) ? 0 : k0 + 2;
  const int Im = (I == 0) ? half - 1 : I - 1, Ip = (I + 1 == half) ? 0 : I + 1;
  int o = 0;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int j = j0 + jj, k = k0 + kk;
      const int rw = (k * n + j) * n, par = (j + k) & 1;
      in[2 * (2 * kk + jj)] = rw + I;
      in[2 * (2 * kk + jj) + 1] = rw + half + I;
      out[o++] = rw + (1 - par) * half + Im;   // (2I-1, j, k)
      out[o++] = rw + par * half + Ip;         // (2I+2, j, k)
    }
  }
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = k0 + kk;
    out[o++] = (k * n + jm) * n + I;           // (2I and 2I+1, j0-1, k)
    out[o++] = (k * n + jm) * n + half + I;
    out[o++] = (k * n + jp) * n + I;           // (2I and 2I+1, j0+2, k)
    out[o++] = (k * n + jp) * n + half + I;
  }
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    const int j = j0 + jj;
    out[o++] = (km * n + j) * n + I;           // (2I and 2I+1, j, k0-1)
    out[o++] = (km * n + j) * n + half + I;
    out[o++] = (kp * n + j) * n + I;           // (2I and 2I+1, j, k0+2)
    out[o++] = (kp * n + j) * n + half + I;
  }
}

// Restricted residual of the linear system: the average over the eight
// children of r - J d, with
//   (J d)1 = d_phi - tau/h^2 Lap d_mu
//   (J d)2 = d_mu - q d_phi - 1/h^2 Lap d_om
//   (J d)3 = d_om - 1/(2h^2) Lap d_phi,
// the averaged Laplacians taken from block sums (summed over the children,
// the 7-point Laplacian's interior faces cancel: sum_children Lap v = s_out -
// 3 s_in, unscaled, with s_in the sum over the eight children and s_out over
// the 24 outside face neighbours) and q d_phi summed cell by cell.  One thread per coarse cell forms all three rows: each of
// d_phi, d_mu, d_om enters one row through its children and another through
// its block sum, so its eight children are loaded once for both (and those
// of d_phi a third time for q d_phi), 128 loads per coarse cell where one
// thread per row needed 160, and every field of a plane is read by the same
// threads.  The sums are formed in the same order as one thread per row did.
// ZERO: d = 0 on entry (no pre-smoothing from a zero start), so rho = r and d
// and q are not read.
template <bool ZERO>
__global__ void k_lin_residual_restrict32(LvlF L, const float* __restrict__ d1,
                                          const float* __restrict__ d2,
                                          const float* __restrict__ d3,
                                          const float* __restrict__ r1,
                                          const float* __restrict__ r2,
                                          const float* __restrict__ r3,
                                          const float* __restrict__ q,
                                          float* __restrict__ c1, float* __restrict__ c2,
                                          float* __restrict__ c3) {
  pdl_wait();
  pdl_trigger();
  const int n = L.n, nc = n >> 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  int K = blockIdx.z;
  const int m = member_of(K, nc);
  if (I >= nc || J >= nc) return;
  const size_t off = (size_t)m * n * n * n, offc = (size_t)m * nc * nc * nc;
  int in[8], out[24];
  block_indices(I, J, K, n, in, out);
  const float* const rr[3] = {r1 + off, r2 + off, r3 + off};
  float a[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += __ldg(rr[f] + in[c]);
    a[f] = s;
  }
  if (!ZERO) {
    const float* const dd[3] = {d1 + off, d2 + off, d3 + off};
    float sin[3], sout[3], p1[8];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      float si = 0.f, so = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float v = __ldg(dd[f] + in[c]);
        if (f == 0) p1[c] = v;
        si += v;
      }
#pragma unroll
      for (int c = 0; c < 24; ++c) so += __ldg(dd[f] + out[c]);
      sin[f] = si;
      sout[f] = so;
    }
    float qp = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) qp = fmaf(__ldg(q + off + in[c]), p1[c], qp);
    // row f: own d_f, the field under the Laplacian (d_mu, d_om, d_phi)
    a[0] = fmaf(L.tg, fmaf(-3.f, sin[1], sout[1]), a[0] - sin[0]);
    a[1] = fmaf(L.g, fmaf(-3.f, sin[2], sout[2]), a[1] - sin[1]) + qp;
    a[2] = fmaf(L.gh, fmaf(-3.f, sin[0], sout[0]), a[2] - sin[2]);
  }
  const int ci = split_index(I, J, K, nc);
  (c1 + offc)[ci] = 0.125f * a[0];
  (c2 + offc)[ci] = 0.125f * a[1];
  (c3 + offc)[ci] = 0.125f * a[2];
}

// The restriction of k_lin_residual_restrict32 followed by EXTRA more
// levels of plain 8-cell averages, in one launch.  Without pre-smoothing
// (nu1 = 0) every coarser level starts its V-cycle from d = 0, so its own
// restriction is the average of its r alone; a block of kChTX x kChTY x kChTZ
// coarse cells keeps its results in shared memory and averages them down to
// (kChTX/2 x kChTY/2 x kChTZ/2) and (kChTX/4 x kChTY/4 x kChTZ/4) cells, in
// the children order of the separate kernel (bit-identical results), and
// each coarser level's separate launch goes.  Coarse size nc a multiple of
// kChTX and kChTZ.
constexpr int kChTX = 16, kChTY = 4, kChTZ = 4;

template <bool ZERO, int EXTRA>
__global__ void __launch_bounds__(kChTX * kChTY * kChTZ) k_lin_restrict_chain32(
    LvlF L, const float* __restrict__ d1, const float* __restrict__ d2,
    const float* __restrict__ d3, const float* __restrict__ r1, const float* __restrict__ r2,
    const float* __restrict__ r3, const float* __restrict__ q, float* __restrict__ c1,
    float* __restrict__ c2, float* __restrict__ c3, float* __restrict__ e1,
    float* __restrict__ e2, float* __restrict__ e3, float* __restrict__ g1,
    float* __restrict__ g2, float* __restrict__ g3) {
  pdl_wait();
  pdl_trigger();
  __shared__ float s1[3][kChTZ][kChTY][kChTX];
  __shared__ float s2[3][kChTZ / 2][kChTY / 2][kChTX / 2];
  const int n = L.n, nc = n >> 1;
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int I = blockIdx.x * kChTX + tx, J = blockIdx.y * kChTY + ty;
  int K = blockIdx.z * kChTZ + tz;
  const int m = member_of(K, nc);
  const size_t off = (size_t)m * n * n * n, offc = (size_t)m * nc * nc * nc;
  int in[8], out[24];
  block_indices(I, J, K, n, in, out);
  const float* const rr[3] = {r1 + off, r2 + off, r3 + off};
  float a[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += __ldg(rr[f] + in[c]);
    a[f] = s;
  }
  if (!ZERO) {
    const float* const dd[3] = {d1 + off, d2 + off, d3 + off};
    float sin[3], sout[3], p1[8];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      float si = 0.f, so = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float v = __ldg(dd[f] + in[c]);
        if (f == 0) p1[c] = v;
        si += v;
      }
#pragma unroll
      for (int c = 0; c < 24; ++c) so += __ldg(dd[f] + out[c]);
      sin[f] = si;
      sout[f] = so;
    }
    float qp = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) qp = fmaf(__ldg(q + off + in[c]), p1[c], qp);
    a[0] = fmaf(L.tg, fmaf(-3.f, sin[1], sout[1]), a[0] - sin[0]);
    a[1] = fmaf(L.g, fmaf(-3.f, sin[2], sout[2]), a[1] - sin[1]) + qp;
    a[2] = fmaf(L.gh, fmaf(-3.f, sin[0], sout[0]), a[2] - sin[2]);
  }
  float* const cc[3] = {c1 + offc, c2 + offc, c3 + offc};
  const int ci = split_index(I, J, K, nc);
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float v = 0.125f * a[f];
    cc[f][ci] = v;
    if (EXTRA > 0) s1[f][tz][ty][tx] = v;
  }
  if (EXTRA == 0) return;
  // averages of the block's cells: children in the order of block_indices
  // (for each child row, the cell of colour half 0 first)
  const int tid = (tz * kChTY + ty) * kChTX + tx;
  const int n2 = nc >> 1;
  const size_t off2 = (size_t)m * n2 * n2 * n2;
  __syncthreads();
  if (tid < (kChTX / 2) * (kChTY / 2) * (kChTZ / 2)) {
    const int x = tid % (kChTX / 2), y = (tid / (kChTX / 2)) % (kChTY / 2),
              z = tid / ((kChTX / 2) * (kChTY / 2));
    float* const ee[3] = {e1 + off2, e2 + off2, e3 + off2};
    const int I2 = blockIdx.x * (kChTX / 2) + x, J2 = blockIdx.y * (kChTY / 2) + y;
    const int K2g = (K - tz) / 2 + z;            // plane within this member's level
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      float sum = 0.f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int par = (jj + kk) & 1;
          sum += s1[f][2 * z + kk][2 * y + jj][2 * x + par];
          sum += s1[f][2 * z + kk][2 * y + jj][2 * x + 1 - par];
        }
      const float v = 0.125f * sum;
      ee[f][split_index(I2, J2, K2g, n2)] = v;
      if (EXTRA > 1) s2[f][z][y][x] = v;
    }
  }
  if (EXTRA < 2) return;
  __syncthreads();
  const int n3 = n2 >> 1;
  const size_t off3 = (size_t)m * n3 * n3 * n3;
  if (tid < (kChTX / 4) * (kChTY / 4) * (kChTZ / 4)) {
    const int x = tid % (kChTX / 4), y = (tid / (kChTX / 4)) % (kChTY / 4),
              z = tid / ((kChTX / 4) * (kChTY / 4));
    float* const gg[3] = {g1 + off3, g2 + off3, g3 + off3};
    const int I3 = blockIdx.x * (kChTX / 4) + x, J3 = blockIdx.y * (kChTY / 4) + y;
    const int K3g = (K - tz) / 4 + z;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      float sum = 0.f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int par = (jj + kk) & 1;
          sum += s2[f][2 * z + kk][2 * y + jj][2 * x + par];
          sum += s2[f][2 * z + kk][2 * y + jj][2 * x + 1 - par];
        }
      gg[f][split_index(I3, J3, K3g, n3)] = 0.125f * sum;
    }
  }
}

// q restricted down up to EXTRA + 1 levels in one launch: a block of kChTX x
// kChTY x kChTZ cells of the first coarse level averages their 8 children
// (the children order of k_restrict32), keeps its averages in shared memory
// and averages them down to (kChTX/2 x kChTY/2 x kChTZ/2) and then
// (kChTX/4 x kChTY/4 x kChTZ/4) cells in the same order: bit-identical to
// EXTRA + 1 launches of k_restrict32.  First coarse size a multiple of kChTX
// and kChTZ.
template <int EXTRA>
__global__ void __launch_bounds__(kChTX * kChTY * kChTZ) k_restrict_chain32(
    int n, const float* __restrict__ f, float* __restrict__ c, float* __restrict__ e,
    float* __restrict__ g) {
  pdl_wait();
  pdl_trigger();
  __shared__ float s1[kChTZ][kChTY][kChTX];
  __shared__ float s2[kChTZ / 2][kChTY / 2][kChTX / 2];
  const int nc = n >> 1;
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int I = blockIdx.x * kChTX + tx, J = blockIdx.y * kChTY + ty;
  int K = blockIdx.z * kChTZ + tz;
  const int m = member_of(K, nc);
  f += (size_t)m * n * n * n;
  float acc = 0.f;
#pragma unroll
  for (int s = 0; s < 8; ++s)
    acc += __ldg(f + split_index(2 * I + (s & 1), 2 * J + ((s >> 1) & 1), 2 * K + (s >> 2), n));
  const float v = 0.125f * acc;
  c[(size_t)m * nc * nc * nc + split_index(I, J, K, nc)] = v;
  if (EXTRA == 0) return;
  s1[tz][ty][tx] = v;
  __syncthreads();
  const int tid = (tz * kChTY + ty) * kChTX + tx;
  const int n2 = nc >> 1;
  if (tid < (kChTX / 2) * (kChTY / 2) * (kChTZ / 2)) {
    const int x = tid % (kChTX / 2), y = (tid / (kChTX / 2)) % (kChTY / 2),
              z = tid / ((kChTX / 2) * (kChTY / 2));
    float a2 = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) a2 += s1[2 * z + (s >> 2)][2 * y + ((s >> 1) & 1)][2 * x + (s & 1)];
    const float v2 = 0.125f * a2;
    const int I2 = blockIdx.x * (kChTX / 2) + x, J2 = blockIdx.y * (kChTY / 2) + y;
    const int K2 = (K - tz) / 2 + z;
    e[(size_t)m * n2 * n2 * n2 + split_index(I2, J2, K2, n2)] = v2;
    if (EXTRA > 1) s2[z][y][x] = v2;
  }
  if (EXTRA < 2) return;
  __syncthreads();
  const int n3 = n2 >> 1;
  if (tid < (kChTX / 4) * (kChTY / 4) * (kChTZ / 4)) {
    const int x = tid % (kChTX / 4), y = (tid / (kChTX / 4)) % (kChTY / 4),
              z = tid / ((kChTX / 4) * (kChTY / 4));
    float a3 = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) a3 += s2[2 * z + (s >> 2)][2 * y + ((s >> 1) & 1)][2 * x + (s & 1)];
    const int I3 = blockIdx.x * (kChTX / 4) + x, J3 = blockIdx.y * (kChTY / 4) + y;
    const int K3 = (K - tz) / 4 + z;
    g[(size_t)m * n3 * n3 * n3 + split_index(I3, J3, K3, n3)] = 0.125f * a3;
  }
}

// d += P e (ASSIGN: d = P e; d was zero and is not read), trilinear
// cell-centred prolongation with the weights 27, 9, 3, 1 over 64 as three
// one-dimensional passes: the child on the low side of an axis takes
// (3 e_0 + e_-1)/4, on the high side (3 e_0 + e_+1)/4.  Split layout on both
// levels.  A block of kPrTI x kPrTJ threads owns that tile of coarse cells
// over `zc` (<= kPrZ) consecutive planes K0.. of one component (the grid's z
// extent covers plane chunks x components x members): it stages the tile's
// neighbourhood (one-cell periodic halo, planes K0-1..K0+zc) in shared
// memory in natural order with one load per value, then each thread writes
// its coarse cells' eight children from there, plane after plane.  The
// children's current values are loaded before the staging, so those loads,
// the staging and the stores of the earlier planes overlap.
//
// SKIP0: the children of colour 0 (the first half of each fine row) are
// neither read nor written.  A red-black pass of colour 0 that follows
// recomputes every colour-0 cell from its colour-1 neighbours alone (the
// pointwise 3x3 solve does not read the cell's own value), so the values the
// prolongation would put there are never used: the pass sees the same inputs
// either way, and half of the fine-level traffic of the prolongation goes.
constexpr int kPrTI = 32, kPrTJ = 4, kPrZ = 8;

template <bool ASSIGN, bool SKIP0>
__global__ void __launch_bounds__(kPrTI * kPrTJ) k_prolong_add32(
    int n, int zc, const float* __restrict__ e1, const float* __restrict__ e2,
    const float* __restrict__ e3, float* __restrict__ d1, float* __restrict__ d2,
    float* __restrict__ d3) {
  pdl_wait();
  pdl_trigger();
  constexpr int kW = kPrTI + 2;
  __shared__ float sh[kPrZ + 2][kPrTJ + 2][kW];
  const int nc = n >> 1, half = n >> 1, hc = nc >> 1;
  const int chunks = (nc + zc - 1) / zc;
  int kb = blockIdx.z;
  const int mf = member_of(kb, chunks);      // member * 3 + component
  const int m = mf / 3, f = mf - 3 * m;
  const int K0 = kb * zc, nz = min(zc, nc - K0);
  const float* __restrict__ e = (f == 0 ? e1 : f == 1 ? e2 : e3) + (size_t)m * nc * nc * nc;
  float* __restrict__ d = (f == 0 ? d1 : f == 1 ? d2 : d3) + (size_t)m * n * n * n;
  const int I0 = blockIdx.x * kPrTI, J0 = blockIdx.y * kPrTJ;
  const int tx = threadIdx.x % kPrTI, ty = threadIdx.x / kPrTI;
  const int I = I0 + tx, J = J0 + ty;
  const bool own = I < nc && J < nc;
  // the children's current values first: old[z][(2 kk + jj) * 2 + a]
  float old[kPrZ][8];
#pragma unroll
  for (int z = 0; z < kPrZ; ++z)
#pragma unroll
    for (int c = 0; c < 8; ++c) old[z][c] = 0.f;
  if (!ASSIGN && own) {
#pragma unroll
    for (int z = 0; z < kPrZ; ++z) {
      if (z < nz) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * J + jj, k = 2 * (K0 + z) + kk;
            const int row = (k * n + j) * n + I, par = (jj + kk) & 1;   // (j + k) & 1
            if (!SKIP0 || par == 1) old[z][(2 * kk + jj) * 2] = d[row + par * half];
            if (!SKIP0 || par == 0) old[z][(2 * kk + jj) * 2 + 1] = d[row + (1 - par) * half];
          }
      }
    }
  }
  // staging: each thread loads its own column (x, y) = (tx + 1, ty + 1) of
  // the tile and the first kHalo threads one cell of the halo ring each, on
  // every plane; the periodic wraps (more than one when nc < kPrTI) and the
  // column offsets are worked out once, so a load costs an add and a select.
  // All loads are issued before any of them is stored, so a block waits for
  // one L2 round trip here instead of one per load.
  {
    constexpr int kHalo = 2 * kW + 2 * kPrTJ;
    static_assert(kHalo <= kPrTI * kPrTJ, "one halo cell per thread at most");
    const int t = threadIdx.x;
    int hx = 0, hy = 0;
    if (t < kW) {
      hx = t;
    } else if (t < 2 * kW) {
      hx = t - kW;
      hy = kPrTJ + 1;
    } else if (t < kHalo) {
      const int r = t - 2 * kW;
      hx = r < kPrTJ ? 0 : kW - 1;
      hy = 1 + (r < kPrTJ ? r : r - kPrTJ);
    }
    const bool halo = t < kHalo;
    // (one conditional add or subtract once the grid is wider than the
    // tile with its halo)
    const auto wrap = [nc](int v) {
      if (nc >= kPrTI + 2) return v < 0 ? v + nc : (v >= nc ? v - nc : v);
      v %= nc;
      return v < 0 ? v + nc : v;
    };
    // offset within a plane of the column (Ig, Jg), and its colour parity
    const int Ia = wrap(I0 + tx), Ja = wrap(J0 + ty);
    const int Ih = wrap(I0 + hx - 1), Jh = wrap(J0 + hy - 1);
    const int oa = Ja * nc + (Ia >> 1), pa_ = (Ia + Ja) & 1;
    const int oh = Jh * nc + (Ih >> 1), ph = (Ih + Jh) & 1;
    const int plane = nc * nc;
    float va[kPrZ + 2], vh[kPrZ + 2];
#pragma unroll
    for (int z = 0; z < kPrZ + 2; ++z) {
      va[z] = 0.f;
      vh[z] = 0.f;
      if (z < nz + 2) {
        int Kg = K0 + z - 1;
        if (Kg < 0) Kg += nc;
        if (Kg >= nc) Kg -= nc;
        const float* const ep = e + Kg * plane;
        va[z] = __ldg(ep + oa + ((pa_ ^ Kg) & 1) * hc);
        if (halo) vh[z] = __ldg(ep + oh + ((ph ^ Kg) & 1) * hc);
      }
    }
#pragma unroll
    for (int z = 0; z < kPrZ + 2; ++z) {
      if (z < nz + 2) {
        sh[z][ty + 1][tx + 1] = va[z];
        if (halo) sh[z][hy][hx] = vh[z];
      }
    }
  }
  __syncthreads();
  if (!own) return;
  // the 3x3 columns of planes z+1 and z+2 carry over to the next plane
  float pa[3][3], pb[3][3];
#pragma unroll
  for (int y = 0; y < 3; ++y)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      pa[y][x] = sh[0][ty + y][tx + x];
      pb[y][x] = sh[1][ty + y][tx + x];
    }
  const int base = ((2 * K0) * n + 2 * J) * n + I;
#pragma unroll
  for (int z = 0; z < kPrZ; ++z) {
    if (z >= nz) break;
    float zx[3][3][2];                       // [y][x][child z]: 3 e_mid + e_lo / e_hi
#pragma unroll
    for (int y = 0; y < 3; ++y) {
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const float v2 = sh[z + 2][ty + y][tx + x];
        zx[y][x][0] = fmaf(3.f, pb[y][x], pa[y][x]);
        zx[y][x][1] = fmaf(3.f, pb[y][x], v2);
        pa[y][x] = pb[y][x];
        pb[y][x] = v2;
      }
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        float yx[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) yx[x] = fmaf(3.f, zx[1][x][kk], zx[2 * jj][x][kk]);
        // fine row (2J + jj, 2(K0 + z) + kk); child a has colour a ^ par
        const int row = base + ((2 * z + kk) * n + jj) * n, par = (jj + kk) & 1;
        const float v0 = (1.f / 64.f) * fmaf(3.f, yx[1], yx[0]);  // a = 0 (i = 2I)
        const float v1 = (1.f / 64.f) * fmaf(3.f, yx[1], yx[2]);  // a = 1 (i = 2I + 1)
        if (!SKIP0 || par == 1) d[row + par * half] = v0 + old[z][(2 * kk + jj) * 2];
        if (!SKIP0 || par == 0)
          d[row + (1 - par) * half] = v1 + old[z][(2 * kk + jj) * 2 + 1];
      }
    }
  }
}

using ProlongKernel = void (*)(int, int, const float*, const float*, const float*, float*,
                               float*, float*);

ProlongKernel prolong_kernel(bool assign, bool skip0) {
  if (assign) return skip0 ? k_prolong_add32<true, true> : k_prolong_add32<true, false>;
  return skip0 ? k_prolong_add32<false, true> : k_prolong_add32<false, false>;
}

// Coarse planes per block of k_prolong_add32: the most (8, 4 or 2) that
// still give about one wave of blocks at five resident blocks per SM, else 2.
// Measured in-graph per launch (us; 2 / 4 / 8 planes): 256^3 add 70.6 / 53.7
// / 42.3, 128^3 add 9.2 / 6.8 / 6.1, 128^3 assign 6.8 / 5.8 / 5.0, 64^3
// assign 2.3 / 2.4 / 2.6, 32^3 assign 1.7 / 2.0 / 2.5 (one plane per block:
// slower everywhere): a block amortises its setup and halo planes over more
// planes, until the short grids of the small levels run out of blocks.
int prolong_planes(int nc, int comps_members) {
  const int64_t tiles = (int64_t)((nc + kPrTI - 1) / kPrTI) * ((nc + kPrTJ - 1) / kPrTJ) *
                        comps_members;
  for (int zc = kPrZ; zc > 2; zc >>= 1)
    if (tiles * ((nc + zc - 1) / zc) >= 5 * 152) return zc;
  return 2;
}

dim3 prolong_grid(int nc, int zc, int comps_members) {
  return dim3((nc + kPrTI - 1) / kPrTI, (nc + kPrTJ - 1) / kPrTJ,
              ((nc + zc - 1) / zc) * comps_members);
}

// ---------------------------------------------------------------------------
// Prolongation fused into the smoothing pass that follows it.  Inside the
// V-cycle the corrected d = d_old + P e of a level is read next by one pass
// only: the first damped Jacobi sweep (d -> t) on a Jacobi level, the
// colour-0 pass on a red-black level (which reads colour-1 cells alone, as
// neighbours; the colour-1 pass after it overwrites them without reading
// them).  So one launch forms d_old + P e on its tile and the tile's one-cell
// halo in shared memory and runs that pass from there: the prolonged values
// never go to global memory, and a launch goes.  Every value is formed with
// the operations of k_prolong_add32 in its order (z, then y, then x, the
// 1/64 scale, then the old value) and of k_lin_jacobi32x2 /
// k_lin_smooth32x2 (sums ((xm + xp) + (ym + yp)) + (zm + zp), lin_point),
// so the result equals the two launches bit for bit.
//
// A block owns a tile of kPsTX x TY x TZ fine cells in natural order (n a
// multiple of kPsTX, TY and TZ) of one ensemble member:
//   1. the coarse values under the tile and its halo, (kPsTX/2 + 2) x
//      (TY/2 + 2) x (TZ/2 + 2) cells of each component;
//   2. their z interpolation onto each of the TZ + 2 fine planes;
//   3. the fine values d_old + P e (P e alone for ASSIGN) on the tile and its
//      halo (the colour-1 cells alone for the red-black pass);
//   4. the pass on the tile's cells, r and q loaded at the start.
// RB0 (red-black): d's colour-0 cells are written, its colour-1 cells keep
// d_old; JACOBI: t = d + w (solve - d), d is not written.
// ---------------------------------------------------------------------------
constexpr int kPsTX = 32;

template <int TY, int TZ>
struct PsTile {
  static constexpr int TX = kPsTX, NT = TX * TY;
  static constexpr int FX = TX + 2, FY = TY + 2, FZ = TZ + 2;             // fine + halo
  static constexpr int CX = TX / 2 + 2, CY = TY / 2 + 2, CZ = TZ / 2 + 2;  // coarse under it
  static constexpr int kF = FZ * FY * FX;          // per component
  static constexpr int kC = CZ * CY * CX;
  static constexpr int kZ = FZ * CY * CX;
  // the coarse values are dead once the fine ones are formed: one buffer
  static constexpr int kFC = 3 * (kF > kC ? kF : kC);
  static constexpr int kSmem = kFC + 3 * kZ;       // floats
  static constexpr int kCols = (FX * FY + NT - 1) / NT;   // halo-tile columns per thread
};

template <int TY, int TZ, bool JACOBI, bool ASSIGN>
__global__ void __launch_bounds__(kPsTX * TY) k_lin_prolong_sweep32(
    LvlF L, float w, const float* __restrict__ e1, const float* __restrict__ e2,
    const float* __restrict__ e3, float* d1, float* d2, float* d3, float* __restrict__ t1,
    float* __restrict__ t2, float* __restrict__ t3, const float* __restrict__ r1,
    const float* __restrict__ r2, const float* __restrict__ r3, const float* __restrict__ q) {
  pdl_wait();
  pdl_trigger();
  using T = PsTile<TY, TZ>;
  constexpr int TX = T::TX, NT = T::NT, FX = T::FX, FY = T::FY, FZ = T::FZ;
  constexpr int CX = T::CX, CY = T::CY;
  // cells of the pass per thread: Jacobi every cell of its column over TZ
  // planes; red-black the colour-0 cells, two threads per column position
  constexpr int kCells = JACOBI ? TZ : TZ / 2;
  static_assert(JACOBI || (TZ % 2 == 0 && NT == 2 * (TX / 2) * TY), "tile");
  __shared__ float sm[T::kSmem];
  float* const sFC = sm;
  float* const sZ = sm + T::kFC;
  const int n = L.n, half = n >> 1, nc = n >> 1, hc = nc >> 1;
  int kz = blockIdx.z;
  const int m = member_of(kz, n / TZ);
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = kz * TZ;
  const size_t offf = (size_t)m * n * n * n, offc = (size_t)m * nc * nc * nc;
  const int tid = threadIdx.x;

  // 0. the pass's cells: split indices, r and q (independent of the rest)
  int px, py, pz0, pstep;
  if (JACOBI) {
    px = tid % TX;
    py = tid / TX;
    pz0 = 0;
    pstep = 1;
  } else {
    const int p = tid % (TX / 2);
    py = (tid / (TX / 2)) % TY;
    pz0 = tid / ((TX / 2) * TY);
    pstep = 2;
    px = 2 * p;                     // + the row's colour-0 offset below
  }
  int sc[kCells], fx[kCells];
  float rq[kCells][4];
#pragma unroll
  for (int s = 0; s < kCells; ++s) {
    const int z = pz0 + s * pstep, j = j0 + py, k = k0 + z;
    const int x = JACOBI ? px : px + ((j + k) & 1);
    const int i = i0 + x, colour = (i + j + k) & 1;
    fx[s] = x;
    sc[s] = (k * n + j) * n + colour * half + (i >> 1);
    rq[s][0] = __ldg(r1 + offf + sc[s]);
    rq[s][1] = __ldg(r2 + offf + sc[s]);
    rq[s][2] = __ldg(r3 + offf + sc[s]);
    rq[s][3] = __ldg(q + offf + sc[s]);
  }

  // 1. coarse values: (I, J, K) = (i0/2 - 1 + cx, j0/2 - 1 + cy, k0/2 - 1 + cz)
  {
    constexpr int kPer = (T::kC + NT - 1) / NT;
    float v[kPer][3];
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int idx = tid + s * NT;
      v[s][0] = v[s][1] = v[s][2] = 0.f;
      if (idx < T::kC) {
        const int cz = idx / (CY * CX), rem = idx - cz * (CY * CX);
        const int cy = rem / CX, cx = rem - cy * CX;
        int I = (i0 >> 1) - 1 + cx, J = (j0 >> 1) - 1 + cy, K = (k0 >> 1) - 1 + cz;
        I = I < 0 ? I + nc : (I >= nc ? I - nc : I);
        J = J < 0 ? J + nc : (J >= nc ? J - nc : J);
        K = K < 0 ? K + nc : (K >= nc ? K - nc : K);
        const int g = (K * nc + J) * nc + ((I + J + K) & 1) * hc + (I >> 1);
        v[s][0] = __ldg(e1 + offc + g);
        v[s][1] = __ldg(e2 + offc + g);
        v[s][2] = __ldg(e3 + offc + g);
      }
    }
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int idx = tid + s * NT;
      if (idx < T::kC) {
        sFC[idx] = v[s][0];
        sFC[T::kC + idx] = v[s][1];
        sFC[2 * T::kC + idx] = v[s][2];
      }
    }
  }
  __syncthreads();

  // 2. z interpolation onto fine plane k0 - 1 + zf: coarse plane index (in
  // the tile) kr = ((zf - 1) >> 1) + 1, the other one below for an even
  // fine plane, above for an odd one
  for (int idx = tid; idx < FZ * CY * CX; idx += NT) {
    const int zf = idx / (CY * CX), col = idx - zf * (CY * CX);
    const int kr = ((zf - 1) >> 1) + 1, k2r = ((zf + 1) & 1) ? kr + 1 : kr - 1;
#pragma unroll
    for (int f = 0; f < 3; ++f)
      sZ[f * T::kZ + idx] = fmaf(3.f, sFC[f * T::kC + kr * (CY * CX) + col],
                                 sFC[f * T::kC + k2r * (CY * CX) + col]);
  }
  __syncthreads();

  // 3. fine values on the tile with its halo: column (xf, yf) = fine (i0 -
  // 1 + xf, j0 - 1 + yf), planes k0 - 1 .. k0 + TZ
  {
    float old[T::kCols][FZ][3];
#pragma unroll
    for (int s = 0; s < T::kCols; ++s)
#pragma unroll
      for (int zf = 0; zf < FZ; ++zf) old[s][zf][0] = old[s][zf][1] = old[s][zf][2] = 0.f;
    if (!ASSIGN) {
#pragma unroll
      for (int s = 0; s < T::kCols; ++s) {
        const int col = tid + s * NT;
        if (col < FX * FY) {
          const int yf = col / FX, xf = col - yf * FX;
          int i = i0 - 1 + xf, j = j0 - 1 + yf;
          const int par = (i + j) & 1;
          i = i < 0 ? i + n : (i >= n ? i - n : i);
          j = j < 0 ? j + n : (j >= n ? j - n : j);
#pragma unroll
          for (int zf = 0; zf < FZ; ++zf) {
            const int colour = (par + k0 - 1 + zf) & 1;
            if (!JACOBI && colour == 0) continue;
            int k = k0 - 1 + zf;
            k = k < 0 ? k + n : (k >= n ? k - n : k);
            const int g = (k * n + j) * n + colour * half + (i >> 1);
            old[s][zf][0] = __ldg(d1 + offf + g);
            old[s][zf][1] = __ldg(d2 + offf + g);
            old[s][zf][2] = __ldg(d3 + offf + g);
          }
        }
      }
    }
    // (the coarse values are dead since the barrier above: their buffer
    // takes the fine values)
#pragma unroll
    for (int s = 0; s < T::kCols; ++s) {
      const int col = tid + s * NT;
      if (col < FX * FY) {
        const int yf = col / FX, xf = col - yf * FX;
        const int par = (i0 - 1 + xf + j0 - 1 + yf) & 1;
        // coarse columns (in the tile) under this fine column: the own one and
        // the other one on the child's side, in x and in y
        const int ir = ((xf - 1) >> 1) + 1, i2r = ((xf + 1) & 1) ? ir + 1 : ir - 1;
        const int jr = ((yf - 1) >> 1) + 1, j2r = ((yf + 1) & 1) ? jr + 1 : jr - 1;
#pragma unroll
        for (int zf = 0; zf < FZ; ++zf) {
          const int colour = (par + k0 - 1 + zf) & 1;
          if (!JACOBI && colour == 0) continue;
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            const float* const Z = sZ + f * T::kZ + zf * (CY * CX);
            const float ya = fmaf(3.f, Z[jr * CX + ir], Z[j2r * CX + ir]);
            const float yb = fmaf(3.f, Z[jr * CX + i2r], Z[j2r * CX + i2r]);
            const float v = (1.f / 64.f) * fmaf(3.f, ya, yb);
            sFC[f * T::kF + (zf * FY + yf) * FX + xf] = v + old[s][zf][f];
          }
        }
      }
    }
  }
  __syncthreads();

  // 4. the pass
#pragma unroll
  for (int s = 0; s < kCells; ++s) {
    const int z = pz0 + s * pstep;
    const int c = ((z + 1) * FY + (py + 1)) * FX + (fx[s] + 1);
    float sum[3], own[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const float* const F = sFC + f * T::kF;
      sum[f] = ((F[c - 1] + F[c + 1]) + (F[c - FX] + F[c + FX])) +
               (F[c - FY * FX] + F[c + FY * FX]);
      own[f] = F[c];
    }
    float dp, dm, dw;
    lin_point(L, sum[0], sum[1], sum[2], rq[s][3], rq[s][0], rq[s][1], rq[s][2], dp, dm, dw);
    if (JACOBI) {
      t1[offf + sc[s]] = fmaf(w, dp - own[0], own[0]);
      t2[offf + sc[s]] = fmaf(w, dm - own[1], own[1]);
      t3[offf + sc[s]] = fmaf(w, dw - own[2], own[2]);
    } else {
      d1[offf + sc[s]] = dp;
      d2[offf + sc[s]] = dm;
      d3[offf + sc[s]] = dw;
    }
  }
}

// Coarsest level of the linear problem when it is not part of a tail launch:
// start from zero, sweeps in one block (red-black, kind 0, or damped Jacobi
// through t, kind 1) until the largest change is below 1e-6 of the largest
// value or max_sweeps.  Split layout.
__global__ void k_lin_coarse_solve32(LvlF L, int kind, float w, int max_sweeps, float* d1,
                                     float* d2, float* d3, float* t1, float* t2, float* t3,
                                     const float* r1, const float* r2, const float* r3,
                                     const float* q) {
  __shared__ float red[2][32];
  __shared__ int done;
  const int n = L.n, half = n >> 1;
  const int cells = n * n * n, ccells = half * n * n;
  const size_t off = (size_t)blockIdx.x * cells;     // one block per member
  d1 += off, d2 += off, d3 += off, t1 += off, t2 += off, t3 += off;
  r1 += off, r2 += off, r3 += off, q += off;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    d1[t] = 0.f;
    d2[t] = 0.f;
    d3[t] = 0.f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float change = 0.f, size = 0.f;
    if (kind == PFC_SWEEP_JACOBI) {
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        int p, j, k, colour;
        split_cell(t, n, p, j, k, colour);
        const Stencil s = split_stencil(p, j, k, colour, n);
        float dp, dm, dw;
        lin_point(L, nbsum_coherent(d1, s), nbsum_coherent(d2, s), nbsum_coherent(d3, s),
                  q[s.c], r1[s.c], r2[s.c], r3[s.c], dp, dm, dw);
        t1[s.c] = fmaf(w, dp - d1[s.c], d1[s.c]);
        t2[s.c] = fmaf(w, dm - d2[s.c], d2[s.c]);
        t3[s.c] = fmaf(w, dw - d3[s.c], d3[s.c]);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        change = fmaxf(change, fmaxf(fabsf(t1[t] - d1[t]),
                                     fmaxf(fabsf(t2[t] - d2[t]), fabsf(t3[t] - d3[t]))));
        size = fmaxf(size, fmaxf(fabsf(t1[t]), fmaxf(fabsf(t2[t]), fabsf(t3[t]))));
        d1[t] = t1[t];
        d2[t] = t2[t];
        d3[t] = t3[t];
      }
      __syncthreads();
    } else {
      for (int colour = 0; colour < 2; ++colour) {
        for (int t = threadIdx.x; t < ccells; t += blockDim.x) {
          const int p = t % half, rr = t / half;
          const Stencil s = split_stencil(p, rr % n, rr / n, colour, n);
          float dp, dm, dw;
          lin_point(L, nbsum_coherent(d1, s), nbsum_coherent(d2, s), nbsum_coherent(d3, s),
                    q[s.c], r1[s.c], r2[s.c], r3[s.c], dp, dm, dw);
          change = fmaxf(change, fmaxf(fabsf(dp - d1[s.c]),
                                       fmaxf(fabsf(dm - d2[s.c]), fabsf(dw - d3[s.c]))));
          size = fmaxf(size, fmaxf(fabsf(dp), fmaxf(fabsf(dm), fabsf(dw))));
          d1[s.c] = dp;
          d2[s.c] = dm;
          d3[s.c] = dw;
        }
        __syncthreads();
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      change = fmaxf(change, __shfl_down_sync(0xffffffffu, change, o));
      size = fmaxf(size, __shfl_down_sync(0xffffffffu, size, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = change;
      red[1][threadIdx.x >> 5] = size;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float c = 0.f, z = 0.f;
      for (int v = 0; v < (int)((blockDim.x + 31) >> 5); ++v) {
        c = fmaxf(c, red[0][v]);
        z = fmaxf(z, red[1][v]);
      }
      done = (c <= 1e-6f * z);
    }
    __syncthreads();
    if (done) break;
  }
}

// ---------------------------------------------------------------------------
// Coarse tail: every level of at most kTailMaxN^3 cells of one FP32 V-cycle
// (pre-smoothing, residual + restriction, coarsest solve, prolongation +
// correction, post-smoothing) in a single launch of one thread block whose
// levels all live in shared memory.  On these grids separate kernels were
// pure launch latency.  Each thread owns a fixed (i, j) column and walks k
// with a stride, so no cell index is divided per cell.
// ---------------------------------------------------------------------------
constexpr int kTailMaxN = 16;
constexpr int kTailMaxLevels = 8;
constexpr int kTailThreads = 1024;

struct TailParams {
  int nlev;          // levels in the tail; the last one is the coarsest
  int nu1, nu2, jfactor, jfactor_top, coarse_sweeps;
  int zero_init;     // the top tail level starts from d = 0
  float w;
  LvlF L[kTailMaxLevels];
  int kind[kTailMaxLevels];
  float* gd[3];      // top level in global memory
  const float* gr[3];
  const float* gq;
};

// Fields of one level in shared memory: d(3), t(3), r(3), q, n^3 floats each.
struct SLev {
  float *d0, *d1, *d2, *t0, *t1, *t2, *r0, *r1, *r2, *q;
};

__device__ __forceinline__ SLev slev(float* smem, const TailParams& P, int l) {
  int off = 0;
  for (int m = 0; m < l; ++m) off += 10 * P.L[m].n * P.L[m].n * P.L[m].n;
  const int c = P.L[l].n * P.L[l].n * P.L[l].n;
  float* b = smem + off;
  SLev S;
  S.d0 = b;
  S.d1 = b + c;
  S.d2 = b + 2 * c;
  S.t0 = b + 3 * c;
  S.t1 = b + 4 * c;
  S.t2 = b + 5 * c;
  S.r0 = b + 6 * c;
  S.r1 = b + 7 * c;
  S.r2 = b + 8 * c;
  S.q = b + 9 * c;
  return S;
}

// Column walker: thread -> (i, j, k0); k advances by kstep.
struct Walk {
  int n, i, j, k0, kstep, im, ip, jm, jp;
  bool active;
  __device__ __forceinline__ Walk(int n_) : n(n_) {
    const int plane = n * n;
    kstep = blockDim.x / plane;
    if (kstep > n) kstep = n;
    const int tid = threadIdx.x;
    k0 = tid / plane;
    const int rem = tid - k0 * plane;
    j = rem / n;
    i = rem - j * n;
    active = k0 < kstep;
    im = (i == 0) ? n - 1 : i - 1;
    ip = (i + 1 == n) ? 0 : i + 1;
    jm = (j == 0) ? n - 1 : j - 1;
    jp = (j + 1 == n) ? 0 : j + 1;
  }
  // linear indices of (i, j, k) and its six neighbours
  __device__ __forceinline__ void at(int k, int& c, int& xm, int& xp, int& ym, int& yp, int& zm,
                                     int& zp) const {
    const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
    const int row = n * (j + n * k);
    c = row + i;
    xm = row + im;
    xp = row + ip;
    ym = i + n * (jm + n * k);
    yp = i + n * (jp + n * k);
    zm = i + n * (j + n * km);
    zp = i + n * (j + n * kp);
  }
};

// Colour walker of a red-black pass (n even, n^2/2 <= blockDim): thread ->
// (p, j, k0) over the n/2 cells of one colour in each x-row; k advances by
// kstep and the cell's x index i = 2p + ((j + k + colour) & 1) follows the
// colour, so every thread has cells of the colour in every pass (a column
// walker leaves idle the half of the threads whose column has the other
// parity, since its k-walk keeps one parity).
struct CWalk {
  int n, p, j, k0, kstep, jm, jp;
  __device__ __forceinline__ CWalk(int n_) : n(n_) {
    const int half = n >> 1, hplane = half * n;
    kstep = blockDim.x / hplane;
    if (kstep > n) kstep = n;
    const int tid = threadIdx.x;
    k0 = tid / hplane;
    const int rem = tid - k0 * hplane;
    j = rem / half;
    p = rem - j * half;
    if (k0 >= kstep) k0 = n;                     // no cell for this thread
    jm = (j == 0) ? n - 1 : j - 1;
    jp = (j + 1 == n) ? 0 : j + 1;
  }
  __device__ __forceinline__ void at(int k, int colour, int& c, int& xm, int& xp, int& ym,
                                     int& yp, int& zm, int& zp) const {
    const int i = 2 * p + ((j + k + colour) & 1);
    const int im = (i == 0) ? n - 1 : i - 1, ip = (i + 1 == n) ? 0 : i + 1;
    const int km = (k == 0) ? n - 1 : k - 1, kp = (k + 1 == n) ? 0 : k + 1;
    const int row = n * (j + n * k);
    c = row + i;
    xm = row + im;
    xp = row + ip;
    ym = n * (jm + n * k) + i;
    yp = n * (jp + n * k) + i;
    zm = n * (j + n * km) + i;
    zp = n * (j + n * kp) + i;
  }
};

__device__ __forceinline__ float nb6(const float* v, int xm, int xp, int ym, int yp, int zm,
                                     int zp) {
  return ((v[xm] + v[xp]) + (v[ym] + v[yp])) + (v[zm] + v[zp]);
}

__device__ void tail_smooth(const LvlF& L, int kind, SLev S, int sweeps, int jfactor, float w,
                            bool zero) {
  if (sweeps <= 0) return;
  const Walk W(L.n);
  int c, xm, xp, ym, yp, zm, zp;
  if (kind == PFC_SWEEP_JACOBI) {
    const int js = sweeps * jfactor;
    float *s0 = S.d0, *s1 = S.d1, *s2 = S.d2, *o0 = S.t0, *o1 = S.t1, *o2 = S.t2;
    for (int s = 0; s < js; ++s) {
      const bool z = zero && s == 0;
      if (W.active) {
        for (int k = W.k0; k < L.n; k += W.kstep) {
          W.at(k, c, xm, xp, ym, yp, zm, zp);
          float sp = 0.f, sm_ = 0.f, sw = 0.f, p0 = 0.f, m0 = 0.f, w0 = 0.f;
          if (!z) {
            sp = nb6(s0, xm, xp, ym, yp, zm, zp);
            sm_ = nb6(s1, xm, xp, ym, yp, zm, zp);
            sw = nb6(s2, xm, xp, ym, yp, zm, zp);
            p0 = s0[c];
            m0 = s1[c];
            w0 = s2[c];
          }
          float dp, dm, dw;
          lin_point(L, sp, sm_, sw, S.q[c], S.r0[c], S.r1[c], S.r2[c], dp, dm, dw);
          o0[c] = fmaf(w, dp - p0, p0);
          o1[c] = fmaf(w, dm - m0, m0);
          o2[c] = fmaf(w, dw - w0, w0);
        }
      }
      __syncthreads();
      float* x;
      x = s0; s0 = o0; o0 = x;
      x = s1; s1 = o1; o1 = x;
      x = s2; s2 = o2; o2 = x;
    }
    if (js & 1) {
      if (W.active) {
        for (int k = W.k0; k < L.n; k += W.kstep) {
          W.at(k, c, xm, xp, ym, yp, zm, zp);
          S.d0[c] = s0[c];
          S.d1[c] = s1[c];
          S.d2[c] = s2[c];
        }
      }
      __syncthreads();
    }
    return;
  }
  const CWalk CW(L.n);
  for (int s = 0; s < sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      const bool z = zero && s == 0 && colour == 0;
      for (int k = CW.k0; k < L.n; k += CW.kstep) {
        CW.at(k, colour, c, xm, xp, ym, yp, zm, zp);
        float sp = 0.f, sm_ = 0.f, sw = 0.f;
        if (!z) {
          sp = nb6(S.d0, xm, xp, ym, yp, zm, zp);
          sm_ = nb6(S.d1, xm, xp, ym, yp, zm, zp);
          sw = nb6(S.d2, xm, xp, ym, yp, zm, zp);
        }
        float dp, dm, dw;
        lin_point(L, sp, sm_, sw, S.q[c], S.r0[c], S.r1[c], S.r2[c], dp, dm, dw);
        S.d0[c] = dp;
        S.d1[c] = dm;
        S.d2[c] = dw;
      }
      __syncthreads();
    }
  }
}

// rho = r - J d on the fine level F, averaged onto the coarse level's r.
__device__ void tail_restrict(const LvlF& L, SLev F, SLev C) {
  const int n = L.n;
  const Walk W(n >> 1);
  if (W.active) {
    for (int K = W.k0; K < W.n; K += W.kstep) {
      float a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int ch = 0; ch < 8; ++ch) {
        const Stencil st = stencil_at(2 * W.i + (ch & 1), 2 * W.j + ((ch >> 1) & 1),
                                      2 * K + (ch >> 2), n);
        const int c = (int)st.c;
        const float p = F.d0[c], m = F.d1[c], w = F.d2[c];
        const float lm = fmaf(-6.f, m, nbsum_coherent(F.d1, st));
        const float lw = fmaf(-6.f, w, nbsum_coherent(F.d2, st));
        const float lp = fmaf(-6.f, p, nbsum_coherent(F.d0, st));
        a1 += F.r0[c] - fmaf(-L.tg, lm, p);
        a2 += F.r1[c] - (fmaf(-F.q[c], p, m) - L.g * lw);
        a3 += F.r2[c] - fmaf(-L.gh, lp, w);
      }
      const int cc = W.i + W.n * (W.j + W.n * K);
      C.r0[cc] = 0.125f * a1;
      C.r1[cc] = 0.125f * a2;
      C.r2[cc] = 0.125f * a3;
    }
  }
  __syncthreads();
}

// d_F += P d_C (trilinear, weights 27, 9, 3, 1 over 64).
__device__ void tail_prolong(int n, SLev C, SLev F) {
  const int nc = n >> 1, nn = nc * nc;
  const Walk W(n);
  if (W.active) {
    const int I = W.i >> 1, J = W.j >> 1;
    const int I2 = ((W.i & 1) ? I + 1 : I - 1 + nc) % nc;
    const int J2 = ((W.j & 1) ? J + 1 : J - 1 + nc) % nc;
    for (int k = W.k0; k < n; k += W.kstep) {
      const int K = k >> 1;
      const int K2 = ((k & 1) ? K + 1 : K - 1 + nc) % nc;
      const int o000 = I + J * nc + K * nn, o100 = I2 + J * nc + K * nn,
                o010 = I + J2 * nc + K * nn, o001 = I + J * nc + K2 * nn,
                o110 = I2 + J2 * nc + K * nn, o101 = I2 + J * nc + K2 * nn,
                o011 = I + J2 * nc + K2 * nn, o111 = I2 + J2 * nc + K2 * nn;
      const int c = W.i + n * (W.j + n * k);
      const float* e[3] = {C.d0, C.d1, C.d2};
      float* d[3] = {F.d0, F.d1, F.d2};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float* x = e[q];
        const float g2 = (x[o100] + x[o010]) + x[o001];
        const float g3 = (x[o110] + x[o101]) + x[o011];
        float acc = fmaf(3.f, g3, x[o111]);
        acc = fmaf(9.f, g2, acc);
        acc = fmaf(27.f, x[o000], acc);
        d[q][c] = fmaf(1.0f / 64.0f, acc, d[q][c]);
      }
    }
  }
  __syncthreads();
}

// Coarsest level: from d = 0, sweeps until the largest change is <= 1e-6 of
// the largest value or `max_sweeps` (the outer FP64 loop absorbs the rest).
__device__ void tail_coarse(const LvlF& L, int kind, SLev S, float w, int max_sweeps,
                            float (*red)[32], int* done) {
  const int n = L.n, cells = n * n * n;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    S.d0[t] = 0.f;
    S.d1[t] = 0.f;
    S.d2[t] = 0.f;
  }
  __syncthreads();
  const Walk W(n);
  const CWalk CW(n);
  int c, xm, xp, ym, yp, zm, zp;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float change = 0.f, size = 0.f;
    if (kind == PFC_SWEEP_JACOBI) {
      if (W.active) {
        for (int k = W.k0; k < n; k += W.kstep) {
          W.at(k, c, xm, xp, ym, yp, zm, zp);
          float dp, dm, dw;
          lin_point(L, nb6(S.d0, xm, xp, ym, yp, zm, zp), nb6(S.d1, xm, xp, ym, yp, zm, zp),
                    nb6(S.d2, xm, xp, ym, yp, zm, zp), S.q[c], S.r0[c], S.r1[c], S.r2[c], dp,
                    dm, dw);
          S.t0[c] = fmaf(w, dp - S.d0[c], S.d0[c]);
          S.t1[c] = fmaf(w, dm - S.d1[c], S.d1[c]);
          S.t2[c] = fmaf(w, dw - S.d2[c], S.d2[c]);
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        change = fmaxf(change, fmaxf(fabsf(S.t0[t] - S.d0[t]),
                                     fmaxf(fabsf(S.t1[t] - S.d1[t]), fabsf(S.t2[t] - S.d2[t]))));
        size = fmaxf(size, fmaxf(fabsf(S.t0[t]), fmaxf(fabsf(S.t1[t]), fabsf(S.t2[t]))));
        S.d0[t] = S.t0[t];
        S.d1[t] = S.t1[t];
        S.d2[t] = S.t2[t];
      }
      __syncthreads();
    } else {
      for (int colour = 0; colour < 2; ++colour) {
        for (int k = CW.k0; k < n; k += CW.kstep) {
          CW.at(k, colour, c, xm, xp, ym, yp, zm, zp);
          float dp, dm, dw;
          lin_point(L, nb6(S.d0, xm, xp, ym, yp, zm, zp), nb6(S.d1, xm, xp, ym, yp, zm, zp),
                    nb6(S.d2, xm, xp, ym, yp, zm, zp), S.q[c], S.r0[c], S.r1[c], S.r2[c],
                    dp, dm, dw);
          change = fmaxf(change, fmaxf(fabsf(dp - S.d0[c]),
                                       fmaxf(fabsf(dm - S.d1[c]), fabsf(dw - S.d2[c]))));
          size = fmaxf(size, fmaxf(fabsf(dp), fmaxf(fabsf(dm), fabsf(dw))));
          S.d0[c] = dp;
          S.d1[c] = dm;
          S.d2[c] = dw;
        }
        __syncthreads();
      }
    }
    if ((sweep & 3) != 3) continue;   // test convergence every fourth sweep
    for (int o = 16; o > 0; o >>= 1) {
      change = fmaxf(change, __shfl_down_sync(0xffffffffu, change, o));
      size = fmaxf(size, __shfl_down_sync(0xffffffffu, size, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = change;
      red[1][threadIdx.x >> 5] = size;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float cmax = 0.f, z = 0.f;
      for (int v = 0; v < (int)((blockDim.x + 31) >> 5); ++v) {
        cmax = fmaxf(cmax, red[0][v]);
        z = fmaxf(z, red[1][v]);
      }
      *done = (cmax <= 1e-6f * z);
    }
    __syncthreads();
    if (*done) break;
  }
}

// q of every tail level below the first, restricted in shared memory.
__device__ void tail_qrestrict(float* smem, const TailParams& P) {
  for (int l = 1; l < P.nlev; ++l) {
    const SLev F = slev(smem, P, l - 1), C = slev(smem, P, l);
    const int n = P.L[l - 1].n;
    const Walk W(n >> 1);
    if (W.active) {
      for (int K = W.k0; K < W.n; K += W.kstep) {
        float acc = 0.f;
        for (int ch = 0; ch < 8; ++ch)
          acc += F.q[(2 * W.i + (ch & 1)) + n * ((2 * W.j + ((ch >> 1) & 1)) + n * (2 * K + (ch >> 2)))];
        C.q[W.i + W.n * (W.j + W.n * K)] = 0.125f * acc;
      }
    }
    __syncthreads();
  }
}

// One V-cycle over the tail levels held in shared memory (one block).
__device__ void tail_vcycle(float* smem, const TailParams& P, bool zero_top, float (*red)[32],
                            int* done) {
  const int last = P.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const SLev S = slev(smem, P, l);
    const bool zero = (l > 0) || zero_top;
    if (P.nu1 > 0) {
      tail_smooth(P.L[l], P.kind[l], S, P.nu1, l == 0 ? P.jfactor_top : P.jfactor, P.w, zero);
    } else if (zero) {
      const int cells = P.L[l].n * P.L[l].n * P.L[l].n;
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        S.d0[t] = 0.f;
        S.d1[t] = 0.f;
        S.d2[t] = 0.f;
      }
      __syncthreads();
    }
    tail_restrict(P.L[l], S, slev(smem, P, l + 1));
  }
  tail_coarse(P.L[last], P.kind[last], slev(smem, P, last), P.w, P.coarse_sweeps, red, done);
  for (int l = last - 1; l >= 0; --l) {
    const SLev S = slev(smem, P, l);
    tail_prolong(P.L[l].n, slev(smem, P, l + 1), S);
    tail_smooth(P.L[l], P.kind[l], S, P.nu2, l == 0 ? P.jfactor_top : P.jfactor, P.w, false);
  }
}

// The whole tail lives in shared memory.  The top level's r and q (and d
// when it does not start from zero) are loaded from global memory, the lower
// levels' q are restricted in shared memory, and the top level's d is stored
// back at the end.
__global__ void __launch_bounds__(kTailThreads) k_lin_tail32(TailParams P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float smem[];
  __shared__ float red[2][32];
  __shared__ int done;
  const bool zero_top = P.zero_init != 0;
  // one block per member of a batched launch; P itself stays unmodified (a
  // written parameter struct would be copied to local memory)
  const size_t off = (size_t)blockIdx.x * P.L[0].n * P.L[0].n * P.L[0].n;
  float* const gd0 = P.gd[0] + off;
  float* const gd1 = P.gd[1] + off;
  float* const gd2 = P.gd[2] + off;
  {
    const float* const gr0 = P.gr[0] + off;
    const float* const gr1 = P.gr[1] + off;
    const float* const gr2 = P.gr[2] + off;
    const float* const gq = P.gq + off;
    const SLev S0 = slev(smem, P, 0);
    const int n0 = P.L[0].n;
    const int cells = n0 * n0 * n0;
    // all of a thread's global loads of a batch before any shared-memory
    // store: one memory round trip per batch instead of one per value
    constexpr int kB = 4;
    for (int t0 = threadIdx.x; t0 < cells; t0 += kB * blockDim.x) {
      float v[7][kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < cells) {
          v[0][u] = gr0[t];
          v[1][u] = gr1[t];
          v[2][u] = gr2[t];
          v[3][u] = gq[t];
          if (!zero_top) {
            v[4][u] = gd0[t];
            v[5][u] = gd1[t];
            v[6][u] = gd2[t];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < cells) {
          int p, j, k, colour;
          split_cell(t, n0, p, j, k, colour);
          const int o = (2 * p + ((j + k + colour) & 1)) + n0 * (j + n0 * k);   // natural index
          S0.r0[o] = v[0][u];
          S0.r1[o] = v[1][u];
          S0.r2[o] = v[2][u];
          S0.q[o] = v[3][u];
          if (!zero_top) {
            S0.d0[o] = v[4][u];
            S0.d1[o] = v[5][u];
            S0.d2[o] = v[6][u];
          }
        }
      }
    }
    __syncthreads();
  }
  tail_qrestrict(smem, P);
  tail_vcycle(smem, P, zero_top, red, &done);
  const SLev S0 = slev(smem, P, 0);
  const int n0 = P.L[0].n;
  const int cells = n0 * n0 * n0;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    int p, j, k, colour;
    split_cell(t, n0, p, j, k, colour);
    const int o = (2 * p + ((j + k + colour) & 1)) + n0 * (j + n0 * k);
    gd0[t] = S0.d0[o];
    gd1[t] = S0.d1[o];
    gd2[t] = S0.d2[o];
  }
}

// Shared memory of the tail starting at level l0 (10 floats per cell per level).
size_t tail_smem_bytes(const int* sizes, int l0, int nl) {
  size_t cells = 0;
  for (int l = l0; l < nl; ++l) cells += (size_t)sizes[l] * sizes[l] * sizes[l];
  return cells * 10 * sizeof(float);
}

constexpr size_t kTailMaxSmem = 200 * 1024;   // + static shared memory <= 227 KiB

// ---------------------------------------------------------------------------
// Cluster tail: the coarse part of an FP32 V-cycle from a level of up to
// kCtMaxN^3 cells down, in one launch of a thread-block cluster of kCtCtas
// CTAs per ensemble member.  The leading levels whose size is a multiple of
// kCtCtas are spread over the cluster in z slabs (CTA r holds planes
// [r nz, (r+1) nz), nz = n / kCtCtas, natural order within the slab); the
// remaining small levels live in CTA 0 and run the single-block tail code.
// A cell's neighbour planes in another CTA are read through distributed
// shared memory (the CTA's shared window mapped with map_shared_rank), and
// every phase whose results another CTA reads ends with a cluster barrier.
// So the 32^3 and 16^3 levels, which as separate launches were pure launch
// latency and as one block kept 151 SMs idle, run on kCtCtas SMs without a
// launch per sweep.  q of every level comes restricted from global memory.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

constexpr int kCtCtas = 8;                      // portable cluster size
constexpr int kCtThreads = 1024;
constexpr int kCtMaxN = 32;
constexpr size_t kCtMaxSmem = 224 * 1024;   // + 272 B static <= 227 KiB

struct CTailParams {
  int nlev;          // levels from the cluster's top level to the coarsest
  int ndist;         // the first ndist levels are spread over the cluster
  int nu1, nu2, jfactor, jfactor_top, zero_init;
  float w;
  LvlF L[kTailMaxLevels];
  int kind[kTailMaxLevels];
  float* gd[3];                         // top level d in global memory (split layout)
  const float* gr[3];                   // top level r
  const float* gq[kTailMaxLevels];      // q of every level (split layout)
  int ga_off;                           // float offset of CTA 0's levels in shared memory
  TailParams G;                         // CTA 0's levels ndist .. nlev-1
};

// This CTA's slab of distributed level l: fields f = 0-2 d, 3-5 t, 6-8 r,
// 9 q at base + f * slab, each nz planes of n^2 cells in natural order.
__device__ __forceinline__ float* ct_base(float* smem, const CTailParams& P, int l) {
  int off = 0;
  for (int m = 0; m < l; ++m) off += 10 * (P.L[m].n / kCtCtas) * P.L[m].n * P.L[m].n;
  return smem + off;
}

// 32-bit shared-window addresses: a shared::cta address of this CTA is also
// its shared::cluster address; mapa gives another CTA's address of the same
// offset.  Loads through these are volatile asm, which keeps them in program
// order with the cluster barriers (themselves volatile asm).
__device__ __forceinline__ unsigned ct_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned ct_mapa(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float ct_ld(unsigned addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void ct_st(unsigned addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// A distributed level as this CTA sees it: its slab (planes [z0, z0 + nz))
// and the cluster addresses of the slabs of the CTAs that hold the planes
// just below and above it (periodic in the rank).  plane_at(k) takes an
// unwrapped plane index within [z0 - nz, z0 + 2 nz) and returns the cluster
// address of its first cell.
struct CtSlab {
  int n, nz, plane, slab, z0;
  float* own;
  unsigned u_own, u_prev, u_next;
  __device__ __forceinline__ CtSlab(unsigned me, float* base, int n_) {
    n = n_;
    nz = n / kCtCtas;
    plane = n * n;
    slab = nz * plane;
    z0 = (int)me * nz;
    own = base;
    u_own = ct_u32(base);
    u_prev = ct_mapa(u_own, (me + kCtCtas - 1) % kCtCtas);
    u_next = ct_mapa(u_own, (me + 1) % kCtCtas);
  }
  __device__ __forceinline__ unsigned plane_at(int k) const {
    const int lz = k - z0;
    if (lz < 0) return u_prev + 4u * (unsigned)((lz + nz) * plane);
    if (lz >= nz) return u_next + 4u * (unsigned)((lz - nz) * plane);
    return u_own + 4u * (unsigned)(lz * plane);
  }
};

// Thread -> fixed (i, j) column of a level with n^2 <= blockDim.x cells per
// plane, first local plane lz0 and plane stride lzs (the Walk of the
// single-block tail); im..jp are the in-plane neighbours' offsets.
struct CtCol {
  int i, j, x, lz0, lzs, im, ip, jm, jp;
  bool on;
  __device__ __forceinline__ CtCol(int n) {
    const int plane = n * n;
    lzs = blockDim.x / plane;
    const int t = threadIdx.x;
    lz0 = t / plane;
    x = t - lz0 * plane;
    j = x / n;
    i = x - j * n;
    on = lz0 < lzs;
    im = (i == 0) ? n - 1 : i - 1;
    ip = (i + 1 == n) ? 0 : i + 1;
    jm = (j == 0) ? n - 1 : j - 1;
    jp = (j + 1 == n) ? 0 : j + 1;
    im += j * n;
    ip += j * n;
    jm = jm * n + i;
    jp = jp * n + i;
  }
};

// Neighbour sum of cell x of a local plane `own` with the planes below and
// above at cluster addresses um, up.
__device__ __forceinline__ float ct_nb(const float* own, unsigned um, unsigned up,
                                       const CtCol& w) {
  return ((own[w.im] + own[w.ip]) + (own[w.jm] + own[w.jp])) +
         (ct_ld(um + 4u * w.x) + ct_ld(up + 4u * w.x));
}

// `sweeps` smoothing sweeps (damped collective Jacobi: kind JACOBI, x jf;
// else red-black) on distributed level l; zero: d = 0 before the first.
// Coarsest: from d = 0, sweeps of the level's kind (Jacobi without the
// factor) until the largest change is <= 1e-6 of the largest value (tested
// every fourth sweep over the whole cluster) or `sweeps`, as the
// single-block coarsest solve.
__device__ void ct_smooth(const cg::cluster_group& cl, unsigned me, float* smem,
                          const CTailParams& P, int l, int sweeps, int jf, bool zero,
                          bool coarsest, float (*red)[32], float* cmax) {
  if (sweeps <= 0) return;
  const LvlF& L = P.L[l];
  const CtSlab S(me, ct_base(smem, P, l), L.n);
  const CtCol w(L.n);
  const bool jac = P.kind[l] == PFC_SWEEP_JACOBI;
  const int nsweep = jac && !coarsest ? sweeps * jf : sweeps;
  const unsigned fb = 4u * (unsigned)S.slab;   // bytes per field
  int s = 0;                                    // d in fields s..s+2 (Jacobi ping-pong)
  for (int sweep = 0; sweep < nsweep; ++sweep) {
    float change = 0.f, size = 0.f;
    for (int pass = 0; pass < (jac ? 1 : 2); ++pass) {
      const bool z = zero && sweep == 0 && pass == 0;
      const int so = s * S.slab, dso = (jac ? 3 - s : 0) * S.slab;
      if (w.on) {
        for (int lz = w.lz0; lz < S.nz; lz += w.lzs) {
          const int k = S.z0 + lz, c = lz * S.plane + w.x;
          if (!jac && ((w.i + w.j + k) & 1) != pass) continue;
          float sum0 = 0.f, sum1 = 0.f, sum2 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
          if (!z) {
            const float* own = S.own + so + lz * S.plane;
            const unsigned um = S.plane_at(k - 1) + 4u * so, up = S.plane_at(k + 1) + 4u * so;
            sum0 = ct_nb(own, um, up, w);
            c0 = own[w.x];
            sum1 = ct_nb(own + S.slab, um + fb, up + fb, w);
            c1 = own[S.slab + w.x];
            sum2 = ct_nb(own + 2 * S.slab, um + 2 * fb, up + 2 * fb, w);
            c2 = own[2 * S.slab + w.x];
          }
          float dp, dm, dw;
          lin_point(L, sum0, sum1, sum2, S.own[9 * S.slab + c], S.own[6 * S.slab + c],
                   S.own[7 * S.slab + c], S.own[8 * S.slab + c], dp, dm, dw);
          if (jac) {
            dp = fmaf(P.w, dp - c0, c0);
            dm = fmaf(P.w, dm - c1, c1);
            dw = fmaf(P.w, dw - c2, c2);
          }
          if (coarsest) {
            // old values: Jacobi's source; a red-black cell's own value (0
            // on the first sweep from d = 0)
            float o0 = c0, o1 = c1, o2 = c2;
            if (!jac) {
              const bool fresh = zero && sweep == 0;
              o0 = fresh ? 0.f : S.own[c];
              o1 = fresh ? 0.f : S.own[S.slab + c];
              o2 = fresh ? 0.f : S.own[2 * S.slab + c];
            }
            change = fmaxf(change, fmaxf(fabsf(dp - o0), fmaxf(fabsf(dm - o1), fabsf(dw - o2))));
            size = fmaxf(size, fmaxf(fabsf(dp), fmaxf(fabsf(dm), fabsf(dw))));
          }
          float* dst = S.own + dso + c;
          dst[0] = dp;
          dst[S.slab] = dm;
          dst[2 * S.slab] = dw;
        }
      }
      cl.sync();
      if (jac) s = 3 - s;
    }
    if (!coarsest || (sweep & 3) != 3) continue;   // convergence test every fourth sweep
    for (int o = 16; o > 0; o >>= 1) {
      change = fmaxf(change, __shfl_down_sync(0xffffffffu, change, o));
      size = fmaxf(size, __shfl_down_sync(0xffffffffu, size, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = change;
      red[1][threadIdx.x >> 5] = size;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float cm = 0.f, zm = 0.f;
      for (int v = 0; v < (int)((blockDim.x + 31) >> 5); ++v) {
        cm = fmaxf(cm, red[0][v]);
        zm = fmaxf(zm, red[1][v]);
      }
      cmax[0] = cm;
      cmax[1] = zm;
    }
    cl.sync();
    float cm = 0.f, zm = 0.f;
    const unsigned uc = ct_u32(cmax);
    for (unsigned r = 0; r < (unsigned)kCtCtas; ++r) {
      const unsigned a = ct_mapa(uc, r);
      cm = fmaxf(cm, ct_ld(a));
      zm = fmaxf(zm, ct_ld(a + 4u));
    }
    cl.sync();                         // every CTA has read the maxima before they change
    if (cm <= 1e-6f * zm) break;
  }
  if (s != 0) {                                 // the result is in t
    if (w.on) {
      for (int lz = w.lz0; lz < S.nz; lz += w.lzs) {
        const int c = lz * S.plane + w.x;
        S.own[c] = S.own[3 * S.slab + c];
        S.own[S.slab + c] = S.own[4 * S.slab + c];
        S.own[2 * S.slab + c] = S.own[5 * S.slab + c];
      }
    }
    cl.sync();
  }
}

// rho = r - J d of distributed level l averaged onto level l+1 (distributed,
// or CTA 0's when l+1 == ndist).  Coarse plane K is formed by the CTA that
// holds fine plane 2K (for a distributed coarse level also its owner).
// dzero: d = 0 on level l, so rho = r.
__device__ void ct_restrict(const cg::cluster_group& cl, unsigned me, float* smem,
                            const CTailParams& P, int l, bool dzero) {
  const LvlF& L = P.L[l];
  const CtSlab S(me, ct_base(smem, P, l), L.n);
  const int n = L.n, nc = n >> 1, pc = nc * nc;
  const bool cdist = l + 1 < P.ndist;
  unsigned ucr;                                 // cluster address of coarse r0, plane 0
  int cstride, cz0 = 0;
  if (cdist) {
    const int cslab = (nc / kCtCtas) * pc;
    ucr = ct_u32(ct_base(smem, P, l + 1) + 6 * cslab);
    cstride = cslab;
    cz0 = (int)me * (nc / kCtCtas);
  } else {
    ucr = ct_mapa(ct_u32(slev(smem + P.ga_off, P.G, 0).r0), 0u);
    cstride = nc * pc;
  }
  const unsigned fb = 4u * (unsigned)S.slab;
  const int K0 = (S.z0 + 1) >> 1, K1 = (S.z0 + S.nz + 1) >> 1;   // 2K in [z0, z0 + nz)
  const CtCol w(nc);
  if (w.on) {
    for (int K = K0 + w.lz0; K < K1; K += w.lzs) {
      float a1 = 0.f, a2 = 0.f, a3 = 0.f;
      for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * K + kk;
        const unsigned pk = S.plane_at(k);     // field 0 of plane k
        const unsigned pm = S.plane_at(k - 1);
        const unsigned pp = S.plane_at(k + 1);
        for (int ch = 0; ch < 4; ++ch) {
          const int i = 2 * w.i + (ch & 1), j = 2 * w.j + (ch >> 1);
          const unsigned x = 4u * (unsigned)(j * n + i);
          a1 += ct_ld(pk + 6 * fb + x);
          a2 += ct_ld(pk + 7 * fb + x);
          a3 += ct_ld(pk + 8 * fb + x);
          if (dzero) continue;
          const int im = (i == 0) ? n - 1 : i - 1, ip = (i + 1 == n) ? 0 : i + 1;
          const int jm = (j == 0) ? n - 1 : j - 1, jp = (j + 1 == n) ? 0 : j + 1;
          const unsigned xm = 4u * (j * n + im), xp = 4u * (j * n + ip);
          const unsigned ym = 4u * (jm * n + i), yp = 4u * (jp * n + i);
          float lap[3], ctr[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const unsigned f = pk + q * fb, fm = pm + q * fb, fp = pp + q * fb;
            ctr[q] = ct_ld(f + x);
            lap[q] = fmaf(-6.f, ctr[q], ((ct_ld(f + xm) + ct_ld(f + xp)) +
                                         (ct_ld(f + ym) + ct_ld(f + yp))) +
                                            (ct_ld(fm + x) + ct_ld(fp + x)));
          }
          // minus (J d): rows 1-3 of the linearised operator
          a1 -= fmaf(-L.tg, lap[1], ctr[0]);
          a2 -= fmaf(-ct_ld(pk + 9 * fb + x), ctr[0], ctr[1]) - L.g * lap[2];
          a3 -= fmaf(-L.gh, lap[0], ctr[2]);
        }
      }
      const unsigned dst = ucr + 4u * (unsigned)((K - cz0) * pc + w.x);
      ct_st(dst, 0.125f * a1);
      ct_st(dst + 4u * cstride, 0.125f * a2);
      ct_st(dst + 8u * cstride, 0.125f * a3);
    }
  }
  cl.sync();
}

// d += P e on distributed level l (assign: d = P e) from level l+1
// (distributed, or CTA 0's): trilinear, weights 27, 9, 3, 1 over 64.
__device__ void ct_prolong(const cg::cluster_group& cl, unsigned me, float* smem,
                           const CTailParams& P, int l, bool assign) {
  const int n = P.L[l].n, nc = n >> 1, pc = nc * nc;
  const CtSlab F(me, ct_base(smem, P, l), n);
  const bool cdist = l + 1 < P.ndist;
  unsigned cown, cprev, cnext, cfb;
  int cz0 = 0, cnz = nc;
  if (cdist) {
    const CtSlab C(me, ct_base(smem, P, l + 1), nc);
    cown = C.u_own;
    cprev = C.u_prev;
    cnext = C.u_next;
    cfb = 4u * (unsigned)C.slab;
    cz0 = C.z0;
    cnz = C.nz;
  } else {
    cown = ct_mapa(ct_u32(slev(smem + P.ga_off, P.G, 0).d0), 0u);
    cprev = cnext = cown;
    cfb = 4u * (unsigned)(nc * pc);
  }
  const CtCol w(n);
  const int I = w.i >> 1, J = w.j >> 1;
  const int I2 = ((w.i & 1) ? I + 1 : I - 1 + nc) % nc;
  const int J2 = ((w.j & 1) ? J + 1 : J - 1 + nc) % nc;
  const unsigned o00 = 4u * (I + J * nc), o10 = 4u * (I2 + J * nc);
  const unsigned o01 = 4u * (I + J2 * nc), o11 = 4u * (I2 + J2 * nc);
  if (w.on) {
    for (int lz = w.lz0; lz < F.nz; lz += w.lzs) {
      const int k = F.z0 + lz, K = k >> 1;
      int K2 = (k & 1) ? K + 1 : K - 1;       // unwrapped
      unsigned a, b;
      if (cdist) {
        a = cown + 4u * (unsigned)((K - cz0) * pc);
        const int l2 = K2 - cz0;
        b = l2 < 0 ? cprev + 4u * (unsigned)((l2 + cnz) * pc)
                   : l2 >= cnz ? cnext + 4u * (unsigned)((l2 - cnz) * pc)
                               : cown + 4u * (unsigned)(l2 * pc);
      } else {
        K2 = (K2 + nc) % nc;
        a = cown + 4u * (unsigned)(K * pc);
        b = cown + 4u * (unsigned)(K2 * pc);
      }
      const int c = lz * F.plane + w.x;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float g2 = (ct_ld(a + o10) + ct_ld(a + o01)) + ct_ld(b + o00);
        const float g3 = (ct_ld(a + o11) + ct_ld(b + o10)) + ct_ld(b + o01);
        float acc = fmaf(3.f, g3, ct_ld(b + o11));
        acc = fmaf(9.f, g2, acc);
        acc = fmaf(27.f, ct_ld(a + o00), acc);
        float* dq = F.own + q * F.slab + c;
        *dq = assign ? (1.0f / 64.0f) * acc : fmaf(1.0f / 64.0f, acc, *dq);
        a += cfb;
        b += cfb;
      }
    }
  }
  cl.sync();
}

__global__ void __launch_bounds__(kCtThreads, 1) k_lin_ctail32(CTailParams P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float smem[];
  __shared__ float red[2][32];
  __shared__ float cmax[2];
  __shared__ int done;
  const cg::cluster_group cl = cg::this_cluster();
  const unsigned me = cl.block_rank();
  const int member = blockIdx.x / kCtCtas;
  const bool zero_top = P.zero_init != 0;
  cl.sync();                                    // every CTA of the cluster is running
  // loads: this CTA's slabs of the distributed levels (top: r, q and d unless
  // it starts from zero; below: q), CTA 0: q of its levels
  for (int l = 0; l < P.ndist; ++l) {
    const int n = P.L[l].n, nz = n / kCtCtas, plane = n * n, z0 = (int)me * nz;
    const size_t off = (size_t)member * n * n * n;
    const int slab = nz * plane;
    float* const f = ct_base(smem, P, l);
    const CtCol w(n);
    for (int lz = w.lz0; w.on && lz < nz; lz += w.lzs) {
      const int c = lz * plane + w.x;
      const int g = split_index(w.i, w.j, z0 + lz, n) + (int)off;
      f[9 * slab + c] = P.gq[l][g];
      if (l == 0) {
        f[6 * slab + c] = P.gr[0][g];
        f[7 * slab + c] = P.gr[1][g];
        f[8 * slab + c] = P.gr[2][g];
        if (!zero_top) {
          f[c] = P.gd[0][g];
          f[slab + c] = P.gd[1][g];
          f[2 * slab + c] = P.gd[2][g];
        }
      }
    }
  }
  if (me == 0) {
    for (int l = P.ndist; l < P.nlev; ++l) {
      const int n = P.L[l].n, cells = n * n * n;
      const size_t off = (size_t)member * cells;
      const SLev S = slev(smem + P.ga_off, P.G, l - P.ndist);
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        int p, j, k, colour;
        split_cell(t, n, p, j, k, colour);
        S.q[(2 * p + ((j + k + colour) & 1)) + n * (j + n * k)] = P.gq[l][t + off];
      }
    }
  }
  cl.sync();
  // down: pre-smoothing and residual restriction on the distributed levels
  // above the coarsest
  const int top = P.ndist < P.nlev ? P.ndist : P.nlev - 1;   // levels with a coarser one
  unsigned dzero_mask = 0;
  for (int l = 0; l < top; ++l) {
    const bool zero = l > 0 || zero_top;
    const int jf = l == 0 ? P.jfactor_top : P.jfactor;
    bool dzero = zero;
    if (P.nu1 > 0) {
      ct_smooth(cl, me, smem, P, l, P.nu1, jf, zero, false, red, cmax);
      dzero = false;
    }
    if (dzero) dzero_mask |= 1u << l;
    ct_restrict(cl, me, smem, P, l, dzero);
  }
  if (P.ndist < P.nlev) {
    // CTA 0: the V-cycle over its levels from d = 0
    if (me == 0) tail_vcycle(smem + P.ga_off, P.G, true, red, &done);
    cl.sync();
  } else {
    ct_smooth(cl, me, smem, P, P.nlev - 1, P.G.coarse_sweeps, 1, true, true, red, cmax);
  }
  // up: prolongation + correction and post-smoothing
  for (int l = top - 1; l >= 0; --l) {
    ct_prolong(cl, me, smem, P, l, (dzero_mask >> l) & 1u);
    ct_smooth(cl, me, smem, P, l, P.nu2, l == 0 ? P.jfactor_top : P.jfactor, false, false,
              red, cmax);
  }
  {
    const int n = P.L[0].n, nz = n / kCtCtas, plane = n * n, z0 = (int)me * nz;
    const size_t off = (size_t)member * n * n * n;
    const int slab = nz * plane;
    const float* d = ct_base(smem, P, 0);
    const CtCol w(n);
    for (int lz = w.lz0; w.on && lz < nz; lz += w.lzs) {
      const int c = lz * plane + w.x;
      const int g = split_index(w.i, w.j, z0 + lz, n) + (int)off;
      P.gd[0][g] = d[c];
      P.gd[1][g] = d[slab + c];
      P.gd[2][g] = d[2 * slab + c];
    }
  }
  cl.sync();                                    // no CTA leaves while its memory is read
}

// u += d: u in the natural layout (FP64), d in the colour-split layout (FP32).

// u += d (FP64 += FP32, colour-split d; the exact widening on the integer
// pipe), per component.
__global__ void k_correct64(int n, double* __restrict__ u1, double* __restrict__ u2,
                            double* __restrict__ u3, const float* __restrict__ d1,
                            const float* __restrict__ d2, const float* __restrict__ d3) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  const size_t off = (size_t)member_of(k, n) * n * n * n;
  if (i >= n || j >= n) return;
  u1 += off, u2 += off, u3 += off, d1 += off, d2 += off, d3 += off;
  const int t = (k * n + j) * n + i;
  const int o = split_index(i, j, k, n);
  u1[t] += f2d(__ldg(d1 + o));
  u2[t] += f2d(__ldg(d2 + o));
  u3[t] += f2d(__ldg(d3 + o));
}

// u += d: df state plus the FP32 correction (colour-split), per component.
__global__ void k_correct_df(int n, float2* __restrict__ u1, float2* __restrict__ u2,
                             float2* __restrict__ u3, const float* __restrict__ d1,
                             const float* __restrict__ d2, const float* __restrict__ d3) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
            k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int t = (k * n + j) * n + i;
  const int o = split_index(i, j, k, n);
  df_st(u1, t, df_add_f(df_ld(u1, t), __ldg(d1 + o)));
  df_st(u2, t, df_add_f(df_ld(u2, t), __ldg(d2 + o)));
  df_st(u3, t, df_add_f(df_ld(u3, t), __ldg(d3 + o)));
}

// Blocks of a grid-stride reduction kernel: one full wave (resident blocks per
// SM from the occupancy calculator times the SM count), no more than the work
// needs and than kReduceBlocks partial-sum slots.
template <class Kernel>
int wave_blocks(Kernel kernel, int64_t cells) {
  int dev = 0, sms = 0, occ = 0;
  int nb = kReduceBlocks;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kReduceThreads, 0) ==
          cudaSuccess &&
      occ > 0 && sms > 0)
    nb = occ * sms;
  if (nb > kReduceBlocks) nb = kReduceBlocks;
  const int64_t need = (cells + kReduceThreads - 1) / kReduceThreads;
  if (need < nb) nb = (int)need;
  return nb < 1 ? 1 : nb;
}

struct Ctx32 {
  MixedBufs* mx;
  const pfc_params* p;
  int nl;
  LvlF L[kMaxLevelsMixed];
  int kind[kMaxLevelsMixed];   // PFC_SWEEP_RB or PFC_SWEEP_JACOBI per level
  float w;                     // Jacobi weight
  int jfactor;                 // Jacobi sweeps per requested sweep (coarse levels)
  int jfactor0;                // the same on the finest level
  cudaStream_t st;
  Prof* pr;
  int nb = 1;                  // members of a batched ensemble (fields member after member)
  double* const* fold_u = nullptr;   // FP64 state the finest level's last pass adds d to
};

// `sweeps` damped Jacobi sweeps d -> t -> d ...; the result ends in d.
// in_t: the current iterate is in t (the sweeps run t -> d -> t ...).
cudaError_t jacobi32(const LvlF& L, int sweeps, float w, bool zero_init, float* const* d,
                     float* const* t, float* const* r, const float* q, cudaStream_t st,
                     bool pdl, int nb = 1, bool in_t = false) {
  const int n = L.n;
  const int64_t cells = (int64_t)n * n * n * nb;
  const bool pairs = n % 4 == 0;                // two cells per thread, float2 moves
  const Launch3 g = launch3(pairs ? n / 2 : n, n, n * nb);
  float* src[3] = {d[0], d[1], d[2]};
  float* dst[3] = {t[0], t[1], t[2]};
  if (in_t)
    for (int c = 0; c < 3; ++c) {
      src[c] = t[c];
      dst[c] = d[c];
    }
  int done = 0;
  cudaError_t e = cudaSuccess;
  while (done < sweeps && e == cudaSuccess) {
    const bool z = zero_init && done == 0;
    if (pairs)
      e = launch_k(pdl, z ? k_lin_jacobi32x2<true> : k_lin_jacobi32x2<false>, g.grid, g.block, 0,
                   st, L, w, src[0], src[1], src[2], dst[0], dst[1], dst[2], r[0], r[1], r[2], q);
    else
      e = launch_k(pdl, z ? k_lin_jacobi32<true> : k_lin_jacobi32<false>, g.grid, g.block, 0,
                   st, L, w, src[0], src[1], src[2], dst[0], dst[1], dst[2], r[0], r[1], r[2], q);
    done += 1;
    for (int c = 0; c < 3; ++c) {
      float* x = src[c];
      src[c] = dst[c];
      dst[c] = x;
    }
  }
  if (e == cudaSuccess && src[0] != d[0])
    e = launch_k(pdl, k_copy3, dim3(grid_for(cells)), dim3(kThreads), 0, st, (int)cells, src[0],
                 src[1], src[2], d[0], d[1], d[2]);
  return e;
}

// One colour pass of a red-black sweep on level l.
cudaError_t rb_pass32(const Ctx32& c, int l, int colour, bool zero) {
  const LvlF& L = c.L[l];
  float* const* d = c.mx->d[l];
  float* const* r = c.mx->r[l];
  const float* q = c.mx->q[l];
  const bool pairs = L.n % 4 == 0;              // two cells per thread, float2 moves
  const Launch3 g = launch3(pairs ? L.n / 4 : L.n / 2, L.n, L.n * c.nb);
  if (pairs)
    return launch_k(c.pr == nullptr, zero ? k_lin_smooth32x2<true> : k_lin_smooth32x2<false>,
                    g.grid, g.block, 0, c.st, L, colour, d[0], d[1], d[2], r[0], r[1], r[2], q);
  return launch_k(c.pr == nullptr, zero ? k_lin_smooth32<true> : k_lin_smooth32<false>, g.grid,
                  g.block, 0, c.st, L, colour, d[0], d[1], d[2], r[0], r[1], r[2], q);
}

// The last colour-1 pass of level l with u += d folded in (c.fold_u).
cudaError_t rb_pass32_correct(const Ctx32& c, int l) {
  const LvlF& L = c.L[l];
  float* const* d = c.mx->d[l];
  float* const* r = c.mx->r[l];
  const Launch3 g = launch3(L.n / 4, L.n, L.n * c.nb);
  return launch_k(c.pr == nullptr, k_lin_smooth32x2_correct, g.grid, g.block, 0, c.st, L,
                  (const float*)d[0], (const float*)d[1], (const float*)d[2], (const float*)r[0],
                  (const float*)r[1], (const float*)r[2], (const float*)c.mx->q[l], c.fold_u[0],
                  c.fold_u[1], c.fold_u[2]);
}

// Whether a correction's u += d can fold into the finest level's last
// post-smoothing pass: a red-black finest level with post-smoothing, wide
// enough that no tail launch takes it (more than 32 cells), its rows a
// multiple of four cells (the paired pass).
bool correction_folds(const Ctx32& c) {
  return c.nl >= 2 && c.kind[0] == PFC_SWEEP_RB && c.p->nu2 > 0 && c.L[0].n > kCtMaxN &&
         c.L[0].n % 4 == 0;
}

// `sweeps` post- (or pre-) smoothing sweeps on level l; fold: the last
// colour-1 pass adds the result to c.fold_u (red-black, n % 4 == 0).
cudaError_t smooth32(const Ctx32& c, int l, int sweeps, bool zero_init, bool fold = false) {
  const LvlF& L = c.L[l];
  float* const* d = c.mx->d[l];
  float* const* r = c.mx->r[l];
  const float* q = c.mx->q[l];
  if (sweeps <= 0) return cudaSuccess;
  prof_begin(c.pr, PFC_K_LIN_SMOOTH, c.st);
  if (c.kind[l] == PFC_SWEEP_JACOBI) {
    const int js = sweeps * (l == 0 ? c.jfactor0 : c.jfactor);
    cudaError_t e =
        jacobi32(L, js, c.w, zero_init, d, c.mx->t[l], r, q, c.st, c.pr == nullptr, c.nb);
    prof_end(c.pr, PFC_K_LIN_SMOOTH, l, js, c.st);
    return e;
  }
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < sweeps && e == cudaSuccess; ++s)
    for (int colour = 0; colour < 2 && e == cudaSuccess; ++colour)
      if (!(fold && s == sweeps - 1 && colour == 1))
        e = rb_pass32(c, l, colour, zero_init && s == 0 && colour == 0);
  prof_end(c.pr, PFC_K_LIN_SMOOTH, l, 2 * sweeps - (fold ? 1 : 0), c.st);
  if (e == cudaSuccess && fold) {
    // timed as the correction it replaces
    prof_begin(c.pr, PFC_K_CORRECT, c.st);
    e = rb_pass32_correct(c, l);
    prof_end(c.pr, PFC_K_CORRECT, l, 1, c.st);
  }
  return e;
}

// Whether the prolongation into a level of n^3 cells fuses with the first
// of `sweeps` post-smoothing sweeps (k_lin_prolong_sweep32's tiles).
bool prolong_fuses(int n, int sweeps) { return sweeps > 0 && n >= kPsTX && n % kPsTX == 0; }

template <int TY, int TZ>
cudaError_t launch_prolong_sweep(const Ctx32& c, int l, bool jacobi, bool assign) {
  MixedBufs& mx = *c.mx;
  const int n = c.L[l].n;
  const dim3 grid(n / kPsTX, n / TY, (n / TZ) * c.nb), block(kPsTX * TY);
  auto k = jacobi ? (assign ? k_lin_prolong_sweep32<TY, TZ, true, true>
                            : k_lin_prolong_sweep32<TY, TZ, true, false>)
                  : (assign ? k_lin_prolong_sweep32<TY, TZ, false, true>
                            : k_lin_prolong_sweep32<TY, TZ, false, false>);
  float* const* e = mx.d[l + 1];
  return launch_k(c.pr == nullptr, k, grid, block, 0, c.st, c.L[l], c.w, (const float*)e[0],
                  (const float*)e[1], (const float*)e[2], mx.d[l][0], mx.d[l][1], mx.d[l][2],
                  mx.t[l][0], mx.t[l][1], mx.t[l][2], (const float*)mx.r[l][0],
                  (const float*)mx.r[l][1], (const float*)mx.r[l][2], (const float*)mx.q[l]);
}

// d (+)= P e from level l + 1, then `sweeps` post-smoothing sweeps on level
// l (damped Jacobi sweeps, or red-black sweeps), the prolongation fused into
// the first pass (prolong_fuses must hold).  The result is in d.
cudaError_t prolong_smooth32(const Ctx32& c, int l, bool assign, int sweeps) {
  const bool jacobi = c.kind[l] == PFC_SWEEP_JACOBI;
  prof_begin(c.pr, PFC_K_LIN_PROLONG, c.st);
  cudaError_t e = c.L[l].n >= 64 ? launch_prolong_sweep<8, 4>(c, l, jacobi, assign)
                                 : launch_prolong_sweep<4, 2>(c, l, jacobi, assign);
  prof_end(c.pr, PFC_K_LIN_PROLONG, l, 1, c.st);
  if (e != cudaSuccess) return e;
  if (jacobi) {
    // the first sweep left its result in t
    prof_begin(c.pr, PFC_K_LIN_SMOOTH, c.st);
    e = jacobi32(c.L[l], sweeps - 1, c.w, false, c.mx->d[l], c.mx->t[l], c.mx->r[l], c.mx->q[l],
                 c.st, c.pr == nullptr, c.nb, true);
    prof_end(c.pr, PFC_K_LIN_SMOOTH, l, sweeps - 1, c.st);
    return e;
  }
  prof_begin(c.pr, PFC_K_LIN_SMOOTH, c.st);
  e = rb_pass32(c, l, 1, false);
  prof_end(c.pr, PFC_K_LIN_SMOOTH, l, 1, c.st);
  if (e == cudaSuccess && sweeps > 1) e = smooth32(c, l, sweeps - 1, false);
  return e;
}

cudaError_t tail32(const Ctx32& c, int l0, bool zero_init) {
  MixedBufs& mx = *c.mx;
  TailParams P;
  P.nlev = c.nl - l0;
  P.nu1 = c.p->nu1;
  P.nu2 = c.p->nu2;
  P.jfactor = c.jfactor;
  P.jfactor_top = l0 == 0 ? c.jfactor0 : c.jfactor;
  P.coarse_sweeps = c.p->coarse_sweeps;
  P.zero_init = zero_init ? 1 : 0;
  P.w = c.w;
  for (int l = l0; l < c.nl; ++l) {
    P.L[l - l0] = c.L[l];
    P.kind[l - l0] = c.kind[l];
  }
  for (int q = 0; q < 3; ++q) {
    P.gd[q] = mx.d[l0][q];
    P.gr[q] = mx.r[l0][q];
  }
  P.gq = mx.q[l0];
  int sizes[kMaxLevelsMixed];
  for (int l = 0; l < c.nl; ++l) sizes[l] = c.L[l].n;
  const size_t smem = tail_smem_bytes(sizes, l0, c.nl);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_lin_tail32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTailMaxSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  prof_begin(c.pr, PFC_K_LIN_COARSE, c.st);
  cudaError_t e =
      launch_k(c.pr == nullptr, k_lin_tail32, dim3(c.nb), dim3(kTailThreads), smem, c.st, P);
  prof_end(c.pr, PFC_K_LIN_COARSE, l0, 1, c.st);
  return e;
}

// Levels from l0 that the cluster tail spreads over its CTAs (n a multiple
// of kCtCtas with at least two planes per CTA), and its shared-memory bytes
// per CTA; 0 distributed levels when the cluster tail does not apply.
int ctail_layout(const Ctx32& c, int l0, size_t* smem, int* ga_off) {
  if (c.L[l0].n > kCtMaxN || c.nl - l0 > kTailMaxLevels) return 0;
  int nd = 0;
  size_t floats = 0;
  for (int l = l0; l < c.nl; ++l) {
    const int n = c.L[l].n;
    if (l - l0 != nd || n % kCtCtas != 0 || n / kCtCtas < 2) break;
    floats += (size_t)10 * (n / kCtCtas) * n * n;
    ++nd;
  }
  if (nd == 0) return 0;
  *ga_off = (int)floats;
  for (int l = l0 + nd; l < c.nl; ++l) floats += (size_t)10 * c.L[l].n * c.L[l].n * c.L[l].n;
  *smem = floats * sizeof(float);
  return *smem <= kCtMaxSmem ? nd : 0;
}

// Whether this device runs a cluster of kCtCtas CTAs of kCtThreads threads
// with the largest shared-memory request (checked once per process).
bool ctail_supported() {
  static int state = -1;
  if (state >= 0) return state == 1;
  state = 0;
  if (cudaFuncSetAttribute(k_lin_ctail32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kCtMaxSmem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCtCtas);
  cfg.blockDim = dim3(kCtThreads);
  cfg.dynamicSmemBytes = kCtMaxSmem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCtCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_lin_ctail32, &cfg) == cudaSuccess &&
      clusters > 0)
    state = 1;
  cudaGetLastError();
  return state == 1;
}

cudaError_t ctail32(const Ctx32& c, int l0, bool zero_init, int nd, size_t smem, int ga_off) {
  MixedBufs& mx = *c.mx;
  CTailParams P;
  P.nlev = c.nl - l0;
  P.ndist = nd;
  P.nu1 = c.p->nu1;
  P.nu2 = c.p->nu2;
  P.jfactor = c.jfactor;
  P.jfactor_top = l0 == 0 ? c.jfactor0 : c.jfactor;
  P.zero_init = zero_init ? 1 : 0;
  P.w = c.w;
  for (int l = l0; l < c.nl; ++l) {
    P.L[l - l0] = c.L[l];
    P.kind[l - l0] = c.kind[l];
    P.gq[l - l0] = mx.q[l];
  }
  for (int q = 0; q < 3; ++q) {
    P.gd[q] = mx.d[l0][q];
    P.gr[q] = mx.r[l0][q];
  }
  P.ga_off = ga_off;
  // CTA 0's levels as a single-block tail (its top starts from zero); with
  // no such level only G.coarse_sweeps is used (distributed coarsest solve)
  TailParams& G = P.G;
  G.nlev = c.nl - l0 - nd;
  G.nu1 = c.p->nu1;
  G.nu2 = c.p->nu2;
  G.jfactor = c.jfactor;
  G.jfactor_top = c.jfactor;
  G.coarse_sweeps = c.p->coarse_sweeps;
  G.zero_init = 1;
  G.w = c.w;
  for (int l = l0 + nd; l < c.nl; ++l) {
    G.L[l - l0 - nd] = c.L[l];
    G.kind[l - l0 - nd] = c.kind[l];
  }
  for (int q = 0; q < 3; ++q) {
    G.gd[q] = nullptr;
    G.gr[q] = nullptr;
  }
  G.gq = nullptr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCtCtas * c.nb);
  cfg.blockDim = dim3(kCtThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCtCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = c.pr == nullptr ? 2 : 1;
  prof_begin(c.pr, PFC_K_LIN_COARSE, c.st);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_lin_ctail32, P);
  prof_end(c.pr, PFC_K_LIN_COARSE, l0, 1, c.st);
  return e;
}

// Whether vcycle32 at level l restricts to l + 1 with a launch of its own
// (not the cluster tail, the shared-memory tail or the coarsest solve).
bool restricts_alone(const Ctx32& c, int l) {
  if (c.p->cluster_tail == 1 || l >= c.nl - 1) return false;
  if (c.L[l].n <= kTailMaxN && c.nl - l <= kTailMaxLevels) {
    int sizes[kMaxLevelsMixed];
    for (int q = 0; q < c.nl; ++q) sizes[q] = c.L[q].n;
    if (tail_smem_bytes(sizes, l, c.nl) <= kTailMaxSmem) return false;
  }
  return true;
}

// Levels below l + 1 whose restriction one k_lin_restrict_chain32 launch at
// level l can take over (0..2): they start from d = 0 (no pre-smoothing) and
// would each restrict in a launch of their own.  Only for coarse levels of
// at most kChainMaxNc^3 cells: there a launch costs more than the traffic,
// while the chain's 16 x 4 x 4 blocks read a large level's rows in 64-byte
// pieces (256^3 -> 128^3 took 107 us against 94 us for the row-wide blocks).
constexpr int kChainMaxNc = 64;

int chain_extra(const Ctx32& c, int l) {
  const int nc = c.L[l].n / 2;
  if (c.p->nu1 > 0 || nc > kChainMaxNc || nc % kChTX != 0 || nc % kChTZ != 0) return 0;
  int extra = 0;
  while (extra < 2 && l + 2 + extra < c.nl && restricts_alone(c, l + 1 + extra)) ++extra;
  return extra;
}

// have: the restrictions of this many levels below l were done by a chain
// launch above (r of levels l+1 .. l+have is in place; d = 0 there).
cudaError_t vcycle32(const Ctx32& c, int l, bool zero_init, int have = 0) {
  MixedBufs& mx = *c.mx;
  const LvlF& L = c.L[l];
  // cluster tail: from the first level of at most kCtMaxN^3 cells (mode 1)
  // or only where the single-block tail would start (mode 2)
  if (c.p->cluster_tail == 1 || (c.p->cluster_tail == 2 && L.n <= kTailMaxN)) {
    size_t smem = 0;
    int ga_off = 0;
    const int nd = ctail_layout(c, l, &smem, &ga_off);
    if (nd > 0 && ctail_supported()) return ctail32(c, l, zero_init, nd, smem, ga_off);
  }
  if (L.n <= kTailMaxN && c.nl - l <= kTailMaxLevels) {
    int sizes[kMaxLevelsMixed];
    for (int q = 0; q < c.nl; ++q) sizes[q] = c.L[q].n;
    if (tail_smem_bytes(sizes, l, c.nl) <= kTailMaxSmem) return tail32(c, l, zero_init);
  }
  if (l == c.nl - 1) {
    const int work = L.n * L.n * L.n;
    int threads = ((work + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    prof_begin(c.pr, PFC_K_LIN_COARSE, c.st);
    k_lin_coarse_solve32<<<c.nb, threads, 0, c.st>>>(
        L, c.kind[l], c.w, 400, mx.d[l][0], mx.d[l][1], mx.d[l][2], mx.t[l][0], mx.t[l][1],
        mx.t[l][2], mx.r[l][0], mx.r[l][1], mx.r[l][2], mx.q[l]);
    prof_end(c.pr, PFC_K_LIN_COARSE, l, 1, c.st);
    return cudaGetLastError();
  }
  cudaError_t e = cudaSuccess;
  // without pre-smoothing from a zero start d stays 0 until the prolongation,
  // which then assigns instead of adding
  const bool dzero = c.p->nu1 <= 0 && zero_init;
  if (c.p->nu1 > 0) e = smooth32(c, l, c.p->nu1, zero_init);
  if (e != cudaSuccess) return e;
  const int nc = L.n / 2;
  int below = 0;
  if (have > 0) {
    below = have - 1;
  } else {
    const int extra = chain_extra(c, l);
    prof_begin(c.pr, PFC_K_LIN_RESTRICT, c.st);
    if (extra > 0) {
      float* const* r2 = mx.r[l + 2];
      float* const* r3 = extra > 1 ? mx.r[l + 3] : mx.r[l + 2];
      const dim3 grid(nc / kChTX, nc / kChTY, (nc / kChTZ) * c.nb);
      const dim3 block(kChTX, kChTY, kChTZ);
      auto kern = dzero ? (extra > 1 ? k_lin_restrict_chain32<true, 2>
                                     : k_lin_restrict_chain32<true, 1>)
                        : (extra > 1 ? k_lin_restrict_chain32<false, 2>
                                     : k_lin_restrict_chain32<false, 1>);
      e = launch_k(c.pr == nullptr, kern, grid, block, 0, c.st, L, mx.d[l][0], mx.d[l][1],
                   mx.d[l][2], mx.r[l][0], mx.r[l][1], mx.r[l][2], mx.q[l], mx.r[l + 1][0],
                   mx.r[l + 1][1], mx.r[l + 1][2], r2[0], r2[1], r2[2], r3[0], r3[1], r3[2]);
      below = extra;
    } else {
      const Launch3 gr = launch3(nc, nc, nc * c.nb);
      e = launch_k(c.pr == nullptr,
                   dzero ? k_lin_residual_restrict32<true> : k_lin_residual_restrict32<false>,
                   gr.grid, gr.block, 0, c.st, L, mx.d[l][0], mx.d[l][1], mx.d[l][2],
                   mx.r[l][0], mx.r[l][1], mx.r[l][2], mx.q[l], mx.r[l + 1][0], mx.r[l + 1][1],
                   mx.r[l + 1][2]);
    }
    prof_end(c.pr, PFC_K_LIN_RESTRICT, l, 1, c.st);
  }
  if (e != cudaSuccess) return e;
  if ((e = vcycle32(c, l + 1, true, below)) != cudaSuccess) return e;
  const int post = c.kind[l] == PFC_SWEEP_JACOBI
                       ? c.p->nu2 * (l == 0 ? c.jfactor0 : c.jfactor)
                       : c.p->nu2;
  // fused on Jacobi levels only: on a red-black level the fused colour-0
  // pass formed every colour-1 value of its tile and halo per cell (25 us
  // per launch at 128^3 against 6.1 + 6.5 us for the prolongation's
  // coarse-column carry and the plain pass)
  if (c.kind[l] == PFC_SWEEP_JACOBI && prolong_fuses(L.n, post))
    return prolong_smooth32(c, l, dzero, post);
  const int pz = prolong_planes(nc, 3 * c.nb);
  // a red-black post-smoothing pass of colour 0 comes next: it recomputes
  // the colour-0 cells without reading them
  const bool skip0 = c.kind[l] != PFC_SWEEP_JACOBI && c.p->nu2 > 0;
  prof_begin(c.pr, PFC_K_LIN_PROLONG, c.st);
  e = launch_k(c.pr == nullptr, prolong_kernel(dzero, skip0), prolong_grid(nc, pz, 3 * c.nb),
               dim3(kPrTI * kPrTJ), 0, c.st, L.n, pz, mx.d[l + 1][0], mx.d[l + 1][1],
               mx.d[l + 1][2], mx.d[l][0], mx.d[l][1], mx.d[l][2]);
  prof_end(c.pr, PFC_K_LIN_PROLONG, l, 1, c.st);
  if (e != cudaSuccess) return e;
  return smooth32(c, l, c.p->nu2, false, l == 0 && c.fold_u != nullptr);
}

}  // namespace

// Planes per block of k_defect64_fx: the split of the n planes of a column
// into chunks that minimises the waves of resident blocks times the planes
// per block, ceil(blocks / (SMs x resident blocks per SM)) x (planes + 1/2
// for the extra plane of z halo); 0 if even whole columns need
// more partial-sum slots than `cap` (blocks = column tiles x chunks x
// members).
int fx_planes(int n, int members, int64_t cap) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    sms = 152;
  // resident blocks per SM: the waves are counted in units of sms * occ
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_defect64_fx, kFxTX * kFxTY,
                                                    kFxSmem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int64_t slots = (int64_t)sms * occ;
  const int64_t tiles =
      (int64_t)((n + kFxTX - 1) / kFxTX) * ((n + kFxTY - 1) / kFxTY) * members;
  int best = 0;
  double best_cost = 0.0;
  for (int chunks = 1; chunks <= n; ++chunks) {
    const int zc = (n + chunks - 1) / chunks;
    if ((n + zc - 1) / zc != chunks) continue;   // same split as a smaller count
    const int64_t blocks = tiles * chunks;
    if (blocks > cap || (int64_t)chunks * members > 65535) break;
    const double cost = (double)((blocks + slots - 1) / slots) * (zc + 0.5);
    if (best == 0 || cost < best_cost) {
      best = zc;
      best_cost = cost;
    }
  }
  return best;
}

cudaError_t launch_defect64(const Lvl& L, const double* phi, const double* mu,
                            const double* om, const double* S1, const double* S2,
                            const double* S3, const double* b, float* r1, float* r2, float* r3,
                            float* q, double* partials, double* out, cudaStream_t st,
                            double* lap, int members, const double* c1m, const double* Mx,
                            const double* My, const double* Mz, double* lapmu,
                            double* lapom, bool pdl, int planes, const DecideArgs* da,
                            bool* decided) {
  if (decided) *decided = false;
  if (!Mx) {
    const int64_t cap = (int64_t)kReduceBlocks * kReduceComps;
    int zc = fx_planes(L.n, members, cap);
    if (planes > 0 && zc > 0) {
      // a fixed choice, where its blocks fit the partial-sum buffer and grid
      const int z = planes < L.n ? planes : L.n, ch = (L.n + z - 1) / z;
      const int64_t blocks = (int64_t)((L.n + kFxTX - 1) / kFxTX) *
                             ((L.n + kFxTY - 1) / kFxTY) * ch * members;
      if (blocks <= cap && (int64_t)ch * members <= 65535) zc = z;
    }
    if (zc > 0) {
      const int chunks = (L.n + zc - 1) / zc;
      const dim3 grid((L.n + kFxTX - 1) / kFxTX, (L.n + kFxTY - 1) / kFxTY, chunks * members);
      cudaError_t e = launch_ex(pdl, k_defect64_fx, grid, dim3(kFxTX * kFxTY), kFxSmem, st, L, zc, phi,
                                mu, om, S1, S2, S3, b, r1, r2, r3, q, partials, lap, c1m, lapmu,
                                lapom);
      if (e == cudaSuccess)
        e = launch_reduce1(pdl, partials, (int)(grid.x * grid.y * chunks), out, members, st, da,
                           decided);
      return e;
    }
  }
  // one resident wave over all members: blocks per member = wave / members
  const int wave = wave_blocks(k_defect64<false>, (int64_t)L.n * L.n * L.n * members);
  int nbx = wave / members;
  const int64_t need = ((int64_t)L.n * L.n * L.n + kReduceThreads - 1) / kReduceThreads;
  if (nbx > need) nbx = (int)need;
  if (nbx < 1) nbx = 1;
  if (Mx)
    k_defect64<true><<<dim3(nbx, members), kReduceThreads, 0, st>>>(
        L, phi, mu, om, S1, S2, S3, b, r1, r2, r3, q, partials, lap, c1m, Mx, My, Mz);
  else
    k_defect64<false><<<dim3(nbx, members), kReduceThreads, 0, st>>>(
        L, phi, mu, om, S1, S2, S3, b, r1, r2, r3, q, partials, lap, c1m, Mx, My, Mz);
  k_reduce1<<<members, kReduceThreads, 0, st>>>(partials, nbx, out);
  return cudaGetLastError();
}

cudaError_t launch_defect64_point(const Lvl& L, const double* b, const double* mu,
                                  const double* om, const double* S2, const double* S3, const double* lapb, const double* lapmu,
                                  const double* lapom, float* r1, float* r2, float* r3, float* q,
                                  double* partials, double* out, double* lap, cudaStream_t st,
                                  int members, const double* c1m, bool pdl,
                                  const DecideArgs* da, bool* decided) {
  const int wave = wave_blocks(k_defect64_point, (int64_t)L.n * L.n * L.n * members);
  int nbx = wave / members;
  const int64_t need = ((int64_t)L.n * L.n * L.n + kReduceThreads - 1) / kReduceThreads;
  if (nbx > need) nbx = (int)need;
  if (nbx < 1) nbx = 1;
  cudaError_t e = launch_ex(pdl, k_defect64_point, dim3(nbx, members), dim3(kReduceThreads), 0,
                            st, L, b, mu, om, S2, S3, lapb, lapmu, lapom, r1, r2, r3, q, partials,
                            lap, c1m);
  if (e == cudaSuccess) e = launch_reduce1(pdl, partials, nbx, out, members, st, da, decided);
  return e;
}

cudaError_t launch_start64_point(const Lvl& L, const double* b, const double* mu,
                                 const double* om, const double* lapb, const double* lapc,
                                 const double* lapmu, const double* lapom, double* S2,
                                 double* S3, double* phi_next, float* r1, float* r2, float* r3,
                                 float* q, double* partials, double* out, double* lap,
                                 cudaStream_t st, int members, const double* c1m, bool pdl,
                                 const DecideArgs* da, bool* decided) {
  const int wave = wave_blocks(k_start64_point, (int64_t)L.n * L.n * L.n * members);
  int nbx = wave / members;
  const int64_t need = ((int64_t)L.n * L.n * L.n + kReduceThreads - 1) / kReduceThreads;
  if (nbx > need) nbx = (int)need;
  if (nbx < 1) nbx = 1;
  cudaError_t e = launch_ex(pdl, k_start64_point, dim3(nbx, members), dim3(kReduceThreads), 0,
                            st, L, b, mu, om, lapb, lapc, lapmu, lapom, S2, S3, phi_next, r1, r2,
                            r3, q, partials, lap, c1m);
  if (e == cudaSuccess) e = launch_reduce1(pdl, partials, nbx, out, members, st, da, decided);
  return e;
}

cudaError_t launch_start64_extrap(const Lvl& L, const double* b, const double* c,
                                  const double* lapb, const double* lapc, const double* mu0,
                                  const double* om0, const double* lapmu0,
                                  const double* lapom0, double* mu1, double* om1,
                                  double* lapmu1, double* lapom1, double* S2, double* S3,
                                  double* phi, float* r1, float* r2, float* r3, float* q,
                                  double* partials, double* out, double* lap, cudaStream_t st,
                                  int members, const double* c1m, bool pdl,
                                  const DecideArgs* da, bool* decided) {
  const int wave = wave_blocks(k_start64_extrap, (int64_t)L.n * L.n * L.n * members);
  int nbx = wave / members;
  const int64_t need = ((int64_t)L.n * L.n * L.n + kReduceThreads - 1) / kReduceThreads;
  if (nbx > need) nbx = (int)need;
  if (nbx < 1) nbx = 1;
  cudaError_t e = launch_ex(pdl, k_start64_extrap, dim3(nbx, members), dim3(kReduceThreads), 0,
                            st, L, b, c, lapb, lapc, mu0, om0, lapmu0, lapom0, mu1, om1, lapmu1,
                            lapom1, S2, S3, phi, r1, r2, r3, q, partials, lap, c1m);
  if (e == cudaSuccess) e = launch_reduce1(pdl, partials, nbx, out, members, st, da, decided);
  return e;
}

cudaError_t launch_face_mobility(int n, double m0, double m2, const double* b, const double* c,
                                 double* Mx, double* My, double* Mz, cudaStream_t st) {
  const Launch3 g = launch3(n, n, n);
  k_face_mobility<<<g.grid, g.block, 0, st>>>(n, m0, m2, b, c, Mx, My, Mz);
  return cudaGetLastError();
}

cudaError_t launch_correct64(int n, double* u1, double* u2, double* u3, const float* d1,
                             const float* d2, const float* d3, cudaStream_t st, bool pdl,
                             int members) {
  const Launch3 g = launch3(n, n, n * members);
  return launch_k(pdl, k_correct64, g.grid, g.block, 0, st, n, u1, u2, u3, d1, d2, d3);
}

cudaError_t launch_adj_defect64(const Lvl& L, const double* z1, const double* z2,
                                const double* z3, const double* g, const double* a,
                                const double* b, float* r1, float* r2, float* r3, float* q,
                                double* partials, double* out, cudaStream_t st) {
  const int nb = wave_blocks(k_adj_defect64, (int64_t)L.n * L.n * L.n);
  k_adj_defect64<<<nb, kReduceThreads, 0, st>>>(L, z1, z2, z3, g, a, b, r1, r2, r3, q,
                                                partials);
  k_reduce1<<<1, kReduceThreads, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_adj_accumulate(const Lvl& L, const double* z1, const double* z2,
                                  const double* z3, const double* a, const double* b,
                                  double* gk, double* gkm1, double* partials, double* out,
                                  cudaStream_t st) {
  const int nb = wave_blocks(k_adj_accumulate, (int64_t)L.n * L.n * L.n);
  k_adj_accumulate<<<nb, kReduceThreads, 0, st>>>(L, z1, z2, z3, a, b, gk, gkm1, partials);
  k_reduce1<<<1, kReduceThreads, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_defect_df(const Lvl& L, const float2* phi, const float2* mu,
                             const float2* om, const float2* S1, const float2* S2,
                             const float2* S3, const float2* b, float* r1, float* r2, float* r3,
                             float* q, double* partials, double* out, cudaStream_t st,
                             float2* lap) {
  const int nb = wave_blocks(k_defect_df, (int64_t)L.n * L.n * L.n);
  k_defect_df<<<nb, kReduceThreads, 0, st>>>(to_df(L), phi, mu, om, S1, S2, S3, b, r1, r2, r3,
                                             q, partials, lap);
  k_reduce1<<<1, kReduceThreads, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_source_df(const Lvl& L, const float2* b, const float2* c, float2* S2,
                             float2* S3, cudaStream_t st) {
  const Launch3 g = launch3(L.n, L.n, L.n);
  k_source_df<<<g.grid, g.block, 0, st>>>(to_df(L), b, c, S2, S3);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics_df(int n, const float2* a, const float2* b, double* partials,
                                  double* out, cudaStream_t st) {
  const int nb = wave_blocks(k_diagnostics_df, (int64_t)n * n * n);
  float2* parts = reinterpret_cast<float2*>(partials);
  k_diagnostics_df<<<nb, kReduceThreads, 0, st>>>(n, a, b, parts);
  k_reduce_df6<<<1, kReduceThreads, 0, st>>>(parts, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_guess_df(const Lvl& L, const float2* b, const float2* c, float2* S2,
                            float2* S3, float2* phig, float2* mug, float2* omg,
                            cudaStream_t st) {
  const Launch3 g = launch3(L.n, L.n, L.n);
  const LvlD D = to_df(L);
  k_source_guess_df<<<g.grid, g.block, 0, st>>>(D, b, c, S2, S3, phig, omg);
  k_mu_guess_df<<<g.grid, g.block, 0, st>>>(D, phig, omg, b, S2, mug);
  return cudaGetLastError();
}

cudaError_t launch_round_f32(int64_t count, const double* x, float* y, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_round_f32<<<grid_for(count), kThreads, 0, st>>>(count, x, y);
  return cudaGetLastError();
}

cudaError_t launch_widen_f64(int64_t count, const float* x, double* y, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_widen_f64<<<grid_for(count), kThreads, 0, st>>>(count, x, y);
  return cudaGetLastError();
}

cudaError_t launch_laplacian_df(int n, const float2* v, float2* lap, cudaStream_t st) {
  const Launch3 g = launch3(n, n, n);
  k_laplacian_df<<<g.grid, g.block, 0, st>>>(n, v, lap);
  return cudaGetLastError();
}

cudaError_t launch_source_cached_df(const Lvl& L, const float2* b, const float2* lapb,
                                    const float2* lapc, float2* S2, float2* S3, cudaStream_t st) {
  k_source_cached_df<<<grid_for((int64_t)L.n * L.n * L.n), kThreads, 0, st>>>(to_df(L), b, lapb,
                                                                              lapc, S2, S3);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics_cached_df(int n, const float2* a, const float2* b,
                                         const float2* lapa, const float2* lapb,
                                         double* partials, double* out, cudaStream_t st) {
  const int nb = wave_blocks(k_diagnostics_cached_df, (int64_t)n * n * n);
  float2* parts = reinterpret_cast<float2*>(partials);
  k_diagnostics_cached_df<<<nb, kReduceThreads, 0, st>>>(n, a, b, lapa, lapb, parts);
  k_reduce_df6<<<1, kReduceThreads, 0, st>>>(parts, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_df_from_f64(int64_t count, const double* x, float2* y, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_df_from_f64<<<grid_for(count), kThreads, 0, st>>>(count, x, y);
  return cudaGetLastError();
}

cudaError_t launch_df_to_f64(int64_t count, const float2* y, double* x, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_df_to_f64<<<grid_for(count), kThreads, 0, st>>>(count, y, x);
  return cudaGetLastError();
}

cudaError_t launch_lin_residual_restrict32(const Lvl& L, bool zero, const float* d1,
                                          const float* d2, const float* d3, const float* r1,
                                          const float* r2, const float* r3, const float* q,
                                          float* c1, float* c2, float* c3, cudaStream_t st) {
  const int nc = L.n / 2;
  const Launch3 g = launch3(nc, nc, nc);
  return launch_k(true,
                  zero ? k_lin_residual_restrict32<true> : k_lin_residual_restrict32<false>,
                  g.grid, g.block, 0, st, to_f32(L), d1, d2, d3, r1, r2, r3, q, c1, c2, c3);
}

cudaError_t launch_lin_restrict_chain32(const Lvl& L, bool zero, int extra, const float* d1,
                                       const float* d2, const float* d3, const float* r1,
                                       const float* r2, const float* r3, const float* q,
                                       float* const c[3], float* const e[3], float* const g[3],
                                       cudaStream_t st) {
  const int nc = L.n / 2;
  const dim3 grid(nc / kChTX, nc / kChTY, nc / kChTZ), block(kChTX, kChTY, kChTZ);
  float* const* g2 = extra > 1 ? g : e;
  auto kern = zero ? (extra > 1 ? k_lin_restrict_chain32<true, 2> : k_lin_restrict_chain32<true, 1>)
                   : (extra > 1 ? k_lin_restrict_chain32<false, 2>
                                : k_lin_restrict_chain32<false, 1>);
  return launch_k(true, kern, grid, block, 0, st, to_f32(L), d1, d2, d3, r1, r2, r3, q, c[0],
                  c[1], c[2], e[0], e[1], e[2], g2[0], g2[1], g2[2]);
}

cudaError_t launch_restrict_q(int n, int extra, const float* q, float* c, float* e, float* g,
                              cudaStream_t st) {
  const int nc = n / 2;
  if (extra == 0) {
    const Launch3 l = launch3(nc, nc, nc);
    return launch_k(true, k_restrict32, l.grid, l.block, 0, st, n, q, c);
  }
  const dim3 grid(nc / kChTX, nc / kChTY, nc / kChTZ), block(kChTX, kChTY, kChTZ);
  return launch_k(true, extra > 1 ? k_restrict_chain32<2> : k_restrict_chain32<1>, grid, block, 0,
                  st, n, q, c, e, extra > 1 ? g : e);
}

cudaError_t launch_prolong32(int n, bool assign, bool skip0, const float* e1, const float* e2,
                             const float* e3, float* d1, float* d2, float* d3, cudaStream_t st) {
  const int nc = n / 2, pz = prolong_planes(nc, 3);
  return launch_k(true, prolong_kernel(assign, skip0), prolong_grid(nc, pz, 3),
                  dim3(kPrTI * kPrTJ), 0, st, n, pz, e1, e2, e3, d1, d2, d3);
}

cudaError_t launch_lin_smooth32(const Lvl& L, int sweeps, bool zero_init, float* d1,
                                float* d2, float* d3, const float* r1, const float* r2,
                                const float* r3, const float* q, cudaStream_t st) {
  MixedBufs mx;
  mx.d[0][0] = d1;
  mx.d[0][1] = d2;
  mx.d[0][2] = d3;
  mx.r[0][0] = (float*)r1;
  mx.r[0][1] = (float*)r2;
  mx.r[0][2] = (float*)r3;
  mx.q[0] = (float*)q;
  Ctx32 c;
  c.mx = &mx;
  c.p = nullptr;
  c.nl = 1;
  c.L[0] = to_f32(L);
  c.kind[0] = PFC_SWEEP_RB;
  c.w = 1.f;
  c.jfactor = 1;
  c.jfactor0 = 1;
  c.st = st;
  c.pr = nullptr;
  return smooth32(c, 0, sweeps, zero_init);
}

cudaError_t launch_lin_smooth_correct32(const Lvl& L, int sweeps, float* d1, float* d2,
                                       float* d3, const float* r1, const float* r2,
                                       const float* r3, const float* q, double* u1, double* u2,
                                       double* u3, cudaStream_t st) {
  MixedBufs mx;
  mx.d[0][0] = d1;
  mx.d[0][1] = d2;
  mx.d[0][2] = d3;
  mx.r[0][0] = (float*)r1;
  mx.r[0][1] = (float*)r2;
  mx.r[0][2] = (float*)r3;
  mx.q[0] = (float*)q;
  double* const u[3] = {u1, u2, u3};
  Ctx32 c;
  c.mx = &mx;
  c.p = nullptr;
  c.nl = 1;
  c.L[0] = to_f32(L);
  c.kind[0] = PFC_SWEEP_RB;
  c.w = 1.f;
  c.jfactor = 1;
  c.jfactor0 = 1;
  c.st = st;
  c.pr = nullptr;
  c.fold_u = u;
  return smooth32(c, 0, sweeps, false, true);
}

cudaError_t launch_lin_prolong_smooth32(const Lvl& L, int kind, bool assign, float w,
                                       const float* e1, const float* e2, const float* e3,
                                       float* d1, float* d2, float* d3, float* t1, float* t2,
                                       float* t3, const float* r1, const float* r2,
                                       const float* r3, const float* q, cudaStream_t st) {
  if (!prolong_fuses(L.n, 1)) return cudaErrorInvalidValue;
  MixedBufs mx;
  mx.d[0][0] = d1;
  mx.d[0][1] = d2;
  mx.d[0][2] = d3;
  mx.t[0][0] = t1;
  mx.t[0][1] = t2;
  mx.t[0][2] = t3;
  mx.r[0][0] = (float*)r1;
  mx.r[0][1] = (float*)r2;
  mx.r[0][2] = (float*)r3;
  mx.q[0] = (float*)q;
  mx.d[1][0] = (float*)e1;
  mx.d[1][1] = (float*)e2;
  mx.d[1][2] = (float*)e3;
  Ctx32 c;
  c.mx = &mx;
  c.p = nullptr;
  c.nl = 2;
  c.L[0] = to_f32(L);
  c.kind[0] = kind;
  c.w = w;
  c.jfactor = 1;
  c.jfactor0 = 1;
  c.st = st;
  c.pr = nullptr;
  return prolong_smooth32(c, 0, assign, 1);
}

cudaError_t launch_lin_jacobi32(const Lvl& L, int sweeps, float w, bool zero_init,
                                float* d1, float* d2, float* d3, float* t1, float* t2,
                                float* t3, const float* r1, const float* r2, const float* r3,
                                const float* q, cudaStream_t st) {
  float* d[3] = {d1, d2, d3};
  float* t[3] = {t1, t2, t3};
  float* r[3] = {(float*)r1, (float*)r2, (float*)r3};
  return jacobi32(to_f32(L), sweeps, w, zero_init, d, t, r, q, st, true);
}

cudaError_t launch_correct_df(int n, float2* u1, float2* u2, float2* u3, const float* d1,
                              const float* d2, const float* d3, cudaStream_t st, bool pdl) {
  const Launch3 g = launch3(n, n, n);
  return launch_k(pdl, k_correct_df, g.grid, g.block, 0, st, n, u1, u2, u3, d1, d2, d3);
}

cudaError_t mixed_enqueue_defect(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                 double* const S[3], const double* b, double* partials,
                                 double* dout, cudaStream_t st, Prof* pr, double* lap,
                                 int members, const double* c1m, double* const M[3],
                                 double* lapmu, double* lapom, int planes,
                                 const DecideArgs* da, bool* decided) {
  prof_begin(pr, PFC_K_DEFECT, st);
  cudaError_t e = launch_defect64(L0, u[0], u[1], u[2], S[0], S[1], S[2], b, mx.r[0][0],
                                  mx.r[0][1], mx.r[0][2], mx.q[0], partials, dout, st, lap,
                                  members, c1m, M ? M[0] : nullptr, M ? M[1] : nullptr,
                                  M ? M[2] : nullptr, lapmu, lapom, !pr || pr->mask == 0,
                                  planes, da, decided);
  prof_end(pr, PFC_K_DEFECT, 0, 2, st);
  return e;
}

cudaError_t mixed_enqueue_defect_point(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                       double* const S[3], const double* b,
                                       const double* lapb, const double* lapmu,
                                       const double* lapom, double* lap, double* partials,
                                       double* dout, cudaStream_t st, Prof* pr, int members,
                                       const double* c1m, const DecideArgs* da,
                                       bool* decided) {
  prof_begin(pr, PFC_K_DEFECT, st);
  cudaError_t e = launch_defect64_point(L0, b, u[1], u[2], S[1], S[2], lapb, lapmu, lapom,
                                        mx.r[0][0], mx.r[0][1], mx.r[0][2], mx.q[0], partials,
                                        dout, lap, st, members, c1m, !pr || pr->mask == 0, da,
                                        decided);
  prof_end(pr, PFC_K_DEFECT, 0, 2, st);
  return e;
}

cudaError_t mixed_enqueue_start_point(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                      double* const S[3], const double* b,
                                      const double* lapb, const double* lapc,
                                      const double* lapmu, const double* lapom, double* lap,
                                      double* partials, double* dout, cudaStream_t st, Prof* pr,
                                      int members, const double* c1m, const DecideArgs* da,
                                      bool* decided) {
  prof_begin(pr, PFC_K_START, st);
  cudaError_t e = launch_start64_point(L0, b, u[1], u[2], lapb, lapc, lapmu, lapom, S[1], S[2],
                                       u[0], mx.r[0][0], mx.r[0][1], mx.r[0][2], mx.q[0],
                                       partials, dout, lap, st, members, c1m,
                                       !pr || pr->mask == 0, da, decided);
  prof_end(pr, PFC_K_START, 0, 2, st);
  return e;
}

cudaError_t mixed_enqueue_start_extrap(MixedBufs& mx, const Lvl& L0, double* const u[3],
                                       double* const S[3], const double* b, const double* c,
                                       const double* lapb, const double* lapc,
                                       const double* mu0, const double* om0,
                                       const double* lapmu0, const double* lapom0,
                                       double* lapmu1, double* lapom1, double* lap,
                                       double* partials, double* dout, cudaStream_t st,
                                       Prof* pr, int members, const double* c1m,
                                       const DecideArgs* da, bool* decided) {
  prof_begin(pr, PFC_K_START, st);
  cudaError_t e = launch_start64_extrap(L0, b, c, lapb, lapc, mu0, om0, lapmu0, lapom0, u[1],
                                        u[2], lapmu1, lapom1, S[1], S[2], u[0], mx.r[0][0],
                                        mx.r[0][1], mx.r[0][2], mx.q[0], partials, dout, lap,
                                        st, members, c1m, !pr || pr->mask == 0, da, decided);
  prof_end(pr, PFC_K_START, 0, 2, st);
  return e;
}

cudaError_t mixed_enqueue_defect(MixedBufs& mx, const Lvl& L0, float2* const u[3],
                                 float2* const S[3], const float2* b, double* partials,
                                 double* dout, cudaStream_t st, Prof* pr, float2* lap) {
  prof_begin(pr, PFC_K_DEFECT, st);
  cudaError_t e = launch_defect_df(L0, u[0], u[1], u[2], S[0], S[1], S[2], b, mx.r[0][0],
                                   mx.r[0][1], mx.r[0][2], mx.q[0], partials, dout, st, lap);
  prof_end(pr, PFC_K_DEFECT, 0, 2, st);
  return e;
}

namespace {

// q restricted to every level, then p.inner_cycles FP32 V-cycles on J d = r
// from d = 0 (the part of a correction shared by both outer precisions).
// The FP32 correction solve of one defect correction: the q restrictions,
// then p.inner_cycles V-cycles from d = 0.  u (FP64 state, or nullptr): where
// correction_folds holds, the last V-cycle's last pass adds d to u (*folded
// set), and the caller's u += d launch goes.
cudaError_t mixed_vcycles(MixedBufs& mx, const pfc_params& p, int nl, const int* sizes,
                          cudaStream_t st, Prof* pr, int members, double tau_scale,
                          double* const* u, bool* folded) {
  Ctx32 c;
  c.nb = members;
  c.mx = &mx;
  c.p = &p;
  c.nl = nl;
  c.st = st;
  c.pr = pr;
  c.w = (float)p.jacobi_weight;
  c.jfactor = p.jacobi_factor;
  c.jfactor0 = p.jacobi_factor0;
  double h = p.L / p.n;
  for (int l = 0; l < nl; ++l) {
    // the FP32 operator uses the reference mobility: tau M_ref in row 1
    c.L[l] = to_f32(make_lvl(sizes[l], h, p.eps, p.dt * tau_scale));
    c.kind[l] = level_kind(&p, h);
    h *= 2.0;
  }
  cudaError_t e = cudaSuccess;
  for (int l = 1; l < nl && e == cudaSuccess;) {
    const int nc = sizes[l];
    // up to two more levels in the same launch where the block tiles the level
    int extra = nl - 1 - l;
    if (extra > 2) extra = 2;
    if (nc % kChTX != 0 || nc % kChTZ != 0 || nc % kChTY != 0) extra = 0;
    prof_begin(pr, PFC_K_RESTRICT, st);
    if (extra > 0) {
      const dim3 grid(nc / kChTX, nc / kChTY, (nc / kChTZ) * members),
          block(kChTX, kChTY, kChTZ);
      float* const g2 = extra > 1 ? mx.q[l + 2] : mx.q[l + 1];
      e = launch_k(pr == nullptr, extra > 1 ? k_restrict_chain32<2> : k_restrict_chain32<1>,
                   grid, block, 0, st, sizes[l - 1], (const float*)mx.q[l - 1], mx.q[l],
                   mx.q[l + 1], g2);
    } else {
      const Launch3 g = launch3(nc, nc, nc * members);
      e = launch_k(pr == nullptr, k_restrict32, g.grid, g.block, 0, st, sizes[l - 1],
                   (const float*)mx.q[l - 1], mx.q[l]);
    }
    prof_end(pr, PFC_K_RESTRICT, l - 1, 1, st);
    l += 1 + extra;
  }
  *folded = u != nullptr && p.inner_cycles > 0 && correction_folds(c);
  for (int ic = 0; ic < p.inner_cycles && e == cudaSuccess; ++ic) {
    c.fold_u = (*folded && ic + 1 == p.inner_cycles) ? u : nullptr;
    e = vcycle32(c, 0, ic == 0);
  }
  return e;
}

}  // namespace

cudaError_t mixed_enqueue_correction(MixedBufs& mx, const pfc_params& p, int nl,
                                     const int* sizes, double* const u[3], cudaStream_t st,
                                     Prof* pr, int members, double tau_scale) {
  bool folded = false;
  cudaError_t e = mixed_vcycles(mx, p, nl, sizes, st, pr, members, tau_scale, u, &folded);
  if (e == cudaSuccess && !folded) {
    prof_begin(pr, PFC_K_CORRECT, st);
    e = launch_correct64(p.n, u[0], u[1], u[2], mx.d[0][0], mx.d[0][1], mx.d[0][2], st,
                         pr == nullptr, members);
    prof_end(pr, PFC_K_CORRECT, 0, 1, st);
  }
  return e;
}

cudaError_t mixed_enqueue_correction(MixedBufs& mx, const pfc_params& p, int nl,
                                     const int* sizes, float2* const u[3], cudaStream_t st,
                                     Prof* pr) {
  bool folded = false;
  cudaError_t e = mixed_vcycles(mx, p, nl, sizes, st, pr, 1, 1.0, nullptr, &folded);
  if (e == cudaSuccess) {
    prof_begin(pr, PFC_K_CORRECT, st);
    e = launch_correct_df(p.n, u[0], u[1], u[2], mx.d[0][0], mx.d[0][1], mx.d[0][2], st,
                          pr == nullptr);
    prof_end(pr, PFC_K_CORRECT, 0, 1, st);
  }
  return e;
}

}  // namespace pfc
