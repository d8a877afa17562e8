// Batched streaming tier of the fine two-grid solve (Algorithm 1 steps 2-4) for meshes of
// 1/32 and finer: one kernel per sweep over all samples of a batch, lockstep across samples.
//
// The per-sample kernel keeps a whole sample inside one CTA; on fine meshes its workspace spills
// out of L2 and every sweep waits on DRAM with few warps in flight.  Here each sweep is a
// grid-wide kernel over [sample][node] arrays instead, so the whole GPU streams every array with
// full memory-level parallelism:
//   * MINRES (preconditioned, symmetric indefinite) in the inner precision T, one iteration =
//     K1 (pending w/x update, q = (A - sigma M) z / gamma, partial <q, z>), S1 (scalars),
//     K2 (v_new; z_j is normalised inside the next pending update), the V-cycle, S2 (Givens
//     rotation, convergence);
//   * the V-cycle (nu = 1 or 2 Jacobi steps before and after, Galerkin coarse levels) streams the
//     meshes finer than 1/32.  nu = 2: four kernels per level -- two fused smoothing steps from
//     zero, residual + restriction, prolongation + correction + one smoothing step, one smoothing
//     step (the last one at the finest level also forms <v, z>).  nu = 1: two kernels per level --
//     the residual of x1 = om D^-1 b restricted, prolongation + correction + one smoothing step
//     (+ <v, z>).  The meshes 1/32 .. 1/2 of each sample run inside one CTA in shared memory;
//   * FP64 iterative refinement around the inner solve and the FP64 Rayleigh quotient.
// Partial sums of every reduction are written per (sample, tile) and added in fixed order by
// the scalar kernels: results do not depend on scheduling.  Converged samples are masked out.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <initializer_list>
#include <vector>

#include "mq_device.cuh"
#include "mq_internal.h"

namespace mq {
namespace {

using namespace dev;

// kernels launched by this thread from this file (read by the host API to report launch counts)
thread_local uint64_t tl_launches = 0;

constexpr int kThreads = 256;
constexpr int kPer = 4;                      // nodes per thread per tile
constexpr int kTile = kThreads * kPer;       // nodes per CTA
constexpr int kSub = 32;                     // meshes up to 1/32 run inside one CTA
constexpr int kSubThreads = 128;             // threads of that CTA (more samples per SM than 256)

// Node arrays of the streaming tier: n + 1 rows of sld(n) = n + 4 entries (a multiple of four,
// so every row of an FP32 array starts on a 16-byte boundary and can be moved as float4), node
// (i, j) at j sld(n) + i; the boundary ring (i or j in {0, n}) and the padding columns n+1..n+3
// hold zeros.  The on-chip sub-cycle keeps its own (n+1) x (n+1) layout (bsub, xsub).
__host__ __device__ inline int sld(int n) { return n + 4; }
__host__ __device__ inline size_t ssz(int n) { return (size_t)(n + 1) * (size_t)sld(n); }

// tiles of kTile interior nodes per sample; n * n / kTile (n a power of two) also covers the
// column walk below, whose threads own one column and kPer rows each
__host__ __device__ inline int tiles_interior(int n) { return n * n > kTile ? n * n / kTile : 1; }
__host__ __device__ inline int tiles_padded(int n) { return (int)((ssz(n) + kTile - 1) / kTile); }

// Column walk over tile ch of mesh n: the thread owns column i and the nr = j1 - j0 (1..kPer)
// rows j0 .. j1-1; consecutive threads own consecutive columns, so every row access is coalesced.
// Stencil kernels load the column strip of every operand once (rows j0-1 .. j1 of the stenciled
// vector, the columns beside it, the weights) as one batch of independent loads, then compute the
// nr nodes from registers: per node three values of the stenciled vector instead of five or
// seven, and all of a thread's memory latency overlapped.  Loads past row j1 - 1 are clamped to
// rows the thread owns (their values are unused).  Returns false when the thread owns no node.
__device__ __forceinline__ bool column_walk(int n, int ch, int& i, int& j0, int& nr) {
  const int g = ch * kThreads + threadIdx.x;
  i = (g & (n - 1)) + 1;
  j0 = (g >> ilog2(n)) * kPer + 1;
  nr = min(kPer, n - j0);
  return i < n && j0 < n;
}

// loop over the interior nodes of tile ch of mesh n
template <class F>
__device__ __forceinline__ void for_tile(int n, int ch, F f) {
  const int lg = ilog2(n);
  const int tot = (n - 1) << lg;
  const int ld = sld(n);
  const int q0 = ch * kTile + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int q = q0 + k * kThreads;
    if (q < tot) {
      const int i = (q & (n - 1)) + 1;
      if (i != n) {
        const int j = (q >> lg) + 1;
        f(j * ld + i, i, j);
      }
    }
  }
}

template <typename T>
struct SS {  // per-sample solver scalars
  T gam, gam_old, eta, eta0, c, c_old, s, s_old, ig, c1, c2, cx, ia1, a2, a3, delta, rs;
  T igp;          // 1 / gamma of the previous step: the pending update normalises z_j on the fly
  T sigm;         // lambda_H h^2 / 12: the mass factor of the shifted operator
  double rnorm, bnorm, lam_h;
  double xnorm;   // ||x64||
  double xax, xmx;  // x.Ax and x.Mx of the last FP64 residual pass (the Rayleigh quotient)
  double xsum;      // sum of the nodal values of x64 in that pass (h^2 xsum = integral of x)
  float amax;     // largest centroid coefficient (for the bound ||A - sigma M|| <= 8 amax + sigma h^2)
  float bmax;     // largest reaction coefficient (the bound gains bmax h^2)
  int act_outer;  // refinement still running
  int act;        // inner MINRES running
  int pend;       // a w/x update is pending
  int iters, outer, flags;
};

// block reduction of NV partial sums to part[(b * nch + ch) * NV + i] (butterfly within each warp,
// then a fixed-order sum over the warps)
template <int NV, typename A>
__device__ __forceinline__ void tile_partials(A (&v)[NV], double* part, size_t slot) {
  __shared__ double red[32 * NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = 0, c = NV;
  Butterfly<NV, 16, A>::run(v, lane, base, c);
  if (c >= 1) red[wid * NV + base] = (double)v[0];
  __syncthreads();
  if (wid == 0 && lane < NV) {
    double s = red[lane];
    for (int w = 1; w < nw; ++w) s += red[w * NV + lane];
    part[slot * NV + lane] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// setup
// v / 2 for a sum v of two valid (positive, finite) coefficients, on the integer units: the
// exponent minus one, exact for every positive normal v (GB300 has few FP64 units).  Coefficients
// that fail the checks below are flagged; their weights are then meaningless but harmless.
__device__ __forceinline__ double half_pos(double v) {
  return __longlong_as_double(__double_as_longlong(v) - (1LL << 52));
}

// weights and inverse diagonal of mesh n from per-triangle coefficients (lower plane, upper plane)
// (with hx: BF16 copies of the weights and of om D^-1 for the V(1,1) sweeps of the FP32 path)
// (with rcells: the reaction term of the second test problem of Sec. 5 -- om D^-1 includes the
// lumped reaction h^2/6 sum_{T at p} b_T, written in BF16 to hr for the V(1,1) sweeps; with rxo also
// the reaction's FP32 edge weights for the operator sweep (b averaged over the two triangles of
// the edges to E, N and NE) and the largest b into ss)
template <typename T, typename S>
__global__ void k_weights(int n, int B, const S* __restrict__ cells, size_t cstride, T* __restrict__ wx,
                          T* __restrict__ wy, T* __restrict__ dinv, T om, double* __restrict__ wx64,
                          double* __restrict__ wy64, const int* __restrict__ act, SS<T>* ss,
                          __nv_bfloat16* __restrict__ hx = nullptr, __nv_bfloat16* __restrict__ hy = nullptr,
                          __nv_bfloat16* __restrict__ hd = nullptr, const S* __restrict__ rcells = nullptr,
                          __nv_bfloat16* __restrict__ hr = nullptr, T* __restrict__ rxo = nullptr,
                          T* __restrict__ ryo = nullptr, T* __restrict__ rdo = nullptr) {
  const int nt = tiles_padded(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || (act && !act[b])) return;
  const S* lo = cells + (size_t)b * cstride;
  const S* up = lo + (size_t)n * n;
  const size_t V = ssz(n);
  const int ld = sld(n);
  int bad = 0;
  const S* rlo = rcells ? rcells + (size_t)b * cstride : nullptr;
  const S* rup = rcells ? rlo + (size_t)n * n : nullptr;
  const double hr6 = 1.0 / (6.0 * (double)n * (double)n);
  long long rbits = 0;  // largest reaction coefficient (bit pattern)
  // largest coefficient as the bit pattern of a double: positive doubles order as their bit patterns
  // (the coefficient checks run on the integer units; GB300 has few FP64 units)
  long long mbits = 0;
  constexpr long long kInfBits = 0x7ff0000000000000LL;
  for (int k = 0; k < kPer; ++k) {
    const size_t q = (size_t)ch * kTile + threadIdx.x + k * kThreads;
    if (q >= V) break;
    const int i = (int)(q % ld), j = (int)(q / ld);
    auto LO = [&](int ii, int jj) { return (double)lo[jj * n + ii]; };
    auto UP = [&](int ii, int jj) { return (double)up[jj * n + ii]; };
    T d = T(0);
    double a64 = 0.0, c64 = 0.0;
    if (i <= n - 1 && j >= 1 && j <= n - 1) a64 = half_pos(LO(i, j) + UP(i, j - 1));
    if (i >= 1 && i <= n - 1 && j <= n - 1) c64 = half_pos(UP(i, j) + LO(i - 1, j));
    const T a = T(a64), c = T(c64);
    if (i <= n - 1 && j <= n - 1) {  // every triangle once: a > 0 and not NaN
      const long long bl = __double_as_longlong(LO(i, j)), bu = __double_as_longlong(UP(i, j));
      bad |= !(bl > 0 && bl <= kInfBits) | !(bu > 0 && bu <= kInfBits);
      mbits = max(mbits, max(bl, bu));
    }
    T dr = T(0);
    if (rlo) {
      auto RL = [&](int ii, int jj) { return (double)rlo[jj * n + ii]; };
      auto RU = [&](int ii, int jj) { return (double)rup[jj * n + ii]; };
      if (i <= n - 1 && j <= n - 1) {  // b >= 0 and not NaN
        const long long bl = __double_as_longlong(RL(i, j)), bu = __double_as_longlong(RU(i, j));
        bad |= !(bl >= 0 && bl <= kInfBits) | !(bu >= 0 && bu <= kInfBits);
        rbits = max(rbits, max(bl, bu));
      }
      if (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1)
        dr = T(hr6 * (RL(i, j) + RU(i, j) + RL(i - 1, j) + RU(i, j - 1) + RL(i - 1, j - 1) + RU(i - 1, j - 1)));
      if (rxo) {
        rxo[(size_t)b * V + q] = (i <= n - 1 && j >= 1 && j <= n - 1) ? T(0.5 * (RL(i, j) + RU(i, j - 1))) : T(0);
        ryo[(size_t)b * V + q] = (i >= 1 && i <= n - 1 && j <= n - 1) ? T(0.5 * (RU(i, j) + RL(i - 1, j))) : T(0);
        rdo[(size_t)b * V + q] = (i <= n - 1 && j <= n - 1) ? T(0.5 * (RL(i, j) + RU(i, j))) : T(0);
      }
      if (hr) hr[(size_t)b * V + q] = __float2bfloat16_rn((float)dr);
    }
    if (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1) {
      // the east and north edges are this node's own (a, c); west and south are the neighbours'
      const T ww = T(half_pos(LO(i - 1, j) + UP(i - 1, j - 1))), ws = T(half_pos(UP(i, j - 1) + LO(i - 1, j - 1)));
      d = om / (a + ww + c + ws + dr);  // the damped Jacobi factor omega D^-1 (with the lumped reaction)
    }
    wx[(size_t)b * V + q] = a;
    wy[(size_t)b * V + q] = c;
    dinv[(size_t)b * V + q] = d;
    if (hx) {
      hx[(size_t)b * V + q] = __float2bfloat16_rn((float)a);
      hy[(size_t)b * V + q] = __float2bfloat16_rn((float)c);
      hd[(size_t)b * V + q] = __float2bfloat16_rn((float)d);
    }
    if (wx64) {
      wx64[(size_t)b * V + q] = a64;
      wy64[(size_t)b * V + q] = c64;
    }
  }
  if (ss) {
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ss[b].flags, kFlagBadCoef);
    float amax = (mbits > 0 && mbits <= kInfBits) ? (float)__longlong_as_double(mbits) * 1.0001f : 0.0f;
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomicMax((int*)&ss[b].amax, __float_as_int(amax));  // positive floats order as ints
    if (rlo) {
      float bmx = (rbits > 0 && rbits <= kInfBits) ? (float)__longlong_as_double(rbits) * 1.0001f : 0.0f;
      for (int o = 16; o > 0; o >>= 1) bmx = fmaxf(bmx, __shfl_xor_sync(0xffffffffu, bmx, o));
      if ((threadIdx.x & 31) == 0 && bmx > 0.0f) atomicMax((int*)&ss[b].bmax, __float_as_int(bmx));
    }
  }
}

// per-triangle coefficients of mesh n/2 as means of the four fine triangles each contains
template <typename S, typename T>
__global__ void k_coarsen(int n, int B, const S* __restrict__ in, size_t istride, T* __restrict__ out) {
  const int m = n / 2;
  const size_t mm = (size_t)m * m;
  const int nt = (int)((mm + kTile - 1) / kTile);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B) return;
  const S* lo = in + (size_t)b * istride;
  const S* up = lo + (size_t)n * n;
  T* o = out + (size_t)b * 2 * mm;
  for (int k = 0; k < kPer; ++k) {
    const size_t q = (size_t)ch * kTile + threadIdx.x + k * kThreads;
    if (q >= mm) break;
    const int I = (int)(q % m), J = (int)(q / m), i = 2 * I, j = 2 * J;
    const double l = (double)lo[j * n + i] + (double)lo[j * n + i + 1] + (double)lo[(j + 1) * n + i + 1] +
                     (double)up[j * n + i + 1];
    const double u = (double)up[j * n + i] + (double)up[(j + 1) * n + i + 1] + (double)up[(j + 1) * n + i] +
                     (double)lo[(j + 1) * n + i];
    o[q] = T(0.25 * l);
    o[mm + q] = T(0.25 * u);
  }
}

template <typename S, typename T>
__global__ void k_convert(size_t count, const S* __restrict__ in, T* __restrict__ out) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x)
    out[q] = T(in[q]);
}

// k 2^-l as a double (0 <= k < 2^l, l <= 30), assembled from its bits on the integer units (the
// barycentric coordinates of nested P1 interpolation are such dyadic fractions, exactly)
__device__ __forceinline__ double dyadic(int k, int l) {
  if (k == 0) return 0.0;
  const int msb = 31 - __clz(k);
  const unsigned long long bits = ((unsigned long long)(msb - l + 1023) << 52) |
                                  (((unsigned long long)k << (52 - msb)) & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// P u_H at the fine nodes (into x64) -- padded arrays, ring zero.  In the coarse cell of fine node
// (i, j), with s = (i mod r) / r and t = (j mod r) / r (r = n / nc): on the lower triangle (s >= t)
// P u_H = u00 + s (u10 - u00) + t (u11 - u10), on the upper u00 + t (u01 - u00) + s (u11 - u01) --
// two FP64 differences and two fused multiply-adds per node, the rest on the integer units
template <typename T>
__global__ void k_interp(int n, int nc, int B, const double* __restrict__ uH, double* __restrict__ x64) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B) return;
  const int lr = ilog2(n / nc), rm = (1 << lr) - 1, ldc = nc + 1;
  const double* __restrict__ u = uH + (size_t)b * gsz(nc);
  double* x = x64 + (size_t)b * ssz(n);
  for_tile(n, ch, [&](int p, int i, int j) {
    const int ki = i & rm, kj = j & rm;
    const int c0 = (j >> lr) * ldc + (i >> lr);
    const bool lower = ki >= kj;
    const double u00 = u[c0], u11 = u[c0 + ldc + 1];
    const double uc = lower ? u[c0 + 1] : u[c0 + ldc];
    const double s1 = dyadic(lower ? ki : kj, lr), s2 = dyadic(lower ? kj : ki, lr);
    x[p] = fma(s2, u11 - uc, fma(s1, uc - u00, u00));
  });
}

// b = M (P u_H); v = T(b); partial ||b||^2; x64 cleared afterwards by the caller
template <typename T>
__global__ void k_rhs(int n, int B, const double* __restrict__ x64, double* __restrict__ b64, T* __restrict__ v,
                      double* part) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B) return;
  const int ld = sld(n);
  const double hm = 1.0 / (12.0 * n * n);
  const size_t off = (size_t)b * ssz(n);
  const double* __restrict__ x = x64 + off;
  double acc[1] = {0.0};
  for_tile(n, ch, [&](int p, int, int) {
    const double bv = hm * mass7(x, p, ld);
    b64[off + p] = bv;
    v[off + p] = T(bv);
    acc[0] += bv * bv;
  });
  tile_partials<1, double>(acc, part, (size_t)b * nt + ch);
}

// Sum of sample b's partial slots k = 0..nch-1 (NV values each, part[(b nch + k) NV + i]) by one
// warp: the lanes stride the slots, then an XOR butterfly.  Every lane returns the same totals
// (the summation order is fixed, and each butterfly step adds the same two values on both lanes).
template <int NV>
__device__ __forceinline__ void warp_sum_slots(const double* __restrict__ part, int b, int nch, double (&s)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) s[i] = 0.0;
#pragma unroll 4
  for (int k = lane; k < nch; k += 32) {
    const double* pk = part + ((size_t)b * nch + k) * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] += pk[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
}

// sample of a warp-per-sample scalar kernel (launched with 32 B threads)
__device__ __forceinline__ int warp_sample() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }

template <typename T>
__global__ void k_sc_start(int B, int n, const double* sigma, int sig_stride, int nch, const double* part,
                           SS<T>* ss) {
  const int b = warp_sample();
  if (b >= B) return;
  double t[1];
  warp_sum_slots<1>(part, b, nch, t);
  if ((threadIdx.x & 31) != 0) return;
  const double s = t[0];
  ss[b].sigm = T(sigma[(size_t)b * sig_stride] / (12.0 * n * n));
  SS<T>& S = ss[b];
  S.bnorm = S.rnorm = sqrt(s);
  S.rs = T(1.0 / S.rnorm);
  S.act_outer = S.rnorm > 0.0;
  S.act = 0;
  S.pend = 0;
  S.iters = 0;
  S.outer = 0;
}

// start of a refinement step: samples above tolerance run an inner solve
__host__ __device__ inline double residual_target(double tol, double bnorm, double knorm, double xnorm, double f) {
  const double floor_ = f * 2.220446049250313e-16 * (knorm * xnorm + bnorm);
  const double t = tol * bnorm;
  return t > floor_ ? t : floor_;
}

template <typename T>
__device__ inline double knorm_of(const SS<T>& S, int n, double sigma) {
  return 8.0 * (double)S.amax + ((double)S.bmax + sigma) / ((double)n * n);
}

// start of a refinement step: samples above the residual target run an inner solve (target: tol
// relative to ||b||, but not below a small multiple of the FP64 floor eps (||K|| ||x|| + ||b||))
template <typename T>
__global__ void k_sc_outer_begin(int B, int n, const double* sigma, int sig_stride, double tol_lin, SS<T>* ss,
                                 int* act, int* count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  SS<T>& S = ss[b];
  const double kn = knorm_of(S, n, sigma[(size_t)b * sig_stride]);
  const int a = S.act_outer && (S.rnorm > residual_target(tol_lin, S.bnorm, kn, S.xnorm, 16.0));
  if (!a) S.act_outer = 0;
  S.act = a;
  act[b] = a;
  if (a) atomicAdd(count, 1);
}

// v *= 1/||r||; clear vo, w, wo, xi
template <typename T>
__global__ void k_inner_init(int n, int B, const int* __restrict__ act, const SS<T>* ss, T* v, T* vo, T* w, T* wo,
                             T* xi) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const T rs = ss[b].rs;
  const size_t off = (size_t)b * ssz(n);
  for_tile(n, ch, [&](int p, int, int) {
    v[off + p] *= rs;
    vo[off + p] = T(0);
    w[off + p] = T(0);
    wo[off + p] = T(0);
    xi[off + p] = T(0);
  });
}

// ---------------------------------------------------------------------------------------------
// V-cycle kernels (mesh n > kSub)
// two damped Jacobi steps from zero: x1 = om D^-1 b, x = x1 + om D^-1 (b - A x1); dinv holds om D^-1
template <typename T>
__global__ void k_smooth2_from_zero(int n, int B, const int* __restrict__ act, const T* __restrict__ wx,
                                    const T* __restrict__ wy, const T* __restrict__ dinv, const T* __restrict__ bb,
                                    T* __restrict__ x) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ D = dinv + off;
  const T* __restrict__ R = bb + off;
  T* __restrict__ X = x + off;
  int i, j0, nr;
  if (!column_walk(n, ch, i, j0, nr)) return;
  const int p0 = j0 * ld + i;
  // x1 = om D^-1 b: centre column rows j0-1 .. j0+kPer (clamped), west and east columns
  T dc[kPer + 2], rc[kPer + 2], dw[kPer], rw[kPer], de[kPer], re[kPer], wE[kPer], wW[kPer], yv[kPer + 1];
#pragma unroll
  for (int k = -1; k <= kPer; ++k) {
    const int q = p0 + min(k, nr) * ld;
    dc[k + 1] = D[q];
    rc[k + 1] = R[q];
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int q = p0 + min(k, nr - 1) * ld;
    dw[k] = D[q - 1];
    rw[k] = R[q - 1];
    de[k] = D[q + 1];
    re[k] = R[q + 1];
    wE[k] = W[q];
    wW[k] = W[q - 1];
  }
#pragma unroll
  for (int k = -1; k < kPer; ++k) yv[k + 1] = Y[p0 + min(k, nr - 1) * ld];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (k < nr) {
      const T xc = dc[k + 1] * rc[k + 1];
      const T ax = wE[k] * (xc - de[k] * re[k]) + wW[k] * (xc - dw[k] * rw[k]) +
                   yv[k + 1] * (xc - dc[k + 2] * rc[k + 2]) + yv[k] * (xc - dc[k] * rc[k]);
      X[p0 + k * ld] = xc + dc[k + 1] * (rc[k + 1] - ax);
    }
  }
}

// residual r = b - A x restricted with P^T to the coarse right-hand side
// bc: rows of ldo entries (sld(n/2) for a streamed level, n/2 + 1 for the sub-cycle's input)
template <typename T>
__global__ void k_restrict(int n, int B, const int* __restrict__ act, const T* __restrict__ wx,
                           const T* __restrict__ wy, const T* __restrict__ bb, const T* __restrict__ x,
                           T* __restrict__ bc, int ldo) {
  const int m = n / 2;
  const int nt = tiles_interior(m);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ R = bb + off;
  const T* __restrict__ X = x + off;
  T* __restrict__ C = bc + (size_t)b * (size_t)(m + 1) * ldo;
  for_tile(m, ch, [&](int, int I, int J) {
    const int p = (2 * J) * ld + 2 * I;
    auto res = [&](int q) { return R[q] - stiff<T, T>(W, Y, X, q, ld); };
    C[J * ldo + I] = res(p) + T(0.5) * ((res(p + 1) + res(p - 1)) + (res(p + ld) + res(p - ld)) +
                              (res(p + ld + 1) + res(p - ld - 1)));
  });
}

// t = x + P xc, then one Jacobi step: out = t + om D^-1 (b - A t)
// xc: rows of ldc entries (sld(n/2) for a streamed level, n/2 + 1 for the sub-cycle's output)
template <typename T>
__global__ void k_prolong_smooth(int n, int B, const int* __restrict__ act, const T* __restrict__ wx,
                                 const T* __restrict__ wy, const T* __restrict__ dinv, const T* __restrict__ bb,
                                 const T* __restrict__ x, const T* __restrict__ xc, T* __restrict__ out, int ldc) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ D = dinv + off;
  const T* __restrict__ R = bb + off;
  const T* __restrict__ X = x + off;
  const T* __restrict__ XC = xc + (size_t)b * (size_t)(n / 2 + 1) * ldc;
  T* __restrict__ O = out + off;
  int i, j0, nr;
  if (!column_walk(n, ch, i, j0, nr)) return;
  auto t = [&](int q, int ii, int jj) {  // x + P xc, branch-free P1 interpolation (see vcycle)
    const int c0 = (jj >> 1) * ldc + (ii >> 1);
    return X[q] + T(0.5) * (XC[c0] + XC[c0 + (ii & 1) + (jj & 1) * ldc]);
  };
  const int p0 = j0 * ld + i;
  T tc[kPer + 2], tw[kPer], te[kPer], wE[kPer], wW[kPer], yv[kPer + 1], dd[kPer], rr[kPer];
#pragma unroll
  for (int k = -1; k <= kPer; ++k) {
    const int kk = min(k, nr);
    tc[k + 1] = t(p0 + kk * ld, i, j0 + kk);
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int kk = min(k, nr - 1);
    const int q = p0 + kk * ld;
    tw[k] = t(q - 1, i - 1, j0 + kk);
    te[k] = t(q + 1, i + 1, j0 + kk);
    wE[k] = W[q];
    wW[k] = W[q - 1];
    dd[k] = D[q];
    rr[k] = R[q];
  }
#pragma unroll
  for (int k = -1; k < kPer; ++k) yv[k + 1] = Y[p0 + min(k, nr - 1) * ld];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (k < nr) {
      const T c = tc[k + 1];
      const T ax = wE[k] * (c - te[k]) + wW[k] * (c - tw[k]) + yv[k + 1] * (c - tc[k + 2]) + yv[k] * (c - tc[k]);
      O[p0 + k * ld] = c + dd[k] * (rr[k] - ax);
    }
  }
}

// V(1,1) down-sweep: the one Jacobi step from zero, x1 = om D^-1 b, is pointwise; its residual
// b - A x1 is formed on the fly and restricted with P^T (nothing stored on the fine mesh)
template <typename WT>
__device__ __forceinline__ float wval(WT v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float wval<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <typename T, typename WT>
__device__ __forceinline__ T wget(const WT* p) {
  if constexpr (sizeof(WT) == 2)
    return T(wval(*p));
  else
    return T(*p);
}

// (weights and om D^-1 of type WT: T, or BF16 copies on the FP32 path -- the V-cycle is only the
// preconditioner, and BF16 keeps it symmetric positive definite and spectrally equivalent)
template <typename T, typename WT = T>
__global__ void k_restrict1(int n, int B, const int* __restrict__ act, const WT* __restrict__ wx,
                            const WT* __restrict__ wy, const WT* __restrict__ dinv, const T* __restrict__ bb,
                            T* __restrict__ bc, int ldo) {
  const int m = n / 2;
  const int nt = tiles_interior(m);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const WT* __restrict__ W = wx + off;
  const WT* __restrict__ Y = wy + off;
  const WT* __restrict__ D = dinv + off;
  const T* __restrict__ R = bb + off;
  T* __restrict__ C = bc + (size_t)b * (size_t)(m + 1) * ldo;
  for_tile(m, ch, [&](int, int I, int J) {
    const int p = (2 * J) * ld + 2 * I;
    auto x1 = [&](int q) { return wget<T>(D + q) * R[q]; };
    auto res = [&](int q) {
      const T xq = x1(q);
      return R[q] - (wget<T>(W + q) * (xq - x1(q + 1)) + wget<T>(W + q - 1) * (xq - x1(q - 1)) +
                     wget<T>(Y + q) * (xq - x1(q + ld)) + wget<T>(Y + q - ld) * (xq - x1(q - ld)));
    };
    C[J * ldo + I] = res(p) + T(0.5) * ((res(p + 1) + res(p - 1)) + (res(p + ld) + res(p - ld)) +
                                        (res(p + ld + 1) + res(p - ld - 1)));
  });
}

// V(1,1) up-sweep: t = om D^-1 b + P xc, then one Jacobi step out = t + om D^-1 (b - A t);
// optionally partial <dotv, out>.  Column strips as in k_prolong_smooth.
template <typename T, bool DOT>
__global__ void k_prolong_smooth1(int n, int B, const int* __restrict__ act, const T* __restrict__ wx,
                                  const T* __restrict__ wy, const T* __restrict__ dinv, const T* __restrict__ bb,
                                  const T* __restrict__ xc, int ldc, T* __restrict__ out, const T* __restrict__ dotv,
                                  double* part) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ D = dinv + off;
  const T* __restrict__ R = bb + off;
  const T* __restrict__ XC = xc + (size_t)b * (size_t)(n / 2 + 1) * ldc;
  T* __restrict__ O = out + off;
  T acc[1] = {T(0)};
  for_tile(n, ch, [&](int p, int i, int j) {
    auto t = [&](int q, int ii, int jj) {
      const int c0 = (jj >> 1) * ldc + (ii >> 1);
      return D[q] * R[q] + T(0.5) * (XC[c0] + XC[c0 + (ii & 1) + (jj & 1) * ldc]);
    };
    const T tp = t(p, i, j);
    const T ax = W[p] * (tp - t(p + 1, i + 1, j)) + W[p - 1] * (tp - t(p - 1, i - 1, j)) +
                 Y[p] * (tp - t(p + ld, i, j + 1)) + Y[p - ld] * (tp - t(p - ld, i, j - 1));
    const T o = tp + D[p] * (R[p] - ax);
    O[p] = o;
    if (DOT) acc[0] += dotv[off + p] * o;
  });
  if (DOT) tile_partials<1, T>(acc, part, (size_t)b * nt + ch);
}

// one Jacobi step out = t + om D^-1 (b - A t); optionally partial <dotv, out>
template <typename T, bool DOT>
__global__ void k_smooth(int n, int B, const int* __restrict__ act, const T* __restrict__ wx,
                         const T* __restrict__ wy, const T* __restrict__ dinv, const T* __restrict__ bb,
                         const T* __restrict__ t, T* __restrict__ out, const T* __restrict__ dotv,
                         double* part) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ D = dinv + off;
  const T* __restrict__ R = bb + off;
  const T* __restrict__ X = t + off;
  T* __restrict__ O = out + off;
  T acc[1] = {T(0)};
  int i, j0, nr;
  if (column_walk(n, ch, i, j0, nr)) {
    const int p0 = j0 * ld + i;
    T xc[kPer + 2], xw[kPer], xe[kPer], wE[kPer], wW[kPer], yv[kPer + 1], dd[kPer], rr[kPer], dv[kPer];
#pragma unroll
    for (int k = -1; k <= kPer; ++k) xc[k + 1] = X[p0 + min(k, nr) * ld];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int q = p0 + min(k, nr - 1) * ld;
      xw[k] = X[q - 1];
      xe[k] = X[q + 1];
      wE[k] = W[q];
      wW[k] = W[q - 1];
      dd[k] = D[q];
      rr[k] = R[q];
      if (DOT) dv[k] = dotv[off + q];
    }
#pragma unroll
    for (int k = -1; k < kPer; ++k) yv[k + 1] = Y[p0 + min(k, nr - 1) * ld];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (k < nr) {
        const T c = xc[k + 1];
        const T ax = wE[k] * (c - xe[k]) + wW[k] * (c - xw[k]) + yv[k + 1] * (c - xc[k + 2]) + yv[k] * (c - xc[k]);
        const T o = c + dd[k] * (rr[k] - ax);
        O[p0 + k * ld] = o;
        if (DOT) acc[0] += dv[k] * o;
      }
    }
  }
  if (DOT) tile_partials<1, T>(acc, part, (size_t)b * nt + ch);
}

// per-sample operator arrays of the meshes 1/ns .. 1/2 (sizes from carve_mg_split; with the
// reaction term also the lumped reaction of every level)
template <typename T>
__host__ __device__ size_t sub_weights_bytes(int ns, bool rxn = false) {
  Carver w(nullptr), v(nullptr);
  MGDesc<T> d;
  carve_mg_split<T>(w, v, ns, d, rxn);
  return (w.used() + 255) & ~(size_t)255;
}
template <typename T>
__host__ __device__ size_t sub_vectors_bytes(int ns, bool rxn = false) {
  Carver w(nullptr), v(nullptr);
  MGDesc<T> d;
  v.take<T>(gsz(ns));
  v.take<T>(gsz(ns));
  carve_mg_split<T>(w, v, ns, d, rxn);
  return v.used() + 64;
}

// builds the operator arrays of meshes 1/ns .. 1/2 of every sample once per solve (rcells: the
// reaction coefficient on the same cells, or NULL)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sub_build(int ns, int B, const T* __restrict__ cells,
                                                        char* __restrict__ subw, size_t wbytes,
                                                        const T* __restrict__ rcells) {
  extern __shared__ __align__(16) char sm[];
  __shared__ double red[kRedSlots];
  __shared__ MGDesc<T> mg;
  const int b = blockIdx.x;
  if (b >= B) return;
  Carver w(subw + (size_t)b * wbytes), v(sm);
  MGDesc<T> d;
  v.take<T>(gsz(ns));
  v.take<T>(gsz(ns));
  carve_mg_split<T>(w, v, ns, d, rcells != nullptr);
  if (threadIdx.x == 0) mg = d;
  __syncthreads();
  build_mg<T, T>(mg, cells + (size_t)b * 2 * ns * ns, ns, red, rcells ? rcells + (size_t)b * 2 * ns * ns : nullptr);
}

// meshes 1/ns .. 1/2 of one sample inside one CTA: x = B^{-1} b (operator arrays read from the
// per-sample block built by k_sub_build, vectors in shared memory)
template <typename T>
__global__ void __launch_bounds__(kSubThreads) k_subcycle(int ns, int B, const int* __restrict__ act,
                                                       const char* __restrict__ subw, size_t wbytes,
                                                       const T* __restrict__ bin, T* __restrict__ xout, int ldio,
                                                       int nu, T om, double* part, const T* __restrict__ dotv,
                                                       int rxn) {
  // bin / xout: rows of ldio entries (ns + 1 for the sub-cycle's own arrays, sld(ns) when the
  // whole V-cycle of a streamed mesh runs here); the shared-memory copies have rows of ns + 1
  extern __shared__ __align__(16) char sm[];
  __shared__ MGDesc<T> mg;
  const int b = blockIdx.x;
  if (b >= B || !act[b]) return;
  const size_t V = gsz(ns);
  const int ld = ns + 1;
  Carver w((char*)subw + (size_t)b * wbytes), v(sm);
  MGDesc<T> d;
  T* b0 = v.take<T>(V);
  T* x0 = v.take<T>(V);
  carve_mg_split<T>(w, v, ns, d, rxn != 0);
  if (threadIdx.x == 0) mg = d;
  const T* src = bin + (size_t)b * (size_t)(ns + 1) * ldio;
  for_all(V, [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    b0[q] = src[j * ldio + i];
    x0[q] = T(0);
  });
  for (int l = 0; l < d.L; ++l) {
    zero_vec(d.t[l], d.n[l]);
    if (l) {
      zero_vec(d.x[l], d.n[l]);
      zero_vec(d.b[l], d.n[l]);
    }
  }
  __syncthreads();
  // with dotv (the right-hand side itself, copied to b0) also <v, x>
  T acc[1] = {vcycle<T>(mg, b0, x0, om, dotv ? b0 : nullptr, nu)};
  T* dst = xout + (size_t)b * (size_t)(ns + 1) * ldio;
  for_all(V, [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    dst[j * ldio + i] = x0[q];
  });
  if (dotv) tile_partials<1, T>(acc, part, (size_t)b);
}

// ---------------------------------------------------------------------------------------------
// MINRES sweeps
// K1: pending w/x update; q = (A - sigma M) z * ig; partial <q, z>
// work: NULL, or a device counter of the algorithmic bytes moved (thread 0 of each active CTA adds
// its tile's interior nodes times the bytes per node: 4 arrays without a pending update, 10 with)
template <typename T>
__global__ void k_minres_q(int n, int B, const int* __restrict__ act, const SS<T>* __restrict__ ss,
                           const T* __restrict__ wx, const T* __restrict__ wy, const double* __restrict__ sigma,
                           int sig_stride, const T* __restrict__ z, const T* __restrict__ zp, T* __restrict__ wo,
                           const T* __restrict__ w, T* __restrict__ xi, T* __restrict__ qv, double* part,
                           unsigned long long* work) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  if (work && threadIdx.x == 0) {
    const long tot = (long)(n - 1) << ilog2(n);
    const long q0 = (long)ch * kTile, q1 = q0 + kTile < tot ? q0 + kTile : tot;
    const long nodes = (q1 - q0) - (q1 / n - q0 / n);  // minus the i == n slots of the walk
    atomicAdd(work, (unsigned long long)(nodes * (ss[b].pend ? 10 : 4) * (long)sizeof(T)));
  }
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const SS<T> S = ss[b];
  const T sigm = S.sigm;
  const T* __restrict__ W = wx + off;
  const T* __restrict__ Y = wy + off;
  const T* __restrict__ Z = z + off;
  T acc[1] = {T(0)};
  for_tile(n, ch, [&](int p, int, int) {
    if (S.pend) {
      const T wnew = (zp[off + p] * S.igp - S.a3 * wo[off + p] - S.a2 * w[off + p]) * S.ia1;
      wo[off + p] = wnew;
      xi[off + p] += S.cx * wnew;
    }
    const T kz = (stiff<T, T>(W, Y, Z, p, ld) - sigm * mass7(Z, p, ld)) * S.ig;
    qv[off + p] = kz;
    acc[0] += kz * Z[p];
  });
  tile_partials<1, T>(acc, part, (size_t)b * nt + ch);
}

// ---------------------------------------------------------------------------------------------
// Vectorised FP32 sweeps: each thread owns four consecutive nodes of one row (columns 4m .. 4m+3,
// one float4 of every operand: rows of the streaming layout start on 16-byte boundaries), so a warp
// moves 512 contiguous bytes per operand and row with one instruction.  Stencil neighbours across
// the four-node group come from the float4s of the rows above and below and from two scalars at
// columns 4m-1 and 4m+4.  Column 0 is the boundary: its outputs are written as zero.
constexpr int kVec = 4;

// CTAs per sample of a vectorised sweep over the interior rows of mesh n
__host__ __device__ inline int tiles_vec(int n) {
  const long t = (long)(n - 1) * (n / kVec);
  return (int)((t + kThreads - 1) / kThreads);
}

// row j (1..n-1) and first column 4m of thread tid of tile ch; false beyond the last row
__device__ __forceinline__ bool vec_walk(int n, int ch, int& j, int& c0) {
  const int per_row = n / kVec;
  const int g = ch * kThreads + threadIdx.x;
  j = g / per_row + 1;
  c0 = (g % per_row) * kVec;
  return j < n;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float at(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// K1, vectorised: the pending w/x update, q = (A - sigma M) z * ig and the partial <q, z>; with RX
// the operator is A + B - sigma M, B the reaction matrix from its edge weights rx, ry, rd (edges to
// E, N and NE)
template <bool RX>
__global__ void k_minres_q4(int n, int B, const int* __restrict__ act, const SS<float>* __restrict__ ss,
                            const float* __restrict__ wx, const float* __restrict__ wy, const float* __restrict__ z,
                            const float* __restrict__ zp, float* __restrict__ wo, const float* __restrict__ w,
                            float* __restrict__ xi, float* __restrict__ qv, double* part, unsigned long long* work,
                            const float* __restrict__ rx, const float* __restrict__ ry, const float* __restrict__ rd) {
  const int nt = tiles_vec(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const SS<float> S = ss[b];
  if (work && threadIdx.x == 0) {
    const long tot = (long)(n - 1) * (n / kVec);
    const long g0 = (long)ch * kThreads, g1 = g0 + kThreads < tot ? g0 + kThreads : tot;
    // interior nodes of the tile: four per thread, minus the boundary column of each row start
    const long per_row = n / kVec;
    const long nodes = kVec * (g1 - g0) - ((g1 + per_row - 1) / per_row - (g0 + per_row - 1) / per_row);
    atomicAdd(work, (unsigned long long)(nodes * ((S.pend ? 10 : 4) + (RX ? 3 : 0)) * (long)sizeof(float)));
  }
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  float acc[1] = {0.0f};
  int j, c0;
  if (vec_walk(n, ch, j, c0)) {
    const size_t p = off + (size_t)j * ld + c0;
    if (S.pend) {
      const float4 a = ld4(zp + p), o = ld4(wo + p), ww = ld4(w + p);
      float4 x = ld4(xi + p);
      float4 wn;
      wn.x = (a.x * S.igp - S.a3 * o.x - S.a2 * ww.x) * S.ia1;
      wn.y = (a.y * S.igp - S.a3 * o.y - S.a2 * ww.y) * S.ia1;
      wn.z = (a.z * S.igp - S.a3 * o.z - S.a2 * ww.z) * S.ia1;
      wn.w = (a.w * S.igp - S.a3 * o.w - S.a2 * ww.w) * S.ia1;
      x.x += S.cx * wn.x;
      x.y += S.cx * wn.y;
      x.z += S.cx * wn.z;
      x.w += S.cx * wn.w;
      st4(wo + p, wn);
      st4(xi + p, x);
    }
    const float4 zc = ld4(z + p), zn = ld4(z + p + ld), zs = ld4(z + p - ld);
    const float4 wc = ld4(wx + p), yc = ld4(wy + p), ys = ld4(wy + p - ld);
    const bool first = c0 == 0;
    const float zw = first ? 0.0f : z[p - 1], ze = z[p + kVec], zne = z[p + ld + kVec];
    const float zsw = first ? 0.0f : z[p - ld - 1], wwest = first ? 0.0f : wx[p - 1];
    float4 rxc, ryc, rys, rdc, rds;
    float rxw = 0.0f, rdsw = 0.0f;
    if (RX) {
      rxc = ld4(rx + p);
      ryc = ld4(ry + p);
      rys = ld4(ry + p - ld);
      rdc = ld4(rd + p);
      rds = ld4(rd + p - ld);
      rxw = first ? 0.0f : rx[p - 1];
      rdsw = first ? 0.0f : rd[p - ld - 1];
    }
    const float hmf = 1.0f / (12.0f * (float)n * (float)n);
    float q[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
      const float xp = at(zc, k);
      const float xe = k < 3 ? at(zc, k + 1) : ze, xw = k > 0 ? at(zc, k - 1) : zw;
      const float xn = at(zn, k), xs = at(zs, k);
      const float xne = k < 3 ? at(zn, k + 1) : zne, xsw = k > 0 ? at(zs, k - 1) : zsw;
      const float we = at(wc, k), wwv = k > 0 ? at(wc, k - 1) : wwest;
      const float st = we * (xp - xe) + wwv * (xp - xw) + at(yc, k) * (xp - xn) + at(ys, k) * (xp - xs);
      const float ms = 6.0f * xp + (xe + xw) + (xn + xs) + (xne + xsw);
      float kz = st - S.sigm * ms;
      if (RX) {
        const float rw = k > 0 ? at(rxc, k - 1) : rxw, rsw = k > 0 ? at(rds, k - 1) : rdsw;
        kz += hmf * (at(rxc, k) * (xp + xe) + rw * (xp + xw) + at(ryc, k) * (xp + xn) + at(rys, k) * (xp + xs) +
                     at(rdc, k) * (xp + xne) + rsw * (xp + xsw));
      }
      kz *= S.ig;
      q[k] = (first && k == 0) ? 0.0f : kz;
      acc[0] += q[k] * xp;
    }
    st4(qv + p, make_float4(q[0], q[1], q[2], q[3]));
  }
  tile_partials<1, float>(acc, part, (size_t)b * nt + ch);
}

// K2, vectorised: v_new = q - c1 v - c2 v_old (into vo)
__global__ void k_minres_v4(int n, int B, const int* __restrict__ act, const SS<float>* __restrict__ ss,
                            const float* __restrict__ q, const float* __restrict__ v, float* __restrict__ vo) {
  const int nt = tiles_vec(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const float c1 = ss[b].c1, c2 = ss[b].c2;
  int j, c0;
  if (!vec_walk(n, ch, j, c0)) return;
  const size_t p = (size_t)b * ssz(n) + (size_t)j * sld(n) + c0;
  const float4 a = ld4(q + p), bv = ld4(v + p), o = ld4(vo + p);
  st4(vo + p, make_float4(a.x - c1 * bv.x - c2 * o.x, a.y - c1 * bv.y - c2 * o.y, a.z - c1 * bv.z - c2 * o.z,
                          a.w - c1 * bv.w - c2 * o.w));
}

// V(1,1) up-sweep, vectorised: t = om D^-1 b + P xc at the four nodes and their stencil
// neighbours, then out = t + om D^-1 (b - A t); with DOT also the partial <dotv, out>.  The coarse
// correction P xc (mean of the two coarse values on the coarse edge through each fine node) reads
// the coarse vector with scalar loads (rows of ldc entries).
// four consecutive weights (16-byte aligned FP32, or 8-byte aligned BF16) as a float4
__device__ __forceinline__ float4 ldw4(const float* p) { return ld4(p); }
__device__ __forceinline__ float4 ldw4(const __nv_bfloat16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
  const __nv_bfloat162 c = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
  const float2 fa = __bfloat1622float2(a), fc = __bfloat1622float2(c);
  return make_float4(fa.x, fa.y, fc.x, fc.y);
}

// CTAs per sample of the vectorised restriction: (m - 1) coarse rows x m/2 pairs of coarse nodes
__host__ __device__ inline int tiles_pairs(int m) {
  const long t = (long)(m - 1) * (m / 2);
  return (int)((t + kThreads - 1) / kThreads);
}

// V(1,1) down-sweep, vectorised: the same restriction as k_restrict1 for two coarse nodes (2t, 2t+1)
// of coarse row J per thread.  The thread loads the fine rows 2J-2 .. 2J+2 at columns 4t-4 ..
// 4t+7 as aligned four-wide vectors (BF16 weights, FP32 right-hand side), forms x1 = om D^-1 b on
// the 5 x 7 block it needs, the residual b - A x1 at the 13 fine nodes of the two 7-point
// restrictions, and writes both coarse values.  Columns left of the row start read as zero (the
// coarse node 0 is the boundary and is not written).
// (RX: the multigrid operator is A + D_B, D_B the lumped reaction in dr)
template <typename WT, bool RX = false>
__global__ void k_restrict1_4(int n, int B, const int* __restrict__ act, const WT* __restrict__ wx,
                              const WT* __restrict__ wy, const WT* __restrict__ dinv, const float* __restrict__ bb,
                              float* __restrict__ bc, int ldo, const WT* __restrict__ dr = nullptr) {
  const int m = n / 2, pairs = m / 2;
  const int nt = tiles_pairs(m);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int g = ch * kThreads + threadIdx.x;
  const int J = g / pairs + 1, t = g % pairs;
  if (J > m - 1) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const int c = 4 * t, jc = 2 * J;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // x1 and r on rows jc-2 .. jc+2 (index 0..4), columns c-2 .. c+4 (index 0..6)
  float x1[5][7], rr[5][7];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const size_t row = off + (size_t)(jc - 2 + r) * ld;
    const float4 d0 = c ? ldw4(dinv + row + c - 4) : z4, r0 = c ? ld4(bb + row + c - 4) : z4;
    const float4 d1 = ldw4(dinv + row + c), r1 = ld4(bb + row + c);
    const float4 d2 = ldw4(dinv + row + c + 4), r2 = ld4(bb + row + c + 4);
    const float dv[7] = {d0.z, d0.w, d1.x, d1.y, d1.z, d1.w, d2.x};
    const float rv[7] = {r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x};
    (void)r2;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      x1[r][q] = dv[q] * rv[q];
      rr[r][q] = rv[q];
    }
  }
  // weights: w_x on rows jc-1 .. jc+1 and w_y on rows jc-2 .. jc+1, columns c-2 .. c+3 (index 0..5)
  float wxv[3][6], wyv[4][6];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const size_t row = off + (size_t)(jc - 1 + r) * ld;
    const float4 a0 = c ? ldw4(wx + row + c - 4) : z4, a1 = ldw4(wx + row + c);
    const float v[6] = {a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int q = 0; q < 6; ++q) wxv[r][q] = v[q];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const size_t row = off + (size_t)(jc - 2 + r) * ld;
    const float4 a0 = c ? ldw4(wy + row + c - 4) : z4, a1 = ldw4(wy + row + c);
    const float v[6] = {a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int q = 0; q < 6; ++q) wyv[r][q] = v[q];
  }
  // lumped reaction on rows jc-1 .. jc+1, columns c-2 .. c+3 (index 0..5)
  float drv[3][6];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int q = 0; q < 6; ++q) drv[r][q] = 0.0f;
    if (RX) {
      const size_t row = off + (size_t)(jc - 1 + r) * ld;
      const float4 a0 = c ? ldw4(dr + row + c - 4) : z4, a1 = ldw4(dr + row + c);
      const float v[6] = {a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int q = 0; q < 6; ++q) drv[r][q] = v[q];
    }
  }
  // residual at fine row jc - 2 + r, column c - 2 + q (r = 1..3, q = 1..5)
  auto res = [&](int r, int q) {
    const float xq = x1[r][q];
    float ax = wxv[r - 1][q] * (xq - x1[r][q + 1]) + wxv[r - 1][q - 1] * (xq - x1[r][q - 1]) +
               wyv[r][q] * (xq - x1[r + 1][q]) + wyv[r - 1][q] * (xq - x1[r - 1][q]);
    if (RX) ax += drv[r - 1][q] * xq;
    return rr[r][q] - ax;
  };
  float* __restrict__ C = bc + (size_t)b * (size_t)(m + 1) * ldo + (size_t)J * ldo;
  // coarse node 2t (fine column c: q = 2) and 2t + 1 (fine column c + 2: q = 4)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = 2 + 2 * h;
    const int I = 2 * t + h;
    if (I < 1) continue;
    C[I] = res(2, q) + 0.5f * ((res(2, q + 1) + res(2, q - 1)) + (res(3, q) + res(1, q)) +
                               (res(3, q + 1) + res(1, q - 1)));
  }
}

template <bool DOT, typename WT = float, bool RX = false>
__global__ void k_prolong_smooth1_4(int n, int B, const int* __restrict__ act, const WT* __restrict__ wx,
                                    const WT* __restrict__ wy, const WT* __restrict__ dinv,
                                    const float* __restrict__ bb, const float* __restrict__ xc, int ldc,
                                    float* __restrict__ out, const float* __restrict__ dotv, double* part,
                                    const WT* __restrict__ dr = nullptr) {
  const int nt = tiles_vec(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const float* __restrict__ XC = xc + (size_t)b * (size_t)(n / 2 + 1) * ldc;
  float acc[1] = {0.0f};
  int j, c0;
  if (vec_walk(n, ch, j, c0)) {
    const size_t p = off + (size_t)j * ld + c0;
    // The coarse values under the tile: rows Jb .. Jb + 2 (Jb = (j - 1) / 2), columns c0/2 - 1 ..
    // c0/2 + 2, loaded once (12 loads for the 14 interpolated nodes).  P xc at fine node (ii, jj) is
    // the mean of the coarse values at the two ends of the coarse edge through it: row jj/2, column
    // ii/2 and row jj/2 + (jj mod 2), column ii/2 + (ii mod 2).
    const int Jb = (j - 1) >> 1, cb = (c0 >> 1) - 1, mh = n >> 1;
    float X[3][4];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        X[r][q] = (Jb + r <= mh && cb + q >= 0) ? XC[(Jb + r) * ldc + cb + q] : 0.0f;
    const bool ev = (j & 1) == 0;
    // the two coarse rows of each fine row j - 1, j, j + 1
    float Am[4], Bm[4], A0[4], B0[4], Ap[4], Bp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Am[q] = X[0][q];
      Bm[q] = ev ? X[1][q] : X[0][q];
      A0[q] = ev ? X[1][q] : X[0][q];
      B0[q] = X[1][q];
      Ap[q] = X[1][q];
      Bp[q] = ev ? X[2][q] : X[1][q];
    }
    // fine column c0 + k, k = -1 .. 4: coarse column index (relative to cb) and parity
    auto pcr = [&](const float (&A)[4], const float (&Bv)[4], int k) {
      const int q = ((k + 4) >> 1) - 1, o = k & 1;
      return 0.5f * (A[q] + Bv[q + o]);
    };
    const bool first = c0 == 0;
    const float4 dc = ldw4(dinv + p), rc = ld4(bb + p);
    const float4 dn = ldw4(dinv + p + ld), rn = ld4(bb + p + ld);
    const float4 ds = ldw4(dinv + p - ld), rs = ld4(bb + p - ld);
    const float4 wc = ldw4(wx + p), yc = ldw4(wy + p), ys = ldw4(wy + p - ld);
    const float wwest = first ? 0.0f : wget<float>(wx + p - 1);
    // t along row j at columns c0-1 .. c0+4, and at rows j+1, j-1 under the four nodes
    float tr[kVec + 2], tn[kVec], ts[kVec];
    tr[0] = first ? 0.0f : wget<float>(dinv + p - 1) * bb[p - 1] + pcr(A0, B0, -1);
    tr[kVec + 1] = wget<float>(dinv + p + kVec) * bb[p + kVec] + pcr(A0, B0, kVec);
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
      tr[k + 1] = at(dc, k) * at(rc, k) + pcr(A0, B0, k);
      tn[k] = at(dn, k) * at(rn, k) + pcr(Ap, Bp, k);
      ts[k] = at(ds, k) * at(rs, k) + pcr(Am, Bm, k);
    }
    const float4 drc = RX ? ldw4(dr + p) : make_float4(0.f, 0.f, 0.f, 0.f);
    float o[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
      const float tp = tr[k + 1];
      const float wwv = k > 0 ? at(wc, k - 1) : wwest;
      float ax = at(wc, k) * (tp - tr[k + 2]) + wwv * (tp - tr[k]) + at(yc, k) * (tp - tn[k]) +
                 at(ys, k) * (tp - ts[k]);
      if (RX) ax += at(drc, k) * tp;
      o[k] = (first && k == 0) ? 0.0f : tp + at(dc, k) * (at(rc, k) - ax);
    }
    st4(out + p, make_float4(o[0], o[1], o[2], o[3]));
    if (DOT) {
      const float4 dv = ld4(dotv + p);
      acc[0] = dv.x * o[0] + dv.y * o[1] + dv.z * o[2] + dv.w * o[3];
    }
  }
  if (DOT) tile_partials<1, float>(acc, part, (size_t)b * nt + ch);
}

// K2: v_new = q - c1 v - c2 v_old (into vo).  z_j stays unnormalised: the next pending update
// scales it by 1 / gamma_j (saves a read and a write of z per step)
template <typename T>
__global__ void k_minres_v(int n, int B, const int* __restrict__ act, const SS<T>* __restrict__ ss,
                           const T* __restrict__ q, const T* __restrict__ v, T* __restrict__ vo) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b]) return;
  const size_t off = (size_t)b * ssz(n);
  const T c1 = ss[b].c1, c2 = ss[b].c2;
  for_tile(n, ch, [&](int p, int, int) { vo[off + p] = q[off + p] - c1 * v[off + p] - c2 * vo[off + p]; });
}

// final pending w/x update
template <typename T>
__global__ void k_minres_finish(int n, int B, const int* __restrict__ act, const SS<T>* __restrict__ ss,
                                const T* __restrict__ zp, const T* __restrict__ wo, const T* __restrict__ w,
                                T* __restrict__ xi) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !act[b] || !ss[b].pend) return;
  const size_t off = (size_t)b * ssz(n);
  const SS<T> S = ss[b];
  for_tile(n, ch, [&](int p, int, int) {
    const T wnew = (zp[off + p] * S.igp - S.a3 * wo[off + p] - S.a2 * w[off + p]) * S.ia1;
    xi[off + p] += S.cx * wnew;
  });
}

template <typename T>
__global__ void k_sc_gamma0(int B, int nch, const double* part, const int* act, SS<T>* ss) {
  const int b = warp_sample();
  if (b >= B || !act[b]) return;
  double t[1];
  warp_sum_slots<1>(part, b, nch, t);
  if ((threadIdx.x & 31) != 0) return;
  const double s = t[0];
  SS<T>& S = ss[b];
  const T t0 = T(s);
  const int brk = !(t0 > T(0));
  const T g = brk ? T(1) : sqrt(t0);
  S.gam = g;
  S.eta = S.eta0 = g;
  S.gam_old = T(1);
  S.c = S.c_old = T(1);
  S.s = S.s_old = T(0);
  S.ig = T(1) / g;
  S.pend = 0;
  if (brk) S.flags |= kFlagBreakdown;
}

template <typename T>
__global__ void k_sc_delta(int B, int nch, const double* part, const int* act, SS<T>* ss) {
  const int b = warp_sample();
  if (b >= B || !act[b]) return;
  double t[1];
  warp_sum_slots<1>(part, b, nch, t);
  if ((threadIdx.x & 31) != 0) return;
  const double s = t[0];
  SS<T>& S = ss[b];
  const T delta = T(s) * S.ig;
  S.c1 = delta * S.ig;
  S.c2 = S.gam / S.gam_old;
  S.delta = delta;
}

// Givens step; a converged sample keeps its pending update and leaves the active set after the
// next K1 (which applies it)
// jc (graph mode): the device iteration counter of the inner loop; iteration *jc + joff is the
// last one allowed when it reaches max_inner - 1, and every sample then counts as done (its pending
// update is applied by the next operator sweep, as the host loop's final update would)
template <typename T>
__global__ void k_sc_givens(int B, int nch, const double* part, int* act, SS<T>* ss, T tol, int* count,
                            const int* jc = nullptr, int joff = 0, int max_inner = 0) {
  const int b = warp_sample();
  if (b >= B || !act[b]) return;
  double t[1];
  warp_sum_slots<1>(part, b, nch, t);
  if ((threadIdx.x & 31) != 0) return;
  const double s = t[0];
  SS<T>& S = ss[b];
  T gnew = T(s);
  if (!(gnew >= T(0))) {
    S.flags |= kFlagBreakdown;
    gnew = T(0);
  }
  gnew = sqrt(gnew);
  const T delta = S.delta, gam = S.gam;
  const T al0 = S.c * delta - S.c_old * S.s * gam;
  const T al1 = sqrt(al0 * al0 + gnew * gnew);
  const T al2 = S.s * delta + S.c_old * S.c * gam;
  const T al3 = S.s_old * gam;
  const T ia1 = T(1) / al1;
  const T cn = al0 * ia1, sn = gnew * ia1;
  S.cx = cn * S.eta;
  S.ia1 = ia1;
  S.a2 = al2;
  S.a3 = al3;
  S.eta = -sn * S.eta;
  S.s_old = S.s;
  S.s = sn;
  S.c_old = S.c;
  S.c = cn;
  S.gam_old = gam;
  S.gam = gnew;
  S.igp = S.ig;
  S.ig = gnew > T(0) ? T(1) / gnew : T(0);
  S.pend = 1;
  S.iters += 1;
  const bool capped = jc && *jc + joff + 1 >= max_inner;
  const bool done = fabs(S.eta) <= tol * S.eta0 || gnew == T(0) || capped;
  if (done) S.act = 0;  // leaves after the next K1
  else atomicAdd(count, 1);
}

// samples that converged in the last Givens step leave the active set (K1 applied their update)
template <typename T>
__global__ void k_sc_retire(int B, int* act, SS<T>* ss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !act[b]) return;
  if (!ss[b].act) {
    act[b] = 0;
    ss[b].pend = 0;
  }
}

// x64 += ||r|| xi for samples that ran an inner solve this step
template <typename T>
__global__ void k_outer_update(int n, int B, const SS<T>* __restrict__ ss, const int* __restrict__ ran,
                               const T* __restrict__ xi, double* __restrict__ x64) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !ran[b]) return;
  const size_t off = (size_t)b * ssz(n);
  const double rn = ss[b].rnorm;
  for_tile(n, ch, [&](int p, int, int) { x64[off + p] += rn * (double)xi[off + p]; });
}

// FP64 residual r = b - (A - sigma M) x64 (FP64 edge weights); v = T(r).
// Partials r.r, x.x, x.Ax, x.Mx, sum x: the last pass of a sample gives its Rayleigh quotient and
// its functional.  The two norms only steer the refinement (stopping tests, the scale of the next
// correction, which the following pass measures again), so each thread sums them in FP32: GB300
// issues FP64 at 1/64 of the FP32 rate.  The nodal sum is formed only for the functional (with_sum).
// (rcb: the reaction coefficient's centroid values [B][2 n^2], or NULL; its seven-point form is added
// to the operator, formed on the fly in FP64)
template <typename T>
__global__ void k_residual(int n, int B, const int* __restrict__ ran, const double* __restrict__ wx64,
                           const double* __restrict__ wy64,
                           const double* __restrict__ sigma, int sig_stride, const double* __restrict__ x64,
                           const double* __restrict__ b64, T* __restrict__ v, double* part,
                           const double* __restrict__ rcb, int with_sum) {
  const int nt = tiles_interior(n);
  const int b = blockIdx.x / nt, ch = blockIdx.x % nt;
  if (b >= B || !ran[b]) return;
  const int ld = sld(n);
  const size_t off = (size_t)b * ssz(n);
  const double hm = 1.0 / (12.0 * n * n);
  const double sg = sigma[(size_t)b * sig_stride];
  const double* __restrict__ WX = wx64 + off;
  const double* __restrict__ WY = wy64 + off;
  const double* __restrict__ X = x64 + off;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  float rr = 0.0f, xx = 0.0f;
  const double* RB = rcb ? rcb + (size_t)b * 2 * n * n : nullptr;
  for_tile(n, ch, [&](int p, int i, int j) {
    const double xv = X[p];
    double ax = stiff<double, double>(WX, WY, X, p, ld);
    if (RB) ax += hm * react_cells(RB, n, X, p, ld, i, j);
    const double mx = hm * mass7(X, p, ld);
    const double r = b64[off + p] - (ax - sg * mx);
    const float rf = (float)r, xf = (float)xv;
    v[off + p] = T(r);
    rr = fmaf(rf, rf, rr);
    xx = fmaf(xf, xf, xx);
    acc[2] += xv * ax;
    acc[3] += xv * mx;
    if (with_sum) acc[4] += xv;
  });
  acc[0] = (double)rr;
  acc[1] = (double)xx;
  tile_partials<5, double>(acc, part, (size_t)b * nt + ch);
}

template <typename T>
__global__ void k_sc_outer_end(int B, int nch, const double* part, const int* ran, SS<T>* ss) {
  const int b = warp_sample();
  if (b >= B || !ran[b]) return;
  double t[5];
  warp_sum_slots<5>(part, b, nch, t);
  if ((threadIdx.x & 31) != 0) return;
  const double s = t[0], sx = t[1], sa = t[2], sm = t[3], su = t[4];
  SS<T>& S = ss[b];
  S.xnorm = sqrt(sx);
  S.xax = sa;
  S.xmx = sm;
  S.xsum = su;
  const double rnew = sqrt(s);
  // No progress: stop refining.  Not on the first step: on fine meshes the FP32 rounding of the
  // first inner solution alone leaves an FP64 residual above ||b|| (the operator amplifies its
  // high-frequency part by O(h^-2)); the next step removes it.
  if (S.outer >= 1 && !(rnew < 0.5 * S.rnorm)) S.act_outer = 0;
  S.rnorm = rnew;
  S.rs = T(1.0 / rnew);
  S.outer += 1;
}

// the Rayleigh quotient x.Ax / x.Mx, or with qoi the functional G(x) = h^2 |sum x| / sqrt(x.Mx)
template <typename T>
__global__ void k_sc_rq(int B, int n, const double* sigma, int sig_stride, const SS<T>* ss, double tol_lin,
                        double* lam_out,
                        int lam_stride, int* it_out, int it_stride, int* outer_out, int outer_stride, int* flags,
                        int flag_stride, int qoi) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const SS<T>& S = ss[b];
  lam_out[(size_t)b * lam_stride] = qoi ? fabs(S.xsum) / ((double)n * n * sqrt(S.xmx)) : S.xax / S.xmx;
  it_out[(size_t)b * it_stride] = S.iters;
  outer_out[(size_t)b * outer_stride] = S.outer;
  int f = S.flags;
  const double kn = knorm_of(S, n, sigma[(size_t)b * sig_stride]);
  if (!(S.rnorm <= residual_target(fmax(1e-5, 10.0 * tol_lin), S.bnorm, kn, S.xnorm, 256.0))) f |= kFlagLinNoConv;
  flags[(size_t)b * flag_stride] |= f;
}

// ---------------------------------------------------------------------------------------------
// loop control of the graph mode: conditional WHILE / IF nodes of a CUDA graph, set on the device
__global__ void k_cond_init(cudaGraphConditionalHandle h, int* counter) {
  *counter = 0;
  cudaGraphSetConditional(h, 1u);
}

// after an outer step: continue while samples are still refining and steps are left
__global__ void k_cond_outer(cudaGraphConditionalHandle h, int* counter, const int* count, int max_iter) {
  const int o = ++*counter;
  cudaGraphSetConditional(h, (*count > 0 && o < max_iter) ? 1u : 0u);
}

// after a pair of inner iterations: continue while samples are active and iterations are left
__global__ void k_cond_inner(cudaGraphConditionalHandle h, int* counter, const int* count, int max_iter) {
  *counter += 2;
  cudaGraphSetConditional(h, (*count > 0 && *counter < max_iter) ? 1u : 0u);
}

template <typename T>
__global__ void k_zero(size_t count, T* p) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x)
    p[q] = T(0);
}

template <typename T>
__global__ void k_set_int(int B, int* p, int v) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) p[b] = v;
}

// ---------------------------------------------------------------------------------------------
// host driver
// The operator sweep and the Lanczos update: vectorised kernels for FP32, the row-mapped ones for
// FP64.  Returns the number of partial-sum slots per sample the sweep wrote (for k_sc_delta).
template <typename T>
int launch_minres_q(int n, int B, const int* act, const SS<T>* ss, const T* wx, const T* wy, const double* lamH,
                    int lam_stride, const T* z, const T* zp, T* wo, const T* w, T* xi, T* q, double* part,
                    unsigned long long* work, cudaStream_t st, const T* rx = nullptr, const T* ry = nullptr,
                    const T* rd = nullptr) {
  if constexpr (sizeof(T) == sizeof(float)) {
    (void)lamH;
    (void)lam_stride;
    if (rx)
      k_minres_q4<true><<<B * tiles_vec(n), kThreads, 0, st>>>(n, B, act, ss, wx, wy, z, zp, wo, w, xi, q, part, work,
                                                              rx, ry, rd);
    else
      k_minres_q4<false><<<B * tiles_vec(n), kThreads, 0, st>>>(n, B, act, ss, wx, wy, z, zp, wo, w, xi, q, part, work,
                                                               nullptr, nullptr, nullptr);
    return tiles_vec(n);
  } else {
    k_minres_q<T><<<B * tiles_interior(n), kThreads, 0, st>>>(n, B, act, ss, wx, wy, lamH, lam_stride, z, zp, wo, w,
                                                            xi, q, part, work);
    return tiles_interior(n);
  }
}

template <typename T>
void launch_minres_v(int n, int B, const int* act, const SS<T>* ss, const T* q, const T* v, T* vo, cudaStream_t st) {
  if constexpr (sizeof(T) == sizeof(float))
    k_minres_v4<<<B * tiles_vec(n), kThreads, 0, st>>>(n, B, act, ss, q, v, vo);
  else
    k_minres_v<T><<<B * tiles_interior(n), kThreads, 0, st>>>(n, B, act, ss, q, v, vo);
}

int grid1(size_t count) {
  size_t g = (count + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

template <typename T>
struct Arena {
  int n, B, Ls;  // Ls streaming multigrid levels (meshes n .. > kSub)
  int nu;        // Jacobi sweeps per side of the V-cycle (1 or 2)
  size_t V0;
  T *v, *vo, *z, *zn, *w, *wo, *q, *xi;
  double *x64, *b64;
  double *wx64, *wy64;  // FP64 edge weights of the finest mesh (the residual operator)
  T *wx[kMaxMG], *wy[kMaxMG], *dinv[kMaxMG], *x[kMaxMG], *t[kMaxMG], *b[kMaxMG];
  // FP32 path: BF16 copies of wx, wy, om D^-1 per streaming level, read by the V(1,1) sweeps
  __nv_bfloat16 *hx[kMaxMG], *hy[kMaxMG], *hd[kMaxMG];
  T* cells[kMaxMG];  // per-triangle coefficients of streaming level l >= 1 and of the sub mesh
  // reaction term (FP32 path): the operator's reaction edge weights on the finest mesh, the lumped
  // reaction per streaming level (BF16, V(1,1) sweeps) and the coarsened reaction coefficients
  int rxn;
  T *rx, *ry, *rd;
  __nv_bfloat16* hr[kMaxMG];
  T* rcells[kMaxMG];
  T *bsub, *xsub;
  char* subw;  // per-sample operator arrays of the sub meshes
  size_t subw_bytes;
  double* part;
  SS<T>* ss;
  int *act, *ran, *count;
};

template <typename T>
size_t carve_arena(void* base, int n, int B, Arena<T>& A, bool rxn = false) {
  Carver c(base);
  A.n = n;
  A.B = B;
  A.rxn = rxn ? 1 : 0;
  A.V0 = ssz(n);
  const size_t Bz = (size_t)B;
  A.v = c.take<T>(Bz * A.V0);
  A.vo = c.take<T>(Bz * A.V0);
  A.z = c.take<T>(Bz * A.V0);
  A.zn = c.take<T>(Bz * A.V0);
  A.w = c.take<T>(Bz * A.V0);
  A.wo = c.take<T>(Bz * A.V0);
  A.q = c.take<T>(Bz * A.V0);
  A.xi = c.take<T>(Bz * A.V0);
  A.x64 = c.take<double>(Bz * A.V0);
  A.b64 = c.take<double>(Bz * A.V0);
  A.wx64 = c.take<double>(Bz * A.V0);
  A.wy64 = c.take<double>(Bz * A.V0);
  A.Ls = 0;
  for (int nl = n; nl > kSub; nl >>= 1) ++A.Ls;
  for (int l = 0; l < (A.Ls > 1 ? A.Ls : 1); ++l) {  // level 0 always: the MINRES operator
    const size_t V = ssz(n >> l);
    A.wx[l] = c.take<T>(Bz * V);
    A.wy[l] = c.take<T>(Bz * V);
    A.dinv[l] = c.take<T>(Bz * V);
    A.t[l] = l < A.Ls ? c.take<T>(Bz * V) : nullptr;
    A.x[l] = l ? c.take<T>(Bz * V) : nullptr;
    A.b[l] = l ? c.take<T>(Bz * V) : nullptr;
    const bool h = sizeof(T) == sizeof(float) && l < A.Ls;
    A.hx[l] = h ? c.take<__nv_bfloat16>(Bz * V) : nullptr;
    A.hy[l] = h ? c.take<__nv_bfloat16>(Bz * V) : nullptr;
    A.hd[l] = h ? c.take<__nv_bfloat16>(Bz * V) : nullptr;
    A.hr[l] = (h && rxn) ? c.take<__nv_bfloat16>(Bz * V) : nullptr;
  }
  A.rx = rxn ? c.take<T>(Bz * A.V0) : nullptr;
  A.ry = rxn ? c.take<T>(Bz * A.V0) : nullptr;
  A.rd = rxn ? c.take<T>(Bz * A.V0) : nullptr;
  for (int l = 0; l < kMaxMG; ++l) A.rcells[l] = nullptr;
  for (int l = 1; l <= A.Ls; ++l) {
    const size_t nl = (size_t)(n >> l);
    A.cells[l] = c.take<T>(Bz * 2 * nl * nl);
    if (rxn) A.rcells[l] = c.take<T>(Bz * 2 * nl * nl);
  }
  const int ns = n >> A.Ls;  // sub mesh (== n when n <= kSub)
  if (A.Ls == 0) {
    A.cells[0] = c.take<T>(Bz * 2 * (size_t)ns * ns);
    if (rxn) A.rcells[0] = c.take<T>(Bz * 2 * (size_t)ns * ns);
  }
  A.bsub = A.Ls ? c.take<T>(Bz * gsz(ns)) : nullptr;
  A.xsub = A.Ls ? c.take<T>(Bz * gsz(ns)) : nullptr;
  A.subw_bytes = sub_weights_bytes<T>(ns, rxn);
  A.subw = c.take<char>(Bz * A.subw_bytes + 256);
  A.subw = (char*)(((uintptr_t)A.subw + 255) & ~(uintptr_t)255);
  const int nch = tiles_interior(n) > 1 ? tiles_interior(n) : 1;
  A.part = c.take<double>(Bz * nch * 5 + Bz);
  A.ss = c.take<SS<T>>(Bz);
  A.act = c.take<int>(Bz);
  A.ran = c.take<int>(Bz);
  A.count = c.take<int>(4);
  return c.used();
}

#define LAUNCH_CHECK()                          \
  do {                                          \
    cudaError_t e_ = cudaGetLastError();        \
    if (e_ != cudaSuccess) return e_;           \
  } while (0)

// V-cycle over the arena hierarchy: x0 = B^{-1} b0; with dotv, partial <dotv, x0> into part
template <typename T>
cudaError_t vcycle_stream(Arena<T>& A, const T* b0, T* x0, const int* act, T om, const T* dotv, double* part,
                          size_t sub_smem, cudaStream_t st) {
  const int n = A.n, B = A.B;
  if (A.Ls == 0) {
    ++tl_launches, k_subcycle<T><<<B, kSubThreads, sub_smem, st>>>(n, B, act, A.subw, A.subw_bytes, b0, x0, sld(n), A.nu,
                                                                   om, part, dotv, A.rxn);
    LAUNCH_CHECK();
    return cudaSuccess;
  }
  if (A.nu == 1) {
    for (int l = 0; l < A.Ls; ++l) {
      const int nl = n >> l;
      const T* b = l ? A.b[l] : b0;
      T* bc = (l + 1 < A.Ls) ? A.b[l + 1] : A.bsub;
      const int ldo = (l + 1 < A.Ls) ? sld(nl / 2) : nl / 2 + 1;
      if constexpr (sizeof(T) == sizeof(float)) {
        if (A.hx[l]) {
          if (A.hr[l])
            ++tl_launches, k_restrict1_4<__nv_bfloat16, true><<<B * tiles_pairs(nl / 2), kThreads, 0, st>>>(
                nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, bc, ldo, A.hr[l]);
          else
            ++tl_launches, k_restrict1_4<__nv_bfloat16><<<B * tiles_pairs(nl / 2), kThreads, 0, st>>>(
                nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, bc, ldo);
          LAUNCH_CHECK();
          continue;
        }
      }
      if (A.hx[l])
        ++tl_launches, k_restrict1<T, __nv_bfloat16><<<B * tiles_interior(nl / 2), kThreads, 0, st>>>(
            nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, bc, ldo);
      else
        ++tl_launches, k_restrict1<T><<<B * tiles_interior(nl / 2), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l],
                                                                                     A.dinv[l], b, bc, ldo);
      LAUNCH_CHECK();
    }
    const int ns = n >> A.Ls;
    ++tl_launches, k_subcycle<T><<<B, kSubThreads, sub_smem, st>>>(ns, B, act, A.subw, A.subw_bytes, A.bsub, A.xsub,
                                                                   ns + 1, 1, om, nullptr, nullptr, A.rxn);
    LAUNCH_CHECK();
    for (int l = A.Ls - 1; l >= 0; --l) {
      const int nl = n >> l;
      const T* b = l ? A.b[l] : b0;
      T* xa = l ? A.x[l] : x0;
      const T* xc = (l + 1 < A.Ls) ? A.x[l + 1] : A.xsub;
      const int ldc = (l + 1 < A.Ls) ? sld(nl / 2) : nl / 2 + 1;
      if constexpr (sizeof(T) == sizeof(float)) {
        if (A.hr[l]) {
          if (l == 0 && dotv)
            ++tl_launches, k_prolong_smooth1_4<true, __nv_bfloat16, true><<<B * tiles_vec(nl), kThreads, 0, st>>>(
                nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, xc, ldc, xa, dotv, part, A.hr[l]);
          else
            ++tl_launches, k_prolong_smooth1_4<false, __nv_bfloat16, true><<<B * tiles_vec(nl), kThreads, 0, st>>>(
                nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, xc, ldc, xa, nullptr, nullptr, A.hr[l]);
        } else if (l == 0 && dotv) {
          ++tl_launches, k_prolong_smooth1_4<true, __nv_bfloat16><<<B * tiles_vec(nl), kThreads, 0, st>>>(
              nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, xc, ldc, xa, dotv, part);
        } else {
          ++tl_launches, k_prolong_smooth1_4<false, __nv_bfloat16><<<B * tiles_vec(nl), kThreads, 0, st>>>(
              nl, B, act, A.hx[l], A.hy[l], A.hd[l], b, xc, ldc, xa, nullptr, nullptr);
        }
      } else {
        if (l == 0 && dotv)
          ++tl_launches, k_prolong_smooth1<T, true><<<B * tiles_interior(nl), kThreads, 0, st>>>(
              nl, B, act, A.wx[l], A.wy[l], A.dinv[l], b, xc, ldc, xa, dotv, part);
        else
          ++tl_launches, k_prolong_smooth1<T, false><<<B * tiles_interior(nl), kThreads, 0, st>>>(
              nl, B, act, A.wx[l], A.wy[l], A.dinv[l], b, xc, ldc, xa, nullptr, nullptr);
      }
      LAUNCH_CHECK();
    }
    return cudaSuccess;
  }
  for (int l = 0; l < A.Ls; ++l) {
    const int nl = n >> l;
    const T* b = l ? A.b[l] : b0;
    T* xa = l ? A.x[l] : x0;
    ++tl_launches, k_smooth2_from_zero<T><<<B * tiles_interior(nl), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l], A.dinv[l],
                                                                       b, xa);
    LAUNCH_CHECK();
    T* bc = (l + 1 < A.Ls) ? A.b[l + 1] : A.bsub;
    const int ldo = (l + 1 < A.Ls) ? sld(nl / 2) : nl / 2 + 1;
    ++tl_launches, k_restrict<T><<<B * tiles_interior(nl / 2), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l], b, xa, bc,
                                                                                ldo);
    LAUNCH_CHECK();
  }
  const int ns = n >> A.Ls;
  ++tl_launches, k_subcycle<T><<<B, kSubThreads, sub_smem, st>>>(ns, B, act, A.subw, A.subw_bytes, A.bsub, A.xsub, ns + 1,
                                                                 A.nu, om, nullptr, nullptr, A.rxn);
  LAUNCH_CHECK();
  for (int l = A.Ls - 1; l >= 0; --l) {
    const int nl = n >> l;
    const T* b = l ? A.b[l] : b0;
    T* xa = l ? A.x[l] : x0;
    const T* xc = (l + 1 < A.Ls) ? A.x[l + 1] : A.xsub;
    const int ldc = (l + 1 < A.Ls) ? sld(nl / 2) : nl / 2 + 1;
    ++tl_launches, k_prolong_smooth<T><<<B * tiles_interior(nl), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l], A.dinv[l], b,
                                                                    xa, xc, A.t[l], ldc);
    LAUNCH_CHECK();
    if (l == 0 && dotv)
      ++tl_launches, k_smooth<T, true><<<B * tiles_interior(nl), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l], A.dinv[l], b,
                                                                    A.t[l], xa, dotv, part);
    else
      ++tl_launches, k_smooth<T, false><<<B * tiles_interior(nl), kThreads, 0, st>>>(nl, B, act, A.wx[l], A.wy[l], A.dinv[l], b,
                                                                     A.t[l], xa, nullptr, nullptr);
    LAUNCH_CHECK();
  }
  return cudaSuccess;
}

int read_count(const int* d_count, cudaStream_t st, cudaError_t& err) {
  int h = 0;
  err = cudaMemcpyAsync(&h, d_count, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  return h;
}

// Graph mode: a WHILE node of the graph being captured on `st`, after the work captured so far; its
// body is captured on `body` until close_while.  The node's condition starts at 1 (k_cond_init
// before the node sets it, and resets the loop counter) and is set by a kernel at the body's end.
// a conditional handle of the graph being captured on st
cudaError_t make_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, 0u, 0u);
}

cudaError_t open_while(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return e;
  return cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
}

cudaError_t close_while(cudaStream_t body) {
  cudaGraph_t g = nullptr;
  return cudaStreamEndCapture(body, &g);
}

template <typename T>
cudaError_t stream_solve_t(const StreamSolve& s, void* arena, cudaStream_t st, const StreamGraph* sg) {
  Arena<T> A;
  // the reaction term runs on the FP32 path with V(1,1) smoothing
  if (s.b && (sizeof(T) != sizeof(float) || s.nu != 1)) return cudaErrorNotSupported;
  carve_arena<T>(arena, s.n, s.B, A, s.b != nullptr);
  A.nu = s.nu == 1 ? 1 : 2;
  const int n = s.n, B = s.B;
  const int nt = tiles_interior(n);
  const size_t Bz = (size_t)B;
  const T om = T(s.omega);
  const int ns = n >> A.Ls;
  const size_t sub_smem = sub_vectors_bytes<T>(ns, A.rxn != 0);
  cudaError_t e = raise_smem_limit((const void*)k_subcycle<T>, (int)sub_smem);
  if (e != cudaSuccess) return e;
  e = raise_smem_limit((const void*)k_sub_build<T>, (int)sub_smem);
  if (e != cudaSuccess) return e;
  const int gs = (B + 255) / 256;
  const int gw = (B + 7) / 8;  // warp-per-sample scalar kernels: 8 samples per 256-thread block
  // ---- clear vectors (boundary rings must be zero), build the operators
  const size_t V0 = A.V0;
  T* const vecs[8] = {A.v, A.vo, A.z, A.zn, A.w, A.wo, A.q, A.xi};
  for (int k = 0; k < 8; ++k) {
    ++tl_launches, k_zero<T><<<grid1(Bz * V0), 256, 0, st>>>(Bz * V0, vecs[k]);
    LAUNCH_CHECK();
  }
  ++tl_launches, k_zero<double><<<grid1(Bz * V0), 256, 0, st>>>(Bz * V0, A.x64);
  ++tl_launches, k_zero<double><<<grid1(Bz * V0), 256, 0, st>>>(Bz * V0, A.b64);
  for (int l = 0; l < A.Ls; ++l) {
    const size_t V = ssz(n >> l);
    T* const lv[3] = {A.t[l], A.x[l], A.b[l]};
    for (int k = 0; k < 3; ++k)
      if (lv[k]) ++tl_launches, k_zero<T><<<grid1(Bz * V), 256, 0, st>>>(Bz * V, lv[k]);
  }
  if (A.Ls) {
    ++tl_launches, k_zero<T><<<grid1(Bz * gsz(ns)), 256, 0, st>>>(Bz * gsz(ns), A.bsub);
    ++tl_launches, k_zero<T><<<grid1(Bz * gsz(ns)), 256, 0, st>>>(Bz * gsz(ns), A.xsub);
  }
  ++tl_launches, k_zero<int><<<grid1(Bz * sizeof(SS<T>) / sizeof(int)), 256, 0, st>>>(Bz * sizeof(SS<T>) / sizeof(int), (int*)A.ss);
  LAUNCH_CHECK();
  const size_t astride = (size_t)2 * n * n;
  for (int l = 0; l < (A.Ls > 1 ? A.Ls : 1); ++l) {
    const int nl = n >> l;
    if (l == 0)
      ++tl_launches, k_weights<T, double><<<B * tiles_padded(nl), kThreads, 0, st>>>(nl, B, s.a, astride, A.wx[0], A.wy[0],
                                                                     A.dinv[0], om, A.wx64, A.wy64, nullptr, A.ss,
                                                                     A.hx[0], A.hy[0], A.hd[0], s.b, A.hr[0], A.rx,
                                                                     A.ry, A.rd);
    else
      ++tl_launches, k_weights<T, T><<<B * tiles_padded(nl), kThreads, 0, st>>>(nl, B, A.cells[l], (size_t)2 * nl * nl, A.wx[l],
                                                                A.wy[l], A.dinv[l], om, nullptr, nullptr, nullptr, nullptr,
                                                                A.hx[l], A.hy[l], A.hd[l], A.rcells[l], A.hr[l]);
    LAUNCH_CHECK();
    if (l >= A.Ls) continue;
    const int m = nl / 2;
    const int ntc = (int)(((size_t)m * m + kTile - 1) / kTile);
    if (l == 0) {
      ++tl_launches, k_coarsen<double, T><<<B * ntc, kThreads, 0, st>>>(nl, B, s.a, astride, A.cells[1]);
      if (A.rxn) ++tl_launches, k_coarsen<double, T><<<B * ntc, kThreads, 0, st>>>(nl, B, s.b, astride, A.rcells[1]);
    } else {
      ++tl_launches, k_coarsen<T, T><<<B * ntc, kThreads, 0, st>>>(nl, B, A.cells[l], (size_t)2 * nl * nl, A.cells[l + 1]);
      if (A.rxn)
        ++tl_launches, k_coarsen<T, T><<<B * ntc, kThreads, 0, st>>>(nl, B, A.rcells[l], (size_t)2 * nl * nl,
                                                                     A.rcells[l + 1]);
    }
    LAUNCH_CHECK();
  }
  if (A.Ls == 0) {
    ++tl_launches, k_convert<double, T><<<grid1(Bz * astride), 256, 0, st>>>(Bz * astride, s.a, A.cells[0]);
    if (A.rxn) ++tl_launches, k_convert<double, T><<<grid1(Bz * astride), 256, 0, st>>>(Bz * astride, s.b, A.rcells[0]);
    LAUNCH_CHECK();
  }
  ++tl_launches, k_sub_build<T><<<B, kThreads, sub_smem, st>>>(ns, B, A.cells[A.Ls], A.subw, A.subw_bytes,
                                                                A.rcells[A.Ls]);
  LAUNCH_CHECK();
  // ---- right-hand side b = M P u_H
  ++tl_launches, k_interp<T><<<B * nt, kThreads, 0, st>>>(n, s.nc, B, s.uH, A.x64);
  LAUNCH_CHECK();
  ++tl_launches, k_rhs<T><<<B * nt, kThreads, 0, st>>>(n, B, A.x64, A.b64, A.v, A.part);
  LAUNCH_CHECK();
  ++tl_launches, k_zero<double><<<grid1(Bz * V0), 256, 0, st>>>(Bz * V0, A.x64);
  ++tl_launches, k_sc_start<T><<<gw, 256, 0, st>>>(B, n, s.lamH, s.lam_stride, nt, A.part, A.ss);
  LAUNCH_CHECK();
  if (sg) {
    // ---- refinement loop as nested WHILE nodes: no host reads.  The inner loop runs iterations in
    // pairs, so the rotating vectors (w/wo, v/vo, z/zn) end every pair where they started; the
    // second iteration of a pair is a no-op for samples that finished in the first (converged, or
    // capped at max_inner by the device counter, which marks every sample done), apart from
    // applying their pending update -- which the host loop's final update does otherwise.  An outer
    // step with nothing left to refine is a no-op too.
    int* oc = sg->counters;      // outer step counter
    int* ic = sg->counters + 1;  // inner iteration counter
    int* cnt_o = A.count;        // samples refining in this step
    int* cnt_i = A.count + 1;    // samples still iterating
    const cudaStream_t b0 = sg->body[0], b1 = sg->body[1];
    cudaGraphConditionalHandle ho, hi;
    if ((e = make_handle(st, &ho)) != cudaSuccess) return e;
    ++tl_launches, k_cond_init<<<1, 1, 0, st>>>(ho, oc);
    LAUNCH_CHECK();
    if ((e = open_while(st, b0, ho)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt_o, 0, sizeof(int), b0)) != cudaSuccess) return e;
    ++tl_launches, k_sc_outer_begin<T><<<gs, 256, 0, b0>>>(B, n, s.lamH, s.lam_stride, s.tol_lin, A.ss, A.act, cnt_o);
    LAUNCH_CHECK();
    if ((e = cudaMemcpyAsync(A.ran, A.act, Bz * sizeof(int), cudaMemcpyDeviceToDevice, b0)) != cudaSuccess) return e;
    ++tl_launches, k_inner_init<T><<<B * nt, kThreads, 0, b0>>>(n, B, A.act, A.ss, A.v, A.vo, A.w, A.wo, A.xi);
    LAUNCH_CHECK();
    T *v = A.v, *vo = A.vo, *z = A.z, *zn = A.zn, *w = A.w, *wo = A.wo;
    if ((e = vcycle_stream<T>(A, v, z, A.act, om, v, A.part, sub_smem, b0)) != cudaSuccess) return e;
    // partial slots per sample of <v, z> (written by the V-cycle's last sweep: the vectorised one for
    // FP32 with V(1,1), the row-mapped one otherwise; one slot when the sub-cycle does it all)
    const int nchd = A.Ls ? ((sizeof(T) == sizeof(float) && A.nu == 1) ? tiles_vec(n) : nt) : 1;
    ++tl_launches, k_sc_gamma0<T><<<gw, 256, 0, b0>>>(B, nchd, A.part, A.act, A.ss);
    LAUNCH_CHECK();
    if ((e = make_handle(b0, &hi)) != cudaSuccess) return e;
    ++tl_launches, k_cond_init<<<1, 1, 0, b0>>>(hi, ic);
    LAUNCH_CHECK();
    if ((e = open_while(b0, b1, hi)) != cudaSuccess) return e;
    for (int half = 0; half < 2; ++half) {
      const int nq = launch_minres_q<T>(n, B, A.act, A.ss, A.wx[0], A.wy[0], s.lamH, s.lam_stride, z, zn, wo, w, A.xi,
                                        A.q, A.part, nullptr, b1, A.rx, A.ry, A.rd);
      ++tl_launches;
      LAUNCH_CHECK();
      ++tl_launches, k_sc_retire<T><<<gs, 256, 0, b1>>>(B, A.act, A.ss);
      { T* tt = wo; wo = w; w = tt; }
      ++tl_launches, k_sc_delta<T><<<gw, 256, 0, b1>>>(B, nq, A.part, A.act, A.ss);
      ++tl_launches, launch_minres_v<T>(n, B, A.act, A.ss, A.q, v, vo, b1);
      LAUNCH_CHECK();
      { T* tt = vo; vo = v; v = tt; }
      if ((e = vcycle_stream<T>(A, v, zn, A.act, om, v, A.part, sub_smem, b1)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(cnt_i, 0, sizeof(int), b1)) != cudaSuccess) return e;
      ++tl_launches, k_sc_givens<T><<<gw, 256, 0, b1>>>(B, nchd, A.part, A.act, A.ss, T(s.tol_inner), cnt_i, ic, half,
                                                       s.max_inner);
      LAUNCH_CHECK();
      { T* tt = z; z = zn; zn = tt; }
    }
    ++tl_launches, k_cond_inner<<<1, 1, 0, b1>>>(hi, ic, cnt_i, s.max_inner);
    LAUNCH_CHECK();
    if ((e = close_while(b1)) != cudaSuccess) return e;
    // an even number of iterations: the rotating vectors are back where they started
    ++tl_launches, k_minres_finish<T><<<B * nt, kThreads, 0, b0>>>(n, B, A.ran, A.ss, zn, wo, w, A.xi);
    ++tl_launches, k_outer_update<T><<<B * nt, kThreads, 0, b0>>>(n, B, A.ss, A.ran, A.xi, A.x64);
    ++tl_launches, k_residual<T><<<B * nt, kThreads, 0, b0>>>(n, B, A.ran, A.wx64, A.wy64, s.lamH, s.lam_stride, A.x64,
                                                             A.b64, A.v, A.part, s.b, s.qoi);
    ++tl_launches, k_sc_outer_end<T><<<gw, 256, 0, b0>>>(B, nt, A.part, A.ran, A.ss);
    ++tl_launches, k_cond_outer<<<1, 1, 0, b0>>>(ho, oc, cnt_o, s.max_outer);
    LAUNCH_CHECK();
    if ((e = close_while(b0)) != cudaSuccess) return e;
  } else {
  // ---- refinement loop
  for (int o = 0; o < s.max_outer; ++o) {
    cudaMemsetAsync(A.count, 0, sizeof(int), st);
    ++tl_launches, k_sc_outer_begin<T><<<gs, 256, 0, st>>>(B, n, s.lamH, s.lam_stride, s.tol_lin, A.ss, A.act, A.count);
    LAUNCH_CHECK();
    int active = read_count(A.count, st, e);
    if (e != cudaSuccess) return e;
    if (active == 0) break;
    cudaMemcpyAsync(A.ran, A.act, Bz * sizeof(int), cudaMemcpyDeviceToDevice, st);
    ++tl_launches, k_inner_init<T><<<B * nt, kThreads, 0, st>>>(n, B, A.act, A.ss, A.v, A.vo, A.w, A.wo, A.xi);
    LAUNCH_CHECK();
    T *v = A.v, *vo = A.vo, *z = A.z, *zn = A.zn, *w = A.w, *wo = A.wo;
    e = vcycle_stream<T>(A, v, z, A.act, om, v, A.part, sub_smem, st);
    if (e != cudaSuccess) return e;
    // partial slots per sample of <v, z> (written by the V-cycle's last sweep: the vectorised one for
    // FP32 with V(1,1), the row-mapped one otherwise; one slot when the sub-cycle does it all)
    const int nchd = A.Ls ? ((sizeof(T) == sizeof(float) && A.nu == 1) ? tiles_vec(n) : nt) : 1;
    ++tl_launches, k_sc_gamma0<T><<<gw, 256, 0, st>>>(B, nchd, A.part, A.act, A.ss);
    LAUNCH_CHECK();
    for (int j = 0; j < s.max_inner; ++j) {
      std::pair<cudaEvent_t, cudaEvent_t>* pe = nullptr;
      if (s.probe) {
        if ((e = s.probe->next(&pe)) != cudaSuccess) return e;
        cudaEventRecord(pe->first, st);
      }
      const int nq = launch_minres_q<T>(n, B, A.act, A.ss, A.wx[0], A.wy[0], s.lamH, s.lam_stride, z, zn, wo, w, A.xi,
                                        A.q, A.part, s.probe ? s.probe->d_bytes : nullptr, st, A.rx, A.ry, A.rd);
      ++tl_launches;
      LAUNCH_CHECK();
      if (pe) cudaEventRecord(pe->second, st);
      // samples that converged in the previous Givens step have now applied their update
      ++tl_launches, k_sc_retire<T><<<gs, 256, 0, st>>>(B, A.act, A.ss);
      { T* tt = wo; wo = w; w = tt; }
      ++tl_launches, k_sc_delta<T><<<gw, 256, 0, st>>>(B, nq, A.part, A.act, A.ss);
      ++tl_launches, launch_minres_v<T>(n, B, A.act, A.ss, A.q, v, vo, st);
      LAUNCH_CHECK();
      { T* tt = vo; vo = v; v = tt; }
      e = vcycle_stream<T>(A, v, zn, A.act, om, v, A.part, sub_smem, st);
      if (e != cudaSuccess) return e;
      cudaMemsetAsync(A.count, 0, sizeof(int), st);
      ++tl_launches, k_sc_givens<T><<<gw, 256, 0, st>>>(B, nchd, A.part, A.act, A.ss, T(s.tol_inner), A.count);
      LAUNCH_CHECK();
      { T* tt = z; z = zn; zn = tt; }
      if ((j & 3) == 3 || j + 1 == s.max_inner) {
        active = read_count(A.count, st, e);
        if (e != cudaSuccess) return e;
        if (active == 0) break;
      }
    }
    // apply the pending updates of every sample that ran this step (converged or capped)
    ++tl_launches, k_minres_finish<T><<<B * nt, kThreads, 0, st>>>(n, B, A.ran, A.ss, zn, wo, w, A.xi);
    LAUNCH_CHECK();
    ++tl_launches, k_outer_update<T><<<B * nt, kThreads, 0, st>>>(n, B, A.ss, A.ran, A.xi, A.x64);
    ++tl_launches, k_residual<T><<<B * nt, kThreads, 0, st>>>(n, B, A.ran, A.wx64, A.wy64, s.lamH, s.lam_stride, A.x64, A.b64, A.v,
                                               A.part, s.b, s.qoi);
    ++tl_launches, k_sc_outer_end<T><<<gw, 256, 0, st>>>(B, nt, A.part, A.ran, A.ss);
    LAUNCH_CHECK();
  }
  }
  // ---- Rayleigh quotient (from each sample's last residual pass)
  ++tl_launches, k_sc_rq<T><<<gs, 256, 0, st>>>(B, n, s.lamH, s.lam_stride, A.ss, s.tol_lin, s.lam_out, s.lam_out_stride, s.iters_out,
                                 s.iters_stride, s.outer_out, s.outer_stride, s.flags, s.flags_stride, s.qoi);
  LAUNCH_CHECK();
  return cudaSuccess;
}

// level difference lambda^l - lambda^{l-1} (lambda^{-1} = 0 without a previous level)
__global__ void k_finalize(int B, double* out, int has_prev) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  out[(size_t)b * 4 + 3] = out[(size_t)b * 4 + 1] - (has_prev ? out[(size_t)b * 4 + 2] : 0.0);
}

}  // namespace

cudaError_t launch_finalize(int B, double* d_out, int has_prev, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  ++tl_launches, k_finalize<<<(B + 255) / 256, 256, 0, st>>>(B, d_out, has_prev);
  return cudaGetLastError();
}

size_t stream_arena_bytes(int n, int B, int mixed, int reaction) {
  if (mixed) {
    Arena<float> A;
    return carve_arena<float>(nullptr, n, B, A, reaction != 0) + 256;
  }
  Arena<double> A;
  return carve_arena<double>(nullptr, n, B, A) + 256;
}

uint64_t stream_launches() { return tl_launches; }

cudaError_t KernelProbe::next(std::pair<cudaEvent_t, cudaEvent_t>** out) {
  if (used == ev.size()) {
    std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&p.first);
    if (e == cudaSuccess) e = cudaEventCreate(&p.second);
    if (e != cudaSuccess) return e;
    ev.push_back(p);
  }
  *out = &ev[used++];
  return cudaSuccess;
}

cudaError_t KernelProbe::collect() {
  for (size_t i = 0; i < used; ++i) {
    float t = 0.0f;
    cudaError_t e = cudaEventElapsedTime(&t, ev[i].first, ev[i].second);
    if (e != cudaSuccess) return e;
    ms += t;
  }
  launches += used;
  used = 0;
  return cudaSuccess;
}

cudaError_t stream_solve(const StreamSolve& s, int mixed, void* arena, cudaStream_t st, const StreamGraph* sg) {
  return mixed ? stream_solve_t<float>(s, arena, st, sg) : stream_solve_t<double>(s, arena, st, sg);
}

}  // namespace mq
