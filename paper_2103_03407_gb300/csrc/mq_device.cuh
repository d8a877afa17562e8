// Device building blocks shared by the per-sample kernel (mq_sample.cu) and the batched
// streaming tier (mq_stream.cu): workspace carving, block-wide loops and reductions, the
// matrix-free P1 stencils, the multigrid hierarchy and the symmetric V-cycle.
//
// Stencils on the SW-NE triangulation with centroid coefficients: the P1 stiffness is the
// weighted five-point edge form (A x)_p = sum_{edges pq} w_pq (x_p - x_q) with
//     w of edge (i,j)-(i+1,j) = (a_low(i,j) + a_up(i,j-1)) / 2,
//     w of edge (i,j)-(i,j+1) = (a_up(i,j) + a_low(i-1,j)) / 2
// (hypotenuses carry no weight) and the consistent mass is the seven-point form
//     (M x)_p = h^2/12 (6 x_p + x_E + x_W + x_N + x_S + x_NE + x_SW).
// Vectors live on the padded (n+1) x (n+1) node grid with a zero boundary ring.  Multigrid
// coarse operators are the Galerkin operators P^T A P, i.e. the coarse P1 stiffness whose
// triangle coefficients are the means of the four fine triangles they contain.
//
// With a reaction term b u (the second test problem of Sec. 5; b constant per triangle) the
// operator gains the reaction matrix B = sum_T b_T M_T, a seven-point form over the six edges pq
// at p:  (B x)_p = h^2/12 sum_{edges pq} r_pq (x_p + x_q),  r_pq = (b_T1 + b_T2) / 2 over the two
// triangles of the edge (b = 1 gives the mass).  The multigrid preconditioner then approximates
// (A + D_B)^{-1} with D_B the lumped reaction, (D_B)_pp = h^2/6 sum_{T at p} b_T (the row sums of
// B), on every level from the coarsened b: symmetric positive definite and spectrally equivalent
// to A + B.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mq_internal.h"

namespace mq {
namespace dev {

// ---------------------------------------------------------------------------------------------
// workspace carving (16-byte aligned arrays)
struct Carver {
  uintptr_t base, cur;
  __host__ __device__ explicit Carver(void* b) : base((uintptr_t)b), cur((uintptr_t)b) {}
  template <typename T>
  __host__ __device__ T* take(size_t count) {
    cur = (cur + 15) & ~(uintptr_t)15;
    T* p = (T*)cur;
    cur += count * sizeof(T);
    return p;
  }
  __host__ __device__ size_t used() const { return (size_t)(cur - base); }
};

__host__ __device__ inline int ilog2(int n) {
#ifdef __CUDA_ARCH__
  return __ffs(n) - 1;  // n is a power of two
#else
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
#endif
}
__host__ __device__ inline size_t gsz(int n) { return (size_t)(n + 1) * (size_t)(n + 1); }

// Multigrid hierarchy for the stiffness A on meshes n, n/2, ..., 2 (level 0 = finest).
template <typename T>
struct MGDesc {
  int L;
  int n[kMaxMG];
  T* wx[kMaxMG];  // weight of edge (i,j)-(i+1,j) at padded node (i,j)
  T* wy[kMaxMG];  // weight of edge (i,j)-(i,j+1)
  T* dinv[kMaxMG];  // 1 / diag(A)
  T* x[kMaxMG];   // level solution (level 0: supplied by the caller)
  T* t[kMaxMG];   // Jacobi partner
  T* b[kMaxMG];   // level right-hand side (level 0: supplied by the caller)
  T* cell[2];     // ping-pong per-triangle coefficients while building
  T* cinv;        // symmetric inverse of the operator on the 3 x 3-unknown mesh 1/4 (exact coarse solve)
  int Lc;         // level solved exactly: mesh 1/4 when present, else mesh 1/2
  T* dr[kMaxMG];  // lumped reaction diagonal D_B per level (NULL: no reaction term)
  T* rcell[2];    // ping-pong per-triangle reaction coefficients while building
};

template <typename T>
__host__ __device__ void carve_mg(Carver& c, int n, MGDesc<T>& d, bool reaction = false) {
  d.L = ilog2(n);
  for (int l = 0; l < d.L; ++l) {
    const int nl = n >> l;
    d.n[l] = nl;
    const size_t V = gsz(nl);
    d.wx[l] = c.take<T>(V);
    d.wy[l] = c.take<T>(V);
    d.dinv[l] = c.take<T>(V);
    d.t[l] = c.take<T>(V);
    d.x[l] = l ? c.take<T>(V) : nullptr;
    d.b[l] = l ? c.take<T>(V) : nullptr;
    d.dr[l] = reaction ? c.take<T>(V) : nullptr;
  }
  const size_t cells = n >= 4 ? (size_t)2 * (n / 2) * (n / 2) : 1;
  d.cell[0] = c.take<T>(cells);
  d.cell[1] = c.take<T>(cells);
  d.rcell[0] = reaction ? c.take<T>(cells) : nullptr;
  d.rcell[1] = reaction ? c.take<T>(cells) : nullptr;
  d.cinv = c.take<T>(81);
  d.Lc = d.L >= 2 ? d.L - 2 : d.L - 1;
}

// Same hierarchy with the operator arrays (weights, inverse diagonals) taken from carver w and
// the vectors (t, x, b) and building buffers taken from carver v.
template <typename T>
__host__ __device__ void carve_mg_split(Carver& w, Carver& v, int n, MGDesc<T>& d, bool reaction = false) {
  d.L = ilog2(n);
  for (int l = 0; l < kMaxMG; ++l) d.dr[l] = nullptr;
  for (int l = 0; l < d.L; ++l) {
    const int nl = n >> l;
    d.n[l] = nl;
    const size_t V = gsz(nl);
    d.wx[l] = w.take<T>(V);
    d.wy[l] = w.take<T>(V);
    d.dinv[l] = w.take<T>(V);
    d.dr[l] = reaction ? w.take<T>(V) : nullptr;
    d.t[l] = v.take<T>(V);
    d.x[l] = l ? v.take<T>(V) : nullptr;
    d.b[l] = l ? v.take<T>(V) : nullptr;
  }
  const size_t cells = n >= 4 ? (size_t)2 * (n / 2) * (n / 2) : 1;
  d.cell[0] = v.take<T>(cells);
  d.cell[1] = v.take<T>(cells);
  d.rcell[0] = reaction ? v.take<T>(cells) : nullptr;
  d.rcell[1] = reaction ? v.take<T>(cells) : nullptr;
  d.cinv = w.take<T>(81);
  d.Lc = d.L >= 2 ? d.L - 2 : d.L - 1;
}

// ---------------------------------------------------------------------------------------------
// block-level helpers
template <class F>
__device__ __forceinline__ void for_interior(int n, F f) {
  const int lg = ilog2(n);
  const int tot = (n - 1) << lg;
  const int ld = n + 1;
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    const int i = (q & (n - 1)) + 1;
    if (i == n) continue;
    const int j = (q >> lg) + 1;
    f(j * ld + i, i, j);
  }
}

template <class F>
__device__ __forceinline__ void for_all(size_t count, F f) {
  for (size_t q = threadIdx.x; q < count; q += blockDim.x) f(q);
}

// size of the shared reduction buffer every block_sum caller must provide
constexpr int kRedSlots = 32 * 12 + 12;

struct NoEp {
  __device__ void operator()(const double*) const {}
};

// Butterfly reduce-scatter of M values over the lanes that differ in bits O, O/2, ..., 1.  At each
// stage a lane keeps one half of the values it carries (the lower half when its bit is clear),
// adds its partner's copy of that half and passes on the other half: M/2 additions per stage
// instead of M, so a warp sums 12 values with 13 additions instead of 60 (FP64 additions are
// scarce on this GPU).  On return v[0] holds the warp total of value index `base` when c >= 1,
// else the lane carries nothing.  Values past a lane's real count c are zeros.
template <int M, int O, typename A>
struct Butterfly {
  static __device__ __forceinline__ void run(A* v, int lane, int& base, int& c) {
    constexpr int H = (M + 1) / 2;
    const bool b = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const A lo = v[i];
      const A hi = (H + i < M) ? v[H + i] : A(0);
      const A send = b ? lo : hi;
      const A keep = b ? hi : lo;
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
    if (b) {
      base += H;
      c = max(0, c - H);
    } else {
      c = min(c, H);
    }
    Butterfly<H, O / 2, A>::run(v, lane, base, c);
  }
};
template <int M, typename A>
struct Butterfly<M, 0, A> {
  static __device__ __forceinline__ void run(A*, int, int&, int&) {}
};

// Sum NV values over the block (fixed order: deterministic).  Thread 0 runs ep(totals) before the
// closing barrier, so scalars it derives are visible to every thread after the call; every thread
// receives the totals in out.  Only threads below nact can hold nonzero values: warps beyond it
// skip the reduction.
template <int NV, typename A, class Ep = NoEp>
__device__ __forceinline__ void block_sum(A (&v)[NV], double (&out)[NV], double* red, Ep ep = Ep(),
                                          int nact = 1 << 30) {
  static_assert(NV <= 12, "block_sum reduces at most 12 values");
  // red: kRedSlots doubles = 32 * 12 partial slots followed by 12 total slots.  The totals never
  // overlap the partials, so two barriers suffice: the next call writes partials only after
  // passing this call's second barrier, and writes totals only after its own first barrier
  // (every thread has read ours).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = min((int)(blockDim.x >> 5), (nact + 31) >> 5);
  double* tot = red + 32 * 12;
  if (wid < nw) {
    int base = 0, c = NV;
    Butterfly<NV, 16, A>::run(v, lane, base, c);
    if (c >= 1) red[wid * NV + base] = (double)v[0];
  }
  __syncthreads();
  if (wid == 0) {
    if (lane < NV) {
      double s = red[lane];
      for (int w = 1; w < nw; ++w) s += red[w * NV + lane];
      tot[lane] = s;
    }
    __syncwarp();
    if (lane == 0) {
      double t[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) t[i] = tot[i];
      ep(t);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = tot[i];
}

// stiffness (weighted five-point edge form) at padded node p
template <typename T, typename X>
__device__ __forceinline__ T stiff(const T* __restrict__ wx, const T* __restrict__ wy, const X* x, int p, int ld) {
  const T xp = (T)x[p];
  return wx[p] * (xp - (T)x[p + 1]) + wx[p - 1] * (xp - (T)x[p - 1]) + wy[p] * (xp - (T)x[p + ld]) +
         wy[p - ld] * (xp - (T)x[p - ld]);
}

// mass seven-point sum without the h^2/12 factor
template <typename T>
__device__ __forceinline__ T mass7(const T* x, int p, int ld) {
  return T(6) * x[p] + (x[p + 1] + x[p - 1]) + (x[p + ld] + x[p - ld]) + (x[p + ld + 1] + x[p - ld - 1]);
}

// FP64 stiffness at interior node (i, j) of mesh n with the edge weights formed from the
// centroid coefficients a (lower triangles first, then upper).
__device__ __forceinline__ double stiff_cells(const double* __restrict__ a, int n, const double* x, int p, int ld,
                                              int i, int j) {
  const double* lo = a;
  const double* up = a + (size_t)n * n;
  const int c = j * n + i;
  const double lij = lo[c], li1j = lo[c - 1], li1j1 = lo[c - n - 1];
  const double uij = up[c], uij1 = up[c - n], ui1j1 = up[c - n - 1];
  const double we = 0.5 * (lij + uij1), ww = 0.5 * (li1j + ui1j1);
  const double wn = 0.5 * (uij + li1j), ws = 0.5 * (uij1 + li1j1);
  const double xp = x[p];
  return we * (xp - x[p + 1]) + ww * (xp - x[p - 1]) + wn * (xp - x[p + ld]) + ws * (xp - x[p - ld]);
}

// reaction seven-point sum without the h^2/12 factor, from the edge weights rx (edge to E), ry (to
// N) and rd (to NE) of the padded nodes
template <typename T, typename X>
__device__ __forceinline__ T react7(const T* __restrict__ rx, const T* __restrict__ ry, const T* __restrict__ rd,
                                    const X* x, int p, int ld) {
  const T xp = (T)x[p];
  return rx[p] * (xp + (T)x[p + 1]) + rx[p - 1] * (xp + (T)x[p - 1]) + ry[p] * (xp + (T)x[p + ld]) +
         ry[p - ld] * (xp + (T)x[p - ld]) + rd[p] * (xp + (T)x[p + ld + 1]) + rd[p - ld - 1] * (xp + (T)x[p - ld - 1]);
}

// FP64 reaction sum (without h^2/12) at interior node (i, j) from the centroid values b of the
// reaction coefficient (lower triangles first, then upper)
__device__ __forceinline__ double react_cells(const double* __restrict__ b, int n, const double* x, int p, int ld,
                                              int i, int j) {
  const double* lo = b;
  const double* up = b + (size_t)n * n;
  const int c = j * n + i;
  const double lij = lo[c], li1j = lo[c - 1], li1j1 = lo[c - n - 1];
  const double uij = up[c], uij1 = up[c - n], ui1j1 = up[c - n - 1];
  const double re = 0.5 * (lij + uij1), rw = 0.5 * (li1j + ui1j1);
  const double rn = 0.5 * (uij + li1j), rs = 0.5 * (uij1 + li1j1);
  const double rne = 0.5 * (lij + uij), rsw = 0.5 * (li1j1 + ui1j1);
  const double xp = x[p];
  return re * (xp + x[p + 1]) + rw * (xp + x[p - 1]) + rn * (xp + x[p + ld]) + rs * (xp + x[p - ld]) +
         rne * (xp + x[p + ld + 1]) + rsw * (xp + x[p - ld - 1]);
}

// ---------------------------------------------------------------------------------------------
// operator setup
template <typename T, typename S>
__device__ void weights_from_cells(int n, const S* low, const S* up, T* wx, T* wy) {
  const int ld = n + 1;
  for_all(gsz(n), [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    T a = T(0), b = T(0);
    if (i <= n - 1 && j >= 1 && j <= n - 1) a = T(0.5 * ((double)low[j * n + i] + (double)up[(j - 1) * n + i]));
    if (i >= 1 && i <= n - 1 && j <= n - 1) b = T(0.5 * ((double)up[j * n + i] + (double)low[j * n + i - 1]));
    wx[q] = a;
    wy[q] = b;
  });
}

// the reaction's edge weights: rx, ry as the stiffness weights of b (same two triangles per edge),
// rd of the hypotenuse (i,j)-(i+1,j+1) = (b_low(i,j) + b_up(i,j)) / 2
template <typename T, typename S>
__device__ void reaction_weights(int n, const S* low, const S* up, T* rx, T* ry, T* rd) {
  weights_from_cells<T, S>(n, low, up, rx, ry);
  const int ld = n + 1;
  for_all(gsz(n), [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    rd[q] = (i <= n - 1 && j <= n - 1) ? T(0.5 * ((double)low[j * n + i] + (double)up[j * n + i])) : T(0);
  });
}

// lumped reaction diagonal h^2/6 sum_{T at p} b_T at the interior nodes, 0 on the ring
template <typename T, typename S>
__device__ void lumped_reaction(int n, const S* low, const S* up, T* dr) {
  const int ld = n + 1;
  const double f = 1.0 / (6.0 * (double)n * (double)n);
  for_all(gsz(n), [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    T v = T(0);
    if (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1) {
      const int c = j * n + i;
      v = T(f * ((double)low[c] + (double)up[c] + (double)low[c - 1] + (double)up[c - n] + (double)low[c - n - 1] +
                 (double)up[c - n - 1]));
    }
    dr[q] = v;
  });
}

template <typename T, typename S>
__device__ void coarsen_cells(int n, const S* low, const S* up, T* out) {
  const int m = n / 2;
  for_all((size_t)m * m, [&](size_t q) {
    const int I = (int)(q % m), J = (int)(q / m);
    const int i = 2 * I, j = 2 * J;
    const double lo = (double)low[j * n + i] + (double)low[j * n + i + 1] + (double)low[(j + 1) * n + i + 1] +
                      (double)up[j * n + i + 1];
    const double hi = (double)up[j * n + i] + (double)up[(j + 1) * n + i + 1] + (double)up[(j + 1) * n + i] +
                      (double)low[(j + 1) * n + i];
    out[q] = T(0.25 * lo);
    out[m * m + q] = T(0.25 * hi);
  });
}

// 1 / diag(A) at the interior nodes and 0 on the boundary ring (the fused smoothing phase of the
// V-cycle reads it at the neighbours of every interior node)
template <typename T>
__device__ void inverse_diagonal(int n, const T* wx, const T* wy, T* dinv, const T* dr = nullptr) {
  const int ld = n + 1;
  for_all(gsz(n), [&](size_t q) {
    const int i = (int)(q % ld), j = (int)(q / ld);
    const int p = (int)q;
    dinv[q] = (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1)
                  ? T(1) / (wx[p] + wx[p - 1] + wy[p] + wy[p - ld] + (dr ? dr[p] : T(0)))
                  : T(0);
  });
}

// Exact coarse solve on mesh 1/4 (3 x 3 unknowns): the inverse of the weighted five-point
// operator by an FP32 Cholesky factorisation (one thread, fully unrolled so the 9 x 9 factor stays
// in registers), written symmetrised.  The V-cycle only needs a symmetric positive definite
// approximation of A^{-1} on this level; this one is exact to FP32 rounding.
template <typename T>
__device__ void coarse_inverse4(const T* wx, const T* wy, T* cinv, const T* dr = nullptr) {
  constexpr int ld = 5;
  float L[9][9];
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int c = 0; c < 9; ++c) L[r][c] = 0.0f;
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const int i = r % 3 + 1, j = r / 3 + 1, p = j * ld + i;
    L[r][r] = (float)(wx[p] + wx[p - 1] + wy[p] + wy[p - ld] + (dr ? dr[p] : T(0)));
    if (i > 1) L[r][r - 1] = -(float)wx[p - 1];
    if (j > 1) L[r][r - 3] = -(float)wy[p - ld];
  }
  // in-place Cholesky of the lower triangle
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float d = L[k][k];
#pragma unroll
    for (int m = 0; m < k; ++m) d -= L[k][m] * L[k][m];
    d = sqrtf(d);
    L[k][k] = d;
    const float id = 1.0f / d;
#pragma unroll
    for (int r = k + 1; r < 9; ++r) {
      float v = L[r][k];
#pragma unroll
      for (int m = 0; m < k; ++m) v -= L[r][m] * L[k][m];
      L[r][k] = v * id;
    }
  }
  // columns of the inverse: L L^T x = e_c
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    float y[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      float v = (r == c) ? 1.0f : 0.0f;
#pragma unroll
      for (int m = 0; m < r; ++m) v -= L[r][m] * y[m];
      y[r] = v / L[r][r];
    }
#pragma unroll
    for (int r = 8; r >= 0; --r) {
      float v = y[r];
#pragma unroll
      for (int m = r + 1; m < 9; ++m) v -= L[m][r] * y[m];
      y[r] = v / L[r][r];
    }
#pragma unroll
    for (int r = 0; r < 9; ++r)
      if (r >= c) cinv[r * 9 + c] = T(y[r]);
  }
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int c = r + 1; c < 9; ++c) cinv[r * 9 + c] = cinv[c * 9 + r];
}

// Builds every level (weights, inverse diagonals) from the fine centroid coefficients a, and with
// rb (hierarchy carved with the reaction arrays) the lumped reaction of every level from the
// centroid values rb of the reaction coefficient.  Returns true when every a is positive
// (Assumption A1) and every b nonnegative.
template <typename T, typename S = double>
__device__ bool build_mg(MGDesc<T>& d, const S* __restrict__ a, int n, double* red, const S* __restrict__ rb = nullptr) {
  int bad = 0;
  const bool rx = rb != nullptr && d.dr[0] != nullptr;
  for_all((size_t)2 * n * n, [&](size_t q) { bad |= !(a[q] > S(0)); });
  if (rx) for_all((size_t)2 * n * n, [&](size_t q) { bad |= !(rb[q] >= S(0)); });
  weights_from_cells<T, S>(n, a, a + (size_t)n * n, d.wx[0], d.wy[0]);
  if (d.L > 1) coarsen_cells<T, S>(n, a, a + (size_t)n * n, d.cell[0]);
  if (rx) {
    lumped_reaction<T, S>(n, rb, rb + (size_t)n * n, d.dr[0]);
    if (d.L > 1) coarsen_cells<T, S>(n, rb, rb + (size_t)n * n, d.rcell[0]);
  }
  __syncthreads();
  for (int l = 1; l < d.L; ++l) {
    const int nl = d.n[l];
    const T* src = d.cell[(l - 1) & 1];
    weights_from_cells<T, T>(nl, src, src + (size_t)nl * nl, d.wx[l], d.wy[l]);
    if (l + 1 < d.L) coarsen_cells<T, T>(nl, src, src + (size_t)nl * nl, d.cell[l & 1]);
    if (rx) {
      const T* rs = d.rcell[(l - 1) & 1];
      lumped_reaction<T, T>(nl, rs, rs + (size_t)nl * nl, d.dr[l]);
      if (l + 1 < d.L) coarsen_cells<T, T>(nl, rs, rs + (size_t)nl * nl, d.rcell[l & 1]);
    }
    inverse_diagonal<T>(d.n[l - 1], d.wx[l - 1], d.wy[l - 1], d.dinv[l - 1], rx ? d.dr[l - 1] : nullptr);
    __syncthreads();
  }
  inverse_diagonal<T>(d.n[d.L - 1], d.wx[d.L - 1], d.wy[d.L - 1], d.dinv[d.L - 1], rx ? d.dr[d.L - 1] : nullptr);
  if (d.L >= 2 && threadIdx.x == 0)
    coarse_inverse4<T>(d.wx[d.L - 2], d.wy[d.L - 2], d.cinv, rx ? d.dr[d.L - 2] : nullptr);
  double v[1] = {(double)bad}, o[1];
  block_sum<1, double>(v, o, red);
  return o[0] == 0.0;
}

// Symmetric V-cycle for A (A + D_B when the hierarchy holds a lumped reaction, which build_mg must
// then have formed) with nu (2 or 1) damped Jacobi steps before and after each coarse-grid
// correction, Galerkin coarse levels and an exact solve on mesh 1/4 (or 1/2): x0 = B^{-1} b0.
// Phases per level: [two Jacobi steps from zero, fused] -> [residual restricted with P^T] going
// down; [prolongation + correction + one Jacobi step, fused] -> [one Jacobi step] going up.
// nu = 1: [residual of x1 = omega D^-1 b, restricted] down, [prolongation + correction + one
// Jacobi step] up -- two phases per level, and x1 is never stored.  With dotv, returns this thread's share of <dotv, x0> (formed in the last phase).
template <typename T>
__device__ __noinline__ T vcycle(const MGDesc<T>& d, const T* b0, T* x0, T omega, const T* dotv = nullptr,
                                int nu = 2) {
  const int Lc = d.Lc;
  for (int l = 0; l < Lc; ++l) {
    const int n = d.n[l], ld = n + 1;
    const T* b = l ? d.b[l] : b0;
    T* xa = l ? d.x[l] : x0;
    const T* __restrict__ wx = d.wx[l];
    const T* __restrict__ wy = d.wy[l];
    const T* __restrict__ di = d.dinv[l];
    const T* __restrict__ dg = d.dr[l];  // lumped reaction (NULL: none)
    if (nu == 1) {
      // V(1,1): the one Jacobi step from zero is x1 = omega D^-1 b, pointwise; the restriction
      // forms it on the fly and nothing is stored
      T* bc = d.b[l + 1];
      for_interior(n >> 1, [&](int P, int I, int J) {
        const int p = (2 * J) * ld + 2 * I;
        auto x1 = [&](int q) { return omega * di[q] * b[q]; };
        auto res = [&](int q) {
          const T xq = x1(q);
          return b[q] - (wx[q] * (xq - x1(q + 1)) + wx[q - 1] * (xq - x1(q - 1)) + wy[q] * (xq - x1(q + ld)) +
                         wy[q - ld] * (xq - x1(q - ld)) + (dg ? dg[q] * xq : T(0)));
        };
        bc[P] = res(p) + T(0.5) * ((res(p + 1) + res(p - 1)) + (res(p + ld) + res(p - ld)) +
                                   (res(p + ld + 1) + res(p - ld - 1)));
      });
      __syncthreads();
      continue;
    }
    for_interior(n, [&](int p, int, int) {
      auto x1 = [&](int q) { return omega * di[q] * b[q]; };
      const T xp = x1(p);
      const T ax = wx[p] * (xp - x1(p + 1)) + wx[p - 1] * (xp - x1(p - 1)) + wy[p] * (xp - x1(p + ld)) +
                   wy[p - ld] * (xp - x1(p - ld)) + (dg ? dg[p] * xp : T(0));
      xa[p] = xp + omega * di[p] * (b[p] - ax);
    });
    __syncthreads();
    T* bc = d.b[l + 1];
    const T* cx = xa;
    for_interior(n >> 1, [&](int P, int I, int J) {
      const int p = (2 * J) * ld + 2 * I;
      auto res = [&](int q) { return b[q] - (stiff<T, T>(wx, wy, cx, q, ld) + (dg ? dg[q] * cx[q] : T(0))); };
      bc[P] = res(p) + T(0.5) * ((res(p + 1) + res(p - 1)) + (res(p + ld) + res(p - ld)) +
                                 (res(p + ld + 1) + res(p - ld - 1)));
    });
    __syncthreads();
  }
  {
    const T* b = Lc ? d.b[Lc] : b0;
    T* x = Lc ? d.x[Lc] : x0;
    if (d.n[Lc] == 4) {
      // 3 x 3 unknowns at padded indices (i, j) -> j * 5 + i
      if (threadIdx.x < 9) {
        const int r = threadIdx.x;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 9; ++c) s += d.cinv[r * 9 + c] * b[(c / 3 + 1) * 5 + (c % 3 + 1)];
        x[(r / 3 + 1) * 5 + (r % 3 + 1)] = s;
      }
    } else if (threadIdx.x == 0) {
      x[4] = b[4] * d.dinv[Lc][4];  // mesh 1/2: one unknown
    }
    __syncthreads();
  }
  T dot = T(0);
  for (int l = Lc - 1; l >= 0; --l) {
    const int n = d.n[l], ld = n + 1;
    const T* b = l ? d.b[l] : b0;
    T* xa = l ? d.x[l] : x0;
    T* tt = d.t[l];
    const T* __restrict__ wx = d.wx[l];
    const T* __restrict__ wy = d.wy[l];
    const T* __restrict__ di = d.dinv[l];
    const T* __restrict__ dg = d.dr[l];
    const T* xc = d.x[l + 1];
    const int ldc = (n >> 1) + 1;
    if (nu == 1) {
      // V(1,1): t = omega D^-1 b + P xc, then the one post-smoothing step, in one phase
      const bool last = (l == 0) && dotv;
      for_interior(n, [&](int p, int i, int j) {
        auto t = [&](int q, int ii, int jj) {
          const int c0 = (jj >> 1) * ldc + (ii >> 1);
          return omega * di[q] * b[q] + T(0.5) * (xc[c0] + xc[c0 + (ii & 1) + (jj & 1) * ldc]);
        };
        const T tp = t(p, i, j);
        const T ax = wx[p] * (tp - t(p + 1, i + 1, j)) + wx[p - 1] * (tp - t(p - 1, i - 1, j)) +
                     wy[p] * (tp - t(p + ld, i, j + 1)) + wy[p - ld] * (tp - t(p - ld, i, j - 1)) +
                     (dg ? dg[p] * tp : T(0));
        const T o = tp + omega * di[p] * (b[p] - ax);
        xa[p] = o;
        if (last) dot += dotv[p] * o;
      });
      __syncthreads();
      continue;
    }
    for_interior(n, [&](int p, int i, int j) {
      // P1 interpolation on the SW-NE mesh, branch-free: the mean of the coarse values at the two
      // ends of the coarse edge through the fine node (both ends coincide at coarse nodes)
      auto t = [&](int q, int ii, int jj) {
        const int c0 = (jj >> 1) * ldc + (ii >> 1);
        return xa[q] + T(0.5) * (xc[c0] + xc[c0 + (ii & 1) + (jj & 1) * ldc]);
      };
      const T tp = t(p, i, j);
      const T ax = wx[p] * (tp - t(p + 1, i + 1, j)) + wx[p - 1] * (tp - t(p - 1, i - 1, j)) +
                   wy[p] * (tp - t(p + ld, i, j + 1)) + wy[p - ld] * (tp - t(p - ld, i, j - 1)) +
                   (dg ? dg[p] * tp : T(0));
      tt[p] = tp + omega * di[p] * (b[p] - ax);
    });
    __syncthreads();
    const bool last = (l == 0) && dotv;
    for_interior(n, [&](int p, int, int) {
      const T o = tt[p] + omega * di[p] * (b[p] - (stiff<T, T>(wx, wy, tt, p, ld) + (dg ? dg[p] * tt[p] : T(0))));
      xa[p] = o;
      if (last) dot += dotv[p] * o;
    });
    __syncthreads();
  }
  if (Lc == 0 && dotv)
    for_interior(d.n[0], [&](int p, int, int) { dot += dotv[p] * x0[p]; });
  return dot;
}

template <typename T>
__device__ void zero_vec(T* v, int n) {
  for_all(gsz(n), [&](size_t q) { v[q] = T(0); });
}

template <typename T>
__device__ void zero_mg(const MGDesc<T>& d) {
  for (int l = 0; l < d.L; ++l) {
    zero_vec(d.t[l], d.n[l]);
    zero_vec(d.dinv[l], d.n[l]);
    if (d.dr[l]) zero_vec(d.dr[l], d.n[l]);
    if (l) {
      zero_vec(d.x[l], d.n[l]);
      zero_vec(d.b[l], d.n[l]);
    }
  }
}

}  // namespace dev
}  // namespace mq
