// Per-sample two-grid kernel: one CTA evaluates whole samples of one MLQMC level.
//
// For each sample (shift r, lattice point k) the CTA
//   1. builds the coarse-mesh operator from the centroid coefficients (truncation S_l) and
//      computes the smallest eigenpair (lambda_H, u_H) by LOBPCG preconditioned with a
//      multigrid V-cycle, warm-started from the eigenvector of the previous lattice point of
//      its chain (Sec. 4.3, "reusing samples from nearby QMC points");
//   2. for the fine mesh of the level (and, on l > 0, the fine mesh of level l-1, from the same
//      coarse pair -- Algorithm 2), forms b = M_h P u_H (P: P1 interpolation), solves
//      (A_h - lambda_H M_h) w = b (eq. 2grid_source) by MINRES preconditioned with a symmetric
//      multigrid V-cycle on A_h, inside FP64 iterative refinement, and returns the Rayleigh
//      quotient w^T A_h w / w^T M_h w (Algorithm 1 steps 3-4, eq. RQ_update);
//   3. writes lambda_H, lambda^l, lambda^{l-1} and the difference.
//
// Operators are matrix-free.  On the SW-NE triangulation with centroid coefficients the P1
// stiffness is the weighted five-point edge form
//     (A x)_p = sum_{edges pq} w_pq (x_p - x_q),
//     w of edge (i,j)-(i+1,j) = (a_low(i,j) + a_up(i,j-1)) / 2,
//     w of edge (i,j)-(i,j+1) = (a_up(i,j) + a_low(i-1,j)) / 2
// (the hypotenuses carry no weight), and the consistent mass is the seven-point form
//     (M x)_p = h^2/12 (6 x_p + x_E + x_W + x_N + x_S + x_NE + x_SW).
// Vectors live on the padded (n+1) x (n+1) node grid with a zero boundary ring, so every
// stencil is branch-free.  The multigrid coarse operators are the Galerkin operators P^T A P,
// which for nested P1 spaces are the coarse P1 stiffness with each coarse triangle's
// coefficient the mean of its four fine triangles.
//
// Workspace: one slab per CTA, carved identically on host (to size it) and device.  The slab
// lives in dynamic shared memory when it fits, otherwise in a global scratch buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mq_internal.h"

namespace mq {
namespace {

// ---------------------------------------------------------------------------------------------
// workspace carving
struct Carver {
  uintptr_t base, cur;
  __host__ __device__ explicit Carver(void* b) : base((uintptr_t)b), cur((uintptr_t)b) {}
  template <typename T>
  __host__ __device__ T* take(size_t count) {
    cur = (cur + 255) & ~(uintptr_t)255;
    T* p = (T*)cur;
    cur += count * sizeof(T);
    return p;
  }
  __host__ __device__ size_t used() const { return (size_t)(cur - base); }
};

__host__ __device__ inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
__host__ __device__ inline size_t gsz(int n) { return (size_t)(n + 1) * (size_t)(n + 1); }

template <typename T>
struct MGDesc {
  int L;
  int n[kMaxMG];
  T* wx[kMaxMG];
  T* wy[kMaxMG];
  T* x[kMaxMG];  // level solution (level 0: supplied by the caller)
  T* t[kMaxMG];  // Jacobi ping-pong partner / residual
  T* b[kMaxMG];  // level right-hand side (level 0: supplied by the caller)
  T* cell[2];    // ping-pong per-triangle coefficients while building
};

template <typename T>
__host__ __device__ void carve_mg(Carver& c, int n, MGDesc<T>& d, T* wx0, T* wy0) {
  d.L = ilog2(n);  // meshes n, n/2, ..., 2
  for (int l = 0; l < d.L; ++l) {
    const int nl = n >> l;
    d.n[l] = nl;
    const size_t V = gsz(nl);
    if (l == 0 && wx0) {
      d.wx[0] = wx0;
      d.wy[0] = wy0;
    } else {
      d.wx[l] = c.take<T>(V);
      d.wy[l] = c.take<T>(V);
    }
    d.t[l] = c.take<T>(V);
    d.x[l] = l ? c.take<T>(V) : nullptr;
    d.b[l] = l ? c.take<T>(V) : nullptr;
  }
  const size_t cells = n >= 4 ? (size_t)2 * (n / 2) * (n / 2) : 1;
  d.cell[0] = c.take<T>(cells);
  d.cell[1] = c.take<T>(cells);
}

struct CoarseWS {
  MGDesc<double> mg;
  double *x, *Ax, *Mx, *w, *Aw, *Mw, *p, *Ap, *Mp, *r, *uprev;
};

__host__ __device__ void carve_coarse(Carver& c, int nc, CoarseWS& ws) {
  const size_t V = gsz(nc);
  ws.x = c.take<double>(V);
  ws.Ax = c.take<double>(V);
  ws.Mx = c.take<double>(V);
  ws.w = c.take<double>(V);
  ws.Aw = c.take<double>(V);
  ws.Mw = c.take<double>(V);
  ws.p = c.take<double>(V);
  ws.Ap = c.take<double>(V);
  ws.Mp = c.take<double>(V);
  ws.r = c.take<double>(V);
  ws.uprev = c.take<double>(V);
  carve_mg<double>(c, nc, ws.mg, nullptr, nullptr);
}

template <typename T>
struct FineWS {
  MGDesc<T> mg;
  double *wx64, *wy64, *x64, *r64, *b64;
  T *vo, *v, *z, *zn, *wo, *w, *q, *xi;
};

template <typename T>
__host__ __device__ void carve_fine(Carver& c, int n, FineWS<T>& ws) {
  const size_t V = gsz(n);
  ws.wx64 = c.take<double>(V);
  ws.wy64 = c.take<double>(V);
  ws.x64 = c.take<double>(V);
  ws.r64 = c.take<double>(V);
  ws.b64 = c.take<double>(V);
  ws.vo = c.take<T>(V);
  ws.v = c.take<T>(V);
  ws.z = c.take<T>(V);
  ws.zn = c.take<T>(V);
  ws.wo = c.take<T>(V);
  ws.w = c.take<T>(V);
  ws.q = c.take<T>(V);
  ws.xi = c.take<T>(V);
  const bool same = sizeof(T) == sizeof(double);
  carve_mg<T>(c, n, ws.mg, same ? (T*)ws.wx64 : nullptr, same ? (T*)ws.wy64 : nullptr);
}

template <typename T>
__host__ __device__ size_t slab_size(int nf, int nc, int np) {
  Carver c(nullptr);
  CoarseWS cw;
  carve_coarse(c, nc, cw);
  const size_t coarse = (c.used() + 255) & ~(size_t)255;
  Carver f(nullptr);
  FineWS<T> fw;
  carve_fine<T>(f, nf > np ? nf : np, fw);
  return coarse + ((f.used() + 255) & ~(size_t)255);
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

// Sum NV values over the block; every thread receives the totals.  Fixed order: deterministic.
template <int NV, typename A>
__device__ __forceinline__ void block_sum(A (&v)[NV], double (&out)[NV], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    A s = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid * NV + i] = (double)s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? red[lane * NV + i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[32 * NV + i] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = red[32 * NV + i];
  __syncthreads();
}

// stiffness (weighted five-point edge form) at padded node p; also returns the diagonal
template <typename T>
__device__ __forceinline__ T stiff(const T* __restrict__ wx, const T* __restrict__ wy, const T* x, int p, int ld,
                                   T& diag) {
  const T we = wx[p], ww = wx[p - 1], wn = wy[p], ws = wy[p - ld];
  const T xp = x[p];
  diag = we + ww + wn + ws;
  return we * (xp - x[p + 1]) + ww * (xp - x[p - 1]) + wn * (xp - x[p + ld]) + ws * (xp - x[p - ld]);
}

// mass seven-point sum without the h^2/12 factor
template <typename T>
__device__ __forceinline__ T mass7(const T* x, int p, int ld) {
  return T(6) * x[p] + (x[p + 1] + x[p - 1]) + (x[p + ld] + x[p - ld]) + (x[p + ld + 1] + x[p - ld - 1]);
}

// ---------------------------------------------------------------------------------------------
// operator setup: edge weights of every multigrid level from the fine centroid coefficients
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

// per-triangle coefficients of the mesh n/2 as means over the four fine triangles they contain
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

// builds all levels; returns true when every fine coefficient is positive (Assumption A1)
template <typename T>
__device__ bool build_mg(MGDesc<T>& d, const double* __restrict__ a, int n, double* red) {
  int bad = 0;
  for_all((size_t)2 * n * n, [&](size_t q) { bad |= !(a[q] > 0.0); });
  weights_from_cells<T, double>(n, a, a + (size_t)n * n, d.wx[0], d.wy[0]);
  if (d.L > 1) coarsen_cells<T, double>(n, a, a + (size_t)n * n, d.cell[0]);
  __syncthreads();
  for (int l = 1; l < d.L; ++l) {
    const int nl = d.n[l];
    const T* src = d.cell[(l - 1) & 1];
    weights_from_cells<T, T>(nl, src, src + (size_t)nl * nl, d.wx[l], d.wy[l]);
    if (l + 1 < d.L) coarsen_cells<T, T>(nl, src, src + (size_t)nl * nl, d.cell[l & 1]);
    __syncthreads();
  }
  double v[1] = {(double)bad}, o[1];
  block_sum<1, double>(v, o, red);
  return o[0] == 0.0;
}

// symmetric V-cycle for A (damped Jacobi, nu sweeps before and after, Galerkin coarse levels,
// exact solve on the one-unknown mesh 1/2): x0 = B^{-1} b0
template <typename T>
__device__ void vcycle(const MGDesc<T>& d, const T* b0, T* x0, int nu, T omega) {
  const int L = d.L;
  for (int l = 0; l < L - 1; ++l) {
    const int n = d.n[l], ld = n + 1;
    const T* b = l ? d.b[l] : b0;
    T* xa = l ? d.x[l] : x0;
    const T* wx = d.wx[l];
    const T* wy = d.wy[l];
    T* cur = d.t[l];
    T* oth = xa;
    for_interior(n, [&](int p, int, int) {
      const T dg = wx[p] + wx[p - 1] + wy[p] + wy[p - ld];
      cur[p] = omega * b[p] / dg;
    });
    __syncthreads();
    for (int k = 1; k < nu; ++k) {
      for_interior(n, [&](int p, int, int) {
        T dg;
        const T ax = stiff(wx, wy, cur, p, ld, dg);
        oth[p] = cur[p] + omega * (b[p] - ax) / dg;
      });
      __syncthreads();
      T* tt = cur;
      cur = oth;
      oth = tt;
    }
    for_interior(n, [&](int p, int, int) {
      T dg;
      oth[p] = b[p] - stiff(wx, wy, cur, p, ld, dg);
    });
    __syncthreads();
    T* bc = d.b[l + 1];
    for_interior(n >> 1, [&](int P, int I, int J) {
      const int p = (2 * J) * ld + 2 * I;
      bc[P] = oth[p] + T(0.5) * ((oth[p + 1] + oth[p - 1]) + (oth[p + ld] + oth[p - ld]) +
                                 (oth[p + ld + 1] + oth[p - ld - 1]));
    });
    __syncthreads();
  }
  {
    // mesh 1/2: one unknown at padded index 4
    const T* b = (L - 1) ? d.b[L - 1] : b0;
    T* x = (L - 1) ? d.x[L - 1] : x0;
    if (threadIdx.x == 0) {
      const T* wx = d.wx[L - 1];
      const T* wy = d.wy[L - 1];
      x[4] = b[4] / (wx[4] + wx[3] + wy[4] + wy[1]);
    }
    __syncthreads();
  }
  for (int l = L - 2; l >= 0; --l) {
    const int n = d.n[l], ld = n + 1;
    const T* b = l ? d.b[l] : b0;
    T* xa = l ? d.x[l] : x0;
    const T* wx = d.wx[l];
    const T* wy = d.wy[l];
    T* cur = ((nu - 1) & 1) ? xa : d.t[l];
    T* oth = ((nu - 1) & 1) ? d.t[l] : xa;
    const T* xc = d.x[l + 1];
    const int ldc = (n >> 1) + 1;
    for_interior(n, [&](int p, int i, int j) {
      const int I = i >> 1, J = j >> 1;
      const int c0 = J * ldc + I;
      T v;
      if (!(i & 1) && !(j & 1)) v = xc[c0];
      else if ((i & 1) && !(j & 1)) v = T(0.5) * (xc[c0] + xc[c0 + 1]);
      else if (!(i & 1)) v = T(0.5) * (xc[c0] + xc[c0 + ldc]);
      else v = T(0.5) * (xc[c0] + xc[c0 + ldc + 1]);
      cur[p] += v;
    });
    __syncthreads();
    for (int k = 0; k < nu; ++k) {
      for_interior(n, [&](int p, int, int) {
        T dg;
        const T ax = stiff(wx, wy, cur, p, ld, dg);
        oth[p] = cur[p] + omega * (b[p] - ax) / dg;
      });
      __syncthreads();
      T* tt = cur;
      cur = oth;
      oth = tt;
    }
  }
}

template <typename T>
__device__ void zero_vec(T* v, int n) {
  for_all(gsz(n), [&](size_t q) { v[q] = T(0); });
}

// ---------------------------------------------------------------------------------------------
// small dense Rayleigh-Ritz for LOBPCG (one thread).  Basis [x, w, p] (k = 2 or 3); returns the
// number of basis vectors kept (0: failure) and c with c^T GM c = 1 for the smallest Ritz value.
__device__ int rayleigh_ritz(const double GA[3][3], const double GM[3][3], int k, double c[3], double& theta) {
  for (; k >= 2; --k) {
    double dsc[3], A[3][3], B[3][3], Lm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    bool ok = true;
    for (int i = 0; i < k; ++i) {
      if (!(GM[i][i] > 0.0)) ok = false;
      dsc[i] = ok ? 1.0 / sqrt(GM[i][i]) : 0.0;
    }
    if (!ok) continue;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        A[i][j] = dsc[i] * GA[i][j] * dsc[j];
        B[i][j] = dsc[i] * GM[i][j] * dsc[j];
      }
    for (int i = 0; i < k && ok; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = B[i][j];
        for (int m = 0; m < j; ++m) s -= Lm[i][m] * Lm[j][m];
        if (i == j) {
          if (!(s > 1e-12)) {
            ok = false;
            break;
          }
          Lm[i][i] = sqrt(s);
        } else {
          Lm[i][j] = s / Lm[j][j];
        }
      }
    if (!ok) continue;
    // C = L^{-1} A L^{-T}
    double Y[3][3], C[3][3];
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        double s = A[i][j];
        for (int m = 0; m < i; ++m) s -= Lm[i][m] * Y[m][j];
        Y[i][j] = s / Lm[i][i];
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double s = Y[i][j];
        for (int m = 0; m < j; ++m) s -= Lm[j][m] * C[i][m];
        C[i][j] = s / Lm[j][j];
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < i; ++j) C[i][j] = C[j][i] = 0.5 * (C[i][j] + C[j][i]);
    // cyclic Jacobi eigen-decomposition of the k x k symmetric C
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int i = 0; i < k; ++i) {
        dia += C[i][i] * C[i][i];
        for (int j = i + 1; j < k; ++j) off += C[i][j] * C[i][j];
      }
      if (off <= 1e-32 * dia) break;
      for (int pI = 0; pI < k - 1; ++pI)
        for (int qI = pI + 1; qI < k; ++qI) {
          const double apq = C[pI][qI];
          if (apq == 0.0) continue;
          const double tau = (C[qI][qI] - C[pI][pI]) / (2.0 * apq);
          const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
          for (int m = 0; m < k; ++m) {
            const double cmp = C[m][pI], cmq = C[m][qI];
            C[m][pI] = cs * cmp - sn * cmq;
            C[m][qI] = sn * cmp + cs * cmq;
          }
          for (int m = 0; m < k; ++m) {
            const double cpm = C[pI][m], cqm = C[qI][m];
            C[pI][m] = cs * cpm - sn * cqm;
            C[qI][m] = sn * cpm + cs * cqm;
          }
          for (int m = 0; m < k; ++m) {
            const double vmp = V[m][pI], vmq = V[m][qI];
            V[m][pI] = cs * vmp - sn * vmq;
            V[m][qI] = sn * vmp + cs * vmq;
          }
        }
    }
    int mi = 0;
    for (int i = 1; i < k; ++i)
      if (C[i][i] < C[mi][mi]) mi = i;
    theta = C[mi][mi];
    // c = D L^{-T} y
    double y[3] = {V[0][mi], V[1][mi], k > 2 ? V[2][mi] : 0.0};
    double cc[3] = {0, 0, 0};
    for (int i = k - 1; i >= 0; --i) {
      double s = y[i];
      for (int m = i + 1; m < k; ++m) s -= Lm[m][i] * cc[m];
      cc[i] = s / Lm[i][i];
    }
    for (int i = 0; i < 3; ++i) c[i] = i < k ? cc[i] * dsc[i] : 0.0;
    return k;
  }
  return 0;
}

struct EigShared {
  double c[3];   // x_new = c0 x + c1 w + c2 p
  double pc[2];  // p_new = pc0 w + pc1 p
  double theta;
  int k;
};

// LOBPCG for the smallest eigenpair of (A_H, M_H); x holds the start vector (not normalised).
// Returns iterations used, or -1 when the tolerance was not reached.  On return x is the
// M-normalised eigenvector with a positive sum and lam its Rayleigh quotient.
__device__ int lobpcg(CoarseWS& ws, int n, double tol, int maxit, int nu, double omega, double* red,
                      EigShared* sh, double& lam) {
  const int ld = n + 1;
  const double hm = 1.0 / (12.0 * n * n);
  const MGDesc<double>& mg = ws.mg;
  const double* wx = mg.wx[0];
  const double* wy = mg.wy[0];
  auto applyAM = [&](const double* u, double* Au, double* Mu, double& uAu, double& uMu) {
    double acc[2] = {0.0, 0.0}, o[2];
    for_interior(n, [&](int p, int, int) {
      double dg;
      const double au = stiff(wx, wy, u, p, ld, dg);
      const double mu = hm * mass7(u, p, ld);
      Au[p] = au;
      Mu[p] = mu;
      acc[0] += u[p] * au;
      acc[1] += u[p] * mu;
    });
    block_sum<2, double>(acc, o, red);
    uAu = o[0];
    uMu = o[1];
  };
  double xAx, xMx;
  applyAM(ws.x, ws.Ax, ws.Mx, xAx, xMx);
  {
    const double s = 1.0 / sqrt(xMx);
    for_interior(n, [&](int p, int, int) {
      ws.x[p] *= s;
      ws.Ax[p] *= s;
      ws.Mx[p] *= s;
    });
    __syncthreads();
  }
  double theta = xAx / xMx;
  bool have_p = false;
  int it = 0, conv = 0;
  for (; it < maxit; ++it) {
    {
      double acc[2] = {0.0, 0.0}, o[2];
      for_interior(n, [&](int p, int, int) {
        const double rv = ws.Ax[p] - theta * ws.Mx[p];
        ws.r[p] = rv;
        acc[0] += rv * rv;
        acc[1] += ws.Mx[p] * ws.Mx[p];
      });
      block_sum<2, double>(acc, o, red);
      if (sqrt(o[0]) <= tol * fabs(theta) * sqrt(o[1])) {
        conv = 1;
        break;
      }
    }
    vcycle<double>(mg, ws.r, ws.w, nu, omega);
    double g[12];
    {
      double acc[12];
      for (int i = 0; i < 12; ++i) acc[i] = 0.0;
      for_interior(n, [&](int p, int, int) {
        double dg;
        const double aw = stiff(wx, wy, ws.w, p, ld, dg);
        const double mw = hm * mass7(ws.w, p, ld);
        ws.Aw[p] = aw;
        ws.Mw[p] = mw;
        const double wv = ws.w[p], xv = ws.x[p];
        acc[0] += wv * aw;
        acc[1] += wv * mw;
        acc[2] += xv * aw;
        acc[3] += xv * mw;
        acc[4] += xv * ws.Ax[p];
        acc[5] += xv * ws.Mx[p];
        if (have_p) {
          const double pv = ws.p[p];
          acc[6] += pv * aw;
          acc[7] += pv * mw;
          acc[8] += xv * ws.Ap[p];
          acc[9] += xv * ws.Mp[p];
          acc[10] += pv * ws.Ap[p];
          acc[11] += pv * ws.Mp[p];
        }
      });
      block_sum<12, double>(acc, g, red);
    }
    if (threadIdx.x == 0) {
      double GA[3][3], GM[3][3];
      GA[0][0] = g[4];
      GM[0][0] = g[5];
      GA[1][1] = g[0];
      GM[1][1] = g[1];
      GA[0][1] = GA[1][0] = g[2];
      GM[0][1] = GM[1][0] = g[3];
      GA[2][2] = g[10];
      GM[2][2] = g[11];
      GA[1][2] = GA[2][1] = g[6];
      GM[1][2] = GM[2][1] = g[7];
      GA[0][2] = GA[2][0] = g[8];
      GM[0][2] = GM[2][0] = g[9];
      double c[3], th;
      const int k = rayleigh_ritz(GA, GM, have_p ? 3 : 2, c, th);
      if (k > 0) {
        if (c[0] < 0) {
          c[0] = -c[0];
          c[1] = -c[1];
          c[2] = -c[2];
        }
        // p_new = c1 w + c2 p, M-normalised
        const double pp = c[1] * c[1] * GM[1][1] + 2 * c[1] * c[2] * GM[1][2] + c[2] * c[2] * GM[2][2];
        const double ps = pp > 0 ? 1.0 / sqrt(pp) : 0.0;
        sh->pc[0] = c[1] * ps;
        sh->pc[1] = (k > 2 ? c[2] : 0.0) * ps;
        sh->c[0] = c[0];
        sh->c[1] = c[1];
        sh->c[2] = k > 2 ? c[2] : 0.0;
        sh->theta = th;
      }
      sh->k = k;
    }
    __syncthreads();
    const int k = sh->k;
    if (k == 0) break;
    const double c0 = sh->c[0], c1 = sh->c[1], c2 = sh->c[2], q0 = sh->pc[0], q1 = sh->pc[1];
    const bool use_p = have_p && k > 2;
    for_interior(n, [&](int p, int, int) {
      const double xv = ws.x[p], axv = ws.Ax[p], mxv = ws.Mx[p];
      const double wv = ws.w[p], awv = ws.Aw[p], mwv = ws.Mw[p];
      const double pv = use_p ? ws.p[p] : 0.0, apv = use_p ? ws.Ap[p] : 0.0, mpv = use_p ? ws.Mp[p] : 0.0;
      ws.x[p] = c0 * xv + c1 * wv + c2 * pv;
      ws.Ax[p] = c0 * axv + c1 * awv + c2 * apv;
      ws.Mx[p] = c0 * mxv + c1 * mwv + c2 * mpv;
      ws.p[p] = q0 * wv + q1 * pv;
      ws.Ap[p] = q0 * awv + q1 * apv;
      ws.Mp[p] = q0 * mwv + q1 * mpv;
    });
    __syncthreads();
    theta = sh->theta;
    have_p = true;
  }
  // final: fresh operator application, normalisation, sign
  double xA, xM;
  applyAM(ws.x, ws.Ax, ws.Mx, xA, xM);
  double sacc[1] = {0.0}, so[1];
  for_interior(n, [&](int p, int, int) { sacc[0] += ws.x[p]; });
  block_sum<1, double>(sacc, so, red);
  const double sc = (so[0] < 0 ? -1.0 : 1.0) / sqrt(xM);
  for_interior(n, [&](int p, int, int) { ws.x[p] *= sc; });
  __syncthreads();
  lam = xA / xM;
  return conv ? it : -1;
}

// ---------------------------------------------------------------------------------------------
// two-grid update on the fine mesh n: returns the Rayleigh quotient of the solution of
// (A - sigma M) w = M P u_H.  iters / outer report the inner MINRES iterations and refinement
// steps; flags receives kFlag* bits.
template <typename T>
__device__ double twogrid_fine(FineWS<T>& ws, char* fine_base, int n, const double* __restrict__ a,
                               const double* uH, int nc, double sigma, const SampleLaunch& P, double* red,
                               int& iters, int& outer, int& flags) {
  const int ld = n + 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    Carver f(fine_base);
    carve_fine<T>(f, n, ws);
  }
  __syncthreads();
  const double hm = 1.0 / (12.0 * n * n);
  // zero every vector of the region (boundary rings must be zero)
  zero_vec(ws.x64, n);
  zero_vec(ws.r64, n);
  zero_vec(ws.b64, n);
  zero_vec(ws.vo, n);
  zero_vec(ws.v, n);
  zero_vec(ws.z, n);
  zero_vec(ws.zn, n);
  zero_vec(ws.wo, n);
  zero_vec(ws.w, n);
  zero_vec(ws.q, n);
  zero_vec(ws.xi, n);
  for (int l = 0; l < ws.mg.L; ++l) {
    zero_vec(ws.mg.t[l], ws.mg.n[l]);
    if (l) {
      zero_vec(ws.mg.x[l], ws.mg.n[l]);
      zero_vec(ws.mg.b[l], ws.mg.n[l]);
    }
  }
  __syncthreads();
  const bool ok = build_mg<T>(ws.mg, a, n, red);
  if (!ok) flags |= kFlagBadCoef;
  if (sizeof(T) != sizeof(double)) {
    weights_from_cells<double, double>(n, a, a + (size_t)n * n, ws.wx64, ws.wy64);
    __syncthreads();
  }
  const double* wx = ws.wx64;
  const double* wy = ws.wy64;
  // b = M P u_H  (P: P1 interpolation from the nested coarse mesh)
  {
    const int lr = ilog2(n / nc);
    const int rm = (1 << lr) - 1;
    const int ldc = nc + 1;
    const double inv = 1.0 / (double)(1 << lr);
    for_interior(n, [&](int p, int i, int j) {
      const int I = i >> lr, J = j >> lr;
      const double xi_ = (double)(i & rm) * inv, et = (double)(j & rm) * inv;
      const int c0 = J * ldc + I;
      double v;
      if (xi_ >= et)
        v = (1.0 - xi_) * uH[c0] + (xi_ - et) * uH[c0 + 1] + et * uH[c0 + ldc + 1];
      else
        v = (1.0 - et) * uH[c0] + (et - xi_) * uH[c0 + ldc] + xi_ * uH[c0 + ldc + 1];
      ws.r64[p] = v;
    });
    __syncthreads();
    double acc[1] = {0.0}, o[1];
    for_interior(n, [&](int p, int, int) {
      const double bv = hm * mass7(ws.r64, p, ld);
      ws.b64[p] = bv;
      acc[0] += bv * bv;
    });
    block_sum<1, double>(acc, o, red);
    for_interior(n, [&](int p, int, int) { ws.r64[p] = ws.b64[p]; });
    __syncthreads();
    outer = 0;
    iters = 0;
    double bnorm = sqrt(o[0]);
    double rnorm = bnorm;
    const T sigm = T(sigma * hm);
    const T om = T(P.omega);
    const T* twx = ws.mg.wx[0];
    const T* twy = ws.mg.wy[0];
    for (; outer < P.max_outer; ++outer) {
      if (!(rnorm > P.tol_lin * bnorm)) break;
      // inner: MINRES on (A - sigma M) xi = r / ||r|| in precision T, preconditioned by the V-cycle
      const double rs = 1.0 / rnorm;
      for_interior(n, [&](int p, int, int) {
        ws.v[p] = T(ws.r64[p] * rs);
        ws.vo[p] = T(0);
        ws.w[p] = T(0);
        ws.wo[p] = T(0);
        ws.xi[p] = T(0);
      });
      __syncthreads();
      T* vo = ws.vo;
      T* v = ws.v;
      T* z = ws.z;
      T* zn = ws.zn;
      T* wo = ws.wo;
      T* w = ws.w;
      vcycle<T>(ws.mg, v, z, P.nu, om);
      double gam;
      {
        T acc1[1] = {T(0)};
        double o1[1];
        for_interior(n, [&](int p, int, int) { acc1[0] += v[p] * z[p]; });
        block_sum<1, T>(acc1, o1, red);
        gam = o1[0];
      }
      if (!(gam > 0.0)) {
        flags |= kFlagBreakdown;
        break;
      }
      gam = sqrt(gam);
      double eta = gam, eta0 = gam, gam_old = 1.0;
      double s_old = 0.0, s = 0.0, c_old = 1.0, c = 1.0;
      int j = 0;
      bool done = false;
      double cx = 0.0, a1 = 1.0, a2 = 0.0, a3 = 0.0;  // pending w/x update
      bool pending = false;
      for (; j < P.max_inner_it && !done; ++j) {
        // [pending update of w, x from the previous iteration] + q = K z / gam, delta
        const T ig = T(1.0 / gam);
        double delta;
        {
          T acc1[1] = {T(0)};
          double o1[1];
          const T ta1 = T(1.0 / a1), ta2 = T(a2), ta3 = T(a3), tcx = T(cx);
          T* zp = zn;  // z of the previous iteration (normalised) is in zn when pending
          for_interior(n, [&](int p, int, int) {
            if (pending) {
              const T wnew = (zp[p] - ta3 * wo[p] - ta2 * w[p]) * ta1;
              wo[p] = wnew;  // becomes w after the pointer swap below
              ws.xi[p] += tcx * wnew;
            }
            T dg;
            const T kz = (stiff(twx, twy, z, p, ld, dg) - sigm * mass7(z, p, ld)) * ig;
            ws.q[p] = kz;
            acc1[0] += kz * z[p];
          });
          block_sum<1, T>(acc1, o1, red);
          delta = o1[0] / gam;
          if (pending) {
            T* tt = wo;
            wo = w;
            w = tt;
          }
          pending = false;
        }
        // v_new = q - (delta/gam) v - (gam/gam_old) v_old ; z normalised in place
        {
          const T c1 = T(delta / gam), c2 = T(gam / gam_old);
          for_interior(n, [&](int p, int, int) {
            vo[p] = ws.q[p] - c1 * v[p] - c2 * vo[p];
            z[p] *= ig;
          });
          __syncthreads();
          T* tt = vo;
          vo = v;
          v = tt;  // v = v_new, vo = v_j
        }
        // zn = B^{-1} v_new, gamma_new
        vcycle<T>(ws.mg, v, zn, P.nu, om);
        double gnew;
        {
          T acc1[1] = {T(0)};
          double o1[1];
          for_interior(n, [&](int p, int, int) { acc1[0] += v[p] * zn[p]; });
          block_sum<1, T>(acc1, o1, red);
          gnew = o1[0];
        }
        if (!(gnew >= 0.0)) {
          flags |= kFlagBreakdown;
          gnew = 0.0;
        }
        gnew = sqrt(gnew);
        const double al0 = c * delta - c_old * s * gam;
        const double al1 = sqrt(al0 * al0 + gnew * gnew);
        const double al2 = s * delta + c_old * c * gam;
        const double al3 = s_old * gam;
        const double cn = al0 / al1, sn = gnew / al1;
        // w_new = (z_j - al3 w_old - al2 w)/al1 ; x += cn eta w_new   (applied lazily)
        // z_j is the normalised z (in buffer z); move it to zn's slot after swapping
        {
          T* tt = z;
          z = zn;
          zn = tt;  // z = z_{j+1} (unnormalised), zn = z_j (normalised)
        }
        cx = cn * eta;
        a1 = al1;
        a2 = al2;
        a3 = al3;
        pending = true;
        eta = -sn * eta;
        s_old = s;
        s = sn;
        c_old = c;
        c = cn;
        gam_old = gam;
        gam = gnew;
        if (fabs(eta) <= P.tol_inner * eta0 || gnew == 0.0) done = true;
      }
      if (pending) {
        const T ta1 = T(1.0 / a1), ta2 = T(a2), ta3 = T(a3), tcx = T(cx);
        for_interior(n, [&](int p, int, int) {
          const T wnew = (zn[p] - ta3 * wo[p] - ta2 * w[p]) * ta1;
          ws.xi[p] += tcx * wnew;
        });
        __syncthreads();
      }
      iters += j;
      if (!done) flags |= kFlagLinNoConv;
      // x64 += ||r|| xi ; r64 = b - (A - sigma M) x64 in FP64
      for_interior(n, [&](int p, int, int) { ws.x64[p] += rnorm * (double)ws.xi[p]; });
      __syncthreads();
      double acc2[1] = {0.0}, o2[1];
      for_interior(n, [&](int p, int, int) {
        double dg;
        const double kx = stiff(wx, wy, ws.x64, p, ld, dg) - sigma * hm * mass7(ws.x64, p, ld);
        const double rv = ws.b64[p] - kx;
        ws.r64[p] = rv;
        acc2[0] += rv * rv;
      });
      block_sum<1, double>(acc2, o2, red);
      const double rnew = sqrt(o2[0]);
      const bool stalled = !(rnew < 0.5 * rnorm);
      rnorm = rnew;
      if (stalled) {
        ++outer;
        break;
      }
    }
    if (!(rnorm <= P.tol_lin * bnorm) && !(rnorm < 1e-6 * bnorm)) flags |= kFlagLinNoConv;
  }
  // Rayleigh quotient in FP64
  double acc[2] = {0.0, 0.0}, o[2];
  for_interior(n, [&](int p, int, int) {
    double dg;
    const double x = ws.x64[p];
    acc[0] += x * stiff(wx, wy, ws.x64, p, ld, dg);
    acc[1] += x * hm * mass7(ws.x64, p, ld);
  });
  block_sum<2, double>(acc, o, red);
  return o[0] / o[1];
}

template <typename T>
__global__ void __launch_bounds__(512) sample_kernel(SampleLaunch P) {
  extern __shared__ __align__(256) char smem_dyn[];
  __shared__ double red[32 * 12 + 12];
  __shared__ EigShared esh;
  __shared__ CoarseWS cws;
  __shared__ FineWS<T> fws;
  char* base = P.use_smem ? smem_dyn : P.gscratch + (size_t)blockIdx.x * P.slab_bytes;
  size_t coarse_bytes;
  {
    Carver c(base);
    carve_coarse(c, P.nc, cws);  // every thread writes the same values
    coarse_bytes = (c.used() + 255) & ~(size_t)255;
  }
  char* fine_base = base + coarse_bytes;
  __syncthreads();
  const int nc = P.nc;
  const int cpr = (P.npts + P.chunk - 1) / P.chunk;
  const int nchunks = cpr * P.R;
  const size_t ncT = (size_t)2 * nc * nc, nfT = (size_t)2 * P.nf * P.nf, npT = (size_t)2 * P.np * P.np;
  // coarse vectors: zero once (rings stay zero; interiors are always written before use)
  {
    CoarseWS& w = cws;
    double* vs[11] = {w.x, w.Ax, w.Mx, w.w, w.Aw, w.Mw, w.p, w.Ap, w.Mp, w.r, w.uprev};
    for (int i = 0; i < 11; ++i) zero_vec(vs[i], nc);
    for (int l = 0; l < w.mg.L; ++l) {
      zero_vec(w.mg.t[l], w.mg.n[l]);
      if (l) {
        zero_vec(w.mg.x[l], w.mg.n[l]);
        zero_vec(w.mg.b[l], w.mg.n[l]);
      }
    }
    __syncthreads();
  }
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int r = ch / cpr;
    const int k0 = (ch % cpr) * P.chunk;
    const int k1 = min(k0 + P.chunk, P.npts);
    for (int kk = k0; kk < k1; ++kk) {
      const size_t b = (size_t)r * P.npts + kk;
      int flags = 0;
      // ---- coarse eigenpair (Algorithm 1 step 1; Algorithm 2 steps 6-7)
      CoarseWS& cw = cws;
      if (!build_mg<double>(cw.mg, P.a_c + b * ncT, nc, red)) flags |= kFlagBadCoef;
      if (kk == k0) {
        for_interior(nc, [&](int p, int i, int j) { cw.x[p] = sinpi((double)i / nc) * sinpi((double)j / nc); });
      } else {
        for_interior(nc, [&](int p, int, int) { cw.x[p] = cw.uprev[p]; });
      }
      __syncthreads();
      double lamH;
      const int eit = lobpcg(cw, nc, P.tol_eig, P.max_eig_it, P.nu, P.omega, red, &esh, lamH);
      if (eit < 0) flags |= kFlagEigNoConv;
      for_interior(nc, [&](int p, int, int) { cw.uprev[p] = cw.x[p]; });
      if (P.u_out) {
        for_interior(nc, [&](int p, int i, int j) { P.u_out[b * (size_t)(nc - 1) * (nc - 1) + (j - 1) * (nc - 1) + (i - 1)] = cw.x[p]; });
      }
      __syncthreads();
      // ---- fine two-grid updates (Algorithm 1 steps 2-4; Algorithm 2 steps 9-14)
      double lf = lamH, lp = 0.0;
      int itf = 0, itp = 0, of = 0, op = 0;
      if (!P.direct_f) lf = twogrid_fine<T>(fws, fine_base, P.nf, P.a_f + b * nfT, cw.x, nc, lamH, P, red, itf, of, flags);
      if (P.np > 0) {
        lp = lamH;
        if (!P.direct_p) lp = twogrid_fine<T>(fws, fine_base, P.np, P.a_p + b * npT, cw.x, nc, lamH, P, red, itp, op, flags);
      }
      if (threadIdx.x == 0) {
        P.out[b * 4 + 0] = lamH;
        P.out[b * 4 + 1] = lf;
        P.out[b * 4 + 2] = lp;
        P.out[b * 4 + 3] = lf - lp;
        P.stat[b * 4 + 0] = eit < 0 ? P.max_eig_it : eit;
        P.stat[b * 4 + 1] = itf;
        P.stat[b * 4 + 2] = itp;
        P.stat[b * 4 + 3] = flags;
        P.outer[b * 2 + 0] = of;
        P.outer[b * 2 + 1] = op;
      }
    }
  }
}

// Operator application for parity checks of the stencils: one CTA per coefficient field; the
// scratch holds three padded grids per field.  Uses the same weight builder and stencils as the
// solver.
__global__ void apply_kernel(int n, const double* __restrict__ a, int which, double sigma,
                             const double* __restrict__ x, double* __restrict__ y, double* scratch) {
  const size_t V = gsz(n);
  const size_t b = blockIdx.x;
  double* wx = scratch + b * 3 * V;
  double* wy = wx + V;
  double* xp = wy + V;
  const size_t nT = (size_t)2 * n * n, nI = (size_t)(n - 1) * (n - 1);
  const double* ab = a + b * nT;
  weights_from_cells<double, double>(n, ab, ab + (size_t)n * n, wx, wy);
  for_all(V, [&](size_t q) { xp[q] = 0.0; });
  __syncthreads();
  for_interior(n, [&](int p, int i, int j) { xp[p] = x[b * nI + (size_t)(j - 1) * (n - 1) + (i - 1)]; });
  __syncthreads();
  const int ld = n + 1;
  const double hm = 1.0 / (12.0 * n * n);
  for_interior(n, [&](int p, int i, int j) {
    double dg;
    const double ax = stiff(wx, wy, xp, p, ld, dg);
    const double mx = hm * mass7(xp, p, ld);
    y[b * nI + (size_t)(j - 1) * (n - 1) + (i - 1)] = which == 0 ? ax : which == 1 ? mx : ax - sigma * mx;
  });
}

// Per-shift sums of the per-sample differences over the points of a batch: one CTA per shift,
// fixed reduction order (deterministic).  flags receives the OR of all sample flags.
__global__ void shift_sums_kernel(const double* __restrict__ out, const int* __restrict__ stat, int npts,
                                  double* __restrict__ sums, int* __restrict__ flags) {
  __shared__ double red[32 * 2 + 2];
  const int r = blockIdx.x;
  double acc[1] = {0.0}, o[1];
  int f = 0;
  for (int k = threadIdx.x; k < npts; k += blockDim.x) {
    const size_t b = (size_t)r * npts + k;
    acc[0] += out[b * 4 + 3];
    f |= stat[b * 4 + 3];
  }
  block_sum<1, double>(acc, o, red);
  if (f) atomicOr(flags, f);
  if (threadIdx.x == 0) sums[r] = o[0];
}

}  // namespace

size_t sample_slab_bytes(int nf, int nc, int np, int mixed) {
  return mixed ? slab_size<float>(nf, nc, np) : slab_size<double>(nf, nc, np);
}

int sample_occupancy(int mixed, int threads, size_t smem) {
  int nb = 0;
  cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<float>, threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<double>, threads, smem);
  return e == cudaSuccess ? nb : 0;
}

int sample_static_smem(int mixed) {
  cudaFuncAttributes fa;
  cudaError_t e = mixed ? cudaFuncGetAttributes(&fa, sample_kernel<float>) : cudaFuncGetAttributes(&fa, sample_kernel<double>);
  return e == cudaSuccess ? (int)fa.sharedSizeBytes : 8192;
}

cudaError_t set_sample_smem(int mixed, int bytes) {
  return mixed ? cudaFuncSetAttribute(sample_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
               : cudaFuncSetAttribute(sample_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_apply_operator(int n, int B, const double* d_a, int which, double sigma, const double* d_x,
                                  double* d_y, double* d_scratch, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  apply_kernel<<<B, 256, 0, st>>>(n, d_a, which, sigma, d_x, d_y, d_scratch);
  return cudaGetLastError();
}

cudaError_t launch_shift_sums(const double* d_out, const int* d_stat, int R, int npts, double* d_sums, int* d_flags,
                              cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  shift_sums_kernel<<<R, 256, 0, st>>>(d_out, d_stat, npts, d_sums, d_flags);
  return cudaGetLastError();
}

cudaError_t launch_sample(const SampleLaunch& p, int mixed, int blocks, int threads, size_t smem, cudaStream_t st) {
  if (mixed)
    sample_kernel<float><<<blocks, threads, smem, st>>>(p);
  else
    sample_kernel<double><<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace mq
