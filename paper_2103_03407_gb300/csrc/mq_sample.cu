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
//   3. writes lambda_H, lambda^l, lambda^{l-1} and the difference (or, for the functional
//      quantity of interest, lambda_H and G of the two eigenfunction approximations and their
//      difference, G(u) = |integral of u| / ||u||_L2).
//
// With a reaction term (the second test problem of Sec. 5) every operator above is A + B, B the
// reaction matrix of b (seven-point form, see mq_device.cuh), and the V-cycles precondition with
// A + D_B (the lumped reaction).
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
#include <map>
#include <mutex>
#include <utility>

#include "mq_device.cuh"
#include "mq_internal.h"

namespace mq {
namespace {

using namespace dev;

// Coarse eigensolve workspace: FP64 LOBPCG basis, FP64 operator weights, FP32 preconditioner.
struct CoarseWS {
  MGDesc<float> mg;
  double *wx, *wy;
  double *rx, *ry, *rd;  // reaction edge weights (NULL without a reaction term)
  double *x, *Ax, *Mx, *w, *Aw, *Mw, *p, *Ap, *Mp, *uprev;
  float *r32, *w32;
};

// uprev comes first: it holds the coarse eigenvector through the fine solves (and as the warm
// start of the next point), while the rest of the coarse workspace is dead during the fine solves
// and shares its memory with the fine workspace.  *persist receives the bytes of that head.
__host__ __device__ void carve_coarse(Carver& c, int nc, CoarseWS& ws, size_t* persist = nullptr,
                                      bool reaction = false) {
  const size_t V = gsz(nc);
  ws.uprev = c.take<double>(V);
  if (persist) *persist = c.used();
  ws.wx = c.take<double>(V);
  ws.wy = c.take<double>(V);
  ws.rx = reaction ? c.take<double>(V) : nullptr;
  ws.ry = reaction ? c.take<double>(V) : nullptr;
  ws.rd = reaction ? c.take<double>(V) : nullptr;
  ws.x = c.take<double>(V);
  ws.Ax = c.take<double>(V);
  ws.Mx = c.take<double>(V);
  ws.w = c.take<double>(V);
  ws.Aw = c.take<double>(V);
  ws.Mw = c.take<double>(V);
  ws.p = c.take<double>(V);
  ws.Ap = c.take<double>(V);
  ws.Mp = c.take<double>(V);
  ws.r32 = c.take<float>(V);
  ws.w32 = c.take<float>(V);
  carve_mg<float>(c, nc, ws.mg, reaction);
}

// Fine shifted-solve workspace: FP64 solution and right-hand side, inner vectors in T.
template <typename T>
struct FineWS {
  MGDesc<T> mg;
  double *x64, *b64;
  T *vo, *v, *z, *zn, *wo, *w, *q, *xi;
  T *rx, *ry, *rd;  // reaction edge weights in the inner precision (NULL without a reaction term)
};

template <typename T>
__host__ __device__ void carve_fine(Carver& c, int n, FineWS<T>& ws, bool reaction = false) {
  const size_t V = gsz(n);
  ws.x64 = c.take<double>(V);
  ws.b64 = c.take<double>(V);
  ws.vo = c.take<T>(V);
  ws.v = c.take<T>(V);
  ws.z = c.take<T>(V);
  ws.zn = c.take<T>(V);
  ws.wo = c.take<T>(V);
  ws.w = c.take<T>(V);
  ws.q = c.take<T>(V);
  ws.xi = c.take<T>(V);
  ws.rx = reaction ? c.take<T>(V) : nullptr;
  ws.ry = reaction ? c.take<T>(V) : nullptr;
  ws.rd = reaction ? c.take<T>(V) : nullptr;
  carve_mg<T>(c, n, ws.mg, reaction);
}

template <typename T>
__host__ __device__ size_t fine_bytes(int n, bool reaction = false) {
  if (n < 2) return 0;
  Carver f(nullptr);
  FineWS<T> fw;
  carve_fine<T>(f, n, fw, reaction);
  return (f.used() + 15) & ~(size_t)15;
}

// workspace of one CTA: the persistent head, then the larger of the rest of the coarse region
// and the largest fine solve it performs in place (mode 0: inner precision T, mode 1: FP64 inner
// solve, 2: not in this kernel).  A multiple of 256 bytes: the slabs of a global scratch lie back
// to back, so every slab then starts as aligned as the scratch itself and the kernel carves it
// exactly as sized here (an unaligned slab start would shift its arrays by up to 15 bytes into
// the next slab).
template <typename T>
__host__ __device__ size_t slab_size(int nf, int nc, int np, int mode_f = 0, int mode_p = 0, bool reaction = false) {
  Carver c(nullptr);
  CoarseWS cw;
  size_t persist = 0;
  carve_coarse(c, nc, cw, &persist, reaction);
  persist = (persist + 15) & ~(size_t)15;  // the fine region starts 16-byte aligned
  const size_t coarse = (c.used() + 15) & ~(size_t)15;
  auto need = [&](int n, int mode) -> size_t {
    if (mode == 2) return 0;
    return mode == 1 ? fine_bytes<double>(n, reaction) : fine_bytes<T>(n, reaction);
  };
  size_t m = coarse - persist;
  const size_t a = need(nf, mode_f), b = need(np, mode_p);
  if (a > m) m = a;
  if (b > m) m = b;
  return (persist + m + 255) & ~(size_t)255;
}

// ---------------------------------------------------------------------------------------------
// Small dense Rayleigh-Ritz for LOBPCG, run by one thread.  The pencil is shifted by the current
// Ritz value in FP64 before it is rounded to FP32: the shifted Gram matrix GA - theta GM has
// entries of the size of the correction, so FP32 resolves the correction to FP32 relative
// accuracy (GB300 executes FP64 at a small fraction of the FP32 rate, and a single thread's FP64
// instruction costs a full warp's issue slot).  Basis [x, w, p] (k = 2 or 3).  Returns the number
// of basis vectors kept (0: failure), the coefficients c of the smallest Ritz vector and mu, the
// smallest eigenvalue of the shifted pencil (theta_new - theta).
__device__ int rayleigh_ritz_shifted(const float GAs[3][3], const float GM[3][3], int k, float c[3], float& mu) {
  for (; k >= 2; --k) {
    float dsc[3], A[3][3], B[3][3], Lm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    bool ok = true;
    for (int i = 0; i < k; ++i) {
      if (!(GM[i][i] > 0.0f)) ok = false;
      dsc[i] = ok ? rsqrtf(GM[i][i]) : 0.0f;
    }
    if (!ok) continue;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        A[i][j] = dsc[i] * GAs[i][j] * dsc[j];
        B[i][j] = dsc[i] * GM[i][j] * dsc[j];
      }
    for (int i = 0; i < k && ok; ++i)
      for (int j = 0; j <= i; ++j) {
        float s = B[i][j];
        for (int m = 0; m < j; ++m) s -= Lm[i][m] * Lm[j][m];
        if (i == j) {
          if (!(s > 1e-5f)) {
            ok = false;
            break;
          }
          Lm[i][i] = sqrtf(s);
        } else {
          Lm[i][j] = s / Lm[j][j];
        }
      }
    if (!ok) continue;
    float Y[3][3], C[3][3];
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        float s = A[i][j];
        for (int m = 0; m < i; ++m) s -= Lm[i][m] * Y[m][j];
        Y[i][j] = s / Lm[i][i];
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        float s = Y[i][j];
        for (int m = 0; m < j; ++m) s -= Lm[j][m] * C[i][m];
        C[i][j] = s / Lm[j][j];
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < i; ++j) C[i][j] = C[j][i] = 0.5f * (C[i][j] + C[j][i]);
    float V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 12; ++sweep) {
      float off = 0.0f, dia = 0.0f;
      for (int i = 0; i < k; ++i) {
        dia += C[i][i] * C[i][i];
        for (int j = i + 1; j < k; ++j) off += C[i][j] * C[i][j];
      }
      if (off <= 1e-14f * dia || off == 0.0f) break;
      for (int pI = 0; pI < k - 1; ++pI)
        for (int qI = pI + 1; qI < k; ++qI) {
          const float apq = C[pI][qI];
          if (apq == 0.0f) continue;
          const float tau = (C[qI][qI] - C[pI][pI]) / (2.0f * apq);
          const float t = (tau >= 0 ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
          const float cs = rsqrtf(1.0f + t * t), sn = t * cs;
          for (int m = 0; m < k; ++m) {
            const float cmp = C[m][pI], cmq = C[m][qI];
            C[m][pI] = cs * cmp - sn * cmq;
            C[m][qI] = sn * cmp + cs * cmq;
          }
          for (int m = 0; m < k; ++m) {
            const float cpm = C[pI][m], cqm = C[qI][m];
            C[pI][m] = cs * cpm - sn * cqm;
            C[qI][m] = sn * cpm + cs * cqm;
          }
          for (int m = 0; m < k; ++m) {
            const float vmp = V[m][pI], vmq = V[m][qI];
            V[m][pI] = cs * vmp - sn * vmq;
            V[m][qI] = sn * vmp + cs * vmq;
          }
        }
    }
    int mi = 0;
    for (int i = 1; i < k; ++i)
      if (C[i][i] < C[mi][mi]) mi = i;
    mu = C[mi][mi];
    float y[3] = {V[0][mi], V[1][mi], k > 2 ? V[2][mi] : 0.0f};
    float cc[3] = {0, 0, 0};
    for (int i = k - 1; i >= 0; --i) {
      float s = y[i];
      for (int m = i + 1; m < k; ++m) s -= Lm[m][i] * cc[m];
      cc[i] = s / Lm[i][i];
    }
    for (int i = 0; i < 3; ++i) c[i] = i < k ? cc[i] * dsc[i] : 0.0f;
    return k;
  }
  return 0;
}

struct EigShared {
  double c[3];   // x_new = c0 x + c1 w + c2 p
  double pc[2];  // p_new = pc0 w + pc1 p
  double theta;
  double scale;  // normalisation factor
  int k;
  int conv;
};

// LOBPCG for the smallest eigenpair of (A_H, M_H), preconditioned by one FP32 V-cycle on A_H
// (A_H + B_H and A_H + D_B with a reaction term).  x holds the start vector.  Returns the
// iterations used, or -1 when the tolerance was not reached.  On return x is the M-normalised
// eigenvector with a positive sum, lam its Rayleigh quotient and g = |integral of x| (= G(x)).
__device__ __noinline__ int lobpcg(CoarseWS& ws, int n, double tol, int maxit, int nu, float omega, double* red, EigShared* sh,
                      double& lam, double& g) {
  const int ld = n + 1;
  const int nact = (n - 1) * n;  // threads for_interior gives work to
  const double hm = 1.0 / (12.0 * n * n);
  const double* __restrict__ wx = ws.wx;
  const double* __restrict__ wy = ws.wy;
  const double* __restrict__ rx = ws.rx;
  const double* __restrict__ ry = ws.ry;
  const double* __restrict__ rd = ws.rd;
  // the operator A (+ B): stiffness and, with a reaction term, the reaction's seven-point form
  auto opA = [&](const double* u, int p) {
    const double au = stiff<double, double>(wx, wy, u, p, ld);
    return rx ? au + hm * react7<double, double>(rx, ry, rd, u, p, ld) : au;
  };
  auto applyAM = [&](const double* u, double* Au, double* Mu, double& uAu, double& uMu) {
    double acc[2] = {0.0, 0.0}, o[2];
    for_interior(n, [&](int p, int, int) {
      const double au = opA(u, p);
      const double mu = hm * mass7(u, p, ld);
      Au[p] = au;
      Mu[p] = mu;
      acc[0] += u[p] * au;
      acc[1] += u[p] * mu;
    });
    block_sum<2, double>(
        acc, o, red, [&](const double* t) { sh->scale = (double)rsqrtf((float)t[1]); sh->theta = t[0] / t[1]; }, nact);
    uAu = o[0];
    uMu = o[1];
  };
  double xAx, xMx;
  applyAM(ws.x, ws.Ax, ws.Mx, xAx, xMx);
  {
    const double s = sh->scale;
    for_interior(n, [&](int p, int, int) {
      ws.x[p] *= s;
      ws.Ax[p] *= s;
      ws.Mx[p] *= s;
    });
    __syncthreads();
  }
  double theta = sh->theta;
  bool have_p = false;
  int it = 0, conv = 0;
  for (; it < maxit; ++it) {
    {
      double acc[2] = {0.0, 0.0}, o[2];
      for_interior(n, [&](int p, int, int) {
        const double rv = ws.Ax[p] - theta * ws.Mx[p];
        ws.r32[p] = (float)rv;
        acc[0] += rv * rv;
        acc[1] += ws.Mx[p] * ws.Mx[p];
      });
      block_sum<2, double>(
          acc, o, red, [&](const double* t) { sh->conv = t[0] <= tol * tol * theta * theta * t[1]; }, nact);
      if (sh->conv) {
        conv = 1;
        break;
      }
    }
    vcycle<float>(ws.mg, ws.r32, ws.w32, omega, nullptr, nu);
    for_interior(n, [&](int p, int, int) { ws.w[p] = (double)ws.w32[p]; });
    __syncthreads();
    double g[12];
    {
      double acc[12];
      for (int i = 0; i < 12; ++i) acc[i] = 0.0;
      for_interior(n, [&](int p, int, int) {
        const double aw = opA(ws.w, p);
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
      const bool hp = have_p;
      block_sum<12, double>(acc, g, red, [&](const double* gg) {
        // Gram matrices of the basis [x, w, p]
        double GA[3][3], GM[3][3];
        GA[0][0] = gg[4];
        GM[0][0] = gg[5];
        GA[1][1] = gg[0];
        GM[1][1] = gg[1];
        GA[0][1] = GA[1][0] = gg[2];
        GM[0][1] = GM[1][0] = gg[3];
        GA[2][2] = gg[10];
        GM[2][2] = gg[11];
        GA[1][2] = GA[2][1] = gg[6];
        GM[1][2] = GM[2][1] = gg[7];
        GA[0][2] = GA[2][0] = gg[8];
        GM[0][2] = GM[2][0] = gg[9];
        const int kk = hp ? 3 : 2;
        const double th0 = GA[0][0] / GM[0][0];  // Rayleigh quotient of the current x
        float As[3][3], Mf[3][3];
        for (int i = 0; i < kk; ++i)
          for (int j = 0; j < kk; ++j) {
            As[i][j] = (float)(GA[i][j] - th0 * GM[i][j]);
            Mf[i][j] = (float)GM[i][j];
          }
        float cf[3], mu;
        const int k = rayleigh_ritz_shifted(As, Mf, kk, cf, mu);
        if (k > 0) {
          if (cf[0] < 0) {
            cf[0] = -cf[0];
            cf[1] = -cf[1];
            cf[2] = -cf[2];
          }
          // Rayleigh quotient of the new iterate from the FP64 Gram matrices; approximate
          // normalisations (the Gram matrices are recomputed every iteration)
          const double c0 = cf[0], c1 = cf[1], c2 = k > 2 ? cf[2] : 0.0;
          double ca = 0.0, cm = 0.0;
          const double cv[3] = {c0, c1, c2};
          for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
              ca += cv[i] * GA[i][j] * cv[j];
              cm += cv[i] * GM[i][j] * cv[j];
            }
          const float xs = rsqrtf((float)cm);
          const float pp = cf[1] * cf[1] * Mf[1][1] + 2 * cf[1] * (k > 2 ? cf[2] : 0.0f) * Mf[1][2] +
                           (k > 2 ? cf[2] * cf[2] * Mf[2][2] : 0.0f);
          const float ps = pp > 0 ? rsqrtf(pp) : 0.0f;
          sh->pc[0] = cf[1] * ps;
          sh->pc[1] = (k > 2 ? cf[2] : 0.0f) * ps;
          sh->c[0] = c0 * xs;
          sh->c[1] = c1 * xs;
          sh->c[2] = c2 * xs;
          sh->theta = ca / cm;
        }
        sh->k = k;
      }, nact);
    }
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
  block_sum<1, double>(sacc, so, red, [&](const double* t) {
    sh->scale = (t[0] < 0 ? -1.0 : 1.0) / sqrt(xM);
    sh->theta = xA / xM;
    // the integral of a P1 function with zero boundary values is h^2 times the sum of its nodal
    // values (each interior hat function integrates to h^2)
    sh->c[0] = fabs(t[0]) / ((double)n * n * sqrt(xM));
  }, nact);
  const double sc = sh->scale;
  for_interior(n, [&](int p, int, int) { ws.x[p] *= sc; });
  __syncthreads();
  lam = sh->theta;
  g = sh->c[0];
  return conv ? it : -1;
}

// MINRES scalars, owned by thread 0 and read by all threads after each reduction.  The
// recurrences run in the inner precision T (FP32 on the mixed path), the refinement norms in FP64.
template <typename T>
struct MinresShared {
  T gam, gam_old, eta, eta0, c, c_old, s, s_old;
  T ig;           // 1 / gamma_j
  T c1, c2;       // v_new = q - c1 v - c2 v_old
  T cx, ia1, a2, a3;  // pending w / x update
  T delta;
  T rs;           // 1 / ||r|| of the refinement residual
  double rnorm, bnorm;
  double knorm, xnorm;  // ||A - sigma M|| bound and ||x|| for the FP64 residual floor
  double xax, xmx;      // x.Ax and x.Mx of the last FP64 residual pass (the Rayleigh quotient)
  double xsum;          // sum of the nodal values of x in that pass (h^2 xsum = integral of x)
  int done, breakdown;
};

// Residual target of the refinement: tol relative to ||b||, but never below a small multiple of
// the FP64 rounding floor eps (||K|| ||x|| + ||b||) of the residual itself (on fine meshes the
// near-singular shifted system puts that floor above 1e-7 ||b||).
__host__ __device__ inline double residual_target(double tol, double bnorm, double knorm, double xnorm, double f) {
  const double floor_ = f * 2.220446049250313e-16 * (knorm * xnorm + bnorm);
  const double t = tol * bnorm;
  return t > floor_ ? t : floor_;
}

// ---------------------------------------------------------------------------------------------
// two-grid update on the fine mesh n: returns the Rayleigh quotient of the solution of
// (A - sigma M) w = M P u_H (A + B - sigma M with the reaction coefficient rb), and in gq the
// functional G(w) = |integral of w| / ||w||_L2.  iters / outer report the inner MINRES iterations
// and refinement steps; flags receives kFlag* bits.
template <typename T>
__device__ __noinline__ double twogrid_fine(FineWS<T>& ws, char* fine_base, int n, const double* __restrict__ a,
                               const double* __restrict__ rb, const double* uH, int nc, double sigma,
                               const SampleLaunch& P, double* red, MinresShared<T>* ms, int& iters, int& outer,
                               int& flags, double& gq) {
  const int ld = n + 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    Carver f(fine_base);
    carve_fine<T>(f, n, ws, rb != nullptr);
  }
  __syncthreads();
  const double hm = 1.0 / (12.0 * n * n);
  zero_vec(ws.x64, n);
  zero_vec(ws.b64, n);
  zero_vec(ws.vo, n);
  zero_vec(ws.v, n);
  zero_vec(ws.z, n);
  zero_vec(ws.zn, n);
  zero_vec(ws.wo, n);
  zero_vec(ws.w, n);
  zero_vec(ws.q, n);
  zero_vec(ws.xi, n);
  if (rb) {
    zero_vec(ws.rx, n);
    zero_vec(ws.ry, n);
    zero_vec(ws.rd, n);
  }
  zero_mg(ws.mg);
  __syncthreads();
  if (!build_mg<T>(ws.mg, a, n, red, rb)) flags |= kFlagBadCoef;
  if (rb) reaction_weights<T, double>(n, rb, rb + (size_t)n * n, ws.rx, ws.ry, ws.rd);
  {
    // ||A + B - sigma M||_inf <= 8 max a + (max b + sigma) h^2 (row sums of the edge form, of the
    // reaction and of the mass)
    double amax = 0.0, bmax = 0.0;
    for_all((size_t)2 * n * n, [&](size_t q) {
      amax = fmax(amax, a[q]);
      if (rb) bmax = fmax(bmax, rb[q]);
    });
    for (int off = 16; off > 0; off >>= 1) {
      amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, off));
      bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = amax;
      red[32 + (threadIdx.x >> 5)] = bmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0, mb = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        m = fmax(m, red[w]);
        mb = fmax(mb, red[32 + w]);
      }
      ms->knorm = 8.0 * m + (mb + sigma) / ((double)n * n);
      ms->xnorm = 0.0;
      ms->xax = ms->xmx = 0.0;
    }
    __syncthreads();
  }
  // FP64 operator for the residual and the Rayleigh quotient: the FP64 weights of level 0 when the
  // inner precision is FP64, otherwise weights formed on the fly from the centroid coefficients
  const bool w64 = sizeof(T) == sizeof(double);
  const double* wx64 = (const double*)ws.mg.wx[0];
  const double* wy64 = (const double*)ws.mg.wy[0];
  auto K64 = [&](const double* x, int p, int i, int j) {
    double k = w64 ? stiff<double, double>(wx64, wy64, x, p, ld) : stiff_cells(a, n, x, p, ld, i, j);
    if (rb)
      k += hm * (w64 ? react7<double, double>((const double*)ws.rx, (const double*)ws.ry, (const double*)ws.rd, x, p, ld)
                     : react_cells(rb, n, x, p, ld, i, j));
    return k;
  };
  // b = M P u_H  (P: P1 interpolation from the nested coarse mesh); x64 holds P u_H for a moment
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
      ws.x64[p] = v;
    });
    __syncthreads();
    double acc[1] = {0.0}, o[1];
    for_interior(n, [&](int p, int, int) {
      const double bv = hm * mass7(ws.x64, p, ld);
      ws.b64[p] = bv;
      ws.v[p] = T(bv);
      acc[0] += bv * bv;
    });
    block_sum<1, double>(acc, o, red, [&](const double* t) {
      ms->bnorm = ms->rnorm = sqrt(t[0]);
      ms->rs = T(1.0 / ms->rnorm);
    });
    for_interior(n, [&](int p, int, int) { ws.x64[p] = 0.0; });
    __syncthreads();
  }
  outer = 0;
  iters = 0;
  const T sigm = T(sigma * hm);
  const T hmt = T(hm);
  const T om = T(P.omega);
  const T* twx = ws.mg.wx[0];
  const T* twy = ws.mg.wy[0];
  const T* trx = ws.rx;
  const T* try_ = ws.ry;
  const T* trd = ws.rd;
  for (; outer < P.max_outer; ++outer) {
    if (!(ms->rnorm > residual_target(P.tol_lin, ms->bnorm, ms->knorm, ms->xnorm, 16.0))) break;
    // inner: MINRES on (A - sigma M) xi = r / ||r|| in precision T, preconditioned by the V-cycle;
    // v holds r (unscaled)
    const T rs = ms->rs;
    for_interior(n, [&](int p, int, int) {
      ws.v[p] *= rs;
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
    {
      T acc1[1] = {vcycle<T>(ws.mg, v, z, om, v, P.nu)};  // z = B^{-1} v and <v, z>
      double o1[1];
      block_sum<1, T>(acc1, o1, red, [&](const double* t) {
        const T t0 = T(t[0]);
        ms->breakdown = !(t0 > T(0));
        const T g = ms->breakdown ? T(1) : sqrt(t0);
        ms->gam = g;
        ms->eta = ms->eta0 = g;
        ms->gam_old = T(1);
        ms->c = ms->c_old = T(1);
        ms->s = ms->s_old = T(0);
        ms->ig = T(1) / g;
        ms->done = ms->breakdown;
      });
    }
    if (ms->breakdown) {
      flags |= kFlagBreakdown;
      break;
    }
    int j = 0;
    bool pending = false;
    for (; j < P.max_inner_it && !ms->done; ++j) {
      // [pending w/x update of the previous iteration] + q = K z / gamma, delta
      {
        T acc1[1] = {T(0)};
        double o1[1];
        const T ig = ms->ig;
        const T ta1 = ms->ia1, ta2 = ms->a2, ta3 = ms->a3, tcx = ms->cx;
        const bool pend = pending;
        const T* zp = zn;
        for_interior(n, [&](int p, int, int) {
          if (pend) {
            const T wnew = (zp[p] - ta3 * wo[p] - ta2 * w[p]) * ta1;
            wo[p] = wnew;
            ws.xi[p] += tcx * wnew;
          }
          T kz = stiff<T, T>(twx, twy, z, p, ld) - sigm * mass7(z, p, ld);
          if (trx) kz += hmt * react7<T, T>(trx, try_, trd, z, p, ld);
          kz *= ig;
          ws.q[p] = kz;
          acc1[0] += kz * z[p];
        });
        block_sum<1, T>(acc1, o1, red, [&](const double* t) {
          const T delta = T(t[0]) * ms->ig;
          ms->c1 = delta * ms->ig;
          ms->c2 = ms->gam / ms->gam_old;
          ms->delta = delta;
        });
        if (pend) {
          T* tt = wo;
          wo = w;
          w = tt;
        }
      }
      // v_new = q - (delta/gam) v - (gam/gam_old) v_old ; z normalised in place
      {
        const T c1 = ms->c1, c2 = ms->c2, ig = ms->ig;
        for_interior(n, [&](int p, int, int) {
          vo[p] = ws.q[p] - c1 * v[p] - c2 * vo[p];
          z[p] *= ig;
        });
        __syncthreads();
        T* tt = vo;
        vo = v;
        v = tt;
      }
      {
        T acc1[1] = {vcycle<T>(ws.mg, v, zn, om, v, P.nu)};  // zn = B^{-1} v_new and <v_new, zn>
        double o1[1];
        const T tol = T(P.tol_inner);
        block_sum<1, T>(acc1, o1, red, [&](const double* t) {
          T gnew = T(t[0]);
          if (!(gnew >= T(0))) {
            ms->breakdown = 1;
            gnew = T(0);
          }
          gnew = sqrt(gnew);
          const T delta = ms->delta, gam = ms->gam;
          const T al0 = ms->c * delta - ms->c_old * ms->s * gam;
          const T al1 = sqrt(al0 * al0 + gnew * gnew);
          const T al2 = ms->s * delta + ms->c_old * ms->c * gam;
          const T al3 = ms->s_old * gam;
          const T ia1 = T(1) / al1;
          const T cn = al0 * ia1, sn = gnew * ia1;
          ms->cx = cn * ms->eta;
          ms->ia1 = ia1;
          ms->a2 = al2;
          ms->a3 = al3;
          ms->eta = -sn * ms->eta;
          ms->s_old = ms->s;
          ms->s = sn;
          ms->c_old = ms->c;
          ms->c = cn;
          ms->gam_old = gam;
          ms->gam = gnew;
          ms->ig = gnew > T(0) ? T(1) / gnew : T(0);
          ms->done = fabs(ms->eta) <= tol * ms->eta0 || gnew == T(0) || ms->breakdown;
        });
        T* tt = z;
        z = zn;
        zn = tt;  // z = z_{j+1} (unnormalised), zn = z_j (normalised)
        pending = true;
      }
    }
    if (pending) {
      const T ta1 = ms->ia1, ta2 = ms->a2, ta3 = ms->a3, tcx = ms->cx;
      for_interior(n, [&](int p, int, int) {
        const T wnew = (zn[p] - ta3 * wo[p] - ta2 * w[p]) * ta1;
        ws.xi[p] += tcx * wnew;
      });
      __syncthreads();
    }
    iters += j;
    if (ms->breakdown) flags |= kFlagBreakdown;
    if (!ms->done) flags |= kFlagLinNoConv;
    // x64 += ||r|| xi ; r = b - (A - sigma M) x64 in FP64, stored (unscaled) in v
    const double rn = ms->rnorm;
    for_interior(n, [&](int p, int, int) { ws.x64[p] += rn * (double)ws.xi[p]; });
    __syncthreads();
    // the same pass forms x.Ax, x.Mx and sum(x): the last one gives the Rayleigh quotient and the
    // functional of the result
    double acc2[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, o2[5];
    for_interior(n, [&](int p, int i, int j) {
      const double xv = ws.x64[p];
      const double ax = K64(ws.x64, p, i, j);
      const double mx = hm * mass7(ws.x64, p, ld);
      const double rv = ws.b64[p] - (ax - sigma * mx);
      ws.v[p] = T(rv);
      acc2[0] += rv * rv;
      acc2[1] += xv * xv;
      acc2[2] += xv * ax;
      acc2[3] += xv * mx;
      acc2[4] += xv;
    });
    int stalled = 0;
    const int first = outer == 0;
    block_sum<5, double>(acc2, o2, red, [&](const double* t) {
      const double rnew = sqrt(t[0]);
      ms->xnorm = sqrt(t[1]);
      ms->xax = t[2];
      ms->xmx = t[3];
      ms->xsum = t[4];
      // no progress: stop refining (not after the first step, whose FP32 rounding noise can
      // leave a residual above ||b|| on fine meshes)
      ms->done = !first && !(rnew < 0.5 * ms->rnorm);
      ms->rnorm = rnew;
      ms->rs = T(1.0 / rnew);
    });
    stalled = ms->done;
    if (stalled) {
      ++outer;
      break;
    }
  }
  // flagged only well above the target (or the FP64 floor): the refinement may stop a little short
  if (!(ms->rnorm <= residual_target(fmax(1e-5, 10.0 * P.tol_lin), ms->bnorm, ms->knorm, ms->xnorm, 256.0)))
    flags |= kFlagLinNoConv;
  // Rayleigh quotient and functional in FP64, from the residual pass over the final iterate
  gq = fabs(ms->xsum) / ((double)n * n * sqrt(ms->xmx));
  return ms->xax / ms->xmx;
}

template <typename T>
__global__ void __launch_bounds__(512) sample_kernel(SampleLaunch P) {
  extern __shared__ __align__(16) char smem_dyn[];
  __shared__ double red[kRedSlots];
  __shared__ EigShared esh;
  __shared__ MinresShared<T> msh;
  __shared__ MinresShared<double> msh64;
  __shared__ CoarseWS cws;
  __shared__ FineWS<T> fws;
  __shared__ FineWS<double> fws64;
  char* base = P.use_smem ? smem_dyn : P.gscratch + (size_t)blockIdx.x * P.slab_bytes;
  size_t persist_bytes;
  const bool rxn = P.reaction != 0;
  {
    Carver c(base);
    CoarseWS tmp;
    carve_coarse(c, P.nc, tmp, &persist_bytes, rxn);
    if (threadIdx.x == 0) cws = tmp;
  }
  char* fine_base = base + ((persist_bytes + 15) & ~(size_t)15);  // the fine workspace overlays the coarse one
  __syncthreads();
  const int nc = P.nc;
  const int cpr = (P.npts + P.chunk - 1) / P.chunk;
  const int nchunks = cpr * P.R;
  const size_t ncT = (size_t)2 * nc * nc, nfT = (size_t)2 * P.nf * P.nf, npT = (size_t)2 * P.np * P.np;
  // the persistent coarse eigenvector: zero once (its ring stays zero)
  zero_vec(cws.uprev, nc);
  __syncthreads();
  const float omega = (float)P.omega;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int r = ch / cpr;
    const int k0 = (ch % cpr) * P.chunk;
    const int k1 = min(k0 + P.chunk, P.npts);
    for (int kk = k0; kk < k1; ++kk) {
      const size_t b = (size_t)r * P.npts + kk;
      int flags = 0;
      // ---- coarse eigenpair (Algorithm 1 step 1; Algorithm 2 steps 6-7), or, in the reuse scheme
      // across levels, the level-0 eigenpair of this point given in u_in / out[b][0]
      CoarseWS& cw = cws;
      double lamH, gH = 0.0;
      int eit = 0;
      if (P.u_in) {
        const size_t Vc = gsz(nc);
        for_all(Vc, [&](size_t q) { cw.uprev[q] = P.u_in[b * Vc + q]; });
        lamH = P.out[b * 4 + 0];
        __syncthreads();
        if (P.qoi && (P.direct_f || (P.np > 0 && P.direct_p && !P.prev_given))) {
          // G(u_H) of the given (M-normalised) eigenvector: h^2 |sum u| / sqrt(u^T M u)
          const double hmc = 1.0 / (12.0 * nc * nc);
          double acc[2] = {0.0, 0.0}, o[2];
          for_interior(nc, [&](int p, int, int) {
            acc[0] += cw.uprev[p];
            acc[1] += cw.uprev[p] * hmc * mass7(cw.uprev, p, nc + 1);
          });
          block_sum<2, double>(acc, o, red);
          gH = fabs(o[0]) / ((double)nc * nc * sqrt(o[1]));
        }
      } else {
        // the fine solves of the previous point reused this memory: clear the coarse vectors
        // (rings must be zero; interiors are written before use)
        double* vs[11] = {cw.wx, cw.wy, cw.x, cw.Ax, cw.Mx, cw.w, cw.Aw, cw.Mw, cw.p, cw.Ap, cw.Mp};
        for (int i = 0; i < 11; ++i) zero_vec(vs[i], nc);
        if (rxn) {
          zero_vec(cw.rx, nc);
          zero_vec(cw.ry, nc);
          zero_vec(cw.rd, nc);
        }
        zero_vec(cw.r32, nc);
        zero_vec(cw.w32, nc);
        zero_mg(cw.mg);
        __syncthreads();
        const double* ac = P.a_c + b * ncT;
        const double* bc = rxn ? P.b_c + b * ncT : nullptr;
        if (!build_mg<float>(cw.mg, ac, nc, red, bc)) flags |= kFlagBadCoef;
        weights_from_cells<double, double>(nc, ac, ac + (size_t)nc * nc, cw.wx, cw.wy);
        if (rxn) reaction_weights<double, double>(nc, bc, bc + (size_t)nc * nc, cw.rx, cw.ry, cw.rd);
        if (kk == k0) {
          const float inc = 1.0f / (float)nc;
          for_interior(nc, [&](int p, int i, int j) { cw.x[p] = (double)(sinpif(i * inc) * sinpif(j * inc)); });
        } else {
          for_interior(nc, [&](int p, int, int) { cw.x[p] = cw.uprev[p]; });
        }
        __syncthreads();
        eit = lobpcg(cw, nc, P.tol_eig, P.max_eig_it, P.nu, omega, red, &esh, lamH, gH);
        if (eit < 0) flags |= kFlagEigNoConv;
        for_interior(nc, [&](int p, int, int) { cw.uprev[p] = cw.x[p]; });
        if (P.u_out) {
          for_interior(nc, [&](int p, int i, int j) {
            P.u_out[b * (size_t)(nc - 1) * (nc - 1) + (j - 1) * (nc - 1) + (i - 1)] = cw.x[p];
          });
        }
        if (P.u_pad) {
          const size_t Vc = gsz(nc);
          for_all(Vc, [&](size_t q) { P.u_pad[b * Vc + q] = cw.x[q]; });
        }
        __syncthreads();
      }
      // ---- fine two-grid updates (Algorithm 1 steps 2-4; Algorithm 2 steps 9-14); a solve of
      // mode 2 runs elsewhere and leaves the coarse eigenvalue as a placeholder
      // the quantity of interest of a level whose eigenpair is the coarse one: lambda_H or G(u_H)
      // (the reuse scheme gives coarse pairs only to levels that solve their own fine problems)
      const double qH = P.qoi ? gH : lamH;
      double lf = qH, lp = P.np > 0 ? qH : 0.0;
      double gf = 0.0, gp = 0.0;
      int itf = 0, itp = 0, of = 0, op = 0;
      const double* rbf = rxn ? P.b_f + b * nfT : nullptr;
      const double* rbp = rxn ? P.b_p + b * npT : nullptr;
      if (!P.direct_f) {
        if (P.mode_f == 0)
          lf = twogrid_fine<T>(fws, fine_base, P.nf, P.a_f + b * nfT, rbf, cw.uprev, nc, lamH, P, red, &msh, itf, of,
                               flags, gf);
        else if (P.mode_f == 1)
          lf = twogrid_fine<double>(fws64, fine_base, P.nf, P.a_f + b * nfT, rbf, cw.uprev, nc, lamH, P, red, &msh64,
                                    itf, of, flags, gf);
        if (P.qoi && P.mode_f != 2) lf = gf;
      }
      if (P.prev_given) {
        lp = P.out[b * 4 + 2];  // every thread reads it before thread 0 rewrites the same value below
      } else if (P.np > 0 && !P.direct_p) {
        if (P.mode_p == 0)
          lp = twogrid_fine<T>(fws, fine_base, P.np, P.a_p + b * npT, rbp, cw.uprev, nc, lamH, P, red, &msh, itp, op,
                               flags, gp);
        else if (P.mode_p == 1)
          lp = twogrid_fine<double>(fws64, fine_base, P.np, P.a_p + b * npT, rbp, cw.uprev, nc, lamH, P, red, &msh64,
                                    itp, op, flags, gp);
        if (P.qoi && P.mode_p != 2) lp = gp;
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
// scratch holds four padded grids per field.  Uses the same weight builders and stencils as the
// solver.  which: 0 stiffness, 1 mass, 2 stiffness - sigma mass; 3 the reaction matrix of the
// field (edge-weight form), 4 the same from the centroid values (the FP64 residual's form).
__global__ void apply_kernel(int n, const double* __restrict__ a, int which, double sigma,
                             const double* __restrict__ x, double* __restrict__ y, double* scratch) {
  const size_t V = gsz(n);
  const size_t b = blockIdx.x;
  double* wx = scratch + b * 4 * V;
  double* wy = wx + V;
  double* xp = wy + V;
  double* wd = xp + V;
  const size_t nT = (size_t)2 * n * n, nI = (size_t)(n - 1) * (n - 1);
  const double* ab = a + b * nT;
  if (which == 3)
    reaction_weights<double, double>(n, ab, ab + (size_t)n * n, wx, wy, wd);
  else
    weights_from_cells<double, double>(n, ab, ab + (size_t)n * n, wx, wy);
  for_all(V, [&](size_t q) { xp[q] = 0.0; });
  __syncthreads();
  for_interior(n, [&](int p, int i, int j) { xp[p] = x[b * nI + (size_t)(j - 1) * (n - 1) + (i - 1)]; });
  __syncthreads();
  const int ld = n + 1;
  const double hm = 1.0 / (12.0 * n * n);
  for_interior(n, [&](int p, int i, int j) {
    double v;
    if (which == 3) {
      v = hm * react7<double, double>(wx, wy, wd, xp, p, ld);
    } else if (which == 4) {
      v = hm * react_cells(ab, n, xp, p, ld, i, j);
    } else {
      const double ax = stiff<double, double>(wx, wy, xp, p, ld);
      const double mx = hm * mass7(xp, p, ld);
      v = which == 0 ? ax : which == 1 ? mx : ax - sigma * mx;
    }
    y[b * nI + (size_t)(j - 1) * (n - 1) + (i - 1)] = v;
  });
}

// Per-shift sums of the per-sample differences over the points of a batch: one CTA per shift,
// fixed reduction order (deterministic).  flags receives the OR of all sample flags.
__global__ void shift_sums_kernel(const double* __restrict__ out, const int* __restrict__ stat, int npts,
                                  double* __restrict__ sums, int* __restrict__ flags, int accumulate) {
  __shared__ double red[kRedSlots];
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
  if (threadIdx.x == 0) sums[r] = accumulate ? sums[r] + o[0] : o[0];
}

// reuse scheme: gather the stored level-0 pairs (and the level below's values) of a pass's samples
__global__ void reuse_gather_kernel(int R, int npts, uint32_t k0, size_t V, const double* __restrict__ u0,
                                    const double* __restrict__ lam0, uint32_t ld0, const double* __restrict__ lamp,
                                    uint32_t ldp, double* __restrict__ upad, double* __restrict__ out,
                                    const uint32_t* dk) {
  if (dk) k0 += *dk;
  const size_t B = (size_t)R * npts, tot = B * V;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const size_t b = q / V, e = q % V;
    const size_t r = b / npts, k = k0 + b % npts;
    upad[q] = u0[(r * ld0 + k) * V + e];
    if (e == 0) {
      out[b * 4 + 0] = lam0[r * ld0 + k];
      out[b * 4 + 2] = lamp ? lamp[r * ldp + k] : 0.0;
    }
  }
}

__global__ void reuse_scatter_kernel(int R, int npts, uint32_t k0, size_t V, const double* __restrict__ upad,
                                     const double* __restrict__ out, double* __restrict__ lam, uint32_t ldl,
                                     double* __restrict__ u0, double* __restrict__ lam0, uint32_t ld0,
                                     const uint32_t* dk) {
  if (dk) k0 += *dk;
  const size_t B = (size_t)R * npts, tot = B * (u0 ? V : 1);
  const size_t per = u0 ? V : 1;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const size_t b = q / per, e = q % per;
    const size_t r = b / npts, k = k0 + b % npts;
    if (u0) u0[(r * ld0 + k) * V + e] = upad[q];
    if (e == 0) {
      lam[r * ldl + k] = out[b * 4 + 1];
      if (lam0) lam0[r * ld0 + k] = out[b * 4 + 0];
    }
  }
}

int grid_of(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

cudaError_t launch_reuse_gather(int R, int npts, uint32_t k0, size_t V, const double* d_u0, const double* d_lam0,
                                uint32_t ld0, const double* d_lamp, uint32_t ldp, double* d_upad, double* d_out,
                                cudaStream_t st, const uint32_t* d_kshift) {
  const size_t tot = (size_t)R * npts * V;
  if (tot == 0) return cudaSuccess;
  reuse_gather_kernel<<<grid_of(tot), 256, 0, st>>>(R, npts, k0, V, d_u0, d_lam0, ld0, d_lamp, ldp, d_upad, d_out,
                                                    d_kshift);
  return cudaGetLastError();
}

cudaError_t launch_reuse_scatter(int R, int npts, uint32_t k0, size_t V, const double* d_upad, const double* d_out,
                                 double* d_lam, uint32_t ldl, double* d_u0, double* d_lam0, uint32_t ld0,
                                 cudaStream_t st, const uint32_t* d_kshift) {
  const size_t tot = (size_t)R * npts * (d_u0 ? V : 1);
  if (tot == 0) return cudaSuccess;
  reuse_scatter_kernel<<<grid_of(tot), 256, 0, st>>>(R, npts, k0, V, d_upad, d_out, d_lam, ldl, d_u0, d_lam0, ld0,
                                                     d_kshift);
  return cudaGetLastError();
}

size_t sample_slab_bytes(int nf, int nc, int np, int mixed) {
  return mixed ? slab_size<float>(nf, nc, np) : slab_size<double>(nf, nc, np);
}

size_t sample_slab_bytes(int nf, int nc, int np, int mixed, int mode_f, int mode_p, int reaction) {
  return mixed ? slab_size<float>(nf, nc, np, mode_f, mode_p, reaction != 0)
               : slab_size<double>(nf, nc, np, mode_f, mode_p, reaction != 0);
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

cudaError_t raise_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;  // (device, kernel) -> limit set so far
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t set_sample_smem(int mixed, int bytes) {
  return mixed ? raise_smem_limit((const void*)sample_kernel<float>, bytes)
               : raise_smem_limit((const void*)sample_kernel<double>, bytes);
}

cudaError_t launch_apply_operator(int n, int B, const double* d_a, int which, double sigma, const double* d_x,
                                  double* d_y, double* d_scratch, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  apply_kernel<<<B, 256, 0, st>>>(n, d_a, which, sigma, d_x, d_y, d_scratch);
  return cudaGetLastError();
}

cudaError_t launch_shift_sums(const double* d_out, const int* d_stat, int R, int npts, double* d_sums, int* d_flags,
                              cudaStream_t st, int accumulate) {
  if (R == 0) return cudaSuccess;
  shift_sums_kernel<<<R, 256, 0, st>>>(d_out, d_stat, npts, d_sums, d_flags, accumulate);
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
