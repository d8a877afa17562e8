// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

namespace mq {

constexpr int kMaxMG = 13;  // multigrid levels: meshes 1/4096 .. 1/2

// Per-launch parameters of the per-sample kernel (one CTA evaluates whole samples).
struct SampleLaunch {
  int nf, nc, np;          // fine mesh 1/h_l, coarse mesh 1/H_l, previous fine mesh (0: none)
  int direct_f, direct_p;  // lambda^l (resp. lambda^{l-1}) equals the coarse eigenvalue
  int R, npts, chunk;      // shifts, points per shift in this batch, points per warm-start chain
  const double* a_f;       // [B][2 nf^2] centroid coefficients, truncation s_l
  const double* a_c;       // [B][2 nc^2] truncation S_l
  const double* a_p;       // [B][2 np^2] truncation s_{l-1}
  double* out;             // [B][4] lambda_H, lambda^l, lambda^{l-1}, difference
  int* stat;               // [B][4] coarse iterations, inner iterations (l, l-1), flags
  int* outer;              // [B][2] refinement steps (l, l-1)
  double* u_out;           // NULL or [B][(nc-1)^2] coarse eigenvectors
  char* gscratch;          // per-CTA workspace slabs when they do not fit in shared memory
  size_t slab_bytes;
  int use_smem;
  double tol_eig;
  int max_eig_it;
  double tol_lin;          // relative FP64 residual target of the shifted solve
  double tol_inner;        // relative reduction of the preconditioned residual per inner solve
  int max_inner_it;
  int max_outer;
  int nu;                  // Jacobi sweeps before and after each coarse-grid correction
  double omega;            // Jacobi damping
  int coarse_only;         // the fine solves of mode 2 run elsewhere (streaming tier)
  double* u_pad;           // NULL or [B][(nc+1)^2]: the padded coarse eigenvectors are written here
  const double* u_in;      // NULL or [B][(nc+1)^2]: coarse pairs given (no coarse eigensolve), with
                           // lambda_H in out[b][0] (the reuse scheme across levels)
  int prev_given;          // lambda^{l-1} given in out[b][2] (no previous-level solve)
  int mode_f, mode_p;      // fine / previous-fine solve: 0 in the kernel (inner precision T),
                           // 1 in the kernel with an FP64 inner solve, 2 elsewhere (streaming)
  int reaction;            // the operator has a reaction term b u (b_f, b_c, b_p hold b)
  const double* b_f;       // [B][2 nf^2] centroid values of the reaction coefficient, like a_f
  const double* b_c;
  const double* b_p;
  int qoi;                 // 0: columns 1-3 of out hold eigenvalues; 1: the functional G(u) of the
                           // eigenfunction approximations (|integral of u| / ||u||_L2)
};

// Live timing of the streaming tier's operator sweep (k_minres_q, the largest kernel of the
// streaming solves): CUDA events around each of its launches (host-driven solves only) and a
// device counter of the algorithmic bytes the launches moved (per active sample and interior node:
// the operator's weights and vector plus the pending MINRES update).
struct KernelProbe {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;  // reused pool
  size_t used = 0;
  double ms = 0.0;
  uint64_t launches = 0;
  unsigned long long* d_bytes = nullptr;  // device counter
  cudaError_t next(std::pair<cudaEvent_t, cudaEvent_t>** out);
  cudaError_t collect();  // after the stream has been synchronised
};

// Batched streaming fine solve (mq_stream.cu): B samples on mesh 1/n, coarse pairs from mesh 1/nc.
struct StreamSolve {
  int n, nc, B;
  const double* a;         // [B][2 n^2] centroid coefficients
  const double* uH;        // [B][(nc+1)^2] padded coarse eigenvectors
  const double* lamH;      // coarse eigenvalue of sample b at lamH[b * lam_stride]
  int lam_stride;
  double* lam_out;         // two-grid eigenvalue of sample b at lam_out[b * lam_out_stride]
  int lam_out_stride;
  int* iters_out;
  int iters_stride;
  int* outer_out;
  int outer_stride;
  int* flags;              // OR-ed with kFlag* bits
  int flags_stride;
  double tol_lin, tol_inner;
  int max_inner, max_outer;
  double omega;
  int nu;                  // Jacobi sweeps before and after each coarse-grid correction (1 or 2)
  KernelProbe* probe;      // NULL, or the live timing of the operator sweep
  int qoi;                 // 1: lam_out receives G(u^h) = |integral of w| / ||w||_L2 instead of the
                           // Rayleigh quotient
  const double* b;         // NULL, or [B][2 n^2] reaction coefficients: the operator is A + B (FP32 path,
                           // V(1,1) smoothing only; cudaErrorNotSupported otherwise)
};
// Graph mode of the streaming solve: the refinement and MINRES loops become conditional WHILE nodes
// of the CUDA graph being captured on the solve's stream (no host reads); their bodies are
// captured on two further streams; two device ints count the loop iterations.
struct StreamGraph {
  cudaStream_t body[2];
  int* counters;
};
size_t stream_arena_bytes(int n, int B, int mixed, int reaction = 0);
cudaError_t stream_solve(const StreamSolve& s, int mixed, void* arena, cudaStream_t st,
                         const StreamGraph* sg = nullptr);
// kernels the streaming tier has launched from the calling thread (monotone counter)
uint64_t stream_launches();
cudaError_t launch_finalize(int B, double* d_out, int has_prev, cudaStream_t st);

// Tensor-core (tcgen05) coefficient GEMM with exact BF16 slices (mq_tc.cu); slices are [7][rows pad][K pad]
size_t tc_slices_bytes(int rows, int k);
int tc_pad_rows(int rows);
int tc_pad_k(int k);
// slices of 2^pexp psi (|2^pexp psi| <= 1 required)
cudaError_t launch_psi_slices(const double* d_psi, int s_rows, int nT, void* d_out, cudaStream_t st, int pexp = 0);
cudaError_t launch_y_slices(const double* d_Y, int B, int ldy, int k, int kpad, void* d_out, cudaStream_t st);
// pexp: the scale exponent the psi slices were built with
cudaError_t launch_coef_tc(const void* d_yslices, int B, int kpad, const void* d_pslices, int nT, int kpad_psi,
                           double a0, double* d_a, int* d_err, cudaStream_t st, const double* d_base = nullptr,
                           int pexp = 0);

// Separable coefficient evaluation for the workload family (mq_tc.cu): the terms grouped by k1
// (device arrays: tlist[k1start[k1] .. k1start[k1+1]) the terms t of wave number k1 in increasing
// t; tk2[t] = k2_t; cj[t] = c_t), and per mesh the tables of both triangle planes (sx: BF16 slices
// of sin(pi k1 x_i), [n][k1pad]; syt: sin(pi k2 y_j), [k2max + 1][n]).
struct SepTerms {
  const int* k1start;
  const int* tlist;
  const int* tk2;
  const double* cj;
};
struct SepTables {
  const void* sx[2];
  const double* syt[2];
  int k1pad;
};
size_t sep_tables_bytes(int n, int k1pad, int k2max);
// builds the tables of mesh n in d_tables (sep_tables_bytes); d_work: n k1pad doubles of scratch
cudaError_t launch_sep_tables(int n, int k1max, int k1pad, int k2max, double* d_work, void* d_tables, SepTables* t,
                              cudaStream_t st);
// a[b][t] for B rows of Y with the first K terms: k1pad >= the padded largest k1 of those terms,
// ey the exponent with |2^ey T| <= 1/2 for every stage-1 value T; d_tslices: sep_scratch_bytes(B,
// n, K, k1pad) bytes of scratch (the stage-1 slices, then the products Y c)
size_t sep_scratch_bytes(int B, int n, int K, int k1pad);
cudaError_t launch_coef_sep(const double* d_Y, int ldy, int B, int K, int k1pad, const SepTerms& terms,
                            const SepTables& tab, int n, double a0, int ey, void* d_tslices, double* d_a, int* d_err,
                            cudaStream_t st);

// Sample flags (stat[b][3])
enum : int {
  kFlagEigNoConv = 1,
  kFlagLinNoConv = 2,
  kFlagBadCoef = 4,
  kFlagBreakdown = 8,
};

size_t sample_slab_bytes(int nf, int nc, int np, int mixed);
size_t sample_slab_bytes(int nf, int nc, int np, int mixed, int mode_f, int mode_p, int reaction = 0);
cudaError_t launch_sample(const SampleLaunch& p, int mixed, int blocks, int threads, size_t smem,
                          cudaStream_t st);
int sample_occupancy(int mixed, int threads, size_t smem);
int sample_static_smem(int mixed);
cudaError_t set_sample_smem(int mixed, int bytes);
// Raises a kernel's dynamic shared memory limit to at least `bytes` on the current device and
// never lowers it, so launches from concurrent host threads (levels evaluated at the same time)
// cannot undo one another's setting between the call and the launch.
cudaError_t raise_smem_limit(const void* func, int bytes);

// FP64 FMA throughput of the device (TFLOP/s) from a kernel of independent FMA chains
cudaError_t measure_fp64_peak(int device, double* tflops, double* ms);

// Coefficient building blocks (mq_coef.cu)
// mbits > 0: embedded rule in radical-inverse order with N = 2^mbits (point k uses index rev(k))
cudaError_t launch_lattice_points(const uint32_t* d_z, uint32_t N, const double* d_delta, int R, int s,
                                  uint32_t k0, int npts, int mbits, double* d_Y, cudaStream_t st,
                                  const uint32_t* d_kshift = nullptr);
// d_region: NULL (every term on all of D), or per term 1 (only on the islands D_f of the second test
// problem of Sec. 5) or 2 (only off them)
cudaError_t launch_psi_table(int n, int s, const int* d_k1, const int* d_k2, const double* d_cj,
                             double* d_psi, cudaStream_t st, const int* d_region = nullptr);
// base[t] = v_in on the triangles whose centroid lies in D_f, v_out elsewhere
cudaError_t launch_island_field(int n, double v_in, double v_out, double* d_base, cudaStream_t st);
// a[b][t] = a0 + sum_j Y[b][j] Psi[j][t], or base[t] + sum_j ... when d_base is not NULL
cudaError_t launch_coef_gemm_f64(const double* d_Y, int ldy, int B, int s, const double* d_psi, int nT,
                                 double a0, double* d_a, cudaStream_t st, const double* d_base = nullptr);
cudaError_t launch_apply_operator(int n, int B, const double* d_a, int which, double sigma,
                                  const double* d_x, double* d_y, double* d_scratch, cudaStream_t st);
// reuse scheme store: u0 [R][N0][V] padded level-0 eigenvectors, lam [R][N_l] per level.
// Gather for the samples b = r * npts + i of a pass (point k = k0 + i): u_pad[b] = u0[r][k],
// out[b][0] = lam0[r][k], out[b][2] = lamp[r][k] (lamp may be NULL).
cudaError_t launch_reuse_gather(int R, int npts, uint32_t k0, size_t V, const double* d_u0, const double* d_lam0,
                                uint32_t ld0, const double* d_lamp, uint32_t ldp, double* d_upad, double* d_out,
                                cudaStream_t st, const uint32_t* d_kshift = nullptr);
// Scatter after a pass: lam[r][k] = out[b][1]; with d_u0, also u0[r][k] = u_pad[b] and
// lam0[r][k] = out[b][0].
cudaError_t launch_reuse_scatter(int R, int npts, uint32_t k0, size_t V, const double* d_upad, const double* d_out,
                                 double* d_lam, uint32_t ldl, double* d_u0, double* d_lam0, uint32_t ld0,
                                 cudaStream_t st, const uint32_t* d_kshift = nullptr);
// (d_kshift: NULL, or a device offset added to k0 -- a captured graph replayed on another range)
// per-shift sums of the level differences of a pass (accumulate: added to d_sums instead of
// overwriting it); d_flags receives the OR of the sample flags
cudaError_t launch_shift_sums(const double* d_out, const int* d_stat, int R, int npts, double* d_sums,
                              int* d_flags, cudaStream_t st, int accumulate = 0);

}  // namespace mq
