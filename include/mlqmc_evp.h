/*
 * mlqmc_evp.h -- C ABI of the GB300 (sm_103a) two-grid MLQMC eigenvalue library.
 *
 * Problem (Sec. 1, eq. evp; Sec. 2, eq. coeff): the smallest eigenvalue lambda(y) of
 *     -div(a(x, y) grad u) = lambda u  on D = (0,1)^2,  u = 0 on the boundary,
 *     a(x, y) = a0 + sum_{j=1}^{s} y_j psi_j(x),  y_j in [-1/2, 1/2),
 * discretised by P1 finite elements on the uniform triangulation of D into n x n squares, each
 * split by its south-west to north-east diagonal (Sec. 2.3), with a evaluated at triangle
 * centroids and the exact consistent mass matrix.
 *
 * The second test problem of Sec. 5 adds a reaction term: -div(a grad u) + b u = lambda u with
 * b(x, y) = b0 + sum_j y_j b_j(x) (mq_set_islands).  Instead of the eigenvalue the quantity of
 * interest can be the linear functional G(u) = integral of u over D of the L2-normalised
 * eigenfunction with positive integral (mq_set_qoi; Sec. 1 and Sec. 4.3: the same estimator).
 *
 * The library evaluates, for a batch of randomly shifted rank-1 lattice points (Sec. 2.5,
 * eq. rqmc, eq. t_kl), the two-grid-truncation eigenvalue approximations of Algorithm 1 and the
 * level differences lambda^l - lambda^{l-1} of Algorithm 2, and forms the shift-averaged MLQMC
 * estimate with its sample-variance standard error (eq. tg-mlqmc, eq. sample_var, eq. ml-var).
 *
 * Conventions
 *   - Every call returns an mq_status; no call aborts the process.  On failure the message of
 *     mq_last_error() says why (valid until the next call on the same context).
 *   - Host arrays passed in are owned by the caller and copied before the call returns.
 *   - The library owns every device buffer it allocates; pointers named d_* are device
 *     pointers owned by the caller, which must stay valid until the call returns (calls that
 *     take them synchronise the context stream before returning).
 *   - Node vectors over a mesh 1/n hold the (n-1)^2 interior nodes row by row:
 *     index (j-1)(n-1) + (i-1) for the node (i/n, j/n), 1 <= i, j <= n-1.
 *   - Per-triangle arrays over a mesh 1/n hold 2 n^2 values: the lower triangle
 *     {(i,j),(i+1,j),(i+1,j+1)} of cell (i,j) at j*n + i and the upper triangle
 *     {(i,j),(i+1,j+1),(i,j+1)} at n*n + j*n + i.
 */
#ifndef MLQMC_EVP_H
#define MLQMC_EVP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mq_ctx mq_ctx;

typedef enum {
  MQ_OK = 0,
  MQ_EINVAL = 1,   /* bad argument: size, range, null pointer, a <= 0 at a centroid */
  MQ_ENOMEM = 2,   /* host or device allocation failed */
  MQ_ECUDA = 3,    /* a CUDA call failed; the message names it */
  MQ_ENOCONV = 4,  /* at least one sample hit an iteration cap; results are still written */
  MQ_ETIMEOUT = 5, /* a bounded device wait ran out (the tensor-core coefficient kernel's waits on
                      its matrix-multiply barriers); the outputs of that call are not valid */
  MQ_ESTATE = 6    /* call out of order (e.g. evaluate before levels, lattice or shifts are set) */
} mq_status;

/* Quantity of interest of the level samples (mq_set_qoi). */
typedef enum {
  MQ_QOI_EIGENVALUE = 0, /* the smallest eigenvalue (default) */
  MQ_QOI_FUNCTIONAL = 1  /* G(u) = |integral of u over D| / ||u||_L2 of the eigenfunction approximation */
} mq_qoi;

typedef enum {
  MQ_PREC_FP64 = 0,  /* every step in FP64 */
  MQ_PREC_MIXED = 1  /* FP32 multigrid-preconditioned MINRES inside FP64 iterative refinement;
                        coefficients, residuals, Rayleigh quotients, coarse eigenpairs in FP64 */
} mq_precision;

/* One MLQMC level (Algorithm 2).  n_fine = 1/h_l and n_coarse = 1/H_l are powers of two with
 * 2 <= n_coarse <= n_fine <= 4096; 1 <= S <= s.  n_coarse == n_fine with S == s makes the level a
 * direct eigensolve (lambda^l = lambda_{h_l, s_l}).  N lattice points (k = 0..N-1), R shifts. */
typedef struct {
  int32_t n_fine, n_coarse;
  int32_t s, S;
  uint32_t N;
  int32_t R;
} mq_level;

/* Per-call statistics (mq_get_stats). */
typedef struct {
  uint64_t samples;          /* samples evaluated by the last evaluation call */
  uint64_t noconv;           /* samples with an iteration cap hit */
  double coarse_iters_mean;  /* coarse eigensolver (LOBPCG) iterations per sample */
  int32_t coarse_iters_max;
  double fine_iters_mean;    /* inner MINRES iterations per fine solve */
  int32_t fine_iters_max;
  double outer_iters_mean;   /* FP64 refinement steps per fine solve */
  int32_t outer_iters_max;
  double kernel_ms;          /* device time of the last evaluation (CUDA events) */
  double coef_ms;            /* of which: coefficient evaluation */
  double sample_ms;          /* of which: per-sample eigen/solve kernel */
  int32_t blocks, threads;   /* launch shape of the per-sample kernel */
  int32_t smem_bytes;        /* dynamic shared memory per block (0 = workspace in global memory) */
  int64_t workspace_bytes;   /* per-block workspace */
} mq_stats;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to launch on, or
 * NULL for a stream the context creates and owns. */
mq_status mq_create(mq_ctx** out, int device, void* cuda_stream);
mq_status mq_destroy(mq_ctx* ctx);

/* Coefficient a(x, y) = a0 + sum_{j<=s} y_j psi_j(x) (Sec. 2, eq. coeff; truncated as in
 * eq. coeff_s), psi_j(x) = j^-decay sin(pi k1_j x1) sin(pi k2_j x2).  family 0: (k1, k2) the
 * j-th pair with k1, k2 >= 1 ordered by k1^2 + k2^2, ties by smaller k1; family 1: (j, j+1), the
 * first test problem of Sec. 5 (decay p~ = 4/3, 2 or 3 there; a0 = pi / sqrt(2) keeps a > 0 for
 * p~ = 4/3).  family 2: the second test problem of Sec. 5 with all four decays equal to `decay`
 * (see mq_set_islands; a0 is then unused but must still be positive).  Other families give
 * MQ_EINVAL.  s_max bounds the truncation of every level.  a0 > 0.  Requires a >= a_min > 0 at all
 * centroids (checked per evaluation: a sample with a non-positive value is flagged and the call
 * returns MQ_EINVAL, its outputs written). */
mq_status mq_set_coefficient(mq_ctx* ctx, double a0, int32_t s_max, int32_t family, double decay);

/* The second test problem of Sec. 5 (coefficient family 2): four islands
 *     D_f = [1/8,3/8]^2 u [5/8,7/8]^2 u [1/8,3/8]x[5/8,7/8] u [5/8,7/8]x[1/8,3/8],
 * the operator -div(a grad u) + b u with
 *     a = a_0 + sum_j y_j a_j,  a_0 = 0.01 on D_f, 0.011 off D_f,
 *     b = b_0 + sum_j y_j b_j,  b_0 = 2 on D_f, 0.3 off D_f,
 *     odd j, k = (j+1)/2:  a_j = 0.01 w_k(p_a),   b_j = 2 w_k(p_b)     on D_f, 0 off D_f,
 *     even j, k = j/2:     a_j = 0.011 w_k(p_a'), b_j = 0.3 w_k(p_b')  off D_f, 0 on D_f,
 *     w_k(q; x) = k^-q sin(8 k pi x1) sin(8 (k+1) pi x2).
 * A zeroth term is multiplied by pi / sqrt(2) on the region whose decay is below 2 (p_a for a_0 on
 * D_f, p_a' off D_f, p_b and p_b' for b_0).  A triangle belongs to D_f when its centroid does (the
 * meshes 1/8 and finer resolve the islands exactly).  The reaction enters every operator as the
 * P1 matrix B = sum_T b_T M_T (b constant per triangle, its centroid value).  Requires a > 0 and
 * b >= 0 at all centroids (checked per evaluation like a).  The fine solves of this family run in
 * the per-sample kernel: levels configured for the streaming tier give MQ_EINVAL when evaluated. */
mq_status mq_set_islands(mq_ctx* ctx, int32_t s_max, double p_a, double p_a_prime, double p_b, double p_b_prime);

/* Quantity of interest (mq_qoi).  MQ_QOI_FUNCTIONAL: the per-sample values and every estimate
 * refer to G(u) = |integral of u| / ||u||_L2 (Sec. 1: each eigenfunction approximation is
 * normalised and given the sign of the eigenfunction, whose integral is positive): G(u_H) of the
 * coarse eigenvector on direct levels, G(w) of the two-grid solution w of Algorithm 1 otherwise.
 * Per-sample records then hold (lambda_H, G^l, G^{l-1}, G^l - G^{l-1}).  Changing the quantity
 * resets the estimator sums and switches the reuse scheme off. */
mq_status mq_set_qoi(mq_ctx* ctx, int32_t qoi);

/* Levels l = 0..L (copied).  Resets the estimator sums, lattices and shifts. */
mq_status mq_set_levels(mq_ctx* ctx, int32_t L_plus_1, const mq_level* levels);

/* Generating vector z[0..s-1] of level `level` (copied), 0 < z_j < N (Sec. 2.5). */
mq_status mq_set_lattice(mq_ctx* ctx, int32_t level, const uint32_t* z, int32_t s);

/* Level `level` uses an embedded lattice rule (Sec. 2.5: one generating vector for every
 * N = 2^m, nested point sets) in radical-inverse order: point k (0 <= k < 2^m_max) is
 *     y_k = {rev(k) z / 2^m_max + Delta_r} - 1/2,  rev(k) = the m_max-bit reversal of k,
 * so the first 2^m points are exactly the 2^m-point rule and doubling the points of a level adds
 * the next 2^m.  z[0..s-1] odd and < 2^m_max (copied); the level's N must be a power of two
 * <= 2^m_max (1 <= m_max <= 31).  mq_set_lattice switches the level back to the plain order. */
mq_status mq_set_lattice_embedded(mq_ctx* ctx, int32_t level, const uint32_t* z, int32_t s, int32_t m_max);

/* Random shifts Delta[R][s_l] of level `level`, row-major, each in [0, 1) (copied). */
mq_status mq_set_shifts(mq_ctx* ctx, int32_t level, const double* delta);

/* The reuse scheme across levels (Sec. 4.3, the closing paragraphs after Algorithm 2): every level
 * uses the same shifts and the same embedded lattice (each level's z and shifts are prefixes of
 * the longest level's), level 0 is a direct eigensolve (n_coarse = n_fine, S = s) and every level
 * l >= 1 has n_coarse = n_fine of level 0 and S = s of level 0.  Point k of level l is then point
 * k of level 0 in the first s_0 components, so the coarse pair of level l at point k is the
 * level-0 eigenpair computed there, and lambda^{l-1} at point k is the value level l-1 computed:
 * levels l >= 1 skip the coarse eigensolve and the previous-level solve (Algorithm 2 steps 6-8 and
 * 12-14) and take both from a device store the library keeps per shift and point.  Consequently
 * mq_eval_level(l, k0, k1) with l >= 1 requires levels 0 and l-1 to have been evaluated at every
 * point of [k0, k1) since the scheme was switched on (MQ_ESTATE otherwise), and N_l must not
 * exceed N_{l-1}.  With shared shifts the levels are not independent: mq_estimate takes the
 * standard error from the per-shift totals sum_l Q^(r)_l (eq. sample_var applied to them)
 * instead of adding the level variances (level_var still reports eq. sample_var per level).
 * on = 1: validate, allocate the store (R N_0 ((n_0+1)^2 + 1) + R sum_l N_l doubles; kept for the next
 * mq_set_reuse(1)) and mark every point empty; on = 0: free the store.  A later mq_set_lattice* or
 * mq_set_shifts switches the scheme off (call mq_set_reuse(1) again after them); mq_set_levels
 * also frees the store.
 * mq_eval_levels_device is not available in this scheme (MQ_ESTATE). */
mq_status mq_set_reuse(mq_ctx* ctx, int32_t on);

/* Precision mode and the relative residual target ||b - (A - lambda_H M) w|| / ||b|| of the fine
 * shifted solve (tol_linear <= 0: default 1e-5 for MQ_PREC_MIXED, 1e-6 for MQ_PREC_FP64).  The
 * Rayleigh quotient lambda^h moves to first order in the solve error with a constant damped by
 * the two-grid error (about 3e-7 on meshes 1/16..1/128), so the defaults keep lambda^h within
 * ~3e-13 of the exact two-grid value.  Samples whose final residual is above max(1e-5,
 * 10 tol_linear) (or a small multiple of the FP64 rounding floor) are flagged. */
mq_status mq_set_precision(mq_ctx* ctx, mq_precision prec, double tol_linear);

/* Inner solver options (values <= 0 keep the defaults): tol_inner is the reduction of the
 * preconditioned MINRES residual per refinement step (default in MQ_PREC_MIXED 1e-4 for fine
 * meshes up to 1/128, 1e-5 beyond; tol_linear/10
 * in MQ_PREC_FP64), max_inner the MINRES iteration cap per step (500), max_outer the cap on FP64
 * refinement steps (10 mixed, 4 FP64). */
mq_status mq_set_solver_options(mq_ctx* ctx, double tol_inner, int32_t max_inner, int32_t max_outer);

/* Coarse eigensolver options (values <= 0 keep the defaults): tol_eig is the target of the
 * relative eigen-residual ||A_H x - theta M_H x|| / (theta ||M_H x||) of LOBPCG, max_eig the
 * iteration cap (200).  The Rayleigh quotient theta = lambda_H is accurate to about the square of
 * tol_eig, the eigenvector (and so G(u_H)) to about tol_eig: the relative eigenvalue error is at
 * most tol_eig^2 kappa(M) theta / (lambda_2 - theta), kappa(M) <= 4 for the P1 mass matrix.
 * Defaults: 1e-6 for level evaluations of eigenvalues with coefficient families 0 and 1
 * (lambda_H within ~3e-12 relative at worst, 5e-14 measured on the six-level workload; the
 * two-grid values depend on u_H only through one shifted inverse-iteration step and stay at FP64
 * rounding); 1e-8 for the islands family of mq_set_islands (its unresolved coarse mesh makes the
 * two-grid values ~1e4 times more sensitive to u_H) and when mq_eval_point returns the
 * eigenvector; 1e-11 for MQ_QOI_FUNCTIONAL. */
mq_status mq_set_eig_options(mq_ctx* ctx, double tol_eig, int32_t max_eig);

/* Damped Jacobi steps before and after each coarse-grid correction of the multigrid V-cycle that
 * preconditions the shifted solves and the coarse eigensolver: 1 or 2 for every solve (0: the
 * default, 2 in the per-sample kernel and 1 in the streaming tier).  The
 * V-cycle is a preconditioner only: results agree to the solver tolerances either way. */
mq_status mq_set_smoothing(mq_ctx* ctx, int32_t nu);

/* Execution tier of the fine solves: fine meshes 1/n with n >= stream_min_n run in
 * the batched streaming tier (one kernel per sweep over all samples of a pass, lockstep across
 * samples); coarser ones run inside the per-sample kernel (one CTA per sample, workspace in
 * shared memory when it fits).  Both tiers compute the same values to rounding.  Default (or
 * stream_min_n = 0): 32 in MQ_PREC_MIXED, 256 in MQ_PREC_FP64. */
mq_status mq_set_tier(mq_ctx* ctx, int32_t stream_min_n);

/* Threads per CTA of the per-sample kernel (one CTA per sample) on level `level` (0 <= level < 64):
 * 0 restores the default (64 when the largest fine mesh solved in the kernel is at most 1/16,
 * 128 for coarse eigensolves on meshes up to 1/16, else 256), otherwise a multiple of 32 in
 * [32, 512].  Fewer threads per sample let more samples share an SM; the results do not depend
 * on it beyond rounding order. */
mq_status mq_set_cta_threads(mq_ctx* ctx, int32_t level, int32_t threads);

/* Launch configuration of one level (0 <= level < 64), overriding the context-wide defaults:
 * tier -1 (fine solve tier by mesh size, mq_set_tier), 0 (fine solves inside the per-sample
 * kernel) or 1 (streaming tier); threads as in mq_set_cta_threads (0: default); nu as in
 * mq_set_smoothing for every solve of the level (0: default).  Results agree to the solver
 * tolerances whatever the configuration. */
mq_status mq_set_level_config(mq_ctx* ctx, int32_t level, int32_t tier, int32_t threads, int32_t nu);

/* Chosen configuration of a level (mq_autotune_level). */
typedef struct {
  int32_t tier, threads, nu;  /* as in mq_set_level_config */
  double ms;                  /* device time of the probe with it (or the cached time) */
  int32_t from_cache;         /* 1: read from the cache file, nothing was timed */
  int32_t tried;              /* configurations timed */
} mq_tune_choice;

/* Autotuner: times the level on its first `points` lattice points (all shifts) with every
 * candidate configuration -- the fine solve's tier when the fine mesh lies between 1/16 and 1/128,
 * the per-sample kernel's threads per CTA (64, 128, 256) and the smoothing (1 or 2 Jacobi steps per
 * side) -- each twice, keeps the fastest (CUDA events around the level's evaluation, second run)
 * and applies it with mq_set_level_config.  cache_path: NULL, or a text file of earlier choices
 * keyed by the GPU, the precision, the level's meshes, truncations, shifts and probe size: a hit
 * applies the stored choice without timing; a miss appends the new one.  The probes leave the
 * estimator sums, timers and launch count as they were. */
mq_status mq_autotune_level(mq_ctx* ctx, int32_t level, uint32_t points, const char* cache_path,
                            mq_tune_choice* choice);

/* Evaluate level `level` at lattice indices k in [k0, k1) for every shift (Algorithm 2, steps
 * 5-15): per sample the coarse eigenpair on (H_l, S_l), lambda^l by Algorithm 1 on (h_l, s_l)
 * and, for l > 0, lambda^{l-1} on (h_{l-1}, s_{l-1}) from the same coarse pair.
 *   per_sample: NULL or host [R][k1-k0][4] = (lambda_H, lambda^l, lambda^{l-1}, difference),
 *               lambda^{-1} = 0 on level 0.
 *   shift_sums: NULL or host [R]; sum over k of the differences is ADDED to each entry.
 * The context also accumulates the sums for mq_estimate.  Returns MQ_ENOCONV (results written)
 * when any sample hit an iteration cap. */
mq_status mq_eval_level(mq_ctx* ctx, int32_t level, uint32_t k0, uint32_t k1, double* per_sample,
                        double* shift_sums);

/* As mq_eval_level with device outputs: d_per_sample [R][k1-k0][4], d_shift_sums [R]
 * (overwritten, not added).  Either may be NULL.  Nothing is copied to the host except the
 * convergence flags; the context sums are still accumulated on the device. */
mq_status mq_eval_level_device(mq_ctx* ctx, int32_t level, uint32_t k0, uint32_t k1,
                               double* d_per_sample, double* d_shift_sums);

/* Evaluate several whole levels (every point k in [0, N_l) of every shift) at the same time
 * (Algorithm 2, steps 4-15 for each listed level; the levels are independent).  Each level runs on
 * its own internal context -- its own CUDA stream, buffers and host thread -- so the latency-bound
 * per-sample kernel of small meshes overlaps the bandwidth-bound streaming solves of large ones.
 *   levels[i]: distinct level indices (lattice and shifts set); d_per_sample[i] and d_shift_sums[i]
 *   as in mq_eval_level_device for levels[i] (either array of pointers, or any entry, may be NULL).
 * Returns after every level has finished; the sums, timers and launch counts of the levels are
 * added to this context (mq_estimate, mq_get_level_timing, mq_get_launch_count).  The internal
 * contexts are built on the first call (and again after any mq_set_* call), share the free device
 * memory equally, and are released by mq_destroy.  Returns the first error of a level
 * (MQ_ENOCONV only if no other error occurred; results are written in that case). */
mq_status mq_eval_levels_device(mq_ctx* ctx, int32_t nlevels, const int32_t* levels, double* const* d_per_sample,
                                double* const* d_shift_sums);

/* Graph schedule (Algorithm 2 over several levels as one CUDA graph).  mq_graph_capture records,
 * as one CUDA graph, the evaluation of the point ranges [k0s[i], k1s[i]) of levels levels[i] in
 * the order given, with the device outputs of mq_eval_level_device (d_per_sample[i],
 * d_shift_sums[i]; either array, or any entry, may be NULL; the buffers must stay valid while
 * the graph is kept).  It first runs the same evaluations once as a rehearsal (which allocates
 * every buffer and builds the tables; the estimator state is put back afterwards), then captures
 * them on the context stream: the streaming tier's refinement and MINRES loops become
 * conditional WHILE nodes whose conditions the kernels set on the device (no host reads), and the
 * per-shift sums and sample flags accumulate on the device.  mq_graph_launch replays the graph
 * with one cudaGraphLaunch, waits for it and adds its sums to the context (mq_estimate), as the
 * level-by-level calls would; the per-sample results equal theirs bit for bit.  k0s: NULL to
 * replay the captured ranges, or new start points for ranges of the captured lengths (the offset
 * reaches the kernels through device memory).  The per-level timers are not updated by the graph.
 * Any setter, and any call that has to enlarge a buffer the graph uses, drops the graph
 * (mq_graph_launch then returns MQ_ESTATE).  The context stream must not be the legacy default
 * stream. */
mq_status mq_graph_capture(mq_ctx* ctx, int32_t nranges, const int32_t* levels, const uint32_t* k0s,
                           const uint32_t* k1s, double* const* d_per_sample, double* const* d_shift_sums);
mq_status mq_graph_launch(mq_ctx* ctx, const uint32_t* k0s);
/* Live timing of the streaming tier's operator sweep (its largest kernel: the MINRES operator
 * application with the pending update, once per inner iteration): with on = 1, every later
 * host-driven streaming solve records CUDA events on the context stream around each launch of
 * that kernel and counts on the device the algorithmic bytes the launches move (per active sample
 * and interior node: weights and operand 4 arrays, plus 6 for the pending MINRES update).  Turning
 * it on (or off) clears the totals.  mq_get_kernel_probe returns the summed launch time (ms), the
 * launches and the algorithmic bytes since then (any output may be NULL).  Graph launches are not
 * timed. */
mq_status mq_set_kernel_probe(mq_ctx* ctx, int32_t on);

/* Measured FP64 throughput of device `device`: a kernel of independent fused multiply-add chains
 * (8 per thread, 8 CTAs of 256 threads per SM), best of three timed launches after a warm-up;
 * tflops counts an FMA as two operations, ms is that launch's time.  The denominator of the FP64
 * roofline of the per-sample kernel. */
mq_status mq_measure_fp64_peak(int device, double* tflops, double* ms);
mq_status mq_get_kernel_probe(mq_ctx* ctx, double* ms, uint64_t* launches, uint64_t* bytes);

/* captured: 1 while a graph is held; kernel_nodes: the kernels captured into it (the loop bodies
 * counted once).  Either output may be NULL. */
mq_status mq_get_graph_info(mq_ctx* ctx, int32_t* captured, uint64_t* kernel_nodes);

/* Estimate from the sums accumulated so far (eq. tg-mlqmc): Q^(r)_l = sum_k diff / n_l where
 * n_l is the number of points evaluated on level l, Qhat_l = mean_r Q^(r)_l, mean = sum_l Qhat_l,
 * level_var[l] = sum_r (Qhat_l - Q^(r)_l)^2 / (R (R - 1)) (eq. sample_var), std_err =
 * sqrt(sum_l level_var[l]) (eq. ml-var).  level_mean / level_var: NULL or host [L+1].
 * MQ_ESTATE if a level has no points yet; MQ_EINVAL if R < 2 on any level. */
mq_status mq_estimate(mq_ctx* ctx, double* mean, double* std_err, double* level_mean,
                      double* level_var);

/* The estimator state of level `level`: sums[r] = sum over the evaluated points of the level
 * differences of shift r (host [R], copied out) and the number of points evaluated.  Several
 * processes that evaluate disjoint sets of shifts of one workload (one per GPU) exchange these and
 * combine them with mq_estimate_sums.  Either output may be NULL. */
mq_status mq_get_sums(mq_ctx* ctx, int32_t level, double* sums, uint64_t* npoints);

/* The estimate of eq. tg-mlqmc from per-level, per-shift sums (no context, no GPU): level l has
 * R[l] >= 2 shifts whose sums are sums[off_l .. off_l + R[l]) with off_l = R[0] + .. + R[l-1], and
 * npoints[l] > 0 points per shift.  Q^(r)_l = sums / npoints, Qhat_l their mean, level_var[l] =
 * eq. sample_var; std_err = sqrt(sum_l level_var[l]) for independent levels (shared = 0), or the
 * standard error of the per-shift totals sum_l Q^(r)_l when every level uses the same shifts
 * (shared = 1, all R[l] equal; as mq_estimate in the reuse scheme).  level_mean / level_var:
 * NULL or host [nlevels]. */
mq_status mq_estimate_sums(int32_t nlevels, const int32_t* R, const double* sums, const uint64_t* npoints,
                           int32_t shared, double* mean, double* std_err, double* level_mean, double* level_var);

/* Result of mq_run_adaptive. */
typedef struct {
  int32_t L;               /* finest level used */
  int32_t converged;       /* 1: variance and bias tests passed; 0: stopped at the last level or at
                              the point capacity of the levels */
  int32_t doublings;       /* point doublings performed */
  int32_t levels_added;    /* levels started (three initial ones included) */
  uint32_t N[32];          /* points per shift on levels 0..L (0 beyond) */
  double mean, std_err;    /* estimate over levels 0..L, std_err = sqrt(sum_l level_var[l]) */
  double level_mean[32], level_var[32];  /* Qhat_l and eq. sample_var per level */
} mq_adaptive_result;

/* The adaptive choice of the point counts N_l and of the number of levels (Sec. 4.2: the paper
 * chooses them with the Giles-Waterhouse algorithm for multilevel QMC).  Reading implemented:
 *   1. levels 0..2 start with n_init points each (every level needs an embedded lattice,
 *      mq_set_lattice_embedded, so its points can be doubled; its N is the largest count allowed);
 *   2. while sum_l level_var > eps^2 / 2 (eq. sample_var): double the points of the level with the
 *      largest level_var / (C_l N_l) among those that can still double (ties: the lower level),
 *      C_l = the fine unknowns solved per sample ((n_l - 1)^2, plus (n_{l-1} - 1)^2 on a two-grid
 *      level l > 0); stop (converged = 0) when no level can double;
 *   3. bias test with weak order alpha (level differences shrink like 2^(-alpha l); 2 for the
 *      O(h^2) eigenvalue error): max(|Qhat_L|, |Qhat_{L-1}| / 2^alpha) <= (2^alpha - 1) eps / sqrt(2)
 *      ends the run (converged = 1); otherwise level L + 1 starts with n_init points and step 2
 *      repeats (converged = 0 when no level is left).
 * Independent shifts per level (MQ_ESTATE in the reuse scheme).  The context's estimator sums are
 * reset first and hold the run's sums afterwards.  Returns MQ_ENOCONV (result written) when any
 * sample hit an iteration cap. */
mq_status mq_run_adaptive(mq_ctx* ctx, double eps, double alpha, uint32_t n_init, mq_adaptive_result* result);

/* Clear the estimator sums and the per-level timers (keeps levels, lattices and shifts). */
mq_status mq_reset_sums(mq_ctx* ctx);

/* Device time accumulated on level `level` since mq_set_levels or mq_reset_sums, measured with
 * CUDA events on the context stream: coefficient evaluation (coef_ms), the per-sample kernel
 * (sample_ms) and the number of per-sample kernel launches.  Any output may be NULL. */
mq_status mq_get_level_timing(mq_ctx* ctx, int32_t level, double* coef_ms, double* sample_ms,
                              uint64_t* launches);

/* The sample_ms of mq_get_level_timing split at the end of the per-sample kernel: percta_ms is the
 * per-sample kernel launch alone (events on either side of it), stream_ms the batched streaming
 * fine solves that follow it (zero when the level runs entirely in the per-sample kernel).  Any
 * output may be NULL. */
mq_status mq_get_kernel_timing(mq_ctx* ctx, int32_t level, double* percta_ms, double* stream_ms);

/* Number of CUDA kernels this context has launched since mq_set_levels or mq_reset_sums (every
 * call that evaluates samples, coefficients, lattice points or operators counts its launches). */
mq_status mq_get_launch_count(mq_ctx* ctx, uint64_t* launches);

/* Single explicit parameter vector y[0..s_l-1] on level `level`: the coarse eigenvalue
 * lambda_{H_l,S_l}(y), lambda^l(y) and (l > 0) lambda^{l-1}(y) (Algorithm 1).  Any output may
 * be NULL.  u_H: NULL or host [(n_coarse-1)^2], the coarse eigenvector, ||u_H||_M = 1, sum > 0. */
mq_status mq_eval_point(mq_ctx* ctx, int32_t level, const double* y, double* lam_H,
                        double* lam_h_twogrid, double* lam_hm1_twogrid, double* u_H);

mq_status mq_get_stats(mq_ctx* ctx, void* stats, size_t bytes);
const char* mq_last_error(const mq_ctx* ctx);

/* ---- building blocks, exposed for step-by-step parity checks ---------------------------- */

/* CBC generating vector (host; Sec. 2.5): product weights gamma_j = j^-decay, squared
 * shift-averaged worst-case error e^2(z) = -1 + (1/N) sum_k prod_j (1 + gamma_j B2({k z_j/N})),
 * B2(x) = x^2 - x + 1/6; component j takes the smallest candidate z in [1, N/2] coprime to N
 * whose error is within an absolute 1e-12 of the minimum.  z_out: host [s].  N >= 2. */
mq_status mq_cbc_lattice(uint32_t N, int32_t s, double decay, uint32_t* z_out);

/* Generating vector of an embedded lattice rule for N = 2^m, m_min <= m <= m_max (host; Sec. 2.5).
 * The paper uses embedded rules without stating their construction criterion; here component j
 * takes the odd candidate c < 2^(m_max-1) minimising max over m of e^2_{2^m}(z_1..z_{j-1}, c) /
 * min_c' e^2_{2^m}(z_1..z_{j-1}, c'), with e^2 the shift-averaged worst-case error of
 * mq_cbc_lattice (product weights gamma_j = j^-decay), formed as the mean of the excess of the
 * running products over one; ratios within a relative 1e-6 of the minimum tie and the smallest
 * candidate wins.
 * 0 <= m_min <= m_max <= 24; z_out: host [s]. */
mq_status mq_cbc_embedded_lattice(int32_t m_min, int32_t m_max, int32_t s, double decay, uint32_t* z_out);

/* Lattice points of level `level` for k in [k0, k1) (eq. t_kl, eq. rqmc; radical-inverse order on
 * a level with an embedded lattice):
 * d_Y [R][k1-k0][s_l], y = {k z / N + Delta_r} - 1/2. */
mq_status mq_lattice_points_device(mq_ctx* ctx, int32_t level, uint32_t k0, uint32_t k1,
                                   double* d_Y);

/* Coefficients at the centroids of mesh 1/n (eq. coeff_s): d_a[b][2n^2] = a0 + sum_{j<s}
 * d_Y[b*ldy + j] psi_{j+1}(c_t), for b < B, with the context's precision mode
 * (FP64: FP64 GEMM; MIXED: tensor-core split GEMM accurate to FP64 rounding of the terms).
 * Family 2: the piecewise a_0 in place of a0. */
mq_status mq_coefficients_device(mq_ctx* ctx, int32_t n, int32_t s, const double* d_Y,
                                 int32_t B, int32_t ldy, double* d_a);

/* The reaction coefficient of family 2 at the centroids of mesh 1/n, as mq_coefficients_device:
 * d_b[b][2n^2] = b_0(c_t) + sum_{j<s} d_Y[b*ldy + j] b_{j+1}(c_t).  MQ_ESTATE for other families. */
mq_status mq_reaction_coefficients_device(mq_ctx* ctx, int32_t n, int32_t s, const double* d_Y,
                                          int32_t B, int32_t ldy, double* d_b);

/* Operator apply on mesh 1/n for B coefficient fields d_a[b][2n^2] (FP64):
 * which = 0: y = A x, 1: y = M x, 2: y = (A - sigma M) x; with d_a holding reaction coefficients b,
 * which = 3: y = B x, the reaction matrix in the edge-weight form the inner solves use, and 4: the
 * same from the centroid values (the form of the FP64 residual).  d_x, d_y: [B][(n-1)^2]. */
mq_status mq_apply_operator_device(mq_ctx* ctx, int32_t n, int32_t B, const double* d_a,
                                   int32_t which, double sigma, const double* d_x, double* d_y);


/* ---- allocation-free entry point ------------------------------------------------------------
 * No counterpart in the paper: an extra way to call the per-sample two-grid kernel for callers
 * that cannot allocate device memory -- code running while someone else captures a CUDA graph,
 * plugins inside a host application with its own fixed memory pool, real-time services that
 * forbid allocation after start-up.  It calls no cudaMalloc, cudaFree or other allocating
 * routine and needs no context: the per-block workspace lives in one fixed 32 MiB device array
 * inside the library, which every GPU that loads the library holds until the process exits.
 *
 * For B samples it computes the coarse eigenpair on mesh 1/n_coarse, the two-grid eigenvalue
 * on mesh 1/n_fine and (n_prev > 0) on mesh 1/n_prev from the same coarse pair (Algorithm 1
 * steps as in mq_eval_level), from caller-evaluated centroid coefficients:
 *   d_a_coarse [B][2 n_coarse^2] (truncation S), d_a_fine [B][2 n_fine^2] (truncation s) or NULL
 *   for a direct level (the fine value is then the coarse eigenvalue), d_a_prev [B][2 n_prev^2]
 *   or NULL (with n_prev > 0: the previous-level value is the coarse eigenvalue).
 * Outputs (device, caller-owned): d_out [B][4] = (lambda_H, lambda^l, lambda^{l-1}, difference);
 * d_stat [B][4] = (coarse iterations, inner iterations on n_fine, on n_prev, flags: 1 eigensolver
 * cap, 2 linear-solver cap, 4 coefficient <= 0, 8 breakdown); d_outer [B][2] refinement steps.
 * Samples are split into chains of consecutive indices; within a chain each coarse eigensolve
 * starts from the previous sample's eigenvector.  precision: MQ_PREC_FP64 or MQ_PREC_MIXED;
 * tol_linear <= 0 selects 1e-10.  The launch is asynchronous on cuda_stream (NULL: the default
 * stream); check d_stat after synchronising.
 *
 * Solver settings are fixed here (they do not follow the mq_set_* options of any context):
 * coarse eigen-residual target 1e-12 with at most 200 LOBPCG iterations, shifted-solve residual
 * target tol_linear (1e-10 by default), inner reduction per refinement step 1e-5 (mixed) or
 * tol_linear / 10 (FP64), at most 500 inner iterations and 10 (mixed) or 4 (FP64) refinement
 * steps, V(2,2) damped Jacobi (omega 0.8).  A solve on the coarse mesh itself (n_fine or n_prev
 * equal to n_coarse) is nearly singular and uses an FP64 inner solve in either precision.  These
 * targets are tighter than mq_eval_level's defaults, so on larger coarse meshes a sample can hit
 * the eigensolver cap (flag 1) where mq_eval_level converges.
 *
 * The first call on each device looks up the device address of the array (with that device
 * current) and caches it; make that first call before any stream capture begins.  The address
 * belongs to the device's context: after cudaDeviceReset the next call looks it up again (that
 * call, too, must come before any capture).  The array
 * keeps the contents of the last call; the kernel clears everything it reads before use.  All
 * calls share the one array, so calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race and corrupt each other's results: serialise them.
 * Returns MQ_EINVAL for bad sizes or null pointers, and when one block's workspace for these
 * meshes exceeds the 32 MiB array (e.g. n_fine = 4096); MQ_ECUDA when the launch fails. */
mq_status mq_twogrid_samples_noalloc(int32_t n_fine, int32_t n_coarse, int32_t n_prev, int32_t precision,
                                     int32_t B, const double* d_a_fine, const double* d_a_coarse,
                                     const double* d_a_prev, double tol_linear, double* d_out,
                                     int32_t* d_stat, int32_t* d_outer, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MLQMC_EVP_H */
