// Host side of the C ABI declared in include/mlqmc_evp.h: context, argument validation, device
// buffers, the coefficient tables, the level evaluation driver and the estimator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/mlqmc_evp.h"
#include "mq_internal.h"

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct mq_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  int smem_optin = 0;
  uint64_t n_launches = 0;  // kernels launched since mq_set_levels / mq_reset_sums
  std::vector<mq_ctx*> lanes;  // per level: child context of mq_eval_levels_device (built lazily)
  bool lanes_stale = true;     // a setter ran since the lanes were built
  int mem_share = 1;           // contexts sharing the free device memory with this one
  std::vector<int> cta_threads;  // per level: threads per CTA of the per-sample kernel (0: default)
  std::vector<int> lvl_tier;     // per level: -1 tier by mesh size, 0 per-sample kernel, 1 streaming tier
  std::vector<int> lvl_nu;       // per level: Jacobi sweeps per side of the V-cycle (0: default)
  std::string err;

  bool coef_set = false;
  double a0 = 1.0, decay = 2.0;
  double decays[4] = {2.0, 2.0, 2.0, 2.0};  // family 2: p_a, p_a', p_b, p_b'
  int s_max = 0, family = 0;
  int* d_k1 = nullptr;
  int* d_k2 = nullptr;
  double* d_cj[2] = {nullptr, nullptr};  // term factors of a (and, family 2, of b)
  int* d_region = nullptr;               // family 2: per term 1 (on D_f) or 2 (off D_f)
  int psi_exp[2] = {0, 0};               // tensor-core slices of a table hold 2^psi_exp psi
  // separable evaluation (family 0): terms grouped by k1, and per truncation K the largest k1 and
  // the sum of |c_t| of the first K terms
  bool sep_ok = false;
  int* d_k1start = nullptr;
  int* d_tlist = nullptr;
  int k1max = 0, k2max = 0;
  std::vector<int> k1prefix;
  std::vector<double> csum;
  std::map<int, std::pair<void*, mq::SepTables>> sep_tab;  // mesh n -> tables
  int qoi = MQ_QOI_EIGENVALUE;

  std::vector<mq_level> levels;
  std::vector<std::vector<uint32_t>> z;
  std::vector<int> mbits;  // per level: 0 = plain lattice order, else the embedded rule of 2^mbits points
  std::vector<uint32_t*> d_z;
  std::vector<std::vector<double>> delta;
  std::vector<double*> d_delta;
  std::vector<std::vector<double>> sums;  // per level, per shift
  std::vector<uint64_t> npoints;          // per level: points evaluated
  std::vector<double> lvl_coef_ms, lvl_sample_ms;  // per level: accumulated device time
  std::vector<uint64_t> lvl_launches;              // per level: per-sample kernel launches
  std::vector<double> lvl_percta_ms, lvl_stream_ms;  // per level: the per-sample kernel alone, the streaming tier

  // reuse scheme across levels (shared shifts, nested points): the level-0 eigenpairs and every
  // level's two-grid values, per shift and point, and which points hold values
  bool reuse = false;
  DevBuf ru0;                            // [R][N_0][(n_0+1)^2] padded level-0 eigenvectors
  DevBuf rlamH;                          // [R][N_0] their eigenvalues (the coarse shifts of levels >= 1)
  std::vector<DevBuf> rlam;              // per level: [R][N_l] the quantity of interest Q^l (lambda^l or G)
  std::vector<std::vector<uint8_t>> rfilled;  // per level: point k has values

  // graph schedule (mq_graph_capture / mq_graph_launch): the captured evaluation, its body-capture
  // streams, the device loop counters of the streaming tier, and the device accumulators of the
  // per-shift sums and sample flags of the captured ranges
  bool capturing = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gbody[2] = {nullptr, nullptr};
  DevBuf gcount, gsums, gflags, gk0;  // gk0: per captured range, the offset of its replayed start
  std::vector<int> g_levels;
  std::vector<uint32_t> g_k0, g_k1;      // the ranges of the last launch
  std::vector<uint32_t> g_cap_k0, g_shift;  // the captured starts; the device offsets (host copy)
  std::vector<size_t> g_off;       // offset of each captured range's sums in gsums
  std::vector<int> last_ppp;       // per level: points per pass of the last evaluation
  uint64_t graph_kernels = 0;      // kernel nodes captured (loop bodies counted once)
  bool probe_on = false;           // live timing of the streaming operator sweep
  mq::KernelProbe probe;
  DevBuf probe_bytes;

  int prec = MQ_PREC_FP64;
  double tol_lin = 0.0;  // 0: default of the precision mode
  double opt_tol_inner = 0.0;  // 0: default of the precision mode
  int opt_max_inner = 0, opt_max_outer = 0;
  double opt_tol_eig = 0.0;  // 0: default
  int opt_max_eig = 0;
  int opt_nu = 0;  // Jacobi sweeps per side of the V-cycle (0: default)

  // per coefficient (0: a, 1: the reaction b of family 2)
  std::map<int, std::pair<int, double*>> psi[2];  // mesh n -> (rows, table [rows][2n^2])
  std::map<int, std::pair<int, void*>> psi_sl[2];  // mesh n -> (K pad, BF16 slices [7][nT pad][K pad])
  std::map<int, double*> base[2];                  // family 2: mesh n -> zeroth term a_0 (b_0) per triangle

  DevBuf Y, af, ac, ap, out, stat, outer, scratch, sums_d, flags_d, uout, misc, upad, arena, ysl, tc_err;
  DevBuf bf, bc, bp;  // reaction coefficients of the fine, coarse and previous meshes (family 2)
  DevBuf tsl, sepw;   // separable evaluation: stage-1 slices, table scratch
  int stream_min = 0;  // fine meshes 1/n with n >= stream_min use the streaming tier (0: default)
  mq_stats stats{};
  size_t last_B = 0;  // samples of the last pass (their per-sample counters are still on the device)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

mq_status fail(mq_ctx* c, mq_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define MQ_CUDA(c, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(c, MQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// a launch wrapper that starts exactly one kernel; counted for mq_get_launch_count
#define MQ_LAUNCH(c, call) \
  do {                     \
    MQ_CUDA(c, call);      \
    ++(c)->n_launches;     \
  } while (0)

// Drops the captured graph (its nodes hold the addresses of the context's buffers and its
// settings): called before any buffer it may use is freed or reallocated and by every setter.
// while a graph is captured: the device offset of the range being captured (the graph can be
// replayed on ranges that start elsewhere); otherwise none
const uint32_t* kshift(const mq_ctx* c) {
  return c->capturing && !c->g_off.empty() ? (const uint32_t*)c->gk0.p + (c->g_off.size() - 1) : nullptr;
}

void graph_release(mq_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->g_levels.clear();
  c->g_k0.clear();
  c->g_k1.clear();
  c->g_off.clear();
}

mq_status grow(mq_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.bytes) return MQ_OK;
  graph_release(c);
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = std::max(bytes, (size_t)256);
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MQ_ENOMEM, "device allocation of %zu bytes failed", want);
  }
  b.bytes = want;
  return MQ_OK;
}

bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

// switches the reuse scheme off but keeps its device store for a later mq_set_reuse(1)
void invalidate_reuse(mq_ctx* c) {
  c->reuse = false;
  c->rfilled.clear();
}

void free_reuse(mq_ctx* c) {
  if (c->ru0.p) cudaFree(c->ru0.p);
  c->ru0 = DevBuf{};
  if (c->rlamH.p) cudaFree(c->rlamH.p);
  c->rlamH = DevBuf{};
  for (DevBuf& b : c->rlam)
    if (b.p) cudaFree(b.p);
  c->rlam.clear();
  c->rfilled.clear();
  c->reuse = false;
}

// frequency pairs of the synthetic family: k1, k2 >= 1 ordered by k1^2 + k2^2, then k1
// Wave numbers (k1, k2) of the first s terms psi_j ~ sin(pi k1 x1) sin(pi k2 x2) of a family:
// 0: all pairs k1, k2 >= 1 ordered by k1^2 + k2^2, ties by smaller k1 (the workload family);
// 1: (j, j+1), the first test problem of Sec. 5.
void psi_pairs(int s, int family, std::vector<int>& k1, std::vector<int>& k2) {
  if (family == 1) {
    k1.resize(s);
    k2.resize(s);
    for (int j = 0; j < s; ++j) {
      k1[j] = j + 1;
      k2[j] = j + 2;
    }
    return;
  }
  const int K = (int)std::ceil(2.0 * std::sqrt((double)std::max(s, 1))) + 2;
  std::vector<std::pair<int, int>> pr;
  for (int a = 1; a <= K; ++a)
    for (int b = 1; b <= K; ++b) pr.emplace_back(a, b);
  std::stable_sort(pr.begin(), pr.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
    const int nx = x.first * x.first + x.second * x.second, ny = y.first * y.first + y.second * y.second;
    return nx != ny ? nx < ny : x.first < y.first;
  });
  k1.resize(s);
  k2.resize(s);
  for (int j = 0; j < s; ++j) {
    k1[j] = pr[j].first;
    k2[j] = pr[j].second;
  }
}

// the second test problem of Sec. 5: four islands, two coefficients with piecewise zeroth terms
constexpr double kSigA[2] = {0.01, 0.011}, kSigB[2] = {2.0, 0.3};  // on D_f, off D_f

void release_tables(mq_ctx* c) {
  for (int w = 0; w < 2; ++w) {
    for (auto& kv : c->psi[w]) cudaFree(kv.second.second);
    c->psi[w].clear();
    for (auto& kv : c->psi_sl[w]) cudaFree(kv.second.second);
    c->psi_sl[w].clear();
    for (auto& kv : c->base[w]) cudaFree(kv.second);
    c->base[w].clear();
  }
  for (auto& kv : c->sep_tab) cudaFree(kv.second.first);
  c->sep_tab.clear();
}

mq_status ensure_psi(mq_ctx* c, int n, int rows, const double** out, int which = 0) {
  auto& tab = c->psi[which];
  auto it = tab.find(n);
  if (it != tab.end() && it->second.first >= rows) {
    *out = it->second.second;
    return MQ_OK;
  }
  if (it != tab.end()) {
    graph_release(c);
    cudaFree(it->second.second);
    tab.erase(it);
  }
  const size_t bytes = (size_t)std::max(rows, 1) * 2 * n * n * sizeof(double);
  double* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MQ_ENOMEM, "psi table for n=%d, s=%d (%zu bytes)", n, rows, bytes);
  }
  MQ_LAUNCH(c, mq::launch_psi_table(n, rows, c->d_k1, c->d_k2, c->d_cj[which], d, c->stream, c->d_region));
  tab[n] = {rows, d};
  *out = d;
  return MQ_OK;
}

// family 2: the zeroth term (a_0 for which = 0, b_0 for 1) on the triangles of mesh n, scaled by
// pi / sqrt(2) on a region whose terms decay with a power below 2
mq_status ensure_base(mq_ctx* c, int n, int which, const double** out) {
  auto it = c->base[which].find(n);
  if (it != c->base[which].end()) {
    *out = it->second;
    return MQ_OK;
  }
  double* d = nullptr;
  const size_t bytes = (size_t)2 * n * n * sizeof(double);
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MQ_ENOMEM, "zeroth-term field for n=%d (%zu bytes)", n, bytes);
  }
  const double* sig = which ? kSigB : kSigA;
  const double p_in = c->decays[2 * which], p_out = c->decays[2 * which + 1];
  const double sc = 3.14159265358979323846 / std::sqrt(2.0);
  MQ_LAUNCH(c, mq::launch_island_field(n, sig[0] * (p_in < 2.0 ? sc : 1.0), sig[1] * (p_out < 2.0 ? sc : 1.0), d,
                                       c->stream));
  c->base[which][n] = d;
  *out = d;
  return MQ_OK;
}

// BF16 slices of the Psi table of mesh n for the tensor-core path (cached per mesh)
mq_status ensure_psi_slices(mq_ctx* c, int n, const void** out, int* kpad, int which = 0) {
  auto it = c->psi_sl[which].find(n);
  const int rows = std::max(c->s_max, 1);
  if (it != c->psi_sl[which].end()) {
    *out = it->second.second;
    *kpad = it->second.first;
    return MQ_OK;
  }
  const double* psi = nullptr;
  mq_status st = ensure_psi(c, n, rows, &psi, which);
  if (st != MQ_OK) return st;
  const int nT = 2 * n * n;
  void* d = nullptr;
  const size_t bytes = mq::tc_slices_bytes(nT, rows);
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MQ_ENOMEM, "psi slices for n=%d (%zu bytes)", n, bytes);
  }
  MQ_LAUNCH(c, mq::launch_psi_slices(psi, rows, nT, d, c->stream, c->psi_exp[which]));
  c->psi_sl[which][n] = {mq::tc_pad_k(rows), d};
  *out = d;
  *kpad = mq::tc_pad_k(rows);
  return MQ_OK;
}

// a[b][t] = a0 + sum_{j<K} Y[b][j] psi_j(c_t) for B rows of Y (stride ldy) on mesh n: FP64 GEMM in
// MQ_PREC_FP64, tensor-core split GEMM in MQ_PREC_MIXED.  which = 1: the reaction coefficient b of
// family 2 (which, like its a, takes a piecewise zeroth term in place of a0).
// The separable evaluation pays off on fine meshes when the terms use few distinct k1: stage 2
// contracts over the padded k1 count instead of K.
bool use_separable(const mq_ctx* c, int n, int K) {
  if (!c->sep_ok || c->prec != MQ_PREC_MIXED || K <= 0 || n < 128) return false;
  return 4 * mq::tc_pad_k(c->k1prefix[K - 1]) <= K;
}

mq_status coefficients_separable(mq_ctx* c, int n, int K, const double* d_Y, int B, int ldy, double* d_a) {
  mq_status st;
  auto it = c->sep_tab.find(n);
  if (it == c->sep_tab.end()) {
    const int kp = mq::tc_pad_k(c->k1max);
    void* mem = nullptr;
    const size_t bytes = mq::sep_tables_bytes(n, kp, c->k2max);
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MQ_ENOMEM, "separable tables for n=%d (%zu bytes)", n, bytes);
    }
    if ((st = grow(c, c->sepw, (size_t)n * kp * sizeof(double))) != MQ_OK) {
      cudaFree(mem);
      return st;
    }
    mq::SepTables t{};
    const cudaError_t e = mq::launch_sep_tables(n, c->k1max, kp, c->k2max, (double*)c->sepw.p, mem, &t, c->stream);
    if (e != cudaSuccess) {
      cudaFree(mem);
      return fail(c, MQ_ECUDA, "separable tables: %s", cudaGetErrorString(e));
    }
    c->n_launches += 6;
    it = c->sep_tab.emplace(n, std::make_pair(mem, t)).first;
  }
  const int k1pad = mq::tc_pad_k(c->k1prefix[K - 1]);
  // |T| <= sum_{t<K} |y_t c_t| < csum / 2: the largest ey with 2^ey csum <= 1 keeps 2^ey |T| <= 1/2
  int ey = 0;
  const double cs = c->csum[K - 1];
  while (std::ldexp(cs, ey) > 1.0) --ey;
  while (std::ldexp(cs, ey + 1) <= 1.0) ++ey;
  if ((st = grow(c, c->tsl, mq::sep_scratch_bytes(B, n, K, k1pad))) != MQ_OK) return st;
  if ((st = grow(c, c->tc_err, sizeof(int))) != MQ_OK) return st;
  const mq::SepTerms terms{c->d_k1start, c->d_tlist, c->d_k2, c->d_cj[0]};
  MQ_CUDA(c, mq::launch_coef_sep(d_Y, ldy, B, K, k1pad, terms, it->second.second, n, c->a0, ey, c->tsl.p, d_a,
                                 (int*)c->tc_err.p, c->stream));
  c->n_launches += 5;  // the products Y c, two stage-1 kernels and two tensor-core launches
  return MQ_OK;
}

mq_status coefficients(mq_ctx* c, int n, int K, const double* d_Y, int B, int ldy, double* d_a, int which = 0) {
  const int nT = 2 * n * n;
  mq_status st;
  const double* base = nullptr;
  if (c->family == 2 && (st = ensure_base(c, n, which, &base)) != MQ_OK) return st;
  if (!base && which == 0 && use_separable(c, n, K)) return coefficients_separable(c, n, K, d_Y, B, ldy, d_a);
  const double a0 = base ? 0.0 : c->a0;
  if (c->prec == MQ_PREC_MIXED && K > 0) {
    const void* ps = nullptr;
    int kps = 0;
    if ((st = ensure_psi_slices(c, n, &ps, &kps, which)) != MQ_OK) return st;
    const int kpad = mq::tc_pad_k(K);
    if ((st = grow(c, c->ysl, mq::tc_slices_bytes(B, K))) != MQ_OK) return st;
    if ((st = grow(c, c->tc_err, sizeof(int))) != MQ_OK) return st;
    MQ_LAUNCH(c, mq::launch_y_slices(d_Y, B, ldy, K, kpad, c->ysl.p, c->stream));
    MQ_LAUNCH(c, mq::launch_coef_tc(c->ysl.p, B, kpad, ps, nT, kps, a0, d_a, (int*)c->tc_err.p, c->stream, base,
                                    c->psi_exp[which]));
    return MQ_OK;
  }
  const double* psi = nullptr;
  if ((st = ensure_psi(c, n, std::max(c->s_max, 1), &psi, which)) != MQ_OK) return st;
  MQ_LAUNCH(c, mq::launch_coef_gemm_f64(d_Y, ldy, B, K, psi, nT, a0, d_a, c->stream, base));
  return MQ_OK;
}

// Zeroes the error word of the tensor-core coefficient kernel (allocated here on first use:
// fresh device memory holds whatever a previous owner left there).
mq_status reset_tc_error(mq_ctx* c) {
  if (c->prec != MQ_PREC_MIXED) return MQ_OK;
  mq_status st = grow(c, c->tc_err, sizeof(int));
  if (st != MQ_OK) return st;
  MQ_CUDA(c, cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
  return MQ_OK;
}

mq_status check_tc_error(mq_ctx* c) {
  if (c->prec != MQ_PREC_MIXED || !c->tc_err.p) return MQ_OK;
  int e = 0;
  MQ_CUDA(c, cudaMemcpyAsync(&e, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  if (e) return fail(c, MQ_ETIMEOUT, "a bounded wait in the tensor-core coefficient kernel ran out");
  return MQ_OK;
}

mq_status check_level_ready(mq_ctx* c, int level) {
  if (!c->coef_set) return fail(c, MQ_ESTATE, "coefficient not set");
  if (c->levels.empty()) return fail(c, MQ_ESTATE, "levels not set");
  if (level < 0 || level >= (int)c->levels.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (c->d_z[level] == nullptr) return fail(c, MQ_ESTATE, "lattice of level %d not set", level);
  if (c->d_delta[level] == nullptr) return fail(c, MQ_ESTATE, "shifts of level %d not set", level);
  return MQ_OK;
}

// Default tier threshold (measured on GB300, 4-level workload): with FP32 inner solves the
// streaming tier wins from 1/32 on (the per-sample kernel fits only two samples of mesh 1/32 per
// SM); the FP64 path is FP64-throughput bound and keeps the per-sample kernel up to 1/128.
int stream_threshold(const mq_ctx* c) {
  if (c->stream_min > 0) return c->stream_min;
  return c->prec == MQ_PREC_MIXED ? 32 : 256;
}

// Threads per CTA of the per-sample kernel: n_fine is the largest mesh solved inside the kernel
// (0: coarse eigensolves only).  Meshes up to 1/16 run with two warps: their workspace (~24 KB)
// lets seven samples share an SM, which hides the barrier latency of the small phases better
// than more threads per sample (measured on GB300).
int threads_for(int n_fine, int n_coarse) {
  if (n_fine > 0 && n_fine <= 16) return 64;
  const int n = n_fine > n_coarse ? n_fine : n_coarse;
  return n <= 16 ? 128 : 256;
}

struct LevelGeom {
  int nf, nc, np, s, S, sp, direct_f, direct_p;
  int threads;  // requested threads per CTA of the per-sample kernel (0: default)
  int tier;     // -1: by mesh size; 0: fine solves in the per-sample kernel; 1: streaming tier
  int nu;       // Jacobi sweeps per side of the V-cycle for this level (0: default)
};

LevelGeom geom(const mq_ctx* c, int level) {
  const mq_level& lv = c->levels[level];
  LevelGeom g{};
  g.nf = lv.n_fine;
  g.nc = lv.n_coarse;
  g.s = lv.s;
  g.S = lv.S;
  g.direct_f = (lv.n_fine == lv.n_coarse && lv.s == lv.S);
  if (level > 0) {
    const mq_level& pv = c->levels[level - 1];
    g.np = pv.n_fine;
    g.sp = pv.s;
    g.direct_p = (pv.n_fine == lv.n_coarse && pv.s == lv.S);
  }
  g.threads = level < (int)c->cta_threads.size() ? c->cta_threads[level] : 0;
  g.tier = level < (int)c->lvl_tier.size() ? c->lvl_tier[level] : -1;
  g.nu = level < (int)c->lvl_nu.size() ? c->lvl_nu[level] : 0;
  return g;
}

// Jacobi sweeps per side of the streaming tier's V-cycle (V(1,1) unless set)
int stream_nu(const mq_ctx* c, const LevelGeom& g) { return g.nu > 0 ? g.nu : (c->opt_nu > 0 ? c->opt_nu : 1); }

// whether the fine solve of mesh g.nf runs in the streaming tier (whose kernels carry the reaction
// term of the second test problem on the FP32 path with V(1,1) smoothing only)
bool streams(const mq_ctx* c, const LevelGeom& g) {
  if (g.direct_f) return false;
  if (c->family == 2 && !(c->prec == MQ_PREC_MIXED && stream_nu(c, g) == 1)) return false;
  if (g.tier >= 0) return g.tier == 1;
  return g.nf >= stream_threshold(c);
}

// Runs the per-sample pipeline on B = R * npts samples whose parameters are in c->Y (ldy = s).
// Writes c->out / c->stat / c->outer; returns timings in stats.  In the reuse scheme, `level`
// and the first point `kbase` of the pass locate the stored level-0 pairs and lower-level values:
// levels l >= 1 take them instead of solving the coarse problem and the previous-level problem.
mq_status run_samples(mq_ctx* c, const LevelGeom& g, int R, int npts, int chunk, bool want_u, int level = -1,
                      uint32_t kbase = 0) {
  const size_t B = (size_t)R * npts;
  mq_status st;
  const bool given = c->reuse && level >= 1;  // coarse pair and lambda^{l-1} come from the store
  const bool rxn = c->family == 2;            // reaction term b u
  if (rxn && g.tier == 1 && !streams(c, g))
    return fail(c, MQ_EINVAL, "the streaming tier carries the reaction term only in mixed precision with V(1,1)");
  const size_t nTf = (size_t)2 * g.nf * g.nf, nTc = (size_t)2 * g.nc * g.nc, nTp = (size_t)2 * g.np * g.np;
  const size_t Vc = (size_t)(g.nc + 1) * (g.nc + 1);
  if (!given && (st = grow(c, c->ac, B * nTc * sizeof(double))) != MQ_OK) return st;
  if (!g.direct_f && (st = grow(c, c->af, B * nTf * sizeof(double))) != MQ_OK) return st;
  if (!given && g.np && !g.direct_p && (st = grow(c, c->ap, B * nTp * sizeof(double))) != MQ_OK) return st;
  if (rxn) {
    if (!given && (st = grow(c, c->bc, B * nTc * sizeof(double))) != MQ_OK) return st;
    if (!g.direct_f && (st = grow(c, c->bf, B * nTf * sizeof(double))) != MQ_OK) return st;
    if (!given && g.np && !g.direct_p && (st = grow(c, c->bp, B * nTp * sizeof(double))) != MQ_OK) return st;
  }
  if ((st = grow(c, c->out, B * 4 * sizeof(double))) != MQ_OK) return st;
  if ((st = grow(c, c->stat, B * 4 * sizeof(int))) != MQ_OK) return st;
  if ((st = grow(c, c->outer, B * 2 * sizeof(int))) != MQ_OK) return st;
  if (want_u && (st = grow(c, c->uout, B * (size_t)(g.nc - 1) * (g.nc - 1) * sizeof(double))) != MQ_OK) return st;
  if (c->reuse && (st = grow(c, c->upad, B * Vc * sizeof(double))) != MQ_OK) return st;

  const int mixed = c->prec == MQ_PREC_MIXED;
  if ((st = reset_tc_error(c)) != MQ_OK) return st;
  if (!c->capturing) MQ_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  const double* Y = (const double*)c->Y.p;
  if (given) {
    const uint32_t N0 = c->levels[0].N, Np = c->levels[level - 1].N;
    MQ_LAUNCH(c, mq::launch_reuse_gather(R, npts, kbase, Vc, (const double*)c->ru0.p, (const double*)c->rlamH.p, N0,
                                         (const double*)c->rlam[level - 1].p, Np, (double*)c->upad.p,
                                         (double*)c->out.p, c->stream, kshift(c)));
    MQ_CUDA(c, cudaMemsetAsync(c->stat.p, 0, B * 4 * sizeof(int), c->stream));
    MQ_CUDA(c, cudaMemsetAsync(c->outer.p, 0, B * 2 * sizeof(int), c->stream));
  } else {
    if ((st = coefficients(c, g.nc, g.S, Y, (int)B, g.s, (double*)c->ac.p)) != MQ_OK) return st;
    if (rxn && (st = coefficients(c, g.nc, g.S, Y, (int)B, g.s, (double*)c->bc.p, 1)) != MQ_OK) return st;
  }
  if (!g.direct_f && (st = coefficients(c, g.nf, g.s, Y, (int)B, g.s, (double*)c->af.p)) != MQ_OK) return st;
  if (rxn && !g.direct_f && (st = coefficients(c, g.nf, g.s, Y, (int)B, g.s, (double*)c->bf.p, 1)) != MQ_OK)
    return st;
  if (!given && g.np && !g.direct_p && (st = coefficients(c, g.np, g.sp, Y, (int)B, g.s, (double*)c->ap.p)) != MQ_OK)
    return st;
  if (rxn && !given && g.np && !g.direct_p &&
      (st = coefficients(c, g.np, g.sp, Y, (int)B, g.s, (double*)c->bp.p, 1)) != MQ_OK)
    return st;
  if (!c->capturing) MQ_CUDA(c, cudaEventRecord(c->ev[1], c->stream));

  mq::SampleLaunch p{};
  // Where each fine solve runs.  A solve on the coarse mesh itself (h = H with a longer
  // truncation) is nearly singular -- lambda_H differs from the fine eigenvalue only by the
  // truncation -- so it always runs in the per-sample kernel with an FP64 inner solve.
  const bool stream = streams(c, g);
  auto mode_of = [&](int n, bool direct) {
    if (direct || n == 0) return 0;
    if (n == g.nc) return mixed ? 1 : 0;
    return stream ? 2 : 0;
  };
  p.mode_f = mode_of(g.nf, g.direct_f);
  p.mode_p = given ? 0 : mode_of(g.np, g.direct_p);
  p.u_in = given ? (const double*)c->upad.p : nullptr;
  p.prev_given = given ? 1 : 0;
  p.nf = g.nf;
  p.nc = g.nc;
  p.np = g.np;
  p.direct_f = g.direct_f;
  p.direct_p = g.direct_p;
  p.R = R;
  p.npts = npts;
  p.chunk = chunk;
  p.a_f = (const double*)c->af.p;
  p.a_c = (const double*)c->ac.p;
  p.a_p = (const double*)c->ap.p;
  p.reaction = rxn ? 1 : 0;
  p.b_f = rxn ? (const double*)c->bf.p : nullptr;
  p.b_c = rxn ? (const double*)c->bc.p : nullptr;
  p.b_p = rxn ? (const double*)c->bp.p : nullptr;
  p.qoi = c->qoi;
  p.out = (double*)c->out.p;
  p.stat = (int*)c->stat.p;
  p.outer = (int*)c->outer.p;
  p.u_out = want_u ? (double*)c->uout.p : nullptr;
  // Default tolerances.  lambda_H is the Rayleigh quotient of the LOBPCG iterate, accurate to the
  // square of its relative eigen-residual (at most tol^2 kappa(M) theta / (lambda_2 - theta), with
  // kappa(M) <= 4): 1e-6 leaves it within ~3e-12 of the exact coarse eigenvalue at worst and within
  // 5e-14 measured on the six-level workload (levels 0-2 and 5), and the two-grid values,
  // which depend on u_H only through one shifted inverse-iteration step, moved by less than 3e-15
  // against 1e-8 -- with 2.6 fewer LOBPCG iterations per sample.  How far lambda^h moves with the
  // eigenvector error grows with the coarse-fine discrepancy: on the second test problem, whose
  // coarse mesh does not resolve the islands (lambda_H ~10 % above lambda^h), 1e-6 moved lambda^h
  // by 1e-10, so that family keeps 1e-8.  When the caller asks for the eigenvector itself
  // (mq_eval_point), 1e-8 keeps it accurate to ~1e-8.  The
  // Rayleigh quotient lambda^h of the shifted-solve iterate is stationary only at an eigenvector;
  // the two-grid iterate is an O(H^4) perturbation of one, so lambda^h moves to first order in the
  // solve error with a small constant: on the 4-level workload (meshes 1/16..1/128) the largest
  // relative change of lambda^h is about 3e-7 times the relative residual.  An FP64 residual of
  // 1e-6 keeps lambda^h within ~3e-13 of the exact two-grid value.  The mixed path refines
  // twice whatever the targets (the FP32 rounding of the first correction, which is
  // amplified by the near-singular shift, leaves a residual of ~1e-4): inner reductions of 1e-4
  // and a target of 1e-5 leave lambda^h within ~2e-13 (1e-5 inner reductions above mesh 1/128).
  // The functional G(u_H) of a direct level is first order in the eigenvector error, which the
  // eigen-residual bounds only to ~tol_eig (lambda_H is second order): it takes 1e-11.
  p.tol_eig = c->opt_tol_eig > 0 ? c->opt_tol_eig : (c->qoi == MQ_QOI_FUNCTIONAL ? 1e-11 : (want_u || rxn ? 1e-8 : 1e-6));
  p.max_eig_it = c->opt_max_eig > 0 ? c->opt_max_eig : 200;
  p.tol_lin = c->tol_lin > 0 ? c->tol_lin : (mixed ? 1e-5 : 1e-6);
  if (mixed) {
    // the preconditioned residual MINRES reduces understates the 2-norm one by a factor growing
    // like 1/h: finer meshes take a smaller inner reduction per refinement step
    p.tol_inner = g.nf > 128 ? 1e-5 : 1e-4;
    p.max_outer = 10;
  } else {
    p.tol_inner = 0.1 * p.tol_lin;
    p.max_outer = 4;
  }
  p.max_inner_it = 500;
  if (c->opt_tol_inner > 0) p.tol_inner = c->opt_tol_inner;
  if (c->opt_max_inner > 0) p.max_inner_it = c->opt_max_inner;
  if (c->opt_max_outer > 0) p.max_outer = c->opt_max_outer;
  // Smoothing per tier, measured on GB300 (4-level workload): V(1,1) needs ~10 % more MINRES
  // iterations than V(2,2) (and ~15 % more LOBPCG iterations) but moves about a third fewer bytes
  // per iteration, so it wins for the bandwidth-bound streaming tier; the latency-bound per-sample
  // kernel keeps V(2,2)
  p.nu = g.nu > 0 ? g.nu : (c->opt_nu > 0 ? c->opt_nu : 2);
  p.omega = 0.8;
  const bool ext = p.mode_f == 2 || p.mode_p == 2;
  if (ext || c->reuse) {
    // the streaming tier (and the reuse store of level 0) reads the padded coarse eigenvectors
    p.coarse_only = ext ? 1 : 0;
    if ((st = grow(c, c->upad, B * Vc * sizeof(double))) != MQ_OK) return st;
    if (!given) p.u_pad = (double*)c->upad.p;
  }
  // FP64 inner solves in the per-sample kernel follow the FP64 defaults
  const int np_k = given ? 0 : g.np;  // the previous-level solve runs here only without the store
  const int in_kernel_n = std::max(p.mode_f != 2 && !g.direct_f ? g.nf : 0, p.mode_p != 2 && !g.direct_p ? np_k : 0);
  const int threads = g.threads > 0 ? g.threads : threads_for(in_kernel_n, g.nc);
  const size_t slab = mq::sample_slab_bytes(g.nf, g.nc, np_k, mixed, p.mode_f, p.mode_p, p.reaction);
  const int static_smem = mq::sample_static_smem(mixed);
  const size_t smem_cap = (size_t)std::max(0, c->smem_optin - static_smem - 1024);
  const bool use_smem = slab <= smem_cap;
  const size_t smem = use_smem ? slab : 0;
  if (use_smem) MQ_CUDA(c, mq::set_sample_smem(mixed, (int)smem));
  int occ = mq::sample_occupancy(mixed, threads, smem);
  if (occ < 1) occ = 1;
  const int cpr = (npts + chunk - 1) / chunk;
  const long nchunks = (long)cpr * R;
  int blocks = (int)std::min<long>(nchunks, (long)c->sm_count * occ);
  if (blocks < 1) blocks = 1;
  if (!use_smem) {
    if ((st = grow(c, c->scratch, (size_t)blocks * slab)) != MQ_OK) return st;
  }
  p.gscratch = (char*)c->scratch.p;
  p.slab_bytes = slab;
  p.use_smem = use_smem;
  // with the coarse pairs and lambda^{l-1} given and the fine solve streamed, the per-sample
  // kernel has nothing to do
  if (!(given && p.mode_f == 2)) MQ_LAUNCH(c, mq::launch_sample(p, mixed, blocks, threads, smem, c->stream));
  if (!c->capturing) MQ_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  if (ext) {
    const uint64_t launched0 = mq::stream_launches();
    if ((st = grow(c, c->arena, mq::stream_arena_bytes(std::max(p.mode_f == 2 ? g.nf : 0, p.mode_p == 2 ? g.np : 0),
                                                       (int)B, mixed, rxn))) != MQ_OK)
      return st;
    mq::StreamSolve s{};
    mq::StreamGraph sg{{c->gbody[0], c->gbody[1]}, (int*)c->gcount.p};
    s.nc = g.nc;
    s.B = (int)B;
    s.uH = (const double*)c->upad.p;
    s.lamH = (const double*)c->out.p;
    s.lam_stride = 4;
    s.lam_out_stride = 4;
    s.iters_stride = 4;
    s.outer_stride = 2;
    s.flags = (int*)c->stat.p + 3;
    s.flags_stride = 4;
    s.tol_lin = p.tol_lin;
    s.tol_inner = p.tol_inner;
    s.max_inner = p.max_inner_it;
    s.max_outer = p.max_outer;
    s.omega = p.omega;
    s.nu = stream_nu(c, g);
    s.probe = (c->probe_on && !c->capturing) ? &c->probe : nullptr;
    s.qoi = c->qoi;
    s.b = nullptr;
    if (p.mode_f == 2) {
      s.n = g.nf;
      s.a = (const double*)c->af.p;
      s.b = rxn ? (const double*)c->bf.p : nullptr;
      s.lam_out = (double*)c->out.p + 1;
      s.iters_out = (int*)c->stat.p + 1;
      s.outer_out = (int*)c->outer.p + 0;
      MQ_CUDA(c, mq::stream_solve(s, mixed, c->arena.p, c->stream, c->capturing ? &sg : nullptr));
    }
    if (p.mode_p == 2 && !given) {
      s.n = g.np;
      s.a = (const double*)c->ap.p;
      s.b = rxn ? (const double*)c->bp.p : nullptr;
      s.lam_out = (double*)c->out.p + 2;
      s.iters_out = (int*)c->stat.p + 2;
      s.outer_out = (int*)c->outer.p + 1;
      MQ_CUDA(c, mq::stream_solve(s, mixed, c->arena.p, c->stream, c->capturing ? &sg : nullptr));
    }
    MQ_CUDA(c, mq::launch_finalize((int)B, (double*)c->out.p, g.np > 0, c->stream));
    c->n_launches += mq::stream_launches() - launched0;
  }
  if (!c->capturing) MQ_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  c->stats.blocks = blocks;
  c->stats.threads = threads;
  c->stats.smem_bytes = (int)smem;
  c->stats.workspace_bytes = (int64_t)slab;
  return MQ_OK;
}

mq_status collect_stats(mq_ctx* c, size_t B, int* any_flags) {
  std::vector<int> st(B * 4), ou(B * 2);
  MQ_CUDA(c, cudaMemcpyAsync(st.data(), c->stat.p, B * 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaMemcpyAsync(ou.data(), c->outer.p, B * 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  mq_stats& s = c->stats;
  double ce = 0, fi = 0, oi = 0;
  long nf = 0;
  int cemax = 0, fimax = 0, oimax = 0, fl = 0;
  uint64_t nc = 0;
  for (size_t b = 0; b < B; ++b) {
    ce += st[b * 4];
    cemax = std::max(cemax, st[b * 4]);
    for (int k = 0; k < 2; ++k) {
      if (ou[b * 2 + k] > 0) {
        fi += st[b * 4 + 1 + k];
        fimax = std::max(fimax, st[b * 4 + 1 + k]);
        oi += ou[b * 2 + k];
        oimax = std::max(oimax, ou[b * 2 + k]);
        ++nf;
      }
    }
    fl |= st[b * 4 + 3];
    if (st[b * 4 + 3] & (mq::kFlagEigNoConv | mq::kFlagLinNoConv | mq::kFlagBreakdown)) ++nc;
  }
  s.samples = B;
  s.noconv = nc;
  s.coarse_iters_mean = B ? ce / B : 0;
  s.coarse_iters_max = cemax;
  s.fine_iters_mean = nf ? fi / nf : 0;
  s.fine_iters_max = fimax;
  s.outer_iters_mean = nf ? oi / nf : 0;
  s.outer_iters_max = oimax;
  *any_flags = fl;
  return MQ_OK;
}

mq_status timing(mq_ctx* c, int level) {
  float t0 = 0, t1 = 0, t2 = 0;
  MQ_CUDA(c, cudaEventSynchronize(c->ev[2]));
  if (c->probe_on) MQ_CUDA(c, c->probe.collect());
  MQ_CUDA(c, cudaEventElapsedTime(&t0, c->ev[0], c->ev[1]));
  MQ_CUDA(c, cudaEventElapsedTime(&t1, c->ev[1], c->ev[2]));
  MQ_CUDA(c, cudaEventElapsedTime(&t2, c->ev[1], c->ev[3]));
  c->stats.coef_ms += t0;
  c->stats.sample_ms += t1;
  c->stats.kernel_ms += t0 + t1;
  if (level >= 0 && level < (int)c->lvl_coef_ms.size()) {
    c->lvl_coef_ms[level] += t0;
    c->lvl_sample_ms[level] += t1;
    c->lvl_percta_ms[level] += t2;
    c->lvl_stream_ms[level] += t1 - t2;
    c->lvl_launches[level] += 1;
  }
  return MQ_OK;
}

mq_status flags_status(mq_ctx* c, int fl) {
  if (fl & mq::kFlagBadCoef)
    return fail(c, MQ_EINVAL, "coefficient a(x, y) <= 0 (or reaction b(x, y) < 0) at a centroid");
  if (fl & (mq::kFlagEigNoConv | mq::kFlagLinNoConv | mq::kFlagBreakdown))
    return fail(c, MQ_ENOCONV, "%llu sample(s) hit an iteration cap or broke down (flags 0x%x)",
                (unsigned long long)c->stats.noconv, fl);
  return MQ_OK;
}

// points per pass so that the coefficient buffers stay within a memory budget
int points_per_pass(const mq_ctx* c, const LevelGeom& g, int R, int npts) {
  // coefficient fields of the three meshes (twice with the reaction coefficient of family 2)
  const size_t fields = (size_t)2 * g.nf * g.nf + (size_t)2 * g.nc * g.nc + (size_t)2 * g.np * g.np;
  size_t per_sample = sizeof(double) * ((c->family == 2 ? 2 : 1) * fields + (size_t)g.s + 8 +
                                        (size_t)(g.nc + 1) * (g.nc + 1));
  if (streams(c, g) && g.nf != g.nc)
    per_sample += mq::stream_arena_bytes(g.nf, 1, c->prec == MQ_PREC_MIXED, c->family == 2);
  size_t free_b = 0, total_b = 0;
  size_t budget = (size_t)24 << 30;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = std::min<size_t>((size_t)(0.4 * free_b), (size_t)64 << 30);
  budget /= (size_t)std::max(1, c->mem_share);
  size_t pts = budget / (per_sample * (size_t)R);
  if (pts < 1) pts = 1;
  return (int)std::min<size_t>(pts, (size_t)npts);
}

int chunk_for(const mq_ctx* c, int R, int npts) {
  // points per warm-start chain: enough chains to fill the GPU, chains as long as possible
  const long want = (long)c->sm_count * 4;
  long ch = ((long)R * npts + want - 1) / want;
  return (int)std::max(1L, std::min<long>(ch, 64));
}

mq_status eval_level_impl(mq_ctx* c, int level, uint32_t k0, uint32_t k1, double* per_sample, double* shift_sums,
                          double* d_per_sample, double* d_shift_sums) {
  mq_status st = check_level_ready(c, level);
  if (st != MQ_OK) return st;
  const mq_level& lv = c->levels[level];
  if (k1 < k0 || k1 > lv.N) return fail(c, MQ_EINVAL, "point range [%u, %u) outside [0, %u)", k0, k1, lv.N);
  MQ_CUDA(c, cudaSetDevice(c->device));
  const LevelGeom g = geom(c, level);
  const int R = lv.R;
  const int npts = (int)(k1 - k0);
  c->stats = mq_stats{};
  if (npts == 0) return MQ_OK;
  if (c->reuse && level >= 1) {
    // the stored level-0 pairs and level l-1 values of these points must exist
    for (uint32_t k = k0; k < k1; ++k)
      if (!c->rfilled[0][k] || !c->rfilled[level - 1][k])
        return fail(c, MQ_ESTATE, "reuse: evaluate levels 0 and %d at point %u before level %d", level - 1, k, level);
  }
  // while a graph is captured nothing may query the device: the pass size of the rehearsal is used
  if ((int)c->last_ppp.size() < (int)c->levels.size()) c->last_ppp.resize(c->levels.size(), 0);
  const int ppp = c->capturing && c->last_ppp[level] > 0 ? std::min(c->last_ppp[level], npts)
                                                         : points_per_pass(c, g, R, npts);
  c->last_ppp[level] = ppp;
  // the captured range's slot in the graph's sum accumulators
  double* gsum = nullptr;
  if (c->capturing) gsum = (double*)c->gsums.p + c->g_off.back();
  std::vector<double> host_out;
  std::vector<double> level_add(R, 0.0);
  int any_flags = 0;
  for (int p0 = 0; p0 < npts; p0 += ppp) {
    const int pn = std::min(ppp, npts - p0);
    const size_t B = (size_t)R * pn;
    if ((st = grow(c, c->Y, B * g.s * sizeof(double))) != MQ_OK) return st;
    const int mb = c->mbits[level];
    MQ_LAUNCH(c, mq::launch_lattice_points(c->d_z[level], mb ? (1u << mb) : lv.N, c->d_delta[level], R, g.s, k0 + p0,
                                         pn, mb, (double*)c->Y.p, c->stream, kshift(c)));
    if ((st = run_samples(c, g, R, pn, chunk_for(c, R, pn), false, level, k0 + p0)) != MQ_OK) return st;
    if (c->reuse) {
      const mq_level& l0 = c->levels[0];
      const size_t V0 = (size_t)(l0.n_fine + 1) * (l0.n_fine + 1);
      MQ_LAUNCH(c, mq::launch_reuse_scatter(R, pn, k0 + p0, V0, (const double*)c->upad.p, (const double*)c->out.p,
                                            (double*)c->rlam[level].p, lv.N, level == 0 ? (double*)c->ru0.p : nullptr,
                                            level == 0 ? (double*)c->rlamH.p : nullptr, l0.N, c->stream, kshift(c)));
    }
    if (c->capturing) {
      // graph schedule: sums and flags accumulate on the device; outputs go to device buffers
      MQ_LAUNCH(c, mq::launch_shift_sums((const double*)c->out.p, (const int*)c->stat.p, R, pn, gsum,
                                       (int*)c->gflags.p, c->stream, 1));
      if (d_per_sample) {
        for (int r = 0; r < R; ++r)
          MQ_CUDA(c, cudaMemcpyAsync(d_per_sample + ((size_t)r * npts + p0) * 4,
                                     (const double*)c->out.p + (size_t)r * pn * 4, (size_t)pn * 4 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c->stream));
      }
      c->last_B = B;
      continue;
    }
    if ((st = grow(c, c->sums_d, R * sizeof(double))) != MQ_OK) return st;
    if ((st = grow(c, c->flags_d, sizeof(int))) != MQ_OK) return st;
    MQ_CUDA(c, cudaMemsetAsync(c->flags_d.p, 0, sizeof(int), c->stream));
    MQ_LAUNCH(c, mq::launch_shift_sums((const double*)c->out.p, (const int*)c->stat.p, R, pn, (double*)c->sums_d.p,
                                     (int*)c->flags_d.p, c->stream));
    std::vector<double> sums(R);
    int fl = 0;
    MQ_CUDA(c, cudaMemcpyAsync(sums.data(), c->sums_d.p, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MQ_CUDA(c, cudaMemcpyAsync(&fl, c->flags_d.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (per_sample) {
      host_out.resize(B * 4);
      MQ_CUDA(c, cudaMemcpyAsync(host_out.data(), c->out.p, B * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    if (d_per_sample) {
      // [R][npts][4] layout of the caller: scatter this pass's [R][pn][4]
      for (int r = 0; r < R; ++r)
        MQ_CUDA(c, cudaMemcpyAsync(d_per_sample + ((size_t)r * npts + p0) * 4,
                                   (const double*)c->out.p + (size_t)r * pn * 4, (size_t)pn * 4 * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->stream));
    }
    MQ_CUDA(c, cudaStreamSynchronize(c->stream));
    if ((st = timing(c, level)) != MQ_OK) return st;
    if ((st = check_tc_error(c)) != MQ_OK) return st;
    if (per_sample) {
      for (int r = 0; r < R; ++r)
        std::memcpy(per_sample + ((size_t)r * npts + p0) * 4, host_out.data() + (size_t)r * pn * 4,
                    (size_t)pn * 4 * sizeof(double));
    }
    for (int r = 0; r < R; ++r) level_add[r] += sums[r];
    any_flags |= fl;
    c->last_B = B;
  }
  if (c->capturing) {
    if (d_shift_sums)
      MQ_CUDA(c, cudaMemcpyAsync(d_shift_sums, gsum, R * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (c->reuse)
      for (uint32_t k = k0; k < k1; ++k) c->rfilled[level][k] = 1;
    return MQ_OK;
  }
  if (d_shift_sums)
    MQ_CUDA(c, cudaMemcpyAsync(d_shift_sums, level_add.data(), R * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int r = 0; r < R; ++r) {
    c->sums[level][r] += level_add[r];
    if (shift_sums) shift_sums[r] += level_add[r];
  }
  c->npoints[level] += (uint64_t)npts;
  if (c->reuse)
    for (uint32_t k = k0; k < k1; ++k) c->rfilled[level][k] = 1;
  if (any_flags) {
    int dummy;
    if ((st = collect_stats(c, c->last_B, &dummy)) != MQ_OK) return st;
  }
  c->stats.samples = (uint64_t)R * npts;
  return flags_status(c, any_flags);
}

// pairwise sum of f(0) .. f(n-1) (rounding error grows like log n, not n)
template <class F>
double pairwise_sum(uint32_t lo, uint32_t n, const F& f) {
  if (n <= 16) {
    double s = 0.0;
    for (uint32_t k = lo; k < lo + n; ++k) s += f(k);
    return s;
  }
  const uint32_t h = n / 2;
  return pairwise_sum(lo, h, f) + pairwise_sum(lo + h, n - h, f);
}

}  // namespace

extern "C" {

mq_status mq_create(mq_ctx** out, int device, void* cuda_stream) {
  if (!out) return MQ_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return MQ_ECUDA;
  }
  if (device < 0 || device >= ndev) return MQ_EINVAL;
  mq_ctx* c = new (std::nothrow) mq_ctx();
  if (!c) return MQ_ENOMEM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return MQ_ECUDA;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MQ_ECUDA;
    }
    c->own_stream = true;
  }
  for (auto& e : c->ev) cudaEventCreate(&e);
  *out = c;
  return MQ_OK;
}

mq_status mq_destroy(mq_ctx* c) {
  if (!c) return MQ_EINVAL;
  for (mq_ctx* l : c->lanes)
    if (l) mq_destroy(l);
  c->lanes.clear();
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  graph_release(c);
  for (cudaStream_t& b : c->gbody)
    if (b) cudaStreamDestroy(b);
  for (auto& pe : c->probe.ev) {
    cudaEventDestroy(pe.first);
    cudaEventDestroy(pe.second);
  }
  for (DevBuf* b : {&c->gcount, &c->gsums, &c->gflags, &c->gk0, &c->probe_bytes})
    if (b->p) cudaFree(b->p);
  for (DevBuf* b : {&c->Y, &c->af, &c->ac, &c->ap, &c->out, &c->stat, &c->outer, &c->scratch, &c->sums_d,
                    &c->flags_d, &c->uout, &c->misc, &c->upad, &c->arena, &c->ysl, &c->tc_err, &c->bf, &c->bc,
                    &c->bp, &c->tsl, &c->sepw})
    if (b->p) cudaFree(b->p);
  release_tables(c);
  free_reuse(c);
  for (auto p : c->d_z)
    if (p) cudaFree(p);
  for (auto p : c->d_delta)
    if (p) cudaFree(p);
  if (c->d_k1) cudaFree(c->d_k1);
  if (c->d_k2) cudaFree(c->d_k2);
  for (double* p : c->d_cj)
    if (p) cudaFree(p);
  if (c->d_region) cudaFree(c->d_region);
  if (c->d_k1start) cudaFree(c->d_k1start);
  if (c->d_tlist) cudaFree(c->d_tlist);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return MQ_OK;
}

const char* mq_last_error(const mq_ctx* c) { return c ? c->err.c_str() : "null context"; }

namespace {

// Term tables of a family: wave numbers, factors of a (and b) and region codes, uploaded once.
mq_status set_terms(mq_ctx* c, double a0, int32_t s_max, int32_t family, double decay, const double* decays4) {
  c->lanes_stale = true;
  graph_release(c);
  if (!(a0 > 0.0) || !std::isfinite(a0)) return fail(c, MQ_EINVAL, "a0 must be positive, got %g", a0);
  if (s_max < 0 || s_max > 65536) return fail(c, MQ_EINVAL, "s_max %d out of range", s_max);
  if (family < 0 || family > 2) return fail(c, MQ_EINVAL, "unknown coefficient family %d", family);
  if (!std::isfinite(decay)) return fail(c, MQ_EINVAL, "decay must be finite");
  if (decays4)
    for (int i = 0; i < 4; ++i)
      if (!std::isfinite(decays4[i])) return fail(c, MQ_EINVAL, "decays must be finite");
  MQ_CUDA(c, cudaSetDevice(c->device));
  const int m = std::max(s_max, 1);
  std::vector<int> k1, k2, region;
  std::vector<double> cj[2];
  cj[0].resize(m);
  if (family == 2) {
    // term j = 1, 2, ...: odd j on D_f with k = (j+1)/2, even j off D_f with k = j/2; w_k has wave
    // numbers 8k and 8(k+1) in the pi-scaled sines
    cj[1].resize(m);
    k1.resize(m);
    k2.resize(m);
    region.resize(m);
    for (int j = 1; j <= m; ++j) {
      const bool odd = j % 2 == 1;
      const int k = odd ? (j + 1) / 2 : j / 2;
      const int r = odd ? 0 : 1;
      k1[j - 1] = 8 * k;
      k2[j - 1] = 8 * (k + 1);
      region[j - 1] = odd ? 1 : 2;
      cj[0][j - 1] = kSigA[r] * std::pow((double)k, -decays4[r]);
      cj[1][j - 1] = kSigB[r] * std::pow((double)k, -decays4[2 + r]);
    }
  } else {
    psi_pairs(m, family, k1, k2);
    for (int j = 0; j < m; ++j) cj[0][j] = std::pow((double)(j + 1), -decay);
  }
  release_tables(c);
  if (c->d_k1) cudaFree(c->d_k1);
  if (c->d_k2) cudaFree(c->d_k2);
  for (double*& p : c->d_cj) {
    if (p) cudaFree(p);
    p = nullptr;
  }
  if (c->d_region) cudaFree(c->d_region);
  c->d_k1 = c->d_k2 = c->d_region = nullptr;
  MQ_CUDA(c, cudaMalloc(&c->d_k1, m * sizeof(int)));
  MQ_CUDA(c, cudaMalloc(&c->d_k2, m * sizeof(int)));
  MQ_CUDA(c, cudaMemcpy(c->d_k1, k1.data(), m * sizeof(int), cudaMemcpyHostToDevice));
  MQ_CUDA(c, cudaMemcpy(c->d_k2, k2.data(), m * sizeof(int), cudaMemcpyHostToDevice));
  for (int w = 0; w < (family == 2 ? 2 : 1); ++w) {
    MQ_CUDA(c, cudaMalloc(&c->d_cj[w], m * sizeof(double)));
    MQ_CUDA(c, cudaMemcpy(c->d_cj[w], cj[w].data(), m * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (family == 2) {
    MQ_CUDA(c, cudaMalloc(&c->d_region, m * sizeof(int)));
    MQ_CUDA(c, cudaMemcpy(c->d_region, region.data(), m * sizeof(int), cudaMemcpyHostToDevice));
  }
  // slice scale of each table: the largest e with 2^e max_j |c_j| <= 1 (|sin sin| <= 1), e = 0 for the
  // families whose factors j^-decay are at most 1
  for (int w = 0; w < 2; ++w) {
    double mx = 0.0;
    for (double v : cj[w]) mx = std::max(mx, std::fabs(v));
    int e = 0;
    if (mx > 0.0 && std::isfinite(mx)) {
      while (std::ldexp(mx, e) > 1.0) --e;
      while (std::ldexp(mx, e + 1) <= 1.0) ++e;
    }
    c->psi_exp[w] = e;
  }
  // separable evaluation (family 0): the terms grouped by k1 in increasing t
  if (c->d_k1start) cudaFree(c->d_k1start);
  if (c->d_tlist) cudaFree(c->d_tlist);
  c->d_k1start = c->d_tlist = nullptr;
  c->sep_ok = false;
  if (family == 0) {
    int k1m = 0, k2m = 0;
    c->k1prefix.assign(m, 0);
    c->csum.assign(m, 0.0);
    double cs = 0.0;
    for (int t = 0; t < m; ++t) {
      k1m = std::max(k1m, k1[t]);
      k2m = std::max(k2m, k2[t]);
      cs += std::fabs(cj[0][t]);
      c->k1prefix[t] = k1m;
      c->csum[t] = cs;
    }
    const int kp = mq::tc_pad_k(k1m);
    // start[v] .. start[v + 1] lists the terms of k1 = v (start[kp + 1] = m closes the last list)
    std::vector<int> start(kp + 2, 0), list;
    list.reserve(m);
    for (int v = 1; v <= kp; ++v) {
      start[v] = (int)list.size();
      for (int t = 0; t < m; ++t)
        if (k1[t] == v) list.push_back(t);
    }
    start[kp + 1] = (int)list.size();
    start[0] = 0;
    MQ_CUDA(c, cudaMalloc(&c->d_k1start, start.size() * sizeof(int)));
    MQ_CUDA(c, cudaMalloc(&c->d_tlist, std::max<size_t>(list.size(), 1) * sizeof(int)));
    MQ_CUDA(c, cudaMemcpy(c->d_k1start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
    MQ_CUDA(c, cudaMemcpy(c->d_tlist, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->k1max = k1m;
    c->k2max = k2m;
    c->sep_ok = true;
  }
  c->a0 = a0;
  c->s_max = s_max;
  c->family = family;
  c->decay = decay;
  for (int i = 0; i < 4; ++i) c->decays[i] = decays4 ? decays4[i] : decay;
  c->coef_set = true;
  return MQ_OK;
}

}  // namespace

mq_status mq_set_coefficient(mq_ctx* c, double a0, int32_t s_max, int32_t family, double decay) {
  if (!c) return MQ_EINVAL;
  const double d4[4] = {decay, decay, decay, decay};
  return set_terms(c, a0, s_max, family, decay, family == 2 ? d4 : nullptr);
}

mq_status mq_set_islands(mq_ctx* c, int32_t s_max, double p_a, double p_a_out, double p_b, double p_b_out) {
  if (!c) return MQ_EINVAL;
  const double d4[4] = {p_a, p_a_out, p_b, p_b_out};
  return set_terms(c, 1.0, s_max, 2, p_a, d4);
}

mq_status mq_set_qoi(mq_ctx* c, int32_t qoi) {
  if (!c) return MQ_EINVAL;
  if (qoi != MQ_QOI_EIGENVALUE && qoi != MQ_QOI_FUNCTIONAL) return fail(c, MQ_EINVAL, "unknown quantity %d", qoi);
  if (qoi == c->qoi) return MQ_OK;
  c->lanes_stale = true;
  graph_release(c);
  invalidate_reuse(c);  // the store holds values of the previous quantity
  c->qoi = qoi;
  return mq_reset_sums(c);
}

mq_status mq_set_levels(mq_ctx* c, int32_t L_plus_1, const mq_level* levels) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (L_plus_1 < 1 || L_plus_1 > 32 || !levels) return fail(c, MQ_EINVAL, "need 1..32 levels");
  if (!c->coef_set) return fail(c, MQ_ESTATE, "set the coefficient before the levels");
  for (int l = 0; l < L_plus_1; ++l) {
    const mq_level& v = levels[l];
    if (!pow2(v.n_fine) || !pow2(v.n_coarse) || v.n_coarse < 2 || v.n_fine > 4096 || v.n_coarse > v.n_fine)
      return fail(c, MQ_EINVAL, "level %d: meshes must be powers of two with 2 <= n_coarse <= n_fine <= 4096", l);
    if (v.S < 1 || v.s < v.S || v.s > c->s_max)
      return fail(c, MQ_EINVAL, "level %d: need 1 <= S <= s <= s_max (%d)", l, c->s_max);
    if (v.N < 1 || v.R < 1) return fail(c, MQ_EINVAL, "level %d: need N >= 1 and R >= 1", l);
    if (l > 0) {
      const mq_level& p = levels[l - 1];
      if (p.n_fine < v.n_coarse || p.n_fine % v.n_coarse)
        return fail(c, MQ_EINVAL, "level %d: coarse mesh must be nested in the fine mesh of level %d", l, l - 1);
      if (p.s > v.s) return fail(c, MQ_EINVAL, "level %d: s must not decrease across levels", l);
    }
  }
  MQ_CUDA(c, cudaSetDevice(c->device));
  for (auto p : c->d_z)
    if (p) cudaFree(p);
  for (auto p : c->d_delta)
    if (p) cudaFree(p);
  free_reuse(c);
  c->levels.assign(levels, levels + L_plus_1);
  c->z.assign(L_plus_1, {});
  c->mbits.assign(L_plus_1, 0);
  c->delta.assign(L_plus_1, {});
  c->d_z.assign(L_plus_1, nullptr);
  c->d_delta.assign(L_plus_1, nullptr);
  c->sums.assign(L_plus_1, {});
  for (int l = 0; l < L_plus_1; ++l) c->sums[l].assign(levels[l].R, 0.0);
  c->npoints.assign(L_plus_1, 0);
  c->lvl_coef_ms.assign(L_plus_1, 0.0);
  c->lvl_sample_ms.assign(L_plus_1, 0.0);
  c->lvl_launches.assign(L_plus_1, 0);
  c->lvl_percta_ms.assign(L_plus_1, 0.0);
  c->n_launches = 0;
  c->lvl_stream_ms.assign(L_plus_1, 0.0);
  return MQ_OK;
}

mq_status mq_set_lattice(mq_ctx* c, int32_t level, const uint32_t* z, int32_t s) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (level < 0 || level >= (int)c->levels.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  const mq_level& lv = c->levels[level];
  if (!z || s != lv.s) return fail(c, MQ_EINVAL, "lattice of level %d needs s = %d components", level, lv.s);
  for (int j = 0; j < s; ++j)
    if (z[j] == 0 || z[j] >= lv.N) return fail(c, MQ_EINVAL, "z[%d] = %u not in (0, N)", j, z[j]);
  MQ_CUDA(c, cudaSetDevice(c->device));
  if (c->d_z[level]) cudaFree(c->d_z[level]);
  c->d_z[level] = nullptr;
  MQ_CUDA(c, cudaMalloc(&c->d_z[level], s * sizeof(uint32_t)));
  MQ_CUDA(c, cudaMemcpy(c->d_z[level], z, s * sizeof(uint32_t), cudaMemcpyHostToDevice));
  c->z[level].assign(z, z + s);
  c->mbits[level] = 0;
  invalidate_reuse(c);
  return MQ_OK;
}

mq_status mq_set_lattice_embedded(mq_ctx* c, int32_t level, const uint32_t* z, int32_t s, int32_t m_max) {
  if (!c) return MQ_EINVAL;
  if (level < 0 || level >= (int)c->levels.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (m_max < 1 || m_max > 31) return fail(c, MQ_EINVAL, "m_max %d not in [1, 31]", m_max);
  const mq_level& lv = c->levels[level];
  if (!pow2((int)std::min<uint32_t>(lv.N, 1u << 30)) || lv.N > (1u << m_max))
    return fail(c, MQ_EINVAL, "level %d: N = %u must be a power of two <= 2^m_max", level, lv.N);
  if (!z || s != lv.s) return fail(c, MQ_EINVAL, "lattice of level %d needs s = %d components", level, lv.s);
  for (int j = 0; j < s; ++j)
    if (z[j] % 2 == 0 || z[j] >= (1u << m_max)) return fail(c, MQ_EINVAL, "z[%d] = %u must be odd and < 2^m_max", j, z[j]);
  const uint32_t N = lv.N;
  c->levels[level].N = 1u << m_max;  // validated against the embedded modulus, then restored
  mq_status st = mq_set_lattice(c, level, z, s);
  c->levels[level].N = N;
  if (st != MQ_OK) return st;
  c->mbits[level] = m_max;
  return MQ_OK;
}

mq_status mq_set_shifts(mq_ctx* c, int32_t level, const double* delta) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (level < 0 || level >= (int)c->levels.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (!delta) return fail(c, MQ_EINVAL, "null shifts");
  const mq_level& lv = c->levels[level];
  const size_t m = (size_t)lv.R * lv.s;
  for (size_t q = 0; q < m; ++q)
    if (!(delta[q] >= 0.0 && delta[q] < 1.0)) return fail(c, MQ_EINVAL, "shift entry %zu = %g not in [0, 1)", q, delta[q]);
  MQ_CUDA(c, cudaSetDevice(c->device));
  if (c->d_delta[level]) cudaFree(c->d_delta[level]);
  c->d_delta[level] = nullptr;
  MQ_CUDA(c, cudaMalloc(&c->d_delta[level], m * sizeof(double)));
  MQ_CUDA(c, cudaMemcpy(c->d_delta[level], delta, m * sizeof(double), cudaMemcpyHostToDevice));
  c->delta[level].assign(delta, delta + m);
  invalidate_reuse(c);
  return MQ_OK;
}

mq_status mq_set_reuse(mq_ctx* c, int32_t on) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (!on) {
    free_reuse(c);
    return MQ_OK;
  }
  invalidate_reuse(c);
  const int L1 = (int)c->levels.size();
  if (L1 == 0) return fail(c, MQ_ESTATE, "levels not set");
  const mq_level& l0 = c->levels[0];
  if (l0.n_coarse != l0.n_fine || l0.S != l0.s) return fail(c, MQ_EINVAL, "reuse: level 0 must be a direct eigensolve");
  int top = 0;
  for (int l = 0; l < L1; ++l) {
    const mq_level& lv = c->levels[l];
    if (l > 0 && (lv.n_coarse != l0.n_fine || lv.S != l0.s))
      return fail(c, MQ_EINVAL, "reuse: level %d must use level 0's coarse problem (n_coarse = %d, S = %d)", l, l0.n_fine,
                  l0.s);
    if (lv.R != l0.R) return fail(c, MQ_EINVAL, "reuse: every level needs the same R");
    if (l > 0 && lv.N > c->levels[l - 1].N) return fail(c, MQ_EINVAL, "reuse: N must not grow with the level");
    if (!c->d_z[l] || !c->d_delta[l]) return fail(c, MQ_ESTATE, "reuse: lattice and shifts of level %d not set", l);
    if (c->mbits[l] == 0 || c->mbits[l] != c->mbits[0])
      return fail(c, MQ_EINVAL, "reuse: every level needs the same embedded lattice (mq_set_lattice_embedded)");
    if (lv.s > c->levels[top].s) top = l;
  }
  // one generating vector and one set of shifts: every level's are prefixes of the longest
  for (int l = 0; l < L1; ++l) {
    const int s = c->levels[l].s, sT = c->levels[top].s;
    for (int j = 0; j < s; ++j)
      if (c->z[l][j] != c->z[top][j]) return fail(c, MQ_EINVAL, "reuse: level %d lattice is not a prefix of level %d's", l, top);
    for (int r = 0; r < l0.R; ++r)
      for (int j = 0; j < s; ++j)
        if (c->delta[l][(size_t)r * s + j] != c->delta[top][(size_t)r * sT + j])
          return fail(c, MQ_EINVAL, "reuse: level %d shifts are not a prefix of level %d's", l, top);
  }
  MQ_CUDA(c, cudaSetDevice(c->device));
  const size_t V0 = (size_t)(l0.n_fine + 1) * (l0.n_fine + 1);
  mq_status st = grow(c, c->ru0, (size_t)l0.R * l0.N * V0 * sizeof(double));
  if (st != MQ_OK) return st;
  if ((st = grow(c, c->rlamH, (size_t)l0.R * l0.N * sizeof(double))) != MQ_OK) return st;
  if ((int)c->rlam.size() != L1) {
    for (DevBuf& b : c->rlam)
      if (b.p) cudaFree(b.p);
    c->rlam.assign(L1, DevBuf{});
  }
  c->rfilled.assign(L1, {});
  for (int l = 0; l < L1; ++l) {
    if ((st = grow(c, c->rlam[l], (size_t)l0.R * c->levels[l].N * sizeof(double))) != MQ_OK) {
      free_reuse(c);
      return st;
    }
    c->rfilled[l].assign(c->levels[l].N, 0);
  }
  c->reuse = true;
  return MQ_OK;
}

mq_status mq_set_precision(mq_ctx* c, mq_precision prec, double tol_linear) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (prec != MQ_PREC_FP64 && prec != MQ_PREC_MIXED) return fail(c, MQ_EINVAL, "unknown precision %d", (int)prec);
  if (!std::isfinite(tol_linear) || tol_linear >= 1.0) return fail(c, MQ_EINVAL, "tolerance must be < 1");
  c->prec = prec;
  c->tol_lin = tol_linear > 0 ? tol_linear : 0.0;
  return MQ_OK;
}

mq_status mq_set_solver_options(mq_ctx* c, double tol_inner, int32_t max_inner, int32_t max_outer) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (!std::isfinite(tol_inner) || tol_inner >= 1.0 || max_inner > 100000 || max_outer > 1000)
    return fail(c, MQ_EINVAL, "bad solver options");
  c->opt_tol_inner = tol_inner > 0 ? tol_inner : 0.0;
  c->opt_max_inner = max_inner > 0 ? max_inner : 0;
  c->opt_max_outer = max_outer > 0 ? max_outer : 0;
  return MQ_OK;
}

mq_status mq_set_eig_options(mq_ctx* c, double tol_eig, int32_t max_eig) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (!std::isfinite(tol_eig) || tol_eig >= 1.0 || max_eig > 100000) return fail(c, MQ_EINVAL, "bad eigensolver options");
  c->opt_tol_eig = tol_eig > 0 ? tol_eig : 0.0;
  c->opt_max_eig = max_eig > 0 ? max_eig : 0;
  return MQ_OK;
}

mq_status mq_set_cta_threads(mq_ctx* c, int32_t level, int32_t threads) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (level < 0 || level >= 64) return fail(c, MQ_EINVAL, "level %d out of range", (int)level);
  if (threads != 0 && (threads < 32 || threads > 512 || threads % 32 != 0))
    return fail(c, MQ_EINVAL, "threads must be 0 or a multiple of 32 in [32, 512]");
  if ((int)c->cta_threads.size() <= level) c->cta_threads.resize(level + 1, 0);
  c->cta_threads[level] = threads;
  return MQ_OK;
}

mq_status mq_set_level_config(mq_ctx* c, int32_t level, int32_t tier, int32_t threads, int32_t nu) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (level < 0 || level >= 64) return fail(c, MQ_EINVAL, "level %d out of range", (int)level);
  if (tier < -1 || tier > 1) return fail(c, MQ_EINVAL, "tier must be -1, 0 or 1");
  if (nu < 0 || nu > 2) return fail(c, MQ_EINVAL, "nu must be 0, 1 or 2");
  mq_status st = mq_set_cta_threads(c, level, threads);
  if (st != MQ_OK) return st;
  if ((int)c->lvl_tier.size() <= level) c->lvl_tier.resize(level + 1, -1);
  if ((int)c->lvl_nu.size() <= level) c->lvl_nu.resize(level + 1, 0);
  c->lvl_tier[level] = tier;
  c->lvl_nu[level] = nu;
  return MQ_OK;
}

mq_status mq_autotune_level(mq_ctx* c, int32_t level, uint32_t points, const char* cache_path, mq_tune_choice* out) {
  if (!c || !out) return MQ_EINVAL;
  mq_status st = check_level_ready(c, level);
  if (st != MQ_OK) return st;
  if (c->reuse) return fail(c, MQ_ESTATE, "autotune: switch the reuse scheme off first");
  const mq_level& lv = c->levels[level];
  if (points < 1 || points > lv.N) return fail(c, MQ_EINVAL, "autotune: need 1 <= points <= N");
  MQ_CUDA(c, cudaSetDevice(c->device));
  *out = mq_tune_choice{};
  // cache key: the GPU, the precision and everything about the level that shapes its kernels
  cudaDeviceProp prop;
  MQ_CUDA(c, cudaGetDeviceProperties(&prop, c->device));
  const LevelGeom g0 = geom(c, level);
  char key[512];
  snprintf(key, sizeof key, "gpu=%s|sms=%d|prec=%d|nf=%d|nc=%d|np=%d|s=%d|S=%d|sp=%d|R=%d|pts=%u|tol=%g|fam=%d",
           prop.name, c->sm_count, c->prec, g0.nf, g0.nc, g0.np, g0.s, g0.S, g0.sp, lv.R, points, c->tol_lin,
           c->family);
  for (char* q = key; *q; ++q)
    if (*q == ' ') *q = '_';
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[1024];
      while (fgets(line, sizeof line, f)) {
        char k[600];
        int tier, threads, nu;
        double ms;
        if (sscanf(line, "%599s %d %d %d %lf", k, &tier, &threads, &nu, &ms) == 5 && strcmp(k, key) == 0) {
          fclose(f);
          out->tier = tier;
          out->threads = threads;
          out->nu = nu;
          out->ms = ms;
          out->from_cache = 1;
          return mq_set_level_config(c, level, tier, threads, nu);
        }
      }
      fclose(f);
    }
  }
  // candidates: the fine solve's tier (when it is a two-grid level whose mesh both tiers handle
  // well), the per-sample kernel's threads per CTA, the smoothing steps
  std::vector<int> tiers = {-1};
  if (!g0.direct_f && g0.nf >= 16 && g0.nf <= 128) tiers = {0, 1};
  const int thr[3] = {64, 128, 256};
  // save the estimator state and the level's settings: probes must leave neither behind
  const auto sums = c->sums;
  const auto npoints = c->npoints;
  const auto t_coef = c->lvl_coef_ms, t_samp = c->lvl_sample_ms, t_pc = c->lvl_percta_ms, t_st = c->lvl_stream_ms;
  const auto t_l = c->lvl_launches;
  const uint64_t nl0 = c->n_launches;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MQ_CUDA(c, cudaEventCreate(&e0));
  MQ_CUDA(c, cudaEventCreate(&e1));
  double best = 1e300;
  int bt = -1, bth = 0, bnu = 0, tried = 0;
  mq_status result = MQ_OK;
  for (int tier : tiers)
    for (int th : thr)
      for (int nu = 1; nu <= 2 && result == MQ_OK; ++nu) {
        // the streaming tier takes the reaction term only in mixed precision with V(1,1)
        if (tier == 1 && c->family == 2 && (c->prec != MQ_PREC_MIXED || nu != 1)) continue;
        if ((result = mq_set_level_config(c, level, tier, th, nu)) != MQ_OK) break;
        double ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {  // the first run also builds tables and buffers
          if (cudaEventRecord(e0, c->stream) != cudaSuccess) result = fail(c, MQ_ECUDA, "event record");
          mq_status s2 = eval_level_impl(c, level, 0, points, nullptr, nullptr, nullptr, nullptr);
          if (s2 != MQ_OK && s2 != MQ_ENOCONV) result = s2;
          if (result != MQ_OK) break;
          cudaEventRecord(e1, c->stream);
          cudaEventSynchronize(e1);
          float t = 0.0f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep == 1 && s2 == MQ_OK) ms = t;
        }
        ++tried;
        if (ms < best) {
          best = ms;
          bt = tier;
          bth = th;
          bnu = nu;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->sums = sums;
  c->npoints = npoints;
  c->lvl_coef_ms = t_coef;
  c->lvl_sample_ms = t_samp;
  c->lvl_percta_ms = t_pc;
  c->lvl_stream_ms = t_st;
  c->lvl_launches = t_l;
  c->n_launches = nl0;
  if (result != MQ_OK) return result;
  if (best >= 1e300) return fail(c, MQ_ENOCONV, "autotune: no configuration converged");
  out->tier = bt;
  out->threads = bth;
  out->nu = bnu;
  out->ms = best;
  out->tried = tried;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s %d %d %d %.6f\n", key, bt, bth, bnu, best);
      fclose(f);
    }
  }
  return mq_set_level_config(c, level, bt, bth, bnu);
}

mq_status mq_set_smoothing(mq_ctx* c, int32_t nu) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (nu < 0 || nu > 2) return fail(c, MQ_EINVAL, "nu must be 0 (default), 1 or 2");
  c->opt_nu = nu;
  return MQ_OK;
}

mq_status mq_set_tier(mq_ctx* c, int32_t stream_min_n) {
  if (!c) return MQ_EINVAL;
  c->lanes_stale = true;
  graph_release(c);
  if (stream_min_n < 0 || stream_min_n == 1) return fail(c, MQ_EINVAL, "stream_min_n must be 0 or >= 2");
  c->stream_min = stream_min_n;
  return MQ_OK;
}

mq_status mq_eval_level(mq_ctx* c, int32_t level, uint32_t k0, uint32_t k1, double* per_sample, double* shift_sums) {
  if (!c) return MQ_EINVAL;
  return eval_level_impl(c, level, k0, k1, per_sample, shift_sums, nullptr, nullptr);
}

mq_status mq_eval_level_device(mq_ctx* c, int32_t level, uint32_t k0, uint32_t k1, double* d_per_sample,
                               double* d_shift_sums) {
  if (!c) return MQ_EINVAL;
  return eval_level_impl(c, level, k0, k1, nullptr, nullptr, d_per_sample, d_shift_sums);
}

mq_status mq_eval_levels_device(mq_ctx* c, int32_t nlev, const int32_t* levels, double* const* d_per_sample,
                                double* const* d_shift_sums) {
  if (!c) return MQ_EINVAL;
  if (nlev < 0 || (nlev > 0 && !levels)) return fail(c, MQ_EINVAL, "bad level list");
  for (int i = 0; i < nlev; ++i) {
    const mq_status st = check_level_ready(c, levels[i]);
    if (st != MQ_OK) return st;
    for (int k = 0; k < i; ++k)
      if (levels[k] == levels[i]) return fail(c, MQ_EINVAL, "level %d listed twice", (int)levels[i]);
  }
  if (nlev == 0) return MQ_OK;
  if (c->reuse) return fail(c, MQ_ESTATE, "reuse: the levels depend on one another; evaluate them in order");
  MQ_CUDA(c, cudaSetDevice(c->device));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));  // earlier work of the caller's stream first
  // one child context per level: its own stream, buffers and host thread
  if (c->lanes_stale) {
    for (mq_ctx* l : c->lanes)
      if (l) mq_destroy(l);
    c->lanes.clear();
    c->lanes_stale = false;
  }
  if (c->lanes.size() < c->levels.size()) c->lanes.resize(c->levels.size(), nullptr);
  for (int i = 0; i < nlev; ++i) {
    const int l = levels[i];
    if (!c->lanes[l]) {
      mq_ctx* ch = nullptr;
      mq_status st = mq_create(&ch, c->device, nullptr);
      if (st != MQ_OK) return fail(c, st, "creating the context of level %d failed", l);
      auto chk = [&](mq_status s2) {
        if (s2 != MQ_OK && st == MQ_OK) st = s2;
      };
      if (c->family == 2)
        chk(mq_set_islands(ch, c->s_max, c->decays[0], c->decays[1], c->decays[2], c->decays[3]));
      else
        chk(mq_set_coefficient(ch, c->a0, c->s_max, c->family, c->decay));
      chk(mq_set_levels(ch, (int32_t)c->levels.size(), c->levels.data()));
      chk(mq_set_qoi(ch, c->qoi));
      if (c->mbits[l])
        chk(mq_set_lattice_embedded(ch, l, c->z[l].data(), (int32_t)c->z[l].size(), c->mbits[l]));
      else
        chk(mq_set_lattice(ch, l, c->z[l].data(), (int32_t)c->z[l].size()));
      chk(mq_set_shifts(ch, l, c->delta[l].data()));
      chk(mq_set_precision(ch, (mq_precision)c->prec, c->tol_lin));
      chk(mq_set_solver_options(ch, c->opt_tol_inner, c->opt_max_inner, c->opt_max_outer));
      chk(mq_set_eig_options(ch, c->opt_tol_eig, c->opt_max_eig));
      chk(mq_set_smoothing(ch, c->opt_nu));
      chk(mq_set_tier(ch, c->stream_min));
      if (l < (int)c->cta_threads.size()) chk(mq_set_cta_threads(ch, l, c->cta_threads[l]));
      if (l < (int)c->lvl_tier.size())
        chk(mq_set_level_config(ch, l, c->lvl_tier[l], l < (int)c->cta_threads.size() ? c->cta_threads[l] : 0,
                                l < (int)c->lvl_nu.size() ? c->lvl_nu[l] : 0));
      if (st != MQ_OK) {
        const std::string m = ch->err;
        mq_destroy(ch);
        return fail(c, st, "configuring the context of level %d: %s", l, m.c_str());
      }
      c->lanes[l] = ch;
    }
    c->lanes[l]->mem_share = nlev;
  }
  std::vector<mq_status> status(nlev, MQ_OK);
  std::vector<std::thread> threads;
  try {
    for (int i = 0; i < nlev; ++i)
      threads.emplace_back([c, levels, d_per_sample, d_shift_sums, i, &status] {
        const int l = levels[i];
        if (cudaSetDevice(c->device) != cudaSuccess) {
          status[i] = MQ_ECUDA;
          return;
        }
        status[i] = mq_eval_level_device(c->lanes[l], l, 0, c->levels[l].N, d_per_sample ? d_per_sample[i] : nullptr,
                                         d_shift_sums ? d_shift_sums[i] : nullptr);
      });
  } catch (...) {
    for (auto& t : threads) t.join();
    return fail(c, MQ_ENOMEM, "could not start the level threads");
  }
  for (auto& t : threads) t.join();
  // fold the levels' sums, timers and counters into this context
  mq_status result = MQ_OK;
  for (int i = 0; i < nlev; ++i) {
    const int l = levels[i];
    mq_ctx* ch = c->lanes[l];
    for (size_t r = 0; r < c->sums[l].size(); ++r) c->sums[l][r] += ch->sums[l][r];
    c->npoints[l] += ch->npoints[l];
    c->lvl_coef_ms[l] += ch->lvl_coef_ms[l];
    c->lvl_sample_ms[l] += ch->lvl_sample_ms[l];
    c->lvl_launches[l] += ch->lvl_launches[l];
    c->lvl_percta_ms[l] += ch->lvl_percta_ms[l];
    c->lvl_stream_ms[l] += ch->lvl_stream_ms[l];
    c->n_launches += ch->n_launches;
    c->stats = ch->stats;
    if (status[i] != MQ_OK && (result == MQ_OK || result == MQ_ENOCONV)) {
      result = status[i];
      c->err = "level " + std::to_string(l) + ": " + ch->err;
    }
    mq_reset_sums(ch);
  }
  return result;
}

mq_status mq_graph_capture(mq_ctx* c, int32_t nlev, const int32_t* levels, const uint32_t* k0s, const uint32_t* k1s,
                           double* const* d_per_sample, double* const* d_shift_sums) {
  if (!c) return MQ_EINVAL;
  if (nlev < 1 || !levels || !k0s || !k1s) return fail(c, MQ_EINVAL, "graph: bad range list");
  for (int i = 0; i < nlev; ++i) {
    mq_status st = check_level_ready(c, levels[i]);
    if (st != MQ_OK) return st;
    if (k1s[i] < k0s[i] || k1s[i] > c->levels[levels[i]].N) return fail(c, MQ_EINVAL, "graph: range %d outside the level", i);
  }
  MQ_CUDA(c, cudaSetDevice(c->device));
  graph_release(c);
  // 1. rehearsal: the same evaluations run normally -- every buffer is allocated, the tables are
  //    built and the pass sizes fixed -- then the estimator state is put back
  const auto sums = c->sums;
  const auto npoints = c->npoints;
  const auto t_coef = c->lvl_coef_ms, t_samp = c->lvl_sample_ms, t_pc = c->lvl_percta_ms, t_st = c->lvl_stream_ms;
  const auto t_l = c->lvl_launches;
  const auto filled = c->rfilled;
  const uint64_t nl0 = c->n_launches;
  auto restore = [&] {
    c->sums = sums;
    c->npoints = npoints;
    c->lvl_coef_ms = t_coef;
    c->lvl_sample_ms = t_samp;
    c->lvl_percta_ms = t_pc;
    c->lvl_stream_ms = t_st;
    c->lvl_launches = t_l;
    c->rfilled = filled;
    c->n_launches = nl0;
  };
  size_t nsum = 0;
  for (int i = 0; i < nlev; ++i) {
    mq_status st = eval_level_impl(c, levels[i], k0s[i], k1s[i], nullptr, nullptr,
                                   d_per_sample ? d_per_sample[i] : nullptr, d_shift_sums ? d_shift_sums[i] : nullptr);
    if (st != MQ_OK && st != MQ_ENOCONV) {
      restore();
      return st;
    }
    nsum += (size_t)c->levels[levels[i]].R;
  }
  restore();
  // 2. the graph's own device state, and the streams its loop bodies are captured on
  mq_status st;
  if ((st = grow(c, c->gcount, 2 * sizeof(int))) != MQ_OK) return st;
  if ((st = grow(c, c->gsums, nsum * sizeof(double))) != MQ_OK) return st;
  if ((st = grow(c, c->gflags, sizeof(int))) != MQ_OK) return st;
  if ((st = grow(c, c->gk0, nlev * sizeof(uint32_t))) != MQ_OK) return st;
  if ((st = grow(c, c->tc_err, sizeof(int))) != MQ_OK) return st;
  MQ_CUDA(c, cudaMemset(c->gk0.p, 0, nlev * sizeof(uint32_t)));
  for (cudaStream_t& b : c->gbody)
    if (!b) MQ_CUDA(c, cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
  // 3. capture
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  MQ_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  c->g_off.clear();
  cudaError_t ce = cudaMemsetAsync(c->gsums.p, 0, nsum * sizeof(double), c->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(c->gflags.p, 0, sizeof(int), c->stream);
  st = ce == cudaSuccess ? MQ_OK : fail(c, MQ_ECUDA, "graph: %s", cudaGetErrorString(ce));
  size_t off = 0;
  for (int i = 0; i < nlev && st == MQ_OK; ++i) {
    c->g_off.push_back(off);
    st = eval_level_impl(c, levels[i], k0s[i], k1s[i], nullptr, nullptr, d_per_sample ? d_per_sample[i] : nullptr,
                         d_shift_sums ? d_shift_sums[i] : nullptr);
    off += (size_t)c->levels[levels[i]].R;
  }
  c->capturing = false;
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(c->stream, &g);
  const uint64_t nodes = c->n_launches - nl0;
  c->n_launches = nl0;
  c->rfilled = filled;  // the graph's launches fill the reuse store, not its capture
  if (st != MQ_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    c->g_off.clear();
    cudaGetLastError();
    return st != MQ_OK ? st : fail(c, MQ_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&c->gexec, g, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(g);
    c->gexec = nullptr;
    c->g_off.clear();
    return fail(c, MQ_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  }
  c->graph = g;
  c->g_levels.assign(levels, levels + nlev);
  c->g_k0.assign(k0s, k0s + nlev);
  c->g_k1.assign(k1s, k1s + nlev);
  c->g_cap_k0.assign(k0s, k0s + nlev);
  c->g_shift.assign(nlev, 0u);
  c->graph_kernels = nodes;
  return MQ_OK;
}

mq_status mq_graph_launch(mq_ctx* c, const uint32_t* k0s) {
  if (!c) return MQ_EINVAL;
  if (!c->gexec) return fail(c, MQ_ESTATE, "graph: nothing captured (or a later call invalidated the graph)");
  MQ_CUDA(c, cudaSetDevice(c->device));
  if (k0s) {
    // replay on ranges of the captured lengths that start at k0s[i]: the kernels add the offset
    // from the captured start (modulo 2^32) that the graph reads from device memory
    for (size_t i = 0; i < c->g_levels.size(); ++i)
      if ((uint64_t)k0s[i] + (c->g_k1[i] - c->g_k0[i]) > c->levels[c->g_levels[i]].N)
        return fail(c, MQ_EINVAL, "graph: range %zu moved outside its level", i);
    for (size_t i = 0; i < c->g_levels.size(); ++i) {
      const uint32_t len = c->g_k1[i] - c->g_k0[i];
      c->g_k0[i] = k0s[i];
      c->g_k1[i] = k0s[i] + len;
      c->g_shift[i] = k0s[i] - c->g_cap_k0[i];
    }
    MQ_CUDA(c, cudaMemcpyAsync(c->gk0.p, c->g_shift.data(), c->g_shift.size() * sizeof(uint32_t),
                               cudaMemcpyHostToDevice, c->stream));
  }
  if (c->reuse) {
    // levels >= 1 of the graph read what its levels below store; both are in the same graph, in order
    for (size_t i = 0; i < c->g_levels.size(); ++i)
      if (c->g_levels[i] >= 1)
        for (uint32_t k = c->g_k0[i]; k < c->g_k1[i]; ++k) {
          bool below = false;
          for (size_t j = 0; j < i; ++j)
            below |= c->g_levels[j] == c->g_levels[i] - 1 && c->g_k0[j] <= k && k < c->g_k1[j];
          if (!below && !c->rfilled[c->g_levels[i] - 1][k])
            return fail(c, MQ_ESTATE, "graph: level %d needs level %d at point %u first", c->g_levels[i],
                        c->g_levels[i] - 1, k);
        }
  }
  MQ_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
  const size_t nsum = c->g_off.empty() ? 0 : c->g_off.back() + (size_t)c->levels[c->g_levels.back()].R;
  std::vector<double> gs(nsum);
  int fl = 0, te = 0;
  MQ_CUDA(c, cudaMemcpyAsync(gs.data(), c->gsums.p, nsum * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaMemcpyAsync(&fl, c->gflags.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (c->prec == MQ_PREC_MIXED)
    MQ_CUDA(c, cudaMemcpyAsync(&te, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  if (te) return fail(c, MQ_ETIMEOUT, "a bounded wait in the tensor-core coefficient kernel ran out");
  uint64_t samples = 0;
  for (size_t i = 0; i < c->g_levels.size(); ++i) {
    const int l = c->g_levels[i];
    for (int r = 0; r < c->levels[l].R; ++r) c->sums[l][r] += gs[c->g_off[i] + r];
    c->npoints[l] += c->g_k1[i] - c->g_k0[i];
    samples += (uint64_t)c->levels[l].R * (c->g_k1[i] - c->g_k0[i]);
    if (c->reuse)
      for (uint32_t k = c->g_k0[i]; k < c->g_k1[i]; ++k) c->rfilled[l][k] = 1;
  }
  c->stats = mq_stats{};
  if (fl) {
    int dummy;
    mq_status st = collect_stats(c, c->last_B, &dummy);
    if (st != MQ_OK) return st;
  }
  c->stats.samples = samples;
  return flags_status(c, fl);
}

mq_status mq_measure_fp64_peak(int device, double* tflops, double* ms) {
  if (!tflops || !ms) return MQ_EINVAL;
  return mq::measure_fp64_peak(device, tflops, ms) == cudaSuccess ? MQ_OK : MQ_ECUDA;
}

mq_status mq_set_kernel_probe(mq_ctx* c, int32_t on) {
  if (!c) return MQ_EINVAL;
  MQ_CUDA(c, cudaSetDevice(c->device));
  mq_status st = grow(c, c->probe_bytes, sizeof(unsigned long long));
  if (st != MQ_OK) return st;
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  MQ_CUDA(c, cudaMemset(c->probe_bytes.p, 0, sizeof(unsigned long long)));
  c->probe.ms = 0.0;
  c->probe.launches = 0;
  c->probe.used = 0;
  c->probe.d_bytes = (unsigned long long*)c->probe_bytes.p;
  c->probe_on = on != 0;
  return MQ_OK;
}

mq_status mq_get_kernel_probe(mq_ctx* c, double* ms, uint64_t* launches, uint64_t* bytes) {
  if (!c) return MQ_EINVAL;
  MQ_CUDA(c, cudaSetDevice(c->device));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  MQ_CUDA(c, c->probe.collect());
  unsigned long long b = 0;
  if (c->probe_bytes.p) MQ_CUDA(c, cudaMemcpy(&b, c->probe_bytes.p, sizeof b, cudaMemcpyDeviceToHost));
  if (ms) *ms = c->probe.ms;
  if (launches) *launches = c->probe.launches;
  if (bytes) *bytes = (uint64_t)b;
  return MQ_OK;
}

mq_status mq_get_graph_info(mq_ctx* c, int32_t* captured, uint64_t* kernel_nodes) {
  if (!c) return MQ_EINVAL;
  if (captured) *captured = c->gexec != nullptr;
  if (kernel_nodes) *kernel_nodes = c->gexec ? c->graph_kernels : 0;
  return MQ_OK;
}

mq_status mq_get_sums(mq_ctx* c, int32_t level, double* sums, uint64_t* npoints) {
  if (!c) return MQ_EINVAL;
  if (level < 0 || level >= (int)c->sums.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (sums) std::copy(c->sums[level].begin(), c->sums[level].end(), sums);
  if (npoints) *npoints = c->npoints[level];
  return MQ_OK;
}

mq_status mq_estimate_sums(int32_t nlevels, const int32_t* R, const double* sums, const uint64_t* npoints,
                           int32_t shared, double* mean, double* std_err, double* level_mean, double* level_var) {
  if (nlevels < 1 || !R || !sums || !npoints) return MQ_EINVAL;
  for (int l = 0; l < nlevels; ++l) {
    if (R[l] < 2 || npoints[l] == 0) return MQ_EINVAL;
    if (shared && R[l] != R[0]) return MQ_EINVAL;
  }
  double tot = 0.0, var = 0.0;
  std::vector<double> qtot(shared ? R[0] : 0, 0.0);
  size_t off = 0;
  for (int l = 0; l < nlevels; ++l) {
    const int Rl = R[l];
    std::vector<double> q(Rl);
    double m = 0.0;
    for (int r = 0; r < Rl; ++r) {
      q[r] = sums[off + r] / (double)npoints[l];
      m += q[r];
    }
    m /= Rl;
    double v = 0.0;
    for (int r = 0; r < Rl; ++r) v += (m - q[r]) * (m - q[r]);
    v /= (double)Rl * (Rl - 1);
    tot += m;
    var += v;
    for (size_t r = 0; r < qtot.size(); ++r) qtot[r] += q[r];
    if (level_mean) level_mean[l] = m;
    if (level_var) level_var[l] = v;
    off += (size_t)Rl;
  }
  if (shared) {
    const int Rs = (int)qtot.size();
    double m = 0.0, v = 0.0;
    for (int r = 0; r < Rs; ++r) m += qtot[r];
    m /= Rs;
    for (int r = 0; r < Rs; ++r) v += (m - qtot[r]) * (m - qtot[r]);
    var = v / ((double)Rs * (Rs - 1));
  }
  if (mean) *mean = tot;
  if (std_err) *std_err = std::sqrt(var);
  return MQ_OK;
}

mq_status mq_run_adaptive(mq_ctx* c, double eps, double alpha, uint32_t n_init, mq_adaptive_result* res) {
  if (!c || !res) return MQ_EINVAL;
  if (!(eps > 0.0) || !std::isfinite(eps) || !(alpha > 0.0) || !std::isfinite(alpha) || n_init < 1)
    return fail(c, MQ_EINVAL, "adaptive: need eps > 0, alpha > 0, n_init >= 1");
  const int L1 = (int)c->levels.size();
  if (L1 == 0) return fail(c, MQ_ESTATE, "levels not set");
  if (L1 > 32) return fail(c, MQ_EINVAL, "adaptive: at most 32 levels");
  if (c->reuse) return fail(c, MQ_ESTATE, "adaptive: switch the reuse scheme off (levels must be independent)");
  for (int l = 0; l < L1; ++l) {
    mq_status st = check_level_ready(c, l);
    if (st != MQ_OK) return st;
    if (c->mbits[l] == 0) return fail(c, MQ_ESTATE, "adaptive: level %d needs an embedded lattice", l);
    if (c->levels[l].R < 2) return fail(c, MQ_EINVAL, "adaptive: level %d needs R >= 2", l);
  }
  // cost per sample: the fine unknowns it solves (the level's mesh, and the previous level's on a
  // two-grid level l > 0)
  std::vector<double> cost(L1);
  for (int l = 0; l < L1; ++l) {
    const mq_level& lv = c->levels[l];
    const double nf = (double)(lv.n_fine - 1) * (lv.n_fine - 1);
    const bool direct = lv.n_fine == lv.n_coarse && lv.s == lv.S;
    cost[l] = nf + (l > 0 && !direct ? (double)(c->levels[l - 1].n_fine - 1) * (c->levels[l - 1].n_fine - 1) : 0.0);
  }
  mq_status st = mq_reset_sums(c);
  if (st != MQ_OK) return st;
  *res = mq_adaptive_result{};
  std::vector<uint32_t> N;
  bool noconv = false;
  auto add = [&](int l, uint32_t n_new) -> mq_status {
    if (l == (int)N.size()) N.push_back(0);
    mq_status s2 = eval_level_impl(c, l, N[l], n_new, nullptr, nullptr, nullptr, nullptr);
    if (s2 == MQ_ENOCONV) noconv = true;
    else if (s2 != MQ_OK) return s2;
    if (n_new > N[l] && N[l] > 0) ++res->doublings;
    else ++res->levels_added;
    N[l] = n_new;
    return MQ_OK;
  };
  auto stats = [&](std::vector<double>& m, std::vector<double>& v) {
    m.assign(N.size(), 0.0);
    v.assign(N.size(), 0.0);
    for (size_t l = 0; l < N.size(); ++l) {
      const int R = c->levels[l].R;
      double mm = 0.0;
      for (int r = 0; r < R; ++r) mm += c->sums[l][r] / (double)N[l];
      mm /= R;
      double vv = 0.0;
      for (int r = 0; r < R; ++r) {
        const double q = c->sums[l][r] / (double)N[l];
        vv += (mm - q) * (mm - q);
      }
      m[l] = mm;
      v[l] = vv / ((double)R * (R - 1));
    }
  };
  for (int l = 0; l < std::min(3, L1); ++l)
    if ((st = add(l, std::min<uint32_t>(n_init, c->levels[l].N))) != MQ_OK) return st;
  std::vector<double> m, v;
  bool converged = false;
  for (;;) {
    stats(m, v);
    bool stuck = false;
    for (;;) {
      double tot = 0.0;
      for (double x : v) tot += x;
      if (!(tot > eps * eps / 2.0)) break;
      int best = -1;
      double bs = -1.0;
      for (size_t l = 0; l < N.size(); ++l) {
        const double sc = 2ull * N[l] <= c->levels[l].N ? v[l] / (cost[l] * N[l]) : -1.0;
        if (sc > bs) {
          bs = sc;
          best = (int)l;
        }
      }
      if (bs < 0.0) {
        stuck = true;
        break;
      }
      if ((st = add(best, 2 * N[best])) != MQ_OK) return st;
      stats(m, v);
    }
    if (stuck) break;
    const int L = (int)N.size() - 1;
    if (L >= 2) {
      const double bias = std::max(std::fabs(m[L]), std::fabs(m[L - 1]) / std::pow(2.0, alpha));
      if (bias <= (std::pow(2.0, alpha) - 1.0) * eps / std::sqrt(2.0)) {
        converged = true;
        break;
      }
    }
    if (L + 1 >= L1) break;
    if ((st = add(L + 1, std::min<uint32_t>(n_init, c->levels[L + 1].N))) != MQ_OK) return st;
  }
  stats(m, v);
  res->L = (int32_t)N.size() - 1;
  res->converged = converged ? 1 : 0;
  double mean = 0.0, var = 0.0;
  for (size_t l = 0; l < N.size(); ++l) {
    res->N[l] = N[l];
    res->level_mean[l] = m[l];
    res->level_var[l] = v[l];
    mean += m[l];
    var += v[l];
  }
  res->mean = mean;
  res->std_err = std::sqrt(var);
  return noconv ? fail(c, MQ_ENOCONV, "adaptive: some samples hit an iteration cap (results written)") : MQ_OK;
}

mq_status mq_reset_sums(mq_ctx* c) {
  if (!c) return MQ_EINVAL;
  for (size_t l = 0; l < c->sums.size(); ++l) std::fill(c->sums[l].begin(), c->sums[l].end(), 0.0);
  std::fill(c->npoints.begin(), c->npoints.end(), 0);
  std::fill(c->lvl_coef_ms.begin(), c->lvl_coef_ms.end(), 0.0);
  std::fill(c->lvl_sample_ms.begin(), c->lvl_sample_ms.end(), 0.0);
  std::fill(c->lvl_launches.begin(), c->lvl_launches.end(), 0);
  std::fill(c->lvl_percta_ms.begin(), c->lvl_percta_ms.end(), 0.0);
  c->n_launches = 0;
  std::fill(c->lvl_stream_ms.begin(), c->lvl_stream_ms.end(), 0.0);
  return MQ_OK;
}

mq_status mq_get_level_timing(mq_ctx* c, int32_t level, double* coef_ms, double* sample_ms, uint64_t* launches) {
  if (!c) return MQ_EINVAL;
  if (level < 0 || level >= (int)c->lvl_coef_ms.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (coef_ms) *coef_ms = c->lvl_coef_ms[level];
  if (sample_ms) *sample_ms = c->lvl_sample_ms[level];
  if (launches) *launches = c->lvl_launches[level];
  return MQ_OK;
}

mq_status mq_get_kernel_timing(mq_ctx* c, int32_t level, double* percta_ms, double* stream_ms) {
  if (!c) return MQ_EINVAL;
  if (level < 0 || level >= (int)c->lvl_percta_ms.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (percta_ms) *percta_ms = c->lvl_percta_ms[level];
  if (stream_ms) *stream_ms = c->lvl_stream_ms[level];
  return MQ_OK;
}

mq_status mq_get_launch_count(mq_ctx* c, uint64_t* launches) {
  if (!c || !launches) return MQ_EINVAL;
  *launches = c->n_launches;
  return MQ_OK;
}

mq_status mq_estimate(mq_ctx* c, double* mean, double* std_err, double* level_mean, double* level_var) {
  if (!c) return MQ_EINVAL;
  if (c->levels.empty()) return fail(c, MQ_ESTATE, "levels not set");
  double tot = 0.0, var = 0.0;
  // reuse scheme: one set of shifts for every level, so the per-shift totals sum_l Q^(r)_l are the
  // independent replicates; their sample variance replaces the sum of the level variances
  std::vector<double> qtot(c->reuse ? c->levels[0].R : 0, 0.0);
  for (size_t l = 0; l < c->levels.size(); ++l) {
    const int R = c->levels[l].R;
    if (c->npoints[l] == 0) return fail(c, MQ_ESTATE, "level %zu has no evaluated points", l);
    if (R < 2) return fail(c, MQ_EINVAL, "level %zu: the standard error needs R >= 2 shifts", l);
    std::vector<double> q(R);
    double m = 0.0;
    for (int r = 0; r < R; ++r) {
      q[r] = c->sums[l][r] / (double)c->npoints[l];
      m += q[r];
    }
    m /= R;
    double v = 0.0;
    for (int r = 0; r < R; ++r) v += (m - q[r]) * (m - q[r]);
    v /= (double)R * (R - 1);
    tot += m;
    var += v;
    for (size_t r = 0; r < qtot.size(); ++r) qtot[r] += q[r];
    if (level_mean) level_mean[l] = m;
    if (level_var) level_var[l] = v;
  }
  if (c->reuse) {
    const int R = (int)qtot.size();
    double m = 0.0, v = 0.0;
    for (int r = 0; r < R; ++r) m += qtot[r];
    m /= R;
    for (int r = 0; r < R; ++r) v += (m - qtot[r]) * (m - qtot[r]);
    var = v / ((double)R * (R - 1));
  }
  if (mean) *mean = tot;
  if (std_err) *std_err = std::sqrt(var);
  return MQ_OK;
}

mq_status mq_eval_point(mq_ctx* c, int32_t level, const double* y, double* lam_H, double* lam_h, double* lam_hm1,
                        double* u_H) {
  if (!c) return MQ_EINVAL;
  if (!c->coef_set) return fail(c, MQ_ESTATE, "coefficient not set");
  if (level < 0 || level >= (int)c->levels.size()) return fail(c, MQ_EINVAL, "level %d out of range", level);
  if (!y) return fail(c, MQ_EINVAL, "null parameter vector");
  MQ_CUDA(c, cudaSetDevice(c->device));
  const LevelGeom g = geom(c, level);
  mq_status st;
  if ((st = grow(c, c->Y, g.s * sizeof(double))) != MQ_OK) return st;
  MQ_CUDA(c, cudaMemcpyAsync(c->Y.p, y, g.s * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->stats = mq_stats{};
  if ((st = run_samples(c, g, 1, 1, 1, u_H != nullptr)) != MQ_OK) return st;
  double o[4];
  MQ_CUDA(c, cudaMemcpyAsync(o, c->out.p, sizeof o, cudaMemcpyDeviceToHost, c->stream));
  if (u_H)
    MQ_CUDA(c, cudaMemcpyAsync(u_H, c->uout.p, (size_t)(g.nc - 1) * (g.nc - 1) * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  if ((st = timing(c, -1)) != MQ_OK) return st;
  if ((st = check_tc_error(c)) != MQ_OK) return st;
  int fl = 0;
  c->last_B = 1;
  if ((st = collect_stats(c, 1, &fl)) != MQ_OK) return st;
  if (lam_H) *lam_H = o[0];
  if (lam_h) *lam_h = o[1];
  if (lam_hm1) *lam_hm1 = o[2];
  return flags_status(c, fl);
}

mq_status mq_get_stats(mq_ctx* c, void* stats, size_t bytes) {
  if (!c || !stats) return MQ_EINVAL;
  if (c->last_B) {
    // iteration counters of the last pass (the sample count stays that of the whole call)
    const uint64_t samples = c->stats.samples;
    int fl = 0;
    mq_status st = collect_stats(c, c->last_B, &fl);
    if (st != MQ_OK) return st;
    c->stats.samples = samples;
  }
  std::memcpy(stats, &c->stats, std::min(bytes, sizeof(mq_stats)));
  return MQ_OK;
}

mq_status mq_cbc_lattice(uint32_t N, int32_t s, double decay, uint32_t* z_out) {
  if (N < 2 || s < 1 || !z_out || !std::isfinite(decay)) return MQ_EINVAL;
  std::vector<uint32_t> cand;
  for (uint32_t q = 1; q <= N / 2; ++q)
    if (std::gcd(q, N) == 1) cand.push_back(q);
  if (cand.empty()) cand.push_back(1);
  std::vector<double> prod(N, 1.0), e2(cand.size());
  auto b2 = [](double x) { return x * x - x + 1.0 / 6.0; };
  for (int j = 0; j < s; ++j) {
    const double gam = std::pow((double)(j + 1), -decay);
    for (size_t ci = 0; ci < cand.size(); ++ci) {
      const uint64_t zc = cand[ci];
      double acc = 0.0;
      for (uint32_t k = 0; k < N; ++k) acc += prod[k] * (1.0 + gam * b2((double)((k * zc) % N) / (double)N));
      e2[ci] = -1.0 + acc / N;
    }
    const double best = *std::min_element(e2.begin(), e2.end());
    size_t pick = 0;
    while (!(e2[pick] <= best + 1e-12)) ++pick;
    z_out[j] = cand[pick];
    const uint64_t zc = cand[pick];
    for (uint32_t k = 0; k < N; ++k) prod[k] *= 1.0 + gam * b2((double)((k * zc) % N) / (double)N);
  }
  return MQ_OK;
}

mq_status mq_cbc_embedded_lattice(int32_t m_min, int32_t m_max, int32_t s, double decay, uint32_t* z_out) {
  if (m_min < 0 || m_max < m_min || m_max > 24 || s < 1 || !z_out || !std::isfinite(decay)) return MQ_EINVAL;
  const uint32_t Nmax = 1u << m_max;
  std::vector<uint32_t> cand;
  for (uint32_t q = 1; q < std::max<uint32_t>(2, Nmax / 2); q += 2) cand.push_back(q);
  const int nm = m_max - m_min + 1;
  // excess[i][k] = prod over the chosen components of (1 + gamma_j B2({k z_j / N})) - 1, N = 2^(m_min+i):
  // the squared error is its mean, formed without cancelling against the constant 1
  std::vector<std::vector<double>> excess(nm), tab(nm);
  for (int i = 0; i < nm; ++i) {
    const uint32_t N = 1u << (m_min + i);
    excess[i].assign(N, 0.0);
    tab[i].resize(N);
    for (uint32_t k = 0; k < N; ++k) {
      const double x = (double)k / (double)N;
      tab[i][k] = x * x - x + 1.0 / 6.0;  // Bernoulli polynomial B2
    }
  }
  std::vector<double> worst(cand.size()), e2(cand.size());
  for (int j = 0; j < s; ++j) {
    const double gam = std::pow((double)(j + 1), -decay);
    std::fill(worst.begin(), worst.end(), 0.0);
    for (int i = 0; i < nm; ++i) {
      const uint32_t N = 1u << (m_min + i), mask = N - 1;
      const double* q = excess[i].data();
      const double* tb = tab[i].data();
      for (size_t ci = 0; ci < cand.size(); ++ci) {
        const uint64_t zc = cand[ci];
        const double acc = pairwise_sum(0, N, [&](uint32_t k) {
          const double a = gam * tb[(uint32_t)(((uint64_t)k * zc) & mask)];
          return q[k] + a * (1.0 + q[k]);
        });
        e2[ci] = acc / N;
      }
      const double emin = *std::min_element(e2.begin(), e2.end());
      for (size_t ci = 0; ci < cand.size(); ++ci) worst[ci] = std::max(worst[ci], e2[ci] / emin);
    }
    const double best = *std::min_element(worst.begin(), worst.end());
    size_t pick = 0;
    while (!(worst[pick] <= best * (1.0 + 1e-6))) ++pick;  // ties within a relative 1e-6: smallest candidate
    z_out[j] = cand[pick];
    for (int i = 0; i < nm; ++i) {
      const uint32_t N = 1u << (m_min + i), mask = N - 1;
      for (uint32_t k = 0; k < N; ++k) {
        const double a = gam * tab[i][(uint32_t)(((uint64_t)k * cand[pick]) & mask)];
        excess[i][k] += a * (1.0 + excess[i][k]);
      }
    }
  }
  return MQ_OK;
}

mq_status mq_lattice_points_device(mq_ctx* c, int32_t level, uint32_t k0, uint32_t k1, double* d_Y) {
  if (!c) return MQ_EINVAL;
  mq_status st = check_level_ready(c, level);
  if (st != MQ_OK) return st;
  const mq_level& lv = c->levels[level];
  if (k1 < k0 || k1 > lv.N || !d_Y) return fail(c, MQ_EINVAL, "bad point range or output");
  MQ_CUDA(c, cudaSetDevice(c->device));
  const int mb = c->mbits[level];
  MQ_LAUNCH(c, mq::launch_lattice_points(c->d_z[level], mb ? (1u << mb) : lv.N, c->d_delta[level], lv.R, lv.s, k0,
                                       (int)(k1 - k0), mb, d_Y, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return MQ_OK;
}

mq_status mq_coefficients_device(mq_ctx* c, int32_t n, int32_t s, const double* d_Y, int32_t B, int32_t ldy,
                                 double* d_a) {
  if (!c) return MQ_EINVAL;
  if (!c->coef_set) return fail(c, MQ_ESTATE, "coefficient not set");
  if (!pow2(n) || n < 2 || n > 4096 || s < 0 || s > c->s_max || B < 0 || ldy < s || (!d_Y && B * s) || (!d_a && B))
    return fail(c, MQ_EINVAL, "bad coefficient arguments");
  MQ_CUDA(c, cudaSetDevice(c->device));
  mq_status st = reset_tc_error(c);
  if (st != MQ_OK) return st;
  st = coefficients(c, n, s, d_Y, B, ldy, d_a);
  if (st != MQ_OK) return st;
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_tc_error(c);
}

mq_status mq_reaction_coefficients_device(mq_ctx* c, int32_t n, int32_t s, const double* d_Y, int32_t B, int32_t ldy,
                                          double* d_b) {
  if (!c) return MQ_EINVAL;
  if (!c->coef_set) return fail(c, MQ_ESTATE, "coefficient not set");
  if (c->family != 2) return fail(c, MQ_ESTATE, "the coefficient family has no reaction term");
  if (!pow2(n) || n < 2 || n > 4096 || s < 0 || s > c->s_max || B < 0 || ldy < s || (!d_Y && B * s) || (!d_b && B))
    return fail(c, MQ_EINVAL, "bad coefficient arguments");
  MQ_CUDA(c, cudaSetDevice(c->device));
  mq_status st = reset_tc_error(c);
  if (st != MQ_OK) return st;
  st = coefficients(c, n, s, d_Y, B, ldy, d_b, 1);
  if (st != MQ_OK) return st;
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_tc_error(c);
}

mq_status mq_apply_operator_device(mq_ctx* c, int32_t n, int32_t B, const double* d_a, int32_t which, double sigma,
                                   const double* d_x, double* d_y) {
  if (!c) return MQ_EINVAL;
  if (!pow2(n) || n < 2 || n > 4096 || B < 0 || which < 0 || which > 4 || (B && (!d_a || !d_x || !d_y)))
    return fail(c, MQ_EINVAL, "bad operator arguments");
  MQ_CUDA(c, cudaSetDevice(c->device));
  mq_status st = grow(c, c->misc, (size_t)B * 4 * (n + 1) * (n + 1) * sizeof(double));
  if (st != MQ_OK) return st;
  MQ_LAUNCH(c, mq::launch_apply_operator(n, B, d_a, which, sigma, d_x, d_y, (double*)c->misc.p, c->stream));
  MQ_CUDA(c, cudaStreamSynchronize(c->stream));
  return MQ_OK;
}

}  // extern "C"
