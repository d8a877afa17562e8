// Allocation-free variant of the per-sample two-grid launch.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being captured by
// someone else, plugins that live inside a host application with its own fixed memory pool,
// and real-time services that forbid allocation after start-up.  For them this file keeps the
// per-block workspace of the per-sample kernel in one file-scope device array of fixed size
// instead of a buffer from cudaMalloc, and takes every input and output from the caller.
//
// In host code the name of the array is only a host-side stand-in for the device symbol, not
// a device address: passing it to a kernel would fault (or, where the GPU can reach host
// memory, silently use the wrong memory).  The device address is therefore looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the first call made on
// that device, and cached.  The cache belongs to the device's primary context: after
// cudaDeviceReset (or anything else that destroys and recreates that context) the cached
// address is stale, so the cache is keyed by the context too and looked up again when the
// current context differs from the one the address was taken in.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/mlqmc_evp.h"
#include "mq_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the cached address belongs to

// Unique id of the current context (never reused by a later context), through the driver entry
// points the runtime hands out (no link-time dependency on the driver library); 0 if unavailable.
unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device (looked up once per device and
// context; with no context id available it is looked up on every call).
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> guard(g_lock);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" mq_status mq_twogrid_samples_noalloc(int32_t n_fine, int32_t n_coarse, int32_t n_prev, int32_t precision,
                                                int32_t B, const double* d_a_fine, const double* d_a_coarse,
                                                const double* d_a_prev, double tol_linear, double* d_out,
                                                int32_t* d_stat, int32_t* d_outer, void* cuda_stream) {
  if (B < 0 || !pow2(n_fine) || !pow2(n_coarse) || n_fine > 4096 || n_coarse > n_fine || n_fine % n_coarse)
    return MQ_EINVAL;
  if (n_prev != 0 && (!pow2(n_prev) || n_prev > n_fine || n_prev < n_coarse || n_prev % n_coarse)) return MQ_EINVAL;
  if (precision != MQ_PREC_FP64 && precision != MQ_PREC_MIXED) return MQ_EINVAL;
  if (!(tol_linear < 1.0)) return MQ_EINVAL;
  if (B == 0) return MQ_OK;
  if (!d_a_coarse || !d_out || !d_stat || !d_outer) return MQ_EINVAL;
  const int mixed = precision == MQ_PREC_MIXED;
  // A solve on the coarse mesh itself (n == n_coarse with a longer truncation) is nearly
  // singular -- the shift is an eigenvalue of a nearby operator -- so in mixed precision it runs
  // with an FP64 inner solve (mode 1), as in mq_eval_level; every other solve uses the inner
  // precision of the mode (mode 0).  The workspace is sized for the modes actually used.
  const int mode_f = (mixed && n_fine == n_coarse && d_a_fine) ? 1 : 0;
  const int mode_p = (mixed && n_prev == n_coarse && d_a_prev) ? 1 : 0;
  const size_t slab = mq::sample_slab_bytes(n_fine, n_coarse, n_prev, mixed, mode_f, mode_p);
  if (slab > kNoAllocScratchBytes) return MQ_EINVAL;  // one block's workspace exceeds the fixed array

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return MQ_ECUDA;
  void* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return MQ_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MQ_ECUDA;

  const int threads = n_fine <= 16 ? 128 : 256;
  int occ = mq::sample_occupancy(mixed, threads, 0);
  if (occ < 1) occ = 1;
  const long fit = (long)(kNoAllocScratchBytes / slab);
  const long blocks = std::max(1L, std::min<long>({(long)B, (long)sms * occ, fit}));
  const int chunk = (int)((B + blocks - 1) / blocks);

  mq::SampleLaunch p{};
  p.nf = n_fine;
  p.nc = n_coarse;
  p.np = n_prev;
  p.direct_f = d_a_fine == nullptr;
  p.direct_p = n_prev != 0 && d_a_prev == nullptr;
  p.R = 1;
  p.npts = B;
  p.chunk = chunk;
  p.a_f = d_a_fine;
  p.a_c = d_a_coarse;
  p.a_p = d_a_prev;
  p.out = d_out;
  p.stat = d_stat;
  p.outer = d_outer;
  p.u_out = nullptr;
  p.gscratch = (char*)scratch;
  p.slab_bytes = slab;
  p.use_smem = 0;
  p.tol_eig = 1e-12;
  p.max_eig_it = 200;
  p.tol_lin = tol_linear > 0 ? tol_linear : 1e-10;
  p.tol_inner = mixed ? 1e-5 : 0.1 * p.tol_lin;
  p.max_outer = mixed ? 10 : 4;
  p.max_inner_it = 500;
  p.nu = 2;
  p.omega = 0.8;
  p.mode_f = mode_f;
  p.mode_p = mode_p;
  const cudaError_t e = mq::launch_sample(p, mixed, (int)blocks, threads, 0, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? MQ_OK : MQ_ECUDA;
}
