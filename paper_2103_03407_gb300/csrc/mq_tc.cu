// Centroid coefficients a = a0 + Y Psi on the 5th-generation tensor cores (tcgen05, sm_103a),
// accurate to FP64 rounding of the terms.
//
// The dense contraction of eq. coeff (samples x truncation) x (truncation x triangles) is split
// into exact BF16 integer slices (an Ozaki-type splitting):
//   y   in [-1/2, 1/2):  y   = sum_{p<7} Y_p 2^{-8(p+1)}  + r,  |r| <= 2^-57,  Y_p integers in [-128, 128]
//   psi in [-1, 1]:      psi = sum_{q<7} P_q 2^{-7-8q}    + r,  |r| <= 2^-64,  P_q integers in [-128, 128]
// Integers of magnitude <= 256 are exact in BF16, products of two are exact in the FP32
// accumulator, and every accumulated sum stays an integer below 2^24 (K is processed in chunks of
// at most 128 and the products are grouped by g = p + q, at most 7 per group: 7 * 128 * 2^14 <
// 2^24), so each group sum
//   S_g = sum_{p+q=g} sum_{j in chunk} Y_p[b][j] P_q[t][j]
// is EXACT whatever the accumulation order of the tensor core.  Groups g <= 6 are kept (28 slice
// products): a = a0 + sum_chunks sum_g 2^{-15-8g} S_g, folded into FP64 registers after every
// chunk.  Dropped products (g >= 7) and slice remainders are below 2^-56 per term: the result
// matches an FP64 GEMM to a few units of FP64 rounding.
//
// Kernel: one CTA (4 warps) computes a 128-sample x 32-triangle tile.  Per 16-wide K step the
// threads stage the seven A slices (128 x 16) and seven B slices (32 x 16) into shared memory in
// the canonical no-swizzle K-major layout (8 x 16-byte core matrices), and one elected thread
// issues the 28 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 32, K = 16) into seven
// TMEM accumulators (32 columns each), then commits to an mbarrier.  After a chunk the
// accumulators are read with tcgen05.ld (each warp its 32 lanes) and folded in FP64.  Every wait
// is bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mq_internal.h"

namespace mq {
namespace {

constexpr int kSlices = 7;   // slices per operand
constexpr int kGroups = 7;   // kept groups g = p + q
constexpr int kTM = 128;     // samples per tile (TMEM lanes)
constexpr int kTN = 32;      // triangles per tile
constexpr int kTK = 16;      // K per MMA
constexpr int kChunk = 128;  // K per exact accumulation chunk
constexpr int kTmemCols = 256;
constexpr long kSpinLimit = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows x 16 bytes;
// lbo = byte distance between core matrices adjacent in K, sbo = between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor core
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 32
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t addr = smem_u32(mbar);
  for (long i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------------------------
// slicing.  out layout [slice][rows_pad][kpad] (K contiguous); zero padding beyond rows / k.
__global__ void k_slice_rows(const double* __restrict__ src, int rows, int k, size_t row_stride, size_t col_stride,
                             double scale, int rows_pad, int kpad, __nv_bfloat16* __restrict__ out) {
  const size_t tot = (size_t)rows_pad * kpad;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / kpad), j = (int)(q % kpad);
    double v = (r < rows && j < k) ? src[(size_t)r * row_stride + (size_t)j * col_stride] * scale : 0.0;
#pragma unroll
    for (int p = 0; p < kSlices; ++p) {
      const double s = rint(v);
      out[(size_t)p * tot + q] = __float2bfloat16_rn((float)s);
      v = (v - s) * 256.0;
    }
  }
}

struct alignas(1024) TcSmem {
  __nv_bfloat16 a[kSlices][kTM * kTK];  // 4 KB per slice
  __nv_bfloat16 b[kSlices][kTN * kTK];  // 1 KB per slice
  uint64_t mbar;
  uint32_t tmem_base;
  int err;
};

// a[b][t] = a0 + sum_j y[b][j] psi[j][t], b < B, t < nT; slices [7][Bpad][Kpad] and [7][nTpad][ldp]
__global__ void __launch_bounds__(128) k_coef_tc(const __nv_bfloat16* __restrict__ ys, const __nv_bfloat16* __restrict__ ps,
                                                 int B, int Bpad, int nT, int nTpad, int Kpad, int ldp, double a0,
                                                 double* __restrict__ out, int* __restrict__ err_flag) {
  extern __shared__ __align__(1024) char dyn[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int t0 = blockIdx.x * kTN, b0 = blockIdx.y * kTM;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&S.mbar, 1);
    S.err = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const uint32_t idesc = instr_desc();
  double acc[kTN];
#pragma unroll
  for (int i = 0; i < kTN; ++i) acc[i] = 0.0;
  uint32_t phase = 0;
  bool ok = true;
  const size_t ysz = (size_t)Bpad * Kpad, psz = (size_t)nTpad * ldp;
  for (int kc = 0; kc < Kpad && ok; kc += kChunk) {
    const int kend = min(Kpad, kc + kChunk);
    for (int k0 = kc; k0 < kend; k0 += kTK) {
      // stage A: row tid, 16 K values = two 16-byte core-matrix rows per slice
      {
        const int r = tid;
        const uint32_t off = (uint32_t)((r >> 3) * 256 + (r & 7) * 16);
#pragma unroll
        for (int p = 0; p < kSlices; ++p) {
          const uint4* src = reinterpret_cast<const uint4*>(ys + p * ysz + (size_t)(b0 + r) * Kpad + k0);
          char* dst = reinterpret_cast<char*>(S.a[p]);
          *reinterpret_cast<uint4*>(dst + off) = src[0];
          *reinterpret_cast<uint4*>(dst + off + 128) = src[1];
        }
      }
      // stage B: slices x 32 rows x 2 halves, 16 bytes each
#pragma unroll
      for (int c = tid; c < kSlices * kTN * 2; c += 128) {
        const int p = c / (kTN * 2), rr = (c >> 1) % kTN, h = c & 1;
        const uint4* src = reinterpret_cast<const uint4*>(ps + p * psz + (size_t)(t0 + rr) * ldp + k0);
        char* dst = reinterpret_cast<char*>(S.b[p]);
        *reinterpret_cast<uint4*>(dst + (rr >> 3) * 256 + (rr & 7) * 16 + h * 128) = src[h];
      }
      async_proxy_fence();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int p = 0; p < kSlices; ++p)
#pragma unroll
          for (int q = 0; q < kSlices; ++q) {
            const int g = p + q;
            if (g >= kGroups) continue;
            const uint64_t ad = smem_desc(smem_u32(S.a[p]), 128, 256);
            const uint64_t bd = smem_desc(smem_u32(S.b[q]), 128, 256);
            // the first product of each group in a chunk overwrites the accumulator
            const uint32_t accum = (k0 != kc) || (p > (g < kSlices ? 0 : g - kSlices + 1));
            mma_bf16(tmem + (uint32_t)(g * kTN), ad, bd, idesc, accum);
          }
        mma_commit(&S.mbar);
      }
      // the shared tiles are reused by the next step: wait for the MMAs that read them
      if (!mbar_wait(&S.mbar, phase)) {
        ok = false;
        if (tid == 0) S.err = 1;
      }
      phase ^= 1;
      tc_fence_after();
      __syncthreads();
      if (!ok) break;
    }
    if (!ok) break;
    // fold the exact group sums of this chunk: they are integers below 2^24, so the combination
    // sum_g S_g 2^{8(6-g)} is formed exactly in two 64-bit integers (groups 0-3 and 4-6) and
    // rounded once to FP64 -- three FP64 operations per output instead of two per group
    long long hi[kTN], lo[kTN];
#pragma unroll
    for (int i = 0; i < kTN; ++i) hi[i] = lo[i] = 0;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * kTN), v);
#pragma unroll
      for (int i = 0; i < kTN; ++i) {
        const long long s = (long long)__float2int_rn(v[i]);
        if (g < 4) hi[i] = hi[i] * 256 + s;
        else lo[i] = lo[i] * 256 + s;
      }
    }
    // value of the chunk = (hi 2^24 + lo) 2^{-15-48}; hi < 2^56 and lo < 2^40 in magnitude
#pragma unroll
    for (int i = 0; i < kTN; ++i) acc[i] += fma((double)hi[i], 0x1p-39, (double)lo[i] * 0x1p-63);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  const int b = b0 + tid;
  if (ok && b < B) {
    double* o = out + (size_t)b * nT;
#pragma unroll
    for (int i = 0; i < kTN; ++i)
      if (t0 + i < nT) o[t0 + i] = a0 + acc[i];
  }
  if (tid == 0 && S.err) {
    atomicOr(err_flag, 1);
    mbar_wait(&S.mbar, phase ^ 1);  // a timed-out wait: give the MMAs in flight one more bounded wait
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

int grid1(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

}  // namespace

size_t tc_slices_bytes(int rows, int k) {
  const size_t rp = ((size_t)rows + 127) / 128 * 128, kp = ((size_t)k + 15) / 16 * 16;
  return (size_t)kSlices * rp * kp * sizeof(__nv_bfloat16);
}

int tc_pad_rows(int rows) { return (rows + 127) / 128 * 128; }
int tc_pad_k(int k) { return (k + 15) / 16 * 16; }

cudaError_t launch_psi_slices(const double* d_psi, int s_rows, int nT, void* d_out, cudaStream_t st) {
  // psi is [s_rows][nT] (row = term j): the slices are [7][nT_pad][K_pad] with K contiguous
  const int rp = tc_pad_rows(nT), kp = tc_pad_k(s_rows);
  k_slice_rows<<<grid1((size_t)rp * kp), 256, 0, st>>>(d_psi, nT, s_rows, 1, (size_t)nT, 128.0, rp, kp,
                                                      (__nv_bfloat16*)d_out);
  return cudaGetLastError();
}

cudaError_t launch_y_slices(const double* d_Y, int B, int ldy, int k, int kpad, void* d_out, cudaStream_t st) {
  const int rp = tc_pad_rows(B);
  k_slice_rows<<<grid1((size_t)rp * kpad), 256, 0, st>>>(d_Y, B, k, (size_t)ldy, 1, 256.0, rp, kpad,
                                                        (__nv_bfloat16*)d_out);
  return cudaGetLastError();
}

// a[B][nT] = a0 + Y psi from slices: y slices [7][Bpad][kpad] built for K = kpad columns, psi
// slices [7][nTpad][kpad_psi] (only the first kpad columns are read)
cudaError_t launch_coef_tc(const void* d_yslices, int B, int kpad, const void* d_pslices, int nT, int kpad_psi,
                           double a0, double* d_a, int* d_err, cudaStream_t st) {
  if (B == 0 || nT == 0) return cudaSuccess;
  if (kpad > kpad_psi || kpad % kTK) return cudaErrorInvalidValue;
  const int Bp = tc_pad_rows(B), nTp = tc_pad_rows(nT);
  const size_t smem = sizeof(TcSmem) + 1024 + 64 * 1024;  // extra space keeps at most two CTAs per SM
  cudaError_t e = cudaFuncSetAttribute(k_coef_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(nTp / kTN, Bp / kTM);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  k_coef_tc<<<grid, 128, smem, st>>>((const __nv_bfloat16*)d_yslices, (const __nv_bfloat16*)d_pslices, B, Bp, nT, nTp,
                                     kpad, kpad_psi, a0, d_a, d_err);
  return cudaGetLastError();
}

}  // namespace mq
