// Centroid coefficients a = a0 + Y Psi on the 5th-generation tensor cores (tcgen05, sm_103a),
// accurate to FP64 rounding of the terms.
//
// The dense contraction of eq. coeff (samples x truncation) x (truncation x triangles) is split
// into exact BF16 integer slices (an Ozaki-type splitting):
//   y   in [-1/2, 1/2):  y   = sum_{p<7} Y_p 2^{-8(p+1)}  + r,  |r| <= 2^-57,  Y_p integers in [-128, 128]
//   psi in [-1, 1]:      psi = sum_{q<7} P_q 2^{-7-8q}    + r,  |r| <= 2^-64,  P_q integers in [-128, 128]
// (a table is scaled by 2^e first, e chosen from its largest term factor so that |2^e psi| <= 1
// with the most bits kept; the result is scaled back by the exact factor 2^-e)
// Integers of magnitude <= 256 are exact in BF16, products of two are exact in the FP32
// accumulator, and every accumulated sum stays an integer below 2^24 (K is processed in chunks of
// at most 128 and the products are grouped by g = p + q, at most 7 per group: 7 * 128 * 2^14 <
// 2^24), so each group sum
//   S_g = sum_{p+q=g} sum_{j in chunk} Y_p[b][j] P_q[t][j]
// is EXACT whatever the accumulation order of the tensor core.  Groups g <= 6 are kept (28 slice
// products): a = a0 + sum_chunks sum_g 2^{-15-8g} S_g, the group sums of a chunk combined exactly
// in 64-bit integers.  A contraction of one chunk (K <= 128: the separable stage, short truncations)
// is then rounded once to FP64 in integer arithmetic; longer ones add their chunks in FP64
// registers.  Dropped products (g >= 7) and slice remainders are below 2^-56 per term: the result
// matches an FP64 GEMM to a few units of FP64 rounding.
//
// Kernel (persistent, one CTA of 8 warps per SM): each CTA walks 128-sample x 64-triangle output
// tiles.  Per 16-wide K step the tensor memory accelerator loads the seven A slices (128 x 16) and
// the seven B slices (64 x 16) into one of four shared-memory stages (slices are stored K-blocked,
// [slice][K/8][row][8], so one 4-D box lands directly in the canonical no-swizzle K-major layout of
// 8 x 16-byte core matrices) and signals the stage's mbarrier with the transferred byte count.  One
// elected thread waits for a stage, issues the 28 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
// M = 128, N = 64, K = 16) into seven TMEM accumulators (64 columns each), commits them to the
// stage's "empty" mbarrier and refills the stage used one step earlier, so loads run up to four
// steps ahead of the tensor cores.  After every 128-wide K chunk the eight warps read the
// accumulators with tcgen05.ld (warp w: TMEM lanes 32 (w mod 4).., columns 32 (w div 4)..) and fold
// them exactly (integer group sums, one rounding per chunk).  Every wait is bounded; a timeout sets an error word, stops the
// issuing of new work, drains what is in flight and frees the tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "mq_internal.h"

namespace mq {
namespace {

constexpr int kSlices = 7;   // slices per operand
constexpr int kGroups = 7;   // kept groups g = p + q
constexpr int kTM = 128;     // samples per tile (TMEM lanes)
constexpr int kTN = 64;      // triangles per tile
constexpr int kTK = 16;      // K per MMA (one pipeline step)
constexpr int kChunk = 128;  // K per exact accumulation chunk
constexpr int kStepsPerChunk = kChunk / kTK;
constexpr int kStages = 5;   // shared-memory pipeline depth (5 x 42 KB)
constexpr int kTcThreads = 256;
constexpr int kTmemCols = 512;  // 7 groups x 64 columns = 448 used
constexpr uint32_t kABytes = kSlices * kTM * kTK * 2;  // 28 KB per stage
constexpr uint32_t kBBytes = kSlices * kTN * kTK * 2;  // 14 KB per stage
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

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 64
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

// arrive once and expect `bytes` of asynchronous (TMA) transfers on the barrier's current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
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

// 4-D tiled TMA load of one box into shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane, without waiting: the registers are valid
// only after tmem_wait on them (several loads can then share one wait)
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// waits for this thread's outstanding TMEM loads; the registers are passed through so that no use
// of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// ---------------------------------------------------------------------------------------------
// slicing.  out layout [slice][kpad / 8][rows_pad][8] (blocks of eight K values per row, the row
// blocks back to back): a TMA box of 8 x rows x 2 x 7 is then one K step of all slices, in the
// core-matrix layout the MMA reads.  Zero padding beyond rows / k.
__global__ void k_slice_rows(const double* __restrict__ src, int rows, int k, size_t row_stride, size_t col_stride,
                             double scale, int rows_pad, int kpad, __nv_bfloat16* __restrict__ out) {
  const size_t tot = (size_t)rows_pad * kpad;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(q & 7);
    const size_t rb = q >> 3;  // jb * rows_pad + r
    const int r = (int)(rb % rows_pad), j = (int)(rb / rows_pad) * 8 + e;
    double v = (r < rows && j < k) ? src[(size_t)r * row_stride + (size_t)j * col_stride] * scale : 0.0;
#pragma unroll
    for (int p = 0; p < kSlices; ++p) {
      const double s = rint(v);
      out[(size_t)p * tot + q] = __float2bfloat16_rn((float)s);
      v = (v - s) * 256.0;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Separable evaluation (families whose terms are c_t sin(pi k1_t x1) sin(pi k2_t x2) with few
// distinct k1, like the workload family, where k1 <= ~2 sqrt(s)).  On one plane of triangles
// (lower or upper: the centroid abscissa x_i depends only on the cell column i, the ordinate y_j
// only on the cell row j)
//     a[b][j][i] = a0 + sum_{k1} T[b][j][k1] sin(pi k1 x_i),
//     T[b][j][k1] = sum_{t < K, k1_t = k1} Y[b][t] c_t sin(pi k2_t y_j),
// the same sum as eq. coeff_s grouped by k1.  Stage 1 forms T in FP64 on the CUDA cores (B n K
// fused multiply-adds per plane) and writes its exact BF16 slices; stage 2 is the tensor-core
// kernel below with rows (b, j), columns i and K = the padded count of k1 values: 2 B n^2 K1
// products per plane instead of 2 B n^2 K.

// centroid numerators over 3n: abscissa of column i, ordinate of row j, per plane
__device__ __forceinline__ int cx_num(int i, int plane) { return 3 * i + (plane == 0 ? 2 : 1); }
__device__ __forceinline__ int cy_num(int j, int plane) { return 3 * j + (plane == 0 ? 1 : 2); }

// syt[k][j] = sin(pi k y_j), k = 0..kmax, j < n (plane `plane`)
__global__ void k_sep_syt(int n, int plane, int kmax, double* __restrict__ syt) {
  const size_t tot = (size_t)(kmax + 1) * n;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / n), j = (int)(q % n);
    syt[q] = sinpi((double)k * (double)cy_num(j, plane) / (double)(3 * n));
  }
}

// sx[i][e] = sin(pi (e+1) x_i) for e + 1 <= k1max, 0 beyond (kpad columns)
__global__ void k_sep_sx(int n, int plane, int k1max, int kpad, double* __restrict__ sx) {
  const size_t tot = (size_t)n * kpad;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / kpad), e = (int)(q % kpad);
    sx[q] = e + 1 <= k1max ? sinpi((double)(e + 1) * (double)cx_num(i, plane) / (double)(3 * n)) : 0.0;
  }
}

// yc[b][t] = Y[b][t] c_t for t < K: the products stage 1 sums, formed once per (sample, term)
// instead of once per (mesh row, term) -- the same roundings, so stage 1 is bit-identical
__global__ void k_sep_yc(const double* __restrict__ Y, int ldy, int B, int K, const double* __restrict__ cj,
                         double* __restrict__ yc) {
  const size_t tot = (size_t)B * K;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / K), t = (int)(q % K);
    yc[q] = Y[(size_t)b * ldy + t] * cj[t];
  }
}

// Stage 1: T[m = b n + j][k1 - 1] for one plane, written as the 7 BF16 slices of scale * T in the
// layout of k_slice_rows ([7][kpad/8][rows_pad][8]); one thread per (row, group of 8 k1 values).
// The terms of each k1 are listed in increasing t: tlist[k1start[k1] .. k1start[k1 + 1]).  The
// slices are the balanced base-256 digits of W = scale T 2^48 rounded to an integer (|W| <= 2^55):
// W = sum_p d_p 2^{8(6-p)}, |d_p| <= 128, formed on the integer units -- the same representation
// error bound (half a unit of the last digit) as digit-by-digit rounding in FP64.
__global__ void k_sep_stage1(const double* __restrict__ yc, int B, int n, int plane, int K, int kpad,
                             const int* __restrict__ k1start, const int* __restrict__ tlist,
                             const int* __restrict__ tk2, const double* __restrict__ syt,
                             double scale, int rows_pad, __nv_bfloat16* __restrict__ out) {
  (void)plane;
  const size_t tot = (size_t)rows_pad * (kpad / 8);
  const size_t sstride = (size_t)rows_pad * kpad;
  const int rows = B * n;
  const double s48 = scale * 281474976710656.0;  // scale 2^48 (a power of two)
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(q % rows_pad), kg = (int)(q / rows_pad);
    __align__(16) __nv_bfloat16 sl[kSlices][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      double v = 0.0;
      if (m < rows) {
        const int b = m / n, j = m % n, k1 = kg * 8 + e + 1;
        const double* yb = yc + (size_t)b * K;
        for (int idx = k1start[k1]; idx < k1start[k1 + 1]; ++idx) {
          const int t = tlist[idx];
          if (t >= K) break;
          v = fma(yb[t], syt[(size_t)tk2[t] * n + j], v);
        }
      }
      long long w = __double2ll_rn(v * s48);
#pragma unroll
      for (int p = 0; p < kSlices - 1; ++p) {
        const int sh = 8 * (kSlices - 1 - p);
        const long long d = (w + (1LL << (sh - 1))) >> sh;  // nearest, |d| <= 128
        w -= d << sh;
        sl[p][e] = __float2bfloat16_rn((float)(int)d);
      }
      sl[kSlices - 1][e] = __float2bfloat16_rn((float)(int)w);
    }
#pragma unroll
    for (int p = 0; p < kSlices; ++p)
      *reinterpret_cast<uint4*>(out + (size_t)p * sstride + ((size_t)kg * rows_pad + m) * 8) =
          *reinterpret_cast<const uint4*>(sl[p]);
  }
}

// (hi 2^24 + lo) 2^e rounded once to the nearest double (ties to even), in integer arithmetic:
// the exact sum of a chunk's group sums, |hi| < 2^56, |lo| < 2^40.  GB300 issues FP64 at 1/64 of
// the FP32 rate; the conversions and the fused multiply-add of the FP64 fold cost more issue time
// than this on the integer units.  The result is finite and normal for every e the tables use.
__device__ __forceinline__ double exact_fold(long long hi, long long lo, int e) {
  const __int128 v = ((__int128)hi << 24) + (__int128)lo;
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
  const int lz = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);
  m <<= lz;  // leading one at bit 127
  const unsigned long long top = (unsigned long long)(m >> 64), rest = (unsigned long long)m;
  unsigned long long mant = top >> 11;  // 53 bits
  const unsigned long long rb = top & 0x7FFull;  // the next 11 bits; rest holds the ones below
  mant += (rb > 0x400ull) || (rb == 0x400ull && (rest != 0ull || (mant & 1ull)));
  int ex = 127 - lz + e;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                  (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

struct alignas(1024) TcSmem {
  __nv_bfloat16 a[kStages][kSlices * kTM * kTK];  // [slice][K half][128 rows][8]
  __nv_bfloat16 b[kStages][kSlices * kTN * kTK];  // [slice][K half][64 rows][8]
  uint64_t full[kStages];   // TMA bytes of a stage landed
  uint64_t empty[kStages];  // the MMAs that read a stage completed
  uint64_t accf;            // the MMAs of a K chunk completed (accumulators readable)
  uint32_t tmem_base;
  int err;
};

// Output placement: element (row b, column t) goes to out[row_off(b) + t] with row_off(b) = b nT,
// or, with mdiv > 0, (b / mdiv) m_hi + (b mod mdiv) m_lo (rows that index (sample, mesh row)
// pairs of a coefficient field).  Rows come in tiles of 128, columns in tiles of 64.
struct TcOut {
  double* out;
  int mdiv;
  long long m_hi, m_lo;
  int cols_fast;  // tile order: 0 row tiles fastest (tiles sharing a column tile run together), 1 columns
};

// a[b][t] = a0 + sum_j y[b][j] psi[j][t], b < B, t < nT (with base: base[t] in place of a0).
// Tiles: tm = tile mod ntm (128 samples), tn = tile div ntm (64 triangles), or the transposed
// order; CTA c takes tiles c, c + grid, ...  Kpad: K of the Y slices.
__global__ void __launch_bounds__(kTcThreads, 1)
    k_coef_tc(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmP, int B, int nT, int Kpad,
              int ntm, int ntiles, double a0, TcOut O, int* __restrict__ err_flag, const double* __restrict__ base,
              int pexp) {
  double* __restrict__ out = O.out;
  const int ntn = ntiles / ntm;
  auto coords = [&](int tile, int& tm, int& tn) {
    if (O.cols_fast) {
      tm = tile / ntn;
      tn = tile % ntn;
    } else {
      tm = tile % ntm;
      tn = tile / ntm;
    }
  };
  extern __shared__ __align__(1024) char dyn[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = Kpad / kTK;  // K steps per tile
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t U = (uint32_t)my_tiles * (uint32_t)T;  // K steps of this CTA
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    mbar_init(&S.accf, 1);
    S.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const uint32_t idesc = instr_desc();
  // producer / issuer state (thread 0 only)
  uint32_t u_load = 0;     // K steps whose loads were issued
  uint32_t u_done = 0;     // K steps whose loads were consumed
  uint32_t commits = 0;    // K steps whose MMAs were committed
  uint32_t chunks = 0;     // accumulator commits (parity of accf)
  auto issue_load = [&](uint32_t u) {
    const int ti = (int)(u / (uint32_t)T), ks = (int)(u % (uint32_t)T);
    const int tile = (int)blockIdx.x + ti * (int)gridDim.x;
    int tm, tn;
    coords(tile, tm, tn);
    const int st = (int)(u % kStages);
    mbar_arrive_expect(&S.full[st], kABytes + kBBytes);
    tma_load4(S.a[st], &tmY, 0, tm * kTM, 2 * ks, 0, &S.full[st]);
    tma_load4(S.b[st], &tmP, 0, tn * kTN, 2 * ks, 0, &S.full[st]);
  };
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmY) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmP) : "memory");
    for (; u_load < U && u_load < (uint32_t)kStages; ++u_load) issue_load(u_load);
  }
  const int q4 = warp & 3, half = warp >> 2;  // TMEM lane quarter, column half
  bool ok = true;
  for (int ti = 0; ti < my_tiles && ok; ++ti) {
    const int tile = (int)blockIdx.x + ti * (int)gridDim.x;
    int tm, tn;
    coords(tile, tm, tn);
    // 2^-39 and 2^-63 of the fold, times the table's exact scale 2^-pexp
    const double chi = ldexp(1.0, -39 - pexp), clo = ldexp(1.0, -63 - pexp);
    const bool single = T <= kStepsPerChunk;
    double acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0;
    for (int kc = 0; kc < T && ok; kc += kStepsPerChunk) {
      const int kend = min(T, kc + kStepsPerChunk);
      if (tid == 0) {
        for (int ks = kc; ks < kend && !S.err; ++ks) {
          const uint32_t u = (uint32_t)ti * (uint32_t)T + (uint32_t)ks;
          const int st = (int)(u % kStages);
          if (!mbar_wait(&S.full[st], (u / kStages) & 1)) {
            S.err = 1;
            break;
          }
          u_done = u + 1;
          tc_fence_after();
          const uint32_t abase = smem_u32(S.a[st]), bbase = smem_u32(S.b[st]);
#pragma unroll
          for (int p = 0; p < kSlices; ++p) {
            const uint64_t ad = smem_desc(abase + p * (kTM * kTK * 2), kTM * 16, 128);
#pragma unroll
            for (int q = 0; q + p < kGroups; ++q) {
              const uint64_t bd = smem_desc(bbase + q * (kTN * kTK * 2), kTN * 16, 128);
              // the first product of each group (p = 0) in a chunk overwrites the accumulator
              mma_bf16(tmem + (uint32_t)((p + q) * kTN), ad, bd, idesc, (ks != kc || p > 0) ? 1u : 0u);
            }
          }
          mma_commit(&S.empty[st]);
          commits = u + 1;
          // refill the stage of the previous step once its MMAs are done (this step's MMAs are
          // queued behind them, so the tensor cores stay busy meanwhile)
          if (u >= 1 && u_load < U) {
            const uint32_t v = u - 1;
            if (!mbar_wait(&S.empty[v % kStages], (v / kStages) & 1)) {
              S.err = 1;
              break;
            }
            issue_load(u_load++);
          }
        }
        mma_commit(&S.accf);  // tracks every MMA issued so far, whether or not an error stopped us
      }
      __syncwarp();
      if (!mbar_wait(&S.accf, chunks & 1)) S.err = 1;
      ++chunks;
      tc_fence_after();
      __syncthreads();
      ok = S.err == 0;
      if (ok) {
        // fold the exact group sums of this chunk: integers below 2^24, combined exactly as
        // sum_g S_g 2^{8(6-g)} in two 64-bit integers (groups 0-3 and 4-6), then rounded once
#pragma unroll
        for (int sh = 0; sh < 2; ++sh) {
          const uint32_t tcol = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(half * 32 + sh * 16);
          long long hi[16], lo[16];
          {
            // groups 0-3: four loads in flight, one wait
            uint32_t r[4][16];
#pragma unroll
            for (int g = 0; g < 4; ++g) tmem_ld16_async(tcol + (uint32_t)(g * kTN), r[g]);
#pragma unroll
            for (int g = 0; g < 4; ++g) tmem_wait(r[g]);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              long long h = 0;
#pragma unroll
              for (int g = 0; g < 4; ++g) h = h * 256 + (long long)__float2int_rn(__uint_as_float(r[g][i]));
              hi[i] = h;
            }
          }
          {
            // groups 4-6
            uint32_t r[3][16];
#pragma unroll
            for (int g = 0; g < 3; ++g) tmem_ld16_async(tcol + (uint32_t)((4 + g) * kTN), r[g]);
#pragma unroll
            for (int g = 0; g < 3; ++g) tmem_wait(r[g]);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              long long l = 0;
#pragma unroll
              for (int g = 0; g < 3; ++g) l = l * 256 + (long long)__float2int_rn(__uint_as_float(r[g][i]));
              lo[i] = l;
            }
          }
          // value of the chunk = (hi 2^24 + lo) 2^{-15-48}; hi < 2^56 and lo < 2^40 in magnitude.  A
          // contraction of one chunk is rounded once in integer arithmetic; longer ones add the
          // chunks in FP64
          if (single) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[sh * 16 + i] = exact_fold(hi[i], lo[i], -63 - pexp);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[sh * 16 + i] += fma((double)hi[i], chi, (double)lo[i] * clo);
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // the accumulators may be overwritten by the next chunk
    }
    if (ok) {
      const int b = tm * kTM + q4 * 32 + lane;
      if (b < B) {
        double* o = out + (O.mdiv > 0 ? (size_t)(b / O.mdiv) * (size_t)O.m_hi + (size_t)(b % O.mdiv) * (size_t)O.m_lo
                                      : (size_t)b * nT);
        const int t0 = tn * kTN + half * 32;
        // t0 is even: pairs are 16-byte aligned whenever the row start is
        if (base) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (t0 + i < nT) o[t0 + i] = base[t0 + i] + acc[i];
        } else if (((uintptr_t)o & 15) == 0) {
#pragma unroll
          for (int i = 0; i < 32; i += 2)
            if (t0 + i < nT) *reinterpret_cast<double2*>(o + t0 + i) = make_double2(a0 + acc[i], a0 + acc[i + 1]);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (t0 + i < nT) o[t0 + i] = a0 + acc[i];
        }
      }
    }
  }
  if (tid == 0) {
    if (S.err) {
      atomicOr(err_flag, 1);
      // drain: loads issued but not consumed, and the last commit of every stage
      for (uint32_t u = u_done; u < u_load; ++u) mbar_wait(&S.full[u % kStages], (u / kStages) & 1);
    }
    for (uint32_t u = commits > kStages ? commits - kStages : 0; u < commits; ++u)
      mbar_wait(&S.empty[u % kStages], (u / kStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

int grid1(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

// cuTensorMapEncodeTiled through the runtime's driver entry points (no link-time dependency)
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)f;
  });
  return fn;
}

// tensor map of slices [7][kpad/8][rows_pad][8] (BF16), box 8 x box_rows x 2 x 7: one K step
cudaError_t slice_map(CUtensorMap* m, const void* base, int rows_pad, int kpad, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dim[4] = {8, (cuuint64_t)rows_pad, (cuuint64_t)(kpad / 8), (cuuint64_t)kSlices};
  const cuuint64_t stride[3] = {16, (cuuint64_t)rows_pad * 16, (cuuint64_t)rows_pad * 16 * (cuuint64_t)(kpad / 8)};
  const cuuint32_t box[4] = {8, (cuuint32_t)box_rows, 2, (cuuint32_t)kSlices};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dim, stride, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

size_t tc_slices_bytes(int rows, int k) {
  const size_t rp = ((size_t)rows + 127) / 128 * 128, kp = ((size_t)k + 15) / 16 * 16;
  return (size_t)kSlices * rp * kp * sizeof(__nv_bfloat16);
}

int tc_pad_rows(int rows) { return (rows + 127) / 128 * 128; }
int tc_pad_k(int k) { return (k + 15) / 16 * 16; }

cudaError_t launch_psi_slices(const double* d_psi, int s_rows, int nT, void* d_out, cudaStream_t st, int pexp) {
  // psi is [s_rows][nT] (row = term j): the slices are [7][K_pad/8][nT_pad][8] of 2^pexp psi
  const int rp = tc_pad_rows(nT), kp = tc_pad_k(s_rows);
  k_slice_rows<<<grid1((size_t)rp * kp), 256, 0, st>>>(d_psi, nT, s_rows, 1, (size_t)nT, std::ldexp(128.0, pexp), rp,
                                                      kp, (__nv_bfloat16*)d_out);
  return cudaGetLastError();
}

cudaError_t launch_y_slices(const double* d_Y, int B, int ldy, int k, int kpad, void* d_out, cudaStream_t st) {
  const int rp = tc_pad_rows(B);
  k_slice_rows<<<grid1((size_t)rp * kpad), 256, 0, st>>>(d_Y, B, k, (size_t)ldy, 1, 256.0, rp, kpad,
                                                        (__nv_bfloat16*)d_out);
  return cudaGetLastError();
}

// a[B][nT] = a0 + Y psi from slices: y slices [7][kpad/8][Bpad][8] built for K = kpad columns, psi
// slices [7][kpad_psi/8][nTpad][8] (only the first kpad columns are read)
namespace {
cudaError_t coef_tc(const void* d_yslices, int B, int kpad, const void* d_pslices, int nT, int kpad_psi, double a0,
                    const TcOut& O, int* d_err, cudaStream_t st, const double* d_base, int pexp) {
  if (B == 0 || nT == 0) return cudaSuccess;
  if (kpad > kpad_psi || kpad % kTK || kpad <= 0) return cudaErrorInvalidValue;
  const int Bp = tc_pad_rows(B), nTp = tc_pad_rows(nT);
  CUtensorMap tmY, tmP;
  cudaError_t e = slice_map(&tmY, d_yslices, Bp, kpad, kTM);
  if (e != cudaSuccess) return e;
  // the psi slices hold kpad_psi columns; the map covers them all, the kernel reads kpad
  e = slice_map(&tmP, d_pslices, nTp, kpad_psi, kTN);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(TcSmem) + 1024;
  // raised once per device (never lowered), so the launch can also be captured into a graph
  if ((e = raise_smem_limit((const void*)k_coef_tc, (int)smem)) != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int ntm = Bp / kTM;
  const long ntiles = (long)ntm * (nTp / kTN);
  if (ntiles > 0x7fffffffL) return cudaErrorInvalidValue;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  k_coef_tc<<<grid, kTcThreads, smem, st>>>(tmY, tmP, B, nT, kpad, ntm, (int)ntiles, a0, O, d_err, d_base, pexp);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_coef_tc(const void* d_yslices, int B, int kpad, const void* d_pslices, int nT, int kpad_psi,
                           double a0, double* d_a, int* d_err, cudaStream_t st, const double* d_base, int pexp) {
  const TcOut O{d_a, 0, 0, 0, 0};
  return coef_tc(d_yslices, B, kpad, d_pslices, nT, kpad_psi, a0, O, d_err, st, d_base, pexp);
}

size_t sep_tables_bytes(int n, int k1pad, int k2max) {
  return 2 * (tc_slices_bytes(n, k1pad) + (size_t)(k2max + 1) * n * sizeof(double)) + 4 * 256;
}

cudaError_t launch_sep_tables(int n, int k1max, int k1pad, int k2max, double* d_work, void* d_tables, SepTables* t,
                              cudaStream_t st) {
  char* p = (char*)d_tables;
  auto take = [&](size_t bytes) {
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    char* r = p;
    p += bytes;
    return r;
  };
  t->k1pad = k1pad;
  for (int plane = 0; plane < 2; ++plane) {
    t->sx[plane] = take(tc_slices_bytes(n, k1pad));
    t->syt[plane] = (double*)take((size_t)(k2max + 1) * n * sizeof(double));
    k_sep_sx<<<grid1((size_t)n * k1pad), 256, 0, st>>>(n, plane, k1max, k1pad, d_work);
    const int rp = tc_pad_rows(n);
    k_slice_rows<<<grid1((size_t)rp * k1pad), 256, 0, st>>>(d_work, n, k1pad, (size_t)k1pad, 1, 128.0, rp, k1pad,
                                                           (__nv_bfloat16*)t->sx[plane]);
    k_sep_syt<<<grid1((size_t)(k2max + 1) * n), 256, 0, st>>>(n, plane, k2max, (double*)t->syt[plane]);
  }
  return cudaGetLastError();
}

size_t sep_scratch_bytes(int B, int n, int K, int k1pad) {
  return ((tc_slices_bytes(B * n, k1pad) + 255) & ~(size_t)255) + (size_t)B * K * sizeof(double);
}

cudaError_t launch_coef_sep(const double* d_Y, int ldy, int B, int K, int k1pad, const SepTerms& terms,
                            const SepTables& tab, int n, double a0, int ey, void* d_tslices, double* d_a, int* d_err,
                            cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  if (k1pad % kTK || k1pad <= 0 || k1pad > tab.k1pad || (long)B * n > 0x7fffffffL - 128) return cudaErrorInvalidValue;
  const int rows = B * n, rp = tc_pad_rows(rows);
  double* yc = (double*)((char*)d_tslices + ((tc_slices_bytes(rows, k1pad) + 255) & ~(size_t)255));
  k_sep_yc<<<grid1((size_t)B * K), 256, 0, st>>>(d_Y, ldy, B, K, terms.cj, yc);
  for (int plane = 0; plane < 2; ++plane) {
    k_sep_stage1<<<grid1((size_t)rp * (k1pad / 8)), 256, 0, st>>>(
        yc, B, n, plane, K, k1pad, terms.k1start, terms.tlist, terms.tk2, tab.syt[plane],
        std::ldexp(256.0, ey), rp, (__nv_bfloat16*)d_tslices);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // rows (b, j) of this plane land at a[b][plane][j][.]: b 2n^2 + plane n^2 + j n
    const TcOut O{d_a + (size_t)plane * n * n, n, 2LL * n * n, (long long)n, 1};
    if ((e = coef_tc(d_tslices, rows, k1pad, tab.sx[plane], n, tab.k1pad, a0, O, d_err, st, nullptr, ey)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace mq
