// Tensor-core (tcgen05) GEMM for the reduced-precision contraction forms.
//
// C[b] = alpha * A[b] * B[b] + beta * C[b] with FP64 operand views (the same
// MatView / OutView as the FP64 kernel).  Operands are first packed into
// K-major, zero-padded buffers of the tensor-core input type.
//
// Exact-slice form BF16X6 (unbiased).  Each row r of A (and each column c of B) is
// scaled by 2^-e_r, e_r the binary exponent of its largest magnitude, and
// written as x 2^-e_r = 2^-7 s_1 + 2^-15 s_2 + 2^-23 s_3 + ..., each slice an
// integer |s_p| <= 128 obtained by rounding to nearest (exact in bf16).
// Slice products s_i t_j are integers below 2^14; the tensor cores sum the
// products of equal weight 2^-(14 + 8 g), g = i + j - 2, into accumulator g,
// and as long as a sum stays below 2^24 the FP32 accumulation is exact.  K is
// therefore cut into chunks (a few k-blocks of 64) whose accumulators are
// combined in FP64 with their weights and the two scales, and the chunks are
// summed in FP64 by the split-K reduction.  The only errors left are the
// dropped high-order slices and products, which are symmetric about zero.
// BF16X6 keeps 3 x 3 slices and the 6 products with g <= 2: ~2^-24 relative
// to the row and column maxima.  BF16X10 keeps 4 x 4 slices, cut from the
// FP64 mantissa by integer arithmetic (x 2^-e_r rounded to a multiple of
// 2^-31, written in balanced base-256 digits), and the 10 products with
// g <= 3 in four accumulators: ~2^-31 relative to the row and column maxima.
// Floating-point forms (FP32 accumulation on the tensor cores, which rounds
// toward zero and therefore drifts):
//   BF16X3 : A = A_hi + A_lo, B = B_hi + B_lo (bf16 each),
//            A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi  (3 MMAs, kind::f16)
//   TF32   : one MMA, kind::tf32
//   TF32X3 : A = A_hi + A_lo (tf32 each), 3 MMAs, kind::tf32
//   BF16   : one MMA, kind::f16
//
// Kernel: one 128 x BN output tile per CTA (4 warps).  Warp 0 (one elected
// thread) streams A/B k-blocks with TMA (128-byte swizzle) into a ring of
// shared-memory stages guarded by mbarriers; warp 1 (one elected thread)
// issues tcgen05.mma from shared-memory descriptors into a TMEM accumulator and
// releases each stage with tcgen05.commit; all four warps then read the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and write
// alpha * acc + beta * C in FP64.  Every mbarrier wait is bounded: on a
// timeout the kernel records an error code, skips the remaining work, frees
// its TMEM and returns.  A split of K writes FP64 partial tiles that the FP64
// reduction kernel sums in a fixed order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "gemm_tc.cuh"

namespace qtt {

namespace {

constexpr int TC_THREADS = 128;
constexpr int BM = 128;
constexpr long long kWaitLimit = 1LL << 26;  // try_wait iterations before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after kWaitLimit polls or 2 s of wall time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && global_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                    // descriptor version of this architecture
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor: D f32, A/B of type `fmt` (bf16 = 1, tf32 = 2),
// both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t bn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Conversions between FP64 and FP32 by bit manipulation.  The FP64 pipe of
// this GPU issues two operations per clock per SM, so the packing and the
// epilogue (which touch every operand and output element) use only integer
// and FP32 instructions.

// float -> double, exact (zero, normal, inf and NaN by bits; denormals, which
// the accumulators of these products do not produce in practice, by the
// hardware conversion).
__device__ __forceinline__ unsigned long long float_to_double_bits(uint32_t f) {
  const uint32_t e = (f >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(f >> 31) << 63;
  if (e == 0u) {
    if ((f & 0x7FFFFFu) == 0u) return sign;
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(f));
  }
  const unsigned long long de = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e + 896u);
  return sign | (de << 52) | ((unsigned long long)(f & 0x7FFFFFu) << 29);
}

// S 2^scale as a double, exact for |S| < 2^53; results below the normal range
// flush to zero.
__device__ __forceinline__ unsigned long long int_to_double_bits(long long S, int scale) {
  if (S == 0) return 0ull;
  const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = (unsigned long long)(S < 0 ? -S : S);
  const int lz = __clzll((long long)a);
  const int ex = (63 - lz) + 1023 + scale;  // a = 1.m 2^(63 - lz)
  if (ex <= 0) return sign;
  if (ex >= 2047) return sign | (0x7FFull << 52);
  const unsigned long long mant = ((a << lz) << 1) >> 12;  // drop the leading one, keep 52 bits
  return sign | ((unsigned long long)ex << 52) | mant;
}

// double -> float, round to nearest even; results below the normal float
// range flush to zero, results above it become infinities.
__device__ __forceinline__ float double_bits_to_float(unsigned long long u) {
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFull);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned long long rem = m & 0x1FFFFFFFull;  // 29 dropped bits
  uint32_t r = ((uint32_t)fe << 23) | (uint32_t)(m >> 29);
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1u))) r += 1u;  // a carry into the exponent is correct
  return __uint_as_float(sign | r);
}

// |x| as an order-preserving integer (the bits of a non-negative double).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// x 2^k by exponent arithmetic (x normal, result normal or flushed to zero).
__device__ __forceinline__ unsigned long long scale_bits(unsigned long long u, int k) {
  const int e = (int)((u >> 52) & 0x7FFull);
  if (e == 0) return u & (1ull << 63);  // zero (or a denormal, flushed)
  const int ne = e + k;
  if (ne <= 0) return u & (1ull << 63);
  if (ne >= 2047) return (u & (1ull << 63)) | (0x7FFull << 52);
  return (u & ~(0x7FFull << 52)) | ((unsigned long long)ne << 52);
}

// na / nb: operand buffers of A and B per k-block; ngroups: TMEM accumulators.
template <int MODE>
struct ModeTraits;
template <>
struct ModeTraits<TC_BF16X3> {
  static constexpr bool tf32 = false, sliced = false;
  static constexpr int na = 2, nb = 2, ngroups = 1, esize = 2;
};
template <>
struct ModeTraits<TC_BF16X6> {
  static constexpr bool tf32 = false, sliced = true;
  static constexpr int na = 3, nb = 3, ngroups = 3, esize = 2;
};
template <>
struct ModeTraits<TC_BF16X10> {
  static constexpr bool tf32 = false, sliced = true;
  static constexpr int na = 4, nb = 4, ngroups = 4, esize = 2;
};
template <>
struct ModeTraits<TC_BF16> {
  static constexpr bool tf32 = false, sliced = false;
  static constexpr int na = 1, nb = 1, ngroups = 1, esize = 2;
};
template <>
struct ModeTraits<TC_TF32> {
  static constexpr bool tf32 = true, sliced = false;
  static constexpr int na = 1, nb = 1, ngroups = 1, esize = 4;
};
template <>
struct ModeTraits<TC_TF32X3> {
  static constexpr bool tf32 = true, sliced = false;
  static constexpr int na = 2, nb = 2, ngroups = 1, esize = 4;
};

__host__ __device__ constexpr int tmem_cols_for(int cols) {
  return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}

template <int MODE, int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmA3,
                   const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                   const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ CUtensorMap tmB3, int M, int N,
                   int kblocks, int kb_per_split, int splitk, int inner, double alpha, double beta, OutView C,
                   double* ws, const int* __restrict__ ea, const int* __restrict__ eb, int a_bs, int b_bs, int* err) {
  using Tr = ModeTraits<MODE>;
  constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
  constexpr int STAGE_BYTES = Tr::na * A_BYTES + Tr::nb * B_BYTES;
  constexpr uint32_t IDESC = make_idesc(Tr::tf32 ? 2u : 1u, (uint32_t)BN);
  constexpr int TMEM_COLS = tmem_cols_for(Tr::ngroups * BN);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int s_abort, s_issued;

  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int z = blockIdx.z;
  const int b = z / splitk, ks = z - b * splitk;
  const int kb0 = ks * kb_per_split;
  const int kb1 = min(kblocks, kb0 + kb_per_split);

  if (threadIdx.x == 0) {
    s_abort = 0;
    s_issued = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();  // operands and outputs are touched only from here on

  if (warp == 0 && lane == 0) {
    // TMA producer; a stage holds the na A tiles, then the nb B tiles
    const CUtensorMap* ma[4] = {&tmA0, &tmA1, &tmA2, &tmA3};
    const CUtensorMap* mb[4] = {&tmB0, &tmB1, &tmB2, &tmB3};
    for (int kb = kb0, i = 0; kb < kb1; ++kb, ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)((i / STAGES) & 1);
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        atomicOr(err, 4);
        s_abort = 1;
        break;
      }
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int kx = kb * (128 / Tr::esize);
#pragma unroll
      for (int t = 0; t < Tr::na; ++t) tma_load_3d(st + t * A_BYTES, ma[t], &full[s], kx, m0, b * a_bs);
#pragma unroll
      for (int t = 0; t < Tr::nb; ++t)
        tma_load_3d(st + Tr::na * A_BYTES + t * B_BYTES, mb[t], &full[s], kx, n0, b * b_bs);
      s_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    for (int kb = kb0, i = 0; kb < kb1; ++kb, ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)((i / STAGES) & 1);
      if (!mbar_wait(&full[s], ph)) {
        atomicOr(err, 8);
        s_abort = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t bst = st + Tr::na * A_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per 128-byte row
        const uint32_t off = kk * 32;
        const bool first = (kb == kb0 && kk == 0);
        if (Tr::sliced) {
          // accumulator g collects the slice products s_i t_j with i + j = g
#pragma unroll
          for (int g = 0; g < Tr::ngroups; ++g) {
            bool fresh = first;
#pragma unroll
            for (int ia = 0; ia < Tr::na; ++ia) {
              const int jb = g - ia;
              if (jb < 0 || jb >= Tr::nb) continue;
              mma_issue<false>(tmem + (uint32_t)(g * BN), desc_sw128(st + ia * A_BYTES + off),
                               desc_sw128(bst + jb * B_BYTES + off), IDESC, fresh ? 0u : 1u);
              fresh = false;
            }
          }
        } else {
          mma_issue<Tr::tf32>(tmem, desc_sw128(st + off), desc_sw128(bst + off), IDESC, first ? 0u : 1u);
          if (Tr::na == 2) {  // hi lo + lo hi
            mma_issue<Tr::tf32>(tmem, desc_sw128(st + off), desc_sw128(bst + B_BYTES + off), IDESC, 1u);
            mma_issue<Tr::tf32>(tmem, desc_sw128(st + A_BYTES + off), desc_sw128(bst + off), IDESC, 1u);
          }
        }
      }
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(done);
  }
  __syncwarp();
  bool have = mbar_wait(done, 0);
  if (!have) atomicOr(err, 16);
  __syncthreads();
  have = have && (s_abort == 0) && (kb1 > kb0);
  tc_fence_after();
  if (s_abort != 0 && threadIdx.x == 0) {
    // give the copies still in flight (the last STAGES issued) a bounded time to land
    const int n_issued = s_issued;
    for (int i = max(0, n_issued - STAGES); i < n_issued; ++i) mbar_wait(&full[i % STAGES], (uint32_t)((i / STAGES) & 1));
  }
  const int wrow0 = m0 + warp * 32;  // first output row of this warp's TMEM lanes
  if (have && wrow0 < M) {
    const int rows_here = min(32, M - wrow0);
    const int bo = b / inner, bi = b - bo * inner;
    double* Cb = C.p + bo * C.so + bi * C.si;
    double* W = ws ? ws + ((long long)b * splitk + ks) * (long long)M * N : nullptr;
    const int m_pad = (int)gridDim.y * BM, n_pad = (int)gridDim.x * BN;
    const int erow = (Tr::sliced && wrow0 + lane < M) ? ea[(long long)(b * a_bs) * m_pad + wrow0 + lane] : 0;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    // 32 x 32 staging tile per warp in the (drained) pipeline buffers: rows are
    // TMEM lanes on the way in, columns are lanes on the way out (coalesced stores)
    unsigned long long* stg = reinterpret_cast<unsigned long long*>(smem) + warp * (32 * 33);
    const bool plain = (beta == 0.0) && (alpha == 1.0 || alpha == -1.0);
    const unsigned long long sign_flip = (alpha == -1.0) ? (1ull << 63) : 0ull;
#pragma unroll 1
    for (int c0 = 0; c0 < BN && n0 + c0 < N; c0 += 32) {
      uint32_t r[Tr::ngroups][32];
#pragma unroll
      for (int g = 0; g < Tr::ngroups; ++g) tmem_ld32(lane_base + (uint32_t)(g * BN + c0), r[g]);
      tmem_ld_wait();
      const int ecol = (Tr::sliced && n0 + c0 + lane < N) ? eb[(long long)(b * b_bs) * n_pad + n0 + c0 + lane] : 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        unsigned long long bits;
        if (Tr::sliced) {
          // exact integer sums I_g of weight 2^-(14 + 8 g) -> one integer
          // S = sum_g I_g 2^(8 (G - 1 - g)) (< 2^41 for G = 3, < 2^49 for
          // G = 4) -> S 2^(e_row + e_col - 14 - 8 (G - 1))
          const int ec = __shfl_sync(0xffffffffu, ecol, j);
          long long S = 0;
#pragma unroll
          for (int g = 0; g < Tr::ngroups; ++g)
            S += (long long)__float2int_rn(__uint_as_float(r[g][j])) << (8 * (Tr::ngroups - 1 - g));
          bits = int_to_double_bits(S, erow + ec - 14 - 8 * (Tr::ngroups - 1));
        } else {
          bits = float_to_double_bits(r[0][j]);
        }
        stg[lane * 33 + j] = bits;
      }
      __syncwarp();
      const int col = n0 + c0 + lane;
      if (col < N) {
        for (int rr = 0; rr < rows_here; ++rr) {
          const unsigned long long bits = stg[rr * 33 + lane];
          const int row = wrow0 + rr;
          if (W) {
            reinterpret_cast<unsigned long long*>(W)[(long long)row * N + col] = bits;
          } else {
            double* c = Cb + (long long)row * C.rs + (long long)col * C.cs;
            if (plain)
              *reinterpret_cast<unsigned long long*>(c) = bits ^ sign_flip;
            else
              *c = alpha * __longlong_as_double((long long)bits) + (beta == 0.0 ? 0.0 : beta * (*c));
          }
        }
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- packing
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Writes the packed form of one element.  Floating-point forms: x is rounded
// to float, then split (hi = x rounded to the operand type, lo = the rest,
// exact in float).  BF16X6: x is first scaled by 2^(ks + 7 - e) (ks: the
// K-index balancing shift; e: exponent of the row's largest balanced
// magnitude, so |t| < 128), then t = s1 + 2^-8 s2 + 2^-16 s3 + O(2^-17) with
// integers |s_p| <= 128 from round-to-nearest; all in FP32.
template <int MODE>
__device__ __forceinline__ void pack_one(double x, int e, int ks, size_t idx, void* o0, void* o1, void* o2,
                                         void* o3) {
  if constexpr (MODE == TC_BF16X10) {
    // T = round(x 2^(31 - e + ks)) from the FP64 bits (|T| <= 2^31), then
    // balanced base-256 digits T = d1 2^24 + d2 2^16 + d3 2^8 + d4 with
    // |d_p| <= 128 (integers, exact in bf16); no FP64 arithmetic.
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((u >> 52) & 0x7FFull);
    long long T = 0;
    if (E != 0) {
      const int sh = 52 - (E - 1023 + 31 - e + ks);  // right shift of the 53-bit mantissa
      const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      unsigned long long a = 0;
      if (sh <= 0) a = m << (-sh > 10 ? 10 : -sh);  // |x| 2^(31-e) < 2^31: cannot happen, kept in range
      else if (sh < 64) a = (m >> sh) + ((m >> (sh - 1)) & 1ull);
      T = (u >> 63) ? -(long long)a : (long long)a;
    }
    long long q = (T + 128) >> 8;
    const long long d4 = T - (q << 8);
    T = q;
    q = (T + 128) >> 8;
    const long long d3 = T - (q << 8);
    T = q;
    q = (T + 128) >> 8;
    const long long d2 = T - (q << 8);
    ((__nv_bfloat16*)o0)[idx] = __float2bfloat16_rn((float)q);
    ((__nv_bfloat16*)o1)[idx] = __float2bfloat16_rn((float)d2);
    ((__nv_bfloat16*)o2)[idx] = __float2bfloat16_rn((float)d3);
    ((__nv_bfloat16*)o3)[idx] = __float2bfloat16_rn((float)d4);
  } else if constexpr (MODE == TC_BF16X6) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const float t = double_bits_to_float(scale_bits(u, 7 - e + ks));
    const float a1 = rintf(t);
    float rr = (t - a1) * 256.0f;
    const float a2 = rintf(rr);
    rr = (rr - a2) * 256.0f;
    ((__nv_bfloat16*)o0)[idx] = __float2bfloat16_rn(a1);
    ((__nv_bfloat16*)o1)[idx] = __float2bfloat16_rn(a2);
    ((__nv_bfloat16*)o2)[idx] = __float2bfloat16_rn(rintf(rr));
  } else {
    const float f = double_bits_to_float((unsigned long long)__double_as_longlong(x));
    if constexpr (MODE == TC_BF16) {
      ((__nv_bfloat16*)o0)[idx] = __float2bfloat16_rn(f);
    } else if constexpr (MODE == TC_BF16X3) {
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      ((__nv_bfloat16*)o0)[idx] = h;
      ((__nv_bfloat16*)o1)[idx] = __float2bfloat16_rn(f - __bfloat162float(h));
    } else if constexpr (MODE == TC_TF32) {
      ((float*)o0)[idx] = to_tf32(f);
    } else {  // TC_TF32X3
      const float h = to_tf32(f);
      ((float*)o0)[idx] = h;
      ((float*)o1)[idx] = to_tf32(f - h);
    }
  }
}

// Row exponent for the exact slices: |x| < 2^e for every x of the row (0 for
// an all-zero row), from the bits of the largest magnitude.
__device__ __forceinline__ int row_exponent(unsigned long long maxbits) {
  const int E = (int)(maxbits >> 52);
  return E == 0 ? 0 : E - 1022;
}

// Loads each thread of the packing and maximum passes issues before it uses
// the first: the passes stream operands once, so they are bound by how many
// bytes are in flight, not by arithmetic.
constexpr int PACK_UNROLL = 8;

// One operand to pack: packed row r, element k is p[b-offset + r * rstr +
// k * kstr].  "cols" layouts (r stride 1) go through a shared tile, 32 rows x
// one k segment per block; the others take one warp per (row, k segment).
struct PackJob {
  const double* p;
  long long rstr, kstr, so, si;
  int inner, rows, K, rows_pad, k_pad, kseg, nseg;
  long long batch, units;  // units: row tiles * batch (cols) or rows * batch (warp layout)
  int cols, ksign;
  const int* kshift;               // K-index balancing shifts (BF16X6), or null
  long long kshift_bstride;        // k_pad, or 0 when the shifts are common to the batch
  unsigned long long* maxbits;     // per packed row: largest balanced magnitude (BF16X6)
  void *o0, *o1, *o2, *o3;
  int* expo;
  int blocks;                      // blocks of this job in the fused launch
};

// The exact slices need, per packed row, the largest balanced magnitude over
// all of K.  It is reduced in a pass of its own (partial maxima of k segments
// combined with atomicMax on the order-preserving bits into a zeroed buffer),
// so that the packing can split K across blocks without re-reading rows.
__device__ void opmax_job(const PackJob& J, int bx) {
  const int lane = threadIdx.x & 31;
  if (J.cols) {
    __shared__ unsigned long long red[8][32];
    const long long u = bx % J.units;
    const int seg = (int)(bx / J.units);
    const int tiles_r = J.rows_pad / 32;
    const long long b = u / tiles_r;
    const int r0 = (int)(u - b * tiles_r) * 32;
    const long long bo = b / J.inner, bi = b - bo * J.inner;
    const double* src = J.p + bo * J.so + bi * J.si;
    const int* ksh = J.kshift + b * J.kshift_bstride;
    const int tx = lane, ty = threadIdx.x >> 5;
    unsigned long long mx = 0;
    if (r0 + tx < J.rows) {
      const int k1 = min(J.K, (seg + 1) * J.kseg);
      for (int k0 = seg * J.kseg + ty; k0 < k1; k0 += 8 * PACK_UNROLL) {
        unsigned long long x[PACK_UNROLL];  // all loads in flight before the first use
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) {
          const int k = k0 + 8 * u;
          x[u] = k < k1 ? scale_bits(abs_bits(src[(r0 + tx) + (long long)k * J.kstr]), J.ksign * ksh[k]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) mx = max(mx, x[u]);
      }
    }
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
      for (int q = 1; q < 8; ++q) mx = max(mx, red[q][tx]);
      if (mx != 0ull) atomicMax(J.maxbits + b * J.rows_pad + r0 + tx, mx);
    }
  } else {
    const long long warps_total = J.units * J.nseg;
    for (long long w = ((long long)bx * blockDim.x + threadIdx.x) >> 5; w < warps_total;
         w += ((long long)J.blocks * blockDim.x) >> 5) {
      const long long rowid = w / J.nseg;
      const int seg = (int)(w - rowid * J.nseg);
      const long long b = rowid / J.rows_pad;
      const int r = (int)(rowid - b * J.rows_pad);
      if (r >= J.rows) continue;  // warp-uniform
      const long long bo = b / J.inner, bi = b - bo * J.inner;
      const double* row = J.p + bo * J.so + bi * J.si + (long long)r * J.rstr;
      const int* ksh = J.kshift + b * J.kshift_bstride;
      unsigned long long mx = 0;
      const int k1 = min(J.K, (seg + 1) * J.kseg);
      for (int k0 = seg * J.kseg + lane; k0 < k1; k0 += 32 * PACK_UNROLL) {
        unsigned long long x[PACK_UNROLL];
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) {
          const int k = k0 + 32 * u;
          x[u] = k < k1 ? scale_bits(abs_bits(row[(long long)k * J.kstr]), J.ksign * ksh[k]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) mx = max(mx, x[u]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx != 0ull) atomicMax(J.maxbits + rowid, mx);
    }
  }
}

template <int MODE>
__device__ void pack_job(const PackJob& J, int bx) {
  const int lane = threadIdx.x & 31;
  if (J.cols) {
    __shared__ double tile[64][33];  // [k][r]
    __shared__ int s_e[32];
    const long long u = bx % J.units;
    const int seg = (int)(bx / J.units);
    const int tiles_r = J.rows_pad / 32;
    const long long b = u / tiles_r;
    const int r0 = (int)(u - b * tiles_r) * 32;
    const long long bo = b / J.inner, bi = b - bo * J.inner;
    const double* src = J.p + bo * J.so + bi * J.si;
    const int tx = lane, ty = threadIdx.x >> 5;  // 32 x 8
    const bool rlive = r0 + tx < J.rows;
    const int* ksh = J.kshift ? J.kshift + b * J.kshift_bstride : nullptr;
    if constexpr (MODE == TC_BF16X6 || MODE == TC_BF16X10) {
      if (ty == 0) {
        const int e = row_exponent(J.maxbits[b * J.rows_pad + r0 + tx]);
        s_e[tx] = e;
        if (seg == 0) J.expo[b * J.rows_pad + r0 + tx] = e;
      }
      __syncthreads();
    }
    const int kend = min(J.k_pad, (seg + 1) * J.kseg);
    for (int k0 = seg * J.kseg; k0 < kend; k0 += 64) {  // kseg is a multiple of 32: the second half may be past kend
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kl = ty + 8 * q, k = k0 + kl;
        tile[kl][tx] = (rlive && k < J.K && k < kend) ? src[(r0 + tx) + (long long)k * J.kstr] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rl = ty + 8 * q;
        const int e = (MODE == TC_BF16X6 || MODE == TC_BF16X10) ? s_e[rl] : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = k0 + 32 * h + tx;
          if (k < kend)
            pack_one<MODE>(tile[32 * h + tx][rl], e, (ksh && k < J.K) ? J.ksign * ksh[k] : 0,
                           ((size_t)b * J.rows_pad + r0 + rl) * J.k_pad + k, J.o0, J.o1, J.o2, J.o3);
        }
      }
      __syncthreads();
    }
  } else {
    const long long warps_total = J.units * J.nseg;
    for (long long w = ((long long)bx * blockDim.x + threadIdx.x) >> 5; w < warps_total;
         w += ((long long)J.blocks * blockDim.x) >> 5) {
      const long long rowid = w / J.nseg;
      const int seg = (int)(w - rowid * J.nseg);
      const long long b = rowid / J.rows_pad;
      const int r = (int)(rowid - b * J.rows_pad);
      const long long bo = b / J.inner, bi = b - bo * J.inner;
      const double* row = J.p + bo * J.so + bi * J.si + (long long)r * J.rstr;
      const int* ksh = J.kshift ? J.kshift + b * J.kshift_bstride : nullptr;
      const bool live = r < J.rows;
      int e = 0;
      if constexpr (MODE == TC_BF16X6 || MODE == TC_BF16X10) {
        e = row_exponent(J.maxbits[rowid]);
        if (lane == 0 && seg == 0) J.expo[rowid] = e;
      }
      const size_t base = (size_t)rowid * J.k_pad;
      const int k1 = min(J.k_pad, (seg + 1) * J.kseg);
      if (MODE == TC_BF16X3 && J.kstr == 1 && !ksh && ((uintptr_t)row & 15) == 0 && (J.kseg & 63) == 0) {
        // contiguous rows: two elements per lane (16-byte loads, 4-byte bf16x2 stores)
        for (int k0 = seg * J.kseg + 2 * lane; k0 < k1; k0 += 64 * (PACK_UNROLL / 2)) {
          double2 x[PACK_UNROLL / 2];
#pragma unroll
          for (int u = 0; u < PACK_UNROLL / 2; ++u) {
            const int k = k0 + 64 * u;
            x[u] = make_double2(0.0, 0.0);
            if (live && k + 1 < J.K && k < k1) x[u] = *reinterpret_cast<const double2*>(row + k);
            else if (live && k < J.K && k < k1) x[u].x = row[k];
          }
#pragma unroll
          for (int u = 0; u < PACK_UNROLL / 2; ++u) {
            const int k = k0 + 64 * u;
            if (k >= k1) continue;
            const float f0 = double_bits_to_float((unsigned long long)__double_as_longlong(x[u].x));
            const float f1 = double_bits_to_float((unsigned long long)__double_as_longlong(x[u].y));
            const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
            const __nv_bfloat162 l = __floats2bfloat162_rn(f0 - __low2float(h), f1 - __high2float(h));
            *reinterpret_cast<__nv_bfloat162*>((__nv_bfloat16*)J.o0 + base + k) = h;
            *reinterpret_cast<__nv_bfloat162*>((__nv_bfloat16*)J.o1 + base + k) = l;
          }
        }
        continue;
      }
      for (int k0 = seg * J.kseg + lane; k0 < k1; k0 += 32 * PACK_UNROLL) {
        double x[PACK_UNROLL];  // all loads in flight before the first use
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) {
          const int k = k0 + 32 * u;
          x[u] = (live && k < J.K && k < k1) ? row[(long long)k * J.kstr] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < PACK_UNROLL; ++u) {
          const int k = k0 + 32 * u;
          if (k < k1) pack_one<MODE>(x[u], e, (ksh && k < J.K) ? J.ksign * ksh[k] : 0, base + k, J.o0, J.o1, J.o2, J.o3);
        }
      }
    }
  }
}

// Both operands in one launch each: blocks [0, a.blocks) serve a, the rest b.
__global__ void __launch_bounds__(256) opmax2_kernel(const PackJob a, const PackJob b) {
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < a.blocks)
    opmax_job(a, blockIdx.x);
  else
    opmax_job(b, blockIdx.x - a.blocks);
}
template <int MODE>
__global__ void __launch_bounds__(256) pack2_kernel(const PackJob a, const PackJob b) {
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < a.blocks)
    pack_job<MODE>(a, blockIdx.x);
  else
    pack_job<MODE>(b, blockIdx.x - a.blocks);
}

// K-index balancing for the exact slices: kshift[b][k] = exponent of
// max_n |B(k, n)| (|B(k, n)| < 2^kshift).  Packing then uses B(k, n) 2^-kshift
// and A(r, k) 2^+kshift, which leaves A B unchanged (powers of two, exact) and
// makes every row of B' of magnitude < 1, so that A''s row exponent follows
// the largest product term a_rk b_kn rather than the largest a_rk.  (In the
// products of this method B is often a right environment whose rows carry
// the bond's singular values.)  B(k, n) at k * rs + n * cs; a warp per k when
// n is contiguous, 32 k per block otherwise.
__global__ void kbalance_kernel(const double* __restrict__ p, long long rs, long long cs, long long so, long long si,
                                int inner, int K, int N, int k_pad, long long batch, int common, int* kshift,
                                unsigned long long* zero_me, long long nzero) {
  // common = 1: one shift per k over the whole batch (batch entries loop inside)
  const long long nb_out = common ? 1 : batch, nb_in = common ? batch : 1;
  pdl_trigger();
  pdl_wait();
  const int lane = threadIdx.x & 31;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nzero; x += (long long)gridDim.x * blockDim.x)
    zero_me[x] = 0ull;  // the row-maximum buffer of the next pass
  if (cs == 1) {
    const long long warps_total = (long long)k_pad * nb_out;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < warps_total;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
      const long long b0 = w / k_pad;
      const int k = (int)(w - b0 * k_pad);
      unsigned long long mx = 0;
      for (long long bb = 0; bb < nb_in && k < K; ++bb) {
        const long long b = b0 + bb;
        const long long bo = b / inner, bi = b - bo * inner;
        const double* row = p + bo * so + bi * si + (long long)k * rs;
        for (int n0 = lane; n0 < N; n0 += 32 * PACK_UNROLL) {
          unsigned long long x[PACK_UNROLL];
#pragma unroll
          for (int u = 0; u < PACK_UNROLL; ++u) x[u] = n0 + 32 * u < N ? abs_bits(row[n0 + 32 * u]) : 0ull;
#pragma unroll
          for (int u = 0; u < PACK_UNROLL; ++u) mx = max(mx, x[u]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) kshift[w] = row_exponent(mx);
    }
  } else {
    // 32 k x 8 n-groups per block (reads coalesce along k when rs == 1)
    __shared__ unsigned long long red[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int ktiles = (k_pad + 31) / 32;
    const long long tiles = (long long)ktiles * nb_out;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
      const long long b0 = t / ktiles;
      const int k = (int)(t - b0 * ktiles) * 32 + tx;
      unsigned long long mx = 0;
      for (long long bb = 0; bb < nb_in && k < K; ++bb) {
        const long long b = b0 + bb;
        const long long bo = b / inner, bi = b - bo * inner;
        const double* row = p + bo * so + bi * si + (long long)k * rs;
        for (int n0 = ty; n0 < N; n0 += 8 * PACK_UNROLL) {
          unsigned long long x[PACK_UNROLL];
#pragma unroll
          for (int u = 0; u < PACK_UNROLL; ++u)
            x[u] = n0 + 8 * u < N ? abs_bits(row[(long long)(n0 + 8 * u) * cs]) : 0ull;
#pragma unroll
          for (int u = 0; u < PACK_UNROLL; ++u) mx = max(mx, x[u]);
        }
      }
      red[ty][tx] = mx;
      __syncthreads();
      if (ty == 0) {
        for (int q = 1; q < 8; ++q) mx = max(mx, red[q][tx]);
        if (k < k_pad) kshift[b0 * k_pad + k] = row_exponent(mx);
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) throw std::runtime_error("CUDA error: cuTensorMapEncodeTiled is unavailable");
}

CUtensorMap make_map(const void* base, int esize, int k_pad, int rows_pad, long long batch, int box_rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[3] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)k_pad * esize, (cuuint64_t)k_pad * esize * (cuuint64_t)rows_pad};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_encode(&m, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("CUDA error: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

template <int MODE, int BN, int STAGES>
void launch_tc(cudaStream_t st, const TcPacked& pk, int M, int N, int kblocks, int kbps, int splitk, int inner,
               long long batch, long long batch_a, long long batch_b, double alpha, double beta, OutView C, double* ws,
               int* err) {
  using Tr = ModeTraits<MODE>;
  constexpr int SMEM = STAGES * (Tr::na * BM * 128 + Tr::nb * BN * 128) + 1024 + 256;
  static_assert(SMEM <= 232448, "shared memory budget");
  static_assert(Tr::ngroups * BN <= 512, "TMEM budget");
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_gemm_kernel<MODE, BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    attr = true;
  }
  CUtensorMap a[4], bm[4];
  for (int i = 0; i < 4; ++i) {
    a[i] = make_map(pk.a[i < Tr::na ? i : 0], Tr::esize, pk.k_pad, pk.m_pad, batch_a, BM);
    bm[i] = make_map(pk.b[i < Tr::nb ? i : 0], Tr::esize, pk.k_pad, pk.n_pad, batch_b, BN);
  }
  dim3 grid(pk.n_pad / BN, pk.m_pad / BM, (unsigned)(batch * splitk));
  launch_pdl(tc_gemm_kernel<MODE, BN, STAGES>, grid, dim3(TC_THREADS), SMEM, st, a[0], a[1], a[2], a[3], bm[0],
             bm[1], bm[2], bm[3], M, N, kblocks, kbps, splitk, inner, alpha, beta, C, ws, (const int*)pk.ea, (const int*)pk.eb,
             batch_a == batch ? 1 : 0, batch_b == batch ? 1 : 0, err);
}

// Packs one operand (rows x K, element (r, k) at r * rstr + k * kstr) into the
// K-major buffers o[0..) (and, for BF16X6, the row exponents).
// Fills the geometry of one packing job: k segments so that about two waves
// of 152 SMs' worth of blocks exist.
PackJob make_job(const MatView& v, long long rstr, long long kstr, int inner, int rows, int K, int rows_pad,
                 int k_pad, long long batch, void* const* o, int* expo, const int* kshift, long long kshift_bstride,
                 int ksign, unsigned long long* maxbits) {
  PackJob J;
  J.kshift_bstride = kshift_bstride;
  J.p = v.p;
  J.rstr = rstr;
  J.kstr = kstr;
  J.so = v.so;
  J.si = v.si;
  J.inner = inner;
  J.rows = rows;
  J.K = K;
  J.rows_pad = rows_pad;
  J.k_pad = k_pad;
  J.batch = batch;
  J.ksign = ksign;
  J.kshift = kshift;
  J.maxbits = maxbits;
  J.o0 = o[0];
  J.o1 = o[1];
  J.o2 = o[2];
  J.o3 = o[3];
  J.expo = expo;
  J.cols = (rstr == 1 && kstr != 1 && rows_pad % 32 == 0) ? 1 : 0;
  const int chunks = (k_pad + 31) / 32;
  J.units = J.cols ? (long long)(rows_pad / 32) * batch : (long long)rows_pad * batch;
  const long long want = J.cols ? 2 * 152 : 2 * 152 * 16;  // blocks (tile layout) / warps (row layout)
  int nseg = (int)std::min<long long>(chunks, std::max<long long>(1, (want + J.units - 1) / J.units));
  J.kseg = 32 * ((chunks + nseg - 1) / nseg);
  J.nseg = (k_pad + J.kseg - 1) / J.kseg;
  long long blocks = J.cols ? J.units * J.nseg : (J.units * J.nseg * 32 + 255) / 256;
  if (!J.cols && blocks > 8192) blocks = 8192;
  J.blocks = (int)blocks;
  return J;
}

struct ModeInfo {
  int na, nb, ngroups, esize;
  bool sliced;
  int exact_kb;  // k-blocks one accumulator may sum exactly (0: no limit)
};

ModeInfo mode_info(int mode) {
  switch (mode) {
    case TC_BF16X3: return {2, 2, 1, 2, false, 0};
    case TC_BF16X6: return {3, 3, 3, 2, true, 5};
    // group 3 sums 4 slice products (|.| <= 2^14 each) per k: 4 k-blocks of 64 stay <= 2^24
    case TC_BF16X10: return {4, 4, 4, 2, true, 4};
    case TC_BF16: return {1, 1, 1, 2, false, 0};
    case TC_TF32: return {1, 1, 1, 4, false, 0};
    default: return {2, 2, 1, 4, false, 0};  // TC_TF32X3
  }
}

int choose_bn(int N, int mode) {
  // smallest padded width among the tile widths whose accumulators fit in TMEM
  const ModeInfo mi = mode_info(mode);
  const int all[4] = {256, 160, 128, 64};
  int best = 64;
  long long bestpad = 1LL << 60;
  for (int c : all) {
    if (mi.ngroups * c > 512) continue;
    const long long pad = (long long)((N + c - 1) / c) * c;
    if (pad < bestpad) {
      bestpad = pad;
      best = c;
    }
  }
  return best;
}

struct PackLayout {
  int bn, m_pad, n_pad, k_pad, kb;
  size_t a_bytes, b_bytes, total;
};

size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

PackLayout pack_layout(int M, int N, int K, long long batch, int mode) {
  const ModeInfo mi = mode_info(mode);
  PackLayout L;
  L.bn = choose_bn(N, mode);
  L.kb = 128 / mi.esize;
  L.k_pad = (K + L.kb - 1) / L.kb * L.kb;
  L.m_pad = (M + BM - 1) / BM * BM;
  L.n_pad = (N + L.bn - 1) / L.bn * L.bn;
  L.a_bytes = (size_t)L.m_pad * L.k_pad * batch * mi.esize;
  L.b_bytes = (size_t)L.n_pad * L.k_pad * batch * mi.esize;
  L.total = mi.na * up256(L.a_bytes) + mi.nb * up256(L.b_bytes) + up256((size_t)L.m_pad * batch * 4) +
            up256((size_t)L.n_pad * batch * 4) + up256((size_t)L.k_pad * batch * 4) +
            up256((size_t)(L.m_pad + L.n_pad) * batch * 8) + 256;
  return L;
}

// shape key of the split-K autotuner and its process-wide cache
struct TuneKey {
  int mode, M, N, K;
  long long batch, ba, bb;
  int cap;
  bool operator<(const TuneKey& o) const {
    if (mode != o.mode) return mode < o.mode;
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    if (K != o.K) return K < o.K;
    if (batch != o.batch) return batch < o.batch;
    if (ba != o.ba) return ba < o.ba;
    if (bb != o.bb) return bb < o.bb;
    return cap < o.cap;
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune;

bool tune_lookup(const TuneKey& k, int& s) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  s = it->second;
  return true;
}
void tune_store(const TuneKey& k, int s) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune[k] = s;
}
bool tune_enabled() {
  const char* e = std::getenv("QTT_TUNE");
  return !(e && e[0] == '0');
}
bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: do not time
  }
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

size_t tc_workspace_bytes(int M, int N, int K, long long batch, int mode) {
  return pack_layout(M, N, K, batch, mode).total + 8192;
}

bool gemm_tc(cudaStream_t st, int mode, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
             double beta, OutView C, void* pack_ws, size_t pack_bytes, double* ws, size_t ws_elems, int* err,
             int max_kb_per_split) {
  if (M <= 0 || N <= 0 || K <= 0 || outer <= 0 || inner <= 0) return false;
  load_encode();
  const long long batch = (long long)outer * inner;
  if (batch > 65535) return false;
  const ModeInfo mi = mode_info(mode);
  const PackLayout L = pack_layout(M, N, K, batch, mode);
  if (L.total > pack_bytes) return false;
  // an operand identical for every batch entry (zero batch strides) is packed once
  const long long batch_a = (A.so == 0 && A.si == 0) ? 1 : batch;
  const long long batch_b = (B.so == 0 && B.si == 0) ? 1 : batch;
  const bool common_shift = batch_a != batch || batch_b != batch;
  TcPacked pk;
  pk.k_pad = L.k_pad;
  pk.m_pad = L.m_pad;
  pk.n_pad = L.n_pad;
  uint8_t* base = (uint8_t*)(((uintptr_t)pack_ws + 255) & ~(uintptr_t)255);
  auto carve = [&](size_t n) {
    uint8_t* q = base;
    base += up256(n);
    return (void*)q;
  };
  for (int i = 0; i < mi.na; ++i) pk.a[i] = carve(L.a_bytes);
  for (int i = 0; i < mi.nb; ++i) pk.b[i] = carve(L.b_bytes);
  pk.ea = (int*)carve((size_t)L.m_pad * batch * 4);
  pk.eb = (int*)carve((size_t)L.n_pad * batch * 4);
  int* kshift = nullptr;
  unsigned long long* maxa = nullptr;
  unsigned long long* maxb = nullptr;
  if (mi.sliced) {
    kshift = (int*)carve((size_t)L.k_pad * batch * 4);
    maxa = (unsigned long long*)carve((size_t)(L.m_pad + L.n_pad) * batch * 8);
    maxb = maxa + (size_t)L.m_pad * batch;
  }
  // A(m, k) = A.p[m * rs + k * cs]; B is packed as B^T: (n, k) = B.p[k * rs + n * cs]
  const long long ksb = common_shift ? 0 : L.k_pad;
  const PackJob ja = make_job(A, A.rs, A.cs, inner, M, K, L.m_pad, L.k_pad, batch_a, pk.a, pk.ea, kshift, ksb, 1, maxa);
  const PackJob jb = make_job(B, B.cs, B.rs, inner, N, K, L.n_pad, L.k_pad, batch_b, pk.b, pk.eb, kshift, ksb, -1, maxb);
  const unsigned pack_blocks = (unsigned)(ja.blocks + jb.blocks);
  if (mi.sliced) {
    const long long kb_batch = common_shift ? 1 : batch;
    const long long items = B.cs == 1 ? 32LL * L.k_pad * kb_batch : 256LL * ((L.k_pad + 31) / 32) * kb_batch;
    long long blocks = (items + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    launch_pdl(kbalance_kernel, dim3((unsigned)blocks), dim3(256), 0, st, B.p, B.rs, B.cs, B.so, B.si, inner, K, N,
               L.k_pad, batch_b, (common_shift && batch_b == batch) ? 1 : 0, kshift, maxa,
               (long long)(L.m_pad + L.n_pad) * batch);
    launch_pdl(opmax2_kernel, dim3(pack_blocks), dim3(256), 0, st, ja, jb);
  }
  switch (mode) {
    case TC_BF16: launch_pdl(pack2_kernel<TC_BF16>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
    case TC_BF16X3: launch_pdl(pack2_kernel<TC_BF16X3>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
    case TC_TF32: launch_pdl(pack2_kernel<TC_TF32>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
    case TC_TF32X3: launch_pdl(pack2_kernel<TC_TF32X3>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
    case TC_BF16X10: launch_pdl(pack2_kernel<TC_BF16X10>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
    default: launch_pdl(pack2_kernel<TC_BF16X6>, dim3(pack_blocks), dim3(256), 0, st, ja, jb); break;
  }
  const int kblocks = L.k_pad / L.kb;
  // split K when the tile grid is small; the exact-slice modes also cap the
  // depth one accumulator sums so that its partial sums stay exact integers.
  // (Capping the floating modes' accumulation depth as well -- 1, 2 or 4
  // k-blocks per accumulator -- did not make BF16X3 more accurate: its error
  // is that of its 16-bit operands; so they keep the tile-grid split only.)
  int cap = max_kb_per_split;
  if (mi.exact_kb > 0 && (cap <= 0 || cap > mi.exact_kb)) cap = mi.exact_kb;
  // The split count minimises a cost model: waves of CTAs x k-blocks per
  // split x the time of one k-block (its operand bytes at ~60 GB/s per SM),
  // plus the FP64 partial tiles written, re-read and reduced (2 s + 1 passes
  // over M x N at ~3 TB/s).  Short K with many tiles stays unsplit.
  auto model_split = [&](int bn) {
    const long long tiles = (long long)(L.m_pad / BM) * (L.n_pad / bn) * batch;
    const double kb_us = (double)(mi.na * BM + mi.nb * bn) * 128.0 / 60e3;
    const double mn_bytes = (double)M * N * batch * 8.0;
    double best = 0.0;
    int sbest = 1;
    for (int s = 1; s <= 64 && s <= kblocks; ++s) {
      const int per = (kblocks + s - 1) / s;
      if (s > 1 && (long long)(s - 1) * per >= kblocks) continue;  // an empty split
      const double waves = (double)((tiles * s + 151) / 152);
      const double t = waves * per * kb_us + (s > 1 ? (2.0 * s + 1.0) * mn_bytes / 3e6 : 0.0);
      if (s == 1 || t < best) {
        best = t;
        sbest = s;
      }
    }
    return sbest;
  };
  int splitk = model_split(L.bn);
  // a split count as launched: k-blocks per split within the exactness cap,
  // partial tiles that fit the workspace (0: not launchable)
  auto legal = [&](int s_req, int& kbps_out) -> int {
    int kb = (kblocks + s_req - 1) / s_req;
    if (cap > 0 && kb > cap) kb = cap;
    const int s2 = (kblocks + kb - 1) / kb;
    if (s2 > 1 && (ws == nullptr || (size_t)s2 * batch * (size_t)M * N > ws_elems || s2 * batch > 65535)) return 0;
    kbps_out = kb;
    return s2;
  };
  auto run = [&](int bn, int sk, int kb, double beta_, OutView C_) {
    double* wsp = sk > 1 ? ws : nullptr;
#define QTT_TC_LAUNCH(MODE_, BN_, ST_) \
  launch_tc<MODE_, BN_, ST_>(st, pk, M, N, kblocks, kb, sk, inner, batch, batch_a, batch_b, alpha, beta_, C_, wsp, err)
#define QTT_TC_BN(MODE_, S256, S160, S128, S64)       \
  switch (bn) {                                       \
    case 256: QTT_TC_LAUNCH(MODE_, 256, S256); break; \
    case 160: QTT_TC_LAUNCH(MODE_, 160, S160); break; \
    case 128: QTT_TC_LAUNCH(MODE_, 128, S128); break; \
    default: QTT_TC_LAUNCH(MODE_, 64, S64); break;    \
  }
#define QTT_TC_BN2(MODE_, S128, S64)                  \
  switch (bn) {                                       \
    case 128: QTT_TC_LAUNCH(MODE_, 128, S128); break; \
    default: QTT_TC_LAUNCH(MODE_, 64, S64); break;    \
  }
#define QTT_TC_BN3(MODE_, S160, S128, S64)            \
  switch (bn) {                                       \
    case 160: QTT_TC_LAUNCH(MODE_, 160, S160); break; \
    case 128: QTT_TC_LAUNCH(MODE_, 128, S128); break; \
    default: QTT_TC_LAUNCH(MODE_, 64, S64); break;    \
  }
    // stages: as many as fit in 227 KB of shared memory
    switch (mode) {
      case TC_BF16X3: QTT_TC_BN(TC_BF16X3, 2, 3, 3, 4); break;
      case TC_BF16X6: QTT_TC_BN3(TC_BF16X6, 2, 2, 3); break;
      case TC_BF16X10: QTT_TC_BN2(TC_BF16X10, 1, 2); break;
      case TC_BF16: QTT_TC_BN(TC_BF16, 4, 4, 6, 8); break;
      case TC_TF32: QTT_TC_BN(TC_TF32, 4, 4, 6, 8); break;
      default: QTT_TC_BN(TC_TF32X3, 2, 3, 3, 4); break;
    }
#undef QTT_TC_BN2
#undef QTT_TC_BN3
#undef QTT_TC_BN
#undef QTT_TC_LAUNCH
    if (sk > 1) splitk_reduce(st, M, N, inner, sk, (int)batch, alpha, ws, beta_, C_);
  };
  int kbps = kblocks;
  splitk = legal(splitk, kbps);
  if (splitk == 0) {
    if (mi.exact_kb > 0) return false;  // exactness needs the FP64 reduction of the chunks
    splitk = 1;
    kbps = kblocks;
  }
  // Autotuner of the tile width and the split-K count: the first time a
  // shape is seen outside a graph capture, the cost model's split for the
  // padding-chosen tile width, half, double and no split of it, and each
  // other tile width whose padded N is the same (the packed operands then
  // serve it unchanged) with its model split and no split, are each timed
  // (CUDA events, three launches after one warm-up, output into a scratch
  // buffer), and the fastest is kept for every later call of that shape.
  // Later steps (and the captured graphs) reuse the choice.
  int bn = L.bn;
  {
    const TuneKey key{mode, M, N, K, batch, batch_a, batch_b, cap};
    int cached = 0;
    if (tune_lookup(key, cached)) {
      int kb2 = kblocks;
      const int s2 = legal(cached % 1000, kb2);
      if (s2 > 0) {
        bn = cached / 1000;
        splitk = s2;
        kbps = kb2;
      }
    } else if (tune_enabled() && !stream_capturing(st)) {
      std::vector<std::pair<int, int>> cands{{bn, splitk}};
      auto add = [&](int b, int c) {
        int kb2 = kblocks;
        const int s2 = c >= 1 ? legal(c, kb2) : 0;
        if (s2 > 0 && std::find(cands.begin(), cands.end(), std::make_pair(b, s2)) == cands.end())
          cands.push_back({b, s2});
      };
      for (int c : {1, splitk / 2, splitk * 2}) add(bn, c);
      for (int b : {256, 160, 128, 64}) {
        if (b == L.bn || mi.ngroups * b > 512 || (mode == TC_BF16X6 && b == 256)) continue;
        if ((N + b - 1) / b * b != L.n_pad) continue;
        add(b, model_split(b));
        add(b, 1);
      }
      std::pair<int, int> best = cands[0];
      if (cands.size() > 1) {
        double* scratch = nullptr;
        const size_t sbytes = (size_t)M * N * batch * sizeof(double);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaMalloc(&scratch, sbytes) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess) {
          OutView Cs;
          Cs.p = scratch;
          Cs.rs = N;
          Cs.cs = 1;
          Cs.si = (long long)M * N;
          Cs.so = Cs.si * inner;
          float best_ms = 1e30f;
          for (const auto& c : cands) {
            int kb2 = kblocks;
            const int s2 = legal(c.second, kb2);
            run(c.first, s2, kb2, 0.0, Cs);  // warm-up
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3; ++r) run(c.first, s2, kb2, 0.0, Cs);
            cudaEventRecord(e1, st);
            float ms = 1e30f;
            if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
              best_ms = ms;
              best = {c.first, s2};
            }
          }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (scratch) {
          cudaStreamSynchronize(st);
          cudaFree(scratch);
        }
        cudaGetLastError();
      }
      tune_store(key, best.first * 1000 + best.second);
      int kb2 = kblocks;
      bn = best.first;
      splitk = legal(best.second, kb2);
      kbps = kb2;
    }
  }
  count_launches(1 + (mi.sliced ? 2 : 0) + (splitk > 1 ? 2 : 1));
  run(bn, splitk, kbps, beta, C);
  return true;
}

}  // namespace qtt
