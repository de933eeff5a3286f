// Tensor-core (tcgen05) GEMM for the reduced-precision contraction forms.
//
// C[b] = alpha * A[b] * B[b] + beta * C[b] with FP64 operand views (the same
// MatView / OutView as the FP64 kernel).  Operands are first packed into
// K-major, zero-padded buffers of the tensor-core input type:
//   BF16X3 : A = A_hi + A_lo, B = B_hi + B_lo (bf16 each),
//            A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi  (3 MMAs, kind::f16)
//   TF32   : one MMA, kind::tf32
//   TF32X3 : A = A_hi + A_lo (tf32 each), 3 MMAs, kind::tf32
//   BF16   : one MMA, kind::f16
// and accumulated in FP32 in tensor memory.
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

#include <cstdio>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <string>

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

template <int MODE>
struct ModeTraits;
template <>
struct ModeTraits<TC_BF16X3> {
  static constexpr bool tf32 = false;
  static constexpr int nops = 2, nmma = 3, esize = 2;
};
template <>
struct ModeTraits<TC_BF16> {
  static constexpr bool tf32 = false;
  static constexpr int nops = 1, nmma = 1, esize = 2;
};
template <>
struct ModeTraits<TC_TF32> {
  static constexpr bool tf32 = true;
  static constexpr int nops = 1, nmma = 1, esize = 4;
};
template <>
struct ModeTraits<TC_TF32X3> {
  static constexpr bool tf32 = true;
  static constexpr int nops = 2, nmma = 3, esize = 4;
};

template <int BN>
struct BnTraits {
  static constexpr int tmem_cols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

template <int MODE, int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1, int M, int N,
                   int kblocks, int kb_per_split, int splitk, int inner, double alpha, double beta, OutView C,
                   double* ws, int* err) {
  using Tr = ModeTraits<MODE>;
  constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
  constexpr int STAGE_BYTES = Tr::nops * (A_BYTES + B_BYTES);
  constexpr uint32_t IDESC = make_idesc(Tr::tf32 ? 2u : 1u, (uint32_t)BN);
  constexpr int TMEM_COLS = BnTraits<BN>::tmem_cols;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int z = blockIdx.z;
  const int b = z / splitk, ks = z - b * splitk;
  const int kb0 = ks * kb_per_split;
  const int kb1 = min(kblocks, kb0 + kb_per_split);

  if (threadIdx.x == 0) {
    s_abort = 0;
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

  if (warp == 0 && lane == 0) {
    // TMA producer
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
      tma_load_3d(st, &tmA0, &full[s], kx, m0, b);
      tma_load_3d(st + Tr::nops * A_BYTES, &tmB0, &full[s], kx, n0, b);
      if (Tr::nops == 2) {
        tma_load_3d(st + A_BYTES, &tmA1, &full[s], kx, m0, b);
        tma_load_3d(st + Tr::nops * A_BYTES + B_BYTES, &tmB1, &full[s], kx, n0, b);
      }
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
      const uint32_t a0 = st, a1 = st + A_BYTES;
      const uint32_t b0 = st + Tr::nops * A_BYTES, b1 = b0 + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per 128-byte row
        const uint32_t off = kk * 32;
        const uint32_t acc0 = (kb > kb0 || kk > 0) ? 1u : 0u;
        mma_issue<Tr::tf32>(tmem, desc_sw128(a0 + off), desc_sw128(b0 + off), IDESC, acc0);
        if (Tr::nmma == 3) {
          mma_issue<Tr::tf32>(tmem, desc_sw128(a0 + off), desc_sw128(b1 + off), IDESC, 1u);
          mma_issue<Tr::tf32>(tmem, desc_sw128(a1 + off), desc_sw128(b0 + off), IDESC, 1u);
        }
      }
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(done);
  }
  __syncwarp();
  // epilogue: every warp waits for the accumulator
  bool have = mbar_wait(done, 0);
  if (!have) atomicOr(err, 16);
  __syncthreads();
  have = have && (s_abort == 0) && (kb1 > kb0);
  tc_fence_after();
  if (have) {
    const int row = m0 + warp * 32 + lane;
    const int bo = b / inner, bi = b - bo * inner;
    double* Cb = C.p + bo * C.so + bi * C.si;
    double* W = ws ? ws + ((long long)b * splitk + ks) * (long long)M * N : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tmem_ld_wait();
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) {
            const double v = (double)__uint_as_float(r[j]);
            if (W) {
              W[(long long)row * N + col] = v;
            } else {
              double* c = Cb + (long long)row * C.rs + (long long)col * C.cs;
              *c = (beta == 0.0) ? alpha * v : alpha * v + beta * (*c);
            }
          }
        }
      }
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

template <int MODE>
__global__ void pack_kernel(const double* p, long long rstr, long long kstr, long long so, long long si, int inner,
                            int rows, int K, int rows_pad, int k_pad, long long batch, void* out0, void* out1) {
  const long long per = (long long)rows_pad * k_pad;
  const long long total = per * batch;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long b = x / per;
    const long long rk = x - b * per;
    const int r = (int)(rk / k_pad), k = (int)(rk - (long long)r * k_pad);
    double v = 0.0;
    if (r < rows && k < K) {
      const long long bo = b / inner, bi = b - bo * inner;
      v = p[bo * so + bi * si + (long long)r * rstr + (long long)k * kstr];
    }
    if (MODE == TC_BF16X3 || MODE == TC_BF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
      ((__nv_bfloat16*)out0)[x] = h;
      if (MODE == TC_BF16X3) ((__nv_bfloat16*)out1)[x] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    } else if (MODE == TC_TF32) {
      ((float*)out0)[x] = to_tf32((float)v);
    } else {
      const float h = to_tf32((float)v);
      ((float*)out0)[x] = h;
      ((float*)out1)[x] = to_tf32((float)(v - (double)h));
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
               long long batch, double alpha, double beta, OutView C, double* ws, int* err) {
  using Tr = ModeTraits<MODE>;
  constexpr int SMEM = STAGES * Tr::nops * (BM * 128 + BN * 128) + 1024 + 256;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_gemm_kernel<MODE, BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    attr = true;
  }
  const CUtensorMap a0 = make_map(pk.a0, Tr::esize, pk.k_pad, pk.m_pad, batch, BM);
  const CUtensorMap a1 = make_map(Tr::nops == 2 ? pk.a1 : pk.a0, Tr::esize, pk.k_pad, pk.m_pad, batch, BM);
  const CUtensorMap b0 = make_map(pk.b0, Tr::esize, pk.k_pad, pk.n_pad, batch, BN);
  const CUtensorMap b1 = make_map(Tr::nops == 2 ? pk.b1 : pk.b0, Tr::esize, pk.k_pad, pk.n_pad, batch, BN);
  dim3 grid(pk.n_pad / BN, pk.m_pad / BM, (unsigned)(batch * splitk));
  tc_gemm_kernel<MODE, BN, STAGES><<<grid, TC_THREADS, SMEM, st>>>(a0, a1, b0, b1, M, N, kblocks, kbps, splitk, inner,
                                                                    alpha, beta, C, ws, err);
}

template <int MODE>
void launch_pack(cudaStream_t st, const MatView& v, long long rstr, long long kstr, int inner, int rows, int K,
                 int rows_pad, int k_pad, long long batch, void* o0, void* o1) {
  const long long total = (long long)rows_pad * k_pad * batch;
  long long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pack_kernel<MODE><<<(int)blocks, 256, 0, st>>>(v.p, rstr, kstr, v.so, v.si, inner, rows, K, rows_pad, k_pad, batch,
                                                o0, o1);
}

int choose_bn(int N) {
  // smallest padded width; ties go to the wider tile
  const int cands[4] = {256, 160, 128, 64};
  int best = 128;
  long long bestpad = 1LL << 60;
  for (int c : cands) {
    const long long pad = (long long)((N + c - 1) / c) * c;
    if (pad < bestpad) {
      bestpad = pad;
      best = c;
    }
  }
  return best;
}

}  // namespace

int tc_mode_esize(int mode) { return (mode == TC_TF32 || mode == TC_TF32X3) ? 4 : 2; }
int tc_mode_nops(int mode) { return (mode == TC_BF16X3 || mode == TC_TF32X3) ? 2 : 1; }

size_t tc_workspace_bytes(int M, int N, int K, long long batch, int mode) {
  const int es = tc_mode_esize(mode), nops = tc_mode_nops(mode);
  const int bn = choose_bn(N);
  const long long kb = 128 / es;
  const long long k_pad = (K + kb - 1) / kb * kb;
  const long long m_pad = (M + BM - 1) / BM * BM;
  const long long n_pad = (N + bn - 1) / bn * bn;
  return (size_t)(nops * (m_pad + n_pad) * k_pad * batch * es) + 4096;
}

bool gemm_tc(cudaStream_t st, int mode, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
             double beta, OutView C, void* pack_ws, size_t pack_bytes, double* ws, size_t ws_elems, int* err,
             int max_kb_per_split) {
  if (M <= 0 || N <= 0 || K <= 0 || outer <= 0 || inner <= 0) return false;
  load_encode();
  const long long batch = (long long)outer * inner;
  if (batch > 65535) return false;
  const int es = tc_mode_esize(mode), nops = tc_mode_nops(mode);
  const int bn = choose_bn(N);
  TcPacked pk;
  const int kb = 128 / es;
  pk.k_pad = (K + kb - 1) / kb * kb;
  pk.m_pad = (M + BM - 1) / BM * BM;
  pk.n_pad = (N + bn - 1) / bn * bn;
  const size_t a_bytes = (size_t)pk.m_pad * pk.k_pad * batch * es;
  const size_t b_bytes = (size_t)pk.n_pad * pk.k_pad * batch * es;
  const size_t need = nops * (a_bytes + b_bytes);
  if (need + 1024 > pack_bytes) return false;
  uint8_t* base = (uint8_t*)(((uintptr_t)pack_ws + 255) & ~(uintptr_t)255);
  auto carve = [&](size_t n) {
    uint8_t* p = base;
    base += (n + 255) & ~(size_t)255;
    return (void*)p;
  };
  pk.a0 = carve(a_bytes);
  pk.a1 = nops == 2 ? carve(a_bytes) : nullptr;
  pk.b0 = carve(b_bytes);
  pk.b1 = nops == 2 ? carve(b_bytes) : nullptr;
  // A(m, k) = A.p[m * rs + k * cs]; B is packed as B^T: (n, k) = B.p[k * rs + n * cs]
  switch (mode) {
    case TC_BF16X3:
      launch_pack<TC_BF16X3>(st, A, A.rs, A.cs, inner, M, K, pk.m_pad, pk.k_pad, batch, pk.a0, pk.a1);
      launch_pack<TC_BF16X3>(st, B, B.cs, B.rs, inner, N, K, pk.n_pad, pk.k_pad, batch, pk.b0, pk.b1);
      break;
    case TC_BF16:
      launch_pack<TC_BF16>(st, A, A.rs, A.cs, inner, M, K, pk.m_pad, pk.k_pad, batch, pk.a0, nullptr);
      launch_pack<TC_BF16>(st, B, B.cs, B.rs, inner, N, K, pk.n_pad, pk.k_pad, batch, pk.b0, nullptr);
      break;
    case TC_TF32:
      launch_pack<TC_TF32>(st, A, A.rs, A.cs, inner, M, K, pk.m_pad, pk.k_pad, batch, pk.a0, nullptr);
      launch_pack<TC_TF32>(st, B, B.cs, B.rs, inner, N, K, pk.n_pad, pk.k_pad, batch, pk.b0, nullptr);
      break;
    default:
      launch_pack<TC_TF32X3>(st, A, A.rs, A.cs, inner, M, K, pk.m_pad, pk.k_pad, batch, pk.a0, pk.a1);
      launch_pack<TC_TF32X3>(st, B, B.cs, B.rs, inner, N, K, pk.n_pad, pk.k_pad, batch, pk.b0, pk.b1);
      break;
  }
  const int kblocks = pk.k_pad / kb;
  // split K when the tile grid is small
  const long long tiles = (long long)(pk.m_pad / BM) * (pk.n_pad / bn) * batch;
  int splitk = 1;
  if (tiles < 152 && kblocks >= 4) {
    long long s = (2 * 152 + tiles - 1) / tiles;
    if (s > kblocks / 2) s = kblocks / 2;
    if (s > 64) s = 64;
    if (s < 1) s = 1;
    splitk = (int)s;
    if (ws == nullptr || (size_t)splitk * batch * (size_t)M * N > ws_elems) splitk = 1;
  }
  int kbps = (kblocks + splitk - 1) / splitk;
  if (max_kb_per_split > 0 && kbps > max_kb_per_split && ws != nullptr &&
      (size_t)((kblocks + max_kb_per_split - 1) / max_kb_per_split) * batch * (size_t)M * N <= ws_elems)
    kbps = max_kb_per_split;
  splitk = (kblocks + kbps - 1) / kbps;
  if ((long long)splitk * batch > 65535) {
    splitk = 1;
    kbps = kblocks;
  }
  double* wsp = splitk > 1 ? ws : nullptr;
  count_launches(2 + (splitk > 1 ? 2 : 1));
#define QTT_TC_LAUNCH(MODE_, BN_, ST_) \
  launch_tc<MODE_, BN_, ST_>(st, pk, M, N, kblocks, kbps, splitk, inner, batch, alpha, beta, C, wsp, err)
#define QTT_TC_BN(MODE_, S256, S160, S128, S64)    \
  switch (bn) {                                    \
    case 256: QTT_TC_LAUNCH(MODE_, 256, S256); break; \
    case 160: QTT_TC_LAUNCH(MODE_, 160, S160); break; \
    case 128: QTT_TC_LAUNCH(MODE_, 128, S128); break; \
    default: QTT_TC_LAUNCH(MODE_, 64, S64); break;    \
  }
  switch (mode) {
    case TC_BF16X3: QTT_TC_BN(TC_BF16X3, 2, 3, 3, 4); break;
    case TC_BF16: QTT_TC_BN(TC_BF16, 4, 4, 6, 8); break;
    case TC_TF32: QTT_TC_BN(TC_TF32, 4, 4, 6, 8); break;
    default: QTT_TC_BN(TC_TF32X3, 2, 3, 3, 4); break;
  }
#undef QTT_TC_BN
#undef QTT_TC_LAUNCH
  if (splitk > 1) splitk_reduce(st, M, N, inner, splitk, (int)batch, alpha, ws, beta, C);
  return true;
}

}  // namespace qtt
