// Contractions with an operator (MPO) bond: batched GEMMs whose M is at most
// 32 and K at most 64 -- the MPO core applied to a site tensor in the sketch
// and zip-up passes (operator bond w <= ~26 for the stencil operators).  These
// are memory-bound (a few FLOPs per loaded element), so they run on the CUDA
// cores without packing: one thread per (batch entry, column n) keeps all M
// outputs in registers, the small A[b] sits in shared memory.  The arithmetic
// type is double for the FP64 form and float (round to nearest, unbiased) for
// the reduced-precision forms; inputs and outputs are FP64.
#include <cstdint>

#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int SG_THREADS = 128;
constexpr int SG_MAXM = 32, SG_MAXK = 64;

// double -> float, round to nearest even, by bits (the FP64 pipe issues two
// operations per clock per SM); below the float normal range -> 0.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFull);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned long long rem = m & 0x1FFFFFFFull;
  uint32_t r = ((uint32_t)fe << 23) | (uint32_t)(m >> 29);
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1u))) r += 1u;
  return __uint_as_float(sign | r);
}

// float -> double, exact, by bits (denormals through the hardware conversion).
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  if (e == 0u) return (b & 0x7FFFFFu) ? (double)f : __longlong_as_double((long long)sign);
  const unsigned long long de = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

template <typename T>
__device__ __forceinline__ T to_t(double x) {
  if constexpr (sizeof(T) == 4)
    return d2f_bits(x);
  else
    return x;
}
template <typename T>
__device__ __forceinline__ double to_d(T x) {
  if constexpr (sizeof(T) == 4)
    return f2d_bits(x);
  else
    return x;
}

template <typename T, int MT>
__global__ void __launch_bounds__(SG_THREADS) small_gemm_kernel(int M, int N, int K, int inner, double alpha,
                                                                MatView A, MatView B, double beta, OutView C) {
  pdl_trigger();
  pdl_wait();
  __shared__ T As[SG_MAXM * SG_MAXK];
  const int b = blockIdx.y;
  const int bo = b / inner, bi = b - bo * inner;
  const double* Ab = A.p + bo * A.so + bi * A.si;
  for (int x = threadIdx.x; x < M * K; x += SG_THREADS) {
    const int m = x / K, k = x - m * K;
    As[x] = to_t<T>(Ab[(long long)m * A.rs + (long long)k * A.cs]);
  }
  __syncthreads();
  const int n = blockIdx.x * SG_THREADS + threadIdx.x;
  if (n >= N) return;
  const double* Bb = B.p + bo * B.so + bi * B.si + (long long)n * B.cs;
  T acc[MT];
#pragma unroll
  for (int m = 0; m < MT; ++m) acc[m] = (T)0;
  for (int k = 0; k < K; ++k) {
    const T bk = to_t<T>(Bb[(long long)k * B.rs]);
#pragma unroll
    for (int m = 0; m < MT; ++m)
      if (m < M) acc[m] += As[m * K + k] * bk;
  }
  double* Cb = C.p + bo * C.so + bi * C.si + (long long)n * C.cs;
  const bool plain = (alpha == 1.0 && beta == 0.0);
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    if (m < M) {
      double* c = Cb + (long long)m * C.rs;
      const double v = to_d<T>(acc[m]);
      *c = plain ? v : alpha * v + (beta == 0.0 ? 0.0 : beta * (*c));
    }
  }
}

template <typename T>
void launch_small(cudaStream_t st, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
                  double beta, OutView C) {
  const dim3 grid((unsigned)((N + SG_THREADS - 1) / SG_THREADS), (unsigned)(outer * inner));
  if (M <= 8)
    launch_pdl(small_gemm_kernel<T, 8>, grid, dim3(SG_THREADS), 0, st, M, N, K, inner, alpha, A, B, beta, C);
  else if (M <= 16)
    launch_pdl(small_gemm_kernel<T, 16>, grid, dim3(SG_THREADS), 0, st, M, N, K, inner, alpha, A, B, beta, C);
  else
    launch_pdl(small_gemm_kernel<T, 32>, grid, dim3(SG_THREADS), 0, st, M, N, K, inner, alpha, A, B, beta, C);
}
}  // namespace

bool small_gemm_fits(int M, int N, int K, int outer, int inner) {
  return M >= 1 && M <= SG_MAXM && K >= 1 && K <= SG_MAXK && N >= 1 && (long long)outer * inner <= 65535;
}

void small_gemm(cudaStream_t st, bool fp32, int M, int N, int K, int outer, int inner, double alpha, MatView A,
                MatView B, double beta, OutView C) {
  count_launches(1);
  if (fp32)
    launch_small<float>(st, M, N, K, outer, inner, alpha, A, B, beta, C);
  else
    launch_small<double>(st, M, N, K, outer, inner, alpha, A, B, beta, C);
}

}  // namespace qtt
