// FP64 strided batched GEMM (CUDA cores, DFMA).  Used by the plain FP64
// path for every core contraction, and by all paths for the small FP64 Gram
// matrices of the SVD truncation sweep.
//
// Tile 64 x 64 x 16, 256 threads, 4 x 4 outputs per thread spread with
// stride 16 so that a warp's shared-memory reads are conflict-free.  The
// operands are read through general (row, column, batch) strides so that
// every reshape / transpose of the contraction is a view, not a copy.
// Split-K writes partial tiles to a workspace that a second kernel reduces
// in a fixed order (deterministic).
#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) gemm_f64_kernel(int M, int N, int K, int inner, int splitk, int kchunk,
                                                      double alpha, MatView A, MatView B, double beta,
                                                      OutView C, double* ws) {
  pdl_trigger();
  pdl_wait();
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int z = blockIdx.z;
  const int b = z / splitk, ks = z - b * splitk;
  const int bo = b / inner, bi = b - bo * inner;
  const double* Ap = A.p + bo * A.so + bi * A.si;
  const double* Bp = B.p + bo * B.so + bi * B.si;
  const int k0 = ks * kchunk;
  const int k1 = min(K, k0 + kchunk);
  const bool a_mfast = (A.rs < 0 ? -A.rs : A.rs) <= (A.cs < 0 ? -A.cs : A.cs);
  const bool b_nfast = (B.cs < 0 ? -B.cs : B.cs) <= (B.rs < 0 ? -B.rs : B.rs);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int kt = k0; kt < k1; kt += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      const int idx = tid + q * NT;
      int mm, kk;
      if (a_mfast) { mm = idx % BM; kk = idx / BM; } else { kk = idx % BK; mm = idx / BK; }
      const int gm = m0 + mm, gk = kt + kk;
      As[kk][mm] = (gm < M && gk < k1) ? Ap[(long long)gm * A.rs + (long long)gk * A.cs] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      const int idx = tid + q * NT;
      int nn, kk;
      if (b_nfast) { nn = idx % BN; kk = idx / BN; } else { kk = idx % BK; nn = idx / BK; }
      const int gn = n0 + nn, gk = kt + kk;
      Bs[kk][nn] = (gn < N && gk < k1) ? Bp[(long long)gk * B.rs + (long long)gn * B.cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (ws) {
    double* W = ws + ((long long)b * splitk + ks) * (long long)M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < M && gn < N) W[(long long)gm * N + gn] = acc[i][j];
      }
  } else {
    double* Cp = C.p + bo * C.so + bi * C.si;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < M && gn < N) {
          double* c = Cp + (long long)gm * C.rs + (long long)gn * C.cs;
          *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
        }
      }
  }
}

__global__ void splitk_reduce_kernel(int M, int N, int inner, int splitk, int batch, double alpha, const double* ws,
                                     double beta, OutView C) {
  pdl_trigger();
  pdl_wait();
  const long long MN = (long long)M * N;
  const long long total = MN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / MN);
    const long long r = e - (long long)b * MN;
    const int gm = (int)(r / N), gn = (int)(r - (long long)gm * N);
    double s = 0.0;
    for (int k = 0; k < splitk; ++k) s += ws[((long long)b * splitk + k) * MN + r];
    const int bo = b / inner, bi = b - bo * inner;
    double* c = C.p + bo * C.so + bi * C.si + (long long)gm * C.rs + (long long)gn * C.cs;
    *c = (beta == 0.0) ? alpha * s : alpha * s + beta * (*c);
  }
}
__global__ void scale_out_kernel(int M, int N, int inner, int batch, double beta, OutView C) {
  pdl_trigger();
  pdl_wait();
  const long long MN = (long long)M * N;
  const long long total = MN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / MN);
    const long long r = e - (long long)b * MN;
    const int gm = (int)(r / N), gn = (int)(r - (long long)gm * N);
    const int bo = b / inner, bi = b - bo * inner;
    double* c = C.p + bo * C.so + bi * C.si + (long long)gm * C.rs + (long long)gn * C.cs;
    *c = (beta == 0.0) ? 0.0 : beta * (*c);
  }
}
}  // namespace

void splitk_reduce(cudaStream_t st, int M, int N, int inner, int splitk, int batch, double alpha, const double* ws,
                   double beta, OutView C) {
  const long long total = (long long)M * N * batch;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  launch_pdl(splitk_reduce_kernel, dim3((unsigned)blocks), dim3(256), 0, st, M, N, inner, splitk, batch, alpha,
             (const double*)ws, beta, C);
}

int gemm_split_k(int M, int N, int K, int batch) {
  const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
  if (tiles >= 152 || K < 2 * BK) return 1;
  // FP64 issues at two operations per clock per SM: spread small products
  // over about two waves of SMs, down to one k-tile per split
  long long s = (304 + tiles - 1) / tiles;
  s = s < (K / BK) ? s : (K / BK);
  if (s > 64) s = 64;
  return s < 1 ? 1 : (int)s;
}

void gemm_f64(cudaStream_t st, int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B,
              double beta, OutView C, double* ws, size_t ws_elems) {
  if (M <= 0 || N <= 0 || outer <= 0 || inner <= 0) return;
  const int batch = outer * inner;
  if (K <= 0) {  // empty contraction: C = beta * C
    const long long total = (long long)M * N * batch;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    count_launches(1);
    scale_out_kernel<<<blocks, 256, 0, st>>>(M, N, inner, batch, beta, C);
    return;
  }
  int splitk = gemm_split_k(M, N, K, batch);
  if (splitk > 1 && (ws == nullptr || (size_t)splitk * batch * (size_t)M * N > ws_elems)) splitk = 1;
  int kchunk = (K + splitk - 1) / splitk;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  splitk = (K + kchunk - 1) / kchunk;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * splitk);
  count_launches(splitk == 1 ? 1 : 2);
  if (splitk == 1) {
    launch_pdl(gemm_f64_kernel, grid, dim3(NT), 0, st, M, N, K, inner, 1, kchunk, alpha, A, B, beta, C,
               (double*)nullptr);
  } else {
    launch_pdl(gemm_f64_kernel, grid, dim3(NT), 0, st, M, N, K, inner, splitk, kchunk, alpha, A, B, beta, C, ws);
    const long long total = (long long)M * N * batch;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    launch_pdl(splitk_reduce_kernel, dim3((unsigned)blocks), dim3(256), 0, st, M, N, inner, splitk, batch, alpha,
             (const double*)ws, beta, C);
  }
}

}  // namespace qtt
