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
#include <algorithm>

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
// Products whose 64 x 64 tile grid is too small for the GPU (the bond-sized
// FP64 products: right Grams of the truncation, 136 x 136 x 272) otherwise
// need a K split and a reduction launch.  16 x 16 output tiles give them
// enough blocks instead, each thread summing its whole dot product (K in
// chunks of 32 staged through shared memory), with the strided views and
// alpha / beta of gemm_f64.
__global__ void __launch_bounds__(256) gemm_f64_t16_kernel(int M, int N, int K, int inner, double alpha, MatView A,
                                                           MatView B, double beta, OutView C) {
  pdl_trigger();
  pdl_wait();
  __shared__ double As[16][33], Bs[32][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16;
  const int b = blockIdx.z, bo = b / inner, bi = b - bo * inner;
  const double* Ap = A.p + bo * A.so + bi * A.si;
  const double* Bp = B.p + bo * B.so + bi * B.si;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int rr = e >> 5, kk = e & 31;  // As[rr][kk] = A(m0 + rr, k0 + kk)
      As[rr][kk] = (m0 + rr < M && k0 + kk < K) ? Ap[(long long)(m0 + rr) * A.rs + (long long)(k0 + kk) * A.cs] : 0.0;
      const int kb = e >> 4, cc = e & 15;  // Bs[kb][cc] = B(k0 + kb, n0 + cc)
      Bs[kb][cc] = (k0 + kb < K && n0 + cc < N) ? Bp[(long long)(k0 + kb) * B.rs + (long long)(n0 + cc) * B.cs] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (m0 + ty < M && n0 + tx < N) {
    double* c = C.p + bo * C.so + bi * C.si + (long long)(m0 + ty) * C.rs + (long long)(n0 + tx) * C.cs;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*c);
  }
}

// One Newton-Schulz step of an almost-orthonormal Q (m x n, row-major):
// out = Q (3 I - Q^T Q) / 2, in two launches.  FP64 issues at two operations
// per clock per SM, so both are sized to one wave of at most 152 blocks with
// one block per SM:
//   ns_gram_kernel: the upper-triangular 16 x 16 tiles of P = Q^T Q only (P is
//     symmetric), each over a slice of the m rows of Q (split s of S), raw
//     partial sums to P_s, written to the tile and to its mirror image;
//   ns_apply_kernel: out = Q G with G = 1.5 I - 0.5 sum_s P_s read row-wise
//     from the partials, 16 x 17 output tiles
//     (17 columns: 136 = 8 x 17 fills 136 blocks where 16 x 16 tiles would
//     make 153, one more than the SMs).
// Operand strips are staged through shared memory in chunks of 32.
constexpr int NS_T = 16;      // Gram tile, and rows of the apply tile
constexpr int NS_C = 17;      // columns of the apply tile
constexpr int NS_MAX_SPLIT = 8;

__global__ void __launch_bounds__(256) ns_gram_kernel(int m, int n, int nt, int rows_per_split,
                                                      const double* __restrict__ Q, double* __restrict__ P) {
  pdl_trigger();
  pdl_wait();
  __shared__ double A[32][NS_T + 1], B[32][NS_T + 1];
  // upper-triangular tile pair (ti <= tj) from the linear block index
  int ti = 0, rem = blockIdx.x;
  while (rem >= nt - ti) {
    rem -= nt - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const int tx = threadIdx.x & (NS_T - 1), ty = threadIdx.x / NS_T;
  const int i0 = ti * NS_T, j0 = tj * NS_T;
  const int kbeg = blockIdx.y * rows_per_split, kend = min(m, kbeg + rows_per_split);
  double acc = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * NS_T; e += blockDim.x) {
      const int kk = e / NS_T, c = e - kk * NS_T, k = k0 + kk;
      A[kk][c] = (k < kend && i0 + c < n) ? Q[(size_t)k * n + i0 + c] : 0.0;
      B[kk][c] = (k < kend && j0 + c < n) ? Q[(size_t)k * n + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = fma(A[kk][ty], B[kk][tx], acc);
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < n && j < n) {
    double* Ps = P + (size_t)blockIdx.y * n * n;
    Ps[(size_t)i * n + j] = acc;
    if (ti != tj) Ps[(size_t)j * n + i] = acc;  // the mirrored tile, so that the apply reads rows
  }
}

__global__ void __launch_bounds__(NS_T * NS_C) ns_apply_kernel(int m, int n, int splits, const double* __restrict__ Q,
                                                               const double* __restrict__ P, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  __shared__ double A[NS_T][33], B[32][NS_C + 1];
  const int tx = threadIdx.x % NS_C, ty = threadIdx.x / NS_C;
  const int r0 = blockIdx.y * NS_T, c0 = blockIdx.x * NS_C;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int e = threadIdx.x; e < NS_T * 32; e += blockDim.x) {
      const int rr = e / 32, kk = e - rr * 32;  // A[rr][kk] = Q[r0 + rr][k0 + kk]
      A[rr][kk] = (r0 + rr < m && k0 + kk < n) ? Q[(size_t)(r0 + rr) * n + k0 + kk] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * NS_C; e += blockDim.x) {
      const int kb = e / NS_C, cc = e - kb * NS_C;  // B[kb][cc] = G[k0 + kb][c0 + cc]
      const int k = k0 + kb, c = c0 + cc;
      double g = 0.0;
      if (k < n && c < n) {
        double p = 0.0;
        for (int sp = 0; sp < splits; ++sp) p += P[(size_t)sp * n * n + (size_t)k * n + c];
        g = (k == c ? 1.5 : 0.0) - 0.5 * p;
      }
      B[kb][cc] = g;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc = fma(A[ty][kk], B[kk][tx], acc);
    __syncthreads();
  }
  if (r0 + ty < m && c0 + tx < n) out[(size_t)(r0 + ty) * n + c0 + tx] = acc;
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
  // The row tiles run along grid.y (at most 65535 blocks): taller products
  // (the dense decompression of a large chain) are issued in row chunks.
  constexpr int kRowsPerCall = 1 << 19;
  if (M > kRowsPerCall) {
    for (int m0 = 0; m0 < M; m0 += kRowsPerCall) {
      MatView Ac = A;
      OutView Cc = C;
      Ac.p += (long long)m0 * A.rs;
      Cc.p += (long long)m0 * C.rs;
      gemm_f64(st, std::min(kRowsPerCall, M - m0), N, K, outer, inner, alpha, Ac, B, beta, Cc, ws, ws_elems);
    }
    return;
  }
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
  {
    const long long t16 = (long long)((M + 15) / 16) * ((N + 15) / 16) * batch;
    if (splitk > 1 && t16 >= 64 && K <= 2048 && batch <= 65535) {
      count_launches(1);
      launch_pdl(gemm_f64_t16_kernel, dim3((N + 15) / 16, (M + 15) / 16, batch), dim3(256), 0, st, M, N, K, inner, alpha,
                 A, B, beta, C);
      return;
    }
  }
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

void gemm_f64_tiles16(cudaStream_t st, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
                      OutView C) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0 || M > 65535 * 16) {  // empty contraction, or more row tiles than grid.y holds
    gemm_f64(st, M, N, K, 1, 1, alpha, A, B, beta, C, nullptr, 0);
    return;
  }
  count_launches(1);
  launch_pdl(gemm_f64_t16_kernel, dim3((N + 15) / 16, (M + 15) / 16, 1), dim3(256), 0, st, M, N, K, 1, alpha, A, B,
             beta, C);
}

void newton_schulz_step(cudaStream_t st, int m, int n, const double* Q, double* G, double* out) {
  if (m <= 0 || n <= 0) return;
  count_launches(2);
  const int nt = (n + NS_T - 1) / NS_T;
  const int pairs = nt * (nt + 1) / 2;
  const int chunks = (m + 31) / 32;  // K slices come in chunks of 32 rows
  int splits = 152 / pairs;
  splits = std::max(1, std::min({splits, chunks, NS_MAX_SPLIT}));
  const int rows = ((chunks + splits - 1) / splits) * 32;
  splits = (m + rows - 1) / rows;
  launch_pdl_chain(ns_gram_kernel, dim3((unsigned)pairs, (unsigned)splits), dim3(256), 0, st, m, n, nt, rows, Q, G);
  const unsigned bc = (unsigned)((n + NS_C - 1) / NS_C), bm = (unsigned)((m + NS_T - 1) / NS_T);
  launch_pdl_chain(ns_apply_kernel, dim3(bc, bm), dim3(NS_T * NS_C), 0, st, m, n, splits, Q, (const double*)G, out);
}

}  // namespace qtt
