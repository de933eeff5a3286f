// Thin Householder QR of a tall matrix in one thread block.
//
// Used by the randomized rounding (left-to-right sweep): the sketch
// Y = T W of the site tensor is orthonormalised, Y = Q R, and Q becomes the
// new left-orthonormal core (paper: "Computational complexity" lists QR
// decompositions that keep the MPS in canonical form).  Householder
// reflections are backward stable, so the error of Q is linear in the unit
// roundoff of T (float for the reduced-precision forms, double otherwise).
//
// Layout: the working copy is column-major (column j contiguous) so that the
// warp-per-column reductions and updates read contiguous memory.
#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int QR_THREADS = 512;

template <typename T>
__device__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_thin_kernel(int m, int n, const double* __restrict__ A,
                                                             double* __restrict__ Qout, T* __restrict__ W,
                                                             int* status) {
  // W: [n][m] reflectors / R (column-major), Q: [n][m] (column-major)
  T* Q = W + (size_t)m * n;
  T* tau = Q + (size_t)m * n;
  __shared__ T s_beta, s_tau, s_v0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = QR_THREADS / 32;
  for (size_t e = tid; e < (size_t)m * n; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    W[(size_t)c * m + i] = (T)A[e];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    T* wj = W + (size_t)j * m;
    if (warp == 0) {
      T s = 0;
      for (int i = j + 1 + lane; i < m; i += 32) s += wj[i] * wj[i];
      s = warp_sum(s);
      if (lane == 0) {
        const T alpha = wj[j];
        if (s == (T)0) {
          s_tau = 0;
          s_v0 = 1;
          s_beta = alpha;
        } else {
          const T mu = sqrt(alpha * alpha + s);
          const T beta = alpha <= (T)0 ? mu : -mu;
          s_tau = (beta - alpha) / beta;
          s_v0 = alpha - beta;
          s_beta = beta;
        }
        tau[j] = s_tau;
        if (!isfinite((double)s_tau)) atomicOr(status, 1);
      }
    }
    __syncthreads();
    const T tj = s_tau;
    if (tj != (T)0) {
      const T inv = (T)1 / s_v0;
      for (int i = j + 1 + tid; i < m; i += QR_THREADS) wj[i] *= inv;
    }
    __syncthreads();
    if (tid == 0) wj[j] = s_beta;
    if (tj != (T)0) {
      for (int c = j + 1 + warp; c < n; c += nwarps) {
        T* wc = W + (size_t)c * m;
        T dot = 0;
        for (int i = j + 1 + lane; i < m; i += 32) dot += wj[i] * wc[i];
        dot = warp_sum(dot) + wc[j];
        dot *= tj;
        if (lane == 0) wc[j] -= dot;
        for (int i = j + 1 + lane; i < m; i += 32) wc[i] -= dot * wj[i];
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{n-1} [I; 0]
  for (size_t e = tid; e < (size_t)m * n; e += QR_THREADS) {
    const int c = (int)(e / m), i = (int)(e - (size_t)c * m);
    Q[e] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == (T)0) continue;
    const T* wj = W + (size_t)j * m;
    for (int c = j + warp; c < n; c += nwarps) {
      T* qc = Q + (size_t)c * m;
      T dot = 0;
      for (int i = j + 1 + lane; i < m; i += 32) dot += wj[i] * qc[i];
      dot = warp_sum(dot) + qc[j];
      dot *= tj;
      if (lane == 0) qc[j] -= dot;
      for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= dot * wj[i];
    }
    __syncthreads();
  }
  for (size_t e = tid; e < (size_t)m * n; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    Qout[e] = (double)Q[(size_t)c * m + i];
  }
}
}  // namespace

void qr_thin(cudaStream_t st, int m, int n, const double* A, double* Qout, void* work, int prec_bits, int* status) {
  if (m <= 0 || n <= 0) return;
  if (m < n) {  // callers only factor tall matrices
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  count_launches(1);
  if (prec_bits == 32)
    qr_thin_kernel<float><<<1, QR_THREADS, 0, st>>>(m, n, A, Qout, (float*)work, status);
  else
    qr_thin_kernel<double><<<1, QR_THREADS, 0, st>>>(m, n, A, Qout, (double*)work, status);
}

}  // namespace qtt
