// Thin Householder QR of a tall matrix in one thread block.
//
// Used by the randomized rounding (left-to-right sweep): the sketch
// Y = T W of the site tensor is orthonormalised, Y = Q R, and Q becomes the
// new left-orthonormal core (the QR decompositions that keep the MPS in
// canonical form, Sec. "Computational complexity").  Householder reflections
// are backward stable, so the error of Q is linear in the unit roundoff of
// the arithmetic (float for the reduced-precision forms, double otherwise).
//
// Column j is reflected by H_j = I - tau_j v_j v_j^T with v_j = (x - beta e_j)
// / (x_j - beta) (so v_j[j] = 1 and |v_j[i]| <= 1), x the rows >= j of the
// current column j, beta = -sign(x_j) ||x|| and tau_j = (beta - x_j) / beta in
// [1, 2].  Only Q is produced (R is not needed by the caller).
//
// Factorisation: one barrier per column.  Warps own trailing columns (lanes
// run down the rows, so the column-major working copy is read contiguously).
// While applying H_j, the warp that updates column j + 1 also forms H_{j+1}
// (norm, tau, scaled v) -- a one-column look-ahead -- so that after the
// barrier every thread finds tau_{j+1} and v_{j+1} ready.  Q = H_0 ... H_{n-1}
// [I; 0] is then accumulated backwards, one barrier per reflector: applying
// H_j touches only the columns c >= j of the partial product.
#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int QR_THREADS = 1024;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr size_t kQrSmemLimit = 200 * 1024;

template <typename T>
__device__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Forms the reflector of column c (rows >= c) in place: rows > c become v,
// tau[c] is set.  Executed by one warp.
template <typename T>
__device__ void make_reflector(T* wc, int c, int m, T* tau, int lane, int* status) {
  T s = 0;
  for (int i = c + 1 + lane; i < m; i += 32) s += wc[i] * wc[i];
  s = warp_sum(s);
  const T alpha = wc[c];
  T t = 0, v0 = 1;
  if (s != (T)0) {
    const T mu = sqrt(alpha * alpha + s);
    const T beta = alpha <= (T)0 ? mu : -mu;
    t = (beta - alpha) / beta;
    v0 = alpha - beta;  // |v0| >= mu >= |x_i|, so x_i / v0 cannot overflow
    for (int i = c + 1 + lane; i < m; i += 32) wc[i] = wc[i] / v0;
  }
  if (lane == 0) {
    tau[c] = t;
    if (!isfinite((double)t)) atomicOr(status, 1);
  }
}

// Work (global, type T): [m n] reflectors, [m n] Q when it does not fit in
// shared memory.  Shared: [m n] matrix (when it fits), then tau.
template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_thin_kernel(int m, int n, const double* __restrict__ A,
                                                             double* __restrict__ Qout, T* __restrict__ Wg,
                                                             int use_smem, int* status) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  const size_t mn = (size_t)m * n;
  T* tau = (T*)(qr_smem + (use_smem ? align16(mn * sizeof(T)) : 0));
  T* W = use_smem ? (T*)qr_smem : Wg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (size_t e = tid; e < mn; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    W[(size_t)c * m + i] = (T)A[e];
  }
  __syncthreads();
  if (warp == 0) make_reflector(W, 0, m, tau, lane, status);
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    const T* vj = W + (size_t)j * m;
    const T tj = tau[j];
    for (int c = j + 1 + warp; c < n; c += QR_WARPS) {
      T* wc = W + (size_t)c * m;
      if (tj != (T)0) {
        const T wcj = wc[j];
        T dot = 0;
        for (int i = j + 1 + lane; i < m; i += 32) dot += vj[i] * wc[i];
        dot = (warp_sum(dot) + wcj) * tj;
        if (lane == 0) wc[j] = wcj - dot;
        for (int i = j + 1 + lane; i < m; i += 32) wc[i] -= dot * vj[i];
      }
      if (c == j + 1) {
        __syncwarp();
        make_reflector(wc, c, m, tau, lane, status);  // look-ahead
      }
    }
    __syncthreads();
  }
  const T* U = Wg;
  T* Q = Wg + mn;
  if (use_smem) {  // move the reflectors to global memory and accumulate Q in shared memory
    for (size_t e = tid; e < mn; e += QR_THREADS) Wg[e] = W[e];
    Q = W;
    __syncthreads();
  }
  for (size_t e = tid; e < mn; e += QR_THREADS) {
    const int c = (int)(e / m), i = (int)(e - (size_t)c * m);
    Q[e] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == (T)0) continue;  // uniform across the block
    const T* vj = U + (size_t)j * m;
    for (int c = j + warp; c < n; c += QR_WARPS) {
      T* qc = Q + (size_t)c * m;
      const T qcj = qc[j];
      T dot = 0;
      for (int i = j + 1 + lane; i < m; i += 32) dot += vj[i] * qc[i];
      dot = (warp_sum(dot) + qcj) * tj;
      if (lane == 0) qc[j] = qcj - dot;
      for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= dot * vj[i];
    }
    __syncthreads();
  }
  for (size_t e = tid; e < mn; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    Qout[e] = (double)Q[(size_t)c * m + i];
  }
}

template <typename T>
void launch_qr(cudaStream_t st, int m, int n, const double* A, double* Qout, void* work, int* status) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(qr_thin_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kQrSmemLimit + 3 * 1024 * sizeof(double) + 64));
    attr = true;
  }
  const size_t wbytes = (size_t)m * n * sizeof(T);
  const int use_smem = wbytes <= kQrSmemLimit ? 1 : 0;
  const size_t smem = (use_smem ? align16(wbytes) : 0) + (size_t)n * sizeof(T);
  qr_thin_kernel<T><<<1, QR_THREADS, smem, st>>>(m, n, A, Qout, (T*)work, use_smem, status);
}
}  // namespace

void qr_thin(cudaStream_t st, int m, int n, const double* A, double* Qout, void* work, int prec_bits, int* status) {
  if (m <= 0 || n <= 0) return;
  if (m < n || n > 1024) {  // callers only factor tall matrices with at most 1024 columns
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  count_launches(1);
  if (prec_bits == 32)
    launch_qr<float>(st, m, n, A, Qout, work, status);
  else
    launch_qr<double>(st, m, n, A, Qout, work, status);
}

}  // namespace qtt
