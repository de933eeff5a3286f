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
// threads per block: 1024 in float, 512 in double (register budget)
template <typename T>
__host__ __device__ constexpr int qr_threads() { return sizeof(T) == 4 ? 1024 : 512; }
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

// Applies H = I - t v v^T (v[j] = 1 implicit, rows > j stored in v) to the
// columns c0, c0 + (warps per block), ... (up to four, c < n) of the
// column-major X, rows >= j.  One warp; the four dot products and their
// shuffle reductions are interleaved so that their latencies overlap.
template <typename T>
__device__ __forceinline__ void reflect4(const T* v, T t, int j, int m, T* X, int c0, int n, int lane) {
  constexpr int QR_WARPS = qr_threads<T>() / 32;
  T* xc[4];
  T dot[4], xj[4];
  bool on[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = c0 + q * QR_WARPS;
    on[q] = c < n;
    xc[q] = X + (size_t)(on[q] ? c : c0) * m;
    xj[q] = on[q] ? xc[q][j] : (T)0;
    dot[q] = 0;
  }
  for (int i = j + 1 + lane; i < m; i += 32) {
    const T vi = v[i];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (on[q]) dot[q] += vi * xc[q][i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < 4; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
  for (int q = 0; q < 4; ++q) dot[q] = (dot[q] + xj[q]) * t;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (on[q]) xc[q][j] = xj[q] - dot[q];
  }
  for (int i = j + 1 + lane; i < m; i += 32) {
    const T vi = v[i];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (on[q]) xc[q][i] -= dot[q] * vi;
  }
}

// Work (global, type T): [m n] reflectors, [m n] Q when it does not fit in
// shared memory.  Shared: [m n] matrix (when it fits), then tau.
template <typename T>
__global__ void __launch_bounds__(qr_threads<T>()) qr_thin_kernel(int m, int n, const double* __restrict__ A,
                                                             double* __restrict__ Qout, T* __restrict__ Wg,
                                                             int use_smem, int* status) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  const size_t mn = (size_t)m * n;
  T* tau = (T*)(qr_smem + (use_smem ? align16(mn * sizeof(T)) : 0));
  T* W = use_smem ? (T*)qr_smem : Wg;
  constexpr int QR_THREADS = qr_threads<T>(), QR_WARPS = QR_THREADS / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (size_t e = tid; e < mn; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    W[(size_t)c * m + i] = (T)A[e];
  }
  __syncthreads();
  if (warp == 0) make_reflector(W, 0, m, tau, lane, status);
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    const T tj = tau[j];
    for (int c0 = j + 1 + warp; c0 < n; c0 += 4 * QR_WARPS) {
      if (tj != (T)0) reflect4(W + (size_t)j * m, tj, j, m, W, c0, n, lane);
      if (c0 == j + 1) {  // look-ahead: this warp holds column j + 1
        __syncwarp();
        make_reflector(W + (size_t)c0 * m, c0, m, tau, lane, status);
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
    for (int c0 = j + warp; c0 < n; c0 += 4 * QR_WARPS) reflect4(U + (size_t)j * m, tj, j, m, Q, c0, n, lane);
    __syncthreads();
  }
  for (size_t e = tid; e < mn; e += QR_THREADS) {
    const int i = (int)(e / n), c = (int)(e - (size_t)i * n);
    Qout[e] = (double)Q[(size_t)c * m + i];
  }
}

// ---------------------------------------------------------------------------
// Float QR with the matrix in registers (m <= 32 RPL, n <= 16 CPW, 512
// threads).  Thread (warp w, lane l) owns rows l + 32 k (k < RPL) of columns
// w + 16 q (q < CPW): a reflector step is RPL FMAs per owned column for the
// dot product, a warp reduction, and RPL FMAs for the update.  The reflectors
// go to shared memory, written once each, so the warps need no block-wide
// barrier: a warp waits only for the flag of the reflector it applies next.
// The owner of column j + 1 applies H_j to that column first, forms H_{j+1}
// and raises its flag before it updates its other columns, which keeps the
// chain of reflectors short (a look-ahead of one column).  Q is accumulated
// backwards in the same register layout, with no synchronisation at all.
constexpr int QRR_WARPS = 16;
constexpr int QRR_THREADS = QRR_WARPS * 32;
constexpr int QRR_SPIN_LIMIT = 1 << 22;  // polls of a reflector flag (with a short sleep) before giving up

// Reflector of the owned column q (global index c) of X (rows lane + 32 k):
// writes v (v_c = 1, zeros above c) to V[c][.] and tau[c], then raises ready[c].
template <int RPL, int CPW>
__device__ __forceinline__ void qrr_reflector(const float (&X)[RPL][CPW], int q, int c, int lane, int ldv, float* V,
                                              float* tau, volatile int* ready, int* status) {
  float s = 0.f, a = 0.f;
#pragma unroll
  for (int qq = 0; qq < CPW; ++qq) {
    if (qq != q) continue;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      if (i > c) s += X[k][qq] * X[k][qq];
      if (i == c) a = X[k][qq];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    a += __shfl_xor_sync(0xffffffffu, a, o);  // one lane holds x_c, the others 0
  }
  float t = 0.f, v0 = 1.f;
  if (s != 0.f) {
    const float mu = sqrtf(a * a + s);
    const float beta = a <= 0.f ? mu : -mu;
    t = (beta - a) / beta;
    v0 = a - beta;
  }
  float* v = V + (size_t)c * ldv;
#pragma unroll
  for (int qq = 0; qq < CPW; ++qq) {
    if (qq != q) continue;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      v[i] = i < c ? 0.f : (i == c ? 1.f : (t != 0.f ? X[k][qq] / v0 : 0.f));
    }
  }
  if (lane == 0) {
    tau[c] = t;
    if (!isfinite(t)) atomicOr(status, 1);
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence_block();
    ready[c] = 1;
  }
}

// Bounded wait for reflector j; false (and status bit 4) if it never comes.
__device__ __forceinline__ bool qrr_wait(volatile int* ready, int j, int lane, int* status) {
  int ok = 1;
  if (lane == 0) {
    int it = 0;
    while (ready[j] == 0 && it < QRR_SPIN_LIMIT) {
      __nanosleep(32);
      ++it;
    }
    ok = ready[j] != 0;
    if (!ok) atomicOr(status, 4);
    __threadfence_block();
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

template <int RPL, int CPW>
__global__ void __launch_bounds__(QRR_THREADS) qr_reg_kernel(int m, int n, const double* __restrict__ A,
                                                             double* __restrict__ Qout, int* status) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char qr_smem[];
  constexpr int LDV = 32 * RPL;
  float* V = (float*)qr_smem;        // [n][LDV] reflectors; first the input, last the output staging
  float* tau = V + (size_t)n * LDV;  // [n]
  volatile int* ready = (volatile int*)(tau + n);  // [n]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // input, column-major in shared memory, then into registers
  for (int e = tid; e < m * n; e += QRR_THREADS) {
    const int i = e / n, c = e - i * n;
    V[(size_t)c * LDV + i] = (float)A[e];
  }
  for (int c = tid; c < n; c += QRR_THREADS) ready[c] = 0;
  __syncthreads();
  float X[RPL][CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + QRR_WARPS * q;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      X[k][q] = (c < n && i < m) ? V[(size_t)c * LDV + i] : 0.f;
    }
  }
  __syncthreads();  // the input copy is dead from here on
  if (warp == 0) qrr_reflector<RPL, CPW>(X, 0, 0, lane, LDV, V, tau, ready, status);
  bool alive = true;
  for (int j = 0; j < n && alive; ++j) {
    alive = qrr_wait(ready, j, lane, status);
    if (!alive) break;
    const float t = tau[j];
    float v[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) v[k] = V[(size_t)j * LDV + lane + 32 * k];
    const int cn = j + 1;
    const bool own_next = cn < n && (cn % QRR_WARPS) == warp;
    const int qn = cn / QRR_WARPS;
    if (own_next) {  // column j + 1 first: apply H_j, then form and publish H_{j+1}
      if (t != 0.f) {
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
          if (q != qn) continue;
          float d = 0.f;
#pragma unroll
          for (int k = 0; k < RPL; ++k) d += v[k] * X[k][q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          const float f = t * d;
#pragma unroll
          for (int k = 0; k < RPL; ++k) X[k][q] -= f * v[k];
        }
      }
      qrr_reflector<RPL, CPW>(X, qn, cn, lane, LDV, V, tau, ready, status);
    }
    if (t != 0.f) {
      float dot[CPW];
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        dot[q] = 0.f;
        const int c = warp + QRR_WARPS * q;
        if (c > cn - (own_next ? 0 : 1) && c < n) {
#pragma unroll
          for (int k = 0; k < RPL; ++k) dot[q] += v[k] * X[k][q];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < CPW; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        const int c = warp + QRR_WARPS * q;
        if (c > cn - (own_next ? 0 : 1) && c < n) {
          const float f = t * dot[q];
#pragma unroll
          for (int k = 0; k < RPL; ++k) X[k][q] -= f * v[k];
        }
      }
    }
  }
  __syncthreads();  // every reflector is published and every warp is done with its columns
  // Q = H_0 ... H_{n-1} [I; 0], accumulated backwards in the same registers
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + QRR_WARPS * q;
#pragma unroll
    for (int k = 0; k < RPL; ++k) X[k][q] = (lane + 32 * k == c) ? 1.f : 0.f;
  }
  for (int j = n - 1; j >= 0; --j) {
    const float t = tau[j];
    if (t == 0.f) continue;  // uniform across the block
    float v[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) v[k] = V[(size_t)j * LDV + lane + 32 * k];
    float dot[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      dot[q] = 0.f;
      const int c = warp + QRR_WARPS * q;
      if (c >= j && c < n) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) dot[q] += v[k] * X[k][q];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < CPW; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + QRR_WARPS * q;
      if (c >= j && c < n) {
        const float f = t * dot[q];
#pragma unroll
        for (int k = 0; k < RPL; ++k) X[k][q] -= f * v[k];
      }
    }
  }
  // stage Q row-major through shared memory (the reflectors are no longer
  // read) and write it out coalesced
  __syncthreads();
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + QRR_WARPS * q;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      if (c < n && i < m) V[(size_t)i * n + c] = X[k][q];
    }
  }
  __syncthreads();
  for (int e = tid; e < m * n; e += QRR_THREADS) Qout[e] = (double)V[e];
}

template <int RPL, int CPW>
bool try_qr_reg(cudaStream_t st, int m, int n, const double* A, double* Qout, int* status) {
  if (m > 32 * RPL || n > QRR_WARPS * CPW) return false;
  const size_t smem = ((size_t)n * 32 * RPL + 2 * (size_t)n) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(qr_reg_kernel<RPL, CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)QRR_WARPS * CPW * 32 * RPL + 2 * QRR_WARPS * CPW) * sizeof(float)));
    attr = true;
  }
  launch_pdl(qr_reg_kernel<RPL, CPW>, dim3(1), dim3(QRR_THREADS), smem, st, m, n, A, Qout, status);
  return true;
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
  qr_thin_kernel<T><<<1, qr_threads<T>(), smem, st>>>(m, n, A, Qout, (T*)work, use_smem, status);
}
}  // namespace

void qr_thin(cudaStream_t st, int m, int n, const double* A, double* Qout, void* work, int prec_bits, int* status) {
  if (m <= 0 || n <= 0) return;
  if (m < n || n > 1024) {  // callers only factor tall matrices with at most 1024 columns
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  count_launches(1);
  if (prec_bits == 32) {
    if (try_qr_reg<3, 3>(st, m, n, A, Qout, status) || try_qr_reg<5, 5>(st, m, n, A, Qout, status) ||
        try_qr_reg<9, 9>(st, m, n, A, Qout, status))
      return;
    launch_qr<float>(st, m, n, A, Qout, work, status);
  }
  else
    launch_qr<double>(st, m, n, A, Qout, work, status);
}

}  // namespace qtt
