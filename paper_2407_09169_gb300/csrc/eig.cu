// Symmetric eigen-decomposition in one thread block: Householder reduction to
// tridiagonal form, implicit-shift QL iteration, back-transformation of the
// leading k eigenvectors.
//
// Used by the SVD truncation sweep (paper: "Matrix product state algorithm" --
// the bond dimension is limited to chi with the singular value
// decomposition): for the bond matrix M the Gram G = M M^T = U diag(lam) U^T
// gives the left singular vectors and lam = sigma^2.
//
// Parallel layout: the reduction uses warp-per-row matrix-vector products and
// a block-wide rank-2 update; the QL iteration's scalar recurrence runs in
// thread 0, which records each sweep's Givens rotations, and all threads then
// apply them to their own rows of the eigenvector matrix; the back-transform
// is warp-per-eigenvector.  Every loop is bounded (QL: at most 60 sweeps per
// eigenvalue, reported through the status word).
#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int EIG_THREADS = 512;
constexpr int EIG_MAXN = 1024;

template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static __device__ double v() { return 2.220446049250313e-16; }
};
template <>
struct Eps<float> {
  static __device__ float v() { return 1.1920929e-7f; }
};

template <typename T>
__device__ T warp_sum_e(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(EIG_THREADS) eig_sym_kernel(int n, int k, const double* __restrict__ G,
                                                              double* __restrict__ Uout, double* __restrict__ lam,
                                                              T* __restrict__ work, int* status) {
  T* A = work;                        // n x n, row-major (row j > ... holds reflector j)
  T* Z = A + (size_t)n * n;           // n x n eigenvectors of the tridiagonal (columns)
  T* ZS = Z + (size_t)n * n;          // k x n selected eigenvectors (rows)
  T* vb = ZS + (size_t)n * n;         // n
  T* pb = vb + n;                     // n
  T* wb = pb + n;                     // n
  __shared__ T d[EIG_MAXN], e[EIG_MAXN], tauv[EIG_MAXN], rc[EIG_MAXN], rs[EIG_MAXN];
  __shared__ int order[EIG_MAXN];
  __shared__ T s_tau, s_v0, s_K;
  __shared__ int s_lo, s_hi, s_done;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = EIG_THREADS / 32;

  for (size_t x = tid; x < (size_t)n * n; x += EIG_THREADS) {
    const int i = (int)(x / n), c = (int)(x - (size_t)i * n);
    A[x] = (T)(0.5 * (G[x] + G[(size_t)c * n + i]));
    Z[x] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();

  // ---- Householder tridiagonalisation (reflector j zeroes row/column j beyond j+1)
  for (int j = 0; j + 2 < n; ++j) {
    T* Aj = A + (size_t)j * n;
    if (warp == 0) {
      T s = 0;
      for (int c = j + 2 + lane; c < n; c += 32) s += Aj[c] * Aj[c];
      s = warp_sum_e(s);
      if (lane == 0) {
        const T alpha = Aj[j + 1];
        d[j] = Aj[j];
        if (s == (T)0) {
          s_tau = 0;
          s_v0 = 1;
          e[j] = alpha;
        } else {
          const T mu = sqrt(alpha * alpha + s);
          const T beta = alpha <= (T)0 ? mu : -mu;
          s_tau = (beta - alpha) / beta;
          s_v0 = alpha - beta;
          e[j] = beta;
        }
        tauv[j] = s_tau;
      }
    }
    __syncthreads();
    const T tau = s_tau;
    if (tau == (T)0) {  // uniform branch: every thread read the same shared value
      __syncthreads();  // s_tau is rewritten by the next step
      continue;
    }
    {
      const T inv = (T)1 / s_v0;
      for (int c = j + 2 + tid; c < n; c += EIG_THREADS) {
        const T v = Aj[c] * inv;
        Aj[c] = v;
        vb[c] = v;
      }
      if (tid == 0) vb[j + 1] = (T)1;
    }
    __syncthreads();
    // p = tau * A22 v
    for (int i = j + 1 + warp; i < n; i += nwarps) {
      const T* Ai = A + (size_t)i * n;
      T acc = 0;
      for (int c = j + 1 + lane; c < n; c += 32) acc += Ai[c] * vb[c];
      acc = warp_sum_e(acc);
      if (lane == 0) pb[i] = tau * acc;
    }
    __syncthreads();
    if (warp == 0) {
      T acc = 0;
      for (int i = j + 1 + lane; i < n; i += 32) acc += pb[i] * vb[i];
      acc = warp_sum_e(acc);
      if (lane == 0) s_K = (T)0.5 * tau * acc;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += EIG_THREADS) wb[i] = pb[i] - s_K * vb[i];
    __syncthreads();
    const int m = n - j - 1;
    for (size_t x = tid; x < (size_t)m * m; x += EIG_THREADS) {
      const int i = j + 1 + (int)(x / m), c = j + 1 + (int)(x % m);
      A[(size_t)i * n + c] -= vb[i] * wb[c] + wb[i] * vb[c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
      e[n - 2] = A[(size_t)(n - 2) * n + (n - 1)];
      tauv[n - 2] = 0;
    }
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0;
    tauv[n - 1] = 0;
  }
  __syncthreads();

  // ---- implicit QL on (d, e); thread 0 runs the recurrence, all apply rotations
  int l = 0, iter = 0;
  bool start = true;
  T f = 0, tst1 = 0;
  const T eps = Eps<T>::v();
  for (;;) {
    if (tid == 0) {
      s_done = 1;
      while (l < n) {
        if (start) {
          const T h = fabs(d[l]) + fabs(e[l]);
          tst1 = h > tst1 ? h : tst1;
          iter = 0;
          start = false;
        }
        int m = l;
        while (m < n - 1 && fabs(e[m]) > eps * tst1) ++m;
        if (m == l || iter >= 60) {
          if (m != l) atomicOr(status, 2);
          d[l] += f;
          e[l] = 0;
          ++l;
          start = true;
          continue;
        }
        ++iter;
        T g = d[l];
        T p = (d[l + 1] - g) / ((T)2 * e[l]);
        T r = hypot(p, (T)1);
        if (p < 0) r = -r;
        d[l] = e[l] / (p + r);
        d[l + 1] = e[l] * (p + r);
        const T dl1 = d[l + 1];
        T h = g - d[l];
        for (int i = l + 2; i < n; ++i) d[i] -= h;
        f += h;
        p = d[m];
        T c = 1, c2 = 1, c3 = 1, s = 0, s2 = 0;
        const T el1 = e[l + 1];
        for (int i = m - 1; i >= l; --i) {
          c3 = c2;
          c2 = c;
          s2 = s;
          g = c * e[i];
          h = c * p;
          r = hypot(p, e[i]);
          e[i + 1] = s * r;
          s = e[i] / r;
          c = p / r;
          p = c * d[i] - s * g;
          d[i + 1] = h + s * (c * g + s * d[i]);
          rc[i] = c;
          rs[i] = s;
        }
        p = -s * s2 * c3 * el1 * e[l] / dl1;
        e[l] = s * p;
        d[l] = c * p;
        s_lo = l;
        s_hi = m - 1;
        s_done = 0;
        break;
      }
    }
    __syncthreads();
    if (s_done) break;
    const int lo = s_lo, hi = s_hi;
    for (int row = tid; row < n; row += EIG_THREADS) {
      T* zr = Z + (size_t)row * n;
      for (int i = hi; i >= lo; --i) {
        const T c = rc[i], s = rs[i];
        const T zi = zr[i], zi1 = zr[i + 1];
        zr[i + 1] = s * zi + c * zi1;
        zr[i] = c * zi - s * zi1;
      }
    }
    __syncthreads();
  }

  // ---- order eigenvalues descending (stable), select the leading k vectors
  for (int i = tid; i < n; i += EIG_THREADS) {
    int rank = 0;
    const T di = d[i];
    for (int q = 0; q < n; ++q) {
      const T dq = d[q];
      rank += (dq > di) || (dq == di && q < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += EIG_THREADS) lam[r] = (double)d[order[r]];
  for (size_t x = tid; x < (size_t)k * n; x += EIG_THREADS) {
    const int r = (int)(x / n), i = (int)(x - (size_t)r * n);
    ZS[x] = Z[(size_t)i * n + order[r]];
  }
  __syncthreads();

  // ---- back-transform: ZS^T <- H_0 ... H_{n-3} ZS^T
  for (int j = n - 3; j >= 0; --j) {
    const T tau = tauv[j];
    if (tau == (T)0) continue;
    const T* Aj = A + (size_t)j * n;
    for (int r = warp; r < k; r += nwarps) {
      T* zr = ZS + (size_t)r * n;
      T acc = 0;
      for (int i = j + 2 + lane; i < n; i += 32) acc += Aj[i] * zr[i];
      acc = warp_sum_e(acc) + zr[j + 1];
      acc *= tau;
      if (lane == 0) zr[j + 1] -= acc;
      for (int i = j + 2 + lane; i < n; i += 32) zr[i] -= acc * Aj[i];
    }
    __syncthreads();
  }
  for (size_t x = tid; x < (size_t)n * k; x += EIG_THREADS) {
    const int i = (int)(x / k), r = (int)(x - (size_t)i * k);
    Uout[x] = (double)ZS[(size_t)r * n + i];
  }
}
}  // namespace

void eig_sym(cudaStream_t st, int n, int k, const double* G, double* U, double* lam, void* work, int prec_bits,
             int* status) {
  if (n <= 0) return;
  if (n > EIG_MAXN || k > n || k < 0) {
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  count_launches(1);
  if (prec_bits == 32)
    eig_sym_kernel<float><<<1, EIG_THREADS, 0, st>>>(n, k, G, U, lam, (float*)work, status);
  else
    eig_sym_kernel<double><<<1, EIG_THREADS, 0, st>>>(n, k, G, U, lam, (double*)work, status);
}

}  // namespace qtt
