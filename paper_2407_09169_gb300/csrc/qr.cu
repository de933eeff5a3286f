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
// chain of reflectors short (a look-ahead of one column).  For the small
// shapes Q is then accumulated backwards in the same register layout, with no
// synchronisation at all; for the larger ones (Vg given) the block hands the
// reflectors to qr_formq_kernel, which forms the columns of Q over several
// blocks.  Both loops pair columns through the packed FP32x2 FMA (FFMA2).

// d0 += a0 * b0, d1 += a1 * b1 in one packed FP32x2 instruction.
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rd, {%0, %1};\n"
      " fma.rn.f32x2 rd, ra, rb, rd;\n mov.b64 {%0, %1}, rd;\n}"
      : "+f"(d0), "+f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Sums each of CPW values over the warp's 32 lanes; every lane gets every
// sum.  For CPW = 9 the first eight go through a butterfly in which pairs of
// values trade halves at each level (lane bit 4 keeps the odd one, bit 3 ...),
// so that after five levels the lane with bits (b4, b3, b2) holds the sum of
// value 4 b2 + 2 b3 + b4, which eight shuffles then broadcast: 22 shuffles
// instead of 45.  Shuffle throughput, not the FMAs, bounds this kernel.
template <int CPW>
__device__ __forceinline__ void qrr_warp_sums(float (&d)[CPW], int lane) {
  constexpr unsigned F = 0xffffffffu;
  if constexpr (CPW == 9) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = (b4 ? d[2 * i + 1] : d[2 * i]) + __shfl_xor_sync(F, b4 ? d[2 * i] : d[2 * i + 1], 16);
    float s8 = d[8] + __shfl_xor_sync(F, d[8], 16);
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) c[i] = (b3 ? a[2 * i + 1] : a[2 * i]) + __shfl_xor_sync(F, b3 ? a[2 * i] : a[2 * i + 1], 8);
    s8 += __shfl_xor_sync(F, s8, 8);
    float e = (b2 ? c[1] : c[0]) + __shfl_xor_sync(F, b2 ? c[0] : c[1], 4);
    s8 += __shfl_xor_sync(F, s8, 4);
    e += __shfl_xor_sync(F, e, 2);
    s8 += __shfl_xor_sync(F, s8, 2);
    e += __shfl_xor_sync(F, e, 1);
    s8 += __shfl_xor_sync(F, s8, 1);
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = __shfl_sync(F, e, ((q & 1) << 4) | (((q >> 1) & 1) << 3) | (((q >> 2) & 1) << 2));
    d[8] = s8;
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < CPW; ++q) d[q] += __shfl_xor_sync(F, d[q], o);
  }
}

constexpr int QRR_WARPS = 16;
constexpr int QRR_THREADS = QRR_WARPS * 32;
constexpr long long QRR_WAIT_LIMIT = 1LL << 24;  // try_wait polls of a reflector barrier before giving up

// One mbarrier per reflector (arrival count 32: every lane of the owning warp
// arrives after its own stores of v, with release semantics); waiters poll
// with try_wait (acquire), which suspends the warp in hardware and resumes it
// as soon as the phase completes, with no sleep quantum on the critical path.
__device__ __forceinline__ uint32_t qrr_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void qrr_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(qrr_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void qrr_bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(qrr_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool qrr_bar_try_wait(uint64_t* bar) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(qrr_smem_u32(bar))
      : "memory");
  return ok != 0;
}

// Reflector of the owned column q (global index c) of X (rows lane + 32 k):
// writes v (v_c = 1, zeros above c) to V[c][.] and tau[c], then arrives on bar[c].
template <int RPL, int CPW>
__device__ __forceinline__ void qrr_reflector(const float (&X)[RPL][CPW], int q, int c, int lane, int ldv, float* V,
                                              float* tau, uint64_t* bar, int* status) {
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
    // On the reflector chain: the approximate reciprocal square root and
    // quotient (a few ulp) where the sum of squares is a normal number.  H
    // stays orthogonal to that level (tau v^T v = 2 up to the error of beta),
    // as with float round-off, which the FP64 Newton-Schulz step removes.
    const float q2 = fmaf(a, a, s);
    const bool normal = q2 > 1e-30f && q2 < 1e30f;
    const float mu = normal ? q2 * rsqrtf(q2) : sqrtf(q2);
    const float beta = a <= 0.f ? mu : -mu;
    t = normal ? __fdividef(beta - a, beta) : (beta - a) / beta;
    v0 = a - beta;
  }
  float* v = V + (size_t)c * ldv;
  // |x_i| <= |v0|: one reciprocal instead of a division per row; the
  // (warp-uniform) branch keeps divisions out of the common case, they run
  // only when v0 is so small that its reciprocal would overflow
  const bool tiny = fabsf(v0) < 1e-30f;
  const float rv0 = (t != 0.f && !tiny) ? __fdividef(1.f, v0) : 0.f;
#pragma unroll
  for (int qq = 0; qq < CPW; ++qq) {
    if (qq != q) continue;
    if (!tiny || t == 0.f) {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int i = lane + 32 * k;
        v[i] = i < c ? 0.f : (i == c ? 1.f : X[k][qq] * rv0);
      }
    } else {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int i = lane + 32 * k;
        v[i] = i < c ? 0.f : (i == c ? 1.f : X[k][qq] / v0);
      }
    }
  }
  if (lane == 0) {
    tau[c] = t;
    if (!isfinite(t)) atomicOr(status, 1);
  }
  qrr_bar_arrive(bar + c);
}

// Bounded wait for reflector j (every lane acquires it); false (and status
// bit 4) if it never comes.
__device__ __forceinline__ bool qrr_wait(uint64_t* bar, int j, int lane, int* status) {
  bool ok = false;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (long long it = 0; it < QRR_WAIT_LIMIT && !ok; ++it) {
    ok = qrr_bar_try_wait(bar + j);
    if (!ok && (it & 255) == 255) {  // and at most about a second of wall time
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) break;
    }
  }
  const bool all = __all_sync(0xffffffffu, ok);
  if (!all && lane == 0) atomicOr(status, 4);
  return all;
}

template <int RPL, int CPW>
__global__ void __launch_bounds__(QRR_THREADS) qr_reg_kernel(int m, int n, const double* __restrict__ A,
                                                             double* __restrict__ Qout, float* __restrict__ Vg,
                                                             int* status) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char qr_smem[];
  constexpr int LDV = 32 * RPL;
  float* V = (float*)qr_smem;        // [n][LDV] reflectors; first the input, last the output staging
  float* tau = V + (size_t)n * LDV;  // [n]
  uint64_t* bar = (uint64_t*)(((uintptr_t)(tau + n) + 7) & ~(uintptr_t)7);  // [n]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // input, column-major in shared memory, then into registers
  for (int e = tid; e < m * n; e += QRR_THREADS) {
    const int i = e / n, c = e - i * n;
    V[(size_t)c * LDV + i] = (float)A[e];
  }
  for (int c = tid; c < n; c += QRR_THREADS) qrr_bar_init(bar + c, 32);
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
  if (warp == 0) qrr_reflector<RPL, CPW>(X, 0, 0, lane, LDV, V, tau, bar, status);
  bool alive = true;
  for (int j = 0; j < n && alive; ++j) {
    alive = qrr_wait(bar, j, lane, status);
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
      qrr_reflector<RPL, CPW>(X, qn, cn, lane, LDV, V, tau, bar, status);
    }
    if (t != 0.f) {
      // the other owned columns c > j (c > j + 1 for the owner of j + 1): the
      // inactive ones form a prefix in q, so columns go in pairs through the
      // packed FP32x2 FMA and a pair with one inactive column gets f = 0 there
      const int cmin = own_next ? cn + 1 : cn;
      float dot[CPW];
#pragma unroll
      for (int q = 0; q < CPW; ++q) dot[q] = 0.f;
#pragma unroll
      for (int q = 0; q + 1 < CPW; q += 2) {
        if (warp + QRR_WARPS * (q + 1) >= cmin && warp + QRR_WARPS * q < n) {
#pragma unroll
          for (int k = 0; k < RPL; ++k) ffma2(dot[q], dot[q + 1], v[k], v[k], X[k][q], X[k][q + 1]);
        }
      }
      if (CPW % 2 == 1) {
        constexpr int q = CPW - 1;
        if (warp + QRR_WARPS * q >= cmin && warp + QRR_WARPS * q < n) {
#pragma unroll
          for (int k = 0; k < RPL; ++k) dot[q] += v[k] * X[k][q];
        }
      }
      qrr_warp_sums<CPW>(dot, lane);
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        const int c = warp + QRR_WARPS * q;
        dot[q] = (c >= cmin && c < n) ? -t * dot[q] : 0.f;  // the update factor
      }
#pragma unroll
      for (int q = 0; q + 1 < CPW; q += 2) {
        if (warp + QRR_WARPS * (q + 1) >= cmin && warp + QRR_WARPS * q < n) {
#pragma unroll
          for (int k = 0; k < RPL; ++k) ffma2(X[k][q], X[k][q + 1], dot[q], dot[q + 1], v[k], v[k]);
        }
      }
      if (CPW % 2 == 1) {
        constexpr int q = CPW - 1;
        if (warp + QRR_WARPS * q >= cmin && warp + QRR_WARPS * q < n) {
#pragma unroll
          for (int k = 0; k < RPL; ++k) X[k][q] += dot[q] * v[k];
        }
      }
    }
  }
  __syncthreads();  // every reflector is published and every warp is done with its columns
  if (Vg) {  // Q is formed by qr_formq_kernel over several blocks: hand over the reflectors and tau
    const int nv = n * LDV / 4;
    for (int e = tid; e < nv; e += QRR_THREADS) reinterpret_cast<float4*>(Vg)[e] = reinterpret_cast<const float4*>(V)[e];
    for (int c = tid; c < n; c += QRR_THREADS) Vg[(size_t)n * LDV + c] = tau[c];
    return;
  }
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
    // columns c >= j (the others are still e_c, orthogonal to v), in pairs as above
    float dot[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) dot[q] = 0.f;
#pragma unroll
    for (int q = 0; q + 1 < CPW; q += 2) {
      if (warp + QRR_WARPS * (q + 1) >= j && warp + QRR_WARPS * q < n) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) ffma2(dot[q], dot[q + 1], v[k], v[k], X[k][q], X[k][q + 1]);
      }
    }
    if (CPW % 2 == 1) {
      constexpr int q = CPW - 1;
      if (warp + QRR_WARPS * q >= j && warp + QRR_WARPS * q < n) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) dot[q] += v[k] * X[k][q];
      }
    }
    qrr_warp_sums<CPW>(dot, lane);
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + QRR_WARPS * q;
      dot[q] = (c >= j && c < n) ? -t * dot[q] : 0.f;
    }
#pragma unroll
    for (int q = 0; q + 1 < CPW; q += 2) {
      if (warp + QRR_WARPS * (q + 1) >= j && warp + QRR_WARPS * q < n) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) ffma2(X[k][q], X[k][q + 1], dot[q], dot[q + 1], v[k], v[k]);
      }
    }
    if (CPW % 2 == 1) {
      constexpr int q = CPW - 1;
      if (warp + QRR_WARPS * q >= j && warp + QRR_WARPS * q < n) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) X[k][q] += dot[q] * v[k];
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

// Q = H_0 ... H_{n-1} [I; 0] from the reflectors that qr_reg_kernel hands over
// (Vg: n rows of LDV = 32 RPL floats, then tau[n]).  The columns of Q are
// independent, Q e_c = H_0 ... H_c e_c (H_j e_c = e_c for j > c, since v_j
// vanishes above row j), so each warp forms one column, 16 per block, over
// ceil(n / 16) blocks; the block stages the reflectors 0 .. its last column in
// shared memory and writes its 16 columns of Q row by row.  The reflectors
// are applied FQ_B at a time in compact form, H_j0 ... H_j0+3 = I - V T V^T
// (T upper triangular: T_kk = tau_k, column k above the diagonal
// -tau_k T V^T v_k, formed once per block of reflectors in the prologue), so
// that one warp reduction of FQ_B dot products replaces FQ_B dependent ones.
// Starting at the block that holds reflector c is exact: the reflectors after
// c in that block meet x = e_c in exact zeros.
constexpr int FQ_B = 4;

template <int RPL>
__host__ __device__ constexpr size_t formq_smem_floats(int nr) {
  return (size_t)nr * 32 * RPL + (size_t)((nr + 3) & ~3) + (size_t)32 * RPL * QRR_WARPS +
         (size_t)((nr + FQ_B - 1) / FQ_B) * FQ_B * FQ_B;
}

template <int RPL>
__global__ void __launch_bounds__(QRR_THREADS) qr_formq_kernel(int m, int n, const float* __restrict__ Vg,
                                                               double* __restrict__ Qout) {
  pdl_trigger();
  pdl_wait();
  constexpr int LDV = 32 * RPL;
  extern __shared__ __align__(16) unsigned char qr_smem[];
  const int c0 = blockIdx.x * QRR_WARPS;
  const int nr = min(n, c0 + QRR_WARPS);  // reflectors 0 .. nr - 1 are needed
  const int nbr = (nr + FQ_B - 1) / FQ_B;  // blocks of FQ_B reflectors
  float* V = (float*)qr_smem;               // [nr][LDV]
  float* tau = V + (size_t)nr * LDV;        // [nr]
  float* S = tau + ((nr + 3) & ~3);         // [32 RPL][QRR_WARPS] staging of the block's columns
  float* T = S + (size_t)32 * RPL * QRR_WARPS;  // [nbr][FQ_B][FQ_B]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nv = nr * LDV / 4;
  for (int e = tid; e < nv; e += QRR_THREADS) reinterpret_cast<float4*>(V)[e] = reinterpret_cast<const float4*>(Vg)[e];
  for (int c = tid; c < nr; c += QRR_THREADS) tau[c] = Vg[(size_t)n * LDV + c];
  __syncthreads();
  // T of each block of reflectors (those at or past nr are absent: tau 0, v 0)
  for (int bb = warp; bb < nbr; bb += QRR_WARPS) {
    const int j0 = bb * FQ_B;
    float g[FQ_B][FQ_B];
#pragma unroll
    for (int r = 0; r < FQ_B; ++r)
#pragma unroll
      for (int k = 0; k < FQ_B; ++k) g[r][k] = 0.f;
#pragma unroll
    for (int kk = 0; kk < RPL; ++kk) {
      float v[FQ_B];
#pragma unroll
      for (int r = 0; r < FQ_B; ++r) v[r] = (j0 + r < nr) ? V[(size_t)(j0 + r) * LDV + lane + 32 * kk] : 0.f;
#pragma unroll
      for (int k = 1; k < FQ_B; ++k)
#pragma unroll
        for (int r = 0; r < k; ++r) g[r][k] += v[r] * v[k];
    }
#pragma unroll
    for (int k = 1; k < FQ_B; ++k)
#pragma unroll
      for (int r = 0; r < k; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[r][k] += __shfl_xor_sync(0xffffffffu, g[r][k], o);
    if (lane == 0) {
      float* Tb = T + (size_t)bb * FQ_B * FQ_B;
      float tk[FQ_B];
#pragma unroll
      for (int k = 0; k < FQ_B; ++k) tk[k] = (j0 + k < nr) ? tau[j0 + k] : 0.f;
#pragma unroll
      for (int k = 0; k < FQ_B; ++k) {
#pragma unroll
        for (int p = 0; p < FQ_B; ++p) Tb[p * FQ_B + k] = 0.f;
        Tb[k * FQ_B + k] = tk[k];
#pragma unroll
        for (int p = 0; p < k; ++p) {
          float acc = 0.f;
#pragma unroll
          for (int r = p; r < k; ++r) acc += Tb[p * FQ_B + r] * g[r][k];
          Tb[p * FQ_B + k] = -tk[k] * acc;
        }
      }
    }
  }
  __syncthreads();
  const int c = c0 + warp;
  float x[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) x[k] = (lane + 32 * k == c) ? 1.f : 0.f;
  if (c < n) {
    for (int bb = c / FQ_B; bb >= 0; --bb) {
      const int j0 = bb * FQ_B;
      float v[FQ_B][RPL], w[FQ_B];
#pragma unroll
      for (int p = 0; p < FQ_B; ++p) {
        w[p] = 0.f;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          v[p][k] = (j0 + p < nr) ? V[(size_t)(j0 + p) * LDV + lane + 32 * k] : 0.f;
          w[p] += v[p][k] * x[k];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int p = 0; p < FQ_B; ++p) w[p] += __shfl_xor_sync(0xffffffffu, w[p], o);
      const float* Tb = T + (size_t)bb * FQ_B * FQ_B;
#pragma unroll
      for (int p = 0; p < FQ_B; ++p) {  // z = T w, then x -= V z
        float z = 0.f;
#pragma unroll
        for (int q = p; q < FQ_B; ++q) z += Tb[p * FQ_B + q] * w[q];
#pragma unroll
        for (int k = 0; k < RPL; ++k) x[k] -= v[p][k] * z;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RPL; ++k) S[(size_t)(lane + 32 * k) * QRR_WARPS + warp] = x[k];
  __syncthreads();
  const int nc = nr - c0;
  for (int e = tid; e < m * QRR_WARPS; e += QRR_THREADS) {
    const int i = e / QRR_WARPS, cc = e - i * QRR_WARPS;
    if (cc < nc) Qout[(size_t)i * n + c0 + cc] = (double)S[e];
  }
}

// split: hand the reflectors over to qr_formq_kernel (work: n (32 RPL + 1)
// floats) instead of accumulating Q in the factorising block.
template <int RPL, int CPW>
bool try_qr_reg(cudaStream_t st, int m, int n, const double* A, double* Qout, int* status, float* split) {
  if (m > 32 * RPL || n > QRR_WARPS * CPW) return false;
  const size_t smem = ((size_t)n * 32 * RPL + (size_t)n) * sizeof(float) + 8 + (size_t)n * sizeof(uint64_t);
  constexpr int NMAX = QRR_WARPS * CPW;
  auto formq_smem = [](int nr) { return formq_smem_floats<RPL>(nr) * sizeof(float); };
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(qr_reg_kernel<RPL, CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)NMAX * 32 * RPL + NMAX) * sizeof(float) + 8 + (size_t)NMAX * sizeof(uint64_t)));
    cudaFuncSetAttribute(qr_formq_kernel<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)formq_smem(NMAX));
    attr = true;
  }
  launch_pdl(qr_reg_kernel<RPL, CPW>, dim3(1), dim3(QRR_THREADS), smem, st, m, n, A, Qout, split, status);
  if (split) {
    const int nb = (n + QRR_WARPS - 1) / QRR_WARPS;
    launch_pdl_chain(qr_formq_kernel<RPL>, dim3(nb), dim3(QRR_THREADS), formq_smem(n), st, m, n, (const float*)split,
                     Qout);
    count_launches(1);
  }
  return true;
}

// ---------------------------------------------------------------------------
// FP64 QR over a cluster of CTAs.  FP64 issues at two FMAs per clock per SM
// on this GPU, so one block needs ~1 ms for the 272 x 136 factorisation
// alone; the factorisation is spread over the P CTAs of a thread-block
// cluster instead.  Column c belongs to warp c / P of CTA c % P (cyclic, so
// every CTA keeps work until the end) and lives in that warp's registers
// (rows lane + 32 k).  A warp applies the reflectors 0 .. c-1 as they appear
// and then forms reflector c itself: the owner of column j + 1 is the first
// to take H_j, which gives the one-column look-ahead with no further
// arrangement.  Reflector c stays in its owner's shared memory (v_c with
// v_c[c] = 1 and zeros above, tau_c); readiness is an mbarrier per reflector
// in every CTA, on which the owner's lane r arrives remotely (release at
// cluster scope) for CTA r, and the consumers read v_c through distributed
// shared memory after an acquire-wait on their local barrier.  Waits are
// bounded (status bit 4 when one gives up).  The reflectors then go to
// global memory (work: n rows of m doubles, then tau), from which
// qr64_formq_kernel forms the columns of Q over n blocks.
constexpr long long QR64_WAIT_POLLS = 1LL << 24;

__device__ __forceinline__ uint32_t qr64_mapa(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ double qr64_ld_remote(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void qr64_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t qr64_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

template <int RPL>
__global__ void __launch_bounds__(512) qr64_cluster_kernel(int m, int n, int P, const double* __restrict__ A, double* __restrict__ Vg,
                                    int ldv, int* status) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  const int wpc = blockDim.x >> 5;                                  // columns (warps) per CTA
  double* V = (double*)qr_smem;                                     // [wpc][32 RPL] own reflectors
  double* tau = V + (size_t)wpc * 32 * RPL;                         // [wpc]
  uint64_t* bar = (uint64_t*)(tau + ((wpc + 1) & ~1));              // [n] one per reflector
  const int rank = (int)qr64_cluster_rank();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int j = tid; j < n; j += blockDim.x)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(qrr_smem_u32(bar + j)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const int c = rank + P * w;  // the column this warp owns
  double X[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int i = lane + 32 * k;
    X[k] = (c < n && i < m) ? A[(size_t)i * n + c] : 0.0;
  }
  qr64_cluster_sync();  // every barrier of every CTA is initialised
  const uint32_t V0 = qrr_smem_u32(V), T0 = qrr_smem_u32(tau);
  bool alive = c < n;
  for (int j = 0; j < c && alive; ++j) {
    // bounded acquire-wait (cluster scope) on the local barrier of reflector j
    const uint32_t b = qrr_smem_u32(bar + j);
    bool ok = false;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (long long it = 0; it < QR64_WAIT_POLLS && !ok; ++it) {
      uint32_t r;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(r)
          : "r"(b)
          : "memory");
      ok = r != 0;
      if (!ok && (it & 255) == 255) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) break;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(status, 4);
      alive = false;
      break;
    }
    const uint32_t owner = (uint32_t)(j % P), slot = (uint32_t)(j / P);
    const uint32_t vb = qr64_mapa(V0 + slot * 32 * RPL * 8, owner);
    const double t = qr64_ld_remote(qr64_mapa(T0 + slot * 8, owner));
    if (t == 0.0) continue;
    double v[RPL], dp[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < RPL; ++k) v[k] = qr64_ld_remote(vb + (lane + 32 * k) * 8);
    // three independent partial sums: the FP64 chain is a third as long
#pragma unroll
    for (int k = 0; k < RPL; ++k) dp[k % 3] = fma(v[k], X[k], dp[k % 3]);
    double d = dp[0] + (dp[1] + dp[2]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const double f = -t * d;
#pragma unroll
    for (int k = 0; k < RPL; ++k) X[k] = fma(f, v[k], X[k]);
  }
  if (alive) {
    // reflector of column c: v = (x - beta e_c) / (x_c - beta) on rows >= c
    double sp[3] = {0.0, 0.0, 0.0}, a = 0.0;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      if (i > c) sp[k % 3] = fma(X[k], X[k], sp[k % 3]);
      if (i == c) a = X[k];  // only lane c % 32 holds row c
    }
    double s = sp[0] + (sp[1] + sp[2]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    a = __shfl_sync(0xffffffffu, a, c & 31);
    double t = 0.0, v0 = 1.0, rv0 = 0.0;
    if (s != 0.0) {
      const double mu = sqrt(fma(a, a, s));
      const double beta = a <= 0.0 ? mu : -mu;
      v0 = a - beta;  // |v0| >= mu >= |x_i|
      // one division for both reciprocals: r = 1 / (beta v0), 1/beta = v0 r,
      // 1/v0 = beta r (two divisions where |beta v0| >= mu^2 could underflow)
      const double bv = beta * v0;
      if (fabs(bv) > 1e-290) {
        const double r = 1.0 / bv;
        t = -v0 * (v0 * r);  // (beta - a) / beta
        rv0 = beta * r;
      } else {
        t = (beta - a) / beta;
        rv0 = 1.0 / v0;
      }
    }
    double* vc = V + (size_t)w * 32 * RPL;
    const bool tiny = fabs(v0) < 1e-300;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int i = lane + 32 * k;
      const double vi = i < c ? 0.0 : (i == c ? 1.0 : (tiny ? X[k] / v0 : X[k] * rv0));
      vc[i] = vi;
      if (i < m) Vg[(size_t)c * ldv + i] = vi;
    }
    if (lane == 0) {
      tau[w] = t;
      Vg[(size_t)n * ldv + c] = t;
      if (!isfinite(t)) atomicOr(status, 1);
    }
    // every lane's stores of v are ordered before the release-arrives below
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    __syncwarp();
    if (lane < P) {
      const uint32_t rb = qr64_mapa(qrr_smem_u32(bar + c), (uint32_t)lane);
      asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rb) : "memory");
    }
  }
  qr64_cluster_sync();  // no CTA leaves while another may still read its reflectors
}

// Q = H_0 ... H_{n-1} [I; 0] column by column: block c forms Q e_c =
// H_0 ... H_c e_c (128 threads, rows t + 128 r), one block reduction per
// reflector; the next reflector's rows are loaded before the reduction.
constexpr int QR64_FQ_THREADS = 128;
__global__ void __launch_bounds__(QR64_FQ_THREADS) qr64_formq_kernel(int m, int n, const double* __restrict__ Vg,
                                                                     int ldv, double* __restrict__ Qout) {
  constexpr int R = 3;  // m <= 384
  __shared__ double part[2][QR64_FQ_THREADS / 32];
  const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const double* tau = Vg + (size_t)n * ldv;
  double x[R], v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = tid + QR64_FQ_THREADS * r;
    x[r] = i == c ? 1.0 : 0.0;
    v[r] = i < m ? Vg[(size_t)c * ldv + i] : 0.0;
  }
  int ph = 0;  // reduction slot: alternates with every block barrier taken
  for (int j = c; j >= 0; --j) {
    const double t = tau[j];
    double vn[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = tid + QR64_FQ_THREADS * r;
      vn[r] = (j > 0 && i < m) ? Vg[(size_t)(j - 1) * ldv + i] : 0.0;
    }
    if (t != 0.0) {  // uniform across the block
      double d = 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) d = fma(v[r], x[r], d);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) part[ph][w] = d;
      __syncthreads();
      d = 0.0;
#pragma unroll
      for (int q = 0; q < QR64_FQ_THREADS / 32; ++q) d += part[ph][q];
      ph ^= 1;
      const double f = -t * d;
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = fma(f, v[r], x[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = vn[r];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = tid + QR64_FQ_THREADS * r;
    if (i < m) Qout[(size_t)i * n + c] = x[r];
  }
}

// Launches the cluster factorisation and the Q formation; false when the
// shape or the GPU does not take it (the caller then uses the one-block QR).
// work: n (m + 1) doubles.
template <int RPL>
bool try_qr64_cluster(cudaStream_t st, int m, int n, const double* A, double* Qout, double* work, int* status) {
  if (m > 32 * RPL || m > 3 * QR64_FQ_THREADS) return false;
  static int P = -1;  // cluster size: 16 where the GPU takes it, else 8, else 0
  const int wpc_max = 16;  // 512 threads: the register file takes every RPL used here
  if (P < 0) {
    P = 0;
    cudaFuncSetAttribute(qr64_cluster_kernel<RPL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    const size_t smem_max = (size_t)wpc_max * 32 * RPL * 8 + (wpc_max + 2) * 8 + (size_t)16 * wpc_max * 8;
    cudaFuncSetAttribute(qr64_cluster_kernel<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    for (int cand : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cand);
      cfg.blockDim = dim3(32 * 9);
      cfg.dynamicSmemBytes = (size_t)9 * 32 * RPL * 8 + 16 * 8 + (size_t)cand * 9 * 8;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cand;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, qr64_cluster_kernel<RPL>, &cfg) == cudaSuccess && nclusters > 0) {
        P = cand;
        break;
      }
      cudaGetLastError();
    }
  }
  if (P == 0) return false;
  const int wpc = (n + P - 1) / P;
  if (wpc > wpc_max) return false;
  const int ldv = m;  // row stride of the reflectors in work (rows >= m are not stored)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(32 * wpc);
  // shared: wpc reflector slots of 32 RPL doubles, tau (rounded up to an even count), n barriers
  cfg.dynamicSmemBytes = (size_t)wpc * 32 * RPL * 8 + (size_t)((wpc + 1) & ~1) * 8 + (size_t)n * 8;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, qr64_cluster_kernel<RPL>, m, n, P, A, work, ldv, status) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  qr64_formq_kernel<<<n, QR64_FQ_THREADS, 0, st>>>(m, n, (const double*)work, ldv, Qout);
  count_launches(1);
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
    float* split = (float*)work;  // n (32 RPL + 1) floats <= 2 m n + n doubles, as m >= 8 RPL where used
    if (try_qr_reg<3, 3>(st, m, n, A, Qout, status, nullptr) || try_qr_reg<5, 5>(st, m, n, A, Qout, status, split) ||
        try_qr_reg<9, 9>(st, m, n, A, Qout, status, split))
      return;
    launch_qr<float>(st, m, n, A, Qout, work, status);
  }
  else {
    if (try_qr64_cluster<3>(st, m, n, A, Qout, (double*)work, status) ||
        try_qr64_cluster<5>(st, m, n, A, Qout, (double*)work, status) ||
        try_qr64_cluster<9>(st, m, n, A, Qout, (double*)work, status) ||
        try_qr64_cluster<12>(st, m, n, A, Qout, (double*)work, status))
      return;
    launch_qr<double>(st, m, n, A, Qout, work, status);
  }
}

}  // namespace qtt
