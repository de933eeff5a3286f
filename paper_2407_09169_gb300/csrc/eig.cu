// Symmetric eigen-decomposition for the SVD truncation sweep.
//
// The sweep truncates a bond through the Gram matrix G = M M^T = U diag(lam) U^T
// of the bond matrix (paper: "Matrix product state algorithm" -- the bond
// dimension is limited to chi with the singular value decomposition;
// lam = sigma^2, U = left singular vectors).
//
// Three kernels, so that the FP64 work does not all sit on one SM:
//   1. eig_tridiag_ql (one block): Householder reduction to tridiagonal form
//      (matrix in shared memory when it fits, lower-triangle updates); for
//      single-precision problems it then runs the implicit-shift QL iteration
//      on (d, e) in warp 0 (one lane carries the rotation chain; lanes of
//      warps 1 and 2 apply each rotation to e and d and record it in a list
//      of every sweep's rotations) and a stable descending order of the
//      eigenvalues;
//   2. FP64: eig_dc (one block), divide and conquer on (d, e) (below), which
//      also orders the eigenvalues; single precision: eig_apply_rotations
//      (one thread per row of the eigenvector matrix Z of the tridiagonal
//      problem, over several blocks), which replays the rotation list on its
//      row;
//   3. eig_back_transform (one warp per kept eigenvector): applies the
//      Householder reflectors, U[:, r] = H_0 ... H_{n-3} Z[:, order[r]].
// Every loop is bounded; a QL iteration stops after 60 sweeps per
// eigenvalue (or when the rotation list is full), a secular root after 100
// steps, and the two QL lanes wait on each other for at most about a second;
// both report through the status word (bits 2 and 8).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace qtt {

namespace {
constexpr int TRI_THREADS = 512;
constexpr int EIG_MAXN = 1024;
constexpr int QL_MAX_SWEEPS = 60;
constexpr size_t EIG_SMEM_LIMIT = 176 * 1024;  // + 6 * EIG_MAXN static values stays below 227 KB

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

__device__ __forceinline__ double rhyp(double a, double b) { return rhypot(a, b); }
__device__ __forceinline__ float rhyp(float a, float b) { return rhypotf(a, b); }
// 1 / sqrt(a^2 + b^2) on the QL recurrence's dependency chain, with b^2
// given (b2 = b * b, computed off the chain): the plain reciprocal square
// root of the sum of squares (fewer dependent operations than the scaled
// rhypot) while the sum stays inside the normal range, else the scaled form.
__device__ __forceinline__ double rhyp_fast_sq(double a, double b, double b2) {
  const double q = fma(a, a, b2);
  const int ex = (__double2hiint(q) >> 20) & 0x7ff;
  return (ex > 27 && ex < 2019) ? rsqrt(q) : rhypot(a, b);
}
__device__ __forceinline__ float rhyp_fast_sq(float a, float b, float b2) {
  const float q = fmaf(a, a, b2);
  return (q > 1e-35f && q < 1e35f) ? rsqrtf(q) : rhypotf(a, b);
}

// Bounded spins on a flag in shared memory, between the QL chain and its
// helper lane: at most ~2^26 polls and about a second of wall time; on expiry
// the abort word is set so that the other side stops too.
constexpr long long QL_SPIN_LIMIT = 1LL << 26;
__device__ __forceinline__ bool ql_spin_expired(long long it, unsigned long long t0) {
  if ((it & 1023) != 1023) return it >= QL_SPIN_LIMIT;
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return it >= QL_SPIN_LIMIT || t - t0 > 1000000000ull;
}
__device__ __forceinline__ unsigned long long ql_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// waits for *w == v; false if it expired or the abort word was set
__device__ inline bool ql_wait_eq(volatile int* w, int v, volatile int* abort_w) {
  const unsigned long long t0 = ql_now();
  for (long long it = 0;; ++it) {
    if (*w == v) return true;
    if (*abort_w || ql_spin_expired(it, t0)) {
      *abort_w = 1;
      return false;
    }
  }
}
// waits for *w >= v
__device__ inline bool ql_wait_ge(volatile int* w, int v, volatile int* abort_w) {
  const unsigned long long t0 = ql_now();
  for (long long it = 0;; ++it) {
    if (*w >= v) return true;
    if (*abort_w || ql_spin_expired(it, t0)) {
      *abort_w = 1;
      return false;
    }
  }
}
// waits for *w != seen; returns the new value, or -2 on expiry / abort
__device__ inline int ql_wait_change(volatile int* w, int seen, volatile int* abort_w) {
  const unsigned long long t0 = ql_now();
  for (long long it = 0;; ++it) {
    const int v = *w;
    if (v != seen) return v;
    if (*abort_w || ql_spin_expired(it, t0)) {
      *abort_w = 1;
      return -2;
    }
  }
}

// Work layout, in elements of T: A n*n | Z n*n | rot_c R | rot_s R | (divide
// and conquer) U n*n | V n*n | vectors 10 n; then ints: seg_lo S | seg_hi S |
// seg_off S | order n | nseg 4 | (divide and conquer) 6 n.  R = 4 n^2 + 64 n
// rotations, S = 60 n sweeps.
struct EigLayout {
  size_t A, Z, rc, rs, R, S;
  size_t dcU, dcV, dcv;
  size_t ints_off;  // bytes
  size_t seg_lo, seg_hi, seg_off, order, nseg, dci;
  size_t bytes;
};

template <typename T>
__host__ __device__ EigLayout eig_layout(int n) {
  EigLayout L;
  const size_t nn = (size_t)n * n;
  L.R = 4 * nn + 64 * (size_t)n;
  L.S = (size_t)QL_MAX_SWEEPS * n;
  L.A = 0;
  L.Z = nn;
  L.rc = 2 * nn;
  L.rs = L.rc + L.R;
  L.dcU = L.rs + L.R;
  L.dcV = L.dcU + nn;
  L.dcv = L.dcV + nn;
  L.ints_off = (L.dcv + 10 * (size_t)n) * sizeof(T);
  L.ints_off = (L.ints_off + 15) & ~(size_t)15;
  L.seg_lo = 0;
  L.seg_hi = L.S;
  L.seg_off = 2 * L.S;
  L.order = 3 * L.S;
  L.nseg = 3 * L.S + n;
  L.dci = L.nseg + 4;
  L.bytes = L.ints_off + (L.dci + 6 * (size_t)n) * sizeof(int);
  return L;
}

template <typename T>
__global__ void __launch_bounds__(TRI_THREADS) eig_tridiag_ql(const EigProblem* __restrict__ probs, int use_smem,
                                                              int* status, int dc) {
  const EigProblem P = probs[blockIdx.x];
  const int n = P.n;
  if (n <= 0) return;
  const double* __restrict__ G = P.G;
  double* __restrict__ lam = P.lam;
  unsigned char* work = P.work;
  const EigLayout L = eig_layout<T>(n);
  T* W = (T*)work;
  int* I = (int*)(work + L.ints_off);
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* A = use_smem ? (T*)dyn_smem : W + L.A;
  T* rcg = W + L.rc;
  T* rsg = W + L.rs;
  int* seg_lo = I + L.seg_lo;
  int* seg_hi = I + L.seg_hi;
  int* seg_off = I + L.seg_off;
  int* order = I + L.order;
  __shared__ T d[EIG_MAXN], e[EIG_MAXN], vb[EIG_MAXN], pb[EIG_MAXN], wb[EIG_MAXN], tauv[EIG_MAXN];
  __shared__ T s_tau, s_v0, s_K;
  __shared__ int ql_ctl[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // row stride of the working copy: n + 1 in shared memory (rows of
  // consecutive threads then fall on different banks), n in global memory
  const int lda = use_smem ? n + 1 : n;
  for (size_t x = tid; x < (size_t)n * n; x += TRI_THREADS) {
    const int i = (int)(x / n), c = (int)(x - (size_t)i * n);
    A[(size_t)i * lda + c] = (T)(0.5 * (G[x] + G[(size_t)c * n + i]));
  }
  __syncthreads();

  // ---- Householder tridiagonalisation.  Only the lower triangle (c <= i) of
  // the trailing block is kept current; reflector j is stored in row j,
  // columns > j + 1 (the strict upper part, unused otherwise).  FP64 issues
  // at a fraction of a lane per clock per scheduler, so the products are laid
  // out to keep whole warps busy: A22 v with four threads per row (no
  // reduction over a warp per row), the rank-2 update over the flattened lower
  // triangle (no lanes idle on short rows).
  for (int j = 0; j + 2 < n; ++j) {
    T* Aj = A + (size_t)j * lda;
    if (warp == 0) {
      T s = 0;
      for (int i = j + 2 + lane; i < n; i += 32) {
        const T v = A[(size_t)i * lda + j];
        s += v * v;
      }
      s = warp_sum_e(s);
      if (lane == 0) {
        const T alpha = A[(size_t)(j + 1) * lda + j];
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
    if (tau == (T)0) {  // uniform branch (shared value)
      __syncthreads();  // s_tau is rewritten by the next step
      continue;
    }
    {
      const T inv = (T)1 / s_v0;
      for (int i = j + 2 + tid; i < n; i += TRI_THREADS) {
        const T v = A[(size_t)i * lda + j] * inv;
        vb[i] = v;
        Aj[i] = v;
      }
      if (tid == 0) vb[j + 1] = (T)1;
    }
    __syncthreads();
    // p = tau * A22 v, A22 symmetric with its lower triangle stored: four
    // threads per row (lanes 4r .. 4r + 3), each over every fourth column
    const int m = n - j - 1;
    const int m4 = (4 * m + 31) & ~31;  // whole warps enter each pass (the shuffles)
    for (int x = tid; x < m4; x += TRI_THREADS) {
      const bool ok = x < 4 * m;
      const int i = j + 1 + (x >> 2), q = x & 3;
      T acc = 0;
      if (ok) {
        for (int c = j + 1 + q; c < n; c += 4) {
          const T a = c <= i ? A[(size_t)i * lda + c] : A[(size_t)c * lda + i];
          acc += a * vb[c];
        }
      }
      // the four partial sums of a row sit in lanes 4r .. 4r + 3 of one warp
      acc += __shfl_xor_sync(0xffffffffu, acc, 1, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2, 4);
      if (ok && q == 0) pb[i] = tau * acc;
    }
    __syncthreads();
    if (warp == 0) {
      T acc = 0;
      for (int i = j + 1 + lane; i < n; i += 32) acc += pb[i] * vb[i];
      acc = warp_sum_e(acc);
      if (lane == 0) s_K = (T)0.5 * tau * acc;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += TRI_THREADS) wb[i] = pb[i] - s_K * vb[i];
    __syncthreads();
    // lower-triangle rank-2 update, rows i >= j+1, columns j+1 <= c <= i,
    // over the flattened triangle: element x is (r, c') with r (r + 1) / 2 <= x
    const int tri = m * (m + 1) / 2;
    for (int x = tid; x < tri; x += TRI_THREADS) {
      int r = (int)((sqrtf(8.f * (float)x + 1.f) - 1.f) * 0.5f);
      while (r * (r + 1) / 2 > x) --r;
      while ((r + 1) * (r + 2) / 2 <= x) ++r;
      const int i = j + 1 + r, c = j + 1 + (x - r * (r + 1) / 2);
      A[(size_t)i * lda + c] -= vb[i] * wb[c] + wb[i] * vb[c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * lda + (n - 2)];
      tauv[n - 2] = 0;
    }
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    e[n - 1] = 0;
    tauv[n - 1] = 0;
  }
  __syncthreads();
  // reflectors (and tau in the diagonal of A) for the back-transform kernel
  for (size_t x = tid; x < (size_t)n * n; x += TRI_THREADS) {
    const int i = (int)(x / n), c = (int)(x - (size_t)i * n);
    if (c > i + 1) W[L.A + x] = A[(size_t)i * lda + c];
    else if (c == i) W[L.A + x] = tauv[i];
  }

  if (dc) {  // the tridiagonal (d, e) for eig_dc, which finds its eigenpairs
    for (int i = tid; i < n; i += TRI_THREADS) {
      W[L.dcv + i] = d[i];
      W[L.dcv + n + i] = e[i];
    }
    return;
  }
  // ---- implicit QL with a Wilkinson-type shift, rotations recorded per sweep.
  // Warp 0 runs it: the search for the next negligible off-diagonal (32
  // entries per ballot) and the shift of the trailing diagonal are spread over
  // its lanes, and lane 0 carries the rotation chain.  FP64 instructions cost
  // the same whatever the number of active lanes, so the chain lane keeps only
  // the operations the next rotation depends on (sum of squares, reciprocal
  // square root, cosine, next p) and hands (p, 1/hypot, e_i) of every
  // rotation to lane 0 of warps 1 and 2, which run on two other schedulers'
  // FP64 pipes one rotation behind: both form the cosine and sine, warp 1
  // updates e[i+1] and records the rotation, warp 2 updates d[i+1] (positions
  // the chain has passed).  The chain waits for both at the end of each
  // sweep.  Every wait is bounded (status bit 8 on expiry).
  {
    T* qlP = vb;  // the tridiagonalisation's vectors are dead from here on
    T* qlR = pb;
    T* qlE2 = wb;
    T* qlEi = tauv;
    volatile int* ctl = ql_ctl;  // 0 sweep number (-1: end), 1 l, 2 m, 3 off, 4 published, 5 / 7 done (e / d), 6 abort
    if (tid == 0) {
      ctl[0] = 0;
      ctl[4] = 0;
      ctl[5] = 0;
      ctl[6] = 0;
      ctl[7] = 0;
    }
    __syncthreads();
    if (warp == 0) {
      const T eps = Eps<T>::v();
      T f = 0, tst1 = 0;
      int nseg = 0, sweep = 0;
      size_t off = 0;
      bool aborted = false;  // warp-uniform (lane 0's view of the abort word)
      for (int l = 0; l < n && !aborted; ++l) {
        const T hl = fabs(d[l]) + fabs(e[l]);
        tst1 = hl > tst1 ? hl : tst1;
        for (int iter = 0;; ++iter) {
          int m = n - 1;
          for (int base = l; base < n - 1; base += 32) {
            const int i = base + lane;
            const bool small = i < n - 1 && !(fabs(e[i]) > eps * tst1);
            const unsigned bal = __ballot_sync(0xffffffffu, small);
            if (bal) {
              m = base + __ffs(bal) - 1;
              break;
            }
          }
          if (m == l) break;
          if (iter >= QL_MAX_SWEEPS || nseg >= (int)L.S || off + (size_t)(m - l) > L.R) {
            if (lane == 0) atomicOr(status, 2);
            break;
          }
          T g = d[l];
          T p = (d[l + 1] - g) / ((T)2 * e[l]);
          T r = (T)1 / rhyp(p, (T)1);
          if (p < 0) r = -r;
          const T dl0 = e[l] / (p + r);
          const T dl1 = e[l] * (p + r);
          const T h = g - dl0;
          __syncwarp();
          if (lane == 0) {
            d[l] = dl0;
            d[l + 1] = dl1;
          }
          for (int i = l + 2 + lane; i < n; i += 32) d[i] -= h;
          for (int i = l + lane; i < m; i += 32) qlE2[i] = e[i] * e[i];  // e_i^2 for the chain
          f += h;
          __syncwarp();
          ++sweep;
          if (lane == 0) {
            p = d[m];
            const T el1 = e[l + 1];
            seg_lo[nseg] = l;
            seg_hi[nseg] = m - 1;
            seg_off[nseg] = (int)off;
            ctl[1] = l;
            ctl[2] = m;
            ctl[3] = (int)off;
            ctl[4] = 0;
            __threadfence_block();
            ctl[0] = sweep;
            // c: cosine of the previous rotation (1 before the first); c2, c3
            // the two before it; (e_i, rr) of the last two for the sines
            T c = 1, c2 = 1, c3 = 1, e1 = 0, r1 = 0, e2 = 0, r2 = 0;
            int k = 0;
            for (int i = m - 1; i >= l; --i, ++k) {
              c3 = c2;
              c2 = c;
              e2 = e1;
              r2 = r1;
              const T ei = e[i], di = d[i], e2 = qlE2[i];
              // the next p = c' d_i - s' g = rr (p d_i - e_i g), e_i g = c e_i^2:
              // the bracket does not wait for rr
              const T tq = fma(p, di, -(c * e2));
              const T rr = rhyp_fast_sq(p, ei, e2);  // 1 / hypot(p, e_i); e_i != 0 inside an unreduced block
              qlP[i] = p;
              qlR[i] = rr;
              qlEi[i] = ei;
              __threadfence_block();
              ctl[4] = k + 1;
              c = p * rr;
              p = rr * tq;
              e1 = ei;
              r1 = rr;
            }
            const T s = e1 * r1, s2 = e2 * r2;  // sines of the last two rotations (0 when absent)
            p = -s * s2 * c3 * el1 * e[l] / dl1;
            // the helper reads e[l] and d[l] in the last rotation and writes
            // d[l+1 ..], e[l+1 ..]: wait for it before e[l], d[l] and the next search
            if (!ql_wait_eq(ctl + 5, sweep, ctl + 6) || !ql_wait_eq(ctl + 7, sweep, ctl + 6)) atomicOr(status, 8);
            __threadfence_block();
            e[l] = s * p;
            d[l] = c * p;
          }
          off += (size_t)(m - l);
          ++nseg;
          __syncwarp();
          __threadfence_block();  // the helper's d and e, seen by lane 0, for every lane
          aborted = __shfl_sync(0xffffffffu, ctl[6], 0) != 0;
          if (aborted) break;
        }
        if (lane == 0) {
          d[l] += f;
          e[l] = 0;
        }
        __syncwarp();
      }
      if (lane == 0) {
        I[L.nseg] = nseg;
        __threadfence_block();
        ctl[0] = -1;
      }
    } else if ((warp == 1 || warp == 2) && lane == 0) {
      // warp 1: e[i+1] and the rotation list; warp 2: d[i+1] (two schedulers'
      // FP64 pipes).  Each reads the original e_i and d_i of its own
      // positions; warp 2 takes e_i from the chain's copy, since warp 1 may
      // already have overwritten it.
      const bool upd_e = warp == 1;
      int seen = 0;
      for (;;) {
        const int sw = ql_wait_change(ctl, seen, ctl + 6);
        if (sw == -2) {  // expired
          atomicOr(status, 8);
          break;
        }
        if (sw < 0) break;
        seen = sw;
        __threadfence_block();
        const int l = ctl[1], m = ctl[2];
        const size_t off = (size_t)ctl[3];
        T c = 1, s = 0;
        bool ok = true;
        for (int k = 0; k < m - l && ok; ++k) {
          ok = ql_wait_ge(ctl + 4, k + 1, ctl + 6);
          if (!ok) break;
          __threadfence_block();
          const int i = m - 1 - k;
          const T p = qlP[i], rr = qlR[i];
          if (upd_e) {
            const T ei = e[i];
            const T cn = p * rr, sn = ei * rr;
            const T r = p * cn + ei * sn;  // hypot(p, e_i)
            e[i + 1] = s * r;               // previous sine
            s = sn;
            c = cn;
            rcg[off + (size_t)k] = c;
            rsg[off + (size_t)k] = s;
          } else {
            const T ei = qlEi[i], di = d[i];
            const T g = c * ei;
            const T hh = c * p;
            const T cn = p * rr, sn = ei * rr;
            s = sn;
            c = cn;
            d[i + 1] = hh + s * (c * g + s * di);
          }
        }
        if (!ok) {
          atomicOr(status, 8);
          break;
        }
        __threadfence_block();
        ctl[upd_e ? 5 : 7] = seen;
      }
    }
  }
  __syncthreads();
  // ---- stable descending order of the eigenvalues
  for (int i = tid; i < n; i += TRI_THREADS) {
    const T di = d[i];
    int rank = 0;
    for (int q = 0; q < n; ++q) {
      const T dq = d[q];
      rank += (dq > di) || (dq == di && q < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRI_THREADS) lam[r] = (double)d[order[r]];
}

// ---------------------------------------------------------------------------
// Divide and conquer on the tridiagonal (FP64): the QL chain above issues one
// dependent FP64 rotation after another, about 1.7k cycles each on this GPU,
// and a full 136 x 136 spectrum takes ~10k of them plus their replay on Z.
// Here the tridiagonal T is cut recursively in halves (Cuppen):
//   T = diag(T1, T2) + beta (e_a + e_b)(e_a + e_b)^T,  beta = T[a][b] at the
// cut, T1's last and T2's first diagonal entries minus beta;
// leaves of at most DC_LEAF rows are solved by the implicit QL iteration in
// one warp each (every lane runs the same scalar recurrence and rotates its
// own row of Z), and two solved halves T1 = Q1 D1 Q1^T, T2 = Q2 D2 Q2^T are
// merged by the eigen-decomposition of D + rho z z^T, z = (last row of Q1,
// first row of Q2): deflation of the negligible components of z and of
// (nearly) equal poles by plane rotations, one root of the secular equation
// 1 + rho sum_i z_i^2 / (d_i - lambda) = 0 per remaining pole (a rational
// model of each side's poles, safeguarded by the bracket), eigenvector
// components from the recomputed z of Gu and Eisenstat (orthogonal vectors
// from computed roots), and the product of the block-diagonal Q with the
// merged vectors.  One block per problem; every loop is bounded.
constexpr int DC_LEAF = 32;
constexpr int DC_SECULAR_ITERS = 100;

// Eigenpairs of the leaf (d[0..m), e[0..m-1)) in place (d <- eigenvalues, e
// overwritten: a copy, e[m - 1] is set to 0), rotating the m x m block of Z
// whose first entry is zb (row stride ldz) from the identity; one warp, lane
// r owns the block's row r.
__device__ void dc_leaf_ql(double* d, double* e, int m, double* zb, int ldz, int lane, int* status) {
  const double eps = Eps<double>::v();
  double* zrow = zb + (size_t)(lane < m ? lane : 0) * ldz;
  if (lane < m) zrow[lane] = 1.0;
  if (lane == 0) e[m - 1] = 0.0;
  __syncwarp();
  double f = 0.0, tst1 = 0.0;
  for (int l = 0; l < m; ++l) {
    const double hl = fabs(d[l]) + fabs(e[l]);
    tst1 = hl > tst1 ? hl : tst1;
    for (int iter = 0;; ++iter) {
      int mm = l;
      while (mm < m - 1 && fabs(e[mm]) > eps * tst1) ++mm;
      if (mm == l) break;
      if (iter >= QL_MAX_SWEEPS) {
        if (lane == 0) atomicOr(status, 2);
        break;
      }
      const double g0 = d[l];
      double p = (d[l + 1] - g0) / (2.0 * e[l]);
      double r = hypot(p, 1.0);
      if (p < 0) r = -r;
      const double dl0 = e[l] / (p + r), dl1 = e[l] * (p + r);
      const double h0 = g0 - dl0;
      __syncwarp();
      if (lane == 0) {
        d[l] = dl0;
        d[l + 1] = dl1;
      }
      for (int i = l + 2 + lane; i < m; i += 32) d[i] -= h0;
      __syncwarp();
      f += h0;
      p = d[mm];
      double c = 1.0, c2 = 1.0, c3 = 1.0, s = 0.0, s2 = 0.0;
      const double el1 = e[l + 1];
      for (int i = mm - 1; i >= l; --i) {
        c3 = c2;
        c2 = c;
        s2 = s;
        const double ei = e[i], di = d[i];
        const double g = c * ei, h = c * p;
        r = hypot(p, ei);
        const double ei1 = s * r, rinv = 1.0 / r;
        s = ei * rinv;
        c = p * rinv;
        p = c * di - s * g;
        const double di1 = h + s * (c * g + s * di);
        __syncwarp();
        if (lane == 0) {
          e[i + 1] = ei1;
          d[i + 1] = di1;
        }
        if (lane < m) {
          const double zi = zrow[i], zi1 = zrow[i + 1];
          zrow[i + 1] = s * zi + c * zi1;
          zrow[i] = c * zi - s * zi1;
        }
        __syncwarp();
      }
      p = -s * s2 * c3 * el1 * e[l] / dl1;
      __syncwarp();
      if (lane == 0) {
        e[l] = s * p;
        d[l] = c * p;
      }
      __syncwarp();
      if (!(fabs(e[l]) > eps * tst1)) break;
    }
    __syncwarp();
    if (lane == 0) {
      d[l] += f;
      e[l] = 0.0;
    }
    __syncwarp();
  }
}

// The root of 1 + rho sum_q z2[q] / (p[q] - lambda) (rho > 0, p increasing,
// kk poles) in (p[i], p[i + 1]), or above p[kk - 1] for i = kk - 1, as
// lambda = p[j] + tau with j the pole nearer to the root, so that the
// differences p[q] - lambda = (p[q] - p[j]) - tau keep their relative
// accuracy.  Each step fits psi (the poles <= i) by q / (p_i - tau) + const
// and phi (the others) by s / (p_{i+1} - tau) + const through their values
// and slopes, and takes the model's root inside the bracket.
__device__ void dc_secular(const double* pole, const double* z2, double zsum, double rho, int i, int kk, int* jout,
                           double* tout) {
  const double eps = Eps<double>::v();
  const bool last = i == kk - 1;
  const double lo = pole[i], hi = last ? pole[i] + rho * zsum : pole[i + 1];
  const double mid = 0.5 * (lo + hi);
  double fmid = 1.0;
  for (int q = 0; q < kk; ++q) fmid += rho * z2[q] / (pole[q] - mid);
  const int j = (!last && fmid < 0) ? i + 1 : i;
  const double org = pole[j];
  double a = lo - org, b = hi - org;
  if (fmid < 0) a = fmax(a, mid - org);
  else b = fmin(b, mid - org);
  double tau = 0.5 * (a + b);
  for (int it = 0; it < DC_SECULAR_ITERS; ++it) {
    double psi = 0, dpsi = 0, phi = 0, dphi = 0;
    for (int q = 0; q < kk; ++q) {
      const double inv = 1.0 / ((pole[q] - org) - tau);
      const double t = z2[q] * inv;
      if (q <= i) {
        psi += t;
        dpsi += t * inv;
      } else {
        phi += t;
        dphi += t * inv;
      }
    }
    const double f = 1.0 + rho * (psi + phi);
    if (fabs(f) <= 8.0 * kk * eps * (1.0 + rho * (fabs(psi) + fabs(phi)))) break;
    if (f < 0) a = fmax(a, tau);
    else b = fmin(b, tau);
    const double di = (pole[i] - org) - tau;
    const double qq = rho * dpsi * di * di;
    double c = f - qq / di;
    double eta;
    if (last) {
      eta = c != 0.0 ? di + qq / c : 0.5 * (a + b) - tau;
    } else {
      const double di1 = (pole[i + 1] - org) - tau;
      const double ss = rho * dphi * di1 * di1;
      c -= ss / di1;
      // c (di - eta)(di1 - eta) + qq (di1 - eta) + ss (di - eta) = 0
      const double A = c, B = -(c * (di + di1) + qq + ss), C = c * di * di1 + qq * di1 + ss * di;
      eta = 0.5 * (di + di1);
      if (fabs(A) < 1e-300) {
        if (B != 0.0) eta = -C / B;
      } else {
        const double sq = sqrt(fmax(B * B - 4.0 * A * C, 0.0));
        const double den = B > 0 ? -B - sq : -B + sq;
        double r1 = den != 0.0 ? den / (2.0 * A) : 0.5 * (di + di1);
        double r2 = (r1 != 0.0) ? C / (A * r1) : 0.5 * (di + di1);
        if (di < r1 && r1 < di1) eta = r1;
        else if (di < r2 && r2 < di1) eta = r2;
      }
    }
    double tn = tau + eta;
    if (!(a < tn && tn < b)) tn = 0.5 * (a + b);
    if (!(a < tn && tn < b)) break;  // the bracket is down to adjacent doubles
    const bool done = fabs(tn - tau) <= 4.0 * eps * fabs(tn);
    tau = tn;
    if (done) break;
  }
  *jout = j;
  *tout = tau;
}

__global__ void __launch_bounds__(TRI_THREADS) eig_dc(const EigProblem* __restrict__ probs, int* status) {
  const EigProblem P = probs[blockIdx.x];
  const int n = P.n;
  if (n <= 0) return;
  double* __restrict__ lam = P.lam;
  unsigned char* work = P.work;
  const EigLayout L = eig_layout<double>(n);
  double* W = (double*)work;
  int* I = (int*)(work + L.ints_off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TRI_THREADS / 32;
  double* Z = W + L.Z;     // n x n, row = coordinate, column = eigenvector
  double* U = W + L.dcU;   // merge scratch, stride n
  double* V = W + L.dcV;   // merge scratch, stride n
  double* vd = W + L.dcv;  // diagonal, then eigenvalues
  double* ve = vd + n;     // off-diagonal (ve[i] couples i, i + 1)
  double* pk = ve + n;     // merge: poles (then the kept, ascending)
  double* zk = pk + n;     // merge: z (then the kept z^2)
  double* ds = zk + n;     // merge: poles in ascending order
  double* zs = ds + n;     // merge: z in the same order
  double* tau = zs + n;    // merge: root offsets
  double* zh = tau + n;    // merge: recomputed z
  double* rcs = zh + n;    // merge: deflation rotations (c, s)
  double* rss = rcs + n;
  int* order = I + L.order;
  int* perm = I + L.dci;   // merge: sorted position -> local coordinate
  int* jr = perm + n;      // merge: root origin pole; deflation flags before
  int* kept = jr + n;      // merge: sorted positions of the kept poles
  int* rl = kept + n;      // merge: deflation rotation pairs
  int* ri = rl + n;
  int* act = ri + n;       // merge: columns that are not a copy of one column of Q
  __shared__ int s_kk, s_nrot;
  __shared__ double s_red[NW], s_rho, s_zsum;
  __shared__ double s_ld[NW][DC_LEAF], s_le[NW][DC_LEAF];

  int depth = 0;
  while (((n + (1 << depth) - 1) >> depth) > DC_LEAF) ++depth;
  // Cuppen cuts of every level: the two diagonal entries beside each cut lose beta
  if (tid == 0)
    for (int dd = 0; dd < depth; ++dd)
      for (int q = 0; q < (1 << dd); ++q) {
        const int sp = ((2 * q + 1) * n) >> (dd + 1);
        const double beta = ve[sp - 1];
        vd[sp - 1] -= beta;
        vd[sp] -= beta;
      }
  for (size_t x = tid; x < (size_t)n * n; x += TRI_THREADS) Z[x] = 0.0;
  __syncthreads();
  // leaves, one warp each, on copies of (d, e) in shared memory (the entry of
  // e at a cut is the coupling its merge needs)
  for (int q = warp; q < (1 << depth); q += NW) {
    const int s0 = (q * n) >> depth, s1 = ((q + 1) * n) >> depth, m = s1 - s0;
    if (lane < m) {
      s_ld[warp][lane] = vd[s0 + lane];
      s_le[warp][lane] = ve[s0 + lane];
    }
    __syncwarp();
    dc_leaf_ql(s_ld[warp], s_le[warp], m, Z + (size_t)s0 * n + s0, n, lane, status);
    if (lane < m) vd[s0 + lane] = s_ld[warp][lane];
    __syncwarp();
  }
  __syncthreads();

  // merges, bottom-up; the whole block on one merge at a time
  for (int dd = depth - 1; dd >= 0; --dd) {
    for (int q = 0; q < (1 << dd); ++q) {
      const int s0 = (q * n) >> dd, s1 = ((q + 1) * n) >> dd, sp = ((2 * q + 1) * n) >> (dd + 1);
      const int k = s1 - s0, n1 = sp - s0;
      const double beta = ve[sp - 1];
      const double sgn = beta < 0 ? -1.0 : 1.0;
      // poles (sign-flipped for beta < 0) and z = (last row of Q1, first row of Q2)
      double part = 0.0;
      for (int j = tid; j < k; j += TRI_THREADS) {
        pk[j] = sgn * vd[s0 + j];
        const double zj = j < n1 ? Z[(size_t)(sp - 1) * n + s0 + j] : Z[(size_t)sp * n + s0 + j];
        zk[j] = zj;
        part += zj * zj;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) s_red[warp] = part;
      __syncthreads();
      if (tid == 0) {
        double z2 = 0.0;
        for (int w = 0; w < NW; ++w) z2 += s_red[w];
        s_rho = fabs(beta) * z2;
        s_red[0] = sqrt(z2);
      }
      __syncthreads();
      const double rho = s_rho, zn = s_red[0];
      // ascending order of the poles (stable)
      for (int j = tid; j < k; j += TRI_THREADS) {
        const double pj = pk[j];
        int rank = 0;
        for (int t = 0; t < k; ++t) {
          const double pt = pk[t];
          rank += (pt < pj) || (pt == pj && t < j);
        }
        perm[rank] = j;
      }
      __syncthreads();
      for (int r = tid; r < k; r += TRI_THREADS) {
        ds[r] = pk[perm[r]];
        zs[r] = zn > 0.0 ? zk[perm[r]] / zn : 0.0;
      }
      __syncthreads();
      // deflation (one thread): negligible rho z_i, and pairs of poles whose
      // rotation onto one z component leaves an off-diagonal below tol
      if (tid == 0) {
        double dmax = 0.0;
        for (int r = 0; r < k; ++r) dmax = fmax(dmax, fabs(ds[r]));
        const double tol = 8.0 * Eps<double>::v() * fmax(dmax, rho);
        int nrot = 0, last = -1;
        for (int r = 0; r < k; ++r) {
          jr[r] = 0;
          if (fabs(rho * zs[r]) <= tol) {
            jr[r] = 1;
            continue;
          }
          // |(d_r - d_last) c s| <= tol with c s = z_last z_r / t^2, tested first
          // without the square root and the divisions (rarely true)
          const double zl = last >= 0 ? zs[last] : 0.0, zr = zs[r];
          if (last >= 0 && fabs((ds[r] - ds[last]) * zl * zr) <= tol * (zl * zl + zr * zr)) {
            const double t = hypot(zl, zr);
            const double c = zl / t, s = zr / t;
            {
              const double dl = ds[last], dr = ds[r];
              zs[r] = t;
              zs[last] = 0.0;
              ds[r] = dl * c * c + dr * s * s;
              ds[last] = dl * s * s + dr * c * c;
              jr[last] = 1;
              rl[nrot] = last;
              ri[nrot] = r;
              rcs[nrot] = c;
              rss[nrot] = s;
              ++nrot;
            }
          }
          last = r;
        }
        int kk = 0;
        for (int r = 0; r < k; ++r) {
          act[r] = !jr[r] ? 1 : 0;
          if (!jr[r]) kept[kk++] = r;
        }
        for (int t = 0; t < nrot; ++t) act[rl[t]] = act[ri[t]] = 1;
        s_kk = kk;
        s_nrot = nrot;
      }
      __syncthreads();
      const int kk = s_kk, nrot = s_nrot;
      // the kept poles in ascending order (a rotation may have moved one by <= tol)
      for (int m = tid; m < kk; m += TRI_THREADS) {
        const double pm = ds[kept[m]];
        int rank = 0;
        for (int t = 0; t < kk; ++t) {
          const double pt = ds[kept[t]];
          rank += (pt < pm) || (pt == pm && t < m);
        }
        jr[rank] = kept[m];  // jr as scratch (flags are no longer needed)
      }
      __syncthreads();
      for (int m = tid; m < kk; m += TRI_THREADS) kept[m] = jr[m];
      __syncthreads();
      double zpart = 0.0;
      for (int m = tid; m < kk; m += TRI_THREADS) {
        pk[m] = ds[kept[m]];
        const double zm = zs[kept[m]];
        zk[m] = zm * zm;
        zh[m] = zm;  // its sign, for the recomputed z
        zpart += zm * zm;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) zpart += __shfl_xor_sync(0xffffffffu, zpart, o);
      if (lane == 0) s_red[warp] = zpart;
      __syncthreads();
      if (tid == 0) {
        double zsum = 0.0;
        for (int w = 0; w < NW; ++w) zsum += s_red[w];
        s_zsum = zsum;
      }
      __syncthreads();
      // one root per kept pole
      for (int m = tid; m < kk; m += TRI_THREADS) dc_secular(pk, zk, s_zsum, rho, m, kk, jr + m, tau + m);
      __syncthreads();
      // recomputed z (Gu-Eisenstat): zhat_m^2 = prod_i (lambda_i - p_m) / (rho prod_{i != m} (p_i - p_m))
      for (int m = tid; m < kk; m += TRI_THREADS) {
        const double pm = pk[m];
        double v = -((pm - pk[jr[m]]) - tau[m]) / rho;
        for (int t = 0; t < kk; ++t)
          if (t != m) v *= -((pm - pk[jr[t]]) - tau[t]) / (pk[t] - pm);
        const double a = sqrt(fabs(v));
        zh[m] = zh[m] < 0 ? -a : a;
      }
      __syncthreads();
      // vectors of the kept part: U[m][i] = zhat_m / (p_m - lambda_i), columns normalised
      for (size_t x = tid; x < (size_t)kk * kk; x += TRI_THREADS) {
        const int m = (int)(x / kk), i = (int)(x - (size_t)m * kk);
        U[(size_t)m * n + i] = zh[m] / ((pk[m] - pk[jr[i]]) - tau[i]);
      }
      __syncthreads();
      for (int i = tid; i < kk; i += TRI_THREADS) {
        double s2 = 0.0;
        for (int m = 0; m < kk; ++m) s2 += U[(size_t)m * n + i] * U[(size_t)m * n + i];
        const double inv = 1.0 / sqrt(s2);
        for (int m = 0; m < kk; ++m) U[(size_t)m * n + i] *= inv;
      }
      __syncthreads();
      // V (sorted coordinates): identity on the deflated positions, U on the
      // kept ones; then the deflation rotations, last first; eigenvalues
      for (size_t x = tid; x < (size_t)k * k; x += TRI_THREADS) {
        const int r = (int)(x / k), c = (int)(x - (size_t)r * k);
        V[(size_t)r * n + c] = r == c ? 1.0 : 0.0;
      }
      __syncthreads();
      for (size_t x = tid; x < (size_t)kk * kk; x += TRI_THREADS) {
        const int m = (int)(x / kk), i = (int)(x - (size_t)m * kk);
        V[(size_t)kept[m] * n + kept[i]] = U[(size_t)m * n + i];
      }
      __syncthreads();
      for (int c = tid; c < k; c += TRI_THREADS) {
        for (int t = nrot - 1; t >= 0; --t) {
          const int a = rl[t], b = ri[t];
          const double cc = rcs[t], ss = rss[t];
          const double va = V[(size_t)a * n + c], vb = V[(size_t)b * n + c];
          V[(size_t)a * n + c] = -ss * va + cc * vb;
          V[(size_t)b * n + c] = cc * va + ss * vb;
        }
      }
      __syncthreads();
      // rows back to the local coordinates: U[perm[r]][c] = V[r][c]
      for (size_t x = tid; x < (size_t)k * k; x += TRI_THREADS) {
        const int r = (int)(x / k), c = (int)(x - (size_t)r * k);
        U[(size_t)perm[r] * n + c] = V[(size_t)r * n + c];
      }
      __syncthreads();
      // Z block <- blockdiag(Q1, Q2) U (through V); a column deflated without a
      // rotation is the unit vector of its pole, so Q's column perm[c] itself
      for (size_t x = tid; x < (size_t)k * k; x += TRI_THREADS) {
        const int r = (int)(x / k), c = (int)(x - (size_t)r * k);
        const double* zr = Z + (size_t)(s0 + r) * n + s0;
        if (!act[c]) {
          V[(size_t)r * n + c] = zr[perm[c]];
          continue;
        }
        const int j0 = r < n1 ? 0 : n1, j1 = r < n1 ? n1 : k;
        double acc = 0.0;
        for (int j = j0; j < j1; ++j) acc += zr[j] * U[(size_t)j * n + c];
        V[(size_t)r * n + c] = acc;
      }
      __syncthreads();
      for (size_t x = tid; x < (size_t)k * k; x += TRI_THREADS) {
        const int r = (int)(x / k), c = (int)(x - (size_t)r * k);
        Z[(size_t)(s0 + r) * n + s0 + c] = V[(size_t)r * n + c];
      }
      // eigenvalue of column c (sorted position c): the root of the kept pole
      // there, or the (rotated) deflated pole itself
      for (int c = tid; c < k; c += TRI_THREADS) vd[s0 + c] = sgn * ds[c];
      __syncthreads();
      for (int m = tid; m < kk; m += TRI_THREADS) vd[s0 + kept[m]] = sgn * (pk[jr[m]] + tau[m]);
      __syncthreads();
    }
  }
  // stable descending order of the eigenvalues
  for (int i = tid; i < n; i += TRI_THREADS) {
    const double di = vd[i];
    int rank = 0;
    for (int q = 0; q < n; ++q) {
      const double dq = vd[q];
      rank += (dq > di) || (dq == di && q < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRI_THREADS) lam[r] = vd[order[r]];
}


// Row `row` of Z (eigenvectors of the tridiagonal matrix as columns) starts as
// e_row and receives every recorded rotation in order.
template <typename T>
__global__ void eig_apply_rotations(const EigProblem* __restrict__ probs) {
  const EigProblem P = probs[blockIdx.y];
  const int n = P.n;
  unsigned char* work = P.work;
  const EigLayout L = eig_layout<T>(n);
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  T* W = (T*)work;
  const int* I = (const int*)(work + L.ints_off);
  const T* rc = W + L.rc;
  const T* rs = W + L.rs;
  T* z = W + L.Z + (size_t)row * n;
  for (int c = 0; c < n; ++c) z[c] = (c == row) ? (T)1 : (T)0;
  const int nseg = I[L.nseg];
  for (int sg = 0; sg < nseg; ++sg) {
    const int lo = I[L.seg_lo + sg], hi = I[L.seg_hi + sg];
    const size_t off = (size_t)I[L.seg_off + sg];
    T zi1 = z[hi + 1];
    for (int i = hi, q = 0; i >= lo; --i, ++q) {
      const T c = rc[off + q], s = rs[off + q];
      const T zi = z[i];
      z[i + 1] = s * zi + c * zi1;
      zi1 = c * zi - s * zi1;
    }
    z[lo] = zi1;
  }
}

// U[:, r] = H_0 ... H_{n-3} Z[:, order[r]] for r < k; one warp per vector.
template <typename T>
__global__ void eig_back_transform(const EigProblem* __restrict__ probs) {
  const EigProblem P = probs[blockIdx.y];
  const int n = P.n, k = P.k;
  unsigned char* work = P.work;
  double* __restrict__ U = P.U;
  const EigLayout L = eig_layout<T>(n);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= k) return;
  const T* W = (const T*)work;
  const int* I = (const int*)(work + L.ints_off);
  const T* A = W + L.A;
  const int col = I[L.order + warp];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* zr = (T*)dyn_smem + (size_t)(threadIdx.x >> 5) * n;
  for (int i = lane; i < n; i += 32) zr[i] = W[L.Z + (size_t)i * n + col];
  __syncwarp();
  for (int j = n - 3; j >= 0; --j) {
    const T tau = A[(size_t)j * n + j];
    if (tau == (T)0) continue;
    const T* Aj = A + (size_t)j * n;
    T acc = 0;
    for (int i = j + 2 + lane; i < n; i += 32) acc += Aj[i] * zr[i];
    acc = warp_sum_e(acc) + zr[j + 1];
    acc *= tau;
    __syncwarp();
    if (lane == 0) zr[j + 1] -= acc;
    for (int i = j + 2 + lane; i < n; i += 32) zr[i] -= acc * Aj[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) U[(size_t)i * k + warp] = (double)zr[i];
}

template <typename T>
void eig_launch(cudaStream_t st, const EigProblem* probs_dev, int nprob, int nmax, int kmax, int* status) {
  const size_t smem_A = (size_t)nmax * (nmax + 1) * sizeof(T);  // row stride n + 1 in shared memory
  const int use_smem = smem_A <= EIG_SMEM_LIMIT ? 1 : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(eig_tridiag_ql<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM_LIMIT);
    attr = true;
  }
  // FP64 problems: tridiagonalisation, then divide and conquer; float ones
  // keep the QL iteration and the replay of its rotations
  constexpr bool dc = sizeof(T) == sizeof(double);
  count_launches(kmax > 0 ? 3 : 2);
  eig_tridiag_ql<T><<<nprob, TRI_THREADS, use_smem ? smem_A : 0, st>>>(probs_dev, use_smem, status, dc ? 1 : 0);
  if constexpr (dc) {
    eig_dc<<<nprob, TRI_THREADS, 0, st>>>(probs_dev, status);
  } else {
    const int rows_per_block = 32;
    eig_apply_rotations<T><<<dim3((nmax + rows_per_block - 1) / rows_per_block, nprob), rows_per_block, 0, st>>>(
        probs_dev);
  }
  if (kmax > 0) {
    const int warps = 4;
    eig_back_transform<T><<<dim3((kmax + warps - 1) / warps, nprob), 32 * warps, (size_t)warps * nmax * sizeof(T),
                            st>>>(probs_dev);
  }
}
}  // namespace

size_t eig_work_bytes(int n, int prec_bits) {
  return prec_bits == 32 ? eig_layout<float>(n).bytes : eig_layout<double>(n).bytes;
}

void eig_sym_batched(cudaStream_t st, const EigProblem* probs_dev, int nprob, int nmax, int kmax, int prec_bits,
                     int* status) {
  if (nprob <= 0 || nmax <= 0) return;
  if (nmax > EIG_MAXN || kmax > nmax || kmax < 0) {
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  if (prec_bits == 32)
    eig_launch<float>(st, probs_dev, nprob, nmax, kmax, status);
  else
    eig_launch<double>(st, probs_dev, nprob, nmax, kmax, status);
}

void eig_sym(cudaStream_t st, int n, int k, const double* G, double* U, double* lam, void* work, int prec_bits,
             int* status) {
  if (n <= 0) return;
  if (n > EIG_MAXN || k > n || k < 0) {
    cudaMemsetAsync(status, 0xff, sizeof(int), st);
    return;
  }
  // the one-problem descriptor lives at the end of the caller's work area
  const size_t wb = eig_work_bytes(n, prec_bits);
  EigProblem P;
  P.n = n;
  P.k = k;
  P.G = G;
  P.U = U;
  P.lam = lam;
  P.work = (unsigned char*)work;
  EigProblem* d = (EigProblem*)((unsigned char*)work + ((wb + 255) & ~(size_t)255));
  cudaMemcpyAsync(d, &P, sizeof(P), cudaMemcpyHostToDevice, st);
  eig_sym_batched(st, d, 1, n, k, prec_bits, status);
}

}  // namespace qtt
