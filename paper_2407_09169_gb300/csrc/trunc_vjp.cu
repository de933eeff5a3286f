// Backward of the simultaneous bond truncation (the derivative of the SVD
// rounding, section "Matrix product state algorithm", with
// Lorentzian-broadened gaps), in tensor-train form on the device.
//
// The truncation keeps, at every cut n of a train X of N binary sites, the
// k_n leading left singular vectors of the unfolding X_(n) and applies all
// the projectors together: T(X) = Pi_1 ... Pi_{N-1} X.  With X held as
// left-orthonormal cores Q_1 .. Q_{N-1} and a last core C (so X_(n) = Q_{<=n}
// M_n with M_n the right part), the projectors come from the eigenpairs
// (V_n, lambda_n) of the right Grams M_n M_n^T: Pi_n = Q_{<=n} P_n Q_{<=n}^T,
// P_n = V_K V_K^T.  The vector-Jacobian product with a cotangent train Ybar
// (bonds s_n) is the train of bond 2 r_n
//     site 1: [Q_1  delta_1],  site n: [[Q_n  delta_n], [0  Q_n]],
//     site N: [[e_{N-1} Ybar_N], [C]],
// built from
//   left environments   Yhat_n = e_{n-1} (x) Ybar_n,  e_n = P_n Q_n^T Yhat_n,
//   right environments  R_{N-1} = Ybar_N C^T,
//                       R_{n-1} = sum_i Ybar_n[:, i, :] R_n (Q_n P_n)[:, i, :]^T,
//   per cut             g = Yhat_n R_n,  Shat = Q_n^T g + g^T Q_n,
//                       A = V_K diag(w0) V_K^T,
//                       Gamma = V_D (W o V_D^T Shat V_K) V_K^T,
//                       delta_n = (I - Q_n Q_n^T) g A + Q_n (Gamma + Gamma^T),
// with w0_i = 1 / lambda_i and W_ji = 1 / (lambda_i - lambda_j) (kept i,
// discarded j), or lambda / (lambda^2 + eps^2) for eps > 0.  The first term
// of delta_n is the part through the null space of X_(n) (outside the range
// of Q_{<=n}), the second the gaps inside it; together with the
// fixed-projector part e_{N-1} Ybar_N they are the exact derivative where
// the kept and discarded eigenvalues are separated.
//
// Everything is FP64: the products through the strided FP64 GEMM (operands
// as strided views, so every transpose and reshape is free), the right
// Grams' eigenpairs through the batched divide-and-conquer eigensolver, and
// four elementwise kernels below.
#include <algorithm>
#include <string>
#include <vector>

#include "engine.hpp"
#include "kernels.cuh"

namespace qtt {

namespace {

constexpr int kThreads = 256;
constexpr int kCutStreams = 4;  // streams the per-cut cores are spread over

int grid_for(long long total) {
  long long b = (total + kThreads - 1) / kThreads;
  return (int)std::max(1LL, std::min(b, 4096LL));
}

// out = H + H^T for an n x n row-major H (out does not alias H).
__global__ void sym_sum_kernel(int n, const double* __restrict__ H, double* __restrict__ out) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (long long)i * n);
    out[e] = H[e] + H[(long long)j * n + i];
  }
}

__device__ __forceinline__ double gap_weight(double d, double eps) {
  return eps > 0.0 ? d / (d * d + eps * eps) : 1.0 / d;
}

// out[i][c] = V[i][c] w0(lam[c]) for i < n, c < k (V row-major, leading
// dimension ldv; out n x k row-major).
__global__ void scale_kept_kernel(int n, int k, const double* __restrict__ V, int ldv, const double* __restrict__ lam,
                                  double eps, double* __restrict__ out) {
  const long long total = (long long)n * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e - (long long)i * k);
    out[e] = V[(long long)i * ldv + c] * gap_weight(lam[c], eps);
  }
}

// B[j][i] *= W(lam[i] - lam[k + j]) for j < nd, i < k (B nd x k row-major).
__global__ void gap_scale_kernel(int nd, int k, const double* __restrict__ lam, double eps, double* __restrict__ B) {
  const long long total = (long long)nd * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / k), i = (int)(e - (long long)j * k);
    B[e] *= gap_weight(lam[i] - lam[k + j], eps);
  }
}

// Core of the output train at a site before the last: Q is the site's
// rl x 2 x rr core of X and D its delta (rows (a, i), rr columns).  The
// first site (rl = 1) gives the 1 x 2 x 2rr core [Q D]; the others the
// 2rl x 2 x 2rr core [[Q D], [0 Q]].
__global__ void assemble_core_kernel(int rl, int rr, int first, const double* __restrict__ Q,
                                     const double* __restrict__ D, double* __restrict__ out) {
  const int orl = first ? 1 : 2 * rl, orr = 2 * rr;
  const long long total = (long long)orl * 2 * orr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / (2 * orr));
    const int rem = (int)(e - (long long)a * 2 * orr);
    const int i = rem / orr, b = rem - i * orr;
    double v;
    if (a < rl)
      v = b < rr ? Q[((long long)a * 2 + i) * rr + b] : D[((long long)a * 2 + i) * rr + (b - rr)];
    else
      v = b < rr ? 0.0 : Q[((long long)(a - rl) * 2 + i) * rr + (b - rr)];
    out[e] = v;
  }
}

// Last core (2rl x 2 x 1): rows a < rl from L (rl x 2), the rest from C.
__global__ void assemble_last_kernel(int rl, const double* __restrict__ L, const double* __restrict__ Cc,
                                     double* __restrict__ out) {
  const int total = 4 * rl;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x)
    out[e] = e < 2 * rl ? L[e] : Cc[e - 2 * rl];
}

MatView mat(const double* p, long long rs, long long cs) {
  MatView v;
  v.p = p;
  v.rs = rs;
  v.cs = cs;
  return v;
}
OutView outm(double* p, long long ld) {
  OutView v;
  v.p = p;
  v.rs = ld;
  v.cs = 1;
  return v;
}

// C (M x N, leading dimension N) = alpha A B + beta C, one product on 16 x 16
// output tiles: the products here are at most a few hundred on a side and
// many are skinny (the discarded block is often a few columns), where a
// 64 x 64 tile would spend most of the scarce FP64 issue on masked rows.
void mm(cudaStream_t st, int M, int N, int K, double alpha, MatView A, MatView B, double beta, double* Cp) {
  gemm_f64_tiles16(st, M, N, K, alpha, A, B, beta, outm(Cp, N));
}

// Streams and events of one call, destroyed on every path out of it.
struct Streams {
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> ev;
  void make(int ns, int nev) {
    for (int i = 0; i < ns; ++i) {
      cudaStream_t x;
      QTT_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      s.push_back(x);
    }
    for (int i = 0; i < nev; ++i) {
      cudaEvent_t e;
      QTT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ev.push_back(e);
    }
  }
  ~Streams() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t x : s) cudaStreamDestroy(x);
  }
};

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

size_t truncate_vjp_out_elems(int N, const int* rx) {
  size_t tot = 0;
  for (int j = 0; j < N; ++j) {
    const size_t bl = j == 0 ? 1 : 2 * (size_t)rx[j];
    const size_t br = j == N - 1 ? 1 : 2 * (size_t)rx[j + 1];
    tot += bl * 2 * br;
  }
  return tot;
}

void truncate_vjp(cudaStream_t st, int N, const int* rx, const double* x, const int* sy, const double* ybar, int chi,
                  double tol, double eps, double* xbar, int* kept) {
  // 1-based sites n = 1 .. N: X site n has bonds r[n-1] x 2 x r[n]
  std::vector<long long> r(N + 1), s(N + 1);
  for (int n = 0; n <= N; ++n) {
    r[n] = rx[n];
    s[n] = sy[n];
  }
  std::vector<size_t> xo(N + 2, 0), yo(N + 2, 0), oo(N + 2, 0);
  for (int n = 1; n <= N; ++n) {
    xo[n + 1] = xo[n] + (size_t)(r[n - 1] * 2 * r[n]);
    yo[n + 1] = yo[n] + (size_t)(s[n - 1] * 2 * s[n]);
    const size_t bl = n == 1 ? 1 : 2 * (size_t)r[n - 1];
    const size_t br = n == N ? 1 : 2 * (size_t)r[n];
    oo[n + 1] = oo[n] + bl * 2 * br;
  }
  auto Xs = [&](int n) { return x + xo[n]; };
  auto Ys = [&](int n) { return ybar + yo[n]; };
  long long rmax = 1, smax = 1;
  for (int n = 0; n <= N; ++n) {
    rmax = std::max(rmax, r[n]);
    smax = std::max(smax, s[n]);
  }
  const long long mx = std::max(rmax, smax);
  const size_t tmax = 2 * (size_t)mx * (size_t)mx;

  // double work area: per-cut Gram, eigenvectors, eigenvalues, P, Q P,
  // Yhat, e, R; then the shared temporaries
  std::vector<size_t> gO(N + 1), uO(N + 1), lO(N + 1), pO(N + 1), qpO(N + 1), yhO(N + 1), eO(N + 1), rO(N + 1);
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += (n + 31) & ~(size_t)31;
    return o;
  };
  for (int n = 1; n < N; ++n) {
    gO[n] = take((size_t)(r[n] * r[n]));
    uO[n] = take((size_t)(r[n] * r[n]));
    lO[n] = take((size_t)r[n]);
    pO[n] = take((size_t)(r[n] * r[n]));
    qpO[n] = take((size_t)(2 * r[n - 1] * r[n]));
    yhO[n] = take((size_t)(2 * r[n - 1] * s[n]));
    rO[n] = take((size_t)(s[n] * r[n]));
  }
  for (int n = 0; n < N; ++n) eO[n] = take((size_t)(r[n] * s[n]));
  const size_t lastO = take((size_t)(2 * r[N - 1]));
  const size_t taO = take(tmax), trO = take(tmax);
  enum { T_G, T_H, T_S, T_VF, T_AM, T_B1, T_B, T_C1, T_GAM, T_U, T_GA, T_COUNT };
  size_t tO[kCutStreams][T_COUNT];
  for (int c = 0; c < kCutStreams; ++c)
    for (int t = 0; t < T_COUNT; ++t) tO[c][t] = take(tmax);
  const size_t ndbl = off;

  // byte work area: eigensolver work per cut, descriptors, status
  std::vector<size_t> wO(N + 1);
  size_t boff = 0;
  for (int n = 1; n < N; ++n) {
    wO[n] = boff;
    boff += (eig_work_bytes((int)r[n], 64) + 255) & ~(size_t)255;
  }
  const size_t descO = boff;
  boff += ((size_t)(N - 1) * sizeof(EigProblem) + 255) & ~(size_t)255;
  const size_t statO = boff;
  boff += 256;

  DevBuf dbuf, bbuf;
  QTT_CUDA(cudaMalloc(&dbuf.p, ndbl * sizeof(double)));
  QTT_CUDA(cudaMalloc(&bbuf.p, boff));
  double* W = (double*)dbuf.p;
  unsigned char* B = (unsigned char*)bbuf.p;
  int* status = (int*)(B + statO);
  QTT_CUDA(cudaMemsetAsync(W, 0, ndbl * sizeof(double), st));
  QTT_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  double* const TA = W + taO;
  double* const TR = W + trO;

  // right Grams: G_{N-1} = C C^T, G_{n-1} = sum_i Q_n[:, i, :] G_n Q_n[:, i, :]^T
  {
    const long long rl = r[N - 1];
    mm(st, (int)rl, (int)rl, 2, 1.0, mat(Xs(N), 2, 1), mat(Xs(N), 1, 2), 0.0, W + gO[N - 1]);
  }
  for (int n = N - 1; n >= 2; --n) {
    const long long rl = r[n - 1], rr = r[n];
    mm(st, (int)(2 * rl), (int)rr, (int)rr, 1.0, mat(Xs(n), rr, 1), mat(W + gO[n], rr, 1), 0.0, TA);
    mm(st, (int)rl, (int)rl, (int)(2 * rr), 1.0, mat(TA, 2 * rr, 1), mat(Xs(n), 1, 2 * rr), 0.0, W + gO[n - 1]);
  }

  // all eigenpairs of every right Gram, one block per cut
  {
    std::vector<EigProblem> probs((size_t)(N - 1));
    for (int n = 1; n < N; ++n) {
      EigProblem& p = probs[(size_t)(n - 1)];
      p.n = (int)r[n];
      p.k = (int)r[n];
      p.G = W + gO[n];
      p.U = W + uO[n];
      p.lam = W + lO[n];
      p.work = B + wO[n];
    }
    EigProblem* dprobs = (EigProblem*)(B + descO);
    QTT_CUDA(cudaMemcpyAsync(dprobs, probs.data(), probs.size() * sizeof(EigProblem), cudaMemcpyHostToDevice, st));
    eig_sym_batched(st, dprobs, N - 1, (int)rmax, (int)rmax, 64, status);
    QTT_CUDA(cudaStreamSynchronize(st));  // the descriptors' host copy may go
  }
  std::vector<std::vector<double>> lamh((size_t)N);
  int hstatus = 0;
  QTT_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  for (int n = 1; n < N; ++n) {
    lamh[(size_t)n].resize((size_t)r[n]);
    QTT_CUDA(cudaMemcpyAsync(lamh[(size_t)n].data(), W + lO[n], (size_t)r[n] * sizeof(double), cudaMemcpyDeviceToHost,
                             st));
  }
  QTT_CUDA(cudaStreamSynchronize(st));
  if (hstatus != 0)
    throw std::runtime_error("the eigen-decomposition of a right Gram failed (status " + std::to_string(hstatus) + ")");

  // kept counts: k_n = min(chi, #{lambda_i > max(tol^2, 1e-24) lambda_0})
  std::vector<int> k((size_t)N, 0);
  for (int n = 1; n < N; ++n) {
    const std::vector<double>& l = lamh[(size_t)n];
    int c = 0;
    if (l[0] > 0.0) {
      const double thr = std::max(tol * tol, 1e-24) * l[0];
      for (double v : l) c += v > thr ? 1 : 0;
    }
    k[(size_t)n] = std::min(chi, c);
    kept[n - 1] = k[(size_t)n];
  }

  // P_n = V_K V_K^T
  for (int n = 1; n < N; ++n) {
    const long long rr = r[n];
    const double* U = W + uO[n];
    mm(st, (int)rr, (int)rr, k[(size_t)n], 1.0, mat(U, rr, 1), mat(U, 1, rr), 0.0, W + pO[n]);
  }

  // the two environment sweeps run side by side, then the cuts over
  // kCutStreams streams; events order them after the projectors and before
  // the end of the call
  Streams ss;
  ss.make(2 + kCutStreams, 3 + kCutStreams);
  cudaStream_t sl_st = ss.s[0], sr_st = ss.s[1];
  cudaEvent_t ev_p = ss.ev[0], ev_l = ss.ev[1], ev_r = ss.ev[2];
  QTT_CUDA(cudaEventRecord(ev_p, st));
  QTT_CUDA(cudaStreamWaitEvent(sl_st, ev_p, 0));
  QTT_CUDA(cudaStreamWaitEvent(sr_st, ev_p, 0));

  // left environments
  fill_value(sl_st, W + eO[0], 1, 1.0);
  for (int n = 1; n < N; ++n) {
    const long long rl = r[n - 1], rr = r[n], sl = s[n - 1], sr = s[n];
    mm(sl_st, (int)rl, (int)(2 * sr), (int)sl, 1.0, mat(W + eO[n - 1], sl, 1), mat(Ys(n), 2 * sr, 1), 0.0,
       W + yhO[n]);
    mm(sl_st, (int)rr, (int)sr, (int)(2 * rl), 1.0, mat(Xs(n), 1, rr), mat(W + yhO[n], sr, 1), 0.0, TA);
    mm(sl_st, (int)rr, (int)sr, (int)rr, 1.0, mat(W + pO[n], rr, 1), mat(TA, sr, 1), 0.0, W + eO[n]);
  }
  {
    const long long rl = r[N - 1], sl = s[N - 1];
    mm(sl_st, (int)rl, 2, (int)sl, 1.0, mat(W + eO[N - 1], sl, 1), mat(Ys(N), 2, 1), 0.0, W + lastO);
  }
  QTT_CUDA(cudaEventRecord(ev_l, sl_st));

  // right environments against X's projected right part
  for (int n = 2; n < N; ++n) {
    const long long rl = r[n - 1], rr = r[n];
    mm(sr_st, (int)(2 * rl), (int)rr, (int)rr, 1.0, mat(Xs(n), rr, 1), mat(W + pO[n], rr, 1), 0.0, W + qpO[n]);
  }
  {
    const long long rl = r[N - 1], sl = s[N - 1];
    mm(sr_st, (int)sl, (int)rl, 2, 1.0, mat(Ys(N), 2, 1), mat(Xs(N), 1, 2), 0.0, W + rO[N - 1]);
  }
  for (int n = N - 1; n >= 2; --n) {
    const long long rl = r[n - 1], rr = r[n], sl = s[n - 1], sr = s[n];
    mm(sr_st, (int)(2 * sl), (int)rr, (int)sr, 1.0, mat(Ys(n), sr, 1), mat(W + rO[n], rr, 1), 0.0, TR);
    mm(sr_st, (int)sl, (int)rl, (int)(2 * rr), 1.0, mat(TR, 2 * rr, 1), mat(W + qpO[n], 1, 2 * rr), 0.0,
       W + rO[n - 1]);
  }
  QTT_CUDA(cudaEventRecord(ev_r, sr_st));
  for (int c = 0; c < kCutStreams; ++c) {
    QTT_CUDA(cudaStreamWaitEvent(ss.s[2 + c], ev_l, 0));
    QTT_CUDA(cudaStreamWaitEvent(ss.s[2 + c], ev_r, 0));
  }

  // one delta core per cut, written into the output train with X's cores
  for (int n = 1; n < N; ++n) {
    const int c = (n - 1) % kCutStreams;
    cudaStream_t cs = ss.s[2 + c];
    double* T[T_COUNT];
    for (int t = 0; t < T_COUNT; ++t) T[t] = W + tO[c][t];
    const long long rl = r[n - 1], rr = r[n], sr = s[n];
    const int kk = k[(size_t)n], nd = (int)rr - kk;
    const double* U = W + uO[n];
    const double* L = W + lO[n];
    const double* Q = Xs(n);
    mm(cs, (int)(2 * rl), (int)rr, (int)sr, 1.0, mat(W + yhO[n], sr, 1), mat(W + rO[n], rr, 1), 0.0, T[T_G]);
    mm(cs, (int)rr, (int)rr, (int)(2 * rl), 1.0, mat(Q, 1, rr), mat(T[T_G], rr, 1), 0.0, T[T_H]);
    count_launches(1);
    sym_sum_kernel<<<grid_for(rr * rr), kThreads, 0, cs>>>((int)rr, T[T_H], T[T_S]);
    if (kk > 0) {
      count_launches(1);
      scale_kept_kernel<<<grid_for(rr * kk), kThreads, 0, cs>>>((int)rr, kk, U, (int)rr, L, eps, T[T_VF]);
    }
    mm(cs, (int)rr, (int)rr, kk, 1.0, mat(T[T_VF], kk, 1), mat(U, 1, rr), 0.0, T[T_AM]);
    if (kk > 0 && nd > 0) {
      mm(cs, nd, (int)rr, (int)rr, 1.0, mat(U + kk, 1, rr), mat(T[T_S], rr, 1), 0.0, T[T_B1]);
      mm(cs, nd, kk, (int)rr, 1.0, mat(T[T_B1], rr, 1), mat(U, rr, 1), 0.0, T[T_B]);
      count_launches(1);
      gap_scale_kernel<<<grid_for((long long)nd * kk), kThreads, 0, cs>>>(nd, kk, L, eps, T[T_B]);
      mm(cs, (int)rr, kk, nd, 1.0, mat(U + kk, rr, 1), mat(T[T_B], kk, 1), 0.0, T[T_C1]);
      mm(cs, (int)rr, (int)rr, kk, 1.0, mat(T[T_C1], kk, 1), mat(U, 1, rr), 0.0, T[T_GAM]);
      count_launches(1);
      sym_sum_kernel<<<grid_for(rr * rr), kThreads, 0, cs>>>((int)rr, T[T_GAM], T[T_U]);
    } else {
      QTT_CUDA(cudaMemsetAsync(T[T_U], 0, (size_t)(rr * rr) * sizeof(double), cs));
    }
    // gA = g A;  u = Gamma + Gamma^T - Q^T gA;  delta = gA + Q u
    mm(cs, (int)(2 * rl), (int)rr, (int)rr, 1.0, mat(T[T_G], rr, 1), mat(T[T_AM], rr, 1), 0.0, T[T_GA]);
    mm(cs, (int)rr, (int)rr, (int)(2 * rl), -1.0, mat(Q, 1, rr), mat(T[T_GA], rr, 1), 1.0, T[T_U]);
    mm(cs, (int)(2 * rl), (int)rr, (int)rr, 1.0, mat(Q, rr, 1), mat(T[T_U], rr, 1), 1.0, T[T_GA]);
    const long long ocore = (n == 1 ? 1 : 2 * rl) * 2 * (2 * rr);
    count_launches(1);
    assemble_core_kernel<<<grid_for(ocore), kThreads, 0, cs>>>((int)rl, (int)rr, n == 1 ? 1 : 0, Q, T[T_GA],
                                                                 xbar + oo[n]);
  }
  QTT_CUDA(cudaStreamWaitEvent(st, ev_l, 0));
  count_launches(1);
  assemble_last_kernel<<<1, kThreads, 0, st>>>((int)r[N - 1], W + lastO, Xs(N), xbar + oo[N]);
  for (int c = 0; c < kCutStreams; ++c) {
    QTT_CUDA(cudaEventRecord(ss.ev[3 + c], ss.s[2 + c]));
    QTT_CUDA(cudaStreamWaitEvent(st, ss.ev[3 + c], 0));
  }
  QTT_CUDA(cudaGetLastError());
  QTT_CUDA(cudaStreamSynchronize(st));
}

}  // namespace qtt
