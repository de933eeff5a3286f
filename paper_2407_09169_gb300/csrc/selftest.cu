// Device self-checks behind qtt_selftest: each kernel family against an
// independent computation on seeded random operands.
#include <cmath>
#include <stdexcept>
#include <string>
#include <vector>

#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace qtt {

namespace {
struct DBuf {
  double* p = nullptr;
  explicit DBuf(size_t n) {
    if (cudaMalloc(&p, (n + 16) * sizeof(double)) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest");
  }
  ~DBuf() { cudaFree(p); }
};

// FP64 throughput probes.  Every thread runs kChains independent dependency
// chains (enough to hide the pipeline latency) for `iters` rounds; the final
// values are summed into *sink so that nothing is dead code.
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) dfma_rate_kernel(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) *sink = s;  // never true for the operands used; keeps the chains live
}

// mma.sync.m8n8k4 in FP64 (one warp: D = A B + C, 8 x 8 x 4, 256 FMAs), four
// independent accumulators per warp.
__global__ void __launch_bounds__(256) dmma_rate_kernel(int iters, double a, double b, double* sink) {
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) d[c][0] = d[c][1] = 1e-3 * (threadIdx.x + c);
  const double av = a + 1e-9 * threadIdx.x, bv = b;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(av), "d"(bv));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  if (s == 12345.678) *sink = s;
}

std::vector<double> down(const double* d, size_t n) {
  std::vector<double> h(n);
  if (cudaMemcpy(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    throw std::runtime_error("CUDA error: selftest copy");
  return h;
}
}  // namespace

// which = 0: tensor-core GEMM modes against the FP64 GEMM.  For every case
// and mode (BF16X3, TF32, TF32X3, BF16, BF16X6, BF16X10) one value:
// max |C_tc - C_64| / max |C_64|.
// which = 1: QR (FP64, FP32, FP32 + one FP64 Newton-Schulz step): ||Q^T Q - I||_max and
//   ||Q Q^T Y - Y|| / ||Y|| per case and run.
// which = 2: eigensolver (FP64 and FP32): ||G U - U diag(lam)|| / ||G|| and ||U^T U - I||_max.
// which = 3: bias of the tensor-core modes (TF32X3, BF16X3, BF16X6) on positive
// operands, K in {32, 256, 2048}, with and without a one-k-block cap per
// accumulator: (mean, max) of the signed relative error (C_tc - C_64) / C_64.
std::vector<double> run_selftest(int which) {
  cudaStream_t st = nullptr;
  std::vector<double> out;
  int* err = nullptr;
  if (cudaMalloc(&err, 16) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest");
  cudaMemset(err, 0, 16);
  if (which == 0) {
    struct Case {
      int M, N, K, outer, inner;
      bool ta, tb;
      double beta;
    };
    const Case cases[] = {
        {128, 128, 64, 1, 1, false, false, 0.0},  {300, 136, 200, 1, 1, false, false, 0.0},
        {130, 70, 100, 3, 2, true, false, 0.0},  {272, 136, 5000, 1, 1, false, true, 0.0},
        {256, 256, 128, 2, 1, false, false, 0.5}, {136, 160, 272, 1, 1, true, true, 1.0},
        {17, 300, 40, 4, 1, false, false, 0.0}};
    const size_t ws_elems = (size_t)32 << 20;
    DBuf ws(ws_elems);
    size_t pack_bytes = (size_t)256 << 20;
    void* pack = nullptr;
    if (cudaMalloc(&pack, pack_bytes) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest pack");
    unsigned long long seed = 12345;
    for (const Case& c : cases) {
      const long long batch = (long long)c.outer * c.inner;
      const size_t asz = (size_t)c.M * c.K * batch, bsz = (size_t)c.K * c.N * batch, csz = (size_t)c.M * c.N * batch;
      DBuf A(asz), B(bsz), C0(csz), C1(csz);
      fill_gaussian(st, A.p, asz, 1.0, seed++, 1);
      fill_gaussian(st, B.p, bsz, 1.0, seed++, 2);
      MatView av, bv;
      av.p = A.p;
      av.rs = c.ta ? 1 : c.K;
      av.cs = c.ta ? c.M : 1;
      av.si = (long long)c.M * c.K;
      av.so = av.si * c.inner;
      bv.p = B.p;
      bv.rs = c.tb ? 1 : c.N;
      bv.cs = c.tb ? c.K : 1;
      bv.si = (long long)c.K * c.N;
      bv.so = bv.si * c.inner;
      for (int mode = 0; mode < 6; ++mode) {
        fill_gaussian(st, C0.p, csz, 1.0, 777, 3);
        fill_gaussian(st, C1.p, csz, 1.0, 777, 3);
        OutView c0, c1;
        c0.p = C0.p;
        c0.rs = c.N;
        c0.cs = 1;
        c0.si = (long long)c.M * c.N;
        c0.so = c0.si * c.inner;
        c1 = c0;
        c1.p = C1.p;
        gemm_f64(st, c.M, c.N, c.K, c.outer, c.inner, 1.5, av, bv, c.beta, c0, ws.p, ws_elems);
        const int tc_mode[6] = {TC_BF16X3, TC_TF32, TC_TF32X3, TC_BF16, TC_BF16X6, TC_BF16X10};
        if (!gemm_tc(st, tc_mode[mode], c.M, c.N, c.K, c.outer, c.inner, 1.5, av, bv, c.beta, c1, pack, pack_bytes,
                     ws.p, ws_elems, err)) {
          out.push_back(-1.0);
          continue;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("CUDA error: selftest gemm");
        std::vector<double> h0 = down(C0.p, csz), h1 = down(C1.p, csz);
        double mx = 0, md = 0;
        for (size_t i = 0; i < csz; ++i) {
          mx = std::fmax(mx, std::fabs(h0[i]));
          md = std::fmax(md, std::fabs(h0[i] - h1[i]));
        }
        out.push_back(md / (mx > 0 ? mx : 1.0));
      }
    }
    cudaFree(pack);
  } else if (which == 1) {
    const int shapes[][2] = {{272, 136}, {64, 33}, {256, 256}, {40, 1}, {288, 143}, {150, 77}, {200, 120}, {96, 2},
                             {288, 144}, {160, 80}, {97, 49}, {161, 81}, {144, 72}};
    for (auto& sh : shapes) {
      const int m = sh[0], n = sh[1];
      DBuf Y((size_t)m * n), Q((size_t)m * n), W((size_t)2 * m * n + n + 64), Qf((size_t)m * n),
          G((size_t)8 * n * n);
      fill_gaussian(st, Y.p, (size_t)m * n, 1.0, 99 + m, 5);
      // FP64 QR; float QR; float QR + one FP64 Newton-Schulz step
      for (int run = 0; run < 3; ++run) {
        if (run < 2) {
          qr_thin(st, m, n, Y.p, Q.p, W.p, run == 0 ? 64 : 32, err);
        } else {
          qr_thin(st, m, n, Y.p, Qf.p, W.p, 32, err);
          newton_schulz_step(st, m, n, Qf.p, G.p, Q.p);
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("CUDA error: selftest qr");
        std::vector<double> y = down(Y.p, (size_t)m * n), q = down(Q.p, (size_t)m * n);
        double orth = 0;
        for (int a = 0; a < n; ++a)
          for (int b2 = 0; b2 < n; ++b2) {
            double s = 0;
            for (int i = 0; i < m; ++i) s += q[(size_t)i * n + a] * q[(size_t)i * n + b2];
            orth = std::fmax(orth, std::fabs(s - (a == b2 ? 1.0 : 0.0)));
          }
        // projection residual ||Y - Q Q^T Y||_F / ||Y||_F
        double num = 0, den = 0;
        for (int c = 0; c < n; ++c) {
          std::vector<double> coef(n, 0.0);
          for (int a = 0; a < n; ++a)
            for (int i = 0; i < m; ++i) coef[a] += q[(size_t)i * n + a] * y[(size_t)i * n + c];
          for (int i = 0; i < m; ++i) {
            double r = y[(size_t)i * n + c];
            for (int a = 0; a < n; ++a) r -= q[(size_t)i * n + a] * coef[a];
            num += r * r;
            den += y[(size_t)i * n + c] * y[(size_t)i * n + c];
          }
        }
        out.push_back(orth);
        out.push_back(std::sqrt(num / den));
      }
    }
  } else if (which == 2) {
    // (size, spectrum): 0 G = X diag(10^(-6 k / n)) X^T (X Gaussian); with Q
    // orthonormal (Gram-Schmidt of a Gaussian X on the host) G = Q diag(w) Q^T
    // for 1: w_k = 10^(-6 k / 20) for k < 20 and 0 beyond (rank 20), 2: w_k =
    // 1/2 for k < 40 (a 40-fold eigenvalue) and 1 + k / n beyond, 3: w_k =
    // 10^(-30 k / n) (graded far below the double precision of the largest)
    const int cases[][2] = {{136, 0}, {64, 0}, {7, 0}, {1, 0}, {200, 0}, {136, 1}, {136, 2}, {136, 3}, {200, 1}, {200, 3}, {520, 0}};
    for (const auto& cs : cases) {
      const int n = cs[0], kind = cs[1];
      std::vector<double> x((size_t)n * n);
      DBuf X((size_t)n * n), G((size_t)n * n), U((size_t)n * n), L(n), W(eig_work_bytes(n, 64) / 8 + 64);
      fill_gaussian(st, X.p, (size_t)n * n, 1.0, 4242 + n + 1000 * kind, 6);
      if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("CUDA error: selftest eig");
      x = down(X.p, (size_t)n * n);
      std::vector<double> w(n);
      for (int k = 0; k < n; ++k)
        w[k] = kind == 0   ? std::pow(10.0, -6.0 * k / n)
               : kind == 1 ? (k < 20 ? std::pow(10.0, -6.0 * k / 20) : 0.0)
               : kind == 2 ? (k < 40 ? 0.5 : 1.0 + (double)k / n)
                           : std::pow(10.0, -30.0 * k / n);
      if (kind != 0) {  // columns of x orthonormal (modified Gram-Schmidt, twice)
        for (int pass = 0; pass < 2; ++pass)
          for (int k = 0; k < n; ++k) {
            for (int j = 0; j < k; ++j) {
              double d = 0;
              for (int i = 0; i < n; ++i) d += x[(size_t)i * n + j] * x[(size_t)i * n + k];
              for (int i = 0; i < n; ++i) x[(size_t)i * n + k] -= d * x[(size_t)i * n + j];
            }
            double nr = 0;
            for (int i = 0; i < n; ++i) nr += x[(size_t)i * n + k] * x[(size_t)i * n + k];
            nr = std::sqrt(nr);
            for (int i = 0; i < n; ++i) x[(size_t)i * n + k] /= nr;
          }
      }
      std::vector<double> g((size_t)n * n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double s = 0;
          for (int k = 0; k < n; ++k) s += x[(size_t)i * n + k] * x[(size_t)j * n + k] * w[k];
          g[(size_t)i * n + j] = s;
        }
      if (cudaMemcpy(G.p, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        throw std::runtime_error("CUDA error: selftest eig upload");
      for (int prec : {64, 32}) {
        eig_sym(st, n, n, G.p, U.p, L.p, W.p, prec, err);
        if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("CUDA error: selftest eig");
        std::vector<double> u = down(U.p, (size_t)n * n), lam = down(L.p, n);
        double gn = 0, res = 0, orth = 0, order = 0;
        for (double v : g) gn = std::fmax(gn, std::fabs(v));
        for (int c = 0; c < n; ++c) {
          if (c > 0 && lam[c] > lam[c - 1]) order = 1;
          for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += g[(size_t)i * n + k] * u[(size_t)k * n + c];
            res = std::fmax(res, std::fabs(s - lam[c] * u[(size_t)i * n + c]));
          }
          for (int c2 = 0; c2 < n; ++c2) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += u[(size_t)k * n + c] * u[(size_t)k * n + c2];
            orth = std::fmax(orth, std::fabs(s - (c == c2 ? 1.0 : 0.0)));
          }
        }
        out.push_back(res / gn);
        out.push_back(orth);
        out.push_back(order);
      }
    }
  } else if (which == 3) {
    // accumulation bias: positive operands, signed mean of (C_tc - C_64) / C_64
    const size_t ws_elems = (size_t)64 << 20;
    DBuf ws(ws_elems);
    size_t pack_bytes = (size_t)128 << 20;
    void* pack = nullptr;
    if (cudaMalloc(&pack, pack_bytes) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest pack");
    const int Ks[3] = {32, 256, 2048};
    for (int K : Ks) {
      const int M = 256, N = 128;
      DBuf A((size_t)M * K), B((size_t)K * N), C0((size_t)M * N), C1((size_t)M * N);
      fill_gaussian(st, A.p, (size_t)M * K, 1.0, 31 + K, 7);
      fill_gaussian(st, B.p, (size_t)K * N, 1.0, 37 + K, 8);
      std::vector<double> ha = down(A.p, (size_t)M * K), hb = down(B.p, (size_t)K * N);
      for (double& v : ha) v = std::fabs(v);
      for (double& v : hb) v = std::fabs(v);
      cudaMemcpy(A.p, ha.data(), ha.size() * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(B.p, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice);
      MatView av, bv;
      av.p = A.p; av.rs = K; av.cs = 1;
      bv.p = B.p; bv.rs = N; bv.cs = 1;
      OutView c0, c1;
      c0.p = C0.p; c0.rs = N; c0.cs = 1;
      c1 = c0; c1.p = C1.p;
      gemm_f64(st, M, N, K, 1, 1, 1.0, av, bv, 0.0, c0, ws.p, ws_elems);
      const int modes[3] = {TC_TF32X3, TC_BF16X3, TC_BF16X6};
      for (int mode : modes)
        for (int chunk : {0, 1}) {
          if (!gemm_tc(st, mode, M, N, K, 1, 1, 1.0, av, bv, 0.0, c1, pack, pack_bytes, ws.p, ws_elems, err, chunk)) {
            out.push_back(-1.0);
            out.push_back(-1.0);
            continue;
          }
          cudaStreamSynchronize(st);
          std::vector<double> h0 = down(C0.p, (size_t)M * N), h1 = down(C1.p, (size_t)M * N);
          double mean = 0, mx = 0;
          for (size_t i = 0; i < h0.size(); ++i) {
            const double r = (h1[i] - h0[i]) / h0[i];
            mean += r;
            mx = std::fmax(mx, std::fabs(r));
          }
          out.push_back(mean / (double)h0.size());
          out.push_back(mx);
        }
    }
    cudaFree(pack);
  } else if (which == 4) {
    // throughput of the tensor-core GEMM on large square products (the
    // contraction kernel on a shape that fills the GPU), per call including the
    // operand packing: for n in {4096, 8192} and modes (BF16, BF16X3):
    // n, mode, TFLOP/s (2 n^3 per call, mean of 5 timed calls after 2 untimed
    // ones), max relative error of 16 sampled entries against FP64 dot products
    const size_t ws_elems = (size_t)32 << 20;
    DBuf ws(ws_elems);
    for (int n : {4096, 8192}) {
      const size_t sz = (size_t)n * n;  // 8192^2 FP64: 512 MiB per operand
      DBuf A(sz), B(sz), C(sz);
      fill_gaussian(st, A.p, sz, 1.0, 4242 + n, 9);
      fill_gaussian(st, B.p, sz, 1.0, 4343 + n, 10);
      MatView av, bv;
      av.p = A.p; av.rs = n; av.cs = 1;
      bv.p = B.p; bv.rs = n; bv.cs = 1;
      OutView cv;
      cv.p = C.p; cv.rs = n; cv.cs = 1;
      const int modes[2] = {TC_BF16, TC_BF16X3};
      for (int mode : modes) {
        const size_t pack_bytes = tc_workspace_bytes(n, n, n, 1, mode);
        void* pack = nullptr;
        if (cudaMalloc(&pack, pack_bytes) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest pack");
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        bool ok = true;
        for (int it = 0; it < 2 && ok; ++it)
          ok = gemm_tc(st, mode, n, n, n, 1, 1, 1.0, av, bv, 0.0, cv, pack, pack_bytes, ws.p, ws_elems, err);
        float ms = 0.f;
        if (ok) {
          cudaEventRecord(e0, st);
          for (int it = 0; it < 5; ++it)
            gemm_tc(st, mode, n, n, n, 1, 1, 1.0, av, bv, 0.0, cv, pack, pack_bytes, ws.p, ws_elems, err);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) throw std::runtime_error("CUDA error: selftest gemm timing");
          cudaEventElapsedTime(&ms, e0, e1);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(pack);
        double err_max = -1.0;
        if (ok) {  // row i of A, column j of B and C(i, j) only
          err_max = 0.0;
          std::vector<double> ar(n), bc(n);
          for (int q = 0; q < 16; ++q) {
            const size_t i = ((size_t)q * 2654435761u) % n, j = ((size_t)q * 40503u + 7) % n;
            double cij = 0.0;
            if (cudaMemcpy(ar.data(), A.p + i * n, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy2D(bc.data(), 8, B.p + j, (size_t)n * 8, 8, n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(&cij, C.p + i * n + j, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
              throw std::runtime_error("CUDA error: selftest gemm sample");
            double ref = 0.0, mag = 0.0;
            for (int k = 0; k < n; ++k) {
              ref += ar[k] * bc[k];
              mag += std::fabs(ar[k] * bc[k]);
            }
            err_max = std::fmax(err_max, std::fabs(cij - ref) / mag);
          }
        }
        out.push_back((double)n);
        out.push_back((double)mode);
        out.push_back(ok && ms > 0.f ? 2.0 * n * (double)n * n * 5.0 / (ms * 1e-3) / 1e12 : -1.0);
        out.push_back(err_max);
      }
    }
  } else if (which == 5) {
    // tensor-core GEMM operands and results for a check on the host in FP64:
    // per case the header (M, N, K, outer, inner, A transposed, B transposed,
    // beta; alpha is 1.5), the operands A, B and the initial C as stored
    // (batch-major, then row-major or, when transposed, column-major), then C
    // after each mode (BF16X3, TF32, TF32X3, BF16, BF16X6, BF16X10; NaN when a mode
    // does not take the shape)
    struct Case {
      int M, N, K, outer, inner;
      bool ta, tb;
      double beta;
    };
    const Case cases[] = {{272, 136, 2176, 1, 1, false, false, 0.0},
                          {4352, 256, 136, 1, 1, false, false, 0.0},
                          {130, 70, 100, 3, 2, true, false, 0.5},
                          {136, 160, 272, 1, 1, true, true, 1.0}};
    const size_t ws_elems = (size_t)32 << 20;
    DBuf ws(ws_elems);
    size_t pack_bytes = (size_t)256 << 20;
    void* pack = nullptr;
    if (cudaMalloc(&pack, pack_bytes) != cudaSuccess) throw std::runtime_error("ENOMEM: selftest pack");
    unsigned long long seed = 24680;
    for (const Case& c : cases) {
      const long long batch = (long long)c.outer * c.inner;
      const size_t asz = (size_t)c.M * c.K * batch, bsz = (size_t)c.K * c.N * batch, csz = (size_t)c.M * c.N * batch;
      DBuf A(asz), B(bsz), C0(csz), C1(csz);
      fill_gaussian(st, A.p, asz, 1.0, seed++, 1);
      fill_gaussian(st, B.p, bsz, 1.0, seed++, 2);
      fill_gaussian(st, C0.p, csz, 1.0, seed++, 3);
      MatView av, bv;
      av.p = A.p;
      av.rs = c.ta ? 1 : c.K;
      av.cs = c.ta ? c.M : 1;
      av.si = (long long)c.M * c.K;
      av.so = av.si * c.inner;
      bv.p = B.p;
      bv.rs = c.tb ? 1 : c.N;
      bv.cs = c.tb ? c.K : 1;
      bv.si = (long long)c.K * c.N;
      bv.so = bv.si * c.inner;
      OutView cv;
      cv.p = C1.p;
      cv.rs = c.N;
      cv.cs = 1;
      cv.si = (long long)c.M * c.N;
      cv.so = cv.si * c.inner;
      const double hdr[8] = {(double)c.M, (double)c.N, (double)c.K, (double)c.outer, (double)c.inner,
                             c.ta ? 1.0 : 0.0, c.tb ? 1.0 : 0.0, c.beta};
      out.insert(out.end(), hdr, hdr + 8);
      for (const DBuf* d : {&A, &B, &C0}) {
        const std::vector<double> h = down(d->p, d == &A ? asz : d == &B ? bsz : csz);
        out.insert(out.end(), h.begin(), h.end());
      }
      const int tc_mode[6] = {TC_BF16X3, TC_TF32, TC_TF32X3, TC_BF16, TC_BF16X6, TC_BF16X10};
      for (int mode = 0; mode < 6; ++mode) {
        if (cudaMemcpy(C1.p, C0.p, csz * sizeof(double), cudaMemcpyDeviceToDevice) != cudaSuccess)
          throw std::runtime_error("CUDA error: selftest copy");
        if (!gemm_tc(st, tc_mode[mode], c.M, c.N, c.K, c.outer, c.inner, 1.5, av, bv, c.beta, cv, pack, pack_bytes,
                     ws.p, ws_elems, err)) {
          out.insert(out.end(), csz, std::nan(""));
          continue;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("CUDA error: selftest gemm");
        const std::vector<double> h = down(C1.p, csz);
        out.insert(out.end(), h.begin(), h.end());
      }
    }
    cudaFree(pack);
  } else if (which == 6) {
    // FP64 arithmetic throughput of the whole GPU: DFMA (CUDA cores) and
    // mma.sync m8n8k4 f64; per probe TFLOP/s (2 flops per FMA) of the best of
    // three timed launches after one untimed one, then the SM count and the
    // number of blocks launched
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    DBuf sink(1);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int probe = 0; probe < 2; ++probe) {
      float best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (probe == 0)
          dfma_rate_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, sink.p);
        else
          dmma_rate_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, sink.p);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) throw std::runtime_error("CUDA error: FP64 rate probe");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
      }
      const double fma_per_thread =
          probe == 0 ? (double)iters * kChains : (double)iters * 4 * 256.0 / 32.0;  // 256 FMAs per warp-MMA
      const double flops = 2.0 * fma_per_thread * threads * (double)blocks;
      out.push_back(flops / (best * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out.push_back((double)sms);
    out.push_back((double)blocks);
  } else {
    cudaFree(err);
    throw std::runtime_error("EINVAL: unknown selftest");
  }
  int herr[4] = {0, 0, 0, 0};
  cudaMemcpy(herr, err, 16, cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (cudaGetLastError() != cudaSuccess) throw std::runtime_error("CUDA error: selftest launch");
  out.push_back((double)herr[0]);
  return out;
}

}  // namespace qtt
