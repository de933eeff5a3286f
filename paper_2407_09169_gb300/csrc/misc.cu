// Small kernels: identity cores, constant / Gaussian fills, the truncation
// selection, weight environments (conditional means and moments), point
// evaluation, finite checks; the launch counter.
#include <cmath>
#include <cstdlib>

#include <algorithm>

#include "kernels.cuh"

namespace qtt {

static unsigned long long g_launches = 0;
unsigned long long launch_count() { return g_launches; }
void count_launches(int n) { g_launches += (unsigned long long)n; }
// Off unless QTT_PDL=1: measured on the 2^8-point chi = 128 workload, the
// early launch of dependents for every kernel cost 4-5% of the step when it
// was built (12.4 -> 11.7 steps/s for BF16X3) and 10% on later kernels (22.3
// -> 20.0) -- waiting CTAs hold SM slots that the running kernel's later CTAs
// need.  (launch_pdl_chain sets it for one short chain regardless.)
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("QTT_PDL");
    return e && e[0] == '1';
  }();
  return on;
}

namespace {

__global__ void identity_left_kernel(double* core, int r) {
  const long long total = (long long)r * 2 * (2 * r);
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long b = x % (2 * r), as = x / (2 * r);
    const long long s = as % 2, a = as / 2;
    core[x] = (b == 2 * a + s) ? 1.0 : 0.0;
  }
}

__global__ void identity_right_kernel(double* core, int c) {
  const long long total = (long long)(2 * c) * 2 * c;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long b = x % c, as = x / c;
    const long long s = as % 2, a = as / 2;
    core[x] = (a == s * c + b) ? 1.0 : 0.0;
  }
}

__global__ void fill_kernel(double* p, size_t n, double v) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
    p[x] = v;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(double* p, size_t n, double sigma, unsigned long long seed,
                                unsigned long long stream_id) {
  const unsigned long long base = mix64(seed ^ mix64(stream_id + 0x632BE59BD9B4E019ull));
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long h1 = mix64(base + 2 * (unsigned long long)x);
    const unsigned long long h2 = mix64(base + 2 * (unsigned long long)x + 1);
    const double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
    p[x] = sigma * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

// All sketch cores of one stage in one launch: blockIdx.y = site n in [1, N).
__global__ void gaussian_sketch_kernel(Chain om, unsigned long long seed, const unsigned long long* step,
                                       int stage) {
  const int n = blockIdx.y;
  if (n == 0 || n >= om.n) return;
  const int bl = om.bond[n], br = om.bond[n + 1];
  const size_t cnt = (size_t)bl * 2 * br;
  const double sigma = rsqrt(2.0 * (double)br);
  const unsigned long long stream_id = ((*step) * 2ull + (unsigned long long)stage) * (unsigned long long)kMaxSites +
                                       (unsigned long long)n;
  const unsigned long long base = mix64(seed ^ mix64(stream_id + 0x632BE59BD9B4E019ull));
  double* p = const_cast<double*>(om.core[n]);  // the sketch MPS is scratch owned by the engine
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < cnt; x += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long h1 = mix64(base + 2 * (unsigned long long)x);
    const unsigned long long h2 = mix64(base + 2 * (unsigned long long)x + 1);
    const double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
    p[x] = sigma * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

__global__ void bump_kernel(unsigned long long* c) { *c += 1ull; }

// out = sum of up to four arrays (the terms' range products of one site).
struct SumArgs {
  const double* in[4];
  int n_in;
};
__global__ void sum_kernel(double* out, SumArgs a, size_t n) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
    double v = a.in[0][x];
    for (int i = 1; i < a.n_in; ++i) v += a.in[i][x];
    out[x] = v;
  }
}

__global__ void eye_kernel(double* p, int n) {
  pdl_trigger();
  pdl_wait();
  const size_t total = (size_t)n * n;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x)
    p[x] = (x / n == x % n) ? 1.0 : 0.0;
}

__global__ void left_weight_env_kernel(Chain f, Chain w, int nsites, int max_bond, double* out, int ldo,
                                       double* work) {
  double* E = work;                    // [4][max_bond]
  double* X = E + 4 * max_bond;        // [4][2][max_bond]
  double* E2 = X + 8 * max_bond;       // [4][max_bond]
  if (threadIdx.x == 0) E[0] = 1.0;
  __syncthreads();
  for (int n = 0; n < nsites; ++n) {
    const int bl = f.bond[n], br = f.bond[n + 1], ql = w.bond[n], qr = w.bond[n + 1];
    const double* A = f.core[n];
    const double* W = w.core[n];
    for (int x = threadIdx.x; x < ql * 2 * br; x += blockDim.x) {
      const int q = x / (2 * br), sb = x - q * 2 * br;
      // four independent partial sums: four loads of A in flight per thread
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int b = 0;
      for (; b + 3 < bl; b += 4) {
        const double v0 = A[(size_t)b * 2 * br + sb], v1 = A[(size_t)(b + 1) * 2 * br + sb];
        const double v2 = A[(size_t)(b + 2) * 2 * br + sb], v3 = A[(size_t)(b + 3) * 2 * br + sb];
        a0 += E[q * max_bond + b] * v0;
        a1 += E[q * max_bond + b + 1] * v1;
        a2 += E[q * max_bond + b + 2] * v2;
        a3 += E[q * max_bond + b + 3] * v3;
      }
      for (; b < bl; ++b) a0 += E[q * max_bond + b] * A[(size_t)b * 2 * br + sb];
      X[q * 2 * max_bond + sb] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < qr * br; x += blockDim.x) {
      const int q2 = x / br, b2 = x - q2 * br;
      double acc = 0.0;
      for (int q = 0; q < ql; ++q)
        for (int s = 0; s < 2; ++s) acc += W[(q * 2 + s) * qr + q2] * X[q * 2 * max_bond + s * br + b2];
      E2[q2 * max_bond + b2] = acc;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < qr * br; x += blockDim.x) {
      const int q2 = x / br, b2 = x - q2 * br;
      E[q2 * max_bond + b2] = E2[q2 * max_bond + b2];
    }
    __syncthreads();
  }
  const int qn = w.bond[nsites], bn = f.bond[nsites];
  for (int x = threadIdx.x; x < qn * bn; x += blockDim.x) {
    const int q = x / bn, b = x - q * bn;
    out[(size_t)q * ldo + b] = E[q * max_bond + b];
  }
}

// Several weight chains at once, one block per chain (block b takes chain
// wchains[b] and writes out + b * out_stride); the environments live in
// shared memory (16 * max_bond doubles).
__global__ void left_weight_envs_kernel(Chain f, const Chain* __restrict__ wchains, int nsites, int max_bond,
                                        double* out, long long out_stride, int ldo) {
  extern __shared__ double env_smem[];
  double* E = env_smem;          // [4][max_bond]
  double* X = E + 4 * max_bond;  // [4][2][max_bond]
  double* E2 = X + 8 * max_bond; // [4][max_bond]
  const Chain& w = wchains[blockIdx.x];
  if (threadIdx.x == 0) E[0] = 1.0;
  __syncthreads();
  for (int n = 0; n < nsites; ++n) {
    const int bl = f.bond[n], br = f.bond[n + 1], ql = w.bond[n], qr = w.bond[n + 1];
    const double* A = f.core[n];
    const double* W = w.core[n];
    for (int x = threadIdx.x; x < ql * 2 * br; x += blockDim.x) {
      const int q = x / (2 * br), sb = x - q * 2 * br;
      // four independent partial sums: four loads of A in flight per thread
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int b = 0;
      for (; b + 3 < bl; b += 4) {
        const double v0 = A[(size_t)b * 2 * br + sb], v1 = A[(size_t)(b + 1) * 2 * br + sb];
        const double v2 = A[(size_t)(b + 2) * 2 * br + sb], v3 = A[(size_t)(b + 3) * 2 * br + sb];
        a0 += E[q * max_bond + b] * v0;
        a1 += E[q * max_bond + b + 1] * v1;
        a2 += E[q * max_bond + b + 2] * v2;
        a3 += E[q * max_bond + b + 3] * v3;
      }
      for (; b < bl; ++b) a0 += E[q * max_bond + b] * A[(size_t)b * 2 * br + sb];
      X[q * 2 * max_bond + sb] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < qr * br; x += blockDim.x) {
      const int q2 = x / br, b2 = x - q2 * br;
      double acc = 0.0;
      for (int q = 0; q < ql; ++q)
        for (int s = 0; s < 2; ++s) acc += W[(q * 2 + s) * qr + q2] * X[q * 2 * max_bond + s * br + b2];
      E2[q2 * max_bond + b2] = acc;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < qr * br; x += blockDim.x) {
      const int q2 = x / br, b2 = x - q2 * br;
      E[q2 * max_bond + b2] = E2[q2 * max_bond + b2];
    }
    __syncthreads();
  }
  const int qn = w.bond[nsites], bn = f.bond[nsites];
  double* o = out + (long long)blockIdx.x * out_stride;
  for (int x = threadIdx.x; x < qn * bn; x += blockDim.x) {
    const int q = x / bn, b = x - q * bn;
    o[(size_t)q * ldo + b] = E[q * max_bond + b];
  }
}

__global__ void right_ones_env_kernel(Chain f, int n0, int max_bond, double* out, double* work) {
  double* R = work;
  double* R2 = work + max_bond;
  if (threadIdx.x == 0) R[0] = 1.0;
  __syncthreads();
  for (int n = f.n - 1; n >= n0; --n) {
    const int bl = f.bond[n], br = f.bond[n + 1];
    const double* A = f.core[n];
    for (int b = threadIdx.x; b < bl; b += blockDim.x) {
      double acc = 0.0;
      for (int s = 0; s < 2; ++s)
        for (int c = 0; c < br; ++c) acc += A[((size_t)b * 2 + s) * br + c] * R[c];
      R2[b] = acc;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bl; b += blockDim.x) R[b] = R2[b];
    __syncthreads();
  }
  for (int b = threadIdx.x; b < f.bond[n0]; b += blockDim.x) out[b] = R[b];
}

__global__ void eval_points_kernel(Chain f, int npts, const unsigned char* bits, int max_bond, double* out,
                                   double* work) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= npts) return;
  double* v = work + (size_t)warp * 2 * max_bond;
  const unsigned char* b = bits + (size_t)warp * f.n;
  const double val = eval_point_warp(f, [b](int n) { return b[n] != 0; }, v, v + max_bond);
  if (lane == 0) out[warp] = val;
}

__global__ void kron_diag_kernel(Chain om, Chain f, Chain out, const double* hf, int kphi) {
  const int j = blockIdx.y, n = kphi + j;
  const int ol = om.bond[j], orr = om.bond[j + 1];
  const int fl = j == 0 ? 2 : f.bond[n], fr = f.bond[n + 1];
  const double* F = j == 0 ? hf : f.core[n];
  const double* O = om.core[j];
  double* X = const_cast<double*>(out.core[n]);
  const long long R = (long long)orr * fr;
  const long long total = (long long)ol * fl * 2 * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e % R, rest = e / R;
    const int s = (int)(rest & 1);
    const long long r = rest >> 1;
    const long long o = r / fl, h = r - o * fl, o2 = c / fr, h2 = c - o2 * fr;
    X[e] = O[(o * 2 + s) * orr + o2] * F[(h * 2 + s) * fr + h2];
  }
}

__global__ void moment_stage_kernel(const double* m0, const double* m, double* out, const double* u, const double* g,
                                    double gamma, int K1, int K2, int K3, double dt, double a, double b, double c) {
  const long long M1 = 1LL << K1, M2 = 1LL << K2, M3 = 1LL << K3, Mx = M1 * M2 * M3;
  const long long st[3] = {M2 * M3, M3, 1};
  const long long Md[3] = {M1, M2, M3};
  const double two_pi = 6.283185307179586476925286766559;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * Mx; e += (long long)gridDim.x * blockDim.x) {
    const long long sp = e / Mx, x = e - sp * Mx;
    const double* ms = m + sp * Mx;
    const double mc = ms[x];
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const long long j = (x / st[i]) % Md[i];
      const long long xp = x + (((j + 1) % Md[i]) - j) * st[i];
      const long long xm = x + (((j + Md[i] - 1) % Md[i]) - j) * st[i];
      const double h = two_pi / (double)Md[i];
      r -= u[i * Mx + x] * (ms[xp] - ms[xm]) / (2.0 * h);
      if (g) {
        const double gp = 0.5 * (g[x] + g[xp]), gm = 0.5 * (g[xm] + g[x]);
        r += (gp * (ms[xp] - mc) - gm * (mc - ms[xm])) / (h * h);
      } else {
        r += gamma * (ms[xp] - 2.0 * mc + ms[xm]) / (h * h);
      }
    }
    out[e] = a * m0[e] + b * mc + c * dt * r;
  }
}

__global__ void error_sums_kernel(const double* fields, const double* ref, long long Mx, double* acc) {
  double v[5] = {0, 0, 0, 0, 0};
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < Mx; x += (long long)gridDim.x * blockDim.x) {
    const double n = fields[x], m1 = fields[Mx + x], m2 = fields[2 * Mx + x];
    const double d1 = m1 - ref[x], d2 = m2 - ref[Mx + x], dn = n - 1.0;
    v[0] += d1 * d1;
    v[1] += d2 * d2;
    v[2] += dn * dn;
    v[3] += m1;
    v[4] += m2;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, v[k]);
  }
}

__global__ void finite_kernel(const double* p, size_t n, int* flag) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(p[x])) {
      atomicOr(flag, 1);
      return;
    }
}

__global__ void truncate_select_kernel(const EigProblem* probs, double tol, double floor_rel, double* discarded,
                                       int* ranks) {
  const EigProblem P = probs[blockIdx.x];
  __shared__ int s_kk;
  if (threadIdx.x == 0) {
    const double l0 = P.lam[0] > 0.0 ? P.lam[0] : 0.0;
    const double rel = tol * tol > floor_rel ? tol * tol : floor_rel;
    const double thr = rel * l0;
    int kk = 0;
    while (kk < P.k && P.lam[kk] > thr && P.lam[kk] > 0.0) ++kk;
    double dis = 0.0;
    for (int i = kk; i < P.n; ++i) dis += P.lam[i] > 0.0 ? P.lam[i] : 0.0;
    atomicAdd(discarded, dis);
    ranks[blockIdx.x] = kk;
    s_kk = kk;
  }
  __syncthreads();
  const int kk = s_kk;
  const int w = P.k - kk;
  if (w <= 0) return;
  for (int x = threadIdx.x; x < P.n * w; x += blockDim.x) {
    const int i = x / w, c = kk + (x - i * w);
    P.U[(size_t)i * P.k + c] = 0.0;
  }
}

int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 2048) b = 2048;
  return (int)b;
}

}  // namespace

void truncate_select(cudaStream_t st, const EigProblem* probs_dev, int nprob, double tol, double floor_rel,
                     double* discarded, int* ranks) {
  if (nprob <= 0) return;
  count_launches(1);
  truncate_select_kernel<<<nprob, 256, 0, st>>>(probs_dev, tol, floor_rel, discarded, ranks);
}
void fill_identity_left(cudaStream_t st, double* core, int r) {
  count_launches(1);
  identity_left_kernel<<<grid_for((size_t)r * 4 * r), 256, 0, st>>>(core, r);
}
void fill_identity_right(cudaStream_t st, double* core, int c) {
  count_launches(1);
  identity_right_kernel<<<grid_for((size_t)c * 4 * c), 256, 0, st>>>(core, c);
}
void fill_value(cudaStream_t st, double* p, size_t n, double v) {
  if (n) count_launches(1);
  if (n) fill_kernel<<<grid_for(n), 256, 0, st>>>(p, n, v);
}
void fill_gaussian(cudaStream_t st, double* p, size_t n, double sigma, unsigned long long seed,
                   unsigned long long stream_id) {
  if (n) count_launches(1);
  if (n) gaussian_kernel<<<grid_for(n), 256, 0, st>>>(p, n, sigma, seed, stream_id);
}
void fill_gaussian_sketch(cudaStream_t st, const Chain& om, size_t max_core, unsigned long long seed,
                          const unsigned long long* step, int stage) {
  if (om.n <= 1) return;
  count_launches(1);
  size_t bx = (max_core + 255) / 256;
  if (bx > 64) bx = 64;
  gaussian_sketch_kernel<<<dim3((unsigned)bx, (unsigned)om.n), 256, 0, st>>>(om, seed, step, stage);
}
void sum_arrays(cudaStream_t st, double* out, const double* const* in, int n_in, size_t n) {
  if (n == 0 || n_in <= 0) return;
  SumArgs a{};
  for (int i = 0; i < n_in && i < 4; ++i) a.in[i] = in[i];
  a.n_in = n_in < 4 ? n_in : 4;
  count_launches(1);
  sum_kernel<<<grid_for(n), 256, 0, st>>>(out, a, n);
}
void fill_eye(cudaStream_t st, double* p, int n) {
  if (n <= 0) return;
  count_launches(1);
  launch_pdl(eye_kernel, dim3(grid_for((size_t)n * n)), dim3(256), 0, st, p, n);
}
void bump_counter(cudaStream_t st, unsigned long long* c) {
  count_launches(1);
  bump_kernel<<<1, 1, 0, st>>>(c);
}
void left_weight_env(cudaStream_t st, const Chain& f, const Chain& w, int nsites, int max_bond, double* out,
                     int ldo, double* work) {
  count_launches(1);
  left_weight_env_kernel<<<1, 256, 0, st>>>(f, w, nsites, max_bond, out, ldo, work);
}
void left_weight_envs(cudaStream_t st, const Chain& f, const Chain* wchains_dev, int nw, int nsites, int max_bond,
                      double* out, long long out_stride, int ldo) {
  if (nw <= 0) return;
  const size_t smem = (size_t)16 * max_bond * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(left_weight_envs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launches(1);
  left_weight_envs_kernel<<<nw, 256, smem, st>>>(f, wchains_dev, nsites, max_bond, out, out_stride, ldo);
}
void right_ones_env(cudaStream_t st, const Chain& f, int n0, int max_bond, double* out, double* work) {
  count_launches(1);
  right_ones_env_kernel<<<1, 256, 0, st>>>(f, n0, max_bond, out, work);
}
void eval_points(cudaStream_t st, const Chain& f, int npts, const unsigned char* bits, int max_bond, double* out,
                 double* work) {
  if (npts <= 0) return;
  const int warps_per_block = 8;
  count_launches(1);
  eval_points_kernel<<<(npts + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
      f, npts, bits, max_bond, out, work);
}
void kron_diag_cores(cudaStream_t st, const Chain& om, const Chain& f, const Chain& out, const double* hf, int kphi) {
  long long most = 1;
  for (int j = 0; j < om.n; ++j) most = std::max<long long>(most, (long long)out.bond[kphi + j] * 2 * out.bond[kphi + j + 1]);
  const unsigned bx = (unsigned)std::min<long long>(1024, (most + 255) / 256);
  count_launches(1);
  kron_diag_kernel<<<dim3(bx, (unsigned)om.n), 256, 0, st>>>(om, f, out, hf, kphi);
}
void moment_stage(cudaStream_t st, const double* m0, const double* m, double* out, const double* u, const double* g,
                  double gamma, const int K[3], double dt, double a, double b, double c) {
  const long long n = 2LL << (K[0] + K[1] + K[2]);
  count_launches(1);
  moment_stage_kernel<<<grid_for((size_t)n), 256, 0, st>>>(m0, m, out, u, g, gamma, K[0], K[1], K[2], dt, a, b, c);
}
void error_sums(cudaStream_t st, const double* fields, const double* ref, size_t Mx, double* acc) {
  count_launches(1);
  error_sums_kernel<<<grid_for(Mx), 256, 0, st>>>(fields, ref, (long long)Mx, acc);
}
void check_finite(cudaStream_t st, const double* p, size_t n, int* flag) {
  if (n) count_launches(1);
  if (n) finite_kernel<<<grid_for(n), 256, 0, st>>>(p, n, flag);
}

}  // namespace qtt
