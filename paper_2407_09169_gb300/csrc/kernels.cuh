// Device kernels of the QTT Fokker-Planck path (launch wrappers).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace qtt {

constexpr int kMaxSites = 64;

// Number of kernels launched by this library since it was loaded.
unsigned long long launch_count();
void count_launches(int n);

// Programmatic dependent launch (optional).  The step is a long chain of
// small kernels on one stream; with programmatic stream serialisation the
// next kernel can be scheduled, and run its prologue (barrier init, TMEM
// allocation), while the previous one finishes.  Every kernel launched
// through launch_pdl calls pdl_trigger() first and pdl_wait() before its first
// global-memory access (read or write), which returns once the preceding
// kernel has completed and its memory is visible.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Whether launch_pdl sets the attribute (environment QTT_PDL=1 turns it on;
// read once).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
// The same with the attribute always set: for the short chain QR factorisation
// -> Q formation -> Newton-Schulz Gram -> apply, whose kernels occupy few SMs
// each, so that the next one is resident (waiting in pdl_wait) when the
// previous one ends.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_chain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Operand view for the strided batched GEMM: element (i, j) of batch
// (bo, bi) lives at p[bo * so + bi * si + i * rs + j * cs].
struct MatView {
  const double* p = nullptr;
  long long rs = 0, cs = 0, so = 0, si = 0;
};
struct OutView {
  double* p = nullptr;
  long long rs = 0, cs = 0, so = 0, si = 0;
};

// A chain of MPS cores passed by value to kernels: core n is
// [bond[n]][2][bond[n+1]] row-major.
struct Chain {
  const double* core[kMaxSites];
  int bond[kMaxSites + 1];
  int n;
};

#ifdef __CUDACC__
// f at one grid point, evaluated by one warp: the row vector v (length of the
// current bond) is carried through the chain, v <- v A_n[:, s_n, :], with s_n
// the n-th index bit of the point, read by bit(n) (any flag type: bytes or
// 0/1 doubles).  v and v2 are two scratch rows of max_bond doubles owned by
// the warp; every entry read has been written first, so the scratch needs no
// clearing.  Returns the value on every lane.
template <typename BitFn>
__device__ __forceinline__ double eval_point_warp(const Chain& f, BitFn bit, double* v, double* v2) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) v[0] = 1.0;
  __syncwarp();
  for (int n = 0; n < f.n; ++n) {
    const int bl = f.bond[n], br = f.bond[n + 1];
    const int s = bit(n) ? 1 : 0;
    const double* A = f.core[n];
    for (int c = lane; c < br; c += 32) {
      double acc = 0.0;
      for (int b = 0; b < bl; ++b) acc += v[b] * A[((size_t)b * 2 + s) * br + c];
      v2[c] = acc;
    }
    __syncwarp();
    for (int c = lane; c < br; c += 32) v[c] = v2[c];
    __syncwarp();
  }
  return v[0];
}
#endif

// C[b] = alpha * A[b] * B[b] + beta * C[b] for b in [0, outer * inner).
// M x K times K x N.  A split of K accumulates partial products in `ws`
// (reduced in a fixed order, so results are deterministic); ws must hold
// split * outer * inner * M * N doubles or the product runs unsplit.
void gemm_f64(cudaStream_t st, int M, int N, int K, int outer, int inner, double alpha, MatView A,
              MatView B, double beta, OutView C, double* ws, size_t ws_elems);
int gemm_split_k(int M, int N, int K, int batch);
// One product (no batch) on 16 x 16 output tiles, whatever its shape: for
// the small and skinny products of short chains, where a 64 x 64 tile would
// issue mostly masked FP64 work (each k is summed in the same order as by
// gemm_f64, so the results are the same).
void gemm_f64_tiles16(cudaStream_t st, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
                      OutView C);
// C = alpha * sum_k ws[b][k] + beta * C: the fixed-order reduction of split-K partial tiles.
void splitk_reduce(cudaStream_t st, int M, int N, int inner, int splitk, int batch, double alpha, const double* ws,
                   double beta, OutView C);

// Batched GEMM with a small M (<= 32) and K (<= 64) on the CUDA cores, same
// views as gemm_f64; fp32 selects float arithmetic (round to nearest).
bool small_gemm_fits(int M, int N, int K, int outer, int inner);
void small_gemm(cudaStream_t st, bool fp32, int M, int N, int K, int outer, int inner, double alpha, MatView A,
                MatView B, double beta, OutView C);

// Thin Householder QR of an m x n row-major matrix (m >= n): Q (m x n,
// row-major) overwrites Qout.  Computed in float (prec_bits 32) or double;
// work must hold 2 * m * n + n doubles.  *status != 0 on failure.
void qr_thin(cudaStream_t st, int m, int n, const double* A, double* Qout, void* work, int prec_bits,
             int* status);

// Symmetric eigen-decomposition of an n x n row-major matrix G (n <= 1024).
// Eigenvalues descending in lam[0..n); eigenvectors of the leading k in the
// columns of U (n x k, row-major).  Computed in float (Householder
// tridiagonalisation, implicit QL) or double (tridiagonalisation, divide and
// conquer with QL on its leaves); work must hold eig_work_bytes(n, prec_bits)
// bytes.  *status |= 2 when a QL iteration hits its cap.
size_t eig_work_bytes(int n, int prec_bits);  // plus 256 + sizeof(EigProblem) for eig_sym
void eig_sym(cudaStream_t st, int n, int k, const double* G, double* U, double* lam, void* work, int prec_bits,
             int* status);
// Many independent problems in one pass (one block per problem); the
// descriptors live in device memory, nmax / kmax bound every n / k.
struct EigProblem {
  int n = 0, k = 0;
  const double* G = nullptr;
  double* U = nullptr;
  double* lam = nullptr;
  unsigned char* work = nullptr;  // eig_work_bytes(n, prec_bits) bytes
};
void eig_sym_batched(cudaStream_t st, const EigProblem* probs_dev, int nprob, int nmax, int kmax, int prec_bits,
                     int* status);

// Rank selection of the bond truncation, one block per problem: with
// lam (descending, n values) and U (n x k, k = kept columns at most), keep
// kk = min(k, #{lam_i > thr}) columns, thr = max(tol^2, floor_rel) * lam_0,
// zero the columns kk..k-1 of U, add sum_{i >= kk} lam_i to *discarded and
// store kk in ranks[problem].
void truncate_select(cudaStream_t st, const EigProblem* probs_dev, int nprob, double tol, double floor_rel,
                     double* discarded, int* ranks);

// core[a][s][b] = (b == 2a + s): an r x 2 x 2r left identity core.
void fill_identity_left(cudaStream_t st, double* core, int r);
// core[a][s][b] = (a == s * c + b): a 2c x 2 x c right identity core.
void fill_identity_right(cudaStream_t st, double* core, int c);
void fill_value(cudaStream_t st, double* p, size_t n, double v);
// Gaussian N(0, sigma^2) entries from a counter-based generator (splitmix64
// hashing of (seed, stream, index), Box-Muller).
void fill_gaussian(cudaStream_t st, double* p, size_t n, double sigma, unsigned long long seed,
                   unsigned long long stream_id);
// The Gaussian sketch cores of one stage: cores n = 1 .. om.n - 1 (bond
// l_n x 2 x l_{n+1}) with sigma_n = 1 / sqrt(2 l_{n+1}), drawn with the same
// generator from the stream ((*step) * 2 + stage) * kMaxSites + n.  The step
// count is read on the device, so a replayed graph draws fresh cores and a
// restart from a checkpoint (which restores the count) draws the same ones.
void fill_gaussian_sketch(cudaStream_t st, const Chain& om, size_t max_core, unsigned long long seed,
                          const unsigned long long* step, int stage);
// out[x] = in[0][x] + ... + in[n_in - 1][x], n_in <= 4.
void sum_arrays(cudaStream_t st, double* out, const double* const* in, int n_in, size_t n);
// p = the n x n identity (row-major).
void fill_eye(cudaStream_t st, double* p, int n);
// One Newton-Schulz step in FP64 of an almost-orthonormal Q (m x n,
// row-major): out = Q (3 I - Q^T Q) / 2.  G is work space of 8 n n doubles
// (split partial sums of Q^T Q).
void newton_schulz_step(cudaStream_t st, int m, int n, const double* Q, double* G, double* out);
// *c += 1 on the device.
void bump_counter(cudaStream_t st, unsigned long long* c);

// out[q * ldo + b] = contraction of the sites [0, nsites) of the weight
// chain w (bond <= 4) with the MPS chain f, left to right; result indexed by
// the weight's last bond q and f's bond b at position nsites.  One block;
// work holds 16 * max_bond doubles.
void left_weight_env(cudaStream_t st, const Chain& f, const Chain& w, int nsites, int max_bond, double* out,
                     int ldo, double* work);
// The same for nw weight chains (device array wchains_dev[0..nw)) in one
// launch, one block per chain, chain i writing out + i * out_stride;
// environments in shared memory (16 * max_bond doubles, max_bond <= 1600).
void left_weight_envs(cudaStream_t st, const Chain& f, const Chain* wchains_dev, int nw, int nsites, int max_bond,
                      double* out, long long out_stride, int ldo);
// u[b] = sum over the indices of sites [n0, N) of f(..)[b]: right environment
// with the all-ones vector.  One block; work holds 2 * max_bond doubles.
void right_ones_env(cudaStream_t st, const Chain& f, int n0, int max_bond, double* out, double* work);
// Evaluates f at npts multi-indices given as bits[p * N + n] (one warp per
// point); work holds npts * 2 * max_bond doubles.
// Diagonal cores of the mixing term under the subgrid closures: the x cores
// of f (the first one replaced by hf, [2][2][b], the conditional means
// absorbed) times the x cores of the Omega_mix(x) train, site by site as a
// Kronecker product: out_n[(o, h)][s][(o', h')] = Om_j[o][s][o'] F_n[h][s][h']
// with j = n - kphi; out's bonds are the products of the two.
void kron_diag_cores(cudaStream_t st, const Chain& om, const Chain& f, const Chain& out, const double* hf, int kphi);
// One explicit RK2 stage of the first-moment equation Eq. FPMoms (S = 0) on
// the dense x grid (x1 slowest, 2^K per dimension), both species at once:
// out = a m0 + b m + c dt R(m), R(m) = -u . D1 m + div(g grad m) with
// periodic CFD2 differences; g = null: the constant gamma times the compact
// second difference, else the flux form with face values averaged from the
// two neighbours.  m0 is read point-wise only, so out may be m0.
void moment_stage(cudaStream_t st, const double* m0, const double* m, double* out, const double* u, const double* g,
                  double gamma, const int K[3], double dt, double a, double b, double c);
// The space sums of an error sample: acc[0..5) += (M1 - r1)^2, (M2 - r2)^2,
// (N - 1)^2, M1, M2 over the x grid (fields [3][Mx] = <1>, <Phi_1>, <Phi_2>;
// ref [2][Mx]); acc must be zeroed first.
void error_sums(cudaStream_t st, const double* fields, const double* ref, size_t Mx, double* acc);
void eval_points(cudaStream_t st, const Chain& f, int npts, const unsigned char* bits, int max_bond, double* out,
                 double* work);
// flag[0] = 1 if any of the n entries is NaN or infinite.
void check_finite(cudaStream_t st, const double* p, size_t n, int* flag);

}  // namespace qtt
