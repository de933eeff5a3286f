// Device engine of the QTT Fokker-Planck solver.
//
// One explicit RK2 stage (paper: "Finite-difference discretisation" -- RK2
// in time; "Matrix product state algorithm" -- the scheme run on the MPS
// manifold with MPO x MPS products, Hadamard products and SVD truncation)
// computes a sum of terms  g = sum_t c_t Op_t f_t, where Op_t is either
//   * the linear stage operator I + dt W_lin (transport, diffusion, the
//     linear composition drift Omega phi_a + reaction, dissipation), or
//   * the mixing term -dt Omega D1phi_a (<Phi_a>(x) f), an element-wise
//     (Hadamard) product of f with the conditional means, whose x-part cores
//     are f's own x cores with the conditional-mean vectors absorbed into the
//     first one (paper: "Computational complexity" -- the element-wise
//     product is the O(chi^4) operation), or
//   * a multiple of the identity (RK combinations).
// The exact sum has bond dimension ~ chi * (w + chi) on the x sites; it is
// never formed.  Instead:
//   1. a right-to-left sketch pass contracts the terms with a Gaussian
//      random MPS of bond ell = chi + oversample (W_n, right environments);
//   2. a left-to-right pass forms each site tensor T = C * (Op core x f core),
//      orthonormalises the sketch Y = T W_{n+1} by Householder QR, keeps
//      Q as the left-orthonormal core and carries C = Q^T T to the next site
//      (randomized "orthogonalise the sketch" rounding of tensor trains);
//   3. a right-to-left sweep truncates every bond to chi with the SVD,
//      obtained from the FP64 Gram matrix M M^T of the bond matrix and its
//      eigen-decomposition, leaving the state right-canonical.
// Exact mode (no truncation, for parity with the finite-difference oracle):
// step 1 uses identity cores instead of random ones up to the centre of the
// chain, step 2 keeps identity cores (no QR) up to the centre and writes the
// centre core as T W, so the whole stage is a chain of exact contractions.
#include "engine.hpp"
#include "gemm_tc.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>

namespace qtt {

struct KernelTimer {
  bool on = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
    double flops;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[8] = {0}, launches[8] = {0}, flops[8] = {0};
  double pending_flops = 0;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void flush() {
    for (auto& r : recs) {
      float t = 0;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.cls] += t;
        launches[r.cls] += 1;
        flops[r.cls] += r.flops;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  ~KernelTimer() {
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};
enum { TM_GEMM = 0, TM_QR = 1, TM_EIG = 2, TM_OTHER = 3, TM_TC = 4, TM_SMALL = 5 };

struct TimeScope {
  KernelTimer* t;
  int cls;
  cudaStream_t st;
  cudaEvent_t b = nullptr;
  TimeScope(KernelTimer* tm, int c, cudaStream_t s, double flops = 0.0) : t(tm), cls(c), st(s) {
    if (t && t->on) {
      cudaEvent_t a = t->get();
      b = t->get();
      cudaEventRecord(a, st);
      t->recs.push_back({cls, a, b, flops});
    }
  }
  ~TimeScope() {
    if (t && t->on && b) cudaEventRecord(b, st);
  }
};

Chain DevMps::chain() const {
  Chain c;
  std::memset(&c, 0, sizeof(c));
  c.n = N;
  for (int n = 0; n < N; ++n) c.core[n] = core(n);
  for (int n = 0; n <= N; ++n) c.bond[n] = b[n];
  return c;
}

static long long pow2(int e) { return e >= 62 ? (1LL << 62) : (1LL << e); }

static std::atomic<unsigned long long> g_engine_ids{0};

Engine::Engine(const Params& p, cudaStream_t stream) : p_(p), st_(stream) {
  id_ = ++g_engine_ids;
  if (st_ == nullptr) {
    // A stream of our own (blocking, so ordered with the legacy default
    // stream) instead of the legacy stream, which cannot be captured.
    if (cudaStreamCreate(&st_) != cudaSuccess) {
      cudaGetLastError();
      throw std::runtime_error("CUDA error: cudaStreamCreate failed");
    }
    own_stream_ = true;
  }
  N_ = p.N();
  kphi_ = p.Kphi();
  exact_ = p.exact != 0;
  prec_bits_ = (p.precision == 0) ? 64 : 32;
  // contraction arithmetic: FP32 -> 3 x 3 exact bf16 slices (unbiased,
  // ~2^-24 of each row's largest term) for the products that carry the state,
  // hi/lo TF32 (~2^-21 per element) for the sketch products; BF16X3 -> the
  // hi/lo bf16 split everywhere; TF32 -> one TF32 pass.  The sketch
  // W_{n+1} = R_{n+1} G must reproduce the right part R_{n+1} of the
  // operator-state product accurately element by element,
  // because T_n R_{n+1} can be far smaller than |T_n| |R_{n+1}| (the stencils
  // cancel) and an error in R_{n+1} steers the range finder away from
  // T_n R_{n+1}; a bias of the sketch, on the other hand, only rescales it.
  const int mode = p.precision == 1   ? TC_BF16X6
                   : p.precision == 2 ? TC_TF32
                   : p.precision == 3 ? TC_BF16X3
                   : p.precision == 4 ? TC_BF16X10
                                      : -1;
  for (int& m : tc_mode_) m = mode;
  if (p.precision == 1 || p.precision == 4) tc_mode_[GEMM_SKETCH] = tc_mode_[GEMM_RANGE] = TC_TF32X3;
  // BF16X10 takes the mixing term's state products (projection and zip-up of
  // the term kind 1, the Hadamard product with the conditional means) in
  // BF16X6.  The term is dt Omega D1phi[(phi - <Phi>) f], of size
  // ~dt Omega |phi - <Phi>| / sigma ~ 4e-3 |f| on the 2^8-point workload, so
  // its products' error (~2^-24 of their operands' row and column maxima)
  // reaches the state ~250 times smaller, at the level BF16X10 leaves on the
  // other terms.  Measured on that workload against the FP64 path after
  // 25 / 100 / 250 steps: 8.3e-7 / 4.1e-6 / 5.3e-6 (all products in BF16X10:
  // 1.0e-6 / 1.9e-6 / 5.4e-6), 6% shorter steps; TF32X3 there gives
  // 9.4e-6 / 2.6e-5 / 5.0e-5.
  tc_mode_[GEMM_MIX] = p.precision == 4 ? TC_BF16X6 : tc_mode_[GEMM_STATE];
  // BF16X10 keeps the operator-bond contractions (CUDA cores) that carry the
  // state in FP64: in FP32 they move the state by ~1e-5 over ten steps of the
  // 2^4-point workload, far above what its sliced products leave.  Those of
  // the sketch pass run in FP32 (measured on the 2^8-point workload: no loss
  // of accuracy, 4% faster steps).
  small_fp32_ = p.precision >= 1 && p.precision <= 3;
  small_sketch_fp32_ = p.precision >= 1;
  // The reduced forms re-orthonormalise the float QR's Q in FP64 (one
  // Newton-Schulz step).  The float Q's departure from orthonormality
  // (~1e-6) otherwise shows up as a drift of the mass <1>: -8.7e-5 against
  // -2.1e-6 after ten BF16X3 steps of the 2^4-point workload.
  qr_refine_ = (p.precision != 0);
  timer_ = new KernelTimer();
  if (const char* e = std::getenv("QTT_KERNEL_TIMING")) timer_->on = (e[0] == '1');
}

Engine::~Engine() {
  for (cudaGraphExec_t& g : graph_)
    if (g) cudaGraphExecDestroy(g);
  for (cudaGraph_t& g : graph_tmpl_)
    if (g) cudaGraphDestroy(g);
  for (void* a : allocs_) cudaFree(a);
  for (void* w : pack_ws_)
    if (w) cudaFree(w);
  for (int l = 1; l < kLanes; ++l) {
    if (lane_st_[l]) cudaStreamDestroy(lane_st_[l]);
    if (ev_join_[l]) cudaEventDestroy(ev_join_[l]);
  }
  if (ev_fork_) cudaEventDestroy(ev_fork_);
  delete timer_;
  if (own_stream_) cudaStreamDestroy(st_);
}

void* Engine::dalloc(size_t bytes) {
  void* ptr = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("ENOMEM: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  allocs_.push_back(ptr);
  return ptr;
}

void Engine::alloc_mps(DevMps& m, const std::vector<int>& bonds) {
  m.N = (int)bonds.size() - 1;
  m.b = bonds;
  m.off.assign(m.N, 0);
  size_t tot = 0;
  for (int n = 0; n < m.N; ++n) {
    m.off[n] = tot;
    tot += (size_t)bonds[n] * 2 * bonds[n + 1];
  }
  m.total = tot;
  m.data = (double*)dalloc(tot * sizeof(double));
  QTT_CUDA(cudaMemsetAsync(m.data, 0, tot * sizeof(double), st_));
}

void Engine::upload_tt_mps(DevMps& m, const TT& t, const std::vector<int>& bonds) {
  // zero-padded copy of a host train into the static profile
  std::vector<double> h(m.total, 0.0);
  for (int n = 0; n < t.N(); ++n) {
    if (t.r[n] > bonds[n] || t.r[n + 1] > bonds[n + 1])
      throw std::runtime_error("EINVAL: host train exceeds the static bond profile");
    for (int a = 0; a < t.r[n]; ++a)
      for (int s = 0; s < 2; ++s)
        for (int c = 0; c < t.r[n + 1]; ++c)
          h[m.off[n] + ((size_t)a * 2 + s) * bonds[n + 1] + c] = t.at(n, a, s, c);
  }
  QTT_CUDA(cudaMemcpy(m.data, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
}

void Engine::upload_op(DevOp& op, const TT& t) {
  op.N = t.N();
  op.w = t.r;
  op.off_t.assign(op.N, 0);
  op.off_ss.assign(op.N, 0);
  size_t tot = 0;
  for (int n = 0; n < op.N; ++n) {
    const size_t sz = (size_t)t.r[n] * 4 * t.r[n + 1];
    op.off_t[n] = tot;
    tot += sz;
    op.off_ss[n] = tot;
    tot += sz;
  }
  std::vector<double> h(tot, 0.0);
  for (int n = 0; n < op.N; ++n) {
    const int wl = t.r[n], wr = t.r[n + 1];
    for (int w = 0; w < wl; ++w)
      for (int s = 0; s < 2; ++s)
        for (int sp = 0; sp < 2; ++sp)
          for (int w2 = 0; w2 < wr; ++w2) {
            const double v = t.at(n, w, s * 2 + sp, w2);
            h[op.off_t[n] + ((size_t)s * wr + w2) * 2 * wl + w * 2 + sp] = v;
            h[op.off_ss[n] + ((size_t)(s * 2 + sp) * wl + w) * wr + w2] = v;
          }
  }
  op.data = (double*)dalloc(tot * sizeof(double));
  QTT_CUDA(cudaMemcpy(op.data, h.data(), tot * sizeof(double), cudaMemcpyHostToDevice));
}

void Engine::gemm64(int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B, double beta,
                    OutView C) {
  TimeScope ts(timer_, TM_GEMM, cur(), 2.0 * M * (double)N * K * outer * inner);
  gemm_f64(cur(), M, N, K, outer, inner, alpha, A, B, beta, C, lane_ws_[lane_], ws_elems_);
}

void Engine::gemm(int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B, double beta,
                  OutView C, int role) {
  const int mode = tc_mode_[role];
  if (small_gemm_fits(M, N, K, outer, inner)) {
    // operator-bond contractions: memory-bound, on the CUDA cores
    TimeScope ts(timer_, TM_SMALL, cur(), 2.0 * M * (double)N * K * outer * inner);
    small_gemm(cur(), mode >= 0 && (small_fp32_ || (small_sketch_fp32_ && role != GEMM_STATE && role != GEMM_MIX)), M, N, K, outer,
               inner, alpha, A, B, beta, C);
    return;
  }
  if (mode < 0) {
    gemm64(M, N, K, outer, inner, alpha, A, B, beta, C);
    return;
  }
  const size_t need = tc_workspace_bytes(M, N, K, (long long)outer * inner, mode);
  void*& pw = pack_ws_[lane_];
  size_t& pb = pack_bytes_[lane_];
  if (need > pb) {  // grows during the first step only (static shapes)
    QTT_CUDA(cudaStreamSynchronize(cur()));
    if (pw) QTT_CUDA(cudaFree(pw));
    pw = nullptr;
    const size_t bytes = need + need / 4;
    if (cudaMalloc(&pw, bytes) != cudaSuccess) {
      cudaGetLastError();
      pw = nullptr;
      pb = 0;
      throw std::runtime_error("ENOMEM: tensor-core packing workspace");
    }
    pb = bytes;
  }
  const double fl = 2.0 * M * (double)N * K * outer * inner;
  if (timer_->on) {
    static const double passes[6] = {3, 2, 6, 1, 6, 10};  // indexed by TcMode, in bf16-pass units
    tc_issued_flops_ += fl * passes[mode];
  }
  TimeScope ts(timer_, TM_TC, cur(), fl);
  if (!gemm_tc(cur(), mode, M, N, K, outer, inner, alpha, A, B, beta, C, pw, pb, lane_ws_[lane_], ws_elems_,
               status_ + 2))
    throw std::runtime_error("EINVAL: tensor-core GEMM shape outside the supported grid or workspace");
}

void Engine::init() {
  std::string why = validate(p_);
  if (!why.empty()) throw std::runtime_error("EINVAL: " + why);
  if (N_ > kMaxSites) throw std::runtime_error("EINVAL: too many sites");
  model_ = build_model(p_);
  const int N = N_;
  // static bond profiles
  D_.assign(N + 1, 1);
  for (int n = 1; n < N; ++n) D_[n] = (int)std::min<long long>({pow2(n), pow2(N - n), (long long)p_.chi_max});
  ell_.assign(N + 1, 1);
  rz_.assign(N + 1, 1);
  if (exact_) {
    nc_ = N / 2;
    for (int n = nc_ + 1; n <= N; ++n) ell_[n] = (int)pow2(N - n);
    for (int n = 0; n <= N; ++n) rz_[n] = (int)(n <= nc_ ? pow2(n) : pow2(N - n));
  } else {
    nc_ = N - 1;
    const int lmax = p_.chi_max + (p_.oversample > 0 ? p_.oversample : 8);
    for (int n = 1; n <= N; ++n) ell_[n] = (int)std::min<long long>((long long)lmax, pow2(N - n));
    rz_[0] = 1;
    for (int n = 0; n + 1 < N; ++n) rz_[n + 1] = std::min(2 * rz_[n], ell_[n + 1]);
    rz_[N] = 1;
  }
  max_bond_ = 1;
  for (int n = 0; n <= N; ++n) max_bond_ = std::max({max_bond_, D_[n], ell_[n], rz_[n]});

  // state
  TT f0 = tt_round(model_.f0, 1e-14, p_.chi_max);
  alloc_mps(f_, D_);
  alloc_mps(fs_, D_);
  alloc_mps(g_, D_);
  upload_tt_mps(f_, f0, D_);
  if (!exact_) {
    alloc_mps(mid_, rz_);
    std::vector<int> ob(N + 1, 1);
    for (int n = 1; n <= N; ++n) ob[n] = ell_[n];
    alloc_mps(omega_, ob);
  }
  // operators
  upload_op(op_lin_, model_.op_lin);
  upload_op(had_, model_.had_phi);
  {
    TT id;
    id.d = 4;
    id.r.assign(N + 1, 1);
    id.c.assign(N, std::vector<double>{1.0, 0.0, 0.0, 1.0});
    upload_op(ident_, id);
  }
  for (int w = 0; w < 6; ++w) {
    alloc_mps(wphi_[w], model_.wphi[w].r);
    upload_tt_mps(wphi_[w], model_.wphi[w], model_.wphi[w].r);
  }
  sgs_ = p_.sgs == 1;
  if (sgs_) {
    const TT& ox = model_.omega_x;
    alloc_mps(omx_, ox.r);
    upload_tt_mps(omx_, ox, ox.r);
    std::vector<int> hb(N + 1, 1);
    hb[kphi_] = 2;
    for (int n = kphi_ + 1; n < N; ++n) hb[n] = ox.r[n - kphi_] * D_[n];
    alloc_mps(hk_, hb);
  }
  if (p_.moment_ref == 1) {
    const size_t Mx = (size_t)1 << (p_.bits[2] + p_.bits[3] + p_.bits[4]);
    mref_ = (double*)dalloc(2 * Mx * sizeof(double));
    mtmp_ = (double*)dalloc(2 * Mx * sizeof(double));
    ux_ = (double*)dalloc(3 * Mx * sizeof(double));
    errs_ = (double*)dalloc(8 * sizeof(double));
    std::vector<double> h(3 * Mx);
    for (int i = 0; i < 3; ++i) {
      const std::vector<double> ui = tt_dense(model_.u[i]);
      std::copy(ui.begin(), ui.end(), h.begin() + i * Mx);
    }
    QTT_CUDA(cudaMemcpy(ux_, h.data(), 3 * Mx * sizeof(double), cudaMemcpyHostToDevice));
    if (sgs_) {
      const std::vector<double> g = subgrid_fields(p_, model_.u).gamma;
      gx_ = (double*)dalloc(Mx * sizeof(double));
      QTT_CUDA(cudaMemcpy(gx_, g.data(), Mx * sizeof(double), cudaMemcpyHostToDevice));
    }
  }

  // per-slot product bonds: slot 0, 3 identity, slot 1 linear, slot 2 mixing
  auto wslot = [&](int slot, int n) -> size_t {
    if (slot == 1) return (size_t)op_lin_.w[n];
    if (slot == 2) return (size_t)(n <= kphi_ ? had_.w[n] : sgs_ ? hk_.b[n] : D_[n]);
    return 1;
  };
  const int nlo = exact_ ? nc_ + 1 : 1;
  size_t x1 = 1, x2 = 1, pp = 1, yy = 1;
  for (int slot = 0; slot < 4; ++slot) {
    Woff_[slot].assign(N + 1, 0);
    size_t tot = 0;
    for (int n = nlo; n <= N; ++n) {
      Woff_[slot][n] = tot;
      tot += (size_t)wslot(slot, n) * D_[n] * ell_[n];
    }
    Wslot_[slot] = (double*)dalloc(tot * sizeof(double));
    size_t cmax = 1, tmax = 1;
    for (int n = 0; n < N; ++n) {
      const bool zipped = exact_ ? (n <= nc_) : true;
      if (zipped) {
        cmax = std::max(cmax, (size_t)rz_[n] * wslot(slot, n) * D_[n]);
        tmax = std::max(tmax, (size_t)2 * rz_[n] * wslot(slot, n + 1) * D_[n + 1]);
        pp = std::max(pp, (size_t)rz_[n] * wslot(slot, n) * 2 * D_[n + 1]);
      }
      if (n >= nlo) {
        x1 = std::max(x1, (size_t)wslot(slot, n + 1) * D_[n + 1] * 2 * ell_[n]);
        x2 = std::max(x2, (size_t)wslot(slot, n + 1) * 2 * D_[n] * 2 * ell_[n]);
      }
    }
    C_[slot] = (double*)dalloc(std::max(cmax, tmax) * sizeof(double));
    T_[slot] = (double*)dalloc(std::max(cmax, tmax) * sizeof(double));
  }
  for (int n = 0; n < N; ++n) {
    yy = std::max(yy, (size_t)2 * rz_[n] * ell_[n + 1]);
  }
  for (int n = 0; n < N; ++n) {
    x1 = std::max(x1, (size_t)2 * rz_[n] * rz_[n + 1]);
    x2 = std::max(x2, (size_t)D_[n] * 2 * rz_[n + 1]);
  }
  pp_elems_ = pp;
  P_ = (double*)dalloc(pp * sizeof(double));
  X1_ = (double*)dalloc(x1 * sizeof(double));
  X2_ = (double*)dalloc(x2 * sizeof(double));
  Y_ = (double*)dalloc(yy * sizeof(double));
  const size_t rmax = (size_t)max_bond_;
  qrwork_ = (double*)dalloc((2 * (2 * rmax) * rmax + rmax) * sizeof(double));
  gq_ = (double*)dalloc(8 * rmax * rmax * sizeof(double));  // Newton-Schulz partial Grams
  {  // the six weight chains as a device array for the batched environment kernel
    std::vector<Chain> wc(6);
    for (int w = 0; w < 6; ++w) wc[w] = wphi_[w].chain();
    wchains_dev_ = (Chain*)dalloc(6 * sizeof(Chain));
    QTT_CUDA(cudaMemcpy(wchains_dev_, wc.data(), 6 * sizeof(Chain), cudaMemcpyHostToDevice));
  }
  // Split-K partial tiles (FP64): a split product writes splits x M x N
  // doubles, and the outputs of this context's products are a few max_bond^2;
  // 512 max_bond^2 (capped at 8 Mi doubles, the size the chi = 128 chains
  // use) leaves room for the splits the cost model picks, without holding
  // 64 MB per lane in the small contexts of a batch.
  ws_elems_ = std::min<size_t>((size_t)8 << 20, std::max<size_t>((size_t)1 << 18, (size_t)512 * max_bond_ * max_bond_));
  ws_ = (double*)dalloc(ws_elems_ * sizeof(double));
  // lanes for the terms' concurrent work (at most 2 terms in the first stage
  // and 3 (Heun) or 4 (midpoint) in the second)
  lane_st_[0] = st_;
  lane_ws_[0] = ws_;
  lane_x1_[0] = X1_;
  lane_x2_[0] = X2_;
  lane_p_[0] = P_;
  lane_y_[0] = (double*)dalloc(yy * sizeof(double));
  nlanes_ = 1 + (p_.rk_variant == 0 ? 3 : 4);
  if (const char* e = std::getenv("QTT_LANES"))
    if (e[0] == '0') nlanes_ = 1;
  if (nlanes_ > 1) QTT_CUDA(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
  for (int l = 1; l < nlanes_; ++l) {
    QTT_CUDA(cudaStreamCreateWithFlags(&lane_st_[l], cudaStreamNonBlocking));
    QTT_CUDA(cudaEventCreateWithFlags(&ev_join_[l], cudaEventDisableTiming));
    lane_ws_[l] = (double*)dalloc(ws_elems_ * sizeof(double));
    lane_x1_[l] = (double*)dalloc(x1 * sizeof(double));
    lane_x2_[l] = (double*)dalloc(x2 * sizeof(double));
    lane_p_[l] = (double*)dalloc(pp * sizeof(double));
    lane_y_[l] = (double*)dalloc(yy * sizeof(double));
  }
  for (int i = 0; i < 2; ++i) {
    v_[i] = (double*)dalloc((size_t)2 * D_[kphi_] * sizeof(double));
    hf_[i] = (double*)dalloc((size_t)4 * D_[kphi_ + 1] * sizeof(double));
  }
  envw_ = (double*)dalloc((size_t)16 * max_bond_ * sizeof(double) + 64);
  envout_ = (double*)dalloc((size_t)(8 * max_bond_ + (size_t)max_bond_ * max_bond_ + 64) * sizeof(double));
  disc_ = (double*)dalloc(sizeof(double) * 4);
  obsA_ = (double*)dalloc((size_t)2 * max_bond_ * max_bond_ * sizeof(double) + 64);
  obsB_ = (double*)dalloc((size_t)2 * max_bond_ * max_bond_ * sizeof(double) + 64);
  obsX_ = (double*)dalloc((size_t)2 * max_bond_ * max_bond_ * sizeof(double) + 64);
  status_ = (int*)dalloc(sizeof(int) * 4);
  dstep_ = (unsigned long long*)dalloc(sizeof(unsigned long long));
  QTT_CUDA(cudaMemsetAsync(dstep_, 0, sizeof(unsigned long long), st_));
  if (const char* e = std::getenv("QTT_GRAPHS")) graphs_ = (e[0] != '0');
  ranks_ = (int*)dalloc(sizeof(int) * (N + 1));
  // truncation: right Gram per bond, eigenvectors / eigenvalues of the bonds that truncate
  gram_.assign(N + 1, nullptr);
  tU_.assign(N + 1, nullptr);
  trunc_bonds_.clear();
  if (!exact_) {
    for (int n = 1; n <= N; ++n) gram_[n] = (double*)dalloc((size_t)rz_[n] * rz_[n] * sizeof(double));
    std::vector<EigProblem> probs;
    trunc_nmax_ = 1;
    trunc_kmax_ = 0;
    for (int n = 1; n < N; ++n) {
      if (rz_[n] <= D_[n]) continue;  // keeps every direction: identity projector
      EigProblem P;
      P.n = rz_[n];
      P.k = D_[n];
      P.G = gram_[n];
      tU_[n] = (double*)dalloc((size_t)rz_[n] * D_[n] * sizeof(double));
      P.U = tU_[n];
      P.lam = (double*)dalloc((size_t)rz_[n] * sizeof(double));
      P.work = (unsigned char*)dalloc(eig_work_bytes(rz_[n], 64) + 256);
      probs.push_back(P);
      trunc_bonds_.push_back(n);
      trunc_nmax_ = std::max(trunc_nmax_, P.n);
      trunc_kmax_ = std::max(trunc_kmax_, P.k);
    }
    trunc_probs_ = (EigProblem*)dalloc(sizeof(EigProblem) * (probs.size() + 1));
    if (!probs.empty())
      QTT_CUDA(cudaMemcpy(trunc_probs_, probs.data(), sizeof(EigProblem) * probs.size(), cudaMemcpyHostToDevice));
  }
  QTT_CUDA(cudaMemsetAsync(disc_, 0, sizeof(double) * 4, st_));
  QTT_CUDA(cudaMemsetAsync(status_, 0, sizeof(int) * 4, st_));
  if (mref_) {  // the reference starts from the initial <Phi_a>(x)
    const size_t Mx = (size_t)1 << (p_.bits[2] + p_.bits[3] + p_.bits[4]);
    double* tmp3 = (double*)dalloc(3 * Mx * sizeof(double));
    means_dev(tmp3);
    QTT_CUDA(cudaMemcpyAsync(mref_, tmp3 + Mx, 2 * Mx * sizeof(double), cudaMemcpyDeviceToDevice, st_));
  }
  QTT_CUDA(cudaStreamSynchronize(st_));
}

void Engine::moment_ref_step() {
  if (!mref_) return;
  TimeScope ts(timer_, TM_OTHER, st_);
  const int K[3] = {p_.bits[2], p_.bits[3], p_.bits[4]};
  const double dt = p_.dt;
  if (p_.rk_variant == 0) {  // Heun
    moment_stage(st_, mref_, mref_, mtmp_, ux_, gx_, p_.gamma, K, dt, 1.0, 0.0, 1.0);
    moment_stage(st_, mref_, mtmp_, mref_, ux_, gx_, p_.gamma, K, dt, 0.5, 0.5, 0.5);
  } else {  // midpoint
    moment_stage(st_, mref_, mref_, mtmp_, ux_, gx_, p_.gamma, K, dt, 1.0, 0.0, 0.5);
    moment_stage(st_, mref_, mtmp_, mref_, ux_, gx_, p_.gamma, K, dt, 1.0, 0.0, 1.0);
  }
}

void Engine::cond_means(const DevMps& f, double* v) {
  // v[a][b] = h1 h2 sum over phi indices of phi_a f(..)[b] at the phi/x cut (Eq. 2)
  TimeScope ts(timer_, TM_OTHER, st_);
  // both alpha in one launch (weight chains 1 and 2)
  left_weight_envs(st_, f.chain(), wchains_dev_ + 1, 2, kphi_, max_bond_, v, D_[kphi_], D_[kphi_]);
}

void Engine::make_hfirst(const DevMps& f, double* v, double* hf) {
  // first x core of diag(<Phi_a>(x)): hf[a][s][b'] = sum_b v[a][b] A_kphi[b][s][b']
  const int bl = D_[kphi_], br = D_[kphi_ + 1];
  gemm64(2, 2 * br, bl, 1, 1, 1.0, mv(v, bl, 1), mv(f.core(kphi_), 2 * br, 1), 0.0, ov(hf, 2 * br, 1));
}

void Engine::mix_cores(const DevMps& f, const double* hf) {
  if (!sgs_) return;
  TimeScope ts(timer_, TM_OTHER, st_);
  kron_diag_cores(st_, omx_.chain(), f.chain(), hk_.chain(), hf, kphi_);
}

void Engine::sketch_site(const Term& t, int n, const double* Wn1, double* Wn, const double* Om, int Ll, int Lr,
                         int role) {
  const int bl = t.bl(n), br = t.br(n);
  const int wl = t.wl(n), wr = t.wr(n);
  const double* A = t.A(n);
  double* X1 = lane_x1_[lane_];
  double* X2 = lane_x2_[lane_];
  // X1[(w',a')][s][l] = sum_l' W_{n+1}[(w',a')][l'] Om[l][s][l']
  gemm(wr * br, Ll, Lr, 1, 2, 1.0, mv(Wn1, Lr, 1), mv(Om, 1, 2LL * Lr, 0, Lr), 0.0, ov(X1, 2LL * Ll, 1, 0, Ll), role);
  if (!t.diag(n)) {
    // X2[w'][(a,s')][(s,l)] = sum_a' A[(a,s')][a'] X1[(w',a')][(s,l)]
    gemm(2 * bl, 2 * Ll, br, wr, 1, 1.0, mv(A, br, 1), mv(X1, 2LL * Ll, 1, (long long)br * 2 * Ll), 0.0,
         ov(X2, 2LL * Ll, 1, 4LL * bl * Ll), role);
    // W_n[(w,a)][l] = sum_{s,s',w'} W[w][s*2+s'][w'] X2[w'][(a,s')][(s,l)]
    const double* Wss = t.op->Wss(n);
    for (int ss = 0; ss < 4; ++ss) {
      const int s = ss >> 1, sp = ss & 1;
      gemm(wl, Ll, wr, bl, 1, 1.0, mv(Wss + (size_t)ss * wl * wr, wr, 1),
           mv(X2 + (size_t)sp * 2 * Ll + (size_t)s * Ll, 4LL * bl * Ll, 1, 4LL * Ll), ss == 0 ? 0.0 : 1.0,
           ov(Wn, (long long)bl * Ll, 1, Ll), role);
    }
  } else {
    const double* H = t.H(n);
    // X2[a][s][h'][l] = sum_a' A[a][s][a'] X1[(h',a')][s][l]
    gemm(bl, Ll, br, wr, 2, 1.0, mv(A, 2LL * br, 1, 0, br), mv(X1, 2LL * Ll, 1, (long long)br * 2 * Ll, Ll), 0.0,
         ov(X2, 2LL * wr * Ll, 1, Ll, (long long)wr * Ll), role);
    // W_n[(h,a)][l] = sum_s sum_h' H[h][s][h'] X2[a][s][h'][l], one product per s
    // accumulated in FP64 (H is shared by every a).
    for (int s = 0; s < 2; ++s)
      gemm(wl, Ll, wr, bl, 1, 1.0, mv(H + (size_t)s * wr, 2LL * wr, 1), mv(X2 + (size_t)s * wr * Ll, Ll, 1, 2LL * wr * Ll),
           s == 0 ? 0.0 : 1.0, ov(Wn, (long long)bl * Ll, 1, Ll), role);
  }
}

void Engine::fork_lanes(int n) {
  QTT_CUDA(cudaEventRecord(ev_fork_, st_));
  for (int l = 1; l <= n; ++l) QTT_CUDA(cudaStreamWaitEvent(lane_st_[l], ev_fork_, 0));
}

void Engine::join_lanes(int n) {
  for (int l = 1; l <= n; ++l) {
    QTT_CUDA(cudaEventRecord(ev_join_[l], lane_st_[l]));
    QTT_CUDA(cudaStreamWaitEvent(st_, ev_join_[l], 0));
  }
}

void Engine::sketch_pass(Term* terms, int nt, int n_stop, const DevMps& om) {
  // right-to-left sketch of every term; the terms' chains are independent,
  // so each runs on a lane of its own when there are enough lanes
  const bool par = nt > 1 && nt < nlanes_;
  if (par) fork_lanes(nt);
  for (int i = 0; i < nt; ++i) {
    lane_ = par ? 1 + i : 0;
    const Term& t = terms[i];
    double* W = Wslot_[t.slot];
    fill_value(cur(), W + Woff_[t.slot][N_], 1, 1.0);
    for (int n = N_ - 1; n > n_stop; --n)
      sketch_site(t, n, W + Woff_[t.slot][n + 1], W + Woff_[t.slot][n], om.core(n), ell_[n], ell_[n + 1],
                  exact_ ? GEMM_STATE : GEMM_SKETCH);
  }
  lane_ = 0;
  if (par) join_lanes(nt);
}

void Engine::zip_site(const Term& t, int n, int r, const double* C, double* T, double alpha) {
  const int bl = t.bl(n), br = t.br(n);
  const int wl = t.wl(n), wr = t.wr(n);
  const double* A = t.A(n);
  double* P = lane_p_[lane_];
  // P[(rho,w)][(s',a')] = sum_a C[(rho,w)][a] A[a][(s',a')]
  const int role = t.kind == 1 ? GEMM_MIX : GEMM_STATE;
  gemm(r * wl, 2 * br, bl, 1, 1, 1.0, mv(C, bl, 1), mv(A, 2LL * br, 1), 0.0, ov(P, 2LL * br, 1), role);
  if (!t.diag(n)) {
    // T[(rho,s)][(w',a')] = sum_{(w,s')} Wt[s][w'][(w,s')] P[rho][(w,s')][a']
    const double* Wt = t.op->Wt(n);
    gemm(wr, br, 2 * wl, r, 2, alpha, mv(Wt, 2LL * wl, 1, 0, (long long)wr * 2 * wl),
         mv(P, br, 1, 2LL * wl * br, 0), 0.0, ov(T, br, 1, 2LL * wr * br, (long long)wr * br), role);
  } else {
    const double* H = t.H(n);
    // T[(rho,s)][(h',a')] = sum_h H[h][s][h'] P[(rho,h)][(s,a')]
    gemm(wr, br, wl, r, 2, alpha, mv(H, 1, 2LL * wr, 0, wr), mv(P, 2LL * br, 1, (long long)wl * 2 * br, br), 0.0,
         ov(T, br, 1, 2LL * wr * br, (long long)wr * br), role);
  }
}

Term Engine::term_dense(int slot, const DevOp* op, const DevMps* f, double scale) const {
  Term t;
  t.f = f;
  t.kind = 0;
  t.op = op;
  t.kphi = kphi_;
  t.slot = slot;
  t.scale = scale;
  return t;
}

Term Engine::term_mix(const DevMps* f, const double* hf, double scale) const {
  Term t;
  t.f = f;
  t.kind = 1;
  t.op = &had_;
  t.hfirst = hf;
  if (sgs_) {  // diag(Omega_mix(x) <Phi_a>(x)): the Kronecker cores built by mix_cores
    t.hsrc = &hk_;
    t.hfirst = hk_.core(kphi_);
  }
  t.kphi = kphi_;
  t.slot = 2;
  t.scale = scale;
  return t;
}

void Engine::run_stage(Term* terms, int nt, DevMps& out, int stage) {
  if (exact_) {
    run_stage_exact(terms, nt, out);
    return;
  }
  const int N = N_;
  {
    TimeScope ts(timer_, TM_OTHER, st_);
    fill_gaussian_sketch(st_, omega_.chain(), omega_.max_core_elems(), p_.seed, dstep_, stage);
  }
  // 1. right-to-left sketch: W_n = (right part of the term) x (right part of the random MPS)
  sketch_pass(terms, nt, 0, omega_);
  // 2. left-to-right orthogonalisation of the sketched site tensors.  The
  // terms' site tensors T_i (and, after the QR, C_i = Q^T T_i together with
  // the next site's T_i) are independent, so each term runs on a lane of its
  // own between the Y = sum_i T_i W_i / QR steps on st_.
  const bool par = nt > 1 && nt < nlanes_;
  for (int i = 0; i < nt; ++i) fill_value(st_, C_[terms[i].slot], 1, 1.0);
  // zip_all(n): each term's site tensor T_i at site n (after C_i = Q^T T_i of
  // site n-1 when `project`), and, when site n truncates, its range product
  // Y_i = T_i W_i; the Y_i are summed on st_ after the join.
  auto zip_all = [&](int n, int r, bool project, int rn) {
    const int rs = project ? rn : r;  // bond entering site n
    const bool range = n + 1 < N && rz_[n + 1] != 2 * rs;
    if (par) fork_lanes(nt);
    for (int i = 0; i < nt; ++i) {
      lane_ = par ? 1 + i : 0;
      const Term& t = terms[i];
      if (project)  // C_i = Q^T T_i at the previous site
        gemm(rn, (int)t.B(n), 2 * r, 1, 1, 1.0, mv(mid_.core(n - 1), 1, rn), mv(T_[t.slot], t.B(n), 1), 0.0,
             ov(C_[t.slot], t.B(n), 1), t.kind == 1 ? GEMM_MIX : GEMM_STATE);
      zip_site(t, n, rs, C_[t.slot], T_[t.slot], n == 0 ? t.scale : 1.0);
      if (range) {
        const int L = ell_[n + 1];
        gemm(2 * rs, L, (int)t.B(n + 1), 1, 1, 1.0, mv(T_[t.slot], t.B(n + 1), 1),
             mv(Wslot_[t.slot] + Woff_[t.slot][n + 1], L, 1), par || i == 0 ? 0.0 : 1.0,
             ov(par ? lane_y_[1 + i] : Y_, L, 1), GEMM_RANGE);
      }
    }
    lane_ = 0;
    if (par) join_lanes(nt);
    if (range && par) {
      const double* ys[4] = {lane_y_[1], lane_y_[2], lane_y_[3], lane_y_[4]};
      TimeScope ts(timer_, TM_OTHER, st_);
      sum_arrays(st_, Y_, ys, nt, (size_t)2 * rs * ell_[n + 1]);
    }
  };
  int r = 1;
  zip_all(0, 1, false, 0);
  for (int n = 0; n < N; ++n) {
    if (n == N - 1) {  // all terms close with bond 1: the last core is their sum
      for (int i = 0; i < nt; ++i) {
        const Term& t = terms[i];
        gemm(2 * r, 1, (int)t.B(N), 1, 1, 1.0, mv(T_[t.slot], t.B(N), 1), mv(Wslot_[t.slot] + Woff_[t.slot][N], 1, 1),
             i == 0 ? 0.0 : 1.0, ov(mid_.core(n), 1, 1));
      }
      break;
    }
    const int rn = rz_[n + 1];
    if (rn == 2 * r) {  // bond still below the sketch size: keep everything
      {
        TimeScope ts(timer_, TM_OTHER, st_);
        fill_identity_left(st_, mid_.core(n), r);
      }
      for (int i = 0; i < nt; ++i) std::swap(C_[terms[i].slot], T_[terms[i].slot]);
      zip_all(n + 1, rn, false, 0);
    } else {
      // Y = sum_i T_i W_i is in Y_ (zip_all)
      {
        TimeScope ts(timer_, TM_QR, st_);
        qr_thin(st_, 2 * r, rn, Y_, qr_refine_ ? X1_ : mid_.core(n), qrwork_, prec_bits_, status_);
      }
      if (qr_refine_) {
        // one Newton-Schulz step in FP64, Q <- Q (3 I - Q^T Q) / 2: the span of
        // the float Q, orthonormal to double round-off
        TimeScope ts(timer_, TM_GEMM, st_, 4.0 * (2.0 * r) * rn * rn);
        newton_schulz_step(st_, 2 * r, rn, X1_, gq_, mid_.core(n));
      }
      if (n + 1 < N) zip_all(n + 1, r, true, rn);
    }
    r = rn;
  }
  // 3. SVD truncation of every bond to chi.  The state is left-orthonormal,
  // so the squared singular values at bond n are the eigenvalues of the
  // Gram matrix R_n of its right part.  All R_n come from one right-to-left
  // FP64 contraction pass; all bond eigensolves run in one batched pass;
  // the projectors U_n U_n^T are then inserted into every core independently.
  gram_pass(mid_);
  if (!trunc_bonds_.empty()) {
    {
      TimeScope ts(timer_, TM_EIG, st_);
      eig_sym_batched(st_, trunc_probs_, (int)trunc_bonds_.size(), trunc_nmax_, trunc_kmax_, 64, status_);
    }
    TimeScope ts(timer_, TM_OTHER, st_);
    truncate_select(st_, trunc_probs_, (int)trunc_bonds_.size(), p_.svd_rel_tol, 1e-24, disc_, ranks_);
  }
  project_cores(mid_, out);
}

void Engine::gram_pass(const DevMps& g) {
  // R_N = [1]; R_n = sum_s A_n[:, s, :] R_{n+1} A_n[:, s, :]^T  (FP64)
  fill_value(st_, gram_[N_], 1, 1.0);
  for (int n = N_ - 1; n >= 1; --n) {
    const int rl = g.b[n], rr = g.b[n + 1];
    gemm64(2 * rl, rr, rr, 1, 1, 1.0, mv(g.core(n), rr, 1), mv(gram_[n + 1], rr, 1), 0.0, ov(X1_, rr, 1));
    gemm64(rl, rl, 2 * rr, 1, 1, 1.0, mv(X1_, 2LL * rr, 1), mv(g.core(n), 1, 2LL * rr), 0.0, ov(gram_[n], rl, 1));
  }
}

void Engine::project_cores(const DevMps& g, DevMps& out) {
  // out core n = U_n^T A_n U_{n+1}, with U = identity on bonds that keep all
  // directions.  The cores are independent: they are spread over the main
  // stream and the lanes (each with its own scratch), then joined.
  const int nl = nlanes_;
  if (nl > 1) fork_lanes(nl - 1);
  for (int n = 0; n < N_; ++n) {
    lane_ = n % nl;
    double* scratch = lane_x2_[lane_];
    const int rl = g.b[n], rr = g.b[n + 1], Dl = out.b[n], Dr = out.b[n + 1];
    const double* U_l = tU_[n];
    const double* U_r = tU_[n + 1];
    const double* X = g.core(n);
    if (U_l) {  // X = U_l^T A_n : [Dl x 2 rr]
      gemm(Dl, 2 * rr, rl, 1, 1, 1.0, mv(U_l, 1, Dl), mv(g.core(n), 2LL * rr, 1), 0.0, ov(scratch, 2LL * rr, 1));
      X = scratch;
    }
    if (U_r) {  // out = X U_r : [(2 Dl) x Dr]
      gemm(2 * Dl, Dr, rr, 1, 1, 1.0, mv(X, rr, 1), mv(U_r, Dr, 1), 0.0, ov(out.core(n), Dr, 1));
    } else {
      QTT_CUDA(cudaMemcpyAsync(out.core(n), X, sizeof(double) * (size_t)Dl * 2 * Dr, cudaMemcpyDeviceToDevice, cur()));
    }
  }
  lane_ = 0;
  if (nl > 1) join_lanes(nl - 1);
}

void Engine::run_stage_exact(Term* terms, int nt, DevMps& out) {
  const int N = N_, nc = nc_;
  {
    TimeScope ts(timer_, TM_OTHER, st_);
    for (int n = nc + 1; n < N; ++n) fill_identity_right(st_, out.core(n), ell_[n + 1]);
  }
  sketch_pass(terms, nt, nc, out);
  for (int i = 0; i < nt; ++i) fill_value(st_, C_[terms[i].slot], 1, 1.0);
  int r = 1;
  for (int n = 0; n <= nc; ++n) {
    for (int i = 0; i < nt; ++i)
      zip_site(terms[i], n, r, C_[terms[i].slot], T_[terms[i].slot], n == 0 ? terms[i].scale : 1.0);
    if (n == nc) {
      const int L = ell_[nc + 1];
      for (int i = 0; i < nt; ++i) {
        const Term& t = terms[i];
        gemm(2 * r, L, (int)t.B(n + 1), 1, 1, 1.0, mv(T_[t.slot], t.B(n + 1), 1),
             mv(Wslot_[t.slot] + Woff_[t.slot][n + 1], L, 1), i == 0 ? 0.0 : 1.0, ov(out.core(n), L, 1));
      }
      break;
    }
    {
      TimeScope ts(timer_, TM_OTHER, st_);
      fill_identity_left(st_, out.core(n), r);
    }
    for (int i = 0; i < nt; ++i) std::swap(C_[terms[i].slot], T_[terms[i].slot]);
    r *= 2;
  }
}

void Engine::step_body() {
  QTT_CUDA(cudaMemsetAsync(disc_, 0, sizeof(double), st_));
  if (p_.rk_variant == 0) {
    // Heun: f* = f + dt L(f);  f_{n+1} = (f + f* + dt L(f*)) / 2
    cond_means(f_, v_[0]);
    make_hfirst(f_, v_[0], hf_[0]);
    mix_cores(f_, hf_[0]);
    Term a[2] = {term_dense(1, &op_lin_, &f_, 1.0), term_mix(&f_, hf_[0], 1.0)};
    run_stage(a, 2, fs_, 0);
    cond_means(fs_, v_[1]);
    make_hfirst(fs_, v_[1], hf_[1]);
    mix_cores(fs_, hf_[1]);
    Term b[3] = {term_dense(0, &ident_, &f_, 0.5), term_dense(1, &op_lin_, &fs_, 0.5), term_mix(&fs_, hf_[1], 0.5)};
    run_stage(b, 3, g_, 1);
  } else {
    // midpoint: f_h = f + dt/2 L(f);  f_{n+1} = f + dt L(f_h)
    cond_means(f_, v_[0]);
    make_hfirst(f_, v_[0], hf_[0]);
    mix_cores(f_, hf_[0]);
    Term a[3] = {term_dense(0, &ident_, &f_, 0.5), term_dense(1, &op_lin_, &f_, 0.5), term_mix(&f_, hf_[0], 0.5)};
    run_stage(a, 3, fs_, 0);
    cond_means(fs_, v_[1]);
    make_hfirst(fs_, v_[1], hf_[1]);
    mix_cores(fs_, hf_[1]);
    Term b[4] = {term_dense(0, &ident_, &f_, 1.0), term_dense(1, &op_lin_, &fs_, 1.0),
                 term_dense(3, &ident_, &fs_, -1.0), term_mix(&fs_, hf_[1], 1.0)};
    run_stage(b, 4, g_, 1);
  }
  moment_ref_step();
  bump_counter(st_, dstep_);
}

bool Engine::capture_step(int parity) {
  // Any failure leaves the stream out of capture, clears the error and turns
  // the graphs off for this context: the step then runs eagerly.
  auto give_up = [&](cudaGraph_t g) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t g2 = nullptr;
      cudaStreamEndCapture(st_, &g2);
      if (g2) cudaGraphDestroy(g2);
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    graph_[parity] = nullptr;
    graphs_ = false;
    return false;
  };
  if (cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return give_up(nullptr);
  try {
    step_body();
  } catch (...) {
    give_up(nullptr);
    throw;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(st_, &g) != cudaSuccess || g == nullptr) return give_up(g);
  if (cudaGraphInstantiate(&graph_[parity], g, 0) != cudaSuccess) return give_up(g);
  if (graph_tmpl_[parity]) cudaGraphDestroy(graph_tmpl_[parity]);
  graph_tmpl_[parity] = g;  // kept for embedding into a batch graph
  ++graph_gen_;
  return true;
}

void Engine::drop_graphs() {
  for (int q = 0; q < 2; ++q) {
    if (graph_[q]) {
      QTT_CUDA(cudaGraphExecDestroy(graph_[q]));
      graph_[q] = nullptr;
    }
    if (graph_tmpl_[q]) {
      cudaGraphDestroy(graph_tmpl_[q]);
      graph_tmpl_[q] = nullptr;
    }
  }
  ++graph_gen_;
}

bool Engine::step_graphs_ready() const {
  return graphs_ && warm_ && !timer_->on && graph_[0] && graph_[1] && graph_tmpl_[0] && graph_tmpl_[1];
}

void Engine::step_launched_externally() {
  count_launches(graph_launches_[parity_]);
  std::swap(f_, g_);
  parity_ ^= 1;
  time_ += p_.dt;
  ++steps_;
}

void Engine::step(int nsteps) {
  for (int k = 0; k < nsteps; ++k) {
    // The step's launches (shapes, pointers, workspaces) are identical from
    // step to step once the first one has sized the workspaces, so later
    // steps replay a captured graph; kernel timing needs the eager path.
    bool replay = false;
    if (graphs_ && warm_ && !timer_->on) {
      // the launch counter counts a graph's kernels once at capture and again at every later replay
      if (graph_[parity_]) {
        count_launches(graph_launches_[parity_]);
        replay = true;
      } else {
        const unsigned long long c0 = launch_count();
        replay = capture_step(parity_);
        const int captured = (int)(launch_count() - c0);
        if (replay) graph_launches_[parity_] = captured;
        else count_launches(-captured);  // nothing ran; the eager step below counts its own
      }
    }
    if (replay) {
      QTT_CUDA(cudaGraphLaunch(graph_[parity_], st_));
    } else {
      step_body();
      warm_ = true;
    }
    std::swap(f_, g_);
    parity_ ^= 1;
    time_ += p_.dt;
    ++steps_;
  }
  QTT_CUDA(cudaGetLastError());
  if (timer_->on) {
    QTT_CUDA(cudaStreamSynchronize(st_));
    timer_->flush();
  }
}

int Engine::check_status(std::string& msg) {
  check_finite(st_, f_.data, f_.total, status_ + 1);
  int h[3] = {0, 0, 0};
  double dis = 0;
  QTT_CUDA(cudaMemcpyAsync(h, status_, sizeof(h), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaMemcpyAsync(&dis, disc_, sizeof(double), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  QTT_CUDA(cudaGetLastError());
  discarded_last_ = dis;
  if (h[2]) {
    msg = "a tensor-core GEMM gave up waiting on a pipeline barrier (code " + std::to_string(h[2]) + ")";
    QTT_CUDA(cudaMemsetAsync(status_ + 2, 0, sizeof(int), st_));
    return 5;  // QTT_ETIMEOUT
  }
  if (h[1]) {
    msg = "non-finite value in the state after step " + std::to_string(steps_);
    return 6;  // QTT_ENAN
  }
  if (h[0] & (4 | 8)) {
    msg = (h[0] & 8) ? "eigensolver: the two QL lanes gave up waiting on each other"
                     : "QR: a warp gave up waiting on a reflector";
    QTT_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), st_));
    return 5;  // QTT_ETIMEOUT
  }
  if (h[0] & 2) {
    msg = "a QL iteration of the eigen-decomposition hit its sweep cap";
    QTT_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), st_));
    return 4;  // QTT_ENOCONV
  }
  if (h[0]) {
    msg = "QR / eigensolver reported an invalid factorisation";
    QTT_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), st_));
    return 4;
  }
  return 0;
}

void Engine::xgram(const DevMps& f, double* E) {
  // E[b][b'] = sum over the x indices of F(x)[b] F(x)[b'] at the phi/x cut
  fill_value(st_, obsA_, 1, 1.0);
  double* cur = obsA_;
  double* nxt = obsB_;
  for (int n = N_ - 1; n >= kphi_; --n) {
    const int bl = f.b[n], br = f.b[n + 1];
    gemm64(2 * bl, br, br, 1, 1, 1.0, mv(f.core(n), br, 1), mv(cur, br, 1), 0.0, ov(obsX_, br, 1));
    gemm64(bl, bl, 2 * br, 1, 1, 1.0, mv(obsX_, 2LL * br, 1), mv(f.core(n), 1, 2LL * br), 0.0, ov(nxt, bl, 1));
    std::swap(cur, nxt);
  }
  QTT_CUDA(cudaMemcpyAsync(E, cur, sizeof(double) * f.b[kphi_] * f.b[kphi_], cudaMemcpyDeviceToDevice, st_));
}

void Engine::scalars(double out[13]) {
  const int b = D_[kphi_];
  double* V = envout_;              // 6 x b weight environments
  double* u = V + 6 * (size_t)b;    // b
  double* E = u + b;                // b x b
  double* res = E + (size_t)b * b;  // 6 + b + 1
  const Chain fc = f_.chain();
  left_weight_envs(st_, fc, wchains_dev_, 6, kphi_, max_bond_, V, b, b);
  right_ones_env(st_, fc, kphi_, max_bond_, u, envw_);
  xgram(f_, E);
  // |f|^2 = sum_bb' G[b][b'] E[b][b'], G the Gram of the phi part (left to right)
  {
    fill_value(st_, obsA_, 1, 1.0);
    double* G = obsA_;
    double* Gn = obsB_;
    for (int n = 0; n < kphi_; ++n) {
      const int bl = f_.b[n], br = f_.b[n + 1];
      gemm64(bl, 2 * br, bl, 1, 1, 1.0, mv(G, bl, 1), mv(f_.core(n), 2LL * br, 1), 0.0, ov(obsX_, 2LL * br, 1));
      gemm64(br, br, 2 * bl, 1, 1, 1.0, mv(f_.core(n), 1, br), mv(obsX_, br, 1), 0.0, ov(Gn, br, 1));
      std::swap(G, Gn);
    }
    gemm64(1, 1, b * b, 1, 1, 1.0, mv(G, (long long)b * b, 1), mv(E, 1, 1), 0.0, ov(obsX_, 1, 1));
  }
  double n2 = 0.0;
  QTT_CUDA(cudaMemcpyAsync(&n2, obsX_, sizeof(double), cudaMemcpyDeviceToHost, st_));
  gemm64(6, 1, b, 1, 1, 1.0, mv(V, b, 1), mv(u, 1, 1), 0.0, ov(res, 1, 1));                 // <w> sums
  gemm64(1, b, b, 1, 1, 1.0, mv(V + b, b, 1), mv(E, b, 1), 0.0, ov(res + 6, b, 1));           // v1^T E
  gemm64(1, 1, b, 1, 1, 1.0, mv(res + 6, b, 1), mv(V + 2 * (size_t)b, 1, 1), 0.0, ov(res + 6 + b, 1, 1));
  double h[6];
  double m12 = 0;
  QTT_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaMemcpyAsync(&m12, res + 6 + b, sizeof(double), cudaMemcpyDeviceToHost, st_));
  std::string msg;
  check_status(msg);
  const double Mx = std::ldexp(1.0, p_.bits[2] + p_.bits[3] + p_.bits[4]);
  for (double& x : h) x /= Mx;
  m12 /= Mx;
  out[0] = time_;
  out[1] = h[0];
  out[2] = h[1];
  out[3] = h[2];
  out[4] = h[3];
  out[5] = h[4];
  out[6] = h[5];
  out[7] = m12 - h[1] * h[2];  // R12
  out[8] = h[5] - m12;         // Y12
  out[9] = h[0] - h[1] - h[2];  // mean of <1 - phi1 - phi2>
  out[10] = discarded_last_;
  out[11] = (double)steps_;
  out[12] = n2;  // sum of f^2 over every grid cell
}

void Engine::chain_dense(const DevMps& f, int n0, const double* head, int head_rows, double* out) {
  size_t rows = head_rows;
  for (int n = n0; n < N_; ++n) rows *= 2;
  double* d = nullptr;
  QTT_CUDA(cudaMalloc(&d, sizeof(double) * rows));
  try {
    chain_dense_dev(f, n0, head, head_rows, d);
    QTT_CUDA(cudaMemcpyAsync(out, d, sizeof(double) * rows, cudaMemcpyDeviceToHost, st_));
    QTT_CUDA(cudaStreamSynchronize(st_));
  } catch (...) {
    cudaFree(d);
    throw;
  }
  cudaFree(d);
}

void Engine::chain_dense_dev(const DevMps& f, int n0, const double* head, int head_rows, double* dout) {
  // rows = multi-index of the processed sites, columns = open bond; out gets head_rows * 2^(N - n0) values
  size_t rows = head_rows;
  for (int n = n0; n < N_; ++n) rows *= 2;
  double* a = nullptr;
  double* b = nullptr;
  QTT_CUDA(cudaMalloc(&a, sizeof(double) * (rows * 1 + 16) * 2));
  QTT_CUDA(cudaMalloc(&b, sizeof(double) * (rows * 1 + 16) * 2));
  // buffer bound: rows_so_far * bond <= head_rows * 2^(N-n0) when bonds follow the structural profile
  size_t R = head_rows;
  int bond = f.b[n0];
  QTT_CUDA(cudaMemcpyAsync(a, head, sizeof(double) * R * bond, cudaMemcpyDeviceToDevice, st_));
  for (int n = n0; n < N_; ++n) {
    const int br = f.b[n + 1];
    gemm64((int)R, 2 * br, bond, 1, 1, 1.0, mv(a, bond, 1), mv(f.core(n), 2LL * br, 1), 0.0, ov(b, 2LL * br, 1));
    std::swap(a, b);
    R *= 2;
    bond = br;
  }
  QTT_CUDA(cudaGetLastError());
  QTT_CUDA(cudaMemcpyAsync(dout, a, sizeof(double) * R, cudaMemcpyDeviceToDevice, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  cudaFree(a);
  cudaFree(b);
}

void Engine::dense(double* out) {
  fill_value(st_, obsA_, 1, 1.0);
  chain_dense(f_, 0, obsA_, 1, out);
}

void Engine::means_dev(double* dout) {
  const int b = D_[kphi_];
  const size_t Mx = (size_t)1 << (p_.bits[2] + p_.bits[3] + p_.bits[4]);
  const Chain fc = f_.chain();
  for (int w = 0; w < 3; ++w) {
    left_weight_env(st_, fc, wphi_[w].chain(), kphi_, max_bond_, envout_, b, envw_);
    chain_dense_dev(f_, kphi_, envout_, 1, dout + w * Mx);
  }
}

void Engine::error_sample(double* out) {
  if (!mref_) throw std::runtime_error("EINVAL: the error measures need moment_ref = 1");
  const size_t Mx = (size_t)1 << (p_.bits[2] + p_.bits[3] + p_.bits[4]);
  double* fields = nullptr;
  QTT_CUDA(cudaMalloc(&fields, 3 * Mx * sizeof(double)));
  double acc[5] = {0, 0, 0, 0, 0};
  try {
    means_dev(fields);
    QTT_CUDA(cudaMemsetAsync(errs_, 0, 5 * sizeof(double), st_));
    error_sums(st_, fields, mref_, Mx, errs_);
    QTT_CUDA(cudaGetLastError());
    QTT_CUDA(cudaMemcpyAsync(acc, errs_, sizeof(acc), cudaMemcpyDeviceToHost, st_));
    QTT_CUDA(cudaStreamSynchronize(st_));
  } catch (...) {
    cudaFree(fields);
    throw;
  }
  cudaFree(fields);
  const double n = (double)Mx, a1 = acc[3] / n, a2 = acc[4] / n;
  out[0] = a1 - 0.5;
  out[1] = a2 - 0.5;
  out[2] = acc[0] / n;
  out[3] = acc[1] / n;
  out[4] = a1 - a2;
  out[5] = acc[2] / n;
}

void Engine::means(double* out) {
  const int b = D_[kphi_];
  const size_t Mx = (size_t)1 << (p_.bits[2] + p_.bits[3] + p_.bits[4]);
  const Chain fc = f_.chain();
  for (int w = 0; w < 3; ++w) {
    left_weight_env(st_, fc, wphi_[w].chain(), kphi_, max_bond_, envout_, b, envw_);
    chain_dense(f_, kphi_, envout_, 1, out + w * Mx);
  }
}

void Engine::points(const std::vector<unsigned char>& bits, int npts, double* out) {
  unsigned char* db = nullptr;
  double *dout = nullptr, *work = nullptr;
  QTT_CUDA(cudaMalloc(&db, bits.size() + 1));
  QTT_CUDA(cudaMalloc(&dout, sizeof(double) * npts));
  QTT_CUDA(cudaMalloc(&work, sizeof(double) * (size_t)npts * 2 * max_bond_));
  QTT_CUDA(cudaMemcpyAsync(db, bits.data(), bits.size(), cudaMemcpyHostToDevice, st_));
  eval_points(st_, f_.chain(), npts, db, max_bond_, dout, work);
  QTT_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * npts, cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  cudaFree(db);
  cudaFree(dout);
  cudaFree(work);
}

double Engine::overlap(const Engine& o) {
  // <this|o> by left environments: E_{n+1} = sum_s A_s^T E_n B_s
  if (o.N_ != N_) throw std::runtime_error("EINVAL: states have different numbers of sites");
  for (int d = 0; d < 5; ++d)
    if (o.p_.bits[d] != p_.bits[d]) throw std::runtime_error("EINVAL: states live on different grids");
  QTT_CUDA(cudaStreamSynchronize(o.st_));
  const DevMps& A = f_;
  const DevMps& B = o.f_;
  size_t need = 1;
  for (int n = 0; n < N_; ++n) {
    const size_t ma = (size_t)std::max(A.b[n], A.b[n + 1]), mb = (size_t)std::max(B.b[n], B.b[n + 1]);
    need = std::max(need, ma * 2 * mb);
  }
  // the observable scratch (2 max_bond^2 doubles each) serves any pair of
  // states no wider than this one; a wider partner gets buffers of its own
  const bool own = need > (size_t)2 * max_bond_ * max_bond_;
  double *e0 = obsA_, *e1 = obsB_, *x = obsX_;
  if (own) {
    QTT_CUDA(cudaMalloc(&e0, need * sizeof(double)));
    QTT_CUDA(cudaMalloc(&e1, need * sizeof(double)));
    QTT_CUDA(cudaMalloc(&x, need * sizeof(double)));
  }
  fill_value(st_, e0, 1, 1.0);
  for (int n = 0; n < N_; ++n) {
    const int ba = A.b[n], bb = B.b[n], ba2 = A.b[n + 1], bb2 = B.b[n + 1];
    gemm64(ba, 2 * bb2, bb, 1, 1, 1.0, mv(e0, bb, 1), mv(B.core(n), 2LL * bb2, 1), 0.0, ov(x, 2LL * bb2, 1));
    gemm64(ba2, bb2, 2 * ba, 1, 1, 1.0, mv(A.core(n), 1, ba2), mv(x, bb2, 1), 0.0, ov(e1, bb2, 1));
    std::swap(e0, e1);
  }
  double r = 0;
  QTT_CUDA(cudaMemcpyAsync(&r, e0, sizeof(double), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  if (own) {
    cudaFree(e0);
    cudaFree(e1);
    cudaFree(x);
  }
  return r;
}

std::vector<double> Engine::download_state() const {
  std::vector<double> h(f_.total);
  QTT_CUDA(cudaMemcpyAsync(h.data(), f_.data, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  return h;
}

void Engine::upload_state(const std::vector<double>& cores) {
  if (cores.size() != f_.total) throw std::runtime_error("EINVAL: checkpoint size does not match the bond profile");
  QTT_CUDA(cudaMemcpyAsync(f_.data, cores.data(), cores.size() * sizeof(double), cudaMemcpyHostToDevice, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
}

std::vector<double> Engine::timings() const {
  std::vector<double> t;
  for (int c = 0; c < 6; ++c) {
    t.push_back(timer_->launches[c]);
    t.push_back(timer_->ms[c]);
    t.push_back(timer_->flops[c]);
  }
  t.push_back((double)launch_count());
  t.push_back(tc_issued_flops_);
  return t;
}

void Engine::set_time(double t, long long s) {
  time_ = t;
  steps_ = s;
  const unsigned long long c = (unsigned long long)s;
  QTT_CUDA(cudaMemcpyAsync(dstep_, &c, sizeof(c), cudaMemcpyHostToDevice, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
}

}  // namespace qtt
