// Device engine: storage of the PDF and operators on the GPU and the RK2
// stage algorithm (see engine.cu).
#pragma once

#include <cuda_runtime.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "model.hpp"

namespace qtt {

// Throws std::runtime_error("CUDA error: ...") when a runtime call fails.
#define QTT_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t _e = (call);                                                                   \
    if (_e != cudaSuccess)                                                                     \
      throw std::runtime_error(std::string("CUDA error: ") + cudaGetErrorString(_e) + " at " + \
                               __FILE__ + ":" + std::to_string(__LINE__));                     \
  } while (0)

// MPS with a static bond profile b[0..N], cores [b[n]][2][b[n+1]] in one allocation.
struct DevMps {
  int N = 0;
  std::vector<int> b;
  std::vector<size_t> off;
  size_t total = 0;
  double* data = nullptr;
  double* core(int n) const { return data + off[n]; }
  size_t core_elems(int n) const { return (size_t)b[n] * 2 * b[n + 1]; }
  size_t max_core_elems() const {
    size_t m = 0;
    for (int n = 0; n + 1 < (int)b.size(); ++n) m = core_elems(n) > m ? core_elems(n) : m;
    return m;
  }
  Chain chain() const;
};

// Dense MPO on the device in the two layouts the contractions read:
// Wt[s][w'][w*2+s'] and Wss[s*2+s'][w][w'] (both = W[w][s*2+s'][w']).
struct DevOp {
  int N = 0;
  std::vector<int> w;
  std::vector<size_t> off_t, off_ss;
  double* data = nullptr;
  const double* Wt(int n) const { return data + off_t[n]; }
  const double* Wss(int n) const { return data + off_ss[n]; }
};

// Arithmetic classes of the contractions (each precision form maps them to a
// tensor-core mode): products carrying the state, products of the random
// sketch environments, and state times sketch (the range finder's Y).
enum GemmRole { GEMM_STATE = 0, GEMM_SKETCH = 1, GEMM_RANGE = 2, GEMM_MIX = 3 };

// One summand c * Op * f of a stage.  kind 0: dense MPO over all sites;
// kind 1: mixing Hadamard term -- dense composition-space MPO on the phi
// sites, then the diagonal operator diag(<Phi_a>(x)) whose cores are the x
// cores of hsrc (the first one mixed with the conditional-mean vectors);
// hsrc is f itself in the forward step and the state the adjoint is
// linearised at in the backward step.  kind 2 (adjoint of the mixing term's
// dependence through <Phi_a>): the output h1 h2 phi_a (x) sum_phi hsrc
// (D1phi_a^T f), i.e. the fixed train aux (weights phi_a on the phi sites,
// then at the first x site a core that already holds the contraction over
// the phi sites) followed by diag(hsrc's x cores) applied to f's x cores.
struct Term {
  const DevMps* f = nullptr;
  int kind = 0;
  const DevOp* op = nullptr;
  const double* hfirst = nullptr;
  const DevMps* hsrc = nullptr;  // kinds 1, 2: source of the diagonal cores (null: f)
  const DevMps* aux = nullptr;   // kind 2: cores 0 .. kphi
  int kphi = 0;
  int slot = 0;  // scratch slot: 0 / 3 identity, 1 linear, 2 mixing, 4 adjoint mixing
  double scale = 1.0;
  const DevMps* hs() const { return hsrc ? hsrc : f; }
  // operated core of site n and its bonds
  const double* A(int n) const { return (kind == 2 && n <= kphi) ? aux->core(n) : f->core(n); }
  int bl(int n) const { return (kind == 2 && n <= kphi) ? aux->b[n] : f->b[n]; }
  int br(int n) const { return (kind == 2 && n <= kphi) ? aux->b[n + 1] : f->b[n + 1]; }
  // operator bond on the left of site n / on the right of site n
  int wl(int n) const {
    if (kind == 0) return op->w[n];
    if (kind == 1) return n <= kphi ? op->w[n] : hs()->b[n];
    return n <= kphi ? 1 : hs()->b[n];
  }
  int wr(int n) const { return (kind == 2 && n == kphi) ? 1 : wl(n + 1); }
  bool diag(int n) const { return (kind == 1 && n >= kphi) || (kind == 2 && n > kphi); }
  const double* H(int n) const { return (kind == 1 && n == kphi) ? hfirst : hs()->core(n); }
  long long B(int n) const { return (long long)wl(n) * bl(n); }
};

// strided views for the contraction calls
inline MatView mv(const double* p, long long rs, long long cs, long long so = 0, long long si = 0) {
  MatView v;
  v.p = p;
  v.rs = rs;
  v.cs = cs;
  v.so = so;
  v.si = si;
  return v;
}
inline OutView ov(double* p, long long rs, long long cs, long long so = 0, long long si = 0) {
  OutView v;
  v.p = p;
  v.rs = rs;
  v.cs = cs;
  v.so = so;
  v.si = si;
  return v;
}

struct KernelTimer;

class Engine {
 public:
  explicit Engine(const Params& p, cudaStream_t stream);
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  void init();                 // uploads the model; throws std::runtime_error
  void step(int nsteps);       // RK2 steps
  int check_status(std::string& msg);  // syncs; returns a qtt_status value
  // observables (host outputs)
  void scalars(double out[13]);
  std::vector<int> bonds() const { return f_.b; }
  void dense(double* out);                     // 2^N values
  void means(double* out);                     // 3 * 2^Kx values
  // the 6 space averages of one error sample (needs moment_ref, see QTT_OBS_ERRORS)
  void error_sample(double* out);
  void points(const std::vector<unsigned char>& bits, int npts, double* out);
  // Point evaluation through the fixed device array of points_static.cu
  // (no allocation); inout holds npts x N 0/1 flags and receives the values.
  void points_noalloc(double* inout, int npts);
  size_t points_noalloc_capacity() const;
  double overlap(const Engine& other);         // <this|other>
  double norm2() { return overlap(*this); }
  std::vector<double> download_state() const;
  void upload_state(const std::vector<double>& cores);
  std::vector<double> timings() const;

  const Params& params() const { return p_; }
  int N() const { return N_; }
  double time() const { return time_; }
  long long steps() const { return steps_; }
  double discarded_last() const { return discarded_last_; }
  cudaStream_t stream() const { return st_; }
  void set_time(double t, long long s);
  // Batched stepping (qtt_step_many): once both step graphs are captured, a
  // caller may launch the captured step itself (embedded in a graph of its
  // own) and then record the step here.  graph_template(q) is the captured
  // graph of parity q (owned by the engine); graph_generation() changes
  // whenever the engine drops or recaptures its graphs; id() is unique per
  // engine in the process.
  bool step_graphs_ready() const;
  int parity() const { return parity_; }
  cudaGraph_t graph_template(int q) const { return graph_tmpl_[q]; }
  unsigned graph_generation() const { return graph_gen_; }
  unsigned long long id() const { return id_; }
  void step_launched_externally();
  // Discrete adjoint (gradient of J = avg_x (<1> - <Phi_1> - <Phi_2>) after
  // nsteps Heun steps from the initial PDF): out[0] = J, out[1..] = dJ/dtheta
  // for Omega, Da, gamma, each velocity mode amplitude and each IC mode
  // amplitude.  The forward states are kept every ckpt_every steps and each
  // segment is recomputed before it is swept backwards.  Leaves the context
  // at the final state.
  std::vector<double> grad(int nsteps, int ckpt_every);
  int n_grad_params() const { return 3 + (int)p_.umodes.size() + (int)p_.icmodes.size(); }

 private:
  void* dalloc(size_t bytes);
  void alloc_mps(DevMps& m, const std::vector<int>& bonds);
  void upload_op(DevOp& op, const TT& t);
  void upload_tt_mps(DevMps& m, const TT& t, const std::vector<int>& bonds);
  // Contraction in the context's precision form (tensor cores for the reduced forms).
  // role: GEMM_STATE (products that carry the state), GEMM_SKETCH (products
  // of the random sketch environments), GEMM_RANGE (state times sketch),
  // GEMM_MIX (state products of the mixing term, which is O(dt))
  void gemm(int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B, double beta, OutView C,
            int role = 0);
  // FP64 product (Gram matrices, norms, masses, observables).
  void gemm64(int M, int N, int K, int outer, int inner, double alpha, MatView A, MatView B, double beta, OutView C);
  void cond_means(const DevMps& f, double* v);
  void make_hfirst(const DevMps& f, double* v, double* hf);
  void mix_cores(const DevMps& f, const double* hf);  // sgs: the mixing term's Kronecker cores into hk_
  void sketch_site(const Term& t, int n, const double* Wn1, double* Wn, const double* Om, int Ll, int Lr, int role);
  void sketch_pass(Term* terms, int nt, int n_stop, const DevMps& om);  // right-to-left, sites N-1 .. n_stop+1
  void zip_site(const Term& t, int n, int r, const double* C, double* T, double alpha);
  void run_stage(Term* terms, int nterms, DevMps& out, int stage);
  void step_body();      // one RK2 step from f_ into g_ (launches only)
  bool capture_step(int parity);  // false: graphs unavailable, run eagerly
  void drop_graphs();             // destroys the step graphs (the next steps recapture them)
  void run_stage_exact(Term* terms, int nterms, DevMps& out);
  void xgram(const DevMps& f, double* E);
  void gram_pass(const DevMps& g);
  void project_cores(const DevMps& g, DevMps& out);
  Term term_dense(int slot, const DevOp* op, const DevMps* f, double scale) const;
  Term term_mix(const DevMps* f, const double* hf, double scale) const;
  void chain_dense(const DevMps& f, int n0, const double* head, int head_rows, double* out);
  // the same into device memory (dout holds head_rows * 2^(N - n0) doubles)
  void chain_dense_dev(const DevMps& f, int n0, const double* head, int head_rows, double* dout);
  void means_dev(double* dout);  // <1>, <Phi_1>, <Phi_2> over x into device memory
  void moment_ref_step();        // one RK2 step of the first-moment reference (moment_ref)
  // adjoint (adjoint.cu)
  void grad_setup();
  void copy_mps(const DevMps& from, DevMps& to);
  void mix_env_core(const DevMps& lam, const DevMps& f);  // the kind-2 core of aux_ at site kphi
  Term term_mix_adj(const DevMps* lam, const DevMps* f, const double* hf, double scale) const;
  Term term_mix_env(const DevMps* lam, const DevMps* f, double scale) const;
  // acc[0 .. w0) += w <a| Term |t.f> (w0 = the term's open left operator bond)
  void sandwich_acc(const DevMps& a, const Term& t, double w, double* acc);
  void grad_terms(const DevMps& a, const DevMps& f, const double* hf, double w);
  void set_step_counter(unsigned long long s);

  Params p_;
  Model model_;
  cudaStream_t st_ = nullptr;
  bool own_stream_ = false;
  int N_ = 0, kphi_ = 0, nc_ = 0;
  int prec_bits_ = 64;
  bool qr_refine_ = false;
  bool small_fp32_ = false;         // operator-bond contractions on the CUDA cores in FP32
  bool small_sketch_fp32_ = false;  // those of the sketch pass in FP32
  bool exact_ = false;
  std::vector<void*> allocs_;
  std::vector<int> D_, ell_, rz_;
  DevMps f_, fs_, g_, mid_, omega_, wphi_[6];
  Chain* wchains_dev_ = nullptr;  // wphi_ chains on the device
  DevOp op_lin_, had_, ident_;
  // subgrid closures: the Omega_mix(x) train over the x sites, and the
  // mixing term's diagonal cores (f's x cores times it, built each stage)
  DevMps omx_, hk_;
  bool sgs_ = false;
  // first-moment reference (moment_ref): m [2][Mx], a stage buffer, the
  // velocity [3][Mx], gamma(x) [Mx] under sgs (else null), error sums [5]
  double *mref_ = nullptr, *mtmp_ = nullptr, *ux_ = nullptr, *gx_ = nullptr, *errs_ = nullptr;
  // scratch
  double *Wslot_[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<size_t> Woff_[5];
  double *C_[5] = {nullptr, nullptr, nullptr, nullptr, nullptr}, *T_[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *P_ = nullptr, *X1_ = nullptr, *X2_ = nullptr, *Y_ = nullptr;
  double *v_[2] = {nullptr, nullptr}, *hf_[2] = {nullptr, nullptr};
  double *envw_ = nullptr, *envout_ = nullptr, *ws_ = nullptr, *qrwork_ = nullptr, *gq_ = nullptr;
  double *disc_ = nullptr, *obsA_ = nullptr, *obsB_ = nullptr, *obsX_ = nullptr;
  int *status_ = nullptr, *ranks_ = nullptr;
  std::vector<double*> gram_, tU_;
  std::vector<int> trunc_bonds_;
  EigProblem* trunc_probs_ = nullptr;
  int trunc_nmax_ = 1, trunc_kmax_ = 0;
  size_t ws_elems_ = 0;
  // Lanes: lane 0 is st_; lanes 1..kLanes-1 are streams of their own on which
  // the terms' independent work (sketch chains; site tensors and projections
  // of the zip-up) runs concurrently, forked from and joined back into st_
  // with events (also inside a captured graph).  Each lane has its own GEMM
  // workspaces and scratch.
  static constexpr int kLanes = 5;
  int lane_ = 0, nlanes_ = 1;
  cudaStream_t lane_st_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork_ = nullptr, ev_join_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* lane_ws_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *lane_x1_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *lane_x2_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *lane_p_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *lane_y_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  void* pack_ws_[kLanes] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t pack_bytes_[kLanes] = {0, 0, 0, 0, 0};
  cudaStream_t cur() const { return lane_st_[lane_]; }
  void fork_lanes(int n);  // lanes 1..n wait for st_
  void join_lanes(int n);  // st_ waits for lanes 1..n
  int tc_mode_[4] = {-1, -1, -1, -1};  // per GEMM role; -1: FP64 kernel
  int max_bond_ = 1;
  unsigned long long* dstep_ = nullptr;  // device copy of the step count (sketch draws)
  // CUDA graphs of one step, indexed by which of the two state buffers is f_
  // (the step swaps them); captured after one step has run eagerly.
  cudaGraphExec_t graph_[2] = {nullptr, nullptr};
  cudaGraph_t graph_tmpl_[2] = {nullptr, nullptr};  // the captured graphs (for embedding)
  unsigned graph_gen_ = 0;
  unsigned long long id_ = 0;
  int graph_launches_[2] = {0, 0};
  bool graphs_ = true, warm_ = false;
  int parity_ = 0;
  double time_ = 0.0;
  long long steps_ = 0;
  double discarded_last_ = 0.0;
  KernelTimer* timer_ = nullptr;
  double tc_issued_flops_ = 0.0;
  // adjoint state (allocated by grad_setup on the first grad call)
  bool adj_ready_ = false;
  AdjointModel adjm_;
  DevOp op_lin_t_, had_t_, had_unit_, dL_stack_;
  std::vector<DevOp> dL_;
  std::vector<DevMps> dic_;
  DevMps lamT_, lam_[2], mu_, aux_, f0_, fin_;
  std::vector<DevMps> ckpt_, segf_, segfs_;
  double *sw_ = nullptr, *sx1_ = nullptr, *sx2_ = nullptr, *senv_[4] = {nullptr, nullptr, nullptr, nullptr};
  double* gacc_ = nullptr;  // [0] J, [1..] dJ/dtheta, [last] the constant 1
  std::vector<size_t> swoff_;
  size_t pp_elems_ = 0;
};

// Backward of the simultaneous bond truncation in tensor-train form
// (trunc_vjp.cu).  x: N cores [rx[n]][2][rx[n+1]] concatenated in site order,
// the first N-1 left-orthonormal; ybar: N cores of bonds sy; xbar receives
// the vector-Jacobian product as a train of bonds 1, 2 rx[1], ..,
// 2 rx[N-1], 1 (truncate_vjp_out_elems doubles); kept[0..N-1) the kept
// counts min(chi, #{lambda_i > max(tol^2, 1e-24) lambda_0}) of the right
// Grams.  Device pointers; synchronises st; throws on failure.
size_t truncate_vjp_out_elems(int N, const int* rx);
void truncate_vjp(cudaStream_t st, int N, const int* rx, const double* x, const int* sy, const double* ybar, int chi,
                  double tol, double eps, double* xbar, int* kept);

}  // namespace qtt
