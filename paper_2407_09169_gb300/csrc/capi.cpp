// C ABI of the QTT Fokker-Planck solver (declared in include/qtt_fp.h).
// Every entry point catches all exceptions and reports a status; nothing
// aborts.  Device work runs in the Engine (engine.cu); this file converts
// parameters, dispatches and formats outputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qtt_fp.h"
#include "engine.hpp"
#include "host_tt.hpp"
#include "model.hpp"

namespace qtt {
std::vector<double> run_selftest(int which);
}

struct qtt_ctx {
  std::unique_ptr<qtt::Engine> eng;
  std::string err;
};

namespace {

thread_local std::string g_init_err;

qtt_status classify(const std::string& m) {
  if (m.rfind("EINVAL", 0) == 0) return QTT_EINVAL;
  if (m.rfind("ENOMEM", 0) == 0) return QTT_ENOMEM;
  if (m.rfind("EIO", 0) == 0) return QTT_EIO;
  if (m.rfind("CUDA", 0) == 0) return QTT_ECUDA;
  return QTT_ESTATE;
}

bool to_params(const qtt_params* in, qtt::Params& p, std::string& err) {
  if (!in) {
    err = "EINVAL: params is NULL";
    return false;
  }
  for (int d = 0; d < 5; ++d) p.bits[d] = in->bits[d];
  p.chi_max = in->chi_max;
  p.svd_rel_tol = in->svd_rel_tol;
  p.precision = in->precision;
  p.oversample = in->oversample > 0 ? in->oversample : 8;
  p.exact = in->exact;
  p.seed = in->seed;
  p.omega = in->omega;
  p.da = in->da;
  p.gamma = in->gamma;
  p.d_phi = in->d_phi;
  p.dt = in->dt;
  p.shear_amp = in->shear_amp;
  if (in->n_umodes < 0 || in->n_umodes > 4096 || in->n_icmodes < 0 || in->n_icmodes > 4096) {
    err = "EINVAL: mode counts out of range";
    return false;
  }
  if (in->n_umodes > 0 && (!in->umode_comp || !in->umode_k || !in->umode_phase || !in->umode_amp)) {
    err = "EINVAL: velocity mode arrays are NULL";
    return false;
  }
  if (in->n_icmodes > 0 && (!in->icmode_k || !in->icmode_phase || !in->icmode_amp)) {
    err = "EINVAL: initial-condition mode arrays are NULL";
    return false;
  }
  p.umodes.clear();
  for (int m = 0; m < in->n_umodes; ++m) {
    qtt::Mode md;
    md.comp = in->umode_comp[m];
    for (int i = 0; i < 3; ++i) md.k[i] = in->umode_k[3 * m + i];
    md.phase = in->umode_phase[m];
    md.amp = in->umode_amp[m];
    p.umodes.push_back(md);
  }
  p.icmodes.clear();
  for (int m = 0; m < in->n_icmodes; ++m) {
    qtt::Mode md;
    for (int i = 0; i < 3; ++i) md.k[i] = in->icmode_k[3 * m + i];
    md.phase = in->icmode_phase[m];
    md.amp = in->icmode_amp[m];
    p.icmodes.push_back(md);
  }
  p.ic_sigma = in->ic_sigma;
  p.ic_blend_width = in->ic_blend_width;
  for (int i = 0; i < 2; ++i) {
    p.ic_c_hi[i] = in->ic_c_hi[i];
    p.ic_c_lo[i] = in->ic_c_lo[i];
  }
  p.rk_variant = in->rk_variant;
  p.flow = in->flow;
  p.u0 = in->u0;
  p.ic_kind = in->ic_kind;
  p.sgs = in->sgs;
  p.c_s = in->c_s;
  p.c_omega = in->c_omega;
  p.delta_cells = in->delta_cells;
  p.moment_ref = in->moment_ref;
  std::string why = qtt::validate(p);
  if (!why.empty()) {
    err = "EINVAL: " + why;
    return false;
  }
  return true;
}

// Dense matrix [row bits][col bits] of an operator train (d = 4).
std::vector<double> op_matrix(const qtt::TT& t) {
  const int N = t.N();
  const size_t M = (size_t)1 << N;
  std::vector<double> raw = qtt::tt_dense(t), out(M * M, 0.0);
  for (size_t idx = 0; idx < raw.size(); ++idx) {
    size_t row = 0, col = 0, x = idx;
    for (int n = N - 1; n >= 0; --n) {
      const size_t i = x & 3;
      x >>= 2;
      row |= (i >> 1) << (N - 1 - n);
      col |= (i & 1) << (N - 1 - n);
    }
    out[row * M + col] = raw[idx];
  }
  return out;
}

qtt_status put(const std::vector<double>& v, double* out, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  if (!out || cap < (int64_t)v.size()) return QTT_EINVAL;
  std::memcpy(out, v.data(), v.size() * sizeof(double));
  if (written) *written = (int64_t)v.size();
  return QTT_OK;
}

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ULL) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ULL;
  }
  return h;
}

}  // namespace

extern "C" {

const char* qtt_version(void) { return "qtt-fp-gb300 0.1 (sm_103a)"; }

const char* qtt_last_error(const qtt_ctx* ctx) {
  if (!ctx) return g_init_err.c_str();
  return ctx->err.c_str();
}

qtt_status qtt_init(const qtt_params* params, qtt_ctx** out) {
  if (!out) {
    g_init_err = "EINVAL: out is NULL";
    return QTT_EINVAL;
  }
  *out = nullptr;
  try {
    qtt::Params p;
    std::string err;
    if (!to_params(params, p, err)) {
      g_init_err = err;
      return QTT_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      g_init_err = std::string("CUDA: no usable CUDA device (") + cudaGetErrorString(e) + ")";
      return QTT_ECUDA;
    }
    std::unique_ptr<qtt_ctx> ctx(new qtt_ctx());
    ctx->eng.reset(new qtt::Engine(p, (cudaStream_t)params->stream));
    ctx->eng->init();
    *out = ctx.release();
    g_init_err.clear();
    return QTT_OK;
  } catch (const std::exception& ex) {
    g_init_err = ex.what();
    return classify(g_init_err);
  } catch (...) {
    g_init_err = "unknown failure in qtt_init";
    return QTT_ESTATE;
  }
}

qtt_status qtt_step(qtt_ctx* ctx, int32_t nsteps) {
  if (!ctx || !ctx->eng) return QTT_EINVAL;
  if (nsteps < 0) {
    ctx->err = "EINVAL: nsteps < 0";
    return QTT_EINVAL;
  }
  try {
    ctx->eng->step(nsteps);
    std::string msg;
    const int st = ctx->eng->check_status(msg);
    if (st != 0) {
      ctx->err = msg;
      return (qtt_status)st;
    }
    return QTT_OK;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

qtt_status qtt_grad(qtt_ctx* ctx, int32_t nsteps, int32_t ckpt_every, double* out, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  if (!ctx || !ctx->eng) return QTT_EINVAL;
  const int64_t need = 1 + ctx->eng->n_grad_params();
  if (written) *written = need;
  if (nsteps < 1 || !out || cap < need) {
    ctx->err = "EINVAL: qtt_grad needs nsteps >= 1 and room for 1 + n_params values";
    return QTT_EINVAL;
  }
  try {
    const std::vector<double> g = ctx->eng->grad(nsteps, ckpt_every);
    std::string msg;
    const int st = ctx->eng->check_status(msg);
    if (st != 0) {
      ctx->err = msg;
      return (qtt_status)st;
    }
    for (size_t i = 0; i < g.size(); ++i) out[i] = g[i];
    return QTT_OK;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

}  // extern "C"

namespace {

// One graph per step for a batch of contexts: once every context has
// captured its two step graphs, the graph of each context's current parity
// is embedded as an independent child node of one parent graph, which is
// launched on a stream of the batch; the next step uses the parent graph of
// the flipped parities.  Both parent graphs are built the first time a set
// of contexts (engine ids, graph generations, parities) is stepped and kept
// for the most recent set.
struct BatchGraph {
  std::vector<unsigned long long> ids;
  std::vector<unsigned> gens;
  std::vector<int> par0;  // parities the exec[0] graph was built for
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<cudaEvent_t> ctx_ev;
  void release() {
    for (cudaGraphExec_t& e : exec)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
  }
};
std::mutex g_batch_mu;
BatchGraph g_batch;

bool batch_build(qtt_ctx* const* ctxs, int32_t n) {
  BatchGraph& B = g_batch;
  B.release();
  if (!B.st && cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (!B.ev && cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming) != cudaSuccess) return false;
  while ((int32_t)B.ctx_ev.size() < n) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    B.ctx_ev.push_back(e);
  }
  B.ids.assign(n, 0);
  B.gens.assign(n, 0);
  B.par0.assign(n, 0);
  for (int32_t i = 0; i < n; ++i) {
    const qtt::Engine& E = *ctxs[i]->eng;
    B.ids[i] = E.id();
    B.gens[i] = E.graph_generation();
    B.par0[i] = E.parity();
  }
  for (int flip = 0; flip < 2; ++flip) {
    cudaGraph_t parent = nullptr;
    if (cudaGraphCreate(&parent, 0) != cudaSuccess) return false;
    bool ok = true;
    for (int32_t i = 0; i < n && ok; ++i) {
      cudaGraphNode_t node;
      ok = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0,
                                      ctxs[i]->eng->graph_template(B.par0[i] ^ flip)) == cudaSuccess;
    }
    ok = ok && cudaGraphInstantiate(&B.exec[flip], parent, 0) == cudaSuccess;
    cudaGraphDestroy(parent);
    if (!ok) {
      cudaGetLastError();
      B.release();
      return false;
    }
  }
  return true;
}

// exec index for the contexts' current parities, or -1 when the cached
// parent graphs do not describe this set of contexts
int batch_match(qtt_ctx* const* ctxs, int32_t n) {
  const BatchGraph& B = g_batch;
  if ((int32_t)B.ids.size() != n || !B.exec[0] || !B.exec[1]) return -1;
  int flip = -1;
  for (int32_t i = 0; i < n; ++i) {
    const qtt::Engine& E = *ctxs[i]->eng;
    if (B.ids[i] != E.id() || B.gens[i] != E.graph_generation()) return -1;
    const int f = E.parity() ^ B.par0[i];
    if (flip >= 0 && f != flip) return -1;
    flip = f;
  }
  return flip;
}

}  // namespace

extern "C" {

qtt_status qtt_step_many(qtt_ctx* const* ctxs, int32_t n, int32_t nsteps, int32_t* failed) {
  if (failed) *failed = -1;
  if (n < 0 || nsteps < 0 || (n > 0 && !ctxs)) return QTT_EINVAL;
  for (int32_t i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->eng) {
      if (failed) *failed = i;
      return QTT_EINVAL;
    }
    for (int32_t k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) {
        ctxs[i]->err = "EINVAL: a context appears twice in qtt_step_many";
        if (failed) *failed = i;
        return QTT_EINVAL;
      }
  }
  // step-major order: every context's step s is enqueued before any step s+1
  std::vector<int> bad(n, 0);
  std::vector<qtt_status> code(n, QTT_OK);
  std::lock_guard<std::mutex> batch_lock(g_batch_mu);
  bool on_batch = false;  // the batch stream holds work the contexts' streams have not waited for
  auto leave_batch = [&]() {
    if (!on_batch) return true;
    on_batch = false;
    if (cudaEventRecord(g_batch.ev, g_batch.st) != cudaSuccess) return false;
    for (int32_t i = 0; i < n; ++i)
      if (cudaStreamWaitEvent(ctxs[i]->eng->stream(), g_batch.ev, 0) != cudaSuccess) return false;
    return true;
  };
  for (int32_t s = 0; s < nsteps; ++s) {
    bool all_ready = n > 1;
    for (int32_t i = 0; i < n && all_ready; ++i) all_ready = !bad[i] && ctxs[i]->eng->step_graphs_ready();
    if (all_ready) {
      int flip = batch_match(ctxs, n);
      if (flip < 0 && batch_build(ctxs, n)) flip = batch_match(ctxs, n);
      if (flip >= 0) {
        bool ok = true;
        if (!on_batch) {  // the batch stream waits for every context's earlier work
          for (int32_t i = 0; i < n && ok; ++i)
            ok = cudaEventRecord(g_batch.ctx_ev[i], ctxs[i]->eng->stream()) == cudaSuccess &&
                 cudaStreamWaitEvent(g_batch.st, g_batch.ctx_ev[i], 0) == cudaSuccess;
        }
        ok = ok && cudaGraphLaunch(g_batch.exec[flip], g_batch.st) == cudaSuccess;
        if (ok) {
          on_batch = true;
          for (int32_t i = 0; i < n; ++i) ctxs[i]->eng->step_launched_externally();
          continue;
        }
        cudaGetLastError();
        g_batch.release();
      }
    }
    if (!leave_batch()) {
      for (int32_t i = 0; i < n; ++i) {
        ctxs[i]->err = "CUDA error: ordering the contexts after the batch graph failed";
        code[i] = QTT_ECUDA;
        bad[i] = 1;
      }
      break;
    }
    for (int32_t i = 0; i < n; ++i) {
      if (bad[i]) continue;
      try {
        ctxs[i]->eng->step(1);
      } catch (const std::exception& ex) {
        ctxs[i]->err = ex.what();
        code[i] = classify(ctxs[i]->err);
        bad[i] = 1;
      }
    }
  }
  if (!leave_batch()) {
    for (int32_t i = 0; i < n; ++i) {
      ctxs[i]->err = "CUDA error: ordering the contexts after the batch graph failed";
      code[i] = QTT_ECUDA;
      bad[i] = 1;
    }
  }
  qtt_status first = QTT_OK;
  for (int32_t i = 0; i < n; ++i) {
    if (!bad[i]) {
      try {
        std::string msg;
        const int st = ctxs[i]->eng->check_status(msg);
        if (st != 0) {
          ctxs[i]->err = msg;
          code[i] = (qtt_status)st;
        }
      } catch (const std::exception& ex) {
        ctxs[i]->err = ex.what();
        code[i] = classify(ctxs[i]->err);
      }
    }
    if (code[i] != QTT_OK && first == QTT_OK) {
      first = code[i];
      if (failed) *failed = i;
    }
  }
  return first;
}

qtt_status qtt_observe(qtt_ctx* ctx, int32_t what, double* out, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  if (!ctx || !ctx->eng) return QTT_EINVAL;
  if (!out) {
    ctx->err = "EINVAL: out is NULL";
    return QTT_EINVAL;
  }
  try {
    qtt::Engine& E = *ctx->eng;
    const qtt::Params& p = E.params();
    const int N = E.N();
    const int Kx = p.bits[2] + p.bits[3] + p.bits[4];
    switch (what) {
      case QTT_OBS_SCALARS: {
        std::vector<double> v(13);
        E.scalars(v.data());
        return put(v, out, cap, written);
      }
      case QTT_OBS_BONDS: {
        std::vector<int> b = E.bonds();
        return put(std::vector<double>(b.begin(), b.end()), out, cap, written);
      }
      case QTT_OBS_DENSE: {
        if (N > 26) {
          ctx->err = "EINVAL: dense output needs N <= 26";
          return QTT_EINVAL;
        }
        const int64_t need = (int64_t)1 << N;
        if (cap < need) {
          ctx->err = "EINVAL: cap < 2^N";
          return QTT_EINVAL;
        }
        E.dense(out);
        if (written) *written = need;
        return QTT_OK;
      }
      case QTT_OBS_MEANS: {
        if (Kx > 26) {
          ctx->err = "EINVAL: mean fields need K3+K4+K5 <= 26";
          return QTT_EINVAL;
        }
        const int64_t need = 3 * ((int64_t)1 << Kx);
        if (cap < need) {
          ctx->err = "EINVAL: cap < 3 * 2^(K3+K4+K5)";
          return QTT_EINVAL;
        }
        E.means(out);
        if (written) *written = need;
        return QTT_OK;
      }
      case QTT_OBS_POINTS: {
        if (cap < N || cap % N != 0) {
          ctx->err = "EINVAL: cap must be a positive multiple of N";
          return QTT_EINVAL;
        }
        const int npts = (int)(cap / N);
        std::vector<unsigned char> bits((size_t)cap);
        for (int64_t i = 0; i < cap; ++i) bits[i] = out[i] != 0.0 ? 1 : 0;
        std::vector<double> vals(npts);
        E.points(bits, npts, vals.data());
        std::memcpy(out, vals.data(), sizeof(double) * npts);
        if (written) *written = npts;
        return QTT_OK;
      }
      case QTT_OBS_NVPP: {
        std::vector<int> b = E.bonds();
        double s1 = 0, s2 = 0;
        for (int n = 1; n <= N; ++n) s1 += 2.0 * b[n - 1] * b[n];
        for (int n = 1; n < N; ++n) s2 += (double)b[n] * b[n];
        return put(std::vector<double>{s1 - s2}, out, cap, written);
      }
      case QTT_OBS_TIMINGS:
        return put(E.timings(), out, cap, written);
      case QTT_OBS_ERRORS: {
        if (p.moment_ref != 1) {
          ctx->err = "EINVAL: the error measures need a context made with moment_ref = 1";
          return QTT_EINVAL;
        }
        std::vector<double> v(6);
        E.error_sample(v.data());
        return put(v, out, cap, written);
      }
      default:
        ctx->err = "EINVAL: unknown observable";
        return QTT_EINVAL;
    }
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

qtt_status qtt_compare(qtt_ctx* a, qtt_ctx* b, double* rel_l2) {
  if (!a || !b || !a->eng || !b->eng || !rel_l2) return QTT_EINVAL;
  try {
    const double aa = a->eng->overlap(*a->eng);
    const double bb = b->eng->overlap(*b->eng);
    const double ab = a->eng->overlap(*b->eng);
    const double d2 = aa + bb - 2.0 * ab;
    *rel_l2 = std::sqrt(d2 > 0 ? d2 : 0.0) / std::sqrt(bb > 0 ? bb : 1e-300);
    return QTT_OK;
  } catch (const std::exception& ex) {
    a->err = ex.what();
    return classify(a->err);
  }
}

qtt_status qtt_save(qtt_ctx* ctx, const char* path) {
  if (!ctx || !ctx->eng || !path) return QTT_EINVAL;
  try {
    qtt::Engine& E = *ctx->eng;
    std::vector<double> data = E.download_state();
    std::vector<int> b = E.bonds();
    std::vector<unsigned char> buf;
    auto app = [&](const void* p, size_t n) {
      const unsigned char* c = (const unsigned char*)p;
      buf.insert(buf.end(), c, c + n);
    };
    const char magic[8] = {'Q', 'T', 'T', 'F', 'P', '0', '0', '1'};
    app(magic, 8);
    const int32_t N = E.N();
    app(&N, 4);
    for (int d = 0; d < 5; ++d) app(&E.params().bits[d], 4);
    const double t = E.time();
    const int64_t st = E.steps();
    app(&t, 8);
    app(&st, 8);
    for (int v : b) app(&v, 4);
    const uint64_t cnt = data.size();
    app(&cnt, 8);
    app(data.data(), data.size() * sizeof(double));
    const uint64_t h = fnv1a(buf.data(), buf.size());
    app(&h, 8);
    FILE* f = std::fopen(path, "wb");
    if (!f) {
      ctx->err = std::string("EIO: cannot open ") + path;
      return QTT_EIO;
    }
    const size_t wr = std::fwrite(buf.data(), 1, buf.size(), f);
    const int cl = std::fclose(f);
    if (wr != buf.size() || cl != 0) {
      ctx->err = "EIO: short write";
      return QTT_EIO;
    }
    return QTT_OK;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

qtt_status qtt_load(qtt_ctx* ctx, const char* path) {
  if (!ctx || !ctx->eng || !path) return QTT_EINVAL;
  try {
    FILE* f = std::fopen(path, "rb");
    if (!f) {
      ctx->err = std::string("EIO: cannot open ") + path;
      return QTT_EIO;
    }
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    std::fclose(f);
    qtt::Engine& E = *ctx->eng;
    const int N = E.N();
    const size_t head = 8 + 4 + 20 + 8 + 8 + 4 * (size_t)(N + 1) + 8;
    if (buf.size() < head + 8 || std::memcmp(buf.data(), "QTTFP001", 8) != 0) {
      ctx->err = "EIO: not a checkpoint of this library";
      return QTT_EIO;
    }
    uint64_t hstored;
    std::memcpy(&hstored, buf.data() + buf.size() - 8, 8);
    if (fnv1a(buf.data(), buf.size() - 8) != hstored) {
      ctx->err = "EIO: checksum mismatch (truncated or corrupted checkpoint)";
      return QTT_EIO;
    }
    size_t o = 8;
    int32_t Nf;
    std::memcpy(&Nf, buf.data() + o, 4);
    o += 4;
    if (Nf != N) {
      ctx->err = "EIO: checkpoint has a different number of sites";
      return QTT_EIO;
    }
    for (int d = 0; d < 5; ++d) {
      int32_t bd;
      std::memcpy(&bd, buf.data() + o, 4);
      o += 4;
      if (bd != E.params().bits[d]) {
        ctx->err = "EIO: checkpoint grid differs";
        return QTT_EIO;
      }
    }
    double t;
    int64_t st;
    std::memcpy(&t, buf.data() + o, 8);
    o += 8;
    std::memcpy(&st, buf.data() + o, 8);
    o += 8;
    std::vector<int> b = E.bonds();
    for (int n = 0; n <= N; ++n) {
      int32_t v;
      std::memcpy(&v, buf.data() + o, 4);
      o += 4;
      if (v != b[n]) {
        ctx->err = "EIO: checkpoint bond profile differs (chi_max mismatch)";
        return QTT_EIO;
      }
    }
    uint64_t cnt;
    std::memcpy(&cnt, buf.data() + o, 8);
    o += 8;
    if (buf.size() != o + cnt * sizeof(double) + 8) {
      ctx->err = "EIO: checkpoint size mismatch";
      return QTT_EIO;
    }
    std::vector<double> data(cnt);
    std::memcpy(data.data(), buf.data() + o, cnt * sizeof(double));
    E.upload_state(data);
    E.set_time(t, st);
    return QTT_OK;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

void qtt_destroy(qtt_ctx* ctx) {
  if (!ctx) return;
  try {
    if (ctx->eng) cudaStreamSynchronize(ctx->eng->stream());
  } catch (...) {
  }
  delete ctx;
}

qtt_status qtt_host_dense(const qtt_params* params, int32_t which, double* out, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  try {
    qtt::Params p;
    std::string err;
    if (!to_params(params, p, err)) {
      g_init_err = err;
      return QTT_EINVAL;
    }
    const int N = p.N();
    if (which == 0) {
      if (N > 26) return QTT_EINVAL;
      qtt::Model m = qtt::build_model(p);
      return put(qtt::tt_dense(m.f0), out, cap, written);
    }
    if (which >= 1 && which <= 3) {
      if (p.bits[2] + p.bits[3] + p.bits[4] > 26) return QTT_EINVAL;
      return put(qtt::tt_dense(qtt::velocity_tt(p, which - 1)), out, cap, written);
    }
    if ((which >= 10 && which <= 14) || (which >= 20 && which <= 24)) {
      const int d = which % 10;
      const int K = p.bits[d];
      const double h = d < 2 ? 1.0 / (double)(1 << K) : 2.0 * 3.14159265358979323846 / (double)(1 << K);
      qtt::TT op;
      if (which < 20) op = d < 2 ? qtt::op_d1_zero_sum(K, h) : qtt::op_d1_periodic(K, h);
      else op = d < 2 ? qtt::op_d2_zero_sum(K, h) : qtt::op_d2_periodic(K, h);
      return put(op_matrix(op), out, cap, written);
    }
    if (which == 30 || which == 31 || which == 40) {
      if (which != 40 && N > 12) return QTT_EINVAL;
      qtt::Model m = qtt::build_model(p);
      if (which == 40) return put(std::vector<double>(m.op_lin.r.begin(), m.op_lin.r.end()), out, cap, written);
      qtt::TT W = which == 30 ? qtt::linear_operator(p, m.u) : m.op_lin;
      return put(op_matrix(W), out, cap, written);
    }
    if (which == 32) {
      if (p.Kphi() > 12) return QTT_EINVAL;
      qtt::Model m = qtt::build_model(p);
      std::vector<double> res;
      for (int a = 0; a < 2; ++a) {
        qtt::TT t = m.had_phi;
        const int L = t.N() - 1;
        // select the open-bond column a of the last core
        std::vector<double> c((size_t)t.r[L] * 4, 0.0);
        for (int x = 0; x < t.r[L]; ++x)
          for (int i = 0; i < 4; ++i) c[(size_t)x * 4 + i] = t.at(L, x, i, a);
        t.c[L] = c;
        t.r[L + 1] = 1;
        std::vector<double> mtx = op_matrix(t);
        res.insert(res.end(), mtx.begin(), mtx.end());
      }
      return put(res, out, cap, written);
    }
    if (which == 41) {
      qtt::Model m = qtt::build_model(p);
      return put(std::vector<double>(m.f0.r.begin(), m.f0.r.end()), out, cap, written);
    }
    if (which == 33 || which == 42) {  // the encoded Omega_mix(x) (sgs), or its bonds
      if (p.sgs != 1) return QTT_EINVAL;
      qtt::Model m = qtt::build_model(p);
      if (which == 42) return put(std::vector<double>(m.omega_x.r.begin(), m.omega_x.r.end()), out, cap, written);
      return put(qtt::tt_dense(m.omega_x), out, cap, written);
    }
    return QTT_EINVAL;
  } catch (const std::exception& ex) {
    g_init_err = ex.what();
    return classify(g_init_err);
  }
}

qtt_status qtt_observe_points_noalloc(qtt_ctx* ctx, double* inout, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  if (!ctx || !ctx->eng || !inout) return QTT_EINVAL;
  try {
    const int N = ctx->eng->N();
    if (cap < N || cap % N != 0) {
      ctx->err = "EINVAL: cap must be a positive multiple of N";
      return QTT_EINVAL;
    }
    const int64_t npts = cap / N;
    if (npts > 0x7fffffff) {
      ctx->err = "EINVAL: too many points";
      return QTT_EINVAL;
    }
    ctx->eng->points_noalloc(inout, (int)npts);
    if (written) *written = npts;
    return QTT_OK;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return classify(ctx->err);
  }
}

qtt_status qtt_truncate_vjp(int32_t N, const int32_t* rx, const double* x, const int32_t* sy, const double* ybar,
                            int32_t chi, double tol, double eps, double* xbar, int64_t cap, int64_t* written,
                            int32_t* kept, void* stream) {
  if (written) *written = 0;
  try {
    if (N < 2 || N > 64) throw std::runtime_error("EINVAL: N must be in [2, 64]");
    if (!rx || !sy || !x || !ybar || !xbar || !kept) throw std::runtime_error("EINVAL: a pointer argument is NULL");
    if (rx[0] != 1 || rx[N] != 1 || sy[0] != 1 || sy[N] != 1)
      throw std::runtime_error("EINVAL: the end bonds of both trains must be 1");
    for (int n = 1; n < N; ++n) {
      if (rx[n] < 1 || sy[n] < 1) throw std::runtime_error("EINVAL: a bond is below 1");
      if (rx[n] > 1024 || sy[n] > 1024) throw std::runtime_error("EINVAL: a bond is above 1024");
      if (rx[n] > 2 * rx[n - 1])
        throw std::runtime_error("EINVAL: rx[n] > 2 rx[n-1]: the cores of x cannot be left-orthonormal");
    }
    if (chi < 1) throw std::runtime_error("EINVAL: chi < 1");
    if (!(tol >= 0.0) || !(eps >= 0.0) || !std::isfinite(tol) || !std::isfinite(eps))
      throw std::runtime_error("EINVAL: tol and eps must be finite and >= 0");
    std::vector<int> r(rx, rx + N + 1), s(sy, sy + N + 1);
    const size_t need = qtt::truncate_vjp_out_elems(N, r.data());
    if (cap < 0 || (size_t)cap < need)
      throw std::runtime_error("EINVAL: xbar has room for " + std::to_string(cap) + " doubles, " +
                               std::to_string(need) + " are needed");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      throw std::runtime_error("CUDA: no usable CUDA device");
    }
    std::vector<int> k((size_t)(N - 1), 0);
    qtt::truncate_vjp((cudaStream_t)stream, N, r.data(), x, s.data(), ybar, chi, tol, eps, xbar, k.data());
    for (int n = 0; n + 1 < N; ++n) kept[n] = k[(size_t)n];
    if (written) *written = (int64_t)need;
    g_init_err.clear();
    return QTT_OK;
  } catch (const std::exception& ex) {
    g_init_err = ex.what();
    return classify(g_init_err);
  }
}

qtt_status qtt_selftest(int32_t which, double* out, int64_t cap, int64_t* written) {
  if (written) *written = 0;
  try {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      g_init_err = "CUDA: no usable CUDA device";
      return QTT_ECUDA;
    }
    return put(qtt::run_selftest(which), out, cap, written);
  } catch (const std::exception& ex) {
    g_init_err = ex.what();
    return classify(g_init_err);
  }
}

}  // extern "C"
