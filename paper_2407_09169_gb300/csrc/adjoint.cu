// Discrete adjoint of the Heun step (gradient of the mean product
// J = avg_x (<1> - <Phi_1> - <Phi_2>), Eqs. 2 and spaceAvg, after nsteps
// steps of Eq. FP2) on the device.
//
// For the Euclidean inner product over all cells, one Heun step
// f_{n+1} = (f + f* + dt L(f*)) / 2, f* = f + dt L(f), has the adjoint
//     mu      = dJ/df*  = (S(f*)^T lambda) / 2
//     lambda' = dJ/df_n = lambda / 2 + S(f_n)^T mu,      S(f)^T = I + dt L'(f)^T
// and contributes dt <lambda, dL/dtheta(f*)> / 2 + dt <mu, dL/dtheta(f_n)> to
// dJ/dtheta.  In train form (all pieces built on the host, model.cpp):
//   S(f)^T g = (I + dt W_lin)^T g                              (MPO transpose)
//            - dt Omega sum_a diag(<Phi_a>[f](x)) D1phi_a^T g   (term kind 1 with
//              the transposed phi-part, diagonal cores from f)
//            - dt Omega h1 h2 sum_a phi_a (x) sum_phi f D1phi_a^T g   (term kind 2)
// The last one is the transpose of the dependence of <Phi_a> (Eq. 2, linear
// in f) inside the mixing drift: its phi part is the fixed weight train
// h1 h2 phi_a, and its x part is the Hadamard product of f's and g's x cores
// started by the partial contraction E_a[i][j] = <g_phi| D1phi_a |f_phi> over
// the phi sites (mix_env_core).  Each adjoint stage is a sum of such terms,
// rounded to chi by the same randomized rounding as the forward stages (its
// Gaussian sketches are drawn for the step and stages 2 and 3), so the
// backward sweep costs about as much as the forward one.  The parameter
// terms are "sandwiches" <a| Op |f> computed with the sketch-site
// contraction, the adjoint state in place of the sketch, in FP64 scalars.
// The forward states are kept every ckpt_every steps; each segment is
// recomputed (same sketches: the step counter is reset) before its backward
// sweep.
#include <algorithm>
#include <cstring>
#include <stdexcept>

#include "engine.hpp"

namespace qtt {

void Engine::copy_mps(const DevMps& from, DevMps& to) {
  if (from.total != to.total) throw std::runtime_error("EINVAL: state profiles differ");
  QTT_CUDA(cudaMemcpyAsync(to.data, from.data, from.total * sizeof(double), cudaMemcpyDeviceToDevice, st_));
}

void Engine::set_step_counter(unsigned long long s) {
  QTT_CUDA(cudaMemcpyAsync(dstep_, &s, sizeof(s), cudaMemcpyHostToDevice, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));  // s lives on the host stack
}

void Engine::grad_setup() {
  if (adj_ready_) return;
  if (p_.rk_variant != 0) throw std::runtime_error("EINVAL: the adjoint is written for the Heun scheme (rk_variant 0)");
  const int N = N_;
  adjm_ = build_adjoint_model(p_, model_);
  upload_op(op_lin_t_, adjm_.op_lin_t);
  upload_op(had_t_, adjm_.had_phi_t);
  upload_op(had_unit_, adjm_.had_unit);
  dL_.resize(adjm_.dL.size());
  for (size_t i = 0; i < dL_.size(); ++i) upload_op(dL_[i], adjm_.dL[i]);
  upload_op(dL_stack_, adjm_.dL_stack);
  dic_.resize(adjm_.dic.size());
  for (size_t i = 0; i < dic_.size(); ++i) {
    alloc_mps(dic_[i], adjm_.dic[i].r);
    upload_tt_mps(dic_[i], adjm_.dic[i], adjm_.dic[i].r);
  }
  alloc_mps(lamT_, D_);
  upload_tt_mps(lamT_, adjm_.lam_T, D_);
  alloc_mps(lam_[0], D_);
  alloc_mps(lam_[1], D_);
  alloc_mps(mu_, D_);
  alloc_mps(fin_, D_);
  alloc_mps(f0_, D_);
  upload_tt_mps(f0_, tt_round(model_.f0, 1e-14, p_.chi_max), D_);
  // aux: the weight train h1 h2 [phi1 (+) phi2] on the phi sites, then the
  // kind-2 core at site kphi (right bond = f bond x adjoint bond)
  const int kp = kphi_;
  const long long dd = (long long)D_[kp + 1] * D_[kp + 1];
  if (dd > (1LL << 26)) throw std::runtime_error("EINVAL: bond too large for the adjoint's mixing core");
  std::vector<int> ab(N + 1, 1);
  for (int n = 0; n <= kp; ++n) ab[n] = adjm_.c_stack.r[n];
  ab[kp + 1] = (int)dd;
  alloc_mps(aux_, ab);
  upload_tt_mps(aux_, adjm_.c_stack, ab);

  // slot 4 (kind-2 term): operated bond <= 4 on the phi sites (aux), the
  // product bond D_n^2 on the x sites; the zip product at site kphi holds
  // rz x 2 x D_{kphi+1}^2.
  auto w4 = [&](int n) -> size_t { return n <= kp ? (size_t)4 : (size_t)D_[n]; };
  const int nlo = exact_ ? nc_ + 1 : 1;
  {
    Woff_[4].assign(N + 1, 0);
    size_t tot = 0;
    for (int n = nlo; n <= N; ++n) {
      Woff_[4][n] = tot;
      tot += w4(n) * D_[n] * ell_[n];
    }
    Wslot_[4] = (double*)dalloc(tot * sizeof(double));
    size_t cmax = 1, tmax = 1, pp = pp_elems_;
    for (int n = 0; n < N; ++n) {
      const bool zipped = exact_ ? (n <= nc_) : true;
      if (!zipped) continue;
      cmax = std::max(cmax, (size_t)rz_[n] * w4(n) * D_[n]);
      tmax = std::max(tmax, (size_t)2 * rz_[n] * w4(n + 1) * D_[n + 1]);
      pp = std::max(pp, (size_t)rz_[n] * w4(n) * 2 * D_[n + 1]);
      if (n == kp) pp = std::max(pp, (size_t)rz_[n] * 2 * (size_t)dd);
    }
    C_[4] = (double*)dalloc(std::max(cmax, tmax) * sizeof(double));
    T_[4] = (double*)dalloc(std::max(cmax, tmax) * sizeof(double));
    if (pp > pp_elems_) {
      for (int l = 0; l < nlanes_; ++l) lane_p_[l] = (double*)dalloc(pp * sizeof(double));
      P_ = lane_p_[0];
      pp_elems_ = pp;
    }
  }
  // sandwich buffers: <a| Op |f> over all sites with a on the D profile and
  // f on the D profile or an IC-mode train
  std::vector<size_t> sb(N + 1), wm(N + 1, 1);
  for (int n = 0; n <= N; ++n) {
    sb[n] = (size_t)D_[n];
    for (const DevMps& m : dic_) sb[n] = std::max(sb[n], (size_t)m.b[n]);
    for (const DevOp& o : dL_) wm[n] = std::max(wm[n], (size_t)o.w[n]);
    wm[n] = std::max(wm[n], (size_t)dL_stack_.w[n]);
    wm[n] = std::max(wm[n], n <= kp ? (size_t)had_unit_.w[n] : (size_t)D_[n]);
  }
  swoff_.assign(N + 1, 0);
  size_t tot = 0, x1 = 1, x2 = 1;
  for (int n = 0; n <= N; ++n) {
    swoff_[n] = tot;
    tot += wm[n] * sb[n] * D_[n];
  }
  for (int n = 0; n < N; ++n) {
    x1 = std::max(x1, wm[n + 1] * sb[n + 1] * 2 * D_[n]);
    x2 = std::max(x2, wm[n + 1] * 4 * sb[n] * D_[n]);
  }
  sw_ = (double*)dalloc(tot * sizeof(double));
  sx1_ = (double*)dalloc(x1 * sizeof(double));
  sx2_ = (double*)dalloc(x2 * sizeof(double));
  // phi-site environments of the kind-2 core (two env buffers [j][w][i], then
  // Y [(w,i)][(s,j')] and Z [s'][w'][i][j']; X [a][j][s][h'] at site kphi)
  size_t e0 = 1, e1 = 1, e2 = 1;
  for (int n = 0; n < kp; ++n) {
    const size_t w = (size_t)had_t_.w[n], w2 = (size_t)had_t_.w[n + 1];
    e0 = std::max(e0, (size_t)D_[n + 1] * w2 * D_[n + 1]);
    e1 = std::max(e1, w * D_[n] * 2 * D_[n + 1]);
    e2 = std::max(e2, 2 * w2 * D_[n] * D_[n + 1]);
  }
  e0 = std::max(e0, (size_t)D_[kp] * 2 * D_[kp]);
  e1 = std::max(e1, (size_t)2 * D_[kp] * 2 * D_[kp + 1]);
  for (int i = 0; i < 4; ++i) senv_[i] = (double*)dalloc(std::max(e0, std::max(e1, e2)) * sizeof(double));
  gacc_ = (double*)dalloc((size_t)(n_grad_params() + 2) * sizeof(double));
  adj_ready_ = true;
}

// The kind-2 core of aux_ at site kphi for the pair (g = lam, f):
//   env[j][a][i] = sum over the phi sites of g[j..] had_phi[a..] f[i..]
//                 (= -dt Omega <g_phi| D1phi_a |f_phi>, bonds open at the cut)
//   X[a][j][s][h'] = sum_i env[j][a][i] f_kphi[i][s][h']
//   G[a][s][(h', j')] = sum_j X[a][j][s][h'] g_kphi[j][s][j']
// All in FP64 (small: the phi sites carry bonds <= chi, operator bond <= 2).
void Engine::mix_env_core(const DevMps& g, const DevMps& f) {
  const int kp = kphi_;
  double* env = senv_[0];
  double* env2 = senv_[1];
  double* Y = senv_[2];
  double* Z = senv_[3];
  fill_value(st_, env, 1, 1.0);
  for (int n = 0; n < kp; ++n) {
    const int bj = g.b[n], bj2 = g.b[n + 1], bi = f.b[n], bi2 = f.b[n + 1];
    const int wl = had_.w[n], wr = had_.w[n + 1];
    // Y[(w,i)][(s,j')] = sum_j env[j][(w,i)] g[j][(s,j')]
    gemm64(wl * bi, 2 * bj2, bj, 1, 1, 1.0, mv(env, 1, (long long)wl * bi), mv(g.core(n), 2LL * bj2, 1), 0.0,
           ov(Y, 2LL * bj2, 1));
    // Z[s'][w'][i][j'] = sum_{s,w} W[w][s,s'][w'] Y[w][i][s][j']   (batch over i)
    const double* Wss = had_.Wss(n);
    for (int sp = 0; sp < 2; ++sp)
      for (int s = 0; s < 2; ++s)
        gemm64(wr, bj2, wl, 1, bi, 1.0, mv(Wss + (size_t)(s * 2 + sp) * wl * wr, 1, wr),
               mv(Y + (size_t)s * bj2, (long long)bi * 2 * bj2, 1, 0, 2LL * bj2), s == 0 ? 0.0 : 1.0,
               ov(Z + (size_t)sp * wr * bi * bj2, (long long)bi * bj2, 1, 0, bj2));
    // env'[j'][w'][i'] = sum_{s',i} Z[s'][w'][i][j'] f[i][s'][i']   (batch over w')
    for (int sp = 0; sp < 2; ++sp)
      gemm64(bj2, bi2, bi, wr, 1, 1.0, mv(Z + (size_t)sp * wr * bi * bj2, 1, bj2, (long long)bi * bj2, 0),
             mv(f.core(n) + (size_t)sp * bi2, 2LL * bi2, 1), sp == 0 ? 0.0 : 1.0,
             ov(env2, (long long)wr * bi2, 1, bi2, 0));
    std::swap(env, env2);
  }
  // the open operator bond at the cut is the species a (2 values)
  const int bj = g.b[kp], bi = f.b[kp], df = f.b[kp + 1], dg = g.b[kp + 1];
  double* X = Y;
  gemm64(bj, 2 * df, bi, 2, 1, 1.0, mv(env, 2LL * bi, 1, bi, 0), mv(f.core(kp), 2LL * df, 1), 0.0,
         ov(X, 2LL * df, 1, (long long)bj * 2 * df, 0));
  gemm64(df, dg, bj, 2, 2, 1.0, mv(X, 1, 2LL * df, (long long)bj * 2 * df, df), mv(g.core(kp), 2LL * dg, 1, 0, dg), 0.0,
         ov(aux_.core(kp), dg, 1, 2LL * df * dg, (long long)df * dg));
}

Term Engine::term_mix_adj(const DevMps* lam, const DevMps* f, const double* hf, double scale) const {
  Term t;
  t.f = lam;
  t.kind = 1;
  t.op = &had_t_;
  t.hfirst = hf;
  t.hsrc = f;
  t.kphi = kphi_;
  t.slot = 2;
  t.scale = scale;
  return t;
}

Term Engine::term_mix_env(const DevMps* lam, const DevMps* f, double scale) const {
  Term t;
  t.f = lam;
  t.kind = 2;
  t.op = &ident_;
  t.hsrc = f;
  t.aux = &aux_;
  t.kphi = kphi_;
  t.slot = 4;
  t.scale = scale;
  return t;
}

// acc += w <a| Term |t.f>: the right-to-left sketch contraction with a in
// place of the random train, down to site 0 (a scalar).
void Engine::sandwich_acc(const DevMps& a, const Term& t, double w, double* acc) {
  const int N = N_;
  const int lane0 = lane_;
  lane_ = 0;
  std::swap(lane_x1_[0], sx1_);
  std::swap(lane_x2_[0], sx2_);
  fill_value(st_, sw_ + swoff_[N], 1, 1.0);
  for (int n = N - 1; n >= 0; --n)
    sketch_site(t, n, sw_ + swoff_[n + 1], sw_ + swoff_[n], a.core(n), a.b[n], a.b[n + 1], GEMM_STATE);
  std::swap(lane_x1_[0], sx1_);
  std::swap(lane_x2_[0], sx2_);
  lane_ = lane0;
  const double* one = gacc_ + n_grad_params() + 1;
  gemm64(t.wl(0), 1, 1, 1, 1, w, mv(sw_ + swoff_[0], 1, 1), mv(one, 1, 1), 1.0, ov(acc, 1, 1));
}

// acc[theta] += w <a| dL/dtheta(f) |f> for Omega, Da, gamma and the velocity
// modes (hf: the first x core of diag(<Phi_a>[f]) for the mixing part of
// dL/dOmega = sum_a D1phi_a[(phi_a - <Phi_a>) f]).
void Engine::grad_terms(const DevMps& a, const DevMps& f, const double* hf, double w) {
  double* g = gacc_ + 1;
  // the linear parts of every parameter in one contraction: the stacked
  // operator's open left bond carries the parameter index
  sandwich_acc(a, term_dense(1, &dL_stack_, &f, 1.0), w, g);
  Term mix = term_mix(&f, hf, 1.0);
  mix.op = &had_unit_;
  sandwich_acc(a, mix, w, g + 0);
}

std::vector<double> Engine::grad(int nsteps, int ckpt_every) {
  if (nsteps < 1) throw std::runtime_error("EINVAL: nsteps must be >= 1");
  if (sgs_) throw std::runtime_error("EINVAL: the discrete adjoint is not available with the subgrid closures (sgs)");
  // The adjoint's products may grow the per-lane packing workspaces (freeing
  // the old ones), which captured step graphs point into: drop the graphs,
  // so that the next qtt_step captures them again.
  QTT_CUDA(cudaStreamSynchronize(st_));
  drop_graphs();
  grad_setup();
  const int k = (ckpt_every < 1 || ckpt_every > nsteps) ? nsteps : ckpt_every;
  const int nseg = (nsteps + k - 1) / k;
  while ((int)ckpt_.size() < nseg) {
    ckpt_.emplace_back();
    alloc_mps(ckpt_.back(), D_);
  }
  while ((int)segf_.size() < k) {
    segf_.emplace_back();
    alloc_mps(segf_.back(), D_);
    segfs_.emplace_back();
    alloc_mps(segfs_.back(), D_);
  }
  const int np = n_grad_params();
  QTT_CUDA(cudaMemsetAsync(gacc_, 0, (size_t)(np + 1) * sizeof(double), st_));
  fill_value(st_, gacc_ + np + 1, 1, 1.0);

  // forward from the initial PDF, keeping every k-th state
  copy_mps(f0_, f_);
  set_step_counter(0);
  for (int s = 0; s < nsteps; ++s) {
    if (s % k == 0) copy_mps(f_, ckpt_[s / k]);
    step_body();
    std::swap(f_, g_);
    parity_ ^= 1;
  }
  copy_mps(f_, fin_);
  sandwich_acc(lamT_, term_dense(0, &ident_, &f_, 1.0), 1.0, gacc_);  // J

  // backward, one recomputed segment at a time
  int cur = 0;
  copy_mps(lamT_, lam_[0]);
  const double dt = p_.dt;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * k, s1 = std::min(nsteps, s0 + k);
    copy_mps(ckpt_[seg], f_);
    set_step_counter((unsigned long long)s0);
    for (int s = s0; s < s1; ++s) {
      copy_mps(f_, segf_[s - s0]);
      step_body();
      copy_mps(fs_, segfs_[s - s0]);
      std::swap(f_, g_);
      parity_ ^= 1;
    }
    for (int s = s1 - 1; s >= s0; --s) {
      const DevMps& fn = segf_[s - s0];
      const DevMps& fsn = segfs_[s - s0];
      DevMps& lam = lam_[cur];
      DevMps& lam2 = lam_[cur ^ 1];
      set_step_counter((unsigned long long)s);
      // mu = S(f*)^T lam / 2
      cond_means(fsn, v_[1]);
      make_hfirst(fsn, v_[1], hf_[1]);
      mix_env_core(lam, fsn);
      {
        Term b1[3] = {term_dense(1, &op_lin_t_, &lam, 0.5), term_mix_adj(&lam, &fsn, hf_[1], 0.5),
                      term_mix_env(&lam, &fsn, 0.5)};
        run_stage(b1, 3, mu_, 2);
      }
      grad_terms(lam, fsn, hf_[1], 0.5 * dt);
      // lam' = lam / 2 + S(f_n)^T mu
      cond_means(fn, v_[0]);
      make_hfirst(fn, v_[0], hf_[0]);
      grad_terms(mu_, fn, hf_[0], dt);
      mix_env_core(mu_, fn);
      {
        Term b2[4] = {term_dense(0, &ident_, &lam, 0.5), term_dense(1, &op_lin_t_, &mu_, 1.0),
                      term_mix_adj(&mu_, &fn, hf_[0], 1.0), term_mix_env(&mu_, &fn, 1.0)};
        run_stage(b2, 4, lam2, 3);
      }
      cur ^= 1;
    }
  }
  // initial-condition amplitudes: <dJ/df_0, g cos(q_m . x + p_m)>
  const size_t ic0 = 1 + 3 + p_.umodes.size();
  for (size_t m = 0; m < dic_.size(); ++m)
    sandwich_acc(lam_[cur], term_dense(0, &ident_, &dic_[m], 1.0), 1.0, gacc_ + ic0 + m);

  // the context continues from the final state
  copy_mps(fin_, f_);
  set_step_counter((unsigned long long)nsteps);
  time_ = nsteps * p_.dt;
  steps_ = nsteps;
  std::vector<double> out((size_t)np + 1);
  QTT_CUDA(cudaMemcpyAsync(out.data(), gacc_, out.size() * sizeof(double), cudaMemcpyDeviceToHost, st_));
  QTT_CUDA(cudaStreamSynchronize(st_));
  QTT_CUDA(cudaGetLastError());
  return out;
}

}  // namespace qtt
