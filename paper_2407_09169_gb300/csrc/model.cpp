// Problem set-up (see model.hpp).
//
// Paper references:
//   Eq. FP0 / FP2     -- the operator: transport -u.grad f, diffusion gamma lap f,
//                        composition drift d/dphi_a [Omega (phi_a - <Phi_a>) f]
//                        and reaction -d/dphi_a (S_a f), S_a = -Da phi1 phi2,
//                        plus the artificial dissipation D_phi d2f/dphi_a^2.
//   Eq. compBCs       -- zero-sum ghost rules for composition derivatives.
//   "Finite-difference discretisation" -- CFD2 stencils, periodic x.
//   "Matrix product state encoding"    -- site order phi1, phi2, x1, x2, x3,
//                        each dimension coarse-to-fine (most significant bit first).
#include "model.hpp"

#include <algorithm>
#include <cmath>
#include <sstream>
#include <stdexcept>

namespace qtt {

static const double kPi = 3.14159265358979323846;
static const double kTol = 1e-14;  // numerical-rank threshold of the exact encodings

std::string validate(const Params& p) {
  std::ostringstream e;
  for (int d = 0; d < 5; ++d)
    if (p.bits[d] < 1 || p.bits[d] > 12) e << "bits[" << d << "]=" << p.bits[d] << " outside 1..12; ";
  if (p.chi_max < 1) e << "chi_max must be >= 1; ";
  if (p.chi_max > 4096) e << "chi_max > 4096 unsupported; ";
  if (!(p.svd_rel_tol >= 0.0) || p.svd_rel_tol >= 1.0) e << "svd_rel_tol must be in [0, 1); ";
  if (p.precision < 0 || p.precision > 4) e << "unknown precision " << p.precision << "; ";
  if (!(p.dt > 0.0) || !std::isfinite(p.dt)) e << "dt must be positive; ";
  if (!(p.ic_sigma > 0.0)) e << "ic_sigma must be positive; ";
  if (p.ic_kind == 2 ? !(p.ic_blend_width >= 0.0) : !(p.ic_blend_width > 0.0))
    e << "ic_blend_width must be positive (ic_kind 2: non-negative); ";
  if (p.flow != 0 && p.flow != 1) e << "flow must be 0 or 1; ";
  if (p.ic_kind < 0 || p.ic_kind > 2) e << "ic_kind must be 0, 1 or 2; ";
  if (!std::isfinite(p.u0)) e << "u0 must be finite; ";
  if (p.oversample < 0 || p.oversample > 256) e << "oversample outside 0..256; ";
  if (p.rk_variant != 0 && p.rk_variant != 1) e << "rk_variant must be 0 or 1; ";
  if (p.sgs != 0 && p.sgs != 1) e << "sgs must be 0 or 1; ";
  if (p.moment_ref != 0 && p.moment_ref != 1) e << "moment_ref must be 0 or 1; ";
  if (p.moment_ref == 1 && p.bits[2] + p.bits[3] + p.bits[4] > 26) e << "moment_ref needs K3 + K4 + K5 <= 26; ";
  if (p.sgs == 1) {
    if (p.bits[2] + p.bits[3] + p.bits[4] > 18) e << "sgs needs K3 + K4 + K5 <= 18 (dense fields at set-up); ";
    if (!(p.c_s >= 0.0) || !(p.c_omega >= 0.0) || !(p.delta_cells > 0.0) || !std::isfinite(p.c_s) ||
        !std::isfinite(p.c_omega) || !std::isfinite(p.delta_cells))
      e << "sgs needs c_s >= 0, c_omega >= 0, delta_cells > 0; ";
  }
  for (const Mode& m : p.umodes) {
    if (m.comp < 0 || m.comp > 2) e << "velocity mode component outside 0..2; ";
    else if (m.k[m.comp] != 0) e << "velocity mode must have k[comp] = 0 (divergence-free); ";
  }
  const double vals[] = {p.omega, p.da, p.gamma, p.d_phi, p.shear_amp};
  for (double v : vals)
    if (!std::isfinite(v)) e << "non-finite coefficient; ";
  if (p.exact) {
    const int N = p.N();
    if (p.svd_rel_tol != 0.0) e << "exact mode requires svd_rel_tol = 0; ";
    if (N > 26) e << "exact mode supports N <= 26; ";
    else if ((long long)p.chi_max < (1LL << (N / 2))) e << "exact mode requires chi_max >= 2^(N/2); ";
  }
  return e.str();
}

// ---------------------------------------------------------------- operators
TT op_shift(int K, int dir, bool periodic) {
  // Core W[c_out][s_out*2 + s_in][c_in]; the carry (dir = +1) or borrow
  // (dir = -1) enters at the least significant (rightmost) site with value 1
  // and leaves at the most significant site, where it is summed (periodic
  // wrap) or required to vanish (no row beyond the lattice).
  std::vector<double> W(2 * 4 * 2, 0.0);
  auto at = [&](int co, int so, int si, int ci) -> double& { return W[(co * 4 + so * 2 + si) * 2 + ci]; };
  for (int s = 0; s < 2; ++s) at(0, s, s, 0) = 1.0;  // no carry: copy the bit
  if (dir > 0) {  // s_in = s_out + 1
    at(0, 0, 1, 1) = 1.0;
    at(1, 1, 0, 1) = 1.0;
  } else {        // s_in = s_out - 1
    at(1, 0, 1, 1) = 1.0;
    at(0, 1, 0, 1) = 1.0;
  }
  const double lv[2] = {1.0, periodic ? 1.0 : 0.0};
  TT t;
  t.d = 4;
  t.r.assign(K + 1, 2);
  t.r[0] = t.r[K] = 1;
  t.c.resize(K);
  for (int n = 0; n < K; ++n) {
    const int L = t.r[n], R = t.r[n + 1];
    t.c[n].assign((size_t)L * 4 * R, 0.0);
    for (int co = 0; co < 2; ++co)
      for (int i = 0; i < 4; ++i)
        for (int ci = 0; ci < 2; ++ci) {
          const double w = W[(co * 4 + i) * 2 + ci];
          if (w == 0.0) continue;
          double lw = (n == 0) ? lv[co] : 1.0;
          double rw = (n == K - 1) ? (ci == 1 ? 1.0 : 0.0) : 1.0;
          const int l = (n == 0) ? 0 : co, r = (n == K - 1) ? 0 : ci;
          t.c[n][((size_t)l * 4 + i) * R + r] += w * lw * rw;
        }
  }
  return t;
}

static TT op_projector(int K, int bit) {
  TT t = mpo_identity(K);
  for (int n = 0; n < K; ++n) t.c[n] = bit ? std::vector<double>{0, 0, 0, 1} : std::vector<double>{1, 0, 0, 0};
  return t;
}

static TT scaled(TT t, double s) {
  tt_scale(t, s);
  return t;
}

TT op_d1_periodic(int K, double h) {
  TT t = tt_add(scaled(op_shift(K, +1, true), 1.0 / (2 * h)), scaled(op_shift(K, -1, true), -1.0 / (2 * h)));
  return tt_round(t, kTol, 0);
}

TT op_d2_periodic(int K, double h) {
  TT t = tt_add(op_shift(K, +1, true), op_shift(K, -1, true));
  t = tt_add(t, scaled(mpo_identity(K), -2.0));
  tt_scale(t, 1.0 / (h * h));
  return tt_round(t, kTol, 0);
}

TT op_d1_zero_sum(int K, double h) {
  // (g_{i+1} - g_{i-1}) / 2h with g_{-1} = -g_0 and g_M = -g_{M-1}:
  // the non-periodic shifts plus (P_0 - P_{M-1}) / 2h on the end rows.
  TT t = tt_add(op_shift(K, +1, false), scaled(op_shift(K, -1, false), -1.0));
  t = tt_add(t, op_projector(K, 0));
  t = tt_add(t, scaled(op_projector(K, 1), -1.0));
  tt_scale(t, 1.0 / (2 * h));
  return tt_round(t, kTol, 0);
}

TT op_d2_zero_sum(int K, double h) {
  // (f_{i+1} - 2 f_i + f_{i-1}) / h^2 with f_{-1} = f_0 and f_M = f_{M-1}.
  TT t = tt_add(op_shift(K, +1, false), op_shift(K, -1, false));
  t = tt_add(t, scaled(mpo_identity(K), -2.0));
  t = tt_add(t, op_projector(K, 0));
  t = tt_add(t, op_projector(K, 1));
  tt_scale(t, 1.0 / (h * h));
  return tt_round(t, kTol, 0);
}

TT embed_op(const Params& p, const TT& op, int dim) {
  TT t;
  for (int d = 0; d < 5; ++d) {
    TT piece = (d == dim) ? op : mpo_identity(p.bits[d]);
    t = (d == 0) ? piece : tt_kron(t, piece);
  }
  return t;
}

// ---------------------------------------------------------------- fields
static std::vector<double> grid_phi(int K) {
  const size_t M = (size_t)1 << K;
  std::vector<double> v(M);
  for (size_t i = 0; i < M; ++i) v[i] = (i + 0.5) / (double)M;
  return v;
}

static std::vector<double> grid_x(int K) {
  const size_t M = (size_t)1 << K;
  std::vector<double> v(M);
  for (size_t i = 0; i < M; ++i) v[i] = 2.0 * kPi * (double)i / (double)M;
  return v;
}

template <typename F>
static TT encode(int K, const std::vector<double>& grid, F fn) {
  std::vector<double> v(grid.size());
  for (size_t i = 0; i < grid.size(); ++i) v[i] = fn(grid[i]);
  return tt_from_vector(v, K, kTol);
}

static TT kron3(const TT& a, const TT& b, const TT& c) { return tt_kron(tt_kron(a, b), c); }

// sum over the 4 separable terms of sin/cos(k1 x1 + k2 x2 + k3 x3 + theta)
static TT fourier_tt(const Params& p, const int k[3], double theta, bool use_sin) {
  const int Kx[3] = {p.bits[2], p.bits[3], p.bits[4]};
  TT c1 = encode(Kx[0], grid_x(Kx[0]), [&](double x) { return std::cos(k[0] * x + theta); });
  TT s1 = encode(Kx[0], grid_x(Kx[0]), [&](double x) { return std::sin(k[0] * x + theta); });
  TT c2 = encode(Kx[1], grid_x(Kx[1]), [&](double x) { return std::cos(k[1] * x); });
  TT s2 = encode(Kx[1], grid_x(Kx[1]), [&](double x) { return std::sin(k[1] * x); });
  TT c3 = encode(Kx[2], grid_x(Kx[2]), [&](double x) { return std::cos(k[2] * x); });
  TT s3 = encode(Kx[2], grid_x(Kx[2]), [&](double x) { return std::sin(k[2] * x); });
  TT t;
  if (use_sin) {
    // sin(a+b+c) = s c c + c s c + c c s - s s s
    t = kron3(s1, c2, c3);
    t = tt_add(t, kron3(c1, s2, c3));
    t = tt_add(t, kron3(c1, c2, s3));
    t = tt_add(t, scaled(kron3(s1, s2, s3), -1.0));
  } else {
    // cos(a+b+c) = c c c - c s s - s c s - s s c
    t = kron3(c1, c2, c3);
    t = tt_add(t, scaled(kron3(c1, s2, s3), -1.0));
    t = tt_add(t, scaled(kron3(s1, c2, s3), -1.0));
    t = tt_add(t, scaled(kron3(s1, s2, c3), -1.0));
  }
  return tt_round(t, kTol, 0);
}

// The paper's flow (Eq. velField) on [0, l0)^3 with l0 = 2 pi: a Taylor-Green
// vortex of wavenumber k = 4 pi / l0 and, in u1, a Gaussian jet of width l0/6
// centred at x2 = x3 = l0 / 2.  Every term is a product of one-dimensional
// functions, so each component is a short sum of Kronecker products.
static TT paper_velocity_tt(const Params& p, int comp) {
  const int Kx[3] = {p.bits[2], p.bits[3], p.bits[4]};
  const double k = 2.0;  // 4 pi / l0
  auto f1 = [&](int d, bool cosine) {
    return encode(Kx[d], grid_x(Kx[d]), [=](double x) { return cosine ? std::cos(k * x) : std::sin(k * x); });
  };
  // (c1 s2 s3, s1 c2 s3, -2 s1 s2 c3)
  TT tg = kron3(f1(0, comp == 0), f1(1, comp == 1), f1(2, comp == 2));
  tt_scale(tg, comp == 2 ? -2.0 * p.u0 : p.u0);
  if (comp != 0) return tg;
  auto jet = [&](int d) {
    return encode(Kx[d], grid_x(Kx[d]), [](double x) {
      const double z = x / (2.0 * kPi) - 0.5;
      return std::exp(-z * z / (2.0 / 36.0));
    });
  };
  TT j = kron3(tt_constant(Kx[0], 1.0), jet(1), jet(2));
  tt_scale(j, -p.u0);
  return tt_round(tt_add(tg, j), kTol, 0);
}

TT velocity_tt(const Params& p, int comp) {
  const int Kx[3] = {p.bits[2], p.bits[3], p.bits[4]};
  TT u = kron3(tt_constant(Kx[0], 0.0), tt_constant(Kx[1], 1.0), tt_constant(Kx[2], 1.0));
  if (p.flow == 1) u = paper_velocity_tt(p, comp);
  if (p.flow == 0 && comp == 0 && p.shear_amp != 0.0) {
    TT sh = kron3(tt_constant(Kx[0], 1.0),
                  encode(Kx[1], grid_x(Kx[1]), [&](double x) { return std::tanh(x - kPi); }),
                  tt_constant(Kx[2], 1.0));
    tt_scale(sh, p.shear_amp);
    u = tt_add(u, sh);
  }
  for (const Mode& m : p.umodes) {
    if (m.comp != comp || m.amp == 0.0) continue;
    u = tt_add(u, scaled(fourier_tt(p, m.k, m.phase, true), m.amp));
  }
  return tt_round(u, kTol, 0);
}

static TT ones_x(const Params& p) {
  return kron3(tt_constant(p.bits[2], 1.0), tt_constant(p.bits[3], 1.0), tt_constant(p.bits[4], 1.0));
}

static TT phi_weight(const Params& p, int e1, int e2) {
  // h1 h2 phi1^e1 phi2^e2 over the phi sites
  const double h1 = 1.0 / (double)(1 << p.bits[0]), h2 = 1.0 / (double)(1 << p.bits[1]);
  TT a = encode(p.bits[0], grid_phi(p.bits[0]), [&](double v) { return std::pow(v, e1); });
  TT b = encode(p.bits[1], grid_phi(p.bits[1]), [&](double v) { return std::pow(v, e2); });
  TT t = tt_kron(a, b);
  tt_scale(t, h1 * h2);
  return t;
}

static TT gaussian_phi(const Params& p, const double c[2]) {
  // normalised separable Gaussian: h1 h2 sum g = 1 on the cell-centred grid
  TT out;
  for (int a = 0; a < 2; ++a) {
    const int K = p.bits[a];
    const std::vector<double> g = grid_phi(K);
    std::vector<double> v(g.size());
    double s = 0;
    for (size_t i = 0; i < g.size(); ++i) {
      v[i] = std::exp(-(g[i] - c[a]) * (g[i] - c[a]) / (2.0 * p.ic_sigma * p.ic_sigma));
      s += v[i];
    }
    const double h = 1.0 / (double)g.size();
    for (double& x : v) x /= (s * h);
    TT t = tt_from_vector(v, K, kTol);
    out = (a == 0) ? t : tt_kron(out, t);
  }
  return out;
}

// ic_kind 2 (ours, not the paper's): a composition-space Gaussian whose
// centre moves with x, c1 = ic_c_hi[0] + A sin(x1) cos(x2),
// c2 = ic_c_hi[1] - A sin(x2 + x3), A = ic_blend_width, std ic_sigma, each
// factor normalised on the phi grid (h_a sum_i G = 1) so that <1>(x) = 1.
// It couples phi with x (not a short sum of products), so it is encoded by
// tensor cross from point evaluations.
static TT moving_gaussian_pdf(const Params& p) {
  const int N = p.N();
  const int K[5] = {p.bits[0], p.bits[1], p.bits[2], p.bits[3], p.bits[4]};
  const size_t M[5] = {(size_t)1 << K[0], (size_t)1 << K[1], (size_t)1 << K[2], (size_t)1 << K[3], (size_t)1 << K[4]};
  const std::vector<double> ph1 = grid_phi(K[0]), ph2 = grid_phi(K[1]);
  const std::vector<double> x1 = grid_x(K[2]), x2 = grid_x(K[3]), x3 = grid_x(K[4]);
  const double A = p.ic_blend_width, s2 = 2.0 * p.ic_sigma * p.ic_sigma;
  auto g = [&](double d) { return std::exp(-d * d / s2); };
  // centres and 1-D normalisations on the x planes they depend on
  std::vector<double> c1(M[2] * M[3]), z1(M[2] * M[3]), c2(M[3] * M[4]), z2(M[3] * M[4]);
  for (size_t a = 0; a < M[2]; ++a)
    for (size_t b = 0; b < M[3]; ++b) {
      const double c = p.ic_c_hi[0] + A * std::sin(x1[a]) * std::cos(x2[b]);
      double z = 0.0;
      for (double v : ph1) z += g(v - c);
      c1[a * M[3] + b] = c;
      z1[a * M[3] + b] = z / (double)M[0];
    }
  for (size_t b = 0; b < M[3]; ++b)
    for (size_t e = 0; e < M[4]; ++e) {
      const double c = p.ic_c_hi[1] - A * std::sin(x2[b] + x3[e]);
      double z = 0.0;
      for (double v : ph2) z += g(v - c);
      c2[b * M[4] + e] = c;
      z2[b * M[4] + e] = z / (double)M[1];
    }
  auto F = [&](const uint8_t* bits) {
    size_t idx[5];
    int o = 0;
    for (int d = 0; d < 5; ++d) {
      size_t v = 0;
      for (int k = 0; k < K[d]; ++k) v = (v << 1) | bits[o + k];
      idx[d] = v;
      o += K[d];
    }
    const size_t i1 = idx[2] * M[3] + idx[3], i2 = idx[3] * M[4] + idx[4];
    return g(ph1[idx[0]] - c1[i1]) / z1[i1] * g(ph2[idx[1]] - c2[i2]) / z2[i2];
  };
  // the state keeps at most chi_max per bond, so the cross needs a little more
  TT t = tt_cross(N, F, p.chi_max + 16, 1e-12, 8, p.seed ^ 0x5eedc0deULL, nullptr);
  return tt_round(t, kTol, 0);
}

static TT initial_pdf(const Params& p) {
  const int Kx[3] = {p.bits[2], p.bits[3], p.bits[4]};
  // ic_kind 0: w(x2) = (1 + tanh((x2 - pi) / width)) / 2.  ic_kind 1 (Eq. initPDF):
  // the band l0/4 <= x1 < 3 l0/4 (l0 = 2 pi) with tanh edges of the given width,
  // w(x1) = (tanh((x1 - pi/2) / width) - tanh((x1 - 3 pi/2) / width)) / 2.
  const int d = p.ic_kind == 1 ? 0 : 1;
  auto w = [&](double x) {
    if (p.ic_kind == 1)
      return 0.5 * (std::tanh((x - 0.5 * kPi) / p.ic_blend_width) - std::tanh((x - 1.5 * kPi) / p.ic_blend_width));
    return 0.5 * (1.0 + std::tanh((x - kPi) / p.ic_blend_width));
  };
  auto blend = [&](bool hi) {
    TT parts[3] = {tt_constant(Kx[0], 1.0), tt_constant(Kx[1], 1.0), tt_constant(Kx[2], 1.0)};
    parts[d] = encode(Kx[d], grid_x(Kx[d]), [&](double x) { return hi ? w(x) : 1.0 - w(x); });
    return kron3(parts[0], parts[1], parts[2]);
  };
  TT f;
  if (p.ic_kind == 2) {
    f = moving_gaussian_pdf(p);
  } else {
    TT whi = blend(true), wlo = blend(false);
    f = tt_add(tt_kron(gaussian_phi(p, p.ic_c_hi), whi), tt_kron(gaussian_phi(p, p.ic_c_lo), wlo));
    f = tt_round(f, kTol, 0);
  }
  bool any = false;
  for (const Mode& m : p.icmodes) any = any || (m.amp != 0.0);
  if (any) {
    TT mod = ones_x(p);
    for (const Mode& m : p.icmodes)
      if (m.amp != 0.0) mod = tt_add(mod, scaled(fourier_tt(p, m.k, m.phase, false), m.amp));
    mod = tt_round(mod, kTol, 0);
    TT phi1 = tt_kron(tt_constant(p.bits[0], 1.0), tt_constant(p.bits[1], 1.0));
    f = tt_round(tt_hadamard(f, tt_kron(phi1, mod)), kTol, 0);
  }
  return f;
}

SubgridFields subgrid_fields(const Params& p, const TT* u3) {
  // Eq. FP0's closures on the sampled velocity: strain rates by periodic CFD2
  // differences, Smagorinsky diffusivity, LMSE mixing rate.
  const int K[3] = {p.bits[2], p.bits[3], p.bits[4]};
  const size_t M[3] = {(size_t)1 << K[0], (size_t)1 << K[1], (size_t)1 << K[2]};
  const size_t Mx = M[0] * M[1] * M[2];
  const double h[3] = {2.0 * kPi / (double)M[0], 2.0 * kPi / (double)M[1], 2.0 * kPi / (double)M[2]};
  std::vector<double> u[3];
  for (int i = 0; i < 3; ++i) u[i] = tt_dense(u3[i]);
  const size_t stride[3] = {M[1] * M[2], M[2], 1};
  auto neighbour = [&](size_t idx, int axis, int dir) {
    const size_t j = (idx / stride[axis]) % M[axis];
    const size_t jn = (j + M[axis] + (size_t)(dir + (int)M[axis])) % M[axis];
    return idx + (jn - j) * stride[axis];  // unsigned wrap-around is exact modulo 2^64
  };
  auto deriv = [&](const std::vector<double>& F, int axis, size_t idx) {
    return (F[neighbour(idx, axis, +1)] - F[neighbour(idx, axis, -1)]) / (2.0 * h[axis]);
  };
  SubgridFields out;
  out.delta = p.delta_cells * std::cbrt(h[0] * h[1] * h[2]);
  out.gamma.assign(Mx, p.gamma);
  out.omega.assign(Mx, 0.0);
  const double c = p.c_s * 0.5 * out.delta * out.delta;
  for (size_t idx = 0; idx < Mx; ++idx) {
    double s2 = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double sij = deriv(u[i], j, idx) + deriv(u[j], i, idx);
        s2 += sij * sij;
      }
    out.gamma[idx] += c * std::sqrt(s2);
    out.omega[idx] = p.c_omega * out.gamma[idx] / (out.delta * out.delta);
  }
  return out;
}

// Tolerance of the TT encodings of the subgrid fields (their ranks grow
// quickly below it; the fields then enter the dynamics at this level).
static const double kFieldTol = 1e-12;

// d/dx_dim [g d/dx_dim] in flux form (periodic): B diag(g_face) F with
// F = (S+ - I) / h, B = (I - S-) / h and g_face(x) = (g(x) + g(x + h e_dim)) / 2.
static TT flux_diffusion_op(const Params& p, const std::vector<double>& g, int dim) {
  const int K[3] = {p.bits[2], p.bits[3], p.bits[4]};
  const int Kx = K[0] + K[1] + K[2];
  const size_t M[3] = {(size_t)1 << K[0], (size_t)1 << K[1], (size_t)1 << K[2]};
  const size_t stride[3] = {M[1] * M[2], M[2], 1};
  std::vector<double> face(g.size());
  for (size_t idx = 0; idx < g.size(); ++idx) {
    const size_t j = (idx / stride[dim]) % M[dim];
    const size_t jn = (j + 1) % M[dim];
    face[idx] = 0.5 * (g[idx] + g[idx + (jn - j) * stride[dim]]);
  }
  const double hh = 2.0 * kPi / (double)M[dim];
  TT F = tt_add(op_shift(K[dim], +1, true), scaled(mpo_identity(K[dim]), -1.0));
  TT B = tt_add(mpo_identity(K[dim]), scaled(op_shift(K[dim], -1, true), -1.0));
  tt_scale(F, 1.0 / hh);
  tt_scale(B, 1.0 / hh);
  const TT diag = tt_kron(mpo_identity(p.bits[0] + p.bits[1]), mpo_diag(tt_from_vector(face, Kx, kFieldTol)));
  TT op = mpo_mul(embed_op(p, tt_round(B, kTol, 0), 2 + dim), tt_round(mpo_mul(diag, embed_op(p, tt_round(F, kTol, 0), 2 + dim)), kTol, 0));
  return tt_round(op, kTol, 0);
}

TT linear_operator(const Params& p, const TT* u3) {
  const int Kphi = p.bits[0] + p.bits[1];
  TT idphi = mpo_identity(Kphi);
  TT W;
  bool have = false;
  auto acc = [&](const TT& t) {
    W = have ? tt_round(tt_add(W, t), kTol, 0) : t;
    have = true;
  };
  SubgridFields sg;
  TT omega_x;
  if (p.sgs == 1) {
    sg = subgrid_fields(p, u3);
    omega_x = tt_from_vector(sg.omega, p.bits[2] + p.bits[3] + p.bits[4], kFieldTol);
  }
  // transport and diffusion in x (periodic CFD2; flux form with gamma(x) under sgs)
  for (int i = 0; i < 3; ++i) {
    const int K = p.bits[2 + i];
    const double h = 2.0 * kPi / (double)(1 << K);
    TT du = tt_kron(idphi, mpo_diag(u3[i]));
    TT adv = mpo_mul(du, embed_op(p, op_d1_periodic(K, h), 2 + i));
    tt_scale(adv, -1.0);
    acc(tt_round(adv, kTol, 0));
    if (p.sgs == 1)
      acc(flux_diffusion_op(p, sg.gamma, i));
    else if (p.gamma != 0.0)
      acc(scaled(embed_op(p, op_d2_periodic(K, h), 2 + i), p.gamma));
  }
  // composition drift (linear part) + reaction + artificial dissipation
  for (int a = 0; a < 2; ++a) {
    const int K = p.bits[a];
    const double h = 1.0 / (double)(1 << K);
    const double h12 = (1.0 / (double)(1 << p.bits[0])) * (1.0 / (double)(1 << p.bits[1]));
    TT dc;
    if (p.sgs == 1) {  // Omega_mix(x) phi_a + Da phi1 phi2
      TT ca = scaled(phi_weight(p, a == 0 ? 1 : 0, a == 1 ? 1 : 0), 1.0 / h12);  // phi_weight carries h1 h2
      TT cr = scaled(phi_weight(p, 1, 1), p.da / h12);
      dc = mpo_diag(tt_round(tt_add(tt_kron(ca, omega_x), tt_kron(cr, ones_x(p))), kTol, 0));
    } else {
      TT c = scaled(phi_weight(p, a == 0 ? 1 : 0, a == 1 ? 1 : 0), p.omega);
      c = tt_add(c, scaled(phi_weight(p, 1, 1), p.da));
      tt_scale(c, 1.0 / h12);  // phi_weight carries h1 h2
      c = tt_round(c, kTol, 0);
      dc = mpo_diag(tt_kron(c, ones_x(p)));
    }
    TT drift = mpo_mul(embed_op(p, op_d1_zero_sum(K, h), a), dc);
    acc(tt_round(drift, kTol, 0));
    if (p.d_phi != 0.0) acc(scaled(embed_op(p, op_d2_zero_sum(K, h), a), p.d_phi));
  }
  return W;
}

Model build_model(const Params& p) {
  Model m;
  m.N = p.N();
  m.off[0] = 0;
  for (int d = 0; d < 5; ++d) m.off[d + 1] = m.off[d] + p.bits[d];
  for (int i = 0; i < 3; ++i) m.u[i] = velocity_tt(p, i);
  m.f0 = initial_pdf(p);
  TT W = linear_operator(p, m.u);
  tt_scale(W, p.dt);
  m.op_lin = tt_round(tt_add(embed_op(p, mpo_identity(p.bits[0]), 0), W), kTol, 0);
  // phi part of the mixing drift -Omega d/dphi_a (<Phi_a> f): D1phi_a on
  // phi_a's sites, the open bond a = 0, 1 carries the choice of species.
  TT d1a = tt_kron(op_d1_zero_sum(p.bits[0], 1.0 / (double)(1 << p.bits[0])), mpo_identity(p.bits[1]));
  TT d1b = tt_kron(mpo_identity(p.bits[0]), op_d1_zero_sum(p.bits[1], 1.0 / (double)(1 << p.bits[1])));
  m.had_phi = tt_stack_right(d1a, d1b);
  // the mixing rate: the constant Omega here, or the field Omega_mix(x) as
  // the x factor of the mixing term (applied with the conditional means)
  tt_scale(m.had_phi, -p.dt * (p.sgs == 1 ? 1.0 : p.omega));
  if (p.sgs == 1)
    m.omega_x = tt_from_vector(subgrid_fields(p, m.u).omega, p.bits[2] + p.bits[3] + p.bits[4], kFieldTol);
  const int ex[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {0, 2}, {1, 1}};
  for (int w = 0; w < 6; ++w) m.wphi[w] = phi_weight(p, ex[w][0], ex[w][1]);
  return m;
}

// ------------------------------------------------------------- adjoint
TT mpo_transpose(const TT& op) {
  TT t = op;
  for (size_t n = 0; n < t.c.size(); ++n) {
    const int L = t.r[n], R = t.r[n + 1];
    for (int l = 0; l < L; ++l)
      for (int r = 0; r < R; ++r) std::swap(t.c[n][((size_t)l * 4 + 1) * R + r], t.c[n][((size_t)l * 4 + 2) * R + r]);
  }
  return t;
}

AdjointModel build_adjoint_model(const Params& p, const Model& m) {
  AdjointModel a;
  a.op_lin_t = mpo_transpose(m.op_lin);
  a.had_phi_t = mpo_transpose(m.had_phi);
  TT d1a = tt_kron(op_d1_zero_sum(p.bits[0], 1.0 / (double)(1 << p.bits[0])), mpo_identity(p.bits[1]));
  TT d1b = tt_kron(mpo_identity(p.bits[0]), op_d1_zero_sum(p.bits[1], 1.0 / (double)(1 << p.bits[1])));
  a.had_unit = tt_stack_right(d1a, d1b);
  tt_scale(a.had_unit, -1.0);
  a.c_stack = tt_stack_right(m.wphi[1], m.wphi[2]);
  const int Kphi = p.bits[0] + p.bits[1];
  TT idphi = mpo_identity(Kphi);
  const double h12 = (1.0 / (double)(1 << p.bits[0])) * (1.0 / (double)(1 << p.bits[1]));
  // dL/dOmega (linear part) = sum_a D1phi_a diag(phi_a); dL/dDa = sum_a D1phi_a diag(phi1 phi2)
  auto drift = [&](int e1a, int e2a, int e1b, int e2b) {
    TT out;
    for (int q = 0; q < 2; ++q) {
      const int K = p.bits[q];
      TT c = scaled(phi_weight(p, q == 0 ? e1a : e1b, q == 0 ? e2a : e2b), 1.0 / h12);
      TT op = mpo_mul(embed_op(p, op_d1_zero_sum(K, 1.0 / (double)(1 << K)), q), mpo_diag(tt_kron(c, ones_x(p))));
      out = q == 0 ? op : tt_add(out, op);
    }
    return tt_round(out, kTol, 0);
  };
  a.dL.push_back(drift(1, 0, 0, 1));
  a.dL.push_back(drift(1, 1, 1, 1));
  {
    TT g;
    for (int i = 0; i < 3; ++i) {
      const int K = p.bits[2 + i];
      TT d2 = embed_op(p, op_d2_periodic(K, 2.0 * kPi / (double)(1 << K)), 2 + i);
      g = i == 0 ? d2 : tt_add(g, d2);
    }
    a.dL.push_back(tt_round(g, kTol, 0));
  }
  for (const Mode& md : p.umodes) {  // dL/da_m = -sin(k_m . x + t_m) D1x_c
    const int K = p.bits[2 + md.comp];
    TT ds = tt_kron(idphi, mpo_diag(fourier_tt(p, md.k, md.phase, true)));
    TT op = mpo_mul(ds, embed_op(p, op_d1_periodic(K, 2.0 * kPi / (double)(1 << K)), 2 + md.comp));
    tt_scale(op, -1.0);
    a.dL.push_back(tt_round(op, kTol, 0));
  }
  a.dL_stack = a.dL[0];
  for (size_t i = 1; i < a.dL.size(); ++i) a.dL_stack = tt_stack_left(a.dL_stack, a.dL[i]);
  {
    Params p0 = p;
    p0.icmodes.clear();
    TT g = initial_pdf(p0);
    TT phi1 = tt_kron(tt_constant(p.bits[0], 1.0), tt_constant(p.bits[1], 1.0));
    for (const Mode& md : p.icmodes)
      a.dic.push_back(tt_round(tt_hadamard(g, tt_kron(phi1, fourier_tt(p, md.k, md.phase, false))), kTol, 0));
  }
  {
    TT w = tt_add(m.wphi[0], scaled(m.wphi[1], -1.0));
    w = tt_add(w, scaled(m.wphi[2], -1.0));
    const double nx = (double)(1LL << (p.bits[2] + p.bits[3] + p.bits[4]));
    a.lam_T = tt_round(tt_kron(w, ones_x(p)), kTol, 0);
    tt_scale(a.lam_T, 1.0 / nx);
  }
  return a;
}

}  // namespace qtt
