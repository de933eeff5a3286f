// Problem set-up for the Fokker-Planck PDF: grids, initial PDF, velocity and
// the operators of Eq. FP2 as trains (host, FP64, once per context).
#pragma once

#include <string>
#include <vector>

#include "host_tt.hpp"

namespace qtt {

struct Mode {
  int comp = 0;
  int k[3] = {0, 0, 0};
  double phase = 0, amp = 0;
};

struct Params {
  int bits[5] = {0, 0, 0, 0, 0};
  int chi_max = 0;
  double svd_rel_tol = 0;
  int precision = 0;
  int oversample = 8;
  int exact = 0;
  unsigned long long seed = 0;
  double omega = 0, da = 0, gamma = 0, d_phi = 0, dt = 0, shear_amp = 0;
  std::vector<Mode> umodes, icmodes;
  double ic_sigma = 0.05, ic_blend_width = 0.2;
  double ic_c_hi[2] = {1, 0}, ic_c_lo[2] = {0, 1};
  int rk_variant = 0;
  int flow = 0;        // 0: shear + seeded modes; 1: jet through a Taylor-Green vortex (Eq. velField)
  double u0 = 1.0;     // velocity scale of flow 1
  int ic_kind = 0;     // 0: tanh blend in x2; 1: Gaussian step function in x1 (Eq. initPDF), smoothed
  int sgs = 0;         // 1: gamma(x) = gamma + gamma_SGS(x) (Smagorinsky), Omega_mix(x) (LMSE)
  double c_s = 0.11, c_omega = 0.5, delta_cells = 3.0;
  int moment_ref = 0;  // 1: step the first-moment equation alongside (error measures)
  int N() const { return bits[0] + bits[1] + bits[2] + bits[3] + bits[4]; }
  int Kphi() const { return bits[0] + bits[1]; }
};

// Validates the parameters; returns an empty string or the reason.
std::string validate(const Params& p);

struct Model {
  int N = 0, off[6] = {0, 0, 0, 0, 0, 0};
  TT f0;        // initial PDF, rounded (right-canonical)
  TT op_lin;    // I + dt * W_lin over all N sites (d = 4)
  TT had_phi;   // -dt * Omega * [D1phi1 (+) D1phi2] over the phi sites, open right bond 2
  TT wphi[6];   // h1 h2 * {1, phi1, phi2, phi1^2, phi2^2, phi1 phi2} over the phi sites
  TT u[3];      // velocity components over the x sites (for checks)
  TT omega_x;   // sgs: Omega_mix(x) over the x sites (the mixing term's x factor); empty otherwise
};

// sgs: gamma(x) = gamma + gamma_SGS(x) and Omega_mix(x) on the x grid
// (x1 slowest), from the sampled velocity components.
struct SubgridFields {
  std::vector<double> gamma, omega;
  double delta = 0.0;
};
SubgridFields subgrid_fields(const Params& p, const TT* u3);

// Trains of the discrete adjoint of the Heun step (gradient of the mean
// product J = avg_x (<1> - <Phi_1> - <Phi_2>), Eqs. 2 and spaceAvg).
struct AdjointModel {
  TT op_lin_t;          // (I + dt W_lin)^T
  TT had_phi_t;         // had_phi with every core transposed (open right bond 2)
  TT had_unit;          // -[D1phi1 (+) D1phi2] (open right bond 2): d/dOmega of the mixing drift
  TT c_stack;           // h1 h2 [phi1 (+) phi2] over the phi sites (open right bond 2)
  std::vector<TT> dL;   // dL/dtheta (linear part) for Omega, Da, gamma, each velocity mode
  TT dL_stack;          // the dL stacked with an open left bond (one per parameter)
  std::vector<TT> dic;  // f0 without modulation times cos(q_m . x + p_m), each IC mode
  TT lam_T;             // dJ/df = (h1 h2 / n_x) (1 - phi1 - phi2)
};
AdjointModel build_adjoint_model(const Params& p, const Model& m);
TT mpo_transpose(const TT& op);

// Single-dimension building blocks (exposed for the host debug entry points).
TT op_shift(int K, int dir, bool periodic);   // (S f)_i = f_{i + dir}, dir = +1 / -1
TT op_d1_periodic(int K, double h);
TT op_d2_periodic(int K, double h);
TT op_d1_zero_sum(int K, double h);           // ghosts g_{-1} = -g_0, g_M = -g_{M-1}
TT op_d2_zero_sum(int K, double h);           // ghosts f_{-1} = f_0, f_M = f_{M-1}
TT embed_op(const Params& p, const TT& op, int dim);  // identity on the other dimensions
TT velocity_tt(const Params& p, int comp);    // over the 3 x dimensions
TT linear_operator(const Params& p, const TT* u3);    // W_lin of Eq. FP2 (no identity, no dt)
Model build_model(const Params& p);

}  // namespace qtt
