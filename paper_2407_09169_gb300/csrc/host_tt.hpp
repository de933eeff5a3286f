// Host-side tensor-train toolkit used once at initialisation: encoding of
// 1-D vectors as quantics tensor trains (TT-SVD), Kronecker products and sums
// of trains, operator (MPO) algebra and rounding.  All FP64; sizes are small
// (bonds of the analytic fields and operators are O(10)).
//
// Paper: "Matrix product state algorithm" -- vectors are MPSs and matrices
// are MPOs; "Computational complexity" -- initial states are prepared once
// at O(chi^3 d log M) cost.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

namespace qtt {

// A train of N cores; core n has shape [r[n]][d][r[n+1]] (row-major).
// d = 2 for vectors (MPS).  d = 4 for operators (MPO) with the physical index
// i = s_out * 2 + s_in.
struct TT {
  int d = 2;
  std::vector<int> r;                   // N + 1 bond dimensions
  std::vector<std::vector<double>> c;   // N cores
  int N() const { return (int)c.size(); }
  double& at(int n, int a, int i, int b) { return c[n][((size_t)a * d + i) * r[n + 1] + b]; }
  double at(int n, int a, int i, int b) const { return c[n][((size_t)a * d + i) * r[n + 1] + b]; }
};

// Dense helpers (row-major).
void svd_jacobi(int m, int n, const double* A, std::vector<double>& U, std::vector<double>& S,
                std::vector<double>& Vt);  // thin SVD, k = min(m, n), S descending
void qr_householder(int m, int n, const double* A, std::vector<double>& Q,
                    std::vector<double>& R);  // thin QR, Q m x k, R k x n, k = min(m, n)

TT tt_from_vector(const std::vector<double>& v, int K, double rel_tol);  // MSB-first TT-SVD
TT tt_constant(int K, double value);
TT tt_kron(const TT& a, const TT& b);
TT tt_add(const TT& a, const TT& b);
TT tt_stack_right(const TT& a, const TT& b);  // direct sum with an open right bond ra + rb
TT tt_stack_left(const TT& a, const TT& b);   // direct sum with an open left bond ra + rb (right ends summed)
void tt_scale(TT& a, double s);
TT tt_round(const TT& a, double rel_tol, int max_rank);  // drop sigma < rel_tol * sigma_1 per bond
TT tt_hadamard(const TT& a, const TT& b);
TT mpo_identity(int K);
TT mpo_diag(const TT& v);
TT mpo_mul(const TT& A, const TT& B);  // operator product A * B
std::vector<double> tt_dense(const TT& a);  // all d^N entries, site 0 most significant
double tt_norm(const TT& a);

// Tensor-train cross interpolation (cross.cpp) of F over N binary indices
// (bits[n] in {0, 1}, site 0 first): two-site sweeps with SVD rank selection
// (relative tolerance rel_tol, cap max_rank) and maximum-volume pivots, at
// most max_sweeps left-to-right sweeps, stopping when the relative error on
// 256 random samples is below 10 rel_tol.  The result is not rounded.
struct CrossStats {
  long long evaluations = 0;
  int sweeps = 0;
  double sample_rel_err = 0.0;
};
TT tt_cross(int N, const std::function<double(const uint8_t*)>& F, int max_rank, double rel_tol, int max_sweeps,
            uint64_t seed, CrossStats* stats);

}  // namespace qtt
