// Tensor-train cross interpolation of a function of N binary indices
// (paper: initial states and fields can be prepared with the tensor-cross
// algorithm at O(chi^3 d log M) cost, "Computational complexity").
//
// Two-site cross with rank adaptation: the train is defined by nested left
// index sets I_k (multi-indices of sites 0..k-1) and right index sets J_k
// (sites k..N-1).  At the bond between sites k and k+1 the "superblock"
// A = F(I_k x {0,1}, {0,1} x J_{k+2}) (2|I_k| x 2|J_{k+2}| samples of F) is
// decomposed by an SVD; its numerical rank plus a few random orthonormal
// directions (relative tolerance, capped) sets the bond, and the maximum-volume rows of
// U and of V (maxvol of Goreinov et al.) become I_{k+1} and J_{k+1}.  Sweeps
// alternate left to right and right to left.  In a left-to-right sweep core
// k is U U[rows]^{-1}: it interpolates the superblock's column space through
// the chosen rows, so the train reproduces F on the pivots, and the last
// core holds F on I_{N-1} x {0,1}.  Its error is checked on random samples
// against F after every left-to-right sweep.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <random>
#include <stdexcept>

#include "host_tt.hpp"

namespace qtt {

namespace {

using Bits = std::vector<uint8_t>;

// Solves X P = B for X (B: m x r, P: r x r, row-major) by Gaussian
// elimination with partial pivoting on P^T.
std::vector<double> right_solve(const std::vector<double>& B, int m, const std::vector<double>& P, int r) {
  // P^T X^T = B^T: columns of X^T are the rows of X
  std::vector<double> A(r * r);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) A[i * r + j] = P[j * r + i];
  std::vector<double> Y(B.size());
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < r; ++j) Y[j * (size_t)m + i] = B[(size_t)i * r + j];  // Y = B^T (r x m)
  for (int c = 0; c < r; ++c) {
    int piv = c;
    for (int i = c + 1; i < r; ++i)
      if (std::fabs(A[i * r + c]) > std::fabs(A[piv * r + c])) piv = i;
    if (A[piv * r + c] == 0.0) throw std::runtime_error("EINVAL: tensor cross met a singular pivot matrix");
    if (piv != c) {
      for (int j = 0; j < r; ++j) std::swap(A[c * r + j], A[piv * r + j]);
      for (int j = 0; j < m; ++j) std::swap(Y[(size_t)c * m + j], Y[(size_t)piv * m + j]);
    }
    for (int i = c + 1; i < r; ++i) {
      const double f = A[i * r + c] / A[c * r + c];
      if (f == 0.0) continue;
      for (int j = c; j < r; ++j) A[i * r + j] -= f * A[c * r + j];
      for (int j = 0; j < m; ++j) Y[(size_t)i * m + j] -= f * Y[(size_t)c * m + j];
    }
  }
  for (int c = r - 1; c >= 0; --c) {
    for (int j = 0; j < m; ++j) {
      double v = Y[(size_t)c * m + j];
      for (int k = c + 1; k < r; ++k) v -= A[c * r + k] * Y[(size_t)k * m + j];
      Y[(size_t)c * m + j] = v / A[c * r + c];
    }
  }
  std::vector<double> X((size_t)m * r);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < r; ++j) X[(size_t)i * r + j] = Y[(size_t)j * m + i];
  return X;
}

// r rows of the m x r matrix U (m >= r) spanning a (locally) maximal-volume
// r x r submatrix: partial-pivoting elimination for a start, then row swaps
// while some entry of U U[rows]^{-1} exceeds 1 + 1e-2 in magnitude.
std::vector<int> maxvol(const std::vector<double>& U, int m, int r) {
  std::vector<int> rows;
  {
    std::vector<double> W = U;
    std::vector<char> used(m, 0);
    for (int c = 0; c < r; ++c) {
      int best = -1;
      double bv = -1.0;
      for (int i = 0; i < m; ++i)
        if (!used[i] && std::fabs(W[(size_t)i * r + c]) > bv) {
          bv = std::fabs(W[(size_t)i * r + c]);
          best = i;
        }
      used[best] = 1;
      rows.push_back(best);
      const double p = W[(size_t)best * r + c];
      if (p == 0.0) continue;
      for (int i = 0; i < m; ++i) {
        if (used[i]) continue;
        const double f = W[(size_t)i * r + c] / p;
        for (int j = c; j < r; ++j) W[(size_t)i * r + j] -= f * W[(size_t)best * r + j];
      }
    }
  }
  std::vector<double> P((size_t)r * r);
  for (int a = 0; a < r; ++a)
    for (int j = 0; j < r; ++j) P[(size_t)a * r + j] = U[(size_t)rows[a] * r + j];
  std::vector<double> B;
  try {
    B = right_solve(U, m, P, r);  // B = U P^{-1}, identity on the chosen rows
  } catch (const std::exception&) {
    return rows;  // rank-deficient start: keep the elimination's rows
  }
  for (int it = 0; it < 4 * m; ++it) {
    int bi = 0, bj = 0;
    double bv = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < r; ++j)
        if (std::fabs(B[(size_t)i * r + j]) > bv) {
          bv = std::fabs(B[(size_t)i * r + j]);
          bi = i;
          bj = j;
        }
    if (bv <= 1.01) break;
    // swap row bi in for rows[bj]: B <- B - B[:, bj] (B[bi, :] - e_bj) / B[bi, bj]
    const double piv = B[(size_t)bi * r + bj];
    std::vector<double> col(m), row(r);
    for (int i = 0; i < m; ++i) col[i] = B[(size_t)i * r + bj];
    for (int j = 0; j < r; ++j) row[j] = B[(size_t)bi * r + j] - (j == bj ? 1.0 : 0.0);
    for (int i = 0; i < m; ++i) {
      const double f = col[i] / piv;
      if (f == 0.0) continue;
      for (int j = 0; j < r; ++j) B[(size_t)i * r + j] -= f * row[j];
    }
    rows[bj] = bi;
  }
  return rows;
}

}  // namespace

TT tt_cross(int N, const std::function<double(const uint8_t*)>& F, int max_rank, double rel_tol, int max_sweeps,
            uint64_t seed, CrossStats* stats) {
  if (N < 2) throw std::runtime_error("EINVAL: tensor cross needs at least 2 sites");
  if (max_rank < 1) max_rank = 1;
  std::mt19937_64 rng(seed);
  std::vector<std::vector<Bits>> I(N + 1), J(N + 1);
  I[0] = {Bits{}};
  J[N] = {Bits{}};
  // nested random right sets to start
  for (int k = N - 1; k >= 1; --k) {
    std::vector<Bits> cand;
    for (int t = 0; t < 2; ++t)
      for (const Bits& b : J[k + 1]) {
        Bits c{(uint8_t)t};
        c.insert(c.end(), b.begin(), b.end());
        cand.push_back(c);
      }
    std::shuffle(cand.begin(), cand.end(), rng);
    cand.resize(std::min<size_t>(cand.size(), 4));
    J[k] = cand;
  }
  long long evals = 0;
  Bits buf(N);
  // superblock at bond k (sites k, k+1): rows (a, s) = a * 2 + s, cols (t, b) = t * |J_{k+2}| + b
  auto superblock = [&](int k, std::vector<double>& A, int& m, int& n) {
    const std::vector<Bits>& L = I[k];
    const std::vector<Bits>& R = J[k + 2];
    m = 2 * (int)L.size();
    n = 2 * (int)R.size();
    A.assign((size_t)m * n, 0.0);
    for (size_t a = 0; a < L.size(); ++a)
      for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t)
          for (size_t b = 0; b < R.size(); ++b) {
            std::copy(L[a].begin(), L[a].end(), buf.begin());
            buf[k] = (uint8_t)s;
            buf[k + 1] = (uint8_t)t;
            std::copy(R[b].begin(), R[b].end(), buf.begin() + k + 2);
            A[(a * 2 + s) * (size_t)n + t * R.size() + b] = F(buf.data());
            ++evals;
          }
  };
  // decompose a superblock: U and V of its leading singular directions (the
  // numerical rank), completed by a few random orthonormal directions, so
  // that the index sets can grow past a rank the current pivots underestimate
  constexpr int kKick = 4;
  std::normal_distribution<double> gauss(0.0, 1.0);
  auto complete = [&](std::vector<double>& Q, int rows_, int have, int want) {
    // columns have .. want-1 of the rows_ x want matrix Q: random, orthonormalised
    for (int j = have; j < want; ++j) {
      for (int i = 0; i < rows_; ++i) Q[(size_t)i * want + j] = gauss(rng);
      for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < j; ++c) {
          double d = 0.0;
          for (int i = 0; i < rows_; ++i) d += Q[(size_t)i * want + c] * Q[(size_t)i * want + j];
          for (int i = 0; i < rows_; ++i) Q[(size_t)i * want + j] -= d * Q[(size_t)i * want + c];
        }
      double nrm = 0.0;
      for (int i = 0; i < rows_; ++i) nrm += Q[(size_t)i * want + j] * Q[(size_t)i * want + j];
      nrm = std::sqrt(nrm);
      for (int i = 0; i < rows_; ++i) Q[(size_t)i * want + j] /= nrm;
    }
  };
  auto decompose = [&](const std::vector<double>& A, int m, int n, std::vector<double>& Ur, std::vector<double>& Vr) {
    std::vector<double> U, S, Vt;
    svd_jacobi(m, n, A.data(), U, S, Vt);
    const int kk = (int)S.size();
    int r0 = 0;  // directions above the tolerance (and above round-off, so that U and V hold them)
    while (r0 < kk && r0 < max_rank && S[r0] > std::max(rel_tol, 1e-14) * S[0] && S[0] > 0.0) ++r0;
    const int r = std::max(1, std::min({kk, r0 + kKick, max_rank}));
    Ur.assign((size_t)m * r, 0.0);
    Vr.assign((size_t)n * r, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < r0; ++j) Ur[(size_t)i * r + j] = U[(size_t)i * kk + j];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < r0; ++j) Vr[(size_t)i * r + j] = Vt[(size_t)j * n + i];
    complete(Ur, m, r0, r);
    complete(Vr, n, r0, r);
    return r;
  };
  auto set_left = [&](int k, const std::vector<int>& rows) {  // I_{k+1} from rows of I_k x {0,1}
    std::vector<Bits> out;
    for (int row : rows) {
      Bits b = I[k][row / 2];
      b.push_back((uint8_t)(row % 2));
      out.push_back(b);
    }
    I[k + 1] = out;
  };
  auto set_right = [&](int k, const std::vector<int>& cols) {  // J_{k+1} from cols of {0,1} x J_{k+2}
    const int nb = (int)J[k + 2].size();
    std::vector<Bits> out;
    for (int col : cols) {
      Bits b{(uint8_t)(col / nb)};
      b.insert(b.end(), J[k + 2][col % nb].begin(), J[k + 2][col % nb].end());
      out.push_back(b);
    }
    J[k + 1] = out;
  };

  TT t;
  double err = 0.0;
  int sweep = 0;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    // left to right: core_k = U (U[rows])^{-1} interpolates the superblock's
    // column space through the chosen rows, which become I_{k+1}
    t = TT();
    t.d = 2;
    t.r.assign(N + 1, 1);
    t.c.resize(N);
    std::vector<double> A, Ur, Vr;
    int m = 0, n = 0;
    for (int k = 0; k + 1 < N; ++k) {
      superblock(k, A, m, n);
      const int r = decompose(A, m, n, Ur, Vr);
      const std::vector<int> rows = maxvol(Ur, m, r);
      std::vector<double> P((size_t)r * r);
      for (int a = 0; a < r; ++a)
        for (int j = 0; j < r; ++j) P[(size_t)a * r + j] = Ur[(size_t)rows[a] * r + j];
      t.c[k] = right_solve(Ur, m, P, r);  // [(a, s)][j] = core [a][s][j]
      t.r[k + 1] = r;
      set_left(k, rows);
      set_right(k, maxvol(Vr, n, r));
      if (k + 2 == N) {  // last core: F(I_{N-1}, s) = rows of the superblock (J_N = {()})
        t.c[N - 1].assign((size_t)r * 2, 0.0);
        for (int a = 0; a < r; ++a)
          for (int s2 = 0; s2 < 2; ++s2) t.c[N - 1][(size_t)a * 2 + s2] = A[(size_t)rows[a] * n + s2];
      }
    }
    // error on random samples
    double emax = 0.0, fmax = 0.0;
    std::uniform_int_distribution<int> bit(0, 1);
    for (int q = 0; q < 256; ++q) {
      for (int i = 0; i < N; ++i) buf[i] = (uint8_t)bit(rng);
      const double fv = F(buf.data());
      ++evals;
      std::vector<double> v{1.0};
      for (int nn = 0; nn < N; ++nn) {
        const int r0 = t.r[nn], r1 = t.r[nn + 1];
        std::vector<double> w(r1, 0.0);
        for (int a = 0; a < r0; ++a)
          for (int b = 0; b < r1; ++b) w[b] += v[a] * t.at(nn, a, buf[nn], b);
        v.swap(w);
      }
      emax = std::max(emax, std::fabs(v[0] - fv));
      fmax = std::max(fmax, std::fabs(fv));
    }
    err = fmax > 0 ? emax / fmax : emax;
    if (err <= 10.0 * rel_tol || sweep == max_sweeps) break;
    // right to left: refresh the right sets
    for (int k = N - 2; k >= 0; --k) {
      superblock(k, A, m, n);
      const int r = decompose(A, m, n, Ur, Vr);
      set_right(k, maxvol(Vr, n, r));
    }
  }
  if (stats) {
    stats->evaluations = evals;
    stats->sweeps = sweep;
    stats->sample_rel_err = err;
  }
  return t;
}

}  // namespace qtt
