// Host tensor-train toolkit (see host_tt.hpp).
#include "host_tt.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace qtt {

// One-sided (Hestenes) Jacobi SVD of a column-rich copy.  For m >= n the
// columns of W = A are rotated until mutually orthogonal; W = U S, and the
// accumulated rotations give V.  For m < n the transpose is decomposed.
void svd_jacobi(int m, int n, const double* A, std::vector<double>& U, std::vector<double>& S,
                std::vector<double>& Vt) {
  if (m < n) {
    std::vector<double> At((size_t)n * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) At[(size_t)j * m + i] = A[(size_t)i * n + j];
    std::vector<double> U2, S2, Vt2;
    svd_jacobi(n, m, At.data(), U2, S2, Vt2);  // A^T = U2 S V2^T  =>  A = V2 S U2^T
    const int k = m;
    U.assign((size_t)m * k, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < k; ++j) U[(size_t)i * k + j] = Vt2[(size_t)j * m + i];
    S = S2;
    Vt.assign((size_t)k * n, 0.0);
    for (int j = 0; j < k; ++j)
      for (int c = 0; c < n; ++c) Vt[(size_t)j * n + c] = U2[(size_t)c * k + j];
    return;
  }
  const int k = n;
  // column-major working copies for cache-friendly column rotations
  std::vector<double> W((size_t)m * n), V((size_t)n * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A[(size_t)i * n + j];
  for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
  const double eps = 2.220446049250313e-16;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double* wp = &W[(size_t)p * m];
        double* wq = &W[(size_t)q * m];
        double a = 0, b = 0, g = 0;
        for (int i = 0; i < m; ++i) {
          a += wp[i] * wp[i];
          b += wq[i] * wq[i];
          g += wp[i] * wq[i];
        }
        if (g == 0.0 || std::fabs(g) <= eps * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < m; ++i) {
          const double x = wp[i], y = wq[i];
          wp[i] = c * x - s * y;
          wq[i] = s * x + c * y;
        }
        double* vp = &V[(size_t)p * n];
        double* vq = &V[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const double x = vp[i], y = vq[i];
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
      }
    }
    if (!rotated) break;
  }
  std::vector<double> sig(n);
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < m; ++i) s2 += W[(size_t)j * m + i] * W[(size_t)j * m + i];
    sig[j] = std::sqrt(s2);
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  U.assign((size_t)m * k, 0.0);
  S.assign(k, 0.0);
  Vt.assign((size_t)k * n, 0.0);
  for (int jj = 0; jj < k; ++jj) {
    const int j = order[jj];
    S[jj] = sig[j];
    if (sig[j] > 0)
      for (int i = 0; i < m; ++i) U[(size_t)i * k + jj] = W[(size_t)j * m + i] / sig[j];
    for (int i = 0; i < n; ++i) Vt[(size_t)jj * n + i] = V[(size_t)j * n + i];
  }
}

// Householder QR with the thin Q formed explicitly.
void qr_householder(int m, int n, const double* A, std::vector<double>& Q, std::vector<double>& R) {
  const int k = std::min(m, n);
  std::vector<double> W(A, A + (size_t)m * n);
  std::vector<double> tau(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double s = 0;
    for (int i = j + 1; i < m; ++i) s += W[(size_t)i * n + j] * W[(size_t)i * n + j];
    const double alpha = W[(size_t)j * n + j];
    if (s == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    const double mu = std::sqrt(alpha * alpha + s);
    const double beta = alpha <= 0 ? mu : -mu;
    const double v0 = alpha - beta;
    tau[j] = (beta - alpha) / beta;
    for (int i = j + 1; i < m; ++i) W[(size_t)i * n + j] /= v0;
    W[(size_t)j * n + j] = beta;
    for (int c = j + 1; c < n; ++c) {
      double dot = W[(size_t)j * n + c];
      for (int i = j + 1; i < m; ++i) dot += W[(size_t)i * n + j] * W[(size_t)i * n + c];
      dot *= tau[j];
      W[(size_t)j * n + c] -= dot;
      for (int i = j + 1; i < m; ++i) W[(size_t)i * n + c] -= dot * W[(size_t)i * n + j];
    }
  }
  R.assign((size_t)k * n, 0.0);
  for (int i = 0; i < k; ++i)
    for (int c = i; c < n; ++c) R[(size_t)i * n + c] = W[(size_t)i * n + c];
  Q.assign((size_t)m * k, 0.0);
  for (int i = 0; i < k; ++i) Q[(size_t)i * k + i] = 1.0;
  for (int j = k - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    for (int c = 0; c < k; ++c) {
      double dot = Q[(size_t)j * k + c];
      for (int i = j + 1; i < m; ++i) dot += W[(size_t)i * n + j] * Q[(size_t)i * k + c];
      dot *= tau[j];
      Q[(size_t)j * k + c] -= dot;
      for (int i = j + 1; i < m; ++i) Q[(size_t)i * k + c] -= dot * W[(size_t)i * n + j];
    }
  }
}

static int choose_rank(const std::vector<double>& S, double rel_tol, int max_rank) {
  int k = 0;
  const double s0 = S.empty() ? 0.0 : S[0];
  for (size_t i = 0; i < S.size(); ++i)
    if (S[i] > rel_tol * s0 && S[i] > 0.0) k = (int)i + 1;
  if (max_rank > 0) k = std::min(k, max_rank);
  return std::max(k, 1);
}

TT tt_from_vector(const std::vector<double>& v, int K, double rel_tol) {
  if ((size_t)1 << K != v.size()) throw std::runtime_error("tt_from_vector: size is not 2^K");
  TT t;
  t.d = 2;
  t.r.assign(K + 1, 1);
  t.c.resize(K);
  std::vector<double> rest = v;  // [r_left * 2^(K-n)]
  int rl = 1;
  for (int n = 0; n < K - 1; ++n) {
    const int rows = rl * 2, cols = (int)(rest.size() / rows);
    std::vector<double> U, S, Vt;
    svd_jacobi(rows, cols, rest.data(), U, S, Vt);
    const int kfull = (int)S.size();
    const int k = choose_rank(S, rel_tol, 0);
    t.r[n + 1] = k;
    t.c[n].assign((size_t)rows * k, 0.0);
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < k; ++j) t.c[n][(size_t)i * k + j] = U[(size_t)i * kfull + j];
    std::vector<double> nr((size_t)k * cols);
    for (int j = 0; j < k; ++j)
      for (int c = 0; c < cols; ++c) nr[(size_t)j * cols + c] = S[j] * Vt[(size_t)j * cols + c];
    rest.swap(nr);
    rl = k;
  }
  t.c[K - 1] = rest;  // [rl * 2]
  return t;
}

TT tt_constant(int K, double value) {
  TT t;
  t.d = 2;
  t.r.assign(K + 1, 1);
  t.c.assign(K, std::vector<double>{1.0, 1.0});
  t.c[0][0] = t.c[0][1] = value;
  return t;
}

TT tt_kron(const TT& a, const TT& b) {
  if (a.d != b.d) throw std::runtime_error("tt_kron: physical dimensions differ");
  if (a.r.back() != 1 || b.r.front() != 1) throw std::runtime_error("tt_kron: open boundary bonds");
  TT t;
  t.d = a.d;
  t.c = a.c;
  t.c.insert(t.c.end(), b.c.begin(), b.c.end());
  t.r = a.r;
  t.r.insert(t.r.end(), b.r.begin() + 1, b.r.end());
  return t;
}

static TT tt_direct_sum(const TT& a, const TT& b, bool open_right, bool open_left = false) {
  if (a.N() != b.N() || a.d != b.d) throw std::runtime_error("tt_add: shape mismatch");
  const int N = a.N(), d = a.d;
  TT t;
  t.d = d;
  t.r.resize(N + 1);
  t.c.resize(N);
  for (int n = 0; n <= N; ++n) t.r[n] = a.r[n] + b.r[n];
  if (!open_left) {
    t.r[0] = 1;
    if (a.r[0] != 1 || b.r[0] != 1) throw std::runtime_error("tt_add: left boundary must be 1");
  }
  if (!open_right) {
    if (a.r[N] != 1 || b.r[N] != 1) throw std::runtime_error("tt_add: right boundary must be 1");
    t.r[N] = 1;
  }
  for (int n = 0; n < N; ++n) {
    const int L = t.r[n], R = t.r[n + 1];
    t.c[n].assign((size_t)L * d * R, 0.0);
    const bool first = (n == 0) && !open_left, last = (n == N - 1) && !open_right;
    for (int which = 0; which < 2; ++which) {
      const TT& s = which ? b : a;
      const int l0 = first ? 0 : (which ? a.r[n] : 0);
      const int r0 = last ? 0 : (which ? a.r[n + 1] : 0);
      for (int x = 0; x < s.r[n]; ++x)
        for (int i = 0; i < d; ++i)
          for (int y = 0; y < s.r[n + 1]; ++y)
            t.c[n][((size_t)(l0 + x) * d + i) * R + (r0 + y)] += s.at(n, x, i, y);
    }
  }
  return t;
}

TT tt_add(const TT& a, const TT& b) { return tt_direct_sum(a, b, false); }
TT tt_stack_right(const TT& a, const TT& b) { return tt_direct_sum(a, b, true); }
TT tt_stack_left(const TT& a, const TT& b) { return tt_direct_sum(a, b, false, true); }

void tt_scale(TT& a, double s) {
  for (double& x : a.c[0]) x *= s;
}

TT tt_round(const TT& a, double rel_tol, int max_rank) {
  TT t = a;
  const int N = t.N(), d = t.d;
  // left-to-right orthogonalisation
  for (int n = 0; n < N - 1; ++n) {
    const int rows = t.r[n] * d, cols = t.r[n + 1];
    std::vector<double> Q, R;
    qr_householder(rows, cols, t.c[n].data(), Q, R);
    const int k = std::min(rows, cols);
    t.c[n] = Q;
    const int cols2 = d * t.r[n + 2];
    std::vector<double> nxt((size_t)k * cols2, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < cols; ++j) {
        const double rij = R[(size_t)i * cols + j];
        if (rij == 0.0) continue;
        const double* src = &t.c[n + 1][(size_t)j * cols2];
        double* dst = &nxt[(size_t)i * cols2];
        for (int c = 0; c < cols2; ++c) dst[c] += rij * src[c];
      }
    t.c[n + 1] = nxt;
    t.r[n + 1] = k;
  }
  // right-to-left truncation
  for (int n = N - 1; n >= 1; --n) {
    const int rows = t.r[n], cols = d * t.r[n + 1];
    std::vector<double> U, S, Vt;
    svd_jacobi(rows, cols, t.c[n].data(), U, S, Vt);
    const int kf = (int)S.size();
    const int k = choose_rank(S, rel_tol, max_rank);
    std::vector<double> core((size_t)k * cols);
    for (int i = 0; i < k; ++i)
      for (int c = 0; c < cols; ++c) core[(size_t)i * cols + c] = Vt[(size_t)i * cols + c];
    t.c[n] = core;
    // previous core times U_k S_k
    const int pr = t.r[n - 1] * d;
    std::vector<double> prev((size_t)pr * k, 0.0);
    for (int i = 0; i < pr; ++i)
      for (int j = 0; j < rows; ++j) {
        const double pij = t.c[n - 1][(size_t)i * rows + j];
        if (pij == 0.0) continue;
        for (int c = 0; c < k; ++c) prev[(size_t)i * k + c] += pij * U[(size_t)j * kf + c] * S[c];
      }
    t.c[n - 1] = prev;
    t.r[n] = k;
  }
  return t;
}

TT tt_hadamard(const TT& a, const TT& b) {
  if (a.N() != b.N() || a.d != 2 || b.d != 2) throw std::runtime_error("tt_hadamard: shape mismatch");
  TT t;
  t.d = 2;
  const int N = a.N();
  t.r.resize(N + 1);
  for (int n = 0; n <= N; ++n) t.r[n] = a.r[n] * b.r[n];
  t.c.resize(N);
  for (int n = 0; n < N; ++n) {
    t.c[n].assign((size_t)t.r[n] * 2 * t.r[n + 1], 0.0);
    for (int x = 0; x < a.r[n]; ++x)
      for (int y = 0; y < b.r[n]; ++y)
        for (int s = 0; s < 2; ++s)
          for (int x2 = 0; x2 < a.r[n + 1]; ++x2)
            for (int y2 = 0; y2 < b.r[n + 1]; ++y2)
              t.c[n][((size_t)(x * b.r[n] + y) * 2 + s) * t.r[n + 1] + (x2 * b.r[n + 1] + y2)] =
                  a.at(n, x, s, x2) * b.at(n, y, s, y2);
  }
  return t;
}

TT mpo_identity(int K) {
  TT t;
  t.d = 4;
  t.r.assign(K + 1, 1);
  t.c.assign(K, std::vector<double>{1.0, 0.0, 0.0, 1.0});
  return t;
}

TT mpo_diag(const TT& v) {
  TT t;
  t.d = 4;
  t.r = v.r;
  const int N = v.N();
  t.c.resize(N);
  for (int n = 0; n < N; ++n) {
    t.c[n].assign((size_t)v.r[n] * 4 * v.r[n + 1], 0.0);
    for (int x = 0; x < v.r[n]; ++x)
      for (int s = 0; s < 2; ++s)
        for (int y = 0; y < v.r[n + 1]; ++y) t.at(n, x, s * 2 + s, y) = v.at(n, x, s, y);
  }
  return t;
}

TT mpo_mul(const TT& A, const TT& B) {
  if (A.N() != B.N() || A.d != 4 || B.d != 4) throw std::runtime_error("mpo_mul: shape mismatch");
  const int N = A.N();
  TT t;
  t.d = 4;
  t.r.resize(N + 1);
  for (int n = 0; n <= N; ++n) t.r[n] = A.r[n] * B.r[n];
  t.c.resize(N);
  for (int n = 0; n < N; ++n) {
    t.c[n].assign((size_t)t.r[n] * 4 * t.r[n + 1], 0.0);
    for (int a = 0; a < A.r[n]; ++a)
      for (int b = 0; b < B.r[n]; ++b)
        for (int a2 = 0; a2 < A.r[n + 1]; ++a2)
          for (int b2 = 0; b2 < B.r[n + 1]; ++b2)
            for (int s = 0; s < 2; ++s)
              for (int s2 = 0; s2 < 2; ++s2) {
                double acc = 0;
                for (int sm = 0; sm < 2; ++sm) acc += A.at(n, a, s * 2 + sm, a2) * B.at(n, b, sm * 2 + s2, b2);
                t.at(n, a * B.r[n] + b, s * 2 + s2, a2 * B.r[n + 1] + b2) = acc;
              }
  }
  return t;
}

std::vector<double> tt_dense(const TT& a) {
  // left-to-right: rows = multi-index of processed sites, cols = open bond
  std::vector<double> cur{1.0};
  size_t rows = 1;
  int bond = 1;
  for (int n = 0; n < a.N(); ++n) {
    const int d = a.d, rn = a.r[n + 1];
    std::vector<double> nxt(rows * d * rn, 0.0);
    for (size_t i = 0; i < rows; ++i)
      for (int x = 0; x < bond; ++x) {
        const double v = cur[i * bond + x];
        if (v == 0.0) continue;
        for (int s = 0; s < d; ++s)
          for (int y = 0; y < rn; ++y) nxt[(i * d + s) * rn + y] += v * a.at(n, x, s, y);
      }
    cur.swap(nxt);
    rows *= d;
    bond = rn;
  }
  return cur;
}

double tt_norm(const TT& a) {
  // <a|a> via left environments
  std::vector<double> E{1.0};
  int b = 1;
  for (int n = 0; n < a.N(); ++n) {
    const int rn = a.r[n + 1];
    std::vector<double> F((size_t)rn * rn, 0.0);
    for (int x = 0; x < b; ++x)
      for (int y = 0; y < b; ++y) {
        const double e = E[(size_t)x * b + y];
        if (e == 0.0) continue;
        for (int s = 0; s < a.d; ++s)
          for (int p = 0; p < rn; ++p) {
            const double ap = a.at(n, x, s, p) * e;
            if (ap == 0.0) continue;
            for (int q = 0; q < rn; ++q) F[(size_t)p * rn + q] += ap * a.at(n, y, s, q);
          }
      }
    E.swap(F);
    b = rn;
  }
  return std::sqrt(std::max(E[0], 0.0));
}

}  // namespace qtt
