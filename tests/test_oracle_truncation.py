"""CPU pins of oracle.truncation: the simultaneous truncation of every bond
and its exact backward, against what the mathematics fixes independently of
the module's formulas:

* central differences of the truncated map (generic tensors, several chi);
* for a tensor whose tensor-train ranks already equal the caps, the
  derivative is the orthogonal projection onto the tangent space of the
  fixed-rank manifold, written in the textbook form
      P_T = sum_k P<=(k-1) (x) I (x) P>=(k+1)  -  sum_k P<=k (x) P>=(k+1)
  with P<=k the projector onto the column space of the unfolding at cut k and
  P>=(k+1) the one onto its row space;
* T(X) = X where nothing is cut, T(T(X)) = T(X), and the single-cut case
  (two sites) equals the Eckart-Young best approximation;
* the Lorentzian broadening tends to the exact backward as eps -> 0.
"""
import numpy as np
import pytest

from oracle import truncation as tr


def _random_tt(N, chi, rng):
    """Dense vector of a random tensor train of bond min(2^n, 2^(N-n), chi)."""
    r = [min(2 ** n, 2 ** (N - n), chi) for n in range(N + 1)]
    T = np.ones((1, 1))
    for n in range(N):
        core = rng.standard_normal((r[n], 2, r[n + 1]))
        T = (T @ core.reshape(r[n], -1)).reshape(-1, r[n + 1])
    return T.reshape(-1)


@pytest.mark.parametrize("N,chi", [(6, 2), (8, 3), (8, 5)])
def test_vjp_matches_central_differences(N, chi):
    rng = np.random.default_rng(100 * N + chi)
    X = rng.standard_normal(2 ** N)
    Yb = rng.standard_normal(2 ** N)
    g = tr.truncate_vjp(X, Yb, N, chi)
    h = 1e-6
    for _ in range(4):
        D = rng.standard_normal(2 ** N)
        fd = (Yb @ tr.truncate(X + h * D, N, chi) - Yb @ tr.truncate(X - h * D, N, chi)) / (2 * h)
        assert abs(fd - g @ D) <= 1e-6 * max(abs(fd), 1.0), (fd, g @ D)


def _tangent_projection(X, Z, N):
    """P_T Z at X (tensor-train tangent space, dense), from the column and
    row spaces of X's unfoldings."""
    Uc, Vr = {0: np.ones((1, 1))}, {N: np.ones((1, 1))}
    for k in range(1, N):
        A = tr.unfold(X, N, k)
        u, s, vt = np.linalg.svd(A, full_matrices=False)
        r = int(np.count_nonzero(s > 1e-10 * s[0]))
        Uc[k], Vr[k] = u[:, :r], vt[:r].T

    def left(Y, k):  # P<=k on the first k sites
        if k == 0:
            return Y
        A = Y.reshape(2 ** k, -1)
        return (Uc[k] @ (Uc[k].T @ A)).reshape(-1)

    def right(Y, k):  # P>=k+1 on the last N-k sites
        if k == N:
            return Y
        A = Y.reshape(2 ** k, -1)
        return ((A @ Vr[k]) @ Vr[k].T).reshape(-1)

    out = np.zeros_like(Z)
    for k in range(1, N + 1):
        out += right(left(Z, k - 1), k)
    for k in range(1, N):
        out -= right(left(Z, k), k)
    return out


@pytest.mark.parametrize("N,chi", [(6, 2), (8, 3)])
def test_vjp_on_the_manifold_is_the_tangent_projection(N, chi):
    rng = np.random.default_rng(7 + N)
    X = _random_tt(N, chi, rng)
    for _ in range(3):
        Yb = rng.standard_normal(2 ** N)
        g = tr.truncate_vjp(X, Yb, N, chi)
        p = _tangent_projection(X, Yb, N)
        assert np.abs(g - p).max() <= 1e-9 * np.abs(p).max()


def test_truncate_identities():
    rng = np.random.default_rng(3)
    N = 8
    X = rng.standard_normal(2 ** N)
    # nothing cut: chi at least every unfolding's rank
    assert np.abs(tr.truncate(X, N, 2 ** (N // 2)) - X).max() <= 1e-12 * np.abs(X).max()
    # a tensor train of bond 3 is kept as it is at chi 3
    Xt = _random_tt(N, 3, rng)
    assert np.abs(tr.truncate(Xt, N, 3) - Xt).max() <= 1e-11 * np.abs(Xt).max()
    # idempotent
    Y = tr.truncate(X, N, 3)
    assert np.abs(tr.truncate(Y, N, 3) - Y).max() <= 1e-11 * np.abs(Y).max()
    # two sites: the best rank-1 approximation of the 2 x 2 matrix
    A = rng.standard_normal((2, 2))
    u, s, vt = np.linalg.svd(A)
    assert np.abs(tr.truncate(A.reshape(-1), 2, 1) - (s[0] * np.outer(u[:, 0], vt[0])).reshape(-1)).max() <= 1e-14


def test_lorentzian_broadening_tends_to_the_exact_backward():
    rng = np.random.default_rng(11)
    N, chi = 8, 3
    X = rng.standard_normal(2 ** N)
    Yb = rng.standard_normal(2 ** N)
    exact = tr.truncate_vjp(X, Yb, N, chi)
    lam1 = max(np.linalg.eigvalsh(tr.unfold(X, N, n) @ tr.unfold(X, N, n).T).max() for n in range(1, N))
    errs = [np.abs(tr.truncate_vjp(X, Yb, N, chi, eps=e * lam1) - exact).max() for e in (1e-2, 1e-4, 1e-6)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-6 * np.abs(exact).max()


@pytest.mark.parametrize("seed", [0, 1])
def test_vjp_at_frozen_rank_below_chi(seed):
    """A tensor train of bond 3 with chi = 5 and tol = 1e-4: the kept count at
    its rank-3 cuts is the rank, held by tol against the O(h) singular values a
    perturbation adds, and the backward runs through the null-space term alone
    there; central differences with h small against tol sigma_1 agree."""
    rng = np.random.default_rng(40 + seed)
    N, chi, tol = 8, 5, 1e-4
    X = _random_tt(N, 3, rng)
    P = tr.projectors(X, N, chi, tol)
    assert [P[n][1] for n in range(1, N)] == [2, 3, 3, 3, 3, 3, 2]
    for n in range(1, N):
        s = np.linalg.svd(tr.unfold(X, N, n), compute_uv=False)
        assert s[P[n][1] - 1] > 100 * tol * s[0]
    Yb = rng.standard_normal(2 ** N)
    g = tr.truncate_vjp(X, Yb, N, chi, tol)
    h = 1e-8 * np.abs(X).max()
    for _ in range(3):
        D = rng.standard_normal(2 ** N)
        fd = (Yb @ tr.truncate(X + h * D, N, chi, tol) - Yb @ tr.truncate(X - h * D, N, chi, tol)) / (2 * h)
        assert abs(fd - g @ D) <= 1e-5 * max(abs(fd), 1.0), (fd, g @ D)
    # tol = 0 keeps the numerical rank: rounding-level singular values are zeros
    P0 = tr.projectors(X, N, chi, 0.0)
    assert [P0[n][1] for n in range(1, N)] == [2, 3, 3, 3, 3, 3, 2]
    g0 = tr.truncate_vjp(X, Yb, N, chi, 0.0)
    assert np.abs(g0 - g).max() <= 1e-10 * np.abs(g).max()
