"""The backward of the simultaneous bond truncation in tensor-train form,
checked against the dense oracle (oracle.truncation.truncate_vjp).

This is the formulation a GPU pass would follow: X is held as left-orthonormal
cores Q_1 .. Q_{N-1} and right parts M_n (what the randomized range finder and
the zip-up leave, bonds r_n possibly above the rank), the cut projectors come
from the eigenpairs (V_n, lambda_n) of the right Grams M_n M_n^T, and the
cotangent Ybar is a tensor train.  With P_n = V_K V_K^T,

* left environments  e_n = P_n Q_n^T (e_{n-1} (x) Ybar_n)                (r_n x s_n)
* right environments R_{n-1} = sum_i Ybar_n[:, i, :] R_n (Q_n P_n)[:, i, :]^T,
  R_{N-1} = Ybar_N M_{N-1}^T                                            (s_n x r_n)
* per cut  g_n = (e_{n-1} (x) Ybar_n) R_n, Shat = Q_n^T g_n + g_n^T Q_n,
  A_n = V_K diag(F0) V_K^T, Gamma_n = V_D (F o V_D^T Shat V_K) V_K^T,
  delta_n = (I - Q_n Q_n^T) g_n A_n + Q_n (Gamma_n + Gamma_n^T),
  with F0_i = 1/lambda_i and F_ji = 1/(lambda_i - lambda_j) (or their
  Lorentzian broadenings),

and Xbar = Q_1 .. Q_{N-1} (e_{N-1} Ybar_N) + sum_n Q_1 .. Q_{n-1} delta_n M_n:
the fixed-projector part, the null-space term (range of X's left basis left
out) and the gap term inside that range, one core per cut.
"""
import numpy as np
import pytest

from oracle import truncation as tr


def _tt(V, N):
    """Cores (r_{n-1}, 2, r_n) of V by a QR sweep without truncation: the first
    N-1 are left-orthonormal, bonds min(2 r_{n-1}, 2^(N-n)) (above the rank
    when V is low-rank, like an oversampled range)."""
    cores, r, A = [], 1, np.asarray(V, dtype=np.float64).reshape(1, -1)
    for _ in range(N - 1):
        A = A.reshape(2 * r, -1)
        Q, R = np.linalg.qr(A)
        cores.append(Q.reshape(r, 2, -1))
        r, A = Q.shape[1], R
    cores.append(A.reshape(r, 2, 1))
    return cores


def _gaps(lk, ld, eps):
    diff = lk[None, :] - ld[:, None]
    return diff / (diff * diff + eps * eps) if eps > 0 else 1.0 / diff


def train_vjp(X, Ybar, N, chi, tol=0.0, eps=0.0):
    Qc = _tt(X, N)              # Q_1 .. Q_{N-1}, then the last core
    Yc = _tt(Ybar, N)           # any tensor train of the cotangent
    Qm = {n: Qc[n - 1].reshape(-1, Qc[n - 1].shape[2]) for n in range(1, N)}  # (2 r_{n-1}) x r_n
    # right parts M_n (r_n x 2^(N-n)) and the right Grams' eigenpairs
    M = {N - 1: Qc[N - 1].reshape(-1, 2)}
    for n in range(N - 2, 0, -1):
        M[n] = np.einsum("aib,bj->aij", Qc[n], M[n + 1]).reshape(Qc[n].shape[0], -1)
    V, lam, k = {}, {}, {}
    for n in range(1, N):
        w, U = np.linalg.eigh(M[n] @ M[n].T)
        lam[n], V[n] = w[::-1].copy(), U[:, ::-1].copy()
        s = np.sqrt(np.clip(lam[n], 0.0, None))
        k[n] = int(min(chi, np.count_nonzero(s > tol * s[0])))
    Pp = {n: V[n][:, : k[n]] @ V[n][:, : k[n]].T for n in range(1, N)}
    # left environments and the stacked (e_{n-1} (x) Ybar_n)
    e, Yhat = {0: np.ones((1, 1))}, {}
    for n in range(1, N):
        Yhat[n] = np.einsum("as,sib->aib", e[n - 1], Yc[n - 1]).reshape(-1, Yc[n - 1].shape[2])
        e[n] = Pp[n] @ Qm[n].T @ Yhat[n]
    # right environments against X's projected right part
    R = {N - 1: Yc[N - 1].reshape(-1, 2) @ M[N - 1].T}
    for n in range(N - 1, 1, -1):
        QP = (Qm[n] @ Pp[n]).reshape(-1, 2, Pp[n].shape[1])
        R[n - 1] = np.einsum("sit,tb,aib->sa", Yc[n - 1], R[n], QP)
    # dense assembly of the train: Q_{<=n} as 2^n x r_n
    Qle = {0: np.ones((1, 1))}
    for n in range(1, N):
        Qle[n] = np.einsum("Ra,aib->Rib", Qle[n - 1], Qc[n - 1]).reshape(2 ** n, -1)
    last = np.einsum("as,sib->aib", e[N - 1], Yc[N - 1]).reshape(-1, 2)
    Xbar = (Qle[N - 1] @ last).reshape(-1)
    for n in range(1, N):
        Qn, kk = Qm[n], k[n]
        g = Yhat[n] @ R[n]
        VK, VD, lk, ld = V[n][:, :kk], V[n][:, kk:], lam[n][:kk], lam[n][kk:]
        A = VK @ np.diag(_gaps(lk, np.zeros(1), eps)[0]) @ VK.T
        Sh = Qn.T @ g + g.T @ Qn
        Gam = VD @ (_gaps(lk, ld, eps) * (VD.T @ Sh @ VK)) @ VK.T
        delta = (np.eye(Qn.shape[0]) - Qn @ Qn.T) @ g @ A + Qn @ (Gam + Gam.T)
        left = np.einsum("Ra,aib->Rib", Qle[n - 1], delta.reshape(-1, 2, delta.shape[1])).reshape(2 ** n, -1)
        Xbar += (left @ M[n]).reshape(-1)
    return Xbar, k


def _random_tt(N, chi, rng):
    r = [min(2 ** n, 2 ** (N - n), chi) for n in range(N + 1)]
    T = np.ones((1, 1))
    for n in range(N):
        T = (T @ rng.standard_normal((r[n], 2, r[n + 1])).reshape(r[n], -1)).reshape(-1, r[n + 1])
    return T.reshape(-1)


@pytest.mark.parametrize("N,chi,eps", [(8, 3, 0.0), (8, 3, 1e-2), (10, 4, 0.0), (9, 6, 1e-3)])
def test_train_backward_equals_dense_backward(N, chi, eps):
    rng = np.random.default_rng(N * 10 + chi)
    X = rng.standard_normal(2 ** N)
    Yb = rng.standard_normal(2 ** N)
    lam1 = max(np.linalg.norm(tr.unfold(X, N, n), 2) ** 2 for n in range(1, N))
    g, k = train_vjp(X, Yb, N, chi, eps=eps * lam1)
    P = tr.projectors(X, N, chi)
    assert [k[n] for n in range(1, N)] == [P[n][1] for n in range(1, N)]
    d = tr.truncate_vjp(X, Yb, N, chi, eps=eps * lam1)
    assert np.abs(g - d).max() <= 1e-10 * np.abs(d).max()


@pytest.mark.parametrize("seed", [0, 1])
def test_train_backward_with_bonds_above_the_rank(seed):
    """X of TT rank 4 held with full QR bonds (noise eigenvalues in the right
    Grams, the in-range discarded set holding both truncated and null
    directions), chi = 3 truncating every rank-4 cut."""
    rng = np.random.default_rng(90 + seed)
    N, chi, tol = 9, 3, 1e-6
    X = _random_tt(N, 4, rng)
    Yb = rng.standard_normal(2 ** N)
    g, k = train_vjp(X, Yb, N, chi, tol)
    P = tr.projectors(X, N, chi, tol)
    assert [k[n] for n in range(1, N)] == [P[n][1] for n in range(1, N)] == [2, 3, 3, 3, 3, 3, 3, 2]
    d = tr.truncate_vjp(X, Yb, N, chi, tol)
    assert np.abs(g - d).max() <= 1e-9 * np.abs(d).max()
