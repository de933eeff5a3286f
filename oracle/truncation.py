"""Dense oracle of the bond truncation and of its exact backward.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import or run this
module.  The product path never calls it, and the two share no code.

The paper limits every bond of the MPS to chi with the singular value
decomposition ("Matrix product state algorithm").  The reading taken here
(the same as the GPU path's) truncates all bonds at once: with X a tensor of
N binary sites stored as the vector X[i_1 ... i_N] (site 1 most significant),
X_(n) its unfolding at cut n (2^n rows, 2^(N-n) columns) and Pi_n the
orthogonal projector onto the k_n leading left singular vectors of X_(n)
(k_n = min(chi, #{sigma > tol sigma_1}), singular values at or below their
FP64 rounding counting as zero), acting on the first n sites,

    T(X) = Pi_1 Pi_2 ... Pi_{N-1} X          (Pi_{N-1} applied first).

Where the leading subspaces are separated from the rest (sigma_k > sigma_{k+1}
at every cut, and, where k_n is below chi, the rank held by tol against the
small singular values a perturbation creates) T is differentiable, and its
adjoint applied to a cotangent
Ybar (the vector-Jacobian product) is the sum of

* the part with the projectors held fixed: Pi_{N-1} ... Pi_1 Ybar;
* for every cut n, the part through Pi_n.  With G = X_(n) X_(n)^T = sum_i
  lambda_i u_i u_i^T (all 2^n eigenpairs, null space included), K the kept
  and D the other eigenvectors, the perturbation of a spectral projector
      dPi = sum_{i in K, j in D} (u_j^T dG u_i) (u_j u_i^T + u_i u_j^T) / (lambda_i - lambda_j)
  gives, with W = (Pi_{n-1} ... Pi_1 Ybar)_(n) (Pi_{n+1} ... Pi_{N-1} X)_(n)^T
  and S = W + W^T,
      Gbar = sum_{i in K, j in D} F_ij (u_j^T S u_i) u_j u_i^T,
      Xbar_(n) += (Gbar + Gbar^T) X_(n),
  F_ij = 1 / (lambda_i - lambda_j), or its Lorentzian broadening
  (lambda_i - lambda_j) / ((lambda_i - lambda_j)^2 + eps^2) that keeps the
  gaps finite where eigenvalues meet.

Plain numpy FP64; singular values and vectors by numpy.linalg.svd of each
unfolding, sizes kept small (tensors of up to ~2^12 entries).
"""
from __future__ import annotations

import numpy as np


def unfold(X, N: int, n: int):
    """X_(n): the 2^n x 2^(N-n) unfolding at cut n (row-major, site 1 first)."""
    return np.asarray(X, dtype=np.float64).reshape(2 ** n, 2 ** (N - n))


def _cut_eig(X, N: int, n: int):
    """All eigenpairs of X_(n) X_(n)^T in descending order, from the SVD of
    X_(n): the squared singular values padded with zeros, and the full set of
    left singular vectors (null space included); also the singular values."""
    A = unfold(X, N, n)
    U, s, _ = np.linalg.svd(A, full_matrices=True)
    lam = np.zeros(A.shape[0])
    lam[: s.size] = s * s
    return lam, U, s


def kept_count(sigma, chi: int, tol: float, shape) -> int:
    """min(chi, #{sigma_i > tol sigma_1}) for the singular values sigma of a
    matrix of the given shape; a singular value at or below its FP64 rounding,
    max(shape) * eps * sigma_1, is zero, so tol = 0 keeps the numerical rank."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0 or sigma[0] <= 0.0:
        return 0
    floor = max(shape) * np.finfo(np.float64).eps * sigma[0]
    resolved = sigma > floor
    return int(min(chi, np.count_nonzero(resolved & (sigma > tol * sigma[0]))))


def projectors(X, N: int, chi: int, tol: float = 0.0):
    """For every cut n = 1 .. N-1: (U_K, k_n, lam, U) of X_(n) -- the kept
    left singular vectors, their count and all eigenpairs of X_(n) X_(n)^T."""
    out = {}
    for n in range(1, N):
        lam, U, sigma = _cut_eig(X, N, n)
        k = kept_count(sigma, chi, tol, (2 ** n, 2 ** (N - n)))
        out[n] = (U[:, :k], k, lam, U)
    return out


def _apply(Y, N: int, n: int, UK):
    """Pi_n Y for the projector U_K U_K^T on the first n sites."""
    A = unfold(Y, N, n)
    return (UK @ (UK.T @ A)).reshape(-1)


def truncate(X, N: int, chi: int, tol: float = 0.0, proj=None):
    """T(X) = Pi_1 ... Pi_{N-1} X (the simultaneous truncation of every bond)."""
    P = projectors(X, N, chi, tol) if proj is None else proj
    Y = np.asarray(X, dtype=np.float64).reshape(-1).copy()
    for n in range(N - 1, 0, -1):
        Y = _apply(Y, N, n, P[n][0])
    return Y


def truncate_vjp(X, Ybar, N: int, chi: int, tol: float = 0.0, eps: float = 0.0):
    """(dT/dX)^T Ybar at X (module docstring); eps > 0 broadens the gaps."""
    X = np.asarray(X, dtype=np.float64).reshape(-1)
    Ybar = np.asarray(Ybar, dtype=np.float64).reshape(-1)
    P = projectors(X, N, chi, tol)
    # the cotangent pulled back through Pi_1 .. Pi_{n-1}, and X pushed through Pi_{N-1} .. Pi_{n+1}
    left = {1: Ybar.copy()}
    for n in range(1, N - 1):
        left[n + 1] = _apply(left[n], N, n, P[n][0])
    right = {N - 1: X.copy()}
    for n in range(N - 1, 1, -1):
        right[n - 1] = _apply(right[n], N, n, P[n][0])
    Xbar = _apply(left[N - 1], N, N - 1, P[N - 1][0])  # Pi_{N-1} ... Pi_1 Ybar
    for n in range(1, N):
        UK, k, lam, U = P[n]
        if k == U.shape[1]:
            continue  # Pi_n = I: no dependence
        W = unfold(left[n], N, n) @ unfold(right[n], N, n).T
        S = W + W.T
        lk, ld = lam[:k], lam[k:]
        diff = lk[None, :] - ld[:, None]  # [j in D, i in K]
        F = diff / (diff * diff + eps * eps) if eps > 0 else 1.0 / diff
        UD = U[:, k:]
        Gbar = UD @ (F * (UD.T @ S @ UK)) @ UK.T
        Xbar += ((Gbar + Gbar.T) @ unfold(X, N, n)).reshape(-1)
    return Xbar
