"""qtt_truncate_vjp (the backward of the simultaneous bond truncation on the
device) against the dense oracle backward (oracle.truncation.truncate_vjp),
element by element after contracting the returned train of bond 2 r_n; and
its argument checks, which fail before any device work (CPU)."""
import numpy as np
import pytest

import paper_2407_09169_gb300 as pkg
from paper_2407_09169_gb300 import _binding as B
from oracle import truncation as tr


def _random_cores(N, bond, rng):
    r = [min(2 ** n, 2 ** (N - n), bond) for n in range(N + 1)]
    return [rng.standard_normal((r[n], 2, r[n + 1])) for n in range(N)]


def _left_orthonormal(cores):
    """QR sweep over the cores (no truncation): the first N-1 become
    left-orthonormal, the bonds min(2 r_{n-1}, r_n)."""
    out, Rm = [], np.ones((1, 1))
    for c in cores[:-1]:
        c = np.einsum("ab,bic->aic", Rm, c)
        Q, Rm = np.linalg.qr(c.reshape(-1, c.shape[2]))
        out.append(Q.reshape(c.shape[0], 2, -1))
    out.append(np.einsum("ab,bic->aic", Rm, cores[-1]))
    return out


def _dense(cores):
    T = np.ones((1, 1))
    for c in cores:
        T = (T @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    return T.reshape(-1)


def _bonds(cores):
    return [c.shape[0] for c in cores] + [1]


def _bound(X, N, kept, eps=0.0):
    """Accuracy reachable from FP64 right Grams: the kept eigenvalues, and
    with them the weights 1 / lambda of the null-space term, carry a relative
    error of about eps64 * lambda_1 / lambda_k (the squared condition of the
    kept singular values; a broadening eps caps it at lambda_1 / eps), so the
    backward is compared to 1e-12 + 50 eps64 max_n lambda_1 / max(lambda_{k_n},
    eps), relative to its largest entry."""
    cond = 1.0
    for n in range(1, N):
        if kept[n - 1] > 0:
            sv = np.linalg.svd(tr.unfold(X, N, n), compute_uv=False)
            cond = max(cond, sv[0] ** 2 / max(sv[kept[n - 1] - 1] ** 2, eps))
    return 1e-12 + 50 * np.finfo(np.float64).eps * cond


def _dense_tt(X, N):
    """Cores of a dense tensor by a QR sweep (left-orthonormal, full bonds)."""
    cores, A, r = [], np.asarray(X).reshape(1, -1), 1
    for _ in range(N - 1):
        Q, R = np.linalg.qr(A.reshape(2 * r, -1))
        cores.append(Q.reshape(r, 2, -1))
        r, A = Q.shape[1], R
    cores.append(A.reshape(r, 2, 1))
    return cores


def _device_vjp(xc, yc, chi, tol, eps):
    torch = pytest.importorskip("torch")
    N = len(xc)
    rx, sy = _bonds(xc), _bonds(yc)
    ro = [1] + [2 * v for v in rx[1:-1]] + [1]
    cap = sum(ro[n] * 2 * ro[n + 1] for n in range(N))
    xd = torch.from_numpy(np.concatenate([c.ravel() for c in xc])).cuda()
    yd = torch.from_numpy(np.concatenate([c.ravel() for c in yc])).cuda()
    out = torch.full((cap,), float("nan"), dtype=torch.float64, device="cuda")
    written, kept = pkg.qtt_truncate_vjp(rx, xd, sy, yd, chi, tol, eps, out, cap)
    assert written == cap
    o = out.cpu().numpy()
    assert np.isfinite(o).all()
    cores, off = [], 0
    for n in range(N):
        sz = ro[n] * 2 * ro[n + 1]
        cores.append(o[off: off + sz].reshape(ro[n], 2, ro[n + 1]))
        off += sz
    return _dense(cores), kept


CASES = [  # N, bond of the random train (0: a dense random tensor), chi, eps relative to lambda_1
    (2, 2, 1, 0.0),
    (8, 16, 3, 0.0),
    (8, 16, 3, 1e-2),
    (10, 7, 5, 0.0),    # ragged bond 7
    (12, 40, 24, 0.0),  # ragged bond 40: 40 x 40 Grams, one merge of the divide and conquer
    (12, 40, 24, 1e-3),
    (12, 64, 16, 0.0),
    (12, 0, 24, 0.0),   # dense random tensor: bonds up to 64, well-conditioned cuts
    (11, 0, 20, 1e-4),
]


def _case(N, bond, chi):
    rng = np.random.default_rng(1000 * N + 10 * bond + chi)
    if bond == 0:
        xc = _dense_tt(rng.standard_normal(2 ** N), N)
    else:
        xc = _left_orthonormal(_random_cores(N, bond, rng))
    return xc, _random_cores(N, 5, rng)


@pytest.mark.gpu
@pytest.mark.parametrize("N,bond,chi,eps", CASES)
def test_truncate_vjp_matches_oracle(N, bond, chi, eps):
    xc, yc = _case(N, bond, chi)
    X, Yb = _dense(xc), _dense(yc)
    lam1 = max(np.linalg.norm(tr.unfold(X, N, n), 2) ** 2 for n in range(1, N))
    got, kept = _device_vjp(xc, yc, chi, 0.0, eps * lam1)
    P = tr.projectors(X, N, chi)
    assert kept == [P[n][1] for n in range(1, N)]
    ref = tr.truncate_vjp(X, Yb, N, chi, eps=eps * lam1)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    bound = _bound(X, N, kept, eps * lam1)
    print(f"N={N} bond={bond} chi={chi} eps={eps}: max rel {err:.2e} (bound {bound:.1e})")
    assert err <= bound


@pytest.mark.gpu
def test_truncate_vjp_bonds_above_the_rank():
    """X of TT rank 4 held at the bonds of a dense QR sweep (noise eigenvalues
    in the right Grams, removed by tol), chi = 3 cutting every rank-4 bond."""
    rng = np.random.default_rng(77)
    N, chi, tol = 9, 3, 1e-6
    X = _dense(_random_cores(N, 4, rng))
    cores = _dense_tt(X, N)
    assert max(_bonds(cores)) == 16
    yc = _random_cores(N, 3, rng)
    got, kept = _device_vjp(cores, yc, chi, tol, 0.0)
    P = tr.projectors(X, N, chi, tol)
    assert kept == [P[n][1] for n in range(1, N)] == [2, 3, 3, 3, 3, 3, 3, 2]
    ref = tr.truncate_vjp(X, _dense(yc), N, chi, tol)
    assert np.abs(got - ref).max() <= _bound(X, N, kept) * np.abs(ref).max()


@pytest.mark.gpu
def test_truncate_vjp_nothing_cut_is_the_identity():
    """chi above every bond of a full-rank X: T is the identity near X, so
    the backward returns the cotangent itself."""
    rng = np.random.default_rng(5)
    N = 8
    xc = _dense_tt(rng.standard_normal(2 ** N), N)
    yc = _random_cores(N, 4, rng)
    got, kept = _device_vjp(xc, yc, 64, 0.0, 0.0)
    assert kept == _bonds(xc)[1:-1]
    Yb = _dense(yc)
    bound = _bound(_dense(xc), N, kept)
    assert bound < 1e-9
    assert np.abs(got - Yb).max() <= bound * np.abs(Yb).max()


# argument checks: all fail before any device work, so they run without a GPU

def _call(rx, sy, chi=2, tol=0.0, eps=0.0, cap=10 ** 6):
    return pkg.qtt_truncate_vjp(rx, 16, sy, 16, chi, tol, eps, 16, cap)


@pytest.mark.parametrize("rx,sy,kw,msg", [
    ([1], [1], {}, "N must be"),
    ([2, 2, 1], [1, 2, 1], {}, "end bonds"),
    ([1, 2, 1], [1, 0, 1], {}, "below 1"),
    ([1, 2, 2048, 2, 1], [1, 2, 2, 2, 1], {}, "above 1024"),
    ([1, 2, 8, 2, 1], [1, 2, 2, 2, 1], {}, "left-orthonormal"),
    ([1, 2, 4, 2, 1], [1, 2, 2, 2, 1], {"chi": 0}, "chi"),
    ([1, 2, 4, 2, 1], [1, 2, 2, 2, 1], {"eps": -1.0}, "eps"),
    ([1, 2, 4, 2, 1], [1, 2, 2, 2, 1], {"tol": float("nan")}, "tol"),
    ([1, 2, 4, 2, 1], [1, 2, 2, 2, 1], {"cap": 10}, "are needed"),
])
def test_truncate_vjp_argument_checks(rx, sy, kw, msg):
    with pytest.raises(B.QttError) as ei:
        _call(rx, sy, **kw)
    assert ei.value.status == B.QTT_EINVAL
    assert msg in str(ei.value)
