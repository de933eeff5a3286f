"""Host-side encodings of the library (initial PDF, velocity, finite-difference
MPOs, the full stage operator) against the oracle's dense constructions.
These run the library's host code only -- no GPU."""
import os
import re

import numpy as np
import pytest

import oracle
import workload

pkg = pytest.importorskip("paper_2407_09169_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_2407_09169_gb300 import build
    build.build()
    pkg.load_library()


def _params(bits, **kw):
    p = workload.make_params("small", **kw)
    p["bits"] = list(bits)
    return p


def _stencil_matrix(fn, M, h):
    I = np.eye(M)
    return np.stack([fn(I[:, j], 0, h) for j in range(M)], axis=1)


def test_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(pkg._binding.LIB_PATH)
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(qtt_\w+)\s*\(", txt, flags=re.M))
    assert {"qtt_init", "qtt_step", "qtt_observe", "qtt_compare", "qtt_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("bits", [[2, 3, 2, 3, 2], [4, 4, 3, 3, 3]])
def test_initial_pdf_encoding(bits):
    p = _params(bits)
    g = oracle.make_grid(bits)
    ref = oracle.initial_pdf(p, g).ravel()
    got = pkg.qtt_host_dense(p, 0, ref.size)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_initial_pdf_with_modulation():
    p = _params([2, 2, 3, 3, 2], icmodes=[dict(k=[1, 0, -1], phase=0.3, amp=0.2), dict(k=[0, 2, 1], phase=1.1, amp=-0.1)])
    g = oracle.make_grid(p["bits"])
    ref = oracle.initial_pdf(p, g).ravel()
    got = pkg.qtt_host_dense(p, 0, ref.size)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("bits,sigma,amp", [([3, 3, 3, 3, 3], 0.1, 0.2), ([4, 3, 3, 2, 3], 0.08, 0.25),
                                             ([3, 3, 3, 3, 3], 0.1, 0.0)])
def test_moving_gaussian_by_tensor_cross(bits, sigma, amp):
    """ic_kind 2 couples phi with x (the Gaussian's centre moves with x), so
    the library encodes it by tensor cross from point samples; the encoding
    must reproduce the oracle's dense array to the cross tolerance."""
    p = _params(bits, ic_kind=2, ic_sigma=sigma, ic_blend_width=amp, ic_c_hi=[0.45, 0.55])
    g = oracle.make_grid(bits)
    ref = oracle.initial_pdf(p, g).ravel()
    got = pkg.qtt_host_dense(p, 0, ref.size)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    ranks = pkg.qtt_host_dense(p, 41, sum(bits) + 1)
    print(f"\nbits {bits} sigma {sigma} amp {amp}: rel err {err:.2e}, max rank {int(ranks.max())}")
    assert err <= 1e-10
    if amp == 0.0:  # separable: rank 1 between the dimensions
        cuts = np.cumsum(bits)[:-1]
        assert all(int(ranks[c]) == 1 for c in cuts), ranks


def test_moving_gaussian_with_modulation():
    p = _params([3, 2, 3, 2, 2], ic_kind=2, ic_sigma=0.12, ic_blend_width=0.15, ic_c_hi=[0.5, 0.45],
                icmodes=[dict(k=[1, 0, -1], phase=0.3, amp=0.2), dict(k=[0, 2, 1], phase=1.1, amp=-0.1)])
    g = oracle.make_grid(p["bits"])
    ref = oracle.initial_pdf(p, g).ravel()
    got = pkg.qtt_host_dense(p, 0, ref.size)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_velocity_encoding():
    p = _params([1, 1, 4, 3, 5])
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    for i in range(3):
        got = pkg.qtt_host_dense(p, 1 + i, u[i].size)
        assert np.abs(got - u[i].ravel()).max() < 1e-12


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_derivative_mpos_match_stencils(K):
    p = _params([K] * 5)
    M = 2 ** K
    for d in range(5):
        if d < 2:
            h = 1.0 / M
            d1 = _stencil_matrix(oracle.d1_zero_sum, M, h)
            d2 = _stencil_matrix(oracle.d2_zero_sum, M, h)
        else:
            h = 2 * np.pi / M
            d1 = _stencil_matrix(oracle.d1_periodic, M, h)
            d2 = _stencil_matrix(oracle.d2_periodic, M, h)
        g1 = pkg.qtt_host_dense(p, 10 + d, M * M).reshape(M, M)
        g2 = pkg.qtt_host_dense(p, 20 + d, M * M).reshape(M, M)
        assert np.abs(g1 - d1).max() <= 1e-12 * max(1.0, np.abs(d1).max())
        assert np.abs(g2 - d2).max() <= 1e-12 * max(1.0, np.abs(d2).max())


@pytest.mark.parametrize("bits,da", [([2, 2, 2, 2, 2], 1.0), ([2, 3, 2, 1, 2], 0.7)])
def test_stage_operator_reproduces_oracle_euler_step(bits, da):
    """(I + dt W_lin) f - dt Omega sum_a D1phi_a(<Phi_a> f) == f + dt L(f) of the oracle,
    for a random PDF: pins every term, sign and coefficient of the operator assembly."""
    p = _params(bits, da=da, gamma=0.03, d_phi=0.01)
    g = oracle.make_grid(bits)
    u = oracle.velocity_field(p, g)
    rng = np.random.default_rng(7)
    f = rng.random(g.shape)
    ref = f + p["dt"] * oracle.rhs(f, g, u, p)
    n = f.size
    op = pkg.qtt_host_dense(p, 31, n * n).reshape(n, n)
    Mphi = g.M[0] * g.M[1]
    had = pkg.qtt_host_dense(p, 32, 2 * Mphi * Mphi).reshape(2, Mphi, Mphi)
    m1, m2 = oracle.conditional_means(f, g)
    fx = f.reshape(Mphi, -1)
    out = op @ f.ravel()
    for a, m in enumerate((m1, m2)):
        out += (had[a] @ (fx * m.ravel()[None, :])).ravel()
    assert np.linalg.norm(out - ref.ravel()) <= 1e-12 * np.linalg.norm(ref)


def _paper(bits, **kw):
    p = workload.make_paper_params(**kw)
    p["bits"] = list(bits)
    return p


def test_paper_flow_encodings():
    """The paper's flow case (Eq. velField velocity, Eq. initPDF initial PDF)
    against the oracle's dense fields."""
    p = _paper([3, 3, 4, 3, 3])
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    for i in range(3):
        got = pkg.qtt_host_dense(p, 1 + i, u[i].size)
        assert np.abs(got - u[i].ravel()).max() < 1e-12
    ref = oracle.initial_pdf(p, g).ravel()
    got = pkg.qtt_host_dense(p, 0, ref.size)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_paper_flow_stage_operator():
    p = _paper([2, 2, 2, 2, 2], da=0.8, gamma=0.03)
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    rng = np.random.default_rng(11)
    f = rng.random(g.shape)
    ref = f + p["dt"] * oracle.rhs(f, g, u, p)
    n = f.size
    op = pkg.qtt_host_dense(p, 31, n * n).reshape(n, n)
    Mphi = g.M[0] * g.M[1]
    had = pkg.qtt_host_dense(p, 32, 2 * Mphi * Mphi).reshape(2, Mphi, Mphi)
    m1, m2 = oracle.conditional_means(f, g)
    fx = f.reshape(Mphi, -1)
    out = op @ f.ravel()
    for a, m in enumerate((m1, m2)):
        out += (had[a] @ (fx * m.ravel()[None, :])).ravel()
    assert np.linalg.norm(out - ref.ravel()) <= 1e-12 * np.linalg.norm(ref)


def test_operator_bonds_are_small():
    p = workload.make_params("large")
    b = pkg.qtt_host_dense(p, 40, 64)
    assert b[0] == 1 and b[-1] == 1 and max(b) <= 64
    ic = pkg.qtt_host_dense(p, 41, 64)
    assert max(ic) <= 64


def test_invalid_params_are_rejected():
    p = _params([2, 2, 2, 2, 2])
    p["bits"][0] = 0
    with pytest.raises(pkg.QttError):
        pkg.qtt_host_dense(p, 0, 1 << 10)
    p = _params([2, 2, 2, 2, 2])
    p["umodes"] = [dict(comp=0, k=[1, 0, 0], phase=0.0, amp=0.1)]  # k_c != 0: not divergence-free
    with pytest.raises(pkg.QttError):
        pkg.qtt_host_dense(p, 1, 1 << 6)


def test_init_fails_loudly_without_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except Exception:
        pass
    with pytest.raises(pkg.QttError):
        pkg.qtt_init(_params([2, 2, 2, 2, 2]))


# ---------------- subgrid closures (Eq. FP0: Smagorinsky gamma_SGS(x), LMSE Omega_mix(x))
def _sgs(bits, **kw):
    base = dict(sgs=1, c_s=0.11, c_omega=0.5, delta_cells=3.0)
    base.update(kw)
    return _paper(bits, **base)


@pytest.mark.parametrize("bits,da", [([2, 2, 2, 2, 2], 0.0), ([2, 3, 2, 3, 2], 0.9)])
def test_subgrid_stage_operator_reproduces_oracle_euler_step(bits, da):
    """Under the subgrid closures the library's encodings -- the stage operator
    (flux-form diffusion with gamma(x), Omega_mix(x) phi_a in the linear
    drift), the composition-space factor -dt D1phi_a and the encoded
    Omega_mix(x) -- assemble f + dt L(f) of the oracle for a random PDF, and
    the encoded Omega_mix(x) equals the oracle's field."""
    p = _sgs(bits, da=da, d_phi=0.01)
    g = oracle.make_grid(bits)
    u = oracle.velocity_field(p, g)
    gam, om = oracle.subgrid_fields(p, g, u)
    om_lib = pkg.qtt_host_dense(p, 33, om.size)
    assert np.abs(om_lib - om.ravel()).max() <= 1e-11 * np.abs(om).max()
    assert np.ptp(gam) > 1e-3 * gam.max()
    rng = np.random.default_rng(9)
    f = rng.random(g.shape)
    ref = f + p["dt"] * oracle.rhs(f, g, u, p)
    n = f.size
    op = pkg.qtt_host_dense(p, 31, n * n).reshape(n, n)
    Mphi = g.M[0] * g.M[1]
    had = pkg.qtt_host_dense(p, 32, 2 * Mphi * Mphi).reshape(2, Mphi, Mphi)
    m1, m2 = oracle.conditional_means(f, g)
    fx = f.reshape(Mphi, -1)
    out = op @ f.ravel()
    for a, m in enumerate((m1, m2)):
        out += (had[a] @ (fx * (om_lib * m.ravel())[None, :])).ravel()
    assert np.linalg.norm(out - ref.ravel()) <= 1e-12 * np.linalg.norm(ref)


def test_subgrid_rejects_large_grids_and_bad_constants():
    p = _sgs([2, 2, 6, 6, 7])
    with pytest.raises(pkg.QttError):
        pkg.qtt_host_dense(p, 40, 64)
    p = _sgs([2, 2, 2, 2, 2], c_omega=-1.0)
    with pytest.raises(pkg.QttError):
        pkg.qtt_host_dense(p, 40, 64)
