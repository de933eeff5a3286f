"""Pins for the CPU oracle: each check compares the oracle with something other
than itself (a Fourier-exact solution, a closed-form variance law, conservation
laws that follow from Eq. compBCs, the separate moment equation Eq. FPMoms,
characteristic solutions of the reaction drift, the paper's NVPP values).
A dropped term, a wrong sign or a wrong ghost rule in the oracle fails at
least one of them."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(bits, **kw):
    p = workload.make_params("small", **kw)
    p["bits"] = list(bits)
    if "dt" not in kw:
        ub = abs(p["shear_amp"]) + sum(abs(m["amp"]) for m in p["umodes"])
        p["dt"] = workload.cfl_dt(p["bits"], p["omega"], p["da"], p["gamma"], p["d_phi"], ub)
    return p


# ---------------------------------------------------------------- stencils (P2)
@pytest.mark.parametrize("M", [2, 4, 8, 16, 32])
def test_phi_stencils_zero_column_sums(M):
    """Eq. compBCs: the sum over the lattice of any discrete phi-derivative is zero."""
    h = 1.0 / M
    I = np.eye(M)
    D1 = np.stack([oracle.d1_zero_sum(I[:, j], 0, h) for j in range(M)], axis=1)
    D2 = np.stack([oracle.d2_zero_sum(I[:, j], 0, h) for j in range(M)], axis=1)
    assert np.abs(D1.sum(axis=0)).max() < 1e-12 * M
    assert np.abs(D2.sum(axis=0)).max() < 1e-12 * M * M
    # interior rows are the CFD2 stencils: exact on linear / quadratic data
    phi = (np.arange(M) + 0.5) * h
    if M >= 3:
        assert np.allclose((D1 @ phi)[1:-1], 1.0, atol=1e-12)
        assert np.allclose((D2 @ phi ** 2)[1:-1], 2.0, atol=1e-9)


def test_phi_stencil_ghost_values():
    """First derivative: antisymmetric ghosts make row 0 read (g1 + g0)/2h and the
    last row -(g_{M-1} + g_{M-2})/2h; second derivative: symmetric ghosts make
    the end rows one-sided differences (values fixed by Eq. compBCs)."""
    M, h = 8, 1.0 / 8
    rng = np.random.default_rng(1)
    g = rng.standard_normal(M)
    d1 = oracle.d1_zero_sum(g, 0, h)
    assert math.isclose(d1[0], (g[1] + g[0]) / (2 * h), rel_tol=1e-14)
    assert math.isclose(d1[-1], -(g[-1] + g[-2]) / (2 * h), rel_tol=1e-14)
    d2 = oracle.d2_zero_sum(g, 0, h)
    assert math.isclose(d2[0], (g[1] - g[0]) / h ** 2, rel_tol=1e-13)
    assert math.isclose(d2[-1], (g[-2] - g[-1]) / h ** 2, rel_tol=1e-13)


@pytest.mark.parametrize("M", [4, 16, 64])
def test_periodic_stencils_fourier_symbols(M):
    """On e^{ikx} the periodic CFD2 operators act as i sin(kh)/h and -2(1-cos kh)/h^2."""
    h = 2 * math.pi / M
    x = np.arange(M) * h
    for k in range(M):
        e = np.exp(1j * k * x)
        assert np.allclose(oracle.d1_periodic(e, 0, h), 1j * math.sin(k * h) / h * e, atol=1e-12)
        assert np.allclose(oracle.d2_periodic(e, 0, h), -2 * (1 - math.cos(k * h)) / h ** 2 * e, atol=1e-10)


# ------------------------------------------------------ Fourier-exact transport (P1)
@pytest.mark.parametrize("rk", [0, 1])
def test_constant_velocity_transport_is_fourier_exact(rk):
    """For constant u and gamma, each Fourier mode of the discrete solution is
    multiplied per step by R(dt*lam), R(z) = 1 + z + z^2/2 (every two-stage RK2),
    lam = sum_i [-i u_i sin(k_i h_i)/h_i - 2 gamma (1 - cos k_i h_i)/h_i^2]."""
    bits = [1, 1, 3, 4, 2]
    p = _params(bits, omega=0.0, da=0.0, d_phi=0.0, gamma=0.07, rk_variant=rk, dt=0.05)
    g = oracle.make_grid(bits)
    uc = [0.7, -0.3, 1.1]
    u = [np.full(g.M[2:], c) for c in uc]
    f0 = np.random.default_rng(3).standard_normal(g.shape)
    n = 9
    f = oracle.solve(p, n, f0=f0, u=u)
    F = np.fft.fftn(f0, axes=(2, 3, 4))
    lam = np.zeros(g.M[2:], dtype=complex)
    for i in range(3):
        k = np.fft.fftfreq(g.M[2 + i]) * g.M[2 + i]
        kh = k * g.h_x[i]
        sym = -1j * uc[i] * np.sin(kh) / g.h_x[i] - 2 * p["gamma"] * (1 - np.cos(kh)) / g.h_x[i] ** 2
        shape = [1, 1, 1]
        shape[i] = -1
        lam = lam + sym.reshape(shape)
    z = p["dt"] * lam
    R = 1 + z + z * z / 2
    ref = np.real(np.fft.ifftn(F * R[None, None] ** n, axes=(2, 3, 4)))
    assert np.abs(f - ref).max() < 1e-12 * np.abs(ref).max()


def test_gaussian_advection_diffusion_second_order():
    """Continuous check: a periodic Gaussian advected and diffused in x1 at
    constant speed; the error against the exact (image-summed) solution falls
    by ~4x per grid doubling (CFD2 in space, dt ~ h^2)."""
    errs = []
    for K in (5, 6, 7):
        bits = [1, 1, K, 1, 1]
        M = 2 ** K
        h = 2 * math.pi / M
        gam, c, s0, T = 0.05, 0.8, 0.4, 0.2
        nsteps = int(round(T / (0.05 * h * h / gam)))
        dt = T / nsteps
        p = _params(bits, omega=0.0, da=0.0, d_phi=0.0, gamma=gam, dt=dt)
        g = oracle.make_grid(bits)
        u = [np.full(g.M[2:], c), np.zeros(g.M[2:]), np.zeros(g.M[2:])]

        def exact(t):
            s2 = s0 * s0 + 2 * gam * t
            x = g.x[0]
            val = sum(np.exp(-(x - math.pi - c * t + 2 * math.pi * j) ** 2 / (2 * s2)) for j in range(-3, 4))
            return val * s0 / math.sqrt(s2)

        f0 = np.broadcast_to(exact(0.0)[None, None, :, None, None], g.shape).copy()
        f = oracle.solve(p, nsteps, f0=f0, u=u)
        errs.append(np.abs(f[0, 0, :, 0, 0] - exact(T)).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), (errs, orders)


# --------------------------------------------------------------- mass (P3)
def test_norm_conserved_pointwise_full_rhs():
    """<1>(x) stays 1 under the full operator (zero column sums in phi, D.1 = 0 in x)."""
    p = _params([4, 4, 3, 3, 3])
    g = oracle.make_grid(p["bits"])
    f = oracle.initial_pdf(p, g)
    o0 = oracle.observables(f, g)
    assert np.abs(o0["norm"] - 1).max() < 1e-13
    f = oracle.solve(p, 6)
    o = oracle.observables(f, g)
    assert np.abs(o["norm"] - 1).max() < 1e-12


# ------------------------------------------------ mixing + dissipation (P4)
@pytest.mark.parametrize("rk", [0, 1])
def test_variance_closed_form(rk):
    """Spatially uniform PDF, u = 0, Da = 0, interior Gaussian: the discrete
    variance obeys Var' = -2 Omega Var + 2 D_phi exactly, so under RK2
    Var_n - Var_inf = (1 - 2 Omega dt + 2 Omega^2 dt^2)^n (Var_0 - Var_inf),
    Var_inf = D_phi / Omega, and the mean stays put."""
    om, dphi = 1.3, 4e-3
    p = _params([6, 6, 1, 1, 1], omega=om, da=0.0, d_phi=dphi, gamma=0.0, shear_amp=0.0,
                umodes=[], ic_c_hi=[0.5, 0.45], ic_c_lo=[0.5, 0.45], rk_variant=rk)
    g = oracle.make_grid(p["bits"])
    f = oracle.initial_pdf(p, g)

    def stats(f):
        o = oracle.observables(f, g)
        return o["mean1_avg"], o["phi11_avg"] - o["mean1_avg"] ** 2, o["mean2_avg"], o["phi22_avg"] - o["mean2_avg"] ** 2

    m10, v10, m20, v20 = stats(f)
    n = 40
    f = oracle.solve(p, n, f0=f)
    m1, v1, m2, v2 = stats(f)
    dt = p["dt"]
    R = 1 - 2 * om * dt + 2 * om * om * dt * dt
    vinf = dphi / om
    assert abs(m1 - m10) < 1e-13 and abs(m2 - m20) < 1e-13
    assert abs(v1 - (vinf + (v10 - vinf) * R ** n)) < 1e-13
    assert abs(v2 - (vinf + (v20 - vinf) * R ** n)) < 1e-13
    assert abs(v1 - v10) > 1e-5  # the law is exercised, not trivially satisfied


# ------------------------------------ interior IC: means, species difference (P5-P7)
def _interior(**kw):
    return _params([5, 5, 3, 3, 3], ic_c_hi=[0.62, 0.4], ic_c_lo=[0.38, 0.6], **kw)


def test_initial_conditional_mean_follows_blend():
    """Interior Gaussians: <Phi_1>(x) = 0.62 w(x2) + 0.38 (1 - w(x2)) with the
    tanh blend (discrete Gaussian means are exact to e^{-2 pi^2 sigma^2/h^2})."""
    p = _interior()
    g = oracle.make_grid(p["bits"])
    o = oracle.observables(oracle.initial_pdf(p, g), g)
    w = 0.5 * (1 + np.tanh((g.x[1] - math.pi) / 0.2))
    exp1 = 0.62 * w + 0.38 * (1 - w)
    assert np.abs(o["mean1"] - exp1[None, :, None]).max() < 1e-12


def test_velocity_divergence_free():
    p = _params([1, 1, 4, 4, 4])
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    div = sum(oracle.d1_periodic(u[i], i, g.h_x[i]) for i in range(3))
    assert np.abs(div).max() < 1e-13
    assert np.abs(u[0]).max() > 0.5


def test_moment_equation_da0():
    """Da = 0: <Phi_a>(x, t) of the 5-D scheme equals the 3-D RK2-CFD2 solution of
    Eq. FPMoms started from <Phi_a>(x, 0); the spatial means are conserved."""
    p = _interior(da=0.0)
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    f = oracle.initial_pdf(p, g)
    m1, m2 = oracle.conditional_means(f, g)
    o0 = oracle.observables(f, g)
    n = 8
    for _ in range(n):
        f = oracle.rk2_step(f, g, u, p)
        m1 = oracle.moment_step(m1, g, u, p)
        m2 = oracle.moment_step(m2, g, u, p)
    f1, f2 = oracle.conditional_means(f, g)
    assert np.abs(f1 - m1).max() < 1e-12
    assert np.abs(f2 - m2).max() < 1e-12
    o = oracle.observables(f, g)
    assert abs(o["mean1_avg"] - o0["mean1_avg"]) < 1e-13
    assert np.abs(m1 - oracle.conditional_means(oracle.initial_pdf(p, g), g)[0]).max() > 1e-4


def test_species_difference_follows_moment_equation():
    """Da > 0: S_1 = S_2, so <Phi_1> - <Phi_2> obeys the linear moment equation
    point-wise, and its space average is conserved (paper: the difference in
    consumption must stay zero for symmetric initial data)."""
    p = _interior(da=1.5)
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    f = oracle.initial_pdf(p, g)
    a, b = oracle.conditional_means(f, g)
    d = a - b
    o0 = oracle.observables(f, g)
    for _ in range(8):
        f = oracle.rk2_step(f, g, u, p)
        d = oracle.moment_step(d, g, u, p)
    a, b = oracle.conditional_means(f, g)
    assert np.abs((a - b) - d).max() < 1e-12
    o = oracle.observables(f, g)
    assert abs((o["mean1_avg"] - o["mean2_avg"]) - (o0["mean1_avg"] - o0["mean2_avg"])) < 1e-13
    assert o["mean1_avg"] < o0["mean1_avg"] - 1e-4  # reaction consumes


def test_reaction_characteristic_logistic():
    """u = 0, Omega = 0: a narrow PDF moves along the characteristic of
    phi_a' = S_a = -Da phi1 phi2, i.e. phi1 - phi2 = c and
    phi1(t) = c / (1 + (c/phi1_0 - 1) exp(-Da c t)); mean error O(sigma^2 Da t)."""
    da, T = 1.0, 0.5
    p = _params([7, 7, 1, 1, 1], omega=0.0, da=da, d_phi=0.0, gamma=0.0, shear_amp=0.0, umodes=[],
                ic_sigma=0.015, ic_c_hi=[0.6, 0.35], ic_c_lo=[0.6, 0.35])
    n = int(math.ceil(T / p["dt"]))
    p["dt"] = T / n
    g = oracle.make_grid(p["bits"])
    f0 = oracle.initial_pdf(p, g)
    o0 = oracle.observables(f0, g)
    f = oracle.solve(p, n, f0=f0)
    o = oracle.observables(f, g)
    a0, b0 = o0["mean1_avg"], o0["mean2_avg"]
    c = a0 - b0
    a_ex = c / (1 + (c / a0 - 1) * math.exp(-da * c * T))
    assert abs(o["mean1_avg"] - a_ex) < 1e-3
    assert abs((o["mean1_avg"] - o["mean2_avg"]) - c) < 1e-12
    assert o["mean1_avg"] < a0 - 0.05


# --------------------------------------------------------------------- NVPP (P8)
def test_nvpp_paper_values():
    with open(os.path.join(GOLDEN, "nvpp.json")) as fh:
        gold = json.load(fh)
    for case in gold["maximal"]:
        assert oracle.nvpp(case["N"], case["chi"]) == case["nvpp"] == 2 ** case["N"]
    o = {c.get("fraction_order", c.get("reduction_order")): c for c in gold["orders"]}
    frac = oracle.nvpp(35, 128) / 2 ** 35
    assert round(math.log10(frac)) == o[-5]["fraction_order"]
    red = 2 ** 35 / oracle.nvpp(35, 32)
    assert round(math.log10(red)) == o[6]["reduction_order"]


def test_nvpp_brute_force_small():
    """Brute force: count the entries of an MPS with the profile p(n) minus the
    gauge dimension sum p(n)^2, for tiny chains."""
    for N in range(1, 9):
        for chi in (1, 2, 3, 4, 8, 16):
            p = oracle.bond_profile(N, chi)
            entries = sum(p[n] * 2 * p[n + 1] for n in range(N))
            gauge = sum(p[n] ** 2 for n in range(1, N))
            assert oracle.nvpp(N, chi) == entries - gauge


# ---- the paper's own flow case (Materials and Methods, Flow case definition)
def _paper_case(bits, **kw):
    p = workload.make_paper_params(**kw)
    p["bits"] = list(bits)
    return p


def test_paper_velocity_values_and_divergence():
    """Eq. velField on [0, 2 pi)^3 (k = 2): u2 peaks at u0 where
    sin(2 x1) = cos(2 x2) = sin(2 x3) = 1, u3 reaches -2 u0 where
    sin(2 x1) = sin(2 x2) = cos(2 x3) = 1, and on the jet axis x2 = x3 = pi the
    vortex term of u1 vanishes so u1 = -u0; the discrete divergence is zero
    (the CFD2 symbols of the three cosine/sine factors cancel, 1 + 1 - 2 = 0)."""
    p = _paper_case([2, 2, 4, 4, 4], u0=1.3)
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    q = g.M[2] // 8  # index of pi / 4
    assert abs(u[1][q, 0, q] - 1.3) < 1e-12 and abs(np.abs(u[1]).max() - 1.3) < 1e-12
    assert abs(u[2][q, q, 0] + 2.6) < 1e-12 and abs(np.abs(u[2]).max() - 2.6) < 1e-12
    c = g.M[2] // 2  # index of pi
    assert np.abs(u[0][:, c, c] + 1.3).max() < 1e-12
    div = sum(oracle.d1_periodic(u[i], i, g.h_x[i]) for i in range(3))
    assert np.abs(div).max() < 1e-12


def test_paper_initial_pdf_mass_and_mirror_symmetry():
    """Eq. initPDF: <1>(x) = 1 everywhere; the two Gaussians are mirror images
    under phi1 <-> phi2 and the band weight satisfies w(pi) = 1 - w(0), so
    <Phi_1>(x1 = pi) = <Phi_2>(x1 = 0) and the band centre carries the inner
    Gaussian (<Phi_1> > 1/2 there)."""
    p = _paper_case([5, 5, 4, 3, 3])
    g = oracle.make_grid(p["bits"])
    o = oracle.observables(oracle.initial_pdf(p, g), g)
    assert np.abs(o["norm"] - 1.0).max() < 1e-13
    c = g.M[2] // 2
    assert np.abs(o["mean1"][c] - o["mean2"][0]).max() < 1e-12
    assert np.abs(o["mean2"][c] - o["mean1"][0]).max() < 1e-12
    assert o["mean1"][c].min() > 0.7 and o["mean1"][0].max() < 0.3


def test_paper_velocity_moment_equation_da0():
    """Da = 0 with the paper's velocity (and the step-function blend in x1):
    <Phi_a>(x, t) of the 5-D scheme equals the RK2-CFD2 solution of Eq. FPMoms.
    The identity needs the composition-space mass to stay clear of the phi
    boundaries (the ghost rules add boundary terms to the first moment), so the
    Gaussians are the interior ones of the other moment pins."""
    p = _paper_case([5, 5, 3, 3, 3], da=0.0, ic_sigma=0.05, ic_c_hi=[0.62, 0.4], ic_c_lo=[0.38, 0.6])
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    f = oracle.initial_pdf(p, g)
    m1, m2 = oracle.conditional_means(f, g)
    for _ in range(6):
        f = oracle.rk2_step(f, g, u, p)
        m1 = oracle.moment_step(m1, g, u, p)
        m2 = oracle.moment_step(m2, g, u, p)
    f1, f2 = oracle.conditional_means(f, g)
    assert np.abs(f1 - m1).max() < 1e-12
    assert np.abs(f2 - m2).max() < 1e-12



def test_moving_gaussian_initial_pdf():
    """ic_kind 2: every x has <1>(x) = 1; with no centre modulation it is the
    separable corner Gaussian of ic_kind 0's construction at the same centre."""
    p = workload.make_params({"bits": 3, "chi_max": 8}, ic_kind=2, ic_sigma=0.1, ic_blend_width=0.2, ic_c_hi=[0.4, 0.6])
    g = oracle.make_grid(p["bits"])
    f = oracle.initial_pdf(p, g)
    norm = f.sum(axis=(0, 1)) * g.h_phi[0] * g.h_phi[1]
    assert np.max(np.abs(norm - 1.0)) < 1e-13
    p0 = dict(p, ic_blend_width=0.0)
    f0 = oracle.initial_pdf(p0, g)
    P1, P2 = np.meshgrid(g.phi[0], g.phi[1], indexing="ij")
    G = np.exp(-((P1 - 0.4) ** 2 + (P2 - 0.6) ** 2) / (2 * 0.1 ** 2))
    G = G / (G.sum() * g.h_phi[0] * g.h_phi[1])
    assert np.max(np.abs(f0 - G[:, :, None, None, None])) < 1e-12 * G.max()
    # the centre moves: the conditional mean of phi1 follows c1 = 0.4 + 0.2 sin(x1) cos(x2) away from the walls
    m1, _ = oracle.conditional_means(f, g)
    X1, X2, _ = np.meshgrid(*g.x, indexing="ij")
    c1 = 0.4 + 0.2 * np.sin(X1) * np.cos(X2)
    assert np.max(np.abs(m1 - c1)) < 0.02


# ------------- integrated statistics (Eqs. spaceAvg, RACov, SGSCov), closed forms
def _blend_pdf_params(**kw):
    return _params([5, 5, 2, 4, 2], ic_c_hi=[0.62, 0.41], ic_c_lo=[0.35, 0.58], **kw)


def test_statistics_of_phi_separable_pdf():
    """f(phi1, phi2; x) = g1(phi1; x) g2(phi2; x) with each 1-D factor
    normalised on its phi grid: <1> = 1, <Phi_1 Phi_2>(x) = m1(x) m2(x) exactly,
    so Y12 = 0 and the space average of <Phi_1 Phi_2> is avg(m1 m2), with
    m_a(x) = h_a sum_i phi_i g_a(phi_i; x) taken from the 1-D factors alone.
    The centres move with x in step, so R12 = Cov_x(m1, m2) is far from zero
    (an R12 / Y12 mix-up or a dropped h_phi factor fails here)."""
    bits = [4, 5, 2, 3, 2]
    g = oracle.make_grid(bits)
    X1, X2, X3 = np.meshgrid(*g.x, indexing="ij")
    c1 = 0.5 + 0.2 * np.sin(X2) * np.cos(X1)
    c2 = 0.45 + 0.15 * np.sin(X2) * np.cos(X1) + 0.05 * np.cos(X3)
    s1, s2 = 0.11, 0.07
    g1 = np.exp(-(g.phi[0][:, None, None, None] - c1[None]) ** 2 / (2 * s1 * s1))
    g2 = np.exp(-(g.phi[1][:, None, None, None] - c2[None]) ** 2 / (2 * s2 * s2))
    g1 /= g1.sum(axis=0, keepdims=True) * g.h_phi[0]
    g2 /= g2.sum(axis=0, keepdims=True) * g.h_phi[1]
    f = g1[:, None] * g2[None, :]
    m1 = g.h_phi[0] * (g.phi[0][:, None, None, None] * g1).sum(axis=0)
    m2 = g.h_phi[1] * (g.phi[1][:, None, None, None] * g2).sum(axis=0)
    o = oracle.observables(f, g)
    assert abs(o["norm_avg"] - 1.0) < 1e-14
    assert abs(o["Y12"]) < 1e-15
    assert abs(o["phi12_avg"] - float((m1 * m2).mean())) < 1e-14
    r12 = float((m1 * m2).mean() - m1.mean() * m2.mean())
    assert abs(o["R12"] - r12) < 1e-14
    assert r12 > 1e-3


def test_statistics_of_x_uniform_two_point_pdf():
    """A PDF that does not depend on x and puts weight 1/2 on each of the two
    cells (i1, i2) = (a1, a2) and (b1, b2): R12 = 0 (no spatial fluctuation of
    the means), and Y12 is the covariance of a two-point distribution,
    (phi1_a - phi1_b)(phi2_a - phi2_b) / 4; <Phi_1 Phi_2> is the mean of the
    two products."""
    bits = [3, 4, 2, 1, 2]
    g = oracle.make_grid(bits)
    a, b = (1, 12), (6, 3)
    f = np.zeros(g.shape)
    w = 0.5 / (g.h_phi[0] * g.h_phi[1])
    f[a[0], a[1]] = w
    f[b[0], b[1]] = w
    pa = (g.phi[0][a[0]], g.phi[1][a[1]])
    pb = (g.phi[0][b[0]], g.phi[1][b[1]])
    o = oracle.observables(f, g)
    assert abs(o["norm_avg"] - 1.0) < 1e-14
    assert abs(o["R12"]) < 1e-16
    assert abs(o["Y12"] - (pa[0] - pb[0]) * (pa[1] - pb[1]) / 4) < 1e-15
    assert abs(o["phi12_avg"] - (pa[0] * pa[1] + pb[0] * pb[1]) / 2) < 1e-15
    assert abs(o["phi11_avg"] - (pa[0] ** 2 + pb[0] ** 2) / 2) < 1e-15
    assert abs(o["Y12"]) > 0.05


def test_statistics_of_interior_tanh_blend():
    """f = w(x2) G_hi + (1 - w(x2)) G_lo with two interior Gaussians (centres
    c_hi, c_lo; uncorrelated, so E[phi1 phi2] = c1 c2 for each): with
    d_a = c_hi,a - c_lo,a the statistics follow from the blend weights alone,
      R12 = d1 d2 (avg(w^2) - avg(w)^2)          (Eq. RACov)
      Y12 = d1 d2 avg(w (1 - w))                 (Eq. SGSCov)
      avg <Phi_1 Phi_2> = avg(w) c_hi,1 c_hi,2 + (1 - avg(w)) c_lo,1 c_lo,2
      J = avg(<1 - phi1 - phi2>) = 1 - sum_a [avg(w) c_hi,a + (1 - avg(w)) c_lo,a]
    (discrete Gaussian moments are exact to e^{-2 pi^2 sigma^2 / h^2} and the
    wall truncation of the tails is below 1e-12)."""
    p = _blend_pdf_params()
    g = oracle.make_grid(p["bits"])
    o = oracle.observables(oracle.initial_pdf(p, g), g)
    w = 0.5 * (1 + np.tanh((g.x[1] - math.pi) / p["ic_blend_width"]))
    hi, lo = p["ic_c_hi"], p["ic_c_lo"]
    d1, d2 = hi[0] - lo[0], hi[1] - lo[1]
    aw, aw2 = float(w.mean()), float((w * w).mean())
    assert abs(o["R12"] - d1 * d2 * (aw2 - aw * aw)) < 1e-12
    assert abs(o["Y12"] - d1 * d2 * float((w * (1 - w)).mean())) < 1e-12
    assert abs(o["phi12_avg"] - (aw * hi[0] * hi[1] + (1 - aw) * lo[0] * lo[1])) < 1e-12
    assert abs(o["product_J"] - (1 - sum(aw * hi[k] + (1 - aw) * lo[k] for k in range(2)))) < 1e-12
    # both covariances are exercised (negative: the centres move in opposite directions)
    assert o["R12"] < -1e-2 and o["Y12"] < -5e-4 and abs(o["R12"] - o["Y12"]) > 1e-3


# ---------------- subgrid closures (Eq. FP0: Smagorinsky gamma_SGS, LMSE Omega_mix)
def _sgs_params(bits, **kw):
    base = dict(sgs=1, c_s=0.11, c_omega=0.5, delta_cells=3.0, gamma=2 * math.pi / 1e3, da=0.0)
    base.update(kw)
    return _paper_case(bits, **base)


def test_subgrid_constant_fields_reduce_to_constant_operator():
    """C_s = 0 makes gamma(x) = gamma and, with C_Omega = Omega Delta^2 / gamma,
    Omega_mix = Omega: the flux-form right-hand side then equals the one with
    constant coefficients (compact CFD2 diffusion, constant Omega)."""
    bits = [3, 3, 2, 3, 2]
    p = _sgs_params(bits, da=0.7)
    g = oracle.make_grid(bits)
    D = oracle.filter_width(p, g)
    p.update(c_s=0.0, c_omega=1.3 * D * D / p["gamma"])
    q = dict(p, sgs=0, omega=1.3)
    u = oracle.velocity_field(p, g)
    f = np.random.default_rng(4).standard_normal(g.shape)
    a, b = oracle.rhs(f, g, u, p), oracle.rhs(f, g, u, q)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_smagorinsky_field_of_shear_modes():
    """u1 = a sin(k x2 + t), u2 = b sin(q x1 + s): the only nonzero strain
    entries are S12 = S21 = d2 u1 + d1 u2, whose CFD2 value is
    a k_h cos(k x2 + t) + b q_h cos(q x1 + s) with k_h = sin(k h)/h, so
    gamma_SGS = C_s Delta^2 / 2 * sqrt(2) |S12| and Omega_mix = C_Omega
    (gamma + gamma_SGS) / Delta^2."""
    bits = [1, 1, 4, 5, 3]
    a, k, t, b, q, s = 0.3, 2, 0.4, -0.2, 3, 1.1
    p = _params(bits, shear_amp=0.0, umodes=[dict(comp=0, k=[0, k, 0], phase=t, amp=a),
                                             dict(comp=1, k=[q, 0, 0], phase=s, amp=b)],
                sgs=1, c_s=0.11, c_omega=0.5, delta_cells=3.0, gamma=0.004)
    g = oracle.make_grid(bits)
    u = oracle.velocity_field(p, g)
    gam, om = oracle.subgrid_fields(p, g, u)
    X1, X2, _ = np.meshgrid(*g.x, indexing="ij")
    s12 = (a * math.sin(k * g.h_x[1]) / g.h_x[1] * np.cos(k * X2 + t)
           + b * math.sin(q * g.h_x[0]) / g.h_x[0] * np.cos(q * X1 + s))
    D = 3.0 * (g.h_x[0] * g.h_x[1] * g.h_x[2]) ** (1 / 3)
    gam_ref = 0.004 + 0.11 * D * D / 2 * math.sqrt(2.0) * np.abs(s12)
    assert np.abs(gam - gam_ref).max() < 1e-14
    assert np.abs(om - 0.5 * gam_ref / (D * D)).max() < 1e-13
    assert np.abs(gam - 0.004).max() > 1e-3


def test_flux_diffusion_conservative_symmetric_and_compact():
    """The flux form d/dx[g df/dx] sums to zero over a periodic axis, is a
    symmetric operator for any g > 0, and equals g D2 for constant g."""
    rng = np.random.default_rng(8)
    M, h = 16, 2 * math.pi / 16
    gf = 1.0 + 0.5 * rng.random((M, 4, 2))
    a, b = rng.standard_normal((M, 4, 2)), rng.standard_normal((M, 4, 2))
    for ax in range(3):
        La = oracle.d2_flux_periodic(a, gf, ax, ax, h)
        Lb = oracle.d2_flux_periodic(b, gf, ax, ax, h)
        assert np.abs(La.sum(axis=ax)).max() < 1e-12
        assert abs(float((a * Lb).sum()) - float((La * b).sum())) < 1e-11 * float(np.abs(a * Lb).sum())
    c = oracle.d2_flux_periodic(a, np.full(gf.shape, 0.7), 0, 0, h)
    assert np.abs(c - 0.7 * oracle.d2_periodic(a, 0, h)).max() < 1e-12 * np.abs(c).max()


def test_subgrid_mixing_rate_acts_pointwise():
    """For an x-uniform PDF transport and diffusion vanish, so the right-hand
    side at each x is the composition-space operator with the constant
    Omega = Omega_mix(x) (and the same dissipation), as computed by the
    constant-coefficient path on a one-point x grid."""
    bits = [4, 4, 2, 2, 2]
    p = _sgs_params(bits, da=0.4, ic_kind=0, ic_c_hi=[0.6, 0.4], ic_c_lo=[0.6, 0.4])
    g = oracle.make_grid(bits)
    u = oracle.velocity_field(p, g)
    f = oracle.initial_pdf(p, g)
    _, om = oracle.subgrid_fields(p, g, u)
    assert np.ptp(om) > 1e-2
    r = oracle.rhs(f, g, u, p)
    g1 = oracle.make_grid([4, 4, 1, 1, 1])
    u0 = [np.zeros((2, 2, 2))] * 3
    for idx in [(0, 0, 0), (1, 2, 3), (3, 1, 2)]:
        q = dict(p, sgs=0, omega=float(om[idx]), bits=[4, 4, 1, 1, 1])
        f1 = np.broadcast_to(f[(slice(None), slice(None)) + idx][:, :, None, None, None], g1.shape).copy()
        r1 = oracle.rhs(f1, g1, u0, q)[:, :, 0, 0, 0]
        assert np.abs(r[(slice(None), slice(None)) + idx] - r1).max() < 1e-11 * np.abs(r1).max()


def test_subgrid_norm_and_moment_equation():
    """With gamma(x) and Omega_mix(x): <1>(x) stays 1 point-wise, and at Da = 0
    the conditional means follow the 3-D flux-form solution of Eq. FPMoms
    (interior Gaussians, so the phi walls add no boundary terms)."""
    bits = [5, 5, 3, 3, 3]
    p = _sgs_params(bits, ic_sigma=0.05, ic_c_hi=[0.62, 0.4], ic_c_lo=[0.38, 0.6])
    g = oracle.make_grid(bits)
    u = oracle.velocity_field(p, g)
    gam, om = oracle.subgrid_fields(p, g, u)
    p["dt"] = workload.cfl_dt(bits, float(om.max()), 0.0, float(gam.max()), p["d_phi"], workload.velocity_bound(p))
    f = oracle.initial_pdf(p, g)
    m1, m2 = oracle.conditional_means(f, g)
    m1_0 = m1.copy()
    for _ in range(6):
        f = oracle.rk2_step(f, g, u, p)
        m1 = oracle.moment_step(m1, g, u, p)
        m2 = oracle.moment_step(m2, g, u, p)
    o = oracle.observables(f, g)
    assert np.abs(o["norm"] - 1.0).max() < 1e-12
    # the Gaussians' tails at the phi walls (e^{-(0.38/0.05)^2/2} ~ 3e-13) enter
    # the boundary terms of the first moment each step
    assert np.abs(o["mean1"] - m1).max() < 5e-12 and np.abs(o["mean2"] - m2).max() < 5e-12
    assert np.abs(m1 - m1_0).max() > 1e-4
    # the field-diffusivity moment solution differs from the constant-gamma one
    mc = m1_0.copy()
    for _ in range(6):
        mc = oracle.moment_step(mc, g, u, dict(p, sgs=0))
    assert np.abs(mc - m1).max() > 1e-6


def test_error_measures_closed_forms():
    """Eqs. RMSE0 / RMSE1 on synthetic samples: constant offsets give the offsets
    back, exact = MPS gives zero, and a norm field 1 + d cos(x) gives |d|/sqrt(2)
    (space-time mean of d^2 cos^2)."""
    x = np.linspace(0, 2 * math.pi, 16, endpoint=False)
    fld = np.broadcast_to(x[:, None, None], (16, 2, 2))
    samples, exact = [], []
    for t in range(17):
        m1 = 0.5 + 0.01 * np.cos(fld)
        samples.append(dict(mean1_avg=0.53, mean2_avg=0.49, mean1=m1, mean2=1.0 - m1,
                            norm=1.0 + 0.02 * np.cos(fld)))
        exact.append((m1 - 0.003, 1.0 - m1 + 0.004))
    e = oracle.error_measures(samples, exact)
    assert abs(e["err_2b_up"] - math.sqrt(0.5 * (0.03 ** 2 + 0.01 ** 2))) < 1e-15
    assert abs(e["err_2b_down"] - math.sqrt(0.5 * (0.003 ** 2 + 0.004 ** 2))) < 1e-15
    assert abs(e["err_2c_up"] - 0.04) < 1e-15
    assert abs(e["err_2c_down"] - 0.02 / math.sqrt(2)) < 1e-15
    assert oracle.error_measures(samples, [(s["mean1"], s["mean2"]) for s in samples])["err_2b_down"] == 0.0


def test_flux_diffusion_second_order_for_smooth_coefficient():
    """Against the analytic d/dx[g f'] for g = 1 + sin(x)/2, f = cos(2x): the
    centred face averages make the flux form second order (error ~h^2); a
    one-sided or shifted face value would make it first order."""
    errs = []
    for M in (32, 64, 128):
        h = 2 * math.pi / M
        x = np.arange(M) * h
        g = 1 + 0.5 * np.sin(x)
        f = np.cos(2 * x)
        exact = -4 * np.cos(2 * x) * (1 + 0.5 * np.sin(x)) - np.sin(2 * x) * np.cos(x)
        errs.append(np.abs(oracle.d2_flux_periodic(f, g, 0, 0, h) - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < o < 2.1 for o in orders), (errs, orders)
