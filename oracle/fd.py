"""Dense finite-difference oracle for the discretised Fokker-Planck equation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import or run this
module.  The product path (the CUDA library and its Python binding) never
calls it, and the two share no code.

What it computes (plain FP64 numpy, no blocking or fusion):

* The PDF f(phi1, phi2; x1, x2, x3) on the full tensor grid, stored as the
  row-major array ``f[i1, i2, j1, j2, j3]`` (paper: "Matrix product state
  encoding" fixes the dimension order phi1, phi2, x1, x2, x3).
* Grids (paper: "Finite-difference discretisation"): x_j = j * 2pi/M,
  periodic; phi_i = (i + 1/2)/M, cell-centred, so that the zero-sum ghost
  rules of Eq. compBCs put the wall half a cell outside the first and last
  nodes.
* Right-hand side of Eq. FP2 (the discretised Eq. FP0 with the artificial
  composition-space dissipation):
      L(f) = - sum_i u_i D1x_i f + gamma sum_i D2x_i f
             + sum_a D1phi_a [ (Omega (phi_a - <Phi_a>(x)) + Da phi1 phi2) f ]
             + D_phi sum_a D2phi_a f
  with S_1 = S_2 = -Da phi1 phi2, so that -d/dphi_a (S_a f) = +D1phi_a(Da phi1 phi2 f).
  D1/D2 are the second-order central differences (CFD2).  In x they are
  periodic.  In phi the ghost points follow Eq. compBCs: g_{-1} = -g_0,
  g_M = -g_{M-1} for a first derivative (applied to the drift flux g) and
  f_{-1} = f_0, f_M = f_{M-1} for the second derivative.
* The conditional mean <Phi_a>(x) = h_phi1 h_phi2 sum_{i1,i2} phi_a f
  (Eq. 2, unnormalised as printed).
* Explicit two-stage Runge-Kutta in time ("Finite-difference discretisation"):
  Heun  f* = f + dt L(f);  f_{n+1} = (f + f* + dt L(f*)) / 2   (default)
  midpoint  f_h = f + dt/2 L(f);  f_{n+1} = f + dt L(f_h)    (rk_variant 1)
* Integrated statistics (Eqs. spaceAvg, RACov, SGSCov) with the space average
  normalised by the domain volume, so that the mean of <1> is one.
* The subgrid closures of Eq. FP0 when params["sgs"] is 1: the Smagorinsky
  diffusivity gamma_SGS(x) = C_s Delta^2/2 sqrt(sum_ij (d_j u_i + d_i u_j)^2)
  (CFD2 derivatives of the sampled velocity) and the LMSE mixing rate
  Omega_mix(x) = C_Omega (gamma + gamma_SGS(x)) / Delta^2, with the filter
  width Delta = delta_cells (h1 h2 h3)^(1/3) (the paper: Delta = 3 l0 / M).
  The diffusion d/dx_i [(gamma + gamma_SGS) df/dx_i] of Eq. FP2 is then taken
  in flux form with face values averaged from the two neighbours,
  [g_{+}(f_{+} - f) - g_{-}(f - f_{-})] / h^2, which for a constant field is
  the CFD2 second difference used otherwise.
* The moment equation Eq. FPMoms for Da = 0 (a separate 3-D RK2-CFD2 solver),
  used as an independent check of the composition-space operators.
* The error measures of Eqs. RMSE0 and RMSE1 (time and space-time averages
  of squared differences over the stored time samples).
* The NVPP count of Eq. MPSdofs.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, Fourier-exact solutions, conservation laws, the moment
equation, brute-force sums and the paper's NVPP values).  The integrated
statistics of ``observables`` (<Phi_1 Phi_2>, R12 of Eq. RACov, Y12 of
Eq. SGSCov, J) are pinned by closed forms of a phi-separable PDF (Y12 = 0),
an x-uniform two-point PDF (R12 = 0, Y12 = the two-point covariance) and the
interior tanh blend (R12 and Y12 from the blend weights alone).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Grid", "make_grid", "velocity_field", "initial_pdf", "d1_periodic",
    "d2_periodic", "d1_zero_sum", "d2_zero_sum", "conditional_means", "rhs",
    "rk2_step", "solve", "observables", "moment_rhs", "moment_step", "nvpp",
    "bond_profile", "filter_width", "subgrid_fields", "d2_flux_periodic", "error_measures",
]


class Grid:
    """Tensor grid: bits per dimension in the order phi1, phi2, x1, x2, x3."""

    def __init__(self, bits):
        self.bits = [int(b) for b in bits]
        self.M = [2 ** b for b in self.bits]
        self.h_phi = [1.0 / m for m in self.M[:2]]
        self.h_x = [2.0 * math.pi / m for m in self.M[2:]]
        self.phi = [(np.arange(m) + 0.5) / m for m in self.M[:2]]
        self.x = [np.arange(m) * (2.0 * math.pi / m) for m in self.M[2:]]

    @property
    def shape(self):
        return tuple(self.M)


def make_grid(bits) -> Grid:
    return Grid(bits)


def velocity_field(params, grid: Grid):
    """flow 0: u_1 = shear_amp * tanh(x2 - pi); flow 1: the jet through a
    Taylor-Green vortex of Eq. velField on [0, l0)^3 with l0 = 2 pi and
    k = 4 pi / l0.  Then the seeded modes a * sin(k . x + theta) are added to
    component c."""
    X1, X2, X3 = np.meshgrid(*grid.x, indexing="ij")
    u = [np.zeros(grid.M[2:]), np.zeros(grid.M[2:]), np.zeros(grid.M[2:])]
    if params.get("flow", 0) == 1:
        u0, l0 = params.get("u0", 1.0), 2.0 * math.pi
        k = 4.0 * math.pi / l0
        jet = np.exp(-((X2 / l0 - 0.5) ** 2 + (X3 / l0 - 0.5) ** 2) / (2.0 * (1.0 / 6.0) ** 2))
        u[0] += u0 * (np.cos(k * X1) * np.sin(k * X2) * np.sin(k * X3) - jet)
        u[1] += u0 * np.sin(k * X1) * np.cos(k * X2) * np.sin(k * X3)
        u[2] += -2.0 * u0 * np.sin(k * X1) * np.sin(k * X2) * np.cos(k * X3)
    else:
        u[0] += params["shear_amp"] * np.tanh(X2 - math.pi)
    for m in params["umodes"]:
        k = m["k"]
        u[m["comp"]] += m["amp"] * np.sin(k[0] * X1 + k[1] * X2 + k[2] * X3 + m["phase"])
    return u


def _gaussian2(grid: Grid, centre, sigma):
    P1, P2 = np.meshgrid(grid.phi[0], grid.phi[1], indexing="ij")
    g = np.exp(-((P1 - centre[0]) ** 2 + (P2 - centre[1]) ** 2) / (2.0 * sigma * sigma))
    return g / (g.sum() * grid.h_phi[0] * grid.h_phi[1])


def _moving_gaussian(params, grid: Grid):
    """ic_kind 2: Gaussian in phi (std ic_sigma) centred at
    c1 = ic_c_hi[0] + A sin(x1) cos(x2), c2 = ic_c_hi[1] - A sin(x2 + x3),
    A = ic_blend_width, each 1-D factor normalised on the phi grid."""
    X1, X2, X3 = np.meshgrid(*grid.x, indexing="ij")
    A, s = params["ic_blend_width"], params["ic_sigma"]
    c1 = params["ic_c_hi"][0] + A * np.sin(X1) * np.cos(X2)
    c2 = params["ic_c_hi"][1] - A * np.sin(X2 + X3)
    g1 = np.exp(-(grid.phi[0][:, None, None, None] - c1[None]) ** 2 / (2 * s * s))
    g2 = np.exp(-(grid.phi[1][:, None, None, None] - c2[None]) ** 2 / (2 * s * s))
    g1 = g1 / (g1.sum(axis=0, keepdims=True) * grid.h_phi[0])
    g2 = g2 / (g2.sum(axis=0, keepdims=True) * grid.h_phi[1])
    f = g1[:, None] * g2[None, :]
    if params.get("icmodes"):
        mod = np.ones(grid.M[2:])
        for m in params["icmodes"]:
            q = m["k"]
            mod += m["amp"] * np.cos(q[0] * X1 + q[1] * X2 + q[2] * X3 + m["phase"])
        f = f * mod[None, None]
    return np.ascontiguousarray(f)


def initial_pdf(params, grid: Grid):
    """f0 = w G_hi(phi) + (1 - w) G_lo(phi), G normalised so that
    h_phi1 h_phi2 sum G = 1.  ic_kind 0: w(x2) = (1 + tanh((x2 - pi)/width))/2.
    ic_kind 1 (Eq. initPDF, smoothed): w(x1) = 1 on l0/4 <= x1 < 3 l0/4
    (l0 = 2 pi), with tanh edges of the given width.  Optionally multiplied
    by (1 + sum_m b_m cos(q_m . x + psi_m)).  ic_kind 2 (ours): see
    _moving_gaussian."""
    if params.get("ic_kind", 0) == 2:
        return _moving_gaussian(params, grid)
    g_hi = _gaussian2(grid, params["ic_c_hi"], params["ic_sigma"])
    g_lo = _gaussian2(grid, params["ic_c_lo"], params["ic_sigma"])
    width = params["ic_blend_width"]
    if params.get("ic_kind", 0) == 1:
        x1 = grid.x[0]
        w = 0.5 * (np.tanh((x1 - 0.5 * math.pi) / width) - np.tanh((x1 - 1.5 * math.pi) / width))
        wx = np.broadcast_to(w[:, None, None], grid.M[2:])
    else:
        w = 0.5 * (1.0 + np.tanh((grid.x[1] - math.pi) / width))
        wx = np.broadcast_to(w[None, :, None], grid.M[2:])
    f = g_hi[:, :, None, None, None] * wx[None, None] + g_lo[:, :, None, None, None] * (1.0 - wx)[None, None]
    if params.get("icmodes"):
        X1, X2, X3 = np.meshgrid(*grid.x, indexing="ij")
        mod = np.ones(grid.M[2:])
        for m in params["icmodes"]:
            q = m["k"]
            mod += m["amp"] * np.cos(q[0] * X1 + q[1] * X2 + q[2] * X3 + m["phase"])
        f = f * mod[None, None]
    return np.ascontiguousarray(f)


def d1_periodic(f, axis, h):
    return (np.roll(f, -1, axis) - np.roll(f, 1, axis)) / (2.0 * h)


def d2_periodic(f, axis, h):
    return (np.roll(f, -1, axis) - 2.0 * f + np.roll(f, 1, axis)) / (h * h)


def _pad(f, axis, lo, hi):
    return np.concatenate([lo, f, hi], axis=axis)


def d1_zero_sum(g, axis, h):
    """CFD2 first derivative with ghosts g_{-1} = -g_0, g_M = -g_{M-1} (Eq. compBCs, n = 1)."""
    first = np.take(g, [0], axis=axis)
    last = np.take(g, [-1], axis=axis)
    gp = _pad(g, axis, -first, -last)
    n = g.shape[axis]
    return (np.take(gp, np.arange(2, n + 2), axis=axis) - np.take(gp, np.arange(0, n), axis=axis)) / (2.0 * h)


def d2_zero_sum(f, axis, h):
    """CFD2 second derivative with ghosts f_{-1} = f_0, f_M = f_{M-1} (Eq. compBCs, n = 2)."""
    first = np.take(f, [0], axis=axis)
    last = np.take(f, [-1], axis=axis)
    fp = _pad(f, axis, first, last)
    n = f.shape[axis]
    return (np.take(fp, np.arange(2, n + 2), axis=axis) - 2.0 * f
            + np.take(fp, np.arange(0, n), axis=axis)) / (h * h)


def d2_flux_periodic(f, g, axis, field_axis, h):
    """d/dx [g df/dx] in flux form on a periodic axis: face value
    g_{i+1/2} = (g_i + g_{i+1}) / 2, result [g_{i+1/2}(f_{i+1} - f_i) -
    g_{i-1/2}(f_i - f_{i-1})] / h^2.  g lives on the 3 x axes (field_axis)
    and is broadcast over the leading phi axes of f when f has more axes."""
    gp = 0.5 * (g + np.roll(g, -1, field_axis))
    lead = f.ndim - g.ndim
    gp = gp.reshape((1,) * lead + gp.shape)
    flux = gp * (np.roll(f, -1, axis) - f)
    return (flux - np.roll(flux, 1, axis)) / (h * h)


def filter_width(params, grid: Grid):
    """LES filter width Delta = delta_cells (h1 h2 h3)^(1/3); the paper takes
    Delta = 3 Delta x on an isotropic grid."""
    return params.get("delta_cells", 3.0) * (grid.h_x[0] * grid.h_x[1] * grid.h_x[2]) ** (1.0 / 3.0)


def subgrid_fields(params, grid: Grid, u):
    """(gamma + gamma_SGS(x), Omega_mix(x)) on the x grid (Eq. FP0 and its
    Smagorinsky / LMSE closures): gamma_SGS = C_s Delta^2 / 2 |S|,
    |S| = sqrt(sum_ij (d_j u_i + d_i u_j)^2) from CFD2 derivatives of the
    sampled velocity, Omega_mix = C_Omega (gamma + gamma_SGS) / Delta^2."""
    D = filter_width(params, grid)
    s2 = np.zeros(grid.M[2:])
    for i in range(3):
        for j in range(3):
            sij = d1_periodic(u[i], j, grid.h_x[j]) + d1_periodic(u[j], i, grid.h_x[i])
            s2 += sij * sij
    gam = params["gamma"] + params["c_s"] * 0.5 * D * D * np.sqrt(s2)
    return gam, params["c_omega"] * gam / (D * D)


def conditional_means(f, grid: Grid):
    """<Phi_a>(x) = h1 h2 sum_{i1,i2} phi_a f  (Eq. 2, unnormalised)."""
    w = grid.h_phi[0] * grid.h_phi[1]
    m1 = w * np.tensordot(grid.phi[0], f.sum(axis=1), axes=(0, 0))
    m2 = w * np.tensordot(grid.phi[1], f.sum(axis=0), axes=(0, 0))
    return m1, m2


def rhs(f, grid: Grid, u, params):
    """L(f) of Eq. FP2 (see the module docstring)."""
    om, da, gam, dphi = params["omega"], params["da"], params["gamma"], params["d_phi"]
    sgs = params.get("sgs", 0) == 1
    if sgs:  # gamma(x) and Omega_mix(x) replace the constants
        gam_x, om_x = subgrid_fields(params, grid, u)
        om = om_x[None, None]
    out = np.zeros_like(f)
    for i in range(3):
        ax = 2 + i
        hx = grid.h_x[i]
        out -= u[i][None, None] * d1_periodic(f, ax, hx)
        if sgs:
            out += d2_flux_periodic(f, gam_x, ax, i, hx)
        elif gam != 0.0:
            out += gam * d2_periodic(f, ax, hx)
    m1, m2 = conditional_means(f, grid)
    P1 = grid.phi[0][:, None, None, None, None]
    P2 = grid.phi[1][None, :, None, None, None]
    react = da * P1 * P2
    g1 = (om * (P1 - m1[None, None]) + react) * f
    g2 = (om * (P2 - m2[None, None]) + react) * f
    out += d1_zero_sum(g1, 0, grid.h_phi[0])
    out += d1_zero_sum(g2, 1, grid.h_phi[1])
    if dphi != 0.0:
        out += dphi * d2_zero_sum(f, 0, grid.h_phi[0])
        out += dphi * d2_zero_sum(f, 1, grid.h_phi[1])
    return out


def rk2_step(f, grid: Grid, u, params):
    dt = params["dt"]
    if params.get("rk_variant", 0) == 1:
        fh = f + 0.5 * dt * rhs(f, grid, u, params)
        return f + dt * rhs(fh, grid, u, params)
    fs = f + dt * rhs(f, grid, u, params)
    return 0.5 * (f + fs + dt * rhs(fs, grid, u, params))


def solve(params, nsteps, f0=None, u=None):
    """Advance the initial PDF (or f0) by nsteps RK2 steps; returns the dense array."""
    grid = make_grid(params["bits"])
    if u is None:
        u = velocity_field(params, grid)
    f = initial_pdf(params, grid) if f0 is None else np.array(f0, dtype=np.float64)
    for _ in range(int(nsteps)):
        f = rk2_step(f, grid, u, params)
    return f


def observables(f, grid: Grid):
    """Point-wise moments and their space averages (Eqs. 2, spaceAvg, RACov, SGSCov).

    Returns a dict with the fields norm(x) = <1>, mean1/mean2 = <Phi_a>,
    and the scalars norm_avg, mean1_avg, mean2_avg, phi11_avg, phi22_avg,
    phi12_avg (space averages of <Phi_a Phi_b>), R12, Y12 and product_J
    (the space average of <1 - phi1 - phi2>)."""
    w = grid.h_phi[0] * grid.h_phi[1]
    P1 = grid.phi[0][:, None, None, None, None]
    P2 = grid.phi[1][None, :, None, None, None]
    norm = w * f.sum(axis=(0, 1))
    m1, m2 = conditional_means(f, grid)
    s11 = w * (P1 * P1 * f).sum(axis=(0, 1))
    s22 = w * (P2 * P2 * f).sum(axis=(0, 1))
    s12 = w * (P1 * P2 * f).sum(axis=(0, 1))
    avg = lambda a: float(a.mean())
    out = dict(norm=norm, mean1=m1, mean2=m2,
               norm_avg=avg(norm), mean1_avg=avg(m1), mean2_avg=avg(m2),
               phi11_avg=avg(s11), phi22_avg=avg(s22), phi12_avg=avg(s12))
    out["R12"] = avg(m1 * m2) - out["mean1_avg"] * out["mean2_avg"]
    out["Y12"] = avg(s12 - m1 * m2)
    out["product_J"] = out["norm_avg"] - out["mean1_avg"] - out["mean2_avg"]
    return out


def moment_rhs(m, grid: Grid, u, gamma):
    """Eq. FPMoms with S = 0 on the 3-D grid: -u . D1x m + gamma sum_i D2x_i m;
    gamma may be a field on the x grid (flux form, see d2_flux_periodic)."""
    out = np.zeros_like(m)
    field = np.ndim(gamma) == 3
    for i in range(3):
        out -= u[i] * d1_periodic(m, i, grid.h_x[i])
        if field:
            out += d2_flux_periodic(m, gamma, i, i, grid.h_x[i])
        elif gamma != 0.0:
            out += gamma * d2_periodic(m, i, grid.h_x[i])
    return out


def moment_step(m, grid: Grid, u, params):
    dt, gam = params["dt"], params["gamma"]
    if params.get("sgs", 0) == 1:
        gam = subgrid_fields(params, grid, u)[0]
    if params.get("rk_variant", 0) == 1:
        mh = m + 0.5 * dt * moment_rhs(m, grid, u, gam)
        return m + dt * moment_rhs(mh, grid, u, gam)
    ms = m + dt * moment_rhs(m, grid, u, gam)
    return 0.5 * (m + ms + dt * moment_rhs(ms, grid, u, gam))


def bond_profile(N, chi):
    """p(n) = min(2^n, 2^(N-n), chi) for n = 0..N (Eq. MPSdofs)."""
    return [min(2 ** n, 2 ** (N - n), chi) for n in range(N + 1)]


def nvpp(N, chi):
    """Number of variables parameterising the PDF, Eq. MPSdofs."""
    p = bond_profile(N, chi)
    return 2 * sum(p[n - 1] * p[n] for n in range(1, N + 1)) - sum(p[n] ** 2 for n in range(1, N))


def error_measures(samples, exact=None):
    """Eqs. RMSE0 / RMSE1: samples is a list (one entry per stored time, the
    paper uses 17 equally spaced ones) of dicts with the space averages
    mean1_avg, mean2_avg and the fields norm, mean1, mean2 (from observables);
    exact the matching list of (<Phi_1>, <Phi_2>) fields of the moment
    equation (or None).  E_t averages squared differences over the samples
    (step quadrature), E_tx also over all grid points.  Returns
    err_2b_up = sqrt(1/2 sum_a E_t[avg<Phi_a> - 1/2]),
    err_2b_down = sqrt(1/2 sum_a E_tx[<Phi_a> - <Phi_a>_exact]) (None
    without exact), err_2c_up = sqrt(E_t[avg<Phi_1> - avg<Phi_2>]),
    err_2c_down = sqrt(E_tx[<1> - 1])."""
    Et = lambda vals: float(np.mean(np.square(vals)))
    out = {}
    out["err_2b_up"] = math.sqrt(0.5 * sum(Et([s[f"mean{a}_avg"] - 0.5 for s in samples]) for a in (1, 2)))
    if exact is not None:
        out["err_2b_down"] = math.sqrt(0.5 * sum(
            float(np.mean([np.mean(np.square(s[f"mean{a}"] - e[a - 1])) for s, e in zip(samples, exact)]))
            for a in (1, 2)))
    else:
        out["err_2b_down"] = None
    out["err_2c_up"] = math.sqrt(Et([s["mean1_avg"] - s["mean2_avg"] for s in samples]))
    out["err_2c_down"] = math.sqrt(float(np.mean([np.mean(np.square(s["norm"] - 1.0)) for s in samples])))
    return out
