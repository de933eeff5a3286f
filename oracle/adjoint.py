"""Discrete adjoint of the dense finite-difference oracle (gradients of a
final-time observable with respect to the model parameters).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import or run this
module.  The product path never calls it, and the two share no code.

What it computes (plain FP64 numpy):

* The observable J = mean over x of <1> - <Phi_1> - <Phi_2>, i.e. the space
  average of h_phi1 h_phi2 sum_phi (1 - phi1 - phi2) f  (the mean final
  product of Eqs. 2 and spaceAvg).  It is linear in f, so its gradient
  lambda_T = dJ/df is the fixed array (h1 h2 / n_x) (1 - phi1 - phi2).
* The adjoint of one Heun step f_{n+1} = (f + f* + dt L(f*)) / 2,
  f* = f + dt L(f), of Eq. FP2, for the Euclidean inner product
  <a, b> = sum over all cells a b:
      mu        = dJ/df*  = (lambda + dt L'(f*)^T lambda) / 2
      dJ/df_n   = lambda / 2 + mu + dt L'(f)^T mu
  and the parameter gradient of the step
      dJ/dtheta += dt <lambda, dL/dtheta(f*)> / 2 + dt <mu, dL/dtheta(f)>.
* L'(f)^T, the transpose of the Jacobian of L (module fd.rhs).  The linear
  part is transposed operator by operator: every 1-D stencil is turned into
  its matrix by applying the forward stencil of fd to the unit vectors, and
  the matrix is transposed.  The mixing drift D1phi_a[-Omega <Phi_a>(x) f] is
  bilinear in f (Eq. 2 is linear in f); its linearisation in the direction v
  is -Omega D1phi_a[<Phi_a>(x) v + <Phi_a>[v](x) f], whose transpose applied
  to lambda, with w = D1phi_a^T lambda, is
      -Omega ( <Phi_a>(x) w  +  h1 h2 phi_a  sum_phi' f w ).
* dL/dtheta for theta = Omega, Da, gamma (diffusivity in x) and the
  amplitude a_m of each velocity Fourier mode u_c += a_m sin(k_m . x + t_m):
      dL/dOmega = sum_a D1phi_a[(phi_a - <Phi_a>(x)) f]
      dL/dDa    = sum_a D1phi_a[phi1 phi2 f]
      dL/dgamma = sum_i D2x_i f
      dL/da_m   = -sin(k_m . x + t_m) D1x_c f
  and, for the amplitude b_m of each initial-condition modulation
  f0 = g(phi, x) (1 + sum_m b_m cos(q_m . x + p_m)),
      dJ/db_m   = <dJ/df_0, g cos(q_m . x + p_m)>.
  The time step is held fixed (it is an input, not a function of theta).

* With the bond truncation in the step (``solve_truncated``,
  ``gradient_truncated``): each stage's sum is truncated as the stages of the
  MPS algorithm are, f* = T(f + dt L(f)) and f_{n+1} = T((f + f* + dt L(f*)) / 2),
  T the simultaneous truncation of every bond of the dense state read as a
  train of N binary sites (module truncation).  The backward passes each
  cotangent through T's vector-Jacobian product first:
      lambda2 = T'(X2)^T lambda,  mu = T'(X1)^T (lambda2 + dt L'(f*)^T lambda2) / 2,
      dJ/df_n = lambda2 / 2 + mu + dt L'(f_n)^T mu,
  with the parameter terms taken against lambda2 and mu.

Parity status: pinned in ``tests/test_oracle_adjoint.py`` against the
forward oracle -- the transpose identity <lambda, L'(f) v> = <L'(f)^T lambda, v>
with L'(f) v from central differences of fd.rhs (exact for a quadratic map),
dL/dtheta against central differences of fd.rhs in theta (exact: L is affine
in each parameter), and the whole gradient against central differences of
J(theta) through fd.solve.  The truncated gradient is pinned in
``tests/test_oracle_truncated_gradient.py`` against central differences of J
through solve_truncated, in a configuration whose kept and discarded
eigenvalues are separated at every stage.
"""
from __future__ import annotations

import copy

import numpy as np

from . import fd
from . import truncation

__all__ = ["param_names", "objective", "objective_gradient", "rhs_transpose", "rhs_param_derivative",
           "gradient", "fd_gradient", "with_param", "solve_truncated", "gradient_truncated"]


def param_names(params):
    """Parameter order of the gradient: Omega, Da, gamma, the velocity mode
    amplitudes (in the order of params['umodes']), the initial-condition
    modulation amplitudes (in the order of params['icmodes'])."""
    names = ["omega", "da", "gamma"]
    names += [f"umode{i}" for i in range(len(params["umodes"]))]
    names += [f"icmode{i}" for i in range(len(params.get("icmodes") or []))]
    return names


def with_param(params, name, value):
    """A copy of params with one parameter replaced (dt unchanged)."""
    p = copy.deepcopy(params)
    if name.startswith("umode"):
        p["umodes"][int(name[5:])]["amp"] = float(value)
    elif name.startswith("icmode"):
        p["icmodes"][int(name[6:])]["amp"] = float(value)
    else:
        p[name] = float(value)
    return p


def param_value(params, name):
    if name.startswith("umode"):
        return params["umodes"][int(name[5:])]["amp"]
    if name.startswith("icmode"):
        return params["icmodes"][int(name[6:])]["amp"]
    return params[name]


def objective(f, grid: fd.Grid):
    """J = space average of <1> - <Phi_1> - <Phi_2>."""
    return float(np.sum(objective_gradient(grid) * f))


def objective_gradient(grid: fd.Grid):
    """dJ/df: (h1 h2 / n_x) (1 - phi1 - phi2), constant in x."""
    P1 = grid.phi[0][:, None, None, None, None]
    P2 = grid.phi[1][None, :, None, None, None]
    nx = grid.M[2] * grid.M[3] * grid.M[4]
    w = grid.h_phi[0] * grid.h_phi[1] / nx
    return np.broadcast_to(w * (1.0 - P1 - P2), grid.shape).copy()


# ------------------------------------------------------------------ operators
def _matrix(stencil, M, h):
    """The M x M matrix of a 1-D stencil of fd: column j = stencil(e_j)."""
    return np.stack([stencil(np.eye(M)[j], 0, h) for j in range(M)], axis=1)


def _apply(mat, arr, axis):
    """mat applied along one axis of arr."""
    return np.moveaxis(np.tensordot(mat, arr, axes=(1, axis)), 0, axis)


class _Ops:
    """1-D matrices of the stencils of Eq. FP2 on a grid, and their transposes."""

    def __init__(self, grid: fd.Grid):
        self.grid = grid
        self.d1x = [_matrix(fd.d1_periodic, grid.M[2 + i], grid.h_x[i]) for i in range(3)]
        self.d2x = [_matrix(fd.d2_periodic, grid.M[2 + i], grid.h_x[i]) for i in range(3)]
        self.d1p = [_matrix(fd.d1_zero_sum, grid.M[a], grid.h_phi[a]) for a in range(2)]
        self.d2p = [_matrix(fd.d2_zero_sum, grid.M[a], grid.h_phi[a]) for a in range(2)]


def _phi_arrays(grid):
    P1 = grid.phi[0][:, None, None, None, None]
    P2 = grid.phi[1][None, :, None, None, None]
    return P1, P2


def _mode_sin(grid, m):
    X1, X2, X3 = np.meshgrid(*grid.x, indexing="ij")
    k = m["k"]
    return np.sin(k[0] * X1 + k[1] * X2 + k[2] * X3 + m["phase"])


def _mode_cos(grid, m):
    X1, X2, X3 = np.meshgrid(*grid.x, indexing="ij")
    q = m["k"]
    return np.cos(q[0] * X1 + q[1] * X2 + q[2] * X3 + m["phase"])


def rhs_transpose(f, lam, grid: fd.Grid, u, params, ops: _Ops | None = None):
    """L'(f)^T lam: the transpose of the Jacobian of fd.rhs at f, applied to lam."""
    ops = ops or _Ops(grid)
    om, da, gam, dphi = params["omega"], params["da"], params["gamma"], params["d_phi"]
    out = np.zeros_like(lam)
    for i in range(3):
        ax = 2 + i
        # -u_i D1x_i f  ->  -D1x_i^T (u_i lam)
        out -= _apply(ops.d1x[i].T, u[i][None, None] * lam, ax)
        if gam != 0.0:
            out += gam * _apply(ops.d2x[i].T, lam, ax)
    P1, P2 = _phi_arrays(grid)
    m1, m2 = fd.conditional_means(f, grid)
    h12 = grid.h_phi[0] * grid.h_phi[1]
    for a, (Pa, ma) in enumerate(((P1, m1), (P2, m2))):
        w = _apply(ops.d1p[a].T, lam, a)  # D1phi_a^T lam
        # linear drift (Omega phi_a + Da phi1 phi2) f
        out += (om * Pa + da * P1 * P2) * w
        # bilinear mixing -Omega <Phi_a>(x) f
        out -= om * ma[None, None] * w
        s = np.sum(f * w, axis=(0, 1))  # sum over phi of f w, a field of x
        out -= om * h12 * Pa * s[None, None]
        if dphi != 0.0:
            out += dphi * _apply(ops.d2p[a].T, lam, a)
    return out


def rhs_param_derivative(f, grid: fd.Grid, u, params, name, ops: _Ops | None = None):
    """dL/dtheta at f for theta = omega, da, gamma or umode<i>."""
    ops = ops or _Ops(grid)
    P1, P2 = _phi_arrays(grid)
    if name == "omega":
        m1, m2 = fd.conditional_means(f, grid)
        return (_apply(ops.d1p[0], (P1 - m1[None, None]) * f, 0)
                + _apply(ops.d1p[1], (P2 - m2[None, None]) * f, 1))
    if name == "da":
        return _apply(ops.d1p[0], P1 * P2 * f, 0) + _apply(ops.d1p[1], P1 * P2 * f, 1)
    if name == "gamma":
        return sum(_apply(ops.d2x[i], f, 2 + i) for i in range(3))
    if name.startswith("umode"):
        m = params["umodes"][int(name[5:])]
        c = m["comp"]
        return -_mode_sin(grid, m)[None, None] * _apply(ops.d1x[c], f, 2 + c)
    raise ValueError(name)


def _ic_derivative(params, grid, name):
    """df0/db_m = g cos(q_m . x + p_m), g the initial PDF without modulation."""
    m = params["icmodes"][int(name[6:])]
    p0 = copy.deepcopy(params)
    p0["icmodes"] = []
    g = fd.initial_pdf(p0, grid)
    return g * _mode_cos(grid, m)[None, None]


def gradient(params, nsteps):
    """(J, dJ/dtheta) after nsteps Heun steps from the initial PDF, theta in
    the order of param_names(params)."""
    if params.get("rk_variant", 0) != 0:
        raise ValueError("the adjoint is written for the Heun scheme")
    grid = fd.make_grid(params["bits"])
    u = fd.velocity_field(params, grid)
    ops = _Ops(grid)
    dt = params["dt"]
    f = fd.initial_pdf(params, grid)
    traj = []
    for _ in range(int(nsteps)):
        fs = f + dt * fd.rhs(f, grid, u, params)
        traj.append((f, fs))
        f = 0.5 * (f + fs + dt * fd.rhs(fs, grid, u, params))
    J = objective(f, grid)
    names = param_names(params)
    dyn = [n for n in names if not n.startswith("icmode")]
    g = dict.fromkeys(names, 0.0)
    lam = objective_gradient(grid)
    for f, fs in reversed(traj):
        mu = 0.5 * (lam + dt * rhs_transpose(fs, lam, grid, u, params, ops))
        for n in dyn:
            g[n] += 0.5 * dt * float(np.sum(lam * rhs_param_derivative(fs, grid, u, params, n, ops)))
            g[n] += dt * float(np.sum(mu * rhs_param_derivative(f, grid, u, params, n, ops)))
        lam = 0.5 * lam + mu + dt * rhs_transpose(f, mu, grid, u, params, ops)
    for n in names:
        if n.startswith("icmode"):
            g[n] = float(np.sum(lam * _ic_derivative(params, grid, n)))
    return J, np.array([g[n] for n in names])


def fd_gradient(params, nsteps, names=None, rel_h=1e-4):
    """Central differences of J through fd.solve, step h = rel_h * max(|theta|, 1)."""
    grid = fd.make_grid(params["bits"])
    names = names or param_names(params)
    out = []
    for n in names:
        v = param_value(params, n)
        h = rel_h * max(abs(v), 1.0)
        jp = objective(fd.solve(with_param(params, n, v + h), nsteps), grid)
        jm = objective(fd.solve(with_param(params, n, v - h), nsteps), grid)
        out.append((jp - jm) / (2.0 * h))
    return np.array(out)


def solve_truncated(params, nsteps, chi, tol=0.0):
    """nsteps Heun steps with both stage sums truncated to chi (module
    truncation, the state read as a train of sum(bits) binary sites, site
    order phi1, phi2, x1, x2, x3, most significant bit first); returns the
    dense final state."""
    grid = fd.make_grid(params["bits"])
    u = fd.velocity_field(params, grid)
    N = int(sum(params["bits"]))
    dt = params["dt"]
    f = fd.initial_pdf(params, grid)
    shape = f.shape
    for _ in range(int(nsteps)):
        fs = truncation.truncate((f + dt * fd.rhs(f, grid, u, params)).ravel(), N, chi, tol).reshape(shape)
        f = truncation.truncate((0.5 * (f + fs + dt * fd.rhs(fs, grid, u, params))).ravel(), N, chi,
                                tol).reshape(shape)
    return f


def gradient_truncated(params, nsteps, chi, tol=0.0, eps=0.0):
    """(J, dJ/dtheta) through solve_truncated (module docstring), theta in the
    order of param_names(params); eps broadens the truncation's gaps."""
    if params.get("rk_variant", 0) != 0:
        raise ValueError("the adjoint is written for the Heun scheme")
    grid = fd.make_grid(params["bits"])
    u = fd.velocity_field(params, grid)
    ops = _Ops(grid)
    N = int(sum(params["bits"]))
    dt = params["dt"]
    f = fd.initial_pdf(params, grid)
    shape = f.shape
    traj = []
    for _ in range(int(nsteps)):
        X1 = f + dt * fd.rhs(f, grid, u, params)
        fs = truncation.truncate(X1.ravel(), N, chi, tol).reshape(shape)
        X2 = 0.5 * (f + fs + dt * fd.rhs(fs, grid, u, params))
        traj.append((f, X1, fs, X2))
        f = truncation.truncate(X2.ravel(), N, chi, tol).reshape(shape)
    J = objective(f, grid)
    names = param_names(params)
    dyn = [n for n in names if not n.startswith("icmode")]
    g = dict.fromkeys(names, 0.0)
    lam = objective_gradient(grid)
    for f, X1, fs, X2 in reversed(traj):
        lam2 = truncation.truncate_vjp(X2.ravel(), lam.ravel(), N, chi, tol, eps).reshape(shape)
        pre = 0.5 * (lam2 + dt * rhs_transpose(fs, lam2, grid, u, params, ops))
        mu = truncation.truncate_vjp(X1.ravel(), pre.ravel(), N, chi, tol, eps).reshape(shape)
        for n in dyn:
            g[n] += 0.5 * dt * float(np.sum(lam2 * rhs_param_derivative(fs, grid, u, params, n, ops)))
            g[n] += dt * float(np.sum(mu * rhs_param_derivative(f, grid, u, params, n, ops)))
        lam = 0.5 * lam2 + mu + dt * rhs_transpose(f, mu, grid, u, params, ops)
    for n in names:
        if n.startswith("icmode"):
            g[n] = float(np.sum(lam * _ic_derivative(params, grid, n)))
    return J, np.array([g[n] for n in names])
