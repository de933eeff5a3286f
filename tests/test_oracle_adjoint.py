"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against the
forward oracle (oracle/fd.py), on CPU.

* The objective is the observable product_J of fd.observables.
* Transpose identity: <lam, L'(f) v> = <L'(f)^T lam, v>, with L'(f) v taken
  as (L(f + v) - L(f - v)) / 2, which is exact for the quadratic map L of
  Eq. FP2 (linear terms plus the bilinear mixing drift).
* dL/dtheta against (L(theta + 1) - L(theta - 1)) / 2: L is affine in each
  parameter, so this is exact too.
* The whole gradient of J after a few Heun steps against central
  differences of J(theta) through fd.solve.
"""
import numpy as np
import pytest

import oracle
import workload
from oracle import adjoint as adj


def _params(bits, n_ic=2, seed=3):
    p = workload.make_params({"bits": 2, "chi_max": 32}, seed=seed, bits=list(bits))
    rng = np.random.default_rng(seed)
    p["icmodes"] = []
    for _ in range(n_ic):
        k = [int(v) for v in rng.integers(-2, 3, size=3)]
        if not any(k):
            k[0] = 1
        p["icmodes"].append(dict(k=k, phase=float(rng.uniform(0, 2 * np.pi)), amp=0.0))
    return p


def test_objective_is_product_j():
    p = _params([3, 2, 2, 3, 2])
    g = oracle.make_grid(p["bits"])
    f = oracle.solve(p, 2)
    assert adj.objective(f, g) == pytest.approx(oracle.observables(f, g)["product_J"], rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("bits", [[2, 2, 2, 2, 2], [3, 2, 2, 3, 2]])
def test_transpose_identity(bits):
    p = _params(bits)
    p["omega"], p["da"], p["gamma"], p["d_phi"] = 1.3, 0.7, 0.05, 0.01
    g = oracle.make_grid(p["bits"])
    u = oracle.velocity_field(p, g)
    rng = np.random.default_rng(1)
    f, v, lam = (rng.standard_normal(g.shape) for _ in range(3))
    jv = 0.5 * (oracle.rhs(f + v, g, u, p) - oracle.rhs(f - v, g, u, p))
    lhs = float(np.sum(lam * jv))
    rhs = float(np.sum(adj.rhs_transpose(f, lam, g, u, p) * v))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), float(np.sum(np.abs(lam * jv))))


@pytest.mark.parametrize("name", ["omega", "da", "gamma", "umode0", "umode2"])
def test_param_derivative(name):
    p = _params([3, 2, 3, 2, 2])
    g = oracle.make_grid(p["bits"])
    rng = np.random.default_rng(2)
    f = rng.standard_normal(g.shape)
    v = adj.param_value(p, name)
    pp, pm = adj.with_param(p, name, v + 1.0), adj.with_param(p, name, v - 1.0)
    ref = 0.5 * (oracle.rhs(f, g, oracle.velocity_field(pp, g), pp) - oracle.rhs(f, g, oracle.velocity_field(pm, g), pm))
    got = adj.rhs_param_derivative(f, g, oracle.velocity_field(p, g), p, name)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_gradient_against_central_differences():
    p = _params([3, 3, 3, 3, 3])
    nsteps = 4
    J, grad = adj.gradient(p, nsteps)
    g = oracle.make_grid(p["bits"])
    assert J == pytest.approx(adj.objective(oracle.solve(p, nsteps), g), rel=1e-13)
    ref = adj.fd_gradient(p, nsteps)
    scale = np.max(np.abs(ref))
    for name, a, b in zip(adj.param_names(p), grad, ref):
        assert abs(a - b) <= 1e-6 * abs(b) + 1e-9 * scale, (name, a, b)
