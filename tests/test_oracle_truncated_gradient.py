"""CPU pins of oracle.adjoint.gradient_truncated: the gradient of J through
Heun steps whose two stage sums are truncated to chi (the MPS algorithm's
rounding), against central differences of J through solve_truncated.

The truncated map is differentiable only where every kept eigenvalue of every
cut's Gram is separated from the discarded ones and the kept counts are held
by tol against the small singular values a perturbation adds.  The analytic
initial PDF with zero modulation has exactly repeated singular values across
the chi boundary (a symmetry), so the configuration here draws nonzero
initial-condition amplitudes, and the test first checks the separation
(smallest relative gap and smallest kept eigenvalue over all stages)."""
import numpy as np
import pytest

import workload
from oracle import adjoint as adj
from oracle import fd
from oracle import truncation as tr

SEED, CHI, TOL, STEPS = 1, 4, 1e-5, 3


def _params():
    p = workload.make_params({"bits": 2, "chi_max": CHI, "steps": STEPS}, seed=SEED)
    p["icmodes"] = workload.draw_ic_modes(SEED, 3)
    rng = np.random.default_rng(100 + SEED)
    for m in p["icmodes"]:
        m["amp"] = float(rng.uniform(0.05, 0.2))
    return p


def _separation(p):
    """Smallest (lambda_k - lambda_{k+1}) / lambda_1 and lambda_k / lambda_1
    over every truncated cut of every stage."""
    grid = fd.make_grid(p["bits"])
    u = fd.velocity_field(p, grid)
    N, dt = int(sum(p["bits"])), p["dt"]
    f = fd.initial_pdf(p, grid)
    gap, low = np.inf, np.inf
    for _ in range(STEPS):
        for stage in (1, 2):
            X = f + dt * fd.rhs(f, grid, u, p) if stage == 1 else 0.5 * (f + fs + dt * fd.rhs(fs, grid, u, p))
            P = tr.projectors(X.ravel(), N, CHI, TOL)
            for n in range(1, N):
                _, k, lam, _ = P[n]
                if k < len(lam):
                    gap = min(gap, (lam[k - 1] - lam[k]) / lam[0])
                    low = min(low, lam[k - 1] / lam[0])
            Y = tr.truncate(X.ravel(), N, CHI, TOL, P).reshape(f.shape)
            if stage == 1:
                fs = Y
            else:
                f = Y
    return gap, low


def test_configuration_is_separated():
    gap, low = _separation(_params())
    assert gap > 1e-6 and low > 1e-6, (gap, low)


def test_truncated_gradient_matches_central_differences():
    p = _params()
    grid = fd.make_grid(p["bits"])
    J, g = adj.gradient_truncated(p, STEPS, CHI, TOL)
    assert J == pytest.approx(adj.objective(adj.solve_truncated(p, STEPS, CHI, TOL), grid), rel=1e-14)
    names = adj.param_names(p)
    fdg = []
    for n in names:
        v = adj.param_value(p, n)
        h = 1e-5 * max(abs(v), 1.0)
        jp = adj.objective(adj.solve_truncated(adj.with_param(p, n, v + h), STEPS, CHI, TOL), grid)
        jm = adj.objective(adj.solve_truncated(adj.with_param(p, n, v - h), STEPS, CHI, TOL), grid)
        fdg.append((jp - jm) / (2 * h))
    fdg = np.array(fdg)
    scale = np.abs(fdg).max()
    assert np.abs(g - fdg).max() <= 1e-6 * scale, np.abs(g - fdg) / scale
    # the truncation's own derivative matters here: the gradient of the
    # untruncated map is far from it
    _, gu = adj.gradient(p, STEPS)
    assert np.abs(gu - fdg).max() > 1e-2 * scale


def test_broadened_truncated_gradient_tends_to_exact():
    p = _params()
    _, g = adj.gradient_truncated(p, STEPS, CHI, TOL)
    grid = fd.make_grid(p["bits"])
    f0 = fd.initial_pdf(p, grid).ravel()
    N = int(sum(p["bits"]))
    lam1 = max(np.linalg.norm(tr.unfold(f0, N, n), 2) ** 2 for n in range(1, N))
    errs = [np.abs(adj.gradient_truncated(p, STEPS, CHI, TOL, e * lam1)[1] - g).max() for e in (1e-6, 1e-9)]
    assert errs[1] < errs[0] and errs[1] <= 1e-6 * np.abs(g).max()
