"""Seeded input generators (CPU): the batched configuration's ranges and
reproducibility."""
import numpy as np

import workload


def test_batch_params_ranges_and_seeding():
    a = workload.make_batch_params(64, seed=0)
    b = workload.make_batch_params(64, seed=0)
    assert a == b
    for i, p in enumerate(a):
        K = p["bits"][0]
        assert p["bits"] == [K] * 5 and K in (5, 6, 7)
        assert p["chi_max"] in (16, 32, 64, 96)
        assert 0.1 <= p["da"] <= 10.0 and 0.5 <= p["omega"] <= 2.0
        assert np.isclose(p["d_phi"], 4e-3 * p["omega"])
        assert p["umodes"] == workload.draw_velocity_modes(i)
        ub = abs(p["shear_amp"]) + sum(abs(m["amp"]) for m in p["umodes"])
        assert p["dt"] == workload.cfl_dt(p["bits"], p["omega"], p["da"], p["gamma"], p["d_phi"], ub)
    # every grid size and chi is drawn
    assert {p["bits"][0] for p in a} == {5, 6, 7}
    assert {p["chi_max"] for p in a} == {16, 32, 64, 96}


def test_truncation_trains_are_left_orthonormal():
    """The inputs of the truncation backward's timing: bonds min(2^n, 2^(N-n),
    ell) and min(.., chi), the first N-1 cores of X with orthonormal columns
    (the precondition of qtt_truncate_vjp), seeded."""
    N, ell, chi = 12, 20, 16
    r, x, s, y = workload.make_truncation_trains(N, ell, chi)
    assert r == [min(2 ** n, 2 ** (N - n), ell) for n in range(N + 1)]
    assert s == [min(2 ** n, 2 ** (N - n), chi) for n in range(N + 1)]
    assert x.size == sum(r[n] * 2 * r[n + 1] for n in range(N))
    assert y.size == sum(s[n] * 2 * s[n + 1] for n in range(N))
    off = 0
    for n in range(N - 1):
        Q = x[off: off + r[n] * 2 * r[n + 1]].reshape(2 * r[n], r[n + 1])
        assert np.abs(Q.T @ Q - np.eye(r[n + 1])).max() < 1e-13
        off += r[n] * 2 * r[n + 1]
    r2, x2, _, y2 = workload.make_truncation_trains(N, ell, chi)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
