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
