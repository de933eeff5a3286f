"""Batched stepping (qtt_step_many): independent PDFs of different grid, chi
and precision advanced together on their own streams give exactly the
states of stepping each alone."""
import pytest

import workload

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")


@pytest.fixture(scope="module", autouse=True)
def lib(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    return pkg.load_library()


def _instances():
    return [
        workload.make_params({"bits": 3, "chi_max": 8}, seed=1, precision="fp32", omega=0.7, da=3.0),
        workload.make_params({"bits": 4, "chi_max": 16}, seed=2, precision="fp64"),
        workload.make_params({"bits": 4, "chi_max": 12}, seed=3, precision="bf16x3", da=0.2),
        workload.make_params({"bits": 3, "chi_max": 128}, seed=4, precision="fp64", exact=1, svd_rel_tol=0.0),
    ]


def test_step_many_matches_separate_steps():
    """The first steps run context by context (eager step, graph captures);
    from then on one parent graph per step embeds every context's step graph.
    Stepping one context alone in between changes the contexts' relative
    parities, so the parent graphs are rebuilt; every state stays bitwise
    equal to stepping the contexts one by one."""
    ps = _instances()
    batch = [pkg.qtt_init(p) for p in ps]
    alone = [pkg.qtt_init(p) for p in ps]
    try:
        pkg.qtt_step_many(batch, 6)
        batch[1].step(1)
        pkg.qtt_step_many(batch, 3)
        for i, c in enumerate(alone):
            c.step(10 if i == 1 else 9)
        for a, b in zip(batch, alone):
            assert a.scalars()["steps"] == b.scalars()["steps"]
            assert a.compare(b) == 0.0
    finally:
        for c in batch + alone:
            c.close()


def test_step_many_rejects_a_repeated_context():
    c = pkg.qtt_init(_instances()[0])
    try:
        with pytest.raises(pkg.QttError) as ei:
            pkg.qtt_step_many([c, c], 1)
        assert "twice" in str(ei.value)
    finally:
        c.close()
