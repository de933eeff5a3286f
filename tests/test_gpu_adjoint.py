"""Discrete adjoint on the GPU (qtt_grad through the C ABI) against the
oracle's dense adjoint (oracle/adjoint.py, itself pinned by
tests/test_oracle_adjoint.py) and against central differences of the GPU
forward map."""
import numpy as np
import pytest

import workload
from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")


@pytest.fixture(scope="module", autouse=True)
def lib(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    return pkg.load_library()


def with_ic_modes(p, n, seed=5):
    rng = np.random.default_rng(seed)
    p["icmodes"] = []
    for _ in range(n):
        k = [int(v) for v in rng.integers(-2, 3, size=3)]
        if not any(k):
            k[0] = 1
        p["icmodes"].append(dict(k=k, phase=float(rng.uniform(0, 2 * np.pi)), amp=0.0))
    return p


def exact_params(bits, **kw):
    p = workload.make_params({"bits": 2, "chi_max": 32}, bits=list(bits), **kw)
    N = sum(p["bits"])
    p["chi_max"] = 2 ** (N // 2)
    p["svd_rel_tol"] = 0.0
    p["exact"] = 1
    return p


@pytest.mark.parametrize("bits,steps,ckpt,flow", [([2, 2, 2, 2, 2], 4, 0, 0), ([2, 2, 3, 2, 3], 3, 2, 0),
                                                  ([2, 2, 2, 2, 2], 3, 1, 1)])
def test_exact_adjoint_matches_oracle(bits, steps, ckpt, flow):
    """Untruncated FP64: the GPU adjoint is the exact gradient of the
    discrete map, like the oracle's (flow 1: the paper's jet through a
    Taylor-Green vortex and its Gaussian step initial PDF, with seeded
    velocity modes added)."""
    if flow == 1:
        p = workload.make_paper_params(bits=2, chi=32, umodes=workload.draw_velocity_modes(0), da=0.7)
        p["bits"] = list(bits)
        N = sum(p["bits"])
        p["chi_max"], p["svd_rel_tol"], p["exact"] = 2 ** (N // 2), 0.0, 1
        p = with_ic_modes(p, 3)
    else:
        p = with_ic_modes(exact_params(bits), 3)
    with pkg.qtt_init(p) as ctx:
        J, g = ctx.grad(steps, ckpt)
        s = ctx.scalars()
    Jr, gr = oadj.gradient(p, steps)
    print("\nJ", J, Jr, "\ngpu   ", g, "\noracle", gr)
    assert abs(J - Jr) <= 1e-12 * abs(Jr) + 1e-15
    assert s["steps"] == steps and abs(s["product_J"] - J) <= 1e-12 * abs(J) + 1e-15
    scale = np.max(np.abs(gr))
    for name, a, b in zip(pkg.grad_param_names(p), g, gr):
        assert abs(a - b) <= 1e-9 * abs(b) + 1e-11 * scale, (name, a, b)


def test_exact_adjoint_vs_central_differences():
    """The untruncated GPU forward map is smooth in every parameter, so its
    central differences (step 1e-4) check the adjoint to O(h^2)."""
    p = with_ic_modes(exact_params([2, 2, 2, 2, 2]), 2)
    steps = 4
    with pkg.qtt_init(p) as ctx:
        _, g = ctx.grad(steps)
    fd = []
    for n in pkg.grad_param_names(p):
        v = oadj.param_value(p, n)
        h = 1e-4 * max(abs(v), 1.0)
        js = []
        for sgn in (1, -1):
            with pkg.qtt_init(oadj.with_param(p, n, v + sgn * h)) as c:
                c.step(steps)
                js.append(c.scalars()["product_J"])
        fd.append((js[0] - js[1]) / (2 * h))
    fd = np.array(fd)
    rel = np.abs(g - fd) / np.max(np.abs(fd))
    print("\nadjoint", g, "\ncentral", fd, "\nrel to max", rel)
    assert np.all(rel <= 1e-6), rel


# Truncated (chi below the full rank 2^7 of the 2^3-point grid): each adjoint
# stage is rounded to chi like a forward stage, so the gradient carries the
# truncation error of the forward and adjoint states.  Measured against the
# oracle's exact gradient, relative to the largest component, over chi 16-64:
# FP64 <= 8.4e-8, FP32 form <= 6.2e-6 (its forward state is 2e-5 from the
# oracle in relative L2).  Bounds: 5e-7 and 5e-5, below the 1e-4 agreement
# asked of the adjoint.
@pytest.mark.parametrize("prec,chi,tol", [("fp64", 24, 5e-7), ("fp32", 24, 5e-5), ("fp32", 64, 5e-5)])
def test_truncated_adjoint_vs_oracle_gradient(prec, chi, tol):
    p = with_ic_modes(workload.make_params({"bits": 3, "chi_max": chi}, precision=prec), 2)
    if prec == "fp64":
        p["svd_rel_tol"] = 0.0
    steps = 6
    with pkg.qtt_init(p) as ctx:
        J, g = ctx.grad(steps, 3)
    Jr, gr = oadj.gradient(p, steps)
    rel = np.abs(g - gr) / np.max(np.abs(gr))
    print(f"\n{prec} chi {chi}: J rel {abs(J - Jr) / abs(Jr):.2e}, gradient rel to max {rel.max():.2e}")
    assert np.all(rel <= tol), rel


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-4), ("fp32", 2.5e-4), ("bf16x10", 1e-4)])
def test_adjoint_at_2p4_vs_oracle_gradient(prec, tol):
    """The adjoint configuration's 23 parameters (Omega, Da, gamma, 4 velocity
    and 16 initial-condition amplitudes) on the 2^20-cell grid (2^4 points per
    dimension), chi 32, 20 Heun steps with checkpoints every 5: the GPU
    gradient agrees with the oracle's FP64 dense-adjoint gradient to 1e-4 of
    the largest component (the agreement asked of the adjoint) in FP64
    (measured 2.2e-6) and BF16X10.  The FP32 form rounds forward and adjoint
    products to 24 bits and drops singular values below 1e-7 sigma_1; its
    distance, 0.8e-4 to 1.4e-4 measured with eigensolvers that differ only in
    rounding order (the ranks its tolerance selects move with the last bits),
    is that form's own accuracy, bounded at 2.5e-4.  J = avg(<1> - <Phi_1> -
    <Phi_2>) ~ 7e-3 is a difference of O(1) means, so it is held to 1e-4 of
    <1> = 1 (FP32: 7.4e-7)."""
    p = workload.make_adjoint_params(seed=0, precision=prec)
    p["bits"], p["chi_max"] = [4] * 5, 32
    p["dt"] = workload.cfl_dt(p["bits"], p["omega"], p["da"], p["gamma"], p["d_phi"], workload.velocity_bound(p))
    steps = 20
    with pkg.qtt_init(p) as ctx:
        J, g = ctx.grad(steps, 5)
    Jr, gr = oadj.gradient(p, steps)
    rel = np.abs(g - gr) / np.max(np.abs(gr))
    print(f"\n2^4 chi 32 {prec}: J rel {abs(J - Jr) / abs(Jr):.2e}, gradient rel to max {rel.max():.2e}")
    assert abs(J - Jr) <= 1e-4
    assert np.all(rel <= tol), rel


def test_autograd_wrapper():
    torch = pytest.importorskip("torch")
    from paper_2407_09169_gb300.autograd import MeanProduct
    p = exact_params([2, 2, 2, 2, 2])
    names = pkg.grad_param_names(p)
    theta = torch.tensor([oadj.param_value(p, n) for n in names], dtype=torch.float64, requires_grad=True)
    J = MeanProduct.apply(theta, p, 3, 0)
    J.backward()
    with pkg.qtt_init(p) as ctx:
        J2, g2 = ctx.grad(3)
    assert float(J.detach()) == pytest.approx(J2, rel=1e-14)
    assert np.allclose(theta.grad.numpy(), g2, rtol=1e-14, atol=0)
