"""Reduced-precision forms (tensor-core contractions, FP32 QR, FP64 Gram and
eigensolver) against the FP64 path at equal chi, and against the oracle."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")


@pytest.fixture(scope="module", autouse=True)
def lib(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    return pkg.load_library()


# Bounds of the current tensor-core forms after 10 steps of the 2^4-point workload
# (chi 32).  The floor ~2e-4 comes from the tensor cores' FP32 accumulation,
# which rounds toward zero (see test_accumulation_bias_is_measured).
@pytest.mark.parametrize("prec,tol", [("bf16x3", 5e-4), ("fp32", 5e-4), ("tf32", 3e-2)])
def test_precision_form_vs_fp64_small(prec, tol):
    p64 = workload.make_params("small")
    pr = workload.make_params("small", precision=prec)
    pr["svd_rel_tol"] = p64["svd_rel_tol"]
    nsteps = 10
    with pkg.qtt_init(p64) as a, pkg.qtt_init(pr) as b:
        a.step(nsteps)
        b.step(nsteps)
        rel = b.compare(a)
        sa, sb = a.scalars(), b.scalars()
        dense_b = b.observe(pkg.OBS_DENSE)
    ref = oracle.solve(p64, nsteps).ravel()
    vs_oracle = float(np.linalg.norm(dense_b - ref) / np.linalg.norm(ref))
    print(f"{prec}: rel-L2 vs fp64 {rel:.2e}, vs oracle {vs_oracle:.2e}, "
          f"norm err {sb['norm_avg'] - 1:.1e}, d<Phi1> {sb['mean1_avg'] - sa['mean1_avg']:.1e}")
    assert rel < tol
    assert abs(sb["norm_avg"] - 1.0) < 2e-2


def test_accumulation_bias_is_measured():
    """Positive operands: the tensor-core product is systematically smaller than
    the FP64 one (mean signed relative error < 0), at the 1e-7..1e-6 level."""
    v = np.array(pkg.qtt_selftest(3)[:-1]).reshape(3, 2, 2, 2)
    means = v[..., 0]
    print("mean signed relative errors:", means.ravel())
    assert np.all(np.abs(v[..., 1]) < 1e-5)
    assert np.all(means < 0) and np.all(means > -5e-6)
