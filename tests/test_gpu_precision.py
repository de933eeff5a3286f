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


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("fp32", 1e-5), ("tf32", 5e-3)])
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
    assert abs(sb["norm_avg"] - 1.0) < 1e-3
