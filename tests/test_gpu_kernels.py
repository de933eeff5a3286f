"""Kernel families on the GPU, through qtt_selftest (C ABI): tensor-core GEMM
modes against the FP64 GEMM, Householder QR, and the eigensolver, each on
seeded random operands including ragged, batched, transposed and split-K shapes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")

MODES = ["bf16x3", "tf32", "tf32x3", "bf16", "bf16x6"]
# per-mode bound on max|C_tc - C_fp64| / max|C_fp64|.  Exact-slice forms: each
# operand element is kept to 2^-16 (2 slices) / 2^-24 (3 slices) of its row's
# (column's) largest power of two, and the dropped slice products are of the
# same order; with rows of Gaussian entries (max ~4 sigma) the error of C is a
# few units of 2^-16 / 2^-24 times 16 relative to max|C|.  TF32X3: 2^-21 plus
# FP32 accumulation; single-pass forms 2^-10 / 2^-7.
TOL = {"bf16x3": 4e-4, "tf32": 4e-3, "tf32x3": 5e-6, "bf16": 3e-2, "bf16x6": 3e-6}


@pytest.fixture(scope="module", autouse=True)
def lib(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    return pkg.load_library()


def test_tensor_core_gemm_modes():
    v = pkg.qtt_selftest(0)
    assert v[-1] == 0, "a bounded wait gave up"
    errs = np.array(v[:-1]).reshape(-1, len(MODES))
    print("\n".join(" ".join(f"{m}={e:.2e}" for m, e in zip(MODES, row)) for row in errs))
    for row in errs:
        for m, e in zip(MODES, row):
            assert 0 <= e <= TOL[m], (m, e)


def test_householder_qr():
    # shape, (FP64 QR, float QR, float QR + one FP64 Newton-Schulz step), (orth, resid)
    v = np.array(pkg.qtt_selftest(1)[:-1]).reshape(-1, 3, 2)
    for case in v:
        (o64, r64), (o32, r32), (ons, rns) = case
        assert o64 < 1e-13 and r64 < 1e-13
        assert o32 < 2e-5 and r32 < 2e-5
        # one step leaves Q^T Q - I = -(3/4) E^2 + O(E^3) for E = Q^T Q - I of
        # the float Q, so max |.| <= (3/4) n max|E|^2 (n <= 256 here), plus the
        # FP64 round-off of two products of length <= 288 (~64 m u <= 2e-12);
        # its span stays the float Q's (residual at the float level)
        assert ons <= 0.75 * 256 * o32 ** 2 + 2e-12 and rns < 2e-5


def test_eigensolver():
    v = np.array(pkg.qtt_selftest(2)[:-1]).reshape(-1, 2, 3)  # size, precision, (res, orth, order)
    for case in v:
        (r64, o64, ord64), (r32, o32, ord32) = case
        assert r64 < 1e-12 and o64 < 1e-12 and ord64 == 0
        assert r32 < 5e-5 and o32 < 5e-5 and ord32 == 0


def test_tensor_core_gemm_large_square():
    """The tensor-core GEMM on square products n = 4096 and 8192 (the shapes
    the contraction kernel reaches its throughput on): sampled entries against
    FP64 dot products, |C - C_fp64| / sum_k |A_ik B_kj|.  BF16: each operand
    rounded to 8 significant bits (2^-8 per product) plus FP32 accumulation
    over K = 8192 (<= K 2^-24 = 4.9e-4): 5e-3.  BF16X3: 16-bit operands
    (2^-16 per product) plus the same accumulation bound: 1e-3."""
    v = np.array(pkg.qtt_selftest(4)[:-1]).reshape(-1, 4)  # n, mode, TFLOP/s, error
    print("\n" + "\n".join(f"n={int(n)} mode={int(m)}: {t:.1f} TFLOP/s, err {e:.2e}" for n, m, t, e in v))
    for n, mode, tflops, err in v:
        assert tflops > 0
        assert 0 <= err <= (5e-3 if int(mode) == 3 else 1e-3), (n, mode, err)
