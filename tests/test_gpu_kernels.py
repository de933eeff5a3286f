"""Kernel families on the GPU, through qtt_selftest (C ABI): tensor-core GEMM
modes against the FP64 GEMM, Householder QR, and the eigensolver, each on
seeded random operands including ragged, batched, transposed and split-K shapes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")

MODES = ["bf16x3", "tf32", "tf32x3", "bf16", "bf16x6", "bf16x10"]
# per-mode bound on max|C_tc - C_fp64| / max|C_fp64|.  Exact-slice forms: each
# operand element is kept to 2^-16 (2 slices) / 2^-24 (3 slices) of its row's
# (column's) largest power of two, and the dropped slice products are of the
# same order; with rows of Gaussian entries (max ~4 sigma) the error of C is a
# few units of 2^-16 / 2^-24 times 16 relative to max|C|.  TF32X3: 2^-21 plus
# FP32 accumulation; single-pass forms 2^-10 / 2^-7.
# BF16X10: four slices, 2^-31 of the row maxima: 2^-31 x 16 ~ 1e-8.
TOL = {"bf16x3": 4e-4, "tf32": 4e-3, "tf32x3": 5e-6, "bf16": 3e-2, "bf16x6": 3e-6, "bf16x10": 2e-8}


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
    """Eleven (size, spectrum) cases: the graded Gram matrices at n = 136, 64,
    7, 1, 200, and, with orthonormal eigenvectors, rank 20, a 40-fold
    eigenvalue and a spectrum graded to 1e-30 (the deflation paths of the FP64
    divide and conquer: negligible z components, equal poles rotated together,
    roots far below the largest eigenvalue's precision), and n = 520 (five
    merge levels; the tridiagonalisation in global memory)."""
    v = np.array(pkg.qtt_selftest(2)[:-1]).reshape(-1, 2, 3)  # case, precision, (res, orth, order)
    assert v.shape[0] == 11
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


def _selftest5_cases(v):
    """Split qtt_selftest(5) output into cases (operands as stored, results per mode)."""
    out, i = [], 0
    while i + 8 <= len(v):
        M, N, K, outer, inner, ta, tb, beta = v[i:i + 8]
        i += 8
        M, N, K, b = int(M), int(N), int(K), int(outer) * int(inner)
        take = lambda n: v[i:i + n]
        A = take(M * K * b); i += M * K * b
        B = take(K * N * b); i += K * N * b
        C0 = take(M * N * b); i += M * N * b
        Cs = []
        for _ in MODES:
            Cs.append(take(M * N * b).reshape(b, M, N)); i += M * N * b
        A = A.reshape(b, K, M).transpose(0, 2, 1) if ta else A.reshape(b, M, K)
        B = B.reshape(b, N, K).transpose(0, 2, 1) if tb else B.reshape(b, K, N)
        out.append((K, beta, A, B, C0.reshape(b, M, N), Cs))
    return out


def test_tensor_core_gemm_against_host_fp64():
    """Every tensor-core mode against a numpy FP64 product of the same seeded
    operands (a long K with split-K, 34 row tiles, a batched product with a
    transposed A and beta, both operands transposed with beta = 1), as
    e = |C_tc - C| / (|alpha| sum_k |a_ik b_kj| + |beta| |c0_ij|).  Bounds from
    the arithmetic: operand representation (unit roundoff of BF16 2^-8 per
    operand, TF32 2^-11; the hi/lo splits leave 2^-16 (BF16X3) / 2^-22
    (TF32X3) per operand plus the dropped lo*lo term of the same size) plus
    FP32 accumulation, at most one rounding of 2^-23 per
    tensor-core instruction (K / 16 of them for BF16, K / 8 for TF32); the
    exact-slice forms accumulate exactly and keep each element to three (BF16X6)
    or four (BF16X10) 8-bit slices of its row's (column's) largest power of
    two, which for Gaussian rows (largest / mean magnitude below 5) is below
    3 * 2^-24 * 25 = 4.5e-6 (BF16X6) and 2^-7 of that (BF16X10) of sum |a b|.  A wrong index, transpose or packing
    gives O(1) errors.  The signed mean errors of the unbiased exact-slice
    forms must also stay far below their bounds."""
    v = np.asarray(pkg.qtt_selftest(5, cap=12_000_000))
    assert v[-1] == 0, "a bounded wait gave up"
    cases = _selftest5_cases(v[:-1])
    assert len(cases) == 4
    alpha, u = 1.5, 2.0 ** -23
    for K, beta, A, B, C0, Cs in cases:
        ref = alpha * np.matmul(A, B) + beta * C0
        mag = abs(alpha) * np.matmul(np.abs(A), np.abs(B)) + abs(beta) * np.abs(C0)
        bound = {"bf16x3": 3 * 2.0 ** -16 + (K / 16) * u, "tf32": 2 * 2.0 ** -11 + (K / 8) * u,
                 "tf32x3": 3 * 2.0 ** -22 + (K / 8) * u, "bf16": 2 * 2.0 ** -8 + (K / 16) * u, "bf16x6": 4.5e-6,
                 "bf16x10": 4.5e-6 * 2.0 ** -7}
        for m, C in zip(MODES, Cs):
            assert not np.isnan(C).any(), (m, K)
            e = (C - ref) / mag
            print(f"K={K} {m}: max {np.abs(e).max():.2e} (bound {bound[m]:.1e}), mean {e.mean():.1e}")
            assert np.abs(e).max() <= bound[m], (m, K, np.abs(e).max())
        for m in ("bf16x6", "bf16x10"):
            em = (Cs[MODES.index(m)] - ref) / mag
            assert abs(em.mean()) <= 0.05 * bound[m]


def test_fp64_throughput_probe():
    """DFMA and f64 mma.sync throughput of the whole GPU (the FP64 roofline's
    denominator): both positive and below the nominal FP64 rate of a GB300
    by a wide margin from above (no probe can beat the hardware: 2 TFLOP/s)."""
    v = pkg.qtt_selftest(6)
    dfma, dmma, sms, blocks = v[:4]
    print(f"\nFP64: DFMA {dfma:.3f} TFLOP/s, DMMA {dmma:.3f} TFLOP/s on {int(sms)} SMs ({int(blocks)} blocks)")
    assert 0.05 < dfma < 2.0 and 0.05 < dmma < 2.0
