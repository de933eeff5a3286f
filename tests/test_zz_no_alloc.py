"""The allocation-free point evaluation (qtt_observe_points_noalloc, C ABI)
against the allocating one (qtt_observe with QTT_OBS_POINTS), on two calls in
a row.  Collected last on purpose: it runs after every other test, and also
passes when run alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")


def _flags(idx, bits):
    rows = []
    for row in idx:
        b = []
        for d in range(5):
            b.extend((int(row[d]) >> (bits[d] - 1 - k)) & 1 for k in range(bits[d]))
        rows.append(b)
    return np.ascontiguousarray(np.array(rows, dtype=np.float64).ravel())


def _noalloc(lib, ctx, flags):
    buf = flags.copy()
    written = C.c_int64(0)
    st = lib.qtt_observe_points_noalloc(ctx._h, buf.ctypes.data_as(C.POINTER(C.c_double)), buf.size,
                                        C.byref(written))
    return st, buf[: written.value]


def test_noalloc_points_match_allocating_points(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    lib = pkg.load_library()
    lib.qtt_observe_points_noalloc.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int64)]
    lib.qtt_observe_points_noalloc.restype = C.c_int
    p = workload.make_params("small")
    rng = np.random.default_rng(11)
    with pkg.qtt_init(p) as ctx:
        ctx.step(2)
        for call in range(2):  # two calls in a row share the fixed scratch
            idx = rng.integers(0, 2 ** p["bits"][0], size=(97 + 31 * call, 5))
            ref = ctx.points(idx)
            st, got = _noalloc(lib, ctx, _flags(idx, p["bits"]))
            assert st == 0, pkg.qtt_last_error(ctx)
            assert got.shape == ref.shape
            assert np.abs(got - ref).max() <= 1e-14 * max(np.abs(ref).max(), 1e-300)
        # requests beyond the fixed capacity are rejected with a clear error
        N = sum(p["bits"])
        huge = np.zeros(N * 200000, dtype=np.float64)
        st, _ = _noalloc(lib, ctx, huge)
        assert st == 1 and "at most" in pkg.qtt_last_error(ctx)
