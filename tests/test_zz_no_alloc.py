"""The allocation-free point evaluation (qtt_observe_points_noalloc, C ABI)
against the allocating one (qtt_observe with QTT_OBS_POINTS), on two calls in
a row and at the exact capacity of its fixed device array.  Callers that
cannot allocate device memory mid-run (a process whose device memory is
entirely held by its own pool allocator, a monitoring loop that cannot pay
cudaFree's device-wide synchronisation) use this entry point.  Collected last
on purpose: it runs after every other test, and also passes when run alone in
a fresh process."""
import ctypes as C
import re

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu
pkg = pytest.importorskip("paper_2407_09169_gb300")

SCRATCH_BYTES = 4 << 20  # the fixed device array of the entry point


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


@pytest.fixture(scope="module")
def lib(gpu_available):
    from paper_2407_09169_gb300 import build
    build.build()
    lib = pkg.load_library()
    lib.qtt_observe_points_noalloc.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int64)]
    lib.qtt_observe_points_noalloc.restype = C.c_int
    return lib


def test_noalloc_points_match_allocating_points(lib):
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


@pytest.mark.parametrize("exact", [0, 1])
def test_noalloc_capacity_boundary(lib, exact):
    """The capacity is floor((4 MiB - 768) / (8 + 8 N + 16 B)), B the largest
    bond of the context (chi_max + oversample when truncating, 2^floor(N/2) in
    exact mode).  Exactly that many points succeed and equal the allocating
    path; one more returns QTT_EINVAL and names the limit."""
    p = workload.make_params("small")
    if exact:
        p["bits"] = [2, 2, 2, 3, 2]
        p["chi_max"], p["svd_rel_tol"], p["exact"] = 2 ** (sum(p["bits"]) // 2), 0.0, 1
    N = sum(p["bits"])
    B = 2 ** (N // 2) if exact else p["chi_max"] + 8
    cap = (SCRATCH_BYTES - 768) // (8 + 8 * N + 16 * B)
    rng = np.random.default_rng(5 + exact)
    with pkg.qtt_init(p) as ctx:
        ctx.step(1)
        st, _ = _noalloc(lib, ctx, np.zeros(N * (cap + 1)))
        assert st == 1
        m = re.search(r"at most (\d+) points", pkg.qtt_last_error(ctx))
        assert m and int(m.group(1)) == cap, pkg.qtt_last_error(ctx)
        idx = np.stack([rng.integers(0, 2 ** b, size=cap) for b in p["bits"]], axis=1)
        ref = ctx.points(idx)
        st, got = _noalloc(lib, ctx, _flags(idx, p["bits"]))
        assert st == 0, pkg.qtt_last_error(ctx)
        assert got.shape == (cap,)
        assert np.abs(got - ref).max() <= 1e-14 * max(np.abs(ref).max(), 1e-300)
