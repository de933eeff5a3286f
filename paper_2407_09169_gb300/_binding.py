"""ctypes binding of libqtt_fp.so (argument marshalling only).

The names follow the C ABI in include/qtt_fp.h.  Every computation runs in
the library's CUDA kernels; when the library is missing or no GPU is
present, the calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqtt_fp.so")

QTT_OK, QTT_EINVAL, QTT_ENOMEM, QTT_ECUDA, QTT_ENOCONV, QTT_ETIMEOUT, QTT_ENAN, QTT_ESTATE, QTT_EIO = range(9)
STATUS_NAMES = ["QTT_OK", "QTT_EINVAL", "QTT_ENOMEM", "QTT_ECUDA", "QTT_ENOCONV", "QTT_ETIMEOUT", "QTT_ENAN",
                "QTT_ESTATE", "QTT_EIO"]
OBS_SCALARS, OBS_BONDS, OBS_DENSE, OBS_MEANS, OBS_POINTS, OBS_NVPP, OBS_TIMINGS, OBS_ERRORS = range(8)
SCALAR_NAMES = ["time", "norm_avg", "mean1_avg", "mean2_avg", "phi11_avg", "phi22_avg", "phi12_avg", "R12", "Y12",
                "product_J", "discarded_weight", "steps", "norm2"]


class QttError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


class QttParams(C.Structure):
    _fields_ = [
        ("bits", C.c_int32 * 5),
        ("chi_max", C.c_int32),
        ("svd_rel_tol", C.c_double),
        ("precision", C.c_int32),
        ("oversample", C.c_int32),
        ("exact", C.c_int32),
        ("seed", C.c_uint64),
        ("omega", C.c_double),
        ("da", C.c_double),
        ("gamma", C.c_double),
        ("d_phi", C.c_double),
        ("dt", C.c_double),
        ("shear_amp", C.c_double),
        ("n_umodes", C.c_int32),
        ("umode_comp", C.POINTER(C.c_int32)),
        ("umode_k", C.POINTER(C.c_int32)),
        ("umode_phase", C.POINTER(C.c_double)),
        ("umode_amp", C.POINTER(C.c_double)),
        ("ic_sigma", C.c_double),
        ("ic_blend_width", C.c_double),
        ("ic_c_hi", C.c_double * 2),
        ("ic_c_lo", C.c_double * 2),
        ("n_icmodes", C.c_int32),
        ("icmode_k", C.POINTER(C.c_int32)),
        ("icmode_phase", C.POINTER(C.c_double)),
        ("icmode_amp", C.POINTER(C.c_double)),
        ("rk_variant", C.c_int32),
        ("flow", C.c_int32),
        ("u0", C.c_double),
        ("ic_kind", C.c_int32),
        ("sgs", C.c_int32),
        ("c_s", C.c_double),
        ("c_omega", C.c_double),
        ("delta_cells", C.c_double),
        ("moment_ref", C.c_int32),
        ("stream", C.c_void_p),
    ]


_lib = None


def load_library(path: str | None = None):
    """Loads libqtt_fp.so (built by paper_2407_09169_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise QttError(QTT_ESTATE, f"{path} is missing: build it with paper_2407_09169_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.qtt_init.argtypes = [P(QttParams), P(C.c_void_p)]
    lib.qtt_step.argtypes = [C.c_void_p, C.c_int32]
    lib.qtt_step_many.argtypes = [P(C.c_void_p), C.c_int32, C.c_int32, P(C.c_int32)]
    lib.qtt_grad.argtypes = [C.c_void_p, C.c_int32, C.c_int32, P(C.c_double), C.c_int64, P(C.c_int64)]
    lib.qtt_observe.argtypes = [C.c_void_p, C.c_int32, P(C.c_double), C.c_int64, P(C.c_int64)]
    lib.qtt_compare.argtypes = [C.c_void_p, C.c_void_p, P(C.c_double)]
    lib.qtt_save.argtypes = [C.c_void_p, C.c_char_p]
    lib.qtt_load.argtypes = [C.c_void_p, C.c_char_p]
    lib.qtt_destroy.argtypes = [C.c_void_p]
    lib.qtt_destroy.restype = None
    lib.qtt_last_error.argtypes = [C.c_void_p]
    lib.qtt_last_error.restype = C.c_char_p
    lib.qtt_version.argtypes = []
    lib.qtt_version.restype = C.c_char_p
    lib.qtt_host_dense.argtypes = [P(QttParams), C.c_int32, P(C.c_double), C.c_int64, P(C.c_int64)]
    lib.qtt_selftest.argtypes = [C.c_int32, P(C.c_double), C.c_int64, P(C.c_int64)]
    lib.qtt_truncate_vjp.argtypes = [C.c_int32, P(C.c_int32), C.c_void_p, P(C.c_int32), C.c_void_p, C.c_int32,
                                     C.c_double, C.c_double, C.c_void_p, C.c_int64, P(C.c_int64), P(C.c_int32),
                                     C.c_void_p]
    for fn in ("qtt_init", "qtt_step", "qtt_step_many", "qtt_grad", "qtt_observe", "qtt_compare", "qtt_save", "qtt_load", "qtt_host_dense",
               "qtt_selftest", "qtt_truncate_vjp"):
        getattr(lib, fn).restype = C.c_int
    _lib = lib
    return lib


def make_c_params(p: dict, stream=None):
    """Packs a parameter dictionary (see workload.make_params) into QttParams.
    Returns (struct, keepalive) -- keep both alive during the call."""
    cp = QttParams()
    for d in range(5):
        cp.bits[d] = int(p["bits"][d])
    cp.chi_max = int(p["chi_max"])
    cp.svd_rel_tol = float(p.get("svd_rel_tol", 0.0))
    cp.precision = int(p.get("precision", 0))
    cp.oversample = int(p.get("oversample", 8))
    cp.exact = int(p.get("exact", 0))
    cp.seed = int(p.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    for key in ("omega", "da", "gamma", "d_phi", "dt", "shear_amp", "ic_sigma", "ic_blend_width"):
        setattr(cp, key, float(p[key]))
    um = p.get("umodes", [])
    comp = np.ascontiguousarray([m["comp"] for m in um] or [0], dtype=np.int32)
    kk = np.ascontiguousarray([v for m in um for v in m["k"]] or [0, 0, 0], dtype=np.int32)
    ph = np.ascontiguousarray([m["phase"] for m in um] or [0.0], dtype=np.float64)
    am = np.ascontiguousarray([m["amp"] for m in um] or [0.0], dtype=np.float64)
    cp.n_umodes = len(um)
    cp.umode_comp = comp.ctypes.data_as(C.POINTER(C.c_int32))
    cp.umode_k = kk.ctypes.data_as(C.POINTER(C.c_int32))
    cp.umode_phase = ph.ctypes.data_as(C.POINTER(C.c_double))
    cp.umode_amp = am.ctypes.data_as(C.POINTER(C.c_double))
    for i in range(2):
        cp.ic_c_hi[i] = float(p["ic_c_hi"][i])
        cp.ic_c_lo[i] = float(p["ic_c_lo"][i])
    im = p.get("icmodes", [])
    ik = np.ascontiguousarray([v for m in im for v in m["k"]] or [0, 0, 0], dtype=np.int32)
    iph = np.ascontiguousarray([m["phase"] for m in im] or [0.0], dtype=np.float64)
    iam = np.ascontiguousarray([m["amp"] for m in im] or [0.0], dtype=np.float64)
    cp.n_icmodes = len(im)
    cp.icmode_k = ik.ctypes.data_as(C.POINTER(C.c_int32))
    cp.icmode_phase = iph.ctypes.data_as(C.POINTER(C.c_double))
    cp.icmode_amp = iam.ctypes.data_as(C.POINTER(C.c_double))
    cp.rk_variant = int(p.get("rk_variant", 0))
    cp.flow = int(p.get("flow", 0))
    cp.u0 = float(p.get("u0", 1.0))
    cp.ic_kind = int(p.get("ic_kind", 0))
    cp.sgs = int(p.get("sgs", 0))
    cp.c_s = float(p.get("c_s", 0.11))
    cp.c_omega = float(p.get("c_omega", 0.5))
    cp.delta_cells = float(p.get("delta_cells", 3.0))
    cp.moment_ref = int(p.get("moment_ref", 0))
    cp.stream = C.c_void_p(int(stream) if stream else 0)
    return cp, (comp, kk, ph, am, ik, iph, iam)


def qtt_version() -> str:
    return load_library().qtt_version().decode()


def qtt_last_error(ctx=None) -> str:
    h = ctx._h if isinstance(ctx, Context) else ctx
    return load_library().qtt_last_error(h).decode(errors="replace")


def _check(status: int, ctx_handle=None):
    if status != QTT_OK:
        raise QttError(status, load_library().qtt_last_error(ctx_handle).decode(errors="replace"))


class Context:
    """A PDF being stepped on the GPU (one qtt_ctx)."""

    def __init__(self, params: dict, stream=None):
        lib = load_library()
        cp, keep = make_c_params(params, stream)
        h = C.c_void_p()
        _check(lib.qtt_init(C.byref(cp), C.byref(h)), None)
        del keep
        self._h = h
        self.params = dict(params)
        self.N = int(sum(params["bits"]))

    def _handle(self):
        if self._h is None:
            raise QttError(QTT_ESTATE, "context destroyed")
        return self._h

    def step(self, nsteps: int = 1):
        _check(load_library().qtt_step(self._handle(), int(nsteps)), self._h)

    def grad(self, nsteps: int, ckpt_every: int = 0):
        """(J, dJ/dtheta) after nsteps Heun steps from the initial PDF; theta in
        the order of grad_param_names(params).  Leaves the context at the final state."""
        n = 1 + len(grad_param_names(self.params))
        out = np.zeros(n, dtype=np.float64)
        written = C.c_int64(0)
        _check(load_library().qtt_grad(self._handle(), int(nsteps), int(ckpt_every),
                                       out.ctypes.data_as(C.POINTER(C.c_double)), out.size, C.byref(written)),
               self._h)
        return float(out[0]), out[1:written.value].copy()

    def observe(self, what: int, cap: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        Kx = sum(self.params["bits"][2:])
        if out is None:
            if cap is None:
                cap = {OBS_SCALARS: len(SCALAR_NAMES), OBS_BONDS: self.N + 1, OBS_DENSE: 2 ** self.N,
                       OBS_MEANS: 3 * 2 ** Kx, OBS_NVPP: 1, OBS_TIMINGS: 20, OBS_ERRORS: 6}[what]
            out = np.zeros(cap, dtype=np.float64)
        written = C.c_int64(0)
        _check(load_library().qtt_observe(self._handle(), int(what), out.ctypes.data_as(C.POINTER(C.c_double)),
                                          out.size, C.byref(written)), self._h)
        return out[: written.value]

    def scalars(self) -> dict:
        v = self.observe(OBS_SCALARS)
        return dict(zip(SCALAR_NAMES, v.tolist()))

    def points(self, idx: np.ndarray) -> np.ndarray:
        """f at multi-indices idx[p] = (i1, i2, j1, j2, j3)."""
        idx = np.atleast_2d(np.asarray(idx, dtype=np.int64))
        bits = self.params["bits"]
        rows = []
        for row in idx:
            b = []
            for d in range(5):
                b.extend((int(row[d]) >> (bits[d] - 1 - k)) & 1 for k in range(bits[d]))
            rows.append(b)
        buf = np.ascontiguousarray(np.array(rows, dtype=np.float64).ravel())
        return self.observe(OBS_POINTS, out=buf).copy()

    def compare(self, other: "Context") -> float:
        r = C.c_double(0.0)
        _check(load_library().qtt_compare(self._handle(), other._handle(), C.byref(r)), self._h)
        return r.value

    def save(self, path: str):
        _check(load_library().qtt_save(self._handle(), path.encode()), self._h)

    def load(self, path: str):
        _check(load_library().qtt_load(self._handle(), path.encode()), self._h)

    def close(self):
        if self._h is not None:
            load_library().qtt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# C-ABI-named functional wrappers
def qtt_init(params: dict, stream=None) -> Context:
    return Context(params, stream)


def qtt_step(ctx: Context, nsteps: int = 1):
    ctx.step(nsteps)


def qtt_step_many(ctxs, nsteps: int = 1):
    """Advances every context of the sequence by nsteps, concurrently on the GPU."""
    ctxs = list(ctxs)
    arr = (C.c_void_p * max(1, len(ctxs)))(*[c._handle() for c in ctxs])
    failed = C.c_int32(-1)
    st = load_library().qtt_step_many(arr, len(ctxs), int(nsteps), C.byref(failed))
    if st != QTT_OK:
        i = failed.value
        _check(st, ctxs[i]._h if 0 <= i < len(ctxs) else None)


def grad_param_names(params: dict) -> list:
    """Order of the gradient of qtt_grad: omega, da, gamma, umode<i>, icmode<i>."""
    return (["omega", "da", "gamma"] + [f"umode{i}" for i in range(len(params.get("umodes") or []))]
            + [f"icmode{i}" for i in range(len(params.get("icmodes") or []))])


def qtt_grad(ctx: Context, nsteps: int, ckpt_every: int = 0):
    return ctx.grad(nsteps, ckpt_every)


def qtt_observe(ctx: Context, what: int, cap: int | None = None) -> np.ndarray:
    return ctx.observe(what, cap)


def qtt_compare(a: Context, b: Context) -> float:
    return a.compare(b)


def qtt_save(ctx: Context, path: str):
    ctx.save(path)


def qtt_load(ctx: Context, path: str):
    ctx.load(path)


def qtt_destroy(ctx: Context):
    ctx.close()


def qtt_host_dense(params: dict, which: int, cap: int) -> np.ndarray:
    """Host-only dense expansion of an encoded object (no GPU needed)."""
    lib = load_library()
    cp, keep = make_c_params(params)
    out = np.zeros(cap, dtype=np.float64)
    written = C.c_int64(0)
    _check(lib.qtt_host_dense(C.byref(cp), int(which), out.ctypes.data_as(C.POINTER(C.c_double)), cap,
                              C.byref(written)), None)
    del keep
    return out[: written.value]


def qtt_selftest(which: int, cap: int = 4096) -> np.ndarray:
    """Device self-checks of the kernel families (see include/qtt_fp.h)."""
    lib = load_library()
    out = np.zeros(cap, dtype=np.float64)
    written = C.c_int64(0)
    _check(lib.qtt_selftest(int(which), out.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(written)), None)
    return out[: written.value]


def _device_ptr(t, name: str) -> int:
    """Device address of a contiguous float64 CUDA tensor (or a raw int)."""
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise QttError(QTT_EINVAL, f"{name} must be a contiguous float64 CUDA tensor")
    return t.data_ptr()


def qtt_truncate_vjp(rx, x, sy, ybar, chi: int, tol: float, eps: float, xbar, cap: int, stream=None):
    """Backward of the bond truncation (see include/qtt_fp.h): x, ybar, xbar
    are device buffers (CUDA tensors or addresses), rx and sy the bond lists.
    Returns (doubles written, kept counts)."""
    lib = load_library()
    rx = [int(v) for v in rx]
    sy = [int(v) for v in sy]
    N = len(rx) - 1
    if len(sy) != N + 1:
        raise QttError(QTT_EINVAL, "rx and sy must have the same length")
    rxa = (C.c_int32 * len(rx))(*rx)
    sya = (C.c_int32 * len(sy))(*sy)
    kept = (C.c_int32 * max(N - 1, 1))()
    written = C.c_int64(0)
    st = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    _check(lib.qtt_truncate_vjp(N, rxa, C.c_void_p(_device_ptr(x, "x")), sya, C.c_void_p(_device_ptr(ybar, "ybar")),
                                int(chi), float(tol), float(eps), C.c_void_p(_device_ptr(xbar, "xbar")), int(cap),
                                C.byref(written), kept, st), None)
    return written.value, [kept[i] for i in range(N - 1)]
