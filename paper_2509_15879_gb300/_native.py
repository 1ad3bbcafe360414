"""ctypes binding of libpolar.so: argument marshalling only.

Every function carries the name of the C entry point it wraps (``include/polar.h``).
Arrays are numpy float64 arrays (host memory) or CUDA tensors exposing ``data_ptr()``
(device memory; torch supplies the memory, the library never allocates for them).
The library has no CPU fallback: loading fails loudly if libpolar.so is missing.
"""
import ctypes as C
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolar.so")

POLAR_OK, POLAR_EINVAL, POLAR_ENOMEM, POLAR_ECUDA = 0, -1, -2, -3
POLAR_ENOCONV, POLAR_ENONFINITE, POLAR_ESTATE = -4, -5, -7
POLAR_SCHEME_CONSERVATIVE, POLAR_SCHEME_PAPER = 0, 1
POLAR_FP64, POLAR_MIXED = 0, 1
POLAR_HOST, POLAR_DEVICE = 0, 1

_dp = C.POINTER(C.c_double)


# device-memory hooks of polar_mesh_desc: alloc(bytes, stream, user) -> ptr, free(ptr, stream, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class polar_mesh_desc(C.Structure):
    _fields_ = [("nr", C.c_int32), ("ntheta", C.c_int32), ("r", _dp), ("theta", _dp),
                ("scheme", C.c_int32), ("precision", C.c_int32), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class polar_coeffs(C.Structure):
    _fields_ = [("memory", C.c_int32), ("d_rface", C.c_void_p), ("d_tface", C.c_void_p),
                ("v_rface", C.c_void_p), ("v_tface", C.c_void_p), ("e_node", C.c_void_p),
                ("b", C.c_void_p), ("d_const", C.c_double), ("b_const", C.c_double),
                ("d0", C.c_double), ("nsrc", C.c_int32), ("src", C.c_void_p * 4),
                ("bnd", C.c_void_p * 4)]


POLAR_SOLVE_AUTO, POLAR_SOLVE_KRYLOV, POLAR_SOLVE_DIRECT = 0, 1, 2


class polar_solver_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("max_refine", C.c_int32),
                ("inner_tol", C.c_double), ("method", C.c_int32), ("reserved", C.c_int32)]


class polar_step_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("status", C.c_int32),
                ("fp64_iters", C.c_int32), ("scaled_resid", C.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, refinements=self.refinements, status=self.status,
                    fp64_iters=self.fp64_iters, scaled_resid=self.scaled_resid)


class polar_gummel_desc(C.Structure):
    _fields_ = [("mobility", C.c_double * 2), ("src_electrons", C.c_int32),
                ("src_holes", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("depth", C.c_int32)]


class polar_gummel_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("change", C.c_double),
                ("phi", polar_step_stats), ("carrier", polar_step_stats * 2)]

    def as_dict(self):
        return dict(iters=self.iters, status=self.status, change=self.change,
                    phi=self.phi.as_dict(),
                    carrier=[self.carrier[0].as_dict(), self.carrier[1].as_dict()])


class PolarError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"polar error {code}: {msg}")
        self.code = code


_lib = None

EXPORTS = {
    "polar_mesh_create": (C.c_int, [C.POINTER(polar_mesh_desc), C.POINTER(C.c_void_p)]),
    "polar_mesh_destroy": (C.c_int, [C.c_void_p]),
    "polar_set_coeffs": (C.c_int, [C.c_void_p, C.POINTER(polar_coeffs)]),
    "polar_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32]),
    "polar_get_state": (C.c_int, [C.c_void_p, C.c_void_p, _dp, C.c_int32]),
    "polar_step": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _dp, _dp,
                             C.POINTER(polar_solver_opts), C.POINTER(polar_step_stats)]),
    "polar_advance": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_double, _dp,
                                C.POINTER(polar_solver_opts), C.POINTER(polar_step_stats)]),
    "polar_apply_operator": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_void_p,
                                       C.c_void_p, C.c_int32]),
    "polar_kernel_launches": (C.c_int64, [C.c_void_p]),
    "polar_is_separable": (C.c_int, [C.c_void_p]),
    "polar_apply_rows_noalloc": (C.c_int, [C.c_int32, C.c_int32] + [C.c_void_p] * 6 +
                                 [C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "polar_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "polar_batch_destroy": (C.c_int, [C.c_void_p]),
    "polar_batch_kernel_launches": (C.c_int64, [C.c_void_p]),
    "polar_batch_advance": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(_dp), _dp, C.POINTER(_dp),
                                      C.POINTER(polar_solver_opts), C.POINTER(polar_step_stats)]),
    "polar_solve_steady": (C.c_int, [C.c_void_p, _dp, C.POINTER(polar_solver_opts),
                                     C.POINTER(polar_step_stats)]),
    "polar_face_drift": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int32]),
    "polar_gummel_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(polar_gummel_desc), C.POINTER(C.c_void_p)]),
    "polar_gummel_step": (C.c_int, [C.c_void_p, _dp, C.c_double, C.POINTER(_dp), _dp,
                                    C.POINTER(polar_solver_opts), C.POINTER(polar_gummel_stats)]),
    "polar_gummel_destroy": (C.c_int, [C.c_void_p]),
    "polar_timing_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "polar_timing_flops": (C.c_int, [C.c_void_p, C.c_int32, _dp]),
    "polar_timing_query": (C.c_int, [C.c_void_p, C.c_int32, C.c_char_p, C.c_size_t,
                                     C.POINTER(C.c_int64), _dp, _dp]),
    "polar_last_error": (C.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Loads libpolar.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "python -m paper_2509_15879_gb300.build")
        lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != POLAR_OK:
        raise PolarError(rc, load().polar_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Arr:
    """Holds a pointer to caller data and keeps the owner alive.

    ``count`` is the number of doubles the C call reads or writes through the pointer:
    every array must be float64, contiguous and hold at least that many.  CUDA tensors must
    live on the current device.  ``out`` marks an array the call writes: it is used in
    place, so a numpy array that would need a converted copy is rejected instead of being
    copied (the result would land in the copy).  Violations raise ValueError before the
    library is called."""

    def __init__(self, a, count, name="array", out=False):
        self.ptr, self.keep, self.device = None, None, None
        if a is None:
            return
        if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):   # torch tensor
            if str(a.dtype) != "torch.float64":
                raise ValueError(f"{name}: tensors must be float64, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError(f"{name}: tensors must be contiguous")
            if a.numel() < count:
                raise ValueError(f"{name}: needs {count} values, the tensor holds {a.numel()}")
            if getattr(a, "is_cuda", False):
                import torch
                if a.device.index != torch.cuda.current_device():
                    raise ValueError(f"{name}: tensor on cuda:{a.device.index}, but the "
                                     f"current device is cuda:{torch.cuda.current_device()}")
                self.device = True
            else:
                self.device = False          # host tensor (e.g. pinned): used in place
            self.ptr, self.keep = a.data_ptr(), a
            return
        if out:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and
                    a.flags.c_contiguous and a.flags.writeable):
                raise ValueError(f"{name}: outputs must be writable contiguous float64 arrays")
            arr = a
        else:
            arr = _f64(a)
        if arr.size < count:
            raise ValueError(f"{name}: needs {count} values, the array holds {arr.size}")
        self.ptr, self.keep, self.device = arr.ctypes.data, arr, False


class Ctx:
    """Handle of a polar_ctx; destroyed with the object or by polar_mesh_destroy.  It keeps
    the allocator hooks the context was created with alive as long as the context."""

    def __init__(self, handle, m, n, hooks=None):
        self.handle, self.m, self.n, self.hooks = handle, m, n, hooks

    @property
    def N(self):
        return self.m * self.n + 1

    def __del__(self):
        # at interpreter exit the allocator behind the hooks may already be gone: the
        # process ends and its device memory with it
        if getattr(self, "handle", None) and _lib is not None and not sys.is_finalizing():
            _lib.polar_mesh_destroy(self.handle)
            self.handle = None


class TorchAllocator:
    """Device memory of a context from PyTorch's caching allocator (the library's buffers
    join torch's memory pool; torch keeps freed blocks cached for reuse)."""

    def alloc(self, nbytes, stream):
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  int(stream or 0))

    def free(self, ptr, stream):
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))


def _hooks(allocator):
    """(alloc, free) ctypes callbacks of an allocator object with alloc(nbytes, stream) ->
    int pointer and free(ptr, stream); null callbacks for None (the library's cudaMalloc)."""
    if allocator is None:
        return ALLOC_FN(), FREE_FN()

    def a(nbytes, stream, user):
        return int(allocator.alloc(nbytes, stream)) or None

    def f(ptr, stream, user):
        allocator.free(ptr, stream)

    return ALLOC_FN(a), FREE_FN(f)


def polar_mesh_create(r, theta, scheme=POLAR_SCHEME_CONSERVATIVE, precision=POLAR_FP64,
                      stream=None, allocator=None) -> Ctx:
    """``allocator``: None (the library allocates with cudaMalloc), "torch" (PyTorch's
    caching allocator) or an object with alloc(nbytes, stream) and free(ptr, stream)."""
    lib = load()
    r, theta = _f64(r), _f64(theta)
    if allocator == "torch":
        allocator = TorchAllocator()
    fa, ff = _hooks(allocator)
    d = polar_mesh_desc(len(r) - 2, len(theta), r.ctypes.data_as(_dp), theta.ctypes.data_as(_dp),
                        scheme, precision, stream, fa, ff, None)
    h = C.c_void_p()
    _check(lib.polar_mesh_create(C.byref(d), C.byref(h)))
    return Ctx(h, len(r) - 2, len(theta), (fa, ff, allocator))


def polar_mesh_destroy(ctx: Ctx):
    if ctx.handle:
        _check(load().polar_mesh_destroy(ctx.handle))
        ctx.handle = None


def polar_set_coeffs(ctx: Ctx, d_rface=None, d_tface=None, v_rface=None, v_tface=None,
                     e_node=None, b=None, d_const=1.0, b_const=0.0, d0=1.0, src=(), bnd=()):
    m, n, N = ctx.m, ctx.n, ctx.N
    if len(src) != len(bnd) or len(src) > 4:
        raise ValueError("src and bnd must have the same length, at most 4")
    sizes = ((m + 1) * n, m * n, (m + 1) * n, m * n, N, N)
    names = ("d_rface", "d_tface", "v_rface", "v_tface", "e_node", "b")
    arrs = [_Arr(x, c, nm) for x, c, nm in zip((d_rface, d_tface, v_rface, v_tface, e_node, b),
                                                sizes, names)]
    srcs = [_Arr(x, N, f"src[{q}]") for q, x in enumerate(src)]
    bnds = [_Arr(x, n, f"bnd[{q}]") for q, x in enumerate(bnd)]
    kinds = {a.device for a in arrs + srcs + bnds if a.ptr is not None}
    if len(kinds) > 1:
        raise ValueError("all coefficient arrays must live in the same memory")
    mem = POLAR_DEVICE if kinds == {True} else POLAR_HOST
    c = polar_coeffs()
    c.memory = mem
    c.d_rface, c.d_tface, c.v_rface, c.v_tface, c.e_node, c.b = [a.ptr for a in arrs]
    c.d_const, c.b_const, c.d0 = float(d_const), float(b_const), float(d0)
    c.nsrc = len(srcs)
    for q in range(len(srcs)):
        c.src[q] = srcs[q].ptr
        c.bnd[q] = bnds[q].ptr
    _check(load().polar_set_coeffs(ctx.handle, C.byref(c)))


def polar_set_state(ctx: Ctx, u, t: float):
    a = _Arr(u, ctx.N, "u")
    _check(load().polar_set_state(ctx.handle, a.ptr, float(t),
                                  POLAR_DEVICE if a.device else POLAR_HOST))


def polar_get_state(ctx: Ctx, out=None):
    """Returns (u, t); u is a new numpy array unless ``out`` (host or device) is given."""
    if out is None:
        out = np.empty(ctx.N, dtype=np.float64)
    a = _Arr(out, ctx.N, "out", out=True)
    t = C.c_double()
    _check(load().polar_get_state(ctx.handle, a.ptr, C.byref(t),
                                  POLAR_DEVICE if a.device else POLAR_HOST))
    return out, t.value


def _opts(opts):
    if opts is None:
        return None
    o = polar_solver_opts(opts.get("tol", 0.0), opts.get("max_iter", 0),
                          opts.get("max_refine", 0), opts.get("inner_tol", 0.0),
                          opts.get("method", POLAR_SOLVE_AUTO), 0)
    return C.byref(o)


def polar_step(ctx: Ctx, dt, theta, w_old=(), w_new=(), opts=None):
    wo, wn = _f64(w_old), _f64(w_new)
    st = polar_step_stats()
    rc = load().polar_step(ctx.handle, float(dt), float(theta), wo.ctypes.data_as(_dp),
                           wn.ctypes.data_as(_dp), _opts(opts), C.byref(st))
    _check(rc)
    return st.as_dict()


def polar_advance(ctx: Ctx, t, theta, w=None, opts=None, check=True):
    t = _f64(t)
    K = len(t) - 1
    w = np.zeros((K + 1, 0)) if w is None else _f64(w)
    stats = (polar_step_stats * max(K, 1))()
    rc = load().polar_advance(ctx.handle, K, t.ctypes.data_as(_dp), float(theta),
                              w.ctypes.data_as(_dp), _opts(opts), stats)
    if check:
        _check(rc)
    return [stats[k].as_dict() for k in range(K)], rc


def polar_apply_operator(ctx: Ctx, alpha, beta, x, out=None):
    if out is None:
        out = np.empty(ctx.N, dtype=np.float64)
    ax, ay = _Arr(x, ctx.N, "x"), _Arr(out, ctx.N, "out", out=True)
    if ax.device != ay.device:
        raise ValueError("x and y must live in the same memory")
    _check(load().polar_apply_operator(ctx.handle, float(alpha), float(beta), ax.ptr, ay.ptr,
                                       POLAR_DEVICE if ax.device else POLAR_HOST))
    return out


def polar_apply_rows_noalloc(m, n, R, W, E, S, N, o, alpha, beta, x, y, stream=None):
    """y = alpha x + beta L x from caller-held device rows (torch CUDA tensors); allocates
    nothing on the device."""
    m, n = int(m), int(n)
    Np = m * n + 1
    arrs = [_Arr(a, c, nm, out=(nm == "y")) for a, c, nm in
            zip((R, W, E, S, N, o, x, y), (Np,) * 5 + (n, Np, Np),
                ("R", "W", "E", "S", "N", "o", "x", "y"))]
    if not all(a.device for a in arrs):
        raise ValueError("polar_apply_rows_noalloc takes device arrays only")
    _check(load().polar_apply_rows_noalloc(int(m), int(n), *[a.ptr for a in arrs[:6]],
                                           float(alpha), float(beta), arrs[6].ptr, arrs[7].ptr,
                                           stream))


def polar_kernel_launches(ctx: Ctx) -> int:
    return int(load().polar_kernel_launches(ctx.handle))


def polar_is_separable(ctx: Ctx) -> bool:
    rc = load().polar_is_separable(ctx.handle)
    if rc < 0:
        _check(rc)
    return rc == 1


class Batch:
    """Handle of a polar_batch over a list of contexts (kept alive with it)."""

    def __init__(self, handle, ctxs):
        self.handle, self.ctxs = handle, list(ctxs)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.polar_batch_destroy(self.handle)
            self.handle = None


def polar_batch_create(ctxs, stream=None) -> Batch:
    arr = (C.c_void_p * len(ctxs))(*[c.handle.value if isinstance(c.handle, C.c_void_p) else c.handle
                                      for c in ctxs])
    h = C.c_void_p()
    _check(load().polar_batch_create(arr, len(ctxs), stream, C.byref(h)))
    return Batch(h, ctxs)


def polar_batch_kernel_launches(batch: Batch) -> int:
    return int(load().polar_batch_kernel_launches(batch.handle))


def polar_batch_destroy(batch: Batch):
    if batch.handle:
        _check(load().polar_batch_destroy(batch.handle))
        batch.handle = None


def polar_batch_advance(batch: Batch, ts, thetas, ws=None, opts=None, check=True):
    """Advances every instance over its own time levels ts[i] (same number of steps);
    returns (stats[i][k] dicts, rc)."""
    count = len(batch.ctxs)
    ts = [_f64(t) for t in ts]
    K = len(ts[0]) - 1
    if any(len(t) != K + 1 for t in ts):
        raise ValueError("every instance needs the same number of steps")
    tptr = (_dp * count)(*[t.ctypes.data_as(_dp) for t in ts])
    th = _f64(thetas)
    keep = []
    wptr = None
    if ws is not None:
        ws = [_f64(w) if w is not None else np.zeros(1) for w in ws]
        keep = ws
        wptr = (_dp * count)(*[w.ctypes.data_as(_dp) for w in ws])
    stats = (polar_step_stats * max(count * K, 1))()
    rc = load().polar_batch_advance(batch.handle, K, tptr, th.ctypes.data_as(_dp), wptr,
                                    _opts(opts), stats)
    del keep
    if check:
        _check(rc)
    return [[stats[i * K + k].as_dict() for k in range(K)] for i in range(count)], rc


def polar_solve_steady(ctx: Ctx, w=(), opts=None):
    """Solves L U = f (sources weighted by w) into the context's state; returns the stats."""
    w = _f64(w)
    st = polar_step_stats()
    _check(load().polar_solve_steady(ctx.handle, w.ctypes.data_as(_dp), _opts(opts),
                                     C.byref(st)))
    return st.as_dict()


def polar_face_drift(ctx: Ctx, mobility, g, v_rface=None, v_tface=None):
    """v = -mobility grad u of the state at the radial and angular faces; g holds u on
    r = 1.  Host arrays unless all three are device tensors; returns (v_rface, v_tface)."""
    m, n = ctx.m, ctx.n
    if v_rface is None:
        v_rface = np.empty((m + 1) * n, dtype=np.float64)
    if v_tface is None:
        v_tface = np.empty(m * n, dtype=np.float64)
    ag = _Arr(g, n, "g")
    ar = _Arr(v_rface, (m + 1) * n, "v_rface", out=True)
    at = _Arr(v_tface, m * n, "v_tface", out=True)
    if len({ag.device, ar.device, at.device}) > 1:
        raise ValueError("g, v_rface and v_tface must live in the same memory")
    _check(load().polar_face_drift(ctx.handle, float(mobility), ag.ptr, ar.ptr, at.ptr,
                                   POLAR_DEVICE if ag.device else POLAR_HOST))
    return v_rface, v_tface


class Gummel:
    """Handle of a polar_gummel (keeps its three contexts alive)."""

    def __init__(self, handle, ctxs):
        self.handle, self.ctxs = handle, ctxs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None and not sys.is_finalizing():
            _lib.polar_gummel_destroy(self.handle)
            self.handle = None


def polar_gummel_create(phi: Ctx, electrons: Ctx, holes: Ctx, mobility, src_electrons,
                        src_holes, tol=1e-10, max_iter=50, depth=0) -> Gummel:
    d = polar_gummel_desc((C.c_double * 2)(*[float(x) for x in mobility]), int(src_electrons),
                          int(src_holes), float(tol), int(max_iter), int(depth))
    h = C.c_void_p()
    _check(load().polar_gummel_create(phi.handle, electrons.handle, holes.handle, C.byref(d),
                                      C.byref(h)))
    return Gummel(h, (phi, electrons, holes))


def polar_gummel_step(g: Gummel, t0, t1, theta, w_electrons=(), w_holes=(), w_phi=(),
                      opts=None, check=True):
    """One coupled step from t0 to t1; w_* hold the carriers' 2 x nsrc weights (levels t0,
    t1) and the potential's nsrc weights.  Returns (stats dict, rc)."""
    t = _f64([t0, t1])
    we, wh, wp = _f64(w_electrons), _f64(w_holes), _f64(w_phi)
    wptr = (_dp * 2)(we.ctypes.data_as(_dp), wh.ctypes.data_as(_dp))
    st = polar_gummel_stats()
    rc = load().polar_gummel_step(g.handle, t.ctypes.data_as(_dp), float(theta), wptr,
                                  wp.ctypes.data_as(_dp), _opts(opts), C.byref(st))
    if check:
        _check(rc)
    return st.as_dict(), rc


def polar_gummel_destroy(g: Gummel):
    if g.handle:
        _check(load().polar_gummel_destroy(g.handle))
        g.handle = None


def polar_timing_enable(ctx: Ctx, on=True):
    _check(load().polar_timing_enable(ctx.handle, 1 if on else 0))


def polar_timing_query(ctx: Ctx):
    """Returns {kernel class: dict(launches, ms, bytes, flops)} of the timed launches."""
    lib, out, k = load(), {}, 0
    while True:
        name = C.create_string_buffer(64)
        nl, ms, by = C.c_int64(), C.c_double(), C.c_double()
        rc = lib.polar_timing_query(ctx.handle, k, name, 64, C.byref(nl), C.byref(ms), C.byref(by))
        if rc != POLAR_OK:
            break
        fl = C.c_double()
        _check(lib.polar_timing_flops(ctx.handle, k, C.byref(fl)))
        out[name.value.decode()] = dict(launches=nl.value, ms=ms.value, bytes=by.value,
                                        flops=fl.value)
        k += 1
    return out


def polar_last_error() -> str:
    return load().polar_last_error().decode()
