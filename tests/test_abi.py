"""The C-ABI library: it loads, exports every function include/polar.h declares, and
rejects bad arguments before any GPU work (these calls need no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polar.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(polar_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_15879_gb300 import _native, build
    if not os.path.exists(_native.LIB_PATH):
        build.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("polar_mesh_create", "polar_set_coeffs", "polar_step", "polar_advance",
                     "polar_mesh_destroy", "polar_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2509_15879_gb300 import _native
    assert set(_declared()) <= set(_native.EXPORTS)


def _desc(P, m, n, r=None, theta=None, scheme=0, precision=0):
    r = np.linspace(0.0, 1.0, m + 2) if r is None else r
    theta = 2 * np.pi * np.arange(n) / n if theta is None else theta
    keep = (r, theta)
    d = P.polar_mesh_desc(m, n, r.ctypes.data_as(P._dp), theta.ctypes.data_as(P._dp), scheme,
                          precision, None)
    return d, keep


@pytest.mark.parametrize("case", ["small_m", "small_n", "bad_r0", "bad_r1", "nonmono_r",
                                  "nonmono_theta", "theta_span", "scheme", "precision",
                                  "n_too_large"])
def test_mesh_create_rejects_bad_meshes_before_gpu_work(lib, case):
    from paper_2509_15879_gb300 import _native as P
    m, n = 8, 16
    r = np.linspace(0.0, 1.0, m + 2)
    th = 2 * np.pi * np.arange(n) / n
    kw = {}
    if case == "small_m":
        m, r = 1, np.linspace(0.0, 1.0, 3)
    elif case == "small_n":
        n, th = 3, 2 * np.pi * np.arange(3) / 3
    elif case == "bad_r0":
        r = r.copy(); r[0] = 1e-3
    elif case == "bad_r1":
        r = r.copy(); r[-1] = 0.999
    elif case == "nonmono_r":
        r = r.copy(); r[3], r[4] = r[4], r[3]
    elif case == "nonmono_theta":
        th = th.copy(); th[2] = th[1]
    elif case == "theta_span":
        th = th.copy(); th[-1] = 2 * np.pi + 0.1
    elif case == "scheme":
        kw["scheme"] = 7
    elif case == "precision":
        kw["precision"] = 9
    elif case == "n_too_large":
        n, th = 20000, 2 * np.pi * np.arange(20000) / 20000
    d, keep = _desc(P, m, n, r, th, **kw)
    h = C.c_void_p()
    rc = lib.polar_mesh_create(C.byref(d), C.byref(h))
    assert rc == P.POLAR_EINVAL, (case, rc)
    assert not h.value
    assert len(lib.polar_last_error()) > 0


def test_null_arguments_are_rejected(lib):
    from paper_2509_15879_gb300 import _native as P
    assert lib.polar_mesh_create(None, None) == P.POLAR_EINVAL
    assert lib.polar_set_coeffs(None, None) == P.POLAR_EINVAL
    assert lib.polar_set_state(None, None, C.c_double(0.0), 0) == P.POLAR_EINVAL
    assert lib.polar_step(None, 0.1, 0.5, None, None, None, None) == P.POLAR_EINVAL
    assert lib.polar_advance(None, 1, None, 0.5, None, None, None) == P.POLAR_EINVAL
    assert lib.polar_mesh_destroy(None) == P.POLAR_OK
    assert lib.polar_kernel_launches(None) == 0


def test_valid_mesh_without_gpu_reports_cuda_error(lib):
    """With no CUDA device the library refuses (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_15879_gb300 import _native as P
    d, keep = _desc(P, 8, 16)
    h = C.c_void_p()
    assert lib.polar_mesh_create(C.byref(d), C.byref(h)) == P.POLAR_ECUDA
    assert not h.value


def test_noalloc_rejects_bad_sizes_and_overlap_before_gpu_work(lib):
    """polar_apply_rows_noalloc checks n against its fixed scratch and the x / y ranges
    before it touches the GPU (the pointers here are never dereferenced)."""
    from paper_2509_15879_gb300 import _native as P
    fake = [C.c_void_p(4096 * (k + 1)) for k in range(6)]
    m, n = 4, 8
    N = m * n + 1
    x = C.c_void_p(1 << 20)
    for y in (x, C.c_void_p((1 << 20) + 8 * (N - 1)), C.c_void_p((1 << 20) - 8 * (N - 1))):
        rc = lib.polar_apply_rows_noalloc(m, n, *fake, 1.0, 1.0, x, y, None)
        assert rc == P.POLAR_EINVAL
    rc = lib.polar_apply_rows_noalloc(m, 16385, *fake, 1.0, 1.0, x, C.c_void_p(1 << 30), None)
    assert rc == P.POLAR_EINVAL
    assert b"16384" in lib.polar_last_error()


def test_mesh_create_rejects_half_an_allocator(lib):
    from paper_2509_15879_gb300 import _native as P
    d, keep = _desc(P, 8, 16)
    d.alloc = P.ALLOC_FN(lambda nbytes, stream, user: None)
    h = C.c_void_p()
    assert lib.polar_mesh_create(C.byref(d), C.byref(h)) == P.POLAR_EINVAL
    assert not h.value


# ------------------------------------------------------------------ binding validation
def test_binding_rejects_wrong_arrays_before_calling_the_library():
    """Arrays the C calls read or write must be float64, contiguous and long enough; an
    output that would need a converted copy is refused (nothing reaches the library)."""
    import torch
    from paper_2509_15879_gb300 import _native as P
    P._Arr(np.zeros(6), 6)                                         # fine
    with pytest.raises(ValueError):
        P._Arr(np.zeros(5), 6, "x")                                # too short
    with pytest.raises(ValueError):
        P._Arr(np.zeros(6, dtype=np.float32), 6, "y", out=True)    # output needs a copy
    with pytest.raises(ValueError):
        P._Arr(np.zeros((6, 2))[:, 0], 6, "y", out=True)           # strided output
    with pytest.raises(ValueError):
        P._Arr(torch.zeros(6, dtype=torch.float32), 6, "u")        # wrong dtype tensor
    with pytest.raises(ValueError):
        P._Arr(torch.zeros(12, dtype=torch.float64)[::2], 6, "u")  # strided tensor
    with pytest.raises(ValueError):
        P._Arr(torch.zeros(5, dtype=torch.float64), 6, "u")        # short tensor
    ctx = P.Ctx(None, 4, 8)                                        # never reaches the library
    N = ctx.N
    with pytest.raises(ValueError):
        P.polar_set_coeffs(ctx, d_rface=np.ones(5 * 8 - 1))
    with pytest.raises(ValueError):
        P.polar_set_coeffs(ctx, src=[np.ones(N)], bnd=[np.ones(7)])
    with pytest.raises(ValueError):
        P.polar_set_state(ctx, np.ones(N - 1), 0.0)
    with pytest.raises(ValueError):
        P.polar_get_state(ctx, np.empty(N - 1))
    with pytest.raises(ValueError):
        P.polar_apply_operator(ctx, 1.0, 1.0, np.ones(N), np.empty(N, dtype=np.float32))
    with pytest.raises(ValueError):
        P.polar_apply_rows_noalloc(4, 8, *[np.ones(N)] * 5, np.ones(8), 1.0, 1.0,
                                   np.ones(N), np.empty(N))
