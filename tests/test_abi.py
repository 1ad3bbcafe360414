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
