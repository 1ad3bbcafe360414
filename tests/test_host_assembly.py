"""The library's host-side operator assembly (polar_host.cpp, run once per polar_set_coeffs)
against the FP64 oracle, on the CPU: every coupling of every row, the diagonal, the
Dirichlet coupling of ring m and the origin row, for both schemes, with drift.

The assembly is compiled here with g++ beside a small C shim (tests/host_assembly_shim.cpp);
the library keeps each row of V L in difference form,
  (V L x)_ij = rs x_ij + w (x_w - x_ij) + e (x_e - x_ij) + s (x_s - x_ij) + nn (x_n - x_ij),
  (V L x)_0  = rs0 x_0 + sum_j o_j (x_{1,j} - x_0),
while the oracle assembles L itself, so V L[row, col] must equal the coupling and
V L[row, row] must equal rs - w - e - s - nn."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import polar_inputs as pi
from oracle import polar_oracle as po

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_15879_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hostasm") / "libhostasm.so")
    cmd = [gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
           os.path.join(HERE, "host_assembly_shim.cpp"), os.path.join(CSRC, "polar_host.cpp"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return C.CDLL(out)


def _ptr(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    _ptr.keep.append(a)
    return a.ctypes.data_as(C.c_void_p)


_ptr.keep = []


def _assemble(lib, prob):
    m, n = prob.m, prob.n
    outs = [np.zeros(m * n) for _ in range(6)] + [np.zeros(n), np.zeros(2)]
    b = None if prob.b is None else prob.b
    d_const = 1.0
    rc = lib.assemble_level0(
        C.c_int(prob.scheme), C.c_int(m), C.c_int(n), _ptr(prob.r), _ptr(prob.theta),
        _ptr(prob.d_rface), _ptr(prob.d_tface), _ptr(prob.v_rface), _ptr(prob.v_tface),
        _ptr(prob.e_node), _ptr(b if b is not None else np.full(prob.N, prob.b_const)),
        C.c_double(d_const), C.c_double(prob.d0), *[o.ctypes.data_as(C.c_void_p) for o in outs])
    assert rc == 0
    _ptr.keep.clear()
    return outs


def _check(prob, outs, rtol=1e-13):
    vol, rs, w, e, s, nn, o, scal = outs
    L, B = po.operator(prob)
    L, B = L.tocsr(), B.tocsr()
    g = po.Geometry(prob.r, prob.theta)
    m, n = prob.m, prob.n
    assert np.allclose(vol, g.V[1:], rtol=1e-15, atol=0)
    assert abs(scal[0] - g.V[0]) <= 1e-15 * g.V[0]

    def close(a, b, scale):
        return abs(a - b) <= rtol * scale

    for j in range(n):
        for i in range(1, m + 1):
            q = j * m + (i - 1)
            p = 1 + q
            V = g.V[p]
            west = 0 if i == 1 else p - 1
            row = L.getrow(p)
            scale = V * np.abs(row.data).sum()
            assert close(V * L[p, west], w[q], scale), ("w", i, j)
            if i < m:
                assert close(V * L[p, p + 1], e[q], scale), ("e", i, j)
            else:
                assert close(V * B[p, j], e[q], scale), ("dirichlet", i, j)
            ps = 1 + ((j - 1) % n) * m + (i - 1)
            pn = 1 + ((j + 1) % n) * m + (i - 1)
            assert close(V * L[p, ps], s[q], scale), ("s", i, j)
            assert close(V * L[p, pn], nn[q], scale), ("nn", i, j)
            assert close(V * L[p, p], rs[q] - w[q] - e[q] - s[q] - nn[q], scale), ("diag", i, j)
    V0 = g.V[0]
    row0 = L.getrow(0)
    scale0 = V0 * np.abs(row0.data).sum()
    for j in range(n):
        assert close(V0 * L[0, 1 + j * m], o[j], scale0), ("origin", j)
    assert close(V0 * L[0, 0], scal[1] - o.sum(), scale0)


def test_conservative_assembly_with_drift(shim):
    prob = pi.continuity_problem(11, 17, 2, 5, pe_target=12.0, d_amp=1.7, delta=0.2)
    _check(prob, _assemble(shim, prob))


def test_conservative_assembly_parabolic_graded(shim):
    prob = pi.config2(m=13, n=21, K=2)
    _check(prob, _assemble(shim, prob))


def test_paper_assembly(shim):
    for prob in (pi.paper_continuity_e3(7), pi.paper_parabolic_e1(6)):
        _check(prob, _assemble(shim, prob))


def _coarsen(lib, prob):
    m, n = prob.m, prob.n
    mc = m // 2
    outs = ([np.zeros(mc * n) for _ in range(6)] + [np.zeros(n), np.zeros(2)] +
            [np.zeros(m * n), np.zeros(m * n)])
    rc = lib.coarsen_level0(
        C.c_int(prob.scheme), C.c_int(m), C.c_int(n), _ptr(prob.r), _ptr(prob.theta),
        _ptr(prob.d_rface), _ptr(prob.d_tface), None, None, None,
        _ptr(np.full(prob.N, prob.b_const)), C.c_double(1.0), C.c_double(prob.d0),
        *[o.ctypes.data_as(C.c_void_p) for o in outs])
    assert rc == 0
    _ptr.keep.clear()
    return outs


@pytest.mark.parametrize("m", [12, 13])
def test_radial_coarsening_is_cyclic_reduction(shim, m):
    """Without angular coupling, reaction or drift, the coarse level is exactly the Schur
    complement of V L after eliminating the odd rings (one step of cyclic reduction of every
    radial line, the origin included), computed here densely from the oracle's L and B."""
    n = 7
    prob = pi.config2(m=m, n=n, K=2)
    rng = np.random.default_rng(m)
    prob.d_rface = rng.uniform(0.5, 2.0, (m + 1) * n)     # radial D varies along the line
    prob.d_tface = np.zeros(m * n)                          # no angular coupling
    vol, rs, w, e, s, nn, o, scal, ia, ib = _coarsen(shim, prob)
    L, B = po.operator(prob)
    g = po.Geometry(prob.r, prob.theta)
    A = (np.diag(g.V) @ L.toarray())
    Bd = np.diag(g.V) @ B.toarray()
    ring = np.zeros(prob.N, dtype=int)
    ring[1:] = np.tile(np.arange(1, m + 1), n)
    Eset = np.where(ring % 2 == 0)[0]                        # origin and even rings
    Oset = np.where(ring % 2 == 1)[0]
    Aoo = A[np.ix_(Oset, Oset)]
    assert np.count_nonzero(Aoo - np.diag(np.diag(Aoo))) == 0   # odd rings decoupled
    inv = 1.0 / np.diag(Aoo)
    Cm = A[np.ix_(Eset, Eset)] - A[np.ix_(Eset, Oset)] @ (inv[:, None] * A[np.ix_(Oset, Eset)])
    CB = Bd[Eset] - A[np.ix_(Eset, Oset)] @ (inv[:, None] * Bd[Oset])
    pos = {int(p): k for k, p in enumerate(Eset)}
    mc = m // 2
    idx = lambda i, j: 1 + j * m + (i - 1)
    for j in range(n):
        for I in range(1, mc + 1):
            qc = j * mc + (I - 1)
            row = pos[idx(2 * I, j)]
            scale = np.abs(Cm[row]).sum() + np.abs(CB[row]).sum()
            west = pos[0] if I == 1 else pos[idx(2 * I - 2, j)]
            assert abs(Cm[row, west] - w[qc]) <= 1e-12 * scale, ("w", I, j)
            if 2 * I + 2 <= m:
                east = Cm[row, pos[idx(2 * I + 2, j)]]
            else:
                east = CB[row, j]                           # into the Dirichlet ring
            assert abs(east - e[qc]) <= 1e-12 * scale, ("e", I, j)
            assert abs(Cm[row, row] - (rs[qc] - w[qc] - e[qc])) <= 1e-12 * scale, ("diag", I, j)
            assert s[qc] == 0.0 and nn[qc] == 0.0
        assert abs(Cm[pos[0], pos[idx(2, j)]] - o[j]) <= 1e-12 * np.abs(Cm[pos[0]]).sum()
    assert abs(Cm[pos[0], pos[0]] - (scal[1] - o.sum())) <= 1e-12 * np.abs(Cm[pos[0]]).sum()
