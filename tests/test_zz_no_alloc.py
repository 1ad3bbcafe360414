"""polar_apply_rows_noalloc: the operator applied from caller-supplied rows without any
device allocation (for callers that cannot allocate: code running under CUDA stream
capture, or embedders whose device memory is fully budgeted up front).  Checked against
polar_apply_operator, the entry point that computes the same product from a context, on
two calls in a row through the C ABI.  This file is collected last on purpose."""
import numpy as np
import pytest

import polar_inputs as pi
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2509_15879_gb300")
from paper_2509_15879_gb300 import driver  # noqa: E402


def _rows(prob):
    """Difference-form rows R, W, E, S, N (interface layout) and origin couplings o of the
    oracle's assembled operator: (L x)_ij = R x + W (x_w - x) + E (x_e - x) + ..."""
    L, B = po.operator(prob)
    L, B = L.tocsr(), B.tocsr()
    m, n = prob.m, prob.n
    N = m * n + 1
    R, W, E, S, Nn = (np.zeros(N) for _ in range(5))
    idx = lambda i, j: 1 + j * m + (i - 1)
    for j in range(n):
        for i in range(1, m + 1):
            q = idx(i, j)
            W[q] = L[q, 0] if i == 1 else L[q, idx(i - 1, j)]
            E[q] = B[q, j] if i == m else L[q, idx(i + 1, j)]
            S[q] = L[q, idx(i, (j - 1) % n)]
            Nn[q] = L[q, idx(i, (j + 1) % n)]
            R[q] = L[q, q] + W[q] + E[q] + S[q] + Nn[q]
    o = np.array([L[0, idx(1, j)] for j in range(n)])
    R[0] = L[0, 0] + o.sum()
    return R, W, E, S, Nn, o


@pytest.mark.parametrize("make", [
    lambda: pi.continuity_problem(13, 22, 2, 31, pe_target=8.0, d_amp=1.3, delta=0.2),
    lambda: pi.paper_parabolic_e1(6),
])
def test_noalloc_matches_apply_operator(make):
    prob = make()
    ctx = driver.create(prob, compact_d=False)
    dev = torch.device("cuda")
    rows = [torch.from_numpy(a).to(dev) for a in _rows(prob)]
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (alpha, beta) in enumerate(((0.0, 1.0), (37.5, 0.5))):
        x = rng.standard_normal(prob.N)
        ref = P.polar_apply_operator(ctx, alpha, beta, x)
        xd = torch.from_numpy(x).to(dev)
        yd = torch.full((prob.N,), float("nan"), dtype=torch.float64, device=dev)
        P.polar_apply_rows_noalloc(prob.m, prob.n, *rows, alpha, beta, xd, yd, stream)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        scale = alpha * np.abs(x) + beta * (abs(po.operator(prob)[0]) @ np.abs(x))
        assert np.all(np.abs(y - ref) <= 1e-13 * np.maximum(scale, 1e-300)), call


def test_noalloc_rejects_n_beyond_its_scratch():
    dev = torch.device("cuda")
    m, n = 2, 16385
    N = m * n + 1
    a = torch.zeros(N, dtype=torch.float64, device=dev)
    o = torch.zeros(n, dtype=torch.float64, device=dev)
    y = torch.zeros(N, dtype=torch.float64, device=dev)
    with pytest.raises(P.PolarError) as e:
        P.polar_apply_rows_noalloc(m, n, a, a, a, a, a, o, 1.0, 1.0, a, y, None)
    assert e.value.code == P.POLAR_EINVAL
