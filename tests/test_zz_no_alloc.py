"""polar_apply_rows_noalloc: the operator applied from caller-supplied rows without any
device allocation, for callers that cannot allocate device memory -- embedders that hand
out a fixed device-memory budget themselves, or pipelines that must not call cudaMalloc /
cudaFree between kernels.  Checked through the C ABI against polar_apply_operator (the
entry point that computes the same product from a context) and against the oracle's
alpha x + beta L x, on two calls in a row (the second sees the scratch the first left),
on meshes of one block, of several blocks with ragged tails, and large enough for the
grid-stride loop (m n above 1024 blocks of 256 threads).  This file is collected last on
purpose."""
import numpy as np
import pytest

import polar_inputs as pi
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2509_15879_gb300")
from paper_2509_15879_gb300 import driver  # noqa: E402


def _rows(L, B, m, n):
    """Difference-form rows R, W, E, S, N (interface layout) and origin couplings o of the
    oracle's assembled operator: (L x)_ij = R x + W (x_w - x) + E (x_e - x) + ..."""
    L, B = L.tocsr(), B.tocsr()
    N = m * n + 1
    j, i = np.divmod(np.arange(m * n), m)
    i = i + 1
    q = 1 + j * m + (i - 1)

    def at(rows, cols):
        return np.asarray(L[rows, cols]).ravel()

    west = np.where(i == 1, 0, q - 1)
    W = at(q, west)
    E = np.where(i == m, np.asarray(B[q, j]).ravel(), at(q, np.minimum(q + 1, N - 1)))
    S = at(q, 1 + ((j - 1) % n) * m + (i - 1))
    Nn = at(q, 1 + ((j + 1) % n) * m + (i - 1))
    R = np.zeros(N)
    out = [np.zeros(N) for _ in range(4)]
    for a, v in zip(out, (W, E, S, Nn)):
        a[1:] = v
    R[1:] = at(q, q) + W + E + S + Nn
    o = at(np.zeros(n, dtype=np.int64), 1 + np.arange(n) * m)
    R[0] = L[0, 0] + o.sum()
    return (R, *out, o)


@pytest.mark.parametrize("make", [
    lambda: pi.continuity_problem(13, 22, 2, 31, pe_target=8.0, d_amp=1.3, delta=0.2),
    lambda: pi.paper_parabolic_e1(6),
    lambda: pi.continuity_problem(300, 1000, 2, 37, pe_target=5.0, d_amp=1.0, delta=0.2),
])
def test_noalloc_matches_apply_operator(make):
    prob = make()
    L, B = po.operator(prob)
    ctx = driver.create(prob, compact_d=False)
    dev = torch.device("cuda")
    rows = [torch.from_numpy(a).to(dev) for a in _rows(L, B, prob.m, prob.n)]
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    absL = abs(L)
    for call, (alpha, beta) in enumerate(((0.0, 1.0), (37.5, 0.5))):
        x = rng.standard_normal(prob.N)
        ref = P.polar_apply_operator(ctx, alpha, beta, x)
        xd = torch.from_numpy(x).to(dev)
        yd = torch.full((prob.N,), float("nan"), dtype=torch.float64, device=dev)
        P.polar_apply_rows_noalloc(prob.m, prob.n, *rows, alpha, beta, xd, yd, stream)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        scale = np.maximum(alpha * np.abs(x) + beta * (absL @ np.abs(x)), 1e-300)
        err_api = float(np.max(np.abs(y - ref) / scale))
        err_orc = float(np.max(np.abs(y - (alpha * x + beta * (L @ x))) / scale))
        print(f"noalloc {prob.m} x {prob.n} call {call}: vs apply_operator {err_api:.1e}, "
              f"vs oracle {err_orc:.1e} (relative to |alpha x| + |beta| |L| |x|)")
        assert err_api <= 1e-13 and err_orc <= 1e-13, call


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
