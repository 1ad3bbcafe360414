"""The direct (Swarztrauber-Sweet) inner solve for separable operators: uniform angles and
ring coefficients independent of the angle (Section 2.1).  Fourier transform along theta
(radix-2 FFT for n a power of two, Bluestein's chirp-z form otherwise), one tridiagonal
solve in r per mode, the origin coupled to the mean mode.  Checked through the C ABI
against the FP64 oracle's sparse LU steps, against the Krylov path of the same library,
and graph against eager execution."""
import math

import numpy as np
import pytest

import polar_inputs as pi
from polar_inputs import meshes
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2509_15879_gb300")
from paper_2509_15879_gb300 import driver  # noqa: E402


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def radial_problem(m, n, K, seed, drift=True):
    """Continuity equation with D, b and the radial drift depending on r only, uniform
    angles, theta-dependent sources and Dirichlet data (random, seeded), time stretch."""
    rng = np.random.default_rng(seed)
    r = meshes.sine_stretch(m, 0.8)
    theta = meshes.uniform_theta(n)
    rh = 0.5 * (r[:-1] + r[1:])
    ri = r[1:m + 1]
    N = m * n + 1
    R, TH = pi.problems.node_coords(r, theta)
    u0 = (1.0 - R ** 2) * (1.0 + 0.3 * R * np.cos(TH) + 0.2 * R * np.sin(2 * TH))
    return pi.Problem(
        name=f"radial_{m}x{n}", r=r, theta=theta, t=meshes.time_stretch(1.0, 1.5, K),
        theta_w=0.6, scheme=po.CONSERVATIVE,
        d_rface=np.tile(0.5 + rh ** 2, n), d_tface=np.tile(0.5 + ri ** 2, n),
        v_rface=np.tile(3.0 * rh * (1.0 - rh), n) if drift else None,
        src=[rng.standard_normal(N), np.cos(3 * TH) * R], bnd=[rng.standard_normal(n), np.ones(n)],
        u0=u0, weights=lambda tt: np.array([math.exp(-tt), 1.0]), b_const=0.7, d0=0.5)


CASES = [
    ("radix2_32x64", lambda: radial_problem(32, 64, 5, 1)),
    ("radix2_40x256", lambda: radial_problem(40, 256, 4, 2)),
    ("bluestein_24x150", lambda: radial_problem(24, 150, 5, 3)),
    ("bluestein_33x1000", lambda: radial_problem(33, 1000, 3, 4)),
    ("radix2_long_16x8192", lambda: radial_problem(16, 8192, 2, 5, drift=False)),
    ("bluestein_long_10x3001", lambda: radial_problem(10, 3001, 2, 6)),
    ("paper_e1_19", lambda: pi.paper_parabolic_e1(19)),
]


def _kappa(prob, k):
    """||(D^-1 A)^-1||_inf of step k's matrix (an M-matrix: the row sums of A^-1 D)."""
    import scipy.sparse.linalg as spla
    L, _ = po.operator(prob)
    A = po.system_matrix(L, prob.t[k + 1] - prob.t[k], prob.theta_w).tocsc()
    return float(np.max(np.abs(spla.splu(A).solve(A.diagonal()))))


@pytest.mark.parametrize("precision", [P.POLAR_FP64, P.POLAR_MIXED])
@pytest.mark.parametrize("name,make", CASES)
def test_direct_steps_match_oracle(name, make, precision):
    """Bar: 1e-12, or 20 kappa eps where the step's matrix is worse conditioned than that
    allows (long rings with large steps: two independent FP64 solves of such a step agree
    only to about kappa eps)."""
    prob = make()
    K = min(len(prob.t) - 1, 5)
    refs = []
    po.run(prob, K, callback=lambda k, U: refs.append(U.copy()))
    ctx = driver.create(prob, precision)
    assert P.polar_is_separable(ctx)
    worst = 0.0
    for k in range(K):
        st = driver.advance(ctx, prob, k, k + 1)[0]
        assert st["status"] == 0 and st["iters"] == 0, st
        assert st["refinements"] <= 4, st
        U, _ = P.polar_get_state(ctx)
        worst = max(worst, _rel(U, refs[k]))
    kappa = max(_kappa(prob, k) for k in range(K))
    bar = max(1e-12, 20 * kappa * np.finfo(float).eps)
    print(f"PARITY direct {name} precision {precision} {K} steps: worst {worst:.2e} (bar "
          f"{bar:.1e}, kappa {kappa:.2e}); refinement sweeps of the last step {st['refinements']}")
    assert worst < bar, worst


def test_config1_direct_full_run():
    """The uniform 32 x 64 parabolic workload, 100 Crank-Nicolson steps, direct solves."""
    prob = pi.config1()
    ref = po.run(prob)
    ctx = driver.create(prob, P.POLAR_FP64)
    assert P.polar_is_separable(ctx)
    stats = driver.advance(ctx, prob)
    assert all(s["status"] == 0 and s["iters"] == 0 for s in stats)
    U, t = P.polar_get_state(ctx)
    print(f"PARITY C1 32x64 direct 100 steps: {_rel(U, ref):.2e} (bar 1e-12)")
    assert _rel(U, ref) < 1e-12


def test_direct_equals_krylov():
    prob = radial_problem(36, 96, 4, 9)
    out = {}
    for method in (P.POLAR_SOLVE_DIRECT, P.POLAR_SOLVE_KRYLOV):
        ctx = driver.create(prob, P.POLAR_FP64)
        stats = driver.advance(ctx, prob, 0, 4, opts=dict(method=method))
        assert all(s["status"] == 0 for s in stats)
        assert all((s["iters"] == 0) == (method == P.POLAR_SOLVE_DIRECT) for s in stats)
        out[method] = P.polar_get_state(ctx)[0]
    d = _rel(out[P.POLAR_SOLVE_DIRECT], out[P.POLAR_SOLVE_KRYLOV])
    print(f"direct vs Krylov 36x96, 4 steps: {d:.2e}")
    assert d < 1e-12


def test_direct_graph_equals_eager():
    prob = radial_problem(20, 150, 4, 10)
    out = []
    for eager in (False, True):
        ctx = driver.create(prob, P.POLAR_FP64)
        if eager:
            P.polar_timing_enable(ctx, True)
        driver.advance(ctx, prob, 0, 4)
        out.append(P.polar_get_state(ctx)[0])
        if eager:
            assert "direct_solve" in P.polar_timing_query(ctx)
    assert np.array_equal(out[0], out[1])


def test_direct_needs_a_separable_operator():
    prob = pi.continuity_problem(12, 20, 2, 3, pe_target=4.0, delta=0.2)
    ctx = driver.create(prob, P.POLAR_FP64)
    assert not P.polar_is_separable(ctx)
    with pytest.raises(P.PolarError) as e:
        driver.advance(ctx, prob, 0, 1, opts=dict(method=P.POLAR_SOLVE_DIRECT))
    assert e.value.code == P.POLAR_EINVAL
    st = driver.advance(ctx, prob, 0, 1)[0]          # AUTO: Krylov
    assert st["status"] == 0 and st["iters"] > 0
