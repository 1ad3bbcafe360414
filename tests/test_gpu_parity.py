"""GPU parity: the CUDA library against the FP64 CPU oracle on the same seeded inputs.

Operator: y = alpha x + beta L x through polar_apply_operator against the oracle's
assembled sparse L (relative 1e-13).  Steps: polar_advance against the oracle's sparse
LU time stepping; FP64 path <= 1e-12 and mixed path <= 1e-9 in the relative max norm.
"""
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


def _rel_wl2(prob, a, b):
    """Relative L2 difference weighted by the control volumes V (origin disk included)."""
    V = po.Geometry(prob.r, prob.theta).V
    return float(np.sqrt(np.sum(V * (a - b) ** 2) / max(np.sum(V * b ** 2), 1e-300)))


def _small_continuity(m, n, K=4, seed=21, pe=6.0, theta_w=0.5):
    return pi.continuity_problem(m, n, K, seed, theta_w=theta_w, pe_target=pe, d_amp=1.3,
                                 delta=0.2)


OPERATOR_CASES = [
    ("parabolic_uniform", lambda: pi.config1()),
    ("parabolic_graded_ragged", lambda: pi.config2(m=37, n=53, K=3)),
    ("continuity_ragged", lambda: _small_continuity(45, 70)),
    ("continuity_tiny", lambda: _small_continuity(2, 4)),
    ("paper_parabolic", lambda: pi.paper_parabolic_e1(19)),
    ("paper_continuity", lambda: pi.paper_continuity_e3(13)),
]


@pytest.mark.parametrize("name,make", OPERATOR_CASES)
def test_operator_matches_assembled_matrix(name, make):
    prob = make()
    L, _ = po.operator(prob)
    ctx = driver.create(prob, compact_d=False)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(prob.N)
    for alpha, beta in ((0.0, 1.0), (37.5, 0.5)):
        y = P.polar_apply_operator(ctx, alpha, beta, x)
        ref = alpha * x + beta * (L @ x)
        scale = alpha * np.abs(x) + beta * (abs(L) @ np.abs(x))
        err = float(np.max(np.abs(y - ref) / np.maximum(scale, 1e-300)))
        print(f"PARITY operator {name} alpha={alpha}: {err:.2e} (bar 1e-13 of |alpha x| + "
              f"|beta| |L| |x|)")
        assert np.all(np.abs(y - ref) <= 1e-13 * scale), name


def _kappa(prob, k):
    """||(D^-1 A)^-1||_inf of step k's matrix (an M-matrix: the row sums of A^-1 D)."""
    import scipy.sparse.linalg as spla
    L, _ = po.operator(prob)
    A = po.system_matrix(L, prob.t[k + 1] - prob.t[k], prob.theta_w).tocsc()
    return float(np.max(np.abs(spla.splu(A).solve(A.diagonal()))))


def _oracle_levels(prob, K):
    out = []
    po.run(prob, K, callback=lambda k, U: out.append(U.copy()))
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_config1_full_run(precision, tol):
    """Uniform 32 x 64 mesh, Crank-Nicolson, dt = 0.01, 100 steps to T = 1."""
    prob = pi.config1()
    ref = po.run(prob)
    ctx = driver.create(prob, precision)
    stats = driver.advance(ctx, prob)
    assert all(s["status"] == 0 for s in stats)
    U, t = P.polar_get_state(ctx)
    assert abs(t - 1.0) < 1e-15
    print(f"PARITY C1 32x64 100 steps precision {precision}: {_rel(U, ref):.2e} (bar {tol:g}), "
          f"V-weighted L2 {_rel_wl2(prob, U, ref):.2e}")
    assert _rel(U, ref) < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("name,make,K", [
    ("C2_shape", lambda: pi.config2(m=64, n=128, K=30), 30),
    ("continuity_drift", lambda: _small_continuity(40, 72, K=12), 12),
    ("continuity_theta06", lambda: _small_continuity(33, 50, K=8, theta_w=0.6, pe=18.0), 8),
    ("paper_e1", lambda: pi.paper_parabolic_e1(19), 10),
    ("paper_e3", lambda: pi.paper_continuity_e3(19), 10),
])
def test_steps_match_oracle(name, make, K, precision, tol):
    prob = make()
    refs = _oracle_levels(prob, K)
    ctx = driver.create(prob, precision)
    worst = worst_l2 = 0.0
    for k in range(K):
        driver.advance(ctx, prob, k, k + 1)
        U, _ = P.polar_get_state(ctx)
        worst = max(worst, _rel(U, refs[k]))
        worst_l2 = max(worst_l2, _rel_wl2(prob, U, refs[k]))
        assert _rel(U, refs[k]) < tol, (name, k, _rel(U, refs[k]))
    print(f"PARITY {name} {prob.m}x{prob.n} {K} steps precision {precision}: worst {worst:.2e} "
          f"(bar {tol:g}), V-weighted L2 {worst_l2:.2e}")


def _stiff_rings():
    """7 rings, the first at r = 1e-4, 16384 angles, one Crank-Nicolson step of dt = 0.2:
    on ring 1 the angular couplings exceed the row sums by many orders more than 1 / eps32,
    so the FP32 refinement cannot reach the FP64 tolerance there."""
    r = np.concatenate([[0.0, 1e-4], np.linspace(1e-4, 1.0, 8)[1:]])
    return pi.parabolic_problem(r, meshes.uniform_theta(16384), np.array([0.0, 0.2]), 0.5,
                                name="stiff_rings")


@pytest.mark.parametrize("precision,make", [(0, lambda: _small_continuity(37, 61, K=6)),
                                            (1, lambda: _small_continuity(37, 61, K=6)),
                                            (1, _stiff_rings)])
def test_graph_step_equals_eager_step(precision, make):
    """A step run as one CUDA graph (device-side refinement and Krylov loops) and the same
    step driven from the host (kernel timing on) execute the same kernels in the same order
    (for the mixed path also when it falls back to the FP64 Krylov solve)."""
    prob = make()
    K = len(prob.t) - 1
    out = []
    for eager in (False, True):
        ctx = driver.create(prob, precision)
        if eager:
            P.polar_timing_enable(ctx, True)
        stats = driver.advance(ctx, prob, 0, K)
        out.append((P.polar_get_state(ctx)[0], stats))
    assert np.array_equal(out[0][0], out[1][0])
    assert [s["iters"] for s in out[0][1]] == [s["iters"] for s in out[1][1]]
    assert [s["fp64_iters"] for s in out[0][1]] == [s["fp64_iters"] for s in out[1][1]]


def test_mixed_fallback_reaches_fp64_tolerance():
    """Where FP32 refinement stalls, the mixed path finishes the step with FP64 Krylov
    solves over its FP32 V-cycle (fp64_iters > 0) and meets the FP64 tolerance; the result
    agrees with the oracle to max(1e-9, 20 kappa eps)."""
    prob = _stiff_rings()
    ref = po.run(prob, 1)
    ctx = driver.create(prob, P.POLAR_MIXED)
    st = driver.advance(ctx, prob, 0, 1)
    assert st[0]["status"] == 0 and st[0]["scaled_resid"] <= 1e-14
    assert st[0]["fp64_iters"] > 0, st[0]
    U, _ = P.polar_get_state(ctx)
    kappa = _kappa(prob, 0)
    tol = max(1e-9, 20 * kappa * np.finfo(float).eps)
    print(f"PARITY stiff rings 7x16384 mixed (FP64 fallback): {_rel(U, ref):.2e} "
          f"(bar {tol:.1e}, kappa {kappa:.2e})")
    assert _rel(U, ref) < tol, (_rel(U, ref), tol)


@pytest.mark.parametrize("timing", [False, True])
def test_failed_step_leaves_state(timing):
    """POLAR_ENOCONV (one refinement sweep cannot reach 1e-18) keeps U and t."""
    prob = _small_continuity(20, 32, K=3)
    ctx = driver.create(prob, P.POLAR_MIXED)
    if timing:
        P.polar_timing_enable(ctx, True)
    U0, t0 = P.polar_get_state(ctx)
    stats, rc = P.polar_advance(ctx, prob.t[:3], prob.theta_w, prob.weight_table()[:3],
                                dict(tol=1e-18, max_refine=1), check=False)
    assert rc == P.POLAR_ENOCONV
    assert stats[0]["status"] == P.POLAR_ENOCONV and stats[1]["status"] == P.POLAR_ESTATE
    U1, t1 = P.polar_get_state(ctx)
    assert t1 == t0 and np.array_equal(U0, U1)
    # the context stays usable
    stats, rc = P.polar_advance(ctx, prob.t[:3], prob.theta_w, prob.weight_table()[:3])
    assert rc == 0


def test_nonfinite_state_rejected():
    prob = _small_continuity(8, 16, K=2)
    ctx = driver.create(prob, P.POLAR_FP64)
    bad = np.array(prob.u0, dtype=np.float64)
    bad[5] = np.nan
    with pytest.raises(P.PolarError) as e:
        P.polar_set_state(ctx, bad, 0.0)
    assert e.value.code == P.POLAR_ENONFINITE


@pytest.mark.parametrize("precision,m,n", [(0, 6, 16384), (1, 20, 16384), (0, 40, 3000),
                                           (1, 40, 3000)])
def test_long_rings(precision, m, n):
    """Rings longer than one CTA covers are split over a thread-block cluster.  The first
    steps of a 2000-level time stretch (dt ~ 1e-5, as in the large continuity workloads).
    On these meshes the small first ring makes the step ill-conditioned: two independent
    FP64 solves can only agree to about kappa eps, kappa = ||(D^-1 A)^-1||_inf (computed
    here from the oracle's factorisation), so the bar is max(stated, 20 kappa eps)."""
    prob = pi.continuity_problem(m, n, 2000, 77, pe_target=4.0, d_amp=1.0, delta=0.2)
    K = 2
    refs = _oracle_levels(prob, K)
    ctx = driver.create(prob, precision)
    kappa = _kappa(prob, 0)
    tol = max(1e-12 if precision == 0 else 1e-9, 20 * kappa * np.finfo(float).eps)
    for k in range(K):
        driver.advance(ctx, prob, k, k + 1)
        U, _ = P.polar_get_state(ctx)
        print(f"PARITY long rings {m}x{n} step {k} precision {precision}: "
              f"{_rel(U, refs[k]):.2e} (bar {tol:.1e}, kappa {kappa:.2e})")
        assert _rel(U, refs[k]) < tol, (m, n, k, _rel(U, refs[k]))


def test_longer_schedule_after_a_short_one():
    """A schedule longer than any before grows the device schedule arrays; the step graph
    captured for the shorter one must not be reused with the old arrays."""
    prob = _small_continuity(24, 40, K=12)
    refs = _oracle_levels(prob, 12)
    ctx = driver.create(prob, P.POLAR_FP64)
    driver.advance(ctx, prob, 0, 1)
    driver.advance(ctx, prob, 1, 3)
    stats = driver.advance(ctx, prob, 3, 12)
    assert [s["status"] for s in stats] == [0] * 9
    assert all(s["iters"] > 0 for s in stats)
    U, t = P.polar_get_state(ctx)
    assert t == prob.t[12]
    assert _rel(U, refs[11]) < 1e-12


@pytest.fixture(scope="module")
def c2_recipe_schedule():
    """The oracle over the whole 1000-level schedule of the 512 x 1024 parabolic workload
    (dt_k = 1e-4 1.01^k, T ~ 209.6), on the same recipe's 64 x 128 mesh: the state at
    k = 100, 200, ..., 1000 and the running maximum of max|U^l| over l <= k."""
    prob = pi.config2(m=64, n=128, K=1000)
    out, run = {}, [float(np.max(np.abs(prob.u0)))]

    def keep(k, U):
        run.append(max(run[-1], float(np.max(np.abs(U)))))
        if k % 100 == 0:
            out[k] = (U.copy(), run[-1])

    po.run(prob, 1000, callback=keep)
    return prob, out


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_c2_recipe_whole_schedule(c2_recipe_schedule, precision, tol):
    """1000 consecutive steps.  u ~ e^{-t} falls to 1e-91 by the end while Crank-Nicolson
    barely damps the stiff modes (amplification near -1 at dt >> h^2), so from about level
    750 on |U| is at the size of what earlier levels left in those modes (~1e-12 of |U^0|,
    the oracle's own state included) and a relative max norm at level k says nothing.  The
    difference is therefore quoted as max|U_gpu^k - U_oracle^k| / max_{l <= k} max|U^l|,
    the size of the state it was made from, at k = 100, ..., 1000."""
    prob, ref = c2_recipe_schedule
    ctx = driver.create(prob, precision)
    worst = 0.0
    for k0 in range(0, 1000, 100):
        stats = driver.advance(ctx, prob, k0, k0 + 100)
        assert all(s["status"] == 0 for s in stats)
        U, t = P.polar_get_state(ctx)
        Uref, runmax = ref[k0 + 100]
        d = float(np.max(np.abs(U - Uref))) / runmax
        worst = max(worst, d)
        print(f"PARITY C2 recipe 64x128 consecutive, level {k0 + 100}, precision {precision}: "
              f"{d:.2e} of max_(l<=k)|U^l| (max|U^k| = {np.max(np.abs(Uref)):.2e}, bar {tol:g})")
        assert d < tol, (k0 + 100, d)


def test_timing_reports_bytes_and_flops():
    # the per-kernel timing carries each class's algorithmic bytes and arithmetic; the
    # rates it implies stay below what the device can do (HBM copy rate, FP64 pipe)
    prob = _small_continuity(40, 72, K=2)
    ctx = driver.create(prob, P.POLAR_FP64)
    driver.advance(ctx, prob, 0, 1)
    P.polar_timing_enable(ctx, True)
    driver.advance(ctx, prob, 1, 2)
    q = P.polar_timing_query(ctx)
    P.polar_timing_enable(ctx, False)
    pts = prob.m * prob.n
    for name in ("ring_pre_odd@L0", "ring_post_even@L0", "stencil_dot", "resid64"):
        d = q[name]
        assert d["launches"] > 0 and d["bytes"] > 0 and d["flops"] > 0
        per_launch = d["flops"] / d["launches"]
        assert pts < per_launch < 40 * pts        # a few to a few tens of flops per point
        assert d["flops"] / (d["ms"] * 1e-3) < 1.3e12   # under GB300's FP64 rate
    assert q["correct"]["flops"] == 0.0             # classes without a model report 0
