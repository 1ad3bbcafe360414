"""Batched instances (parameter sweep of uneven meshes) advanced by one CUDA graph per
step: every instance matches the same instance advanced alone (bit for bit: same kernels
in the same order) and the FP64 CPU oracle."""
import numpy as np
import pytest

import polar_inputs as pi
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2509_15879_gb300")
from paper_2509_15879_gb300 import driver  # noqa: E402


def _instances():
    # uneven sizes, D amplitudes and Peclet numbers (the shape of the 256-instance sweep)
    return [pi.config4_instance(i, K=6, scale=0.06) for i in range(5)]


@pytest.mark.parametrize("precision", [P.POLAR_FP64, P.POLAR_MIXED])
def test_batch_matches_single_and_oracle(precision):
    probs = _instances()
    K = 4
    ctxs = [driver.create(p, precision) for p in probs]
    batch = P.polar_batch_create(ctxs)
    stats, rc = driver.batch_advance(batch, probs, 0, K)
    assert rc == 0
    assert all(s["status"] == 0 for row in stats for s in row)
    tol = 1e-12 if precision == P.POLAR_FP64 else 1e-9
    for p, c, row in zip(probs, ctxs, stats):
        U, t = P.polar_get_state(c)
        assert t == p.t[K]
        alone = driver.create(p, precision)
        st_alone = driver.advance(alone, p, 0, K)
        Ua, _ = P.polar_get_state(alone)
        assert np.array_equal(U, Ua)
        assert [s["iters"] for s in row] == [s["iters"] for s in st_alone]
        ref = po.run(p, K)
        err = np.max(np.abs(U - ref)) / np.max(np.abs(ref))
        print(f"PARITY batch instance {p.m}x{p.n} precision {precision}: {err:.2e} (bar {tol:g})")
        assert err < tol


def test_batch_failure_is_per_instance():
    probs = _instances()[:3]
    ctxs = [driver.create(p, P.POLAR_FP64) for p in probs]
    batch = P.polar_batch_create(ctxs)
    stats, rc = driver.batch_advance(batch, probs, 0, 2, check=False)
    assert rc == 0
    # no instance can meet an impossible tolerance in one sweep: each stops at its first
    # step, keeps its state, and the rest of its schedule is reported as not run
    bad = P.polar_batch_advance(batch, [p.t[2:5] for p in probs], [p.theta_w for p in probs],
                                [p.weight_table()[2:5] for p in probs],
                                dict(tol=1e-18, max_refine=1), check=False)
    stats, rc = bad
    assert rc == P.POLAR_ENOCONV
    for c, p, row in zip(ctxs, probs, stats):
        assert row[0]["status"] == P.POLAR_ENOCONV
        assert row[1]["status"] == P.POLAR_ESTATE
        assert P.polar_get_state(c)[1] == p.t[2]


def test_batch_longer_schedule_after_a_short_one():
    """The batch graph is captured again when a longer schedule grows the instances'
    schedule arrays (it holds their device addresses)."""
    probs = _instances()[:3]
    ctxs = [driver.create(p, P.POLAR_MIXED) for p in probs]
    batch = P.polar_batch_create(ctxs)
    driver.batch_advance(batch, probs, 0, 1)
    stats, rc = driver.batch_advance(batch, probs, 1, 5)
    assert rc == 0
    assert all(s["status"] == 0 and s["iters"] > 0 for row in stats for s in row)
    for p, c in zip(probs, ctxs):
        U, t = P.polar_get_state(c)
        assert t == p.t[5]
        ref = po.run(p, 5)
        assert np.max(np.abs(U - ref)) / np.max(np.abs(ref)) < 1e-9


def test_mixed_path_completes_the_hard_sweep_instances():
    # instances 196 and 240 of the 256-instance sweep: once the mixed path's FP32 smoother
    # could not finish steps 149 and 377 of their schedules; the mixed path now carries on
    # in FP64 where the FP32 solve stalls.  Both advance as a batch, in mixed precision,
    # through those steps; every step must succeed and the states must equal the FP64
    # path's at the mixed bar (1e-9 relative; both stop at the same FP64 tolerance)
    K = 380
    probs = [pi.config4_instance(i, K=500) for i in (196, 240)]
    states = {}
    for precision in (P.POLAR_MIXED, P.POLAR_FP64):
        ctxs = [driver.create(p, precision) for p in probs]
        batch = P.polar_batch_create(ctxs)
        stats, rc = driver.batch_advance(batch, probs, 0, K)
        assert rc == 0
        assert all(s["status"] == 0 for row in stats for s in row)
        states[precision] = [P.polar_get_state(c)[0] for c in ctxs]
        worst = [max(s["iters"] for s in row) for row in stats]
        print(f"HARD instances precision {precision}: most Krylov iterations in a step {worst}")
    for a, b in zip(states[P.POLAR_MIXED], states[P.POLAR_FP64]):
        err = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        print(f"PARITY hard instance mixed vs FP64 after {K} steps: {err:.2e} (bar 1e-9)")
        assert err < 1e-9
