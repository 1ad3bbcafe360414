"""GPU parity of the coupled electron-hole-potential path against the oracle.

polar_solve_steady (the steady problem, with and without drift), polar_face_drift and
polar_gummel_step (Gummel's iteration over one theta-step of the carrier pair, plain or
Anderson-accelerated, the pair advanced as a 2-instance batch) are compared with oracle/coupled.py on the seeded pair of
polar_inputs.coupled_pair.  Bars: the steady solves max(1e-12, 20 kappa eps) relative
(kappa = ||(D^-1 A)^-1||_inf of the oracle's matrix: two FP64 solves of the same system
agree to about kappa eps); the face drift 1e-13 relative (the same difference quotients);
the coupled steps 1e-9 relative (both sides stop Gummel's iteration at a change of 1e-12,
which bounds their distance to the fixed point by about 1e-12 / (1 - 0.2)).
"""
from dataclasses import replace

import numpy as np
import pytest

import polar_inputs as pi
from oracle import coupled as oc
from oracle import polar_oracle as po

pytestmark = pytest.mark.gpu


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver
    return P, driver


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _kappa_bar(prob, stated=1e-12):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    L, _ = po.operator(prob)
    A = L.tocsc()
    Dinv = sp.diags(1.0 / A.diagonal())
    inv = spla.inv((Dinv @ A).tocsc()).toarray()
    kappa = float(np.max(np.sum(np.abs(inv), axis=1)))
    return max(stated, 20.0 * kappa * np.finfo(np.float64).eps), kappa


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("drift", [False, True])
def test_steady_solve_matches_oracle(precision, drift):
    P, driver = _lib()
    cp = pi.coupled_pair(m=20, n=40)
    prob = cp.electrons
    if drift:
        rng = np.random.default_rng(7)
        prob = replace(prob, v_rface=rng.uniform(-3, 3, (prob.m + 1) * prob.n),
                       v_tface=rng.uniform(-3, 3, prob.m * prob.n))
    prec = P.POLAR_FP64 if precision == "fp64" else P.POLAR_MIXED
    ctx = driver.create(prob, prec)
    P.polar_set_state(ctx, np.zeros(prob.N), 0.0)
    w = np.array([0.8])
    st = P.polar_solve_steady(ctx, w)
    got, t = P.polar_get_state(ctx)
    want = oc.steady(prob, w)
    bar, kappa = _kappa_bar(prob)
    err = _rel(got, want)
    print(f"PARITY steady {precision} drift={drift}: rel err {err:.3e} (bar {bar:.1e}, "
          f"kappa {kappa:.2e}), iters {st['iters']}")
    assert st["status"] == 0 and t == 0.0
    assert err <= bar


def test_face_drift_matches_oracle():
    P, driver = _lib()
    cp = pi.coupled_pair(m=20, n=40)
    ctx = driver.create(cp.phi, P.POLAR_FP64)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(cp.phi.N)
    g = rng.standard_normal(cp.phi.n)
    P.polar_set_state(ctx, u, 0.0)
    for mob in (1.5, -2.0):
        vr, vt = P.polar_face_drift(ctx, mob, g)
        wr, wt = oc.face_drift(cp.phi.r, cp.phi.theta, u, g, mob)
        err = max(_rel(vr, wr), _rel(vt, wt))
        print(f"PARITY face drift mobility {mob}: rel err {err:.3e}")
        assert err <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("depth,scale", [(0, 1.0), (3, 1.0), (3, 4.0)])
def test_gummel_steps_match_oracle(precision, depth, scale):
    P, driver = _lib()
    cp = pi.coupled_pair(m=24, n=48, K=3, scale=scale)
    prec = P.POLAR_FP64 if precision == "fp64" else P.POLAR_MIXED
    ph = driver.create(cp.phi, prec)
    el = driver.create(cp.electrons, prec)
    ho = driver.create(cp.holes, prec)
    P.polar_set_state(ph, np.zeros(cp.phi.N), 0.0)
    tol = 1e-12
    g = P.polar_gummel_create(ph, el, ho, cp.mobility, cp.slots[0], cp.slots[1], tol=tol,
                              max_iter=60, depth=depth)
    U = [cp.electrons.u0.copy(), cp.holes.u0.copy()]
    w = [np.array([1.0, 1.0]), np.array([1.0, 1.0])]
    for k in range(len(cp.t) - 1):
        st, rc = P.polar_gummel_step(g, cp.t[k], cp.t[k + 1], cp.theta_w, w[0], w[1], cp.w_phi)
        U, phi, iters, change, ok = oc.gummel_step(
            cp.phi, [cp.electrons, cp.holes], U, cp.t[k], cp.t[k + 1], cp.theta_w, w,
            cp.w_phi, cp.mobility, cp.slots, tol, 60, depth=depth)
        assert ok and rc == 0 and st["status"] == 0
        e_err = _rel(P.polar_get_state(el)[0], U[0])
        h_err = _rel(P.polar_get_state(ho)[0], U[1])
        p_err = _rel(P.polar_get_state(ph)[0], phi)
        print(f"PARITY gummel {precision} depth {depth} scale {scale} step {k}: electrons "
              f"{e_err:.3e}, holes {h_err:.3e}, phi {p_err:.3e}; potential solves GPU "
              f"{st['iters']} oracle {iters}")
        assert max(e_err, h_err, p_err) <= 1e-9
        assert abs(st["iters"] - iters) <= (1 if depth == 0 else 2)
        assert P.polar_get_state(el)[1] == cp.t[k + 1]
    P.polar_gummel_destroy(g)


def test_gummel_rejects_bad_setups():
    P, driver = _lib()
    cp = pi.coupled_pair(m=8, n=16)
    ph = driver.create(cp.phi, P.POLAR_FP64)
    el = driver.create(cp.electrons, P.POLAR_FP64)
    other = pi.coupled_pair(m=9, n=16)
    ho = driver.create(other.holes, P.POLAR_FP64)
    with pytest.raises(P.PolarError):        # meshes differ
        P.polar_gummel_create(ph, el, ho, cp.mobility, 0, 1)
    ho = driver.create(cp.holes, P.POLAR_FP64)
    with pytest.raises(P.PolarError):        # one slot for both densities
        P.polar_gummel_create(ph, el, ho, cp.mobility, 0, 0)
    with pytest.raises(P.PolarError):        # slot out of range
        P.polar_gummel_create(ph, el, ho, cp.mobility, 0, 3)
    g = P.polar_gummel_create(ph, el, ho, cp.mobility, 0, 1, max_iter=1)
    with pytest.raises(P.PolarError):        # one potential solve cannot test convergence
        P.polar_gummel_step(g, 0.0, 0.02, 0.5, [1.0, 1.0], [1.0, 1.0], cp.w_phi)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_assembly_matches_host_assembly(precision):
    # A Gummel step with an enormous tol stops after its second potential solve, so the
    # carriers keep the operators the step assembled on the device from phi_0, the
    # potential of the initial densities.  The same drift, built here through the host
    # path (polar_face_drift to host arrays, polar_set_coeffs), must give the same
    # operator and the same next step
    P, driver = _lib()
    cp = pi.coupled_pair(m=24, n=48, K=3)
    prec = P.POLAR_FP64 if precision == "fp64" else P.POLAR_MIXED
    ph = driver.create(cp.phi, prec)
    el = driver.create(cp.electrons, prec)
    ho = driver.create(cp.holes, prec)
    P.polar_set_state(ph, np.zeros(cp.phi.N), 0.0)
    g = P.polar_gummel_create(ph, el, ho, cp.mobility, cp.slots[0], cp.slots[1], tol=1e300,
                              max_iter=5)
    w1 = [1.0, 1.0]
    st, _ = P.polar_gummel_step(g, cp.t[0], cp.t[1], cp.theta_w, w1, w1, cp.w_phi)
    assert st["iters"] == 2
    # phi_0 from the initial densities, through the host upload of the sources
    src = [cp.electrons.u0, cp.holes.u0, cp.phi.src[2]]
    phi0 = driver.create(replace(cp.phi, src=src), prec)
    P.polar_set_state(phi0, np.zeros(cp.phi.N), 0.0)
    P.polar_solve_steady(phi0, cp.w_phi)
    gb = sum(wq * bq for wq, bq in zip(cp.w_phi, cp.phi.bnd))
    rng = np.random.default_rng(11)
    x = rng.standard_normal(cp.phi.N)
    for k, (ctx, prob) in enumerate(((el, cp.electrons), (ho, cp.holes))):
        vr, vt = P.polar_face_drift(phi0, cp.mobility[k], gb)
        host = driver.create(replace(prob, v_rface=vr, v_tface=vt), prec)
        y_dev = P.polar_apply_operator(ctx, 50.0, 0.5, x)
        y_host = P.polar_apply_operator(host, 50.0, 0.5, x)
        op_err = _rel(y_dev, y_host)
        # one more step of both from the same state
        P.polar_set_state(ctx, prob.u0, cp.t[0])
        P.polar_set_state(host, prob.u0, cp.t[0])
        sd, _ = P.polar_advance(ctx, cp.t[0:2], cp.theta_w, np.ones((2, 1)))
        sh, _ = P.polar_advance(host, cp.t[0:2], cp.theta_w, np.ones((2, 1)))
        st_err = _rel(P.polar_get_state(ctx)[0], P.polar_get_state(host)[0])
        print(f"PARITY device vs host assembly {precision} carrier {k}: operator {op_err:.2e}, "
              f"step {st_err:.2e}, iterations {sd[0]['iters']} / {sh[0]['iters']}")
        assert op_err <= 1e-13
        assert st_err <= (1e-12 if precision == "fp64" else 1e-9)
        assert abs(sd[0]["iters"] - sh[0]["iters"]) <= 1
    P.polar_gummel_destroy(g)
