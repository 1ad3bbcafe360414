"""Pins of the coupled-system oracle (steady solve, face drift, Gummel step).

The steady solve is pinned to a closed form the conservative scheme reproduces exactly
(phi = 1 - r^2 on uniform radii) and to a dense LAPACK solve of the matrix assembled node
by node from the printed formulas; the face drift to closed forms (linear in r:
exact; r cos(theta) on uniform angles: the angular difference quotient equals
sin(theta_{j+1/2}) sin(dtheta/2) / (dtheta/2)); the Gummel step to special cases whose
answer is known without it (zero mobility decouples the carriers; a symmetric pair has
zero net charge and so zero field) and to the direction of the drift each sign selects;
the Anderson-accelerated step to a least-squares solve, to the plain iteration's fixed
point, and to convergence where the plain iteration fails (a fixed point of the map).
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import polar_inputs as pi
from polar_inputs import meshes
from polar_inputs.problems import node_coords
from oracle import coupled as oc
from oracle import polar_oracle as po

from test_oracle_dense import _dense_conservative, _small_problem


def _poisson(r, theta, d, source, g):
    m, n = len(r) - 2, len(theta)
    N = m * n + 1
    return pi.Problem(name="poisson", r=r, theta=theta, t=np.array([0.0, 1.0]), theta_w=1.0,
                      scheme=po.CONSERVATIVE, d_rface=np.full((m + 1) * n, d),
                      d_tface=np.full(m * n, d), src=[source], bnd=[g], u0=np.zeros(N),
                      weights=lambda tt: np.array([1.0]))


@pytest.mark.parametrize("m,n,angles", [(8, 16, "uniform"), (13, 21, "stretched"),
                                        (32, 48, "density")])
@pytest.mark.parametrize("d", [1.0, 0.37])
def test_steady_reproduces_quadratic_on_uniform_radii(m, n, angles, d):
    # -div(d grad phi) = 4 d with phi = 0 on r = 1 has phi = 1 - r^2; the control-volume
    # balance is exact for it on uniform radii (face fluxes 2 d r_{i+1/2}^2 w_j, volumes
    # r_i h w_j, origin disk pi h^2 / 4)
    r = meshes.uniform_r(m)
    theta = {"uniform": meshes.uniform_theta(n), "stretched": meshes.angular_stretch(n, 1.4),
             "density": meshes.density_theta(n, 1.1)}[angles]
    R, _ = node_coords(r, theta)
    prob = _poisson(r, theta, d, np.full(m * n + 1, 4.0 * d), np.zeros(n))
    phi = oc.steady(prob, [1.0])
    assert np.max(np.abs(phi - (1.0 - R ** 2))) < 1e-13


def test_steady_quadratic_is_not_exact_on_graded_radii():
    # the same problem on stretched radii carries a truncation error: the pin above is a
    # property of the uniform mesh, not of any solver
    r = meshes.sine_stretch(16, 0.8)
    theta = meshes.uniform_theta(32)
    R, _ = node_coords(r, theta)
    phi = oc.steady(_poisson(r, theta, 1.0, np.full(16 * 32 + 1, 4.0), np.zeros(32)), [1.0])
    assert np.max(np.abs(phi - (1.0 - R ** 2))) > 1e-6


@pytest.mark.parametrize("m,n", [(3, 5), (4, 8), (6, 5)])
@pytest.mark.parametrize("drift", [False, True])
def test_steady_equals_dense_solve(m, n, drift):
    prob = _small_problem(m, n, po.CONSERVATIVE, drift, uniform_angles=False, seed=100 * m + n)
    L, B = _dense_conservative(prob)
    w = np.array([0.7, -1.3])
    f = w[0] * prob.src[0] + w[1] * prob.src[1]
    g = w[0] * prob.bnd[0] + w[1] * prob.bnd[1]
    dense = np.linalg.solve(L, f - B @ g)
    got = oc.steady(prob, w)
    assert np.max(np.abs(got - dense)) / np.max(np.abs(dense)) < 1e-12


@pytest.mark.parametrize("mob", [1.0, -2.5])
def test_face_drift_linear_in_r_is_exact(mob):
    r = meshes.capped_geometric(20, 1.03, True)
    theta = meshes.density_theta(24, 0.4)
    R, _ = node_coords(r, theta)
    a, b = 0.3, -1.7
    vr, vt = oc.face_drift(r, theta, a + b * R, np.full(24, a + b), mob)
    assert np.max(np.abs(vr + mob * b)) < 1e-13
    assert np.max(np.abs(vt)) == 0.0


@pytest.mark.parametrize("n", [16, 40])
def test_face_drift_of_x_coordinate(n):
    # u = r cos(theta): radial quotients are cos(theta_j) exactly (u is linear in r along
    # a line, origin value 0); angular ones are sin(theta_{j+1/2}) sinc(dtheta / 2)
    m, mob = 12, 0.8
    r = meshes.sine_stretch(m, 0.7)
    theta = meshes.uniform_theta(n)
    R, TH = node_coords(r, theta)
    vr, vt = oc.face_drift(r, theta, R * np.cos(TH), np.cos(theta), mob)
    vr = vr.reshape(n, m + 1)
    vt = vt.reshape(n, m)
    assert np.max(np.abs(vr + mob * np.cos(theta)[:, None])) < 1e-13  # rounding / h
    dth = 2.0 * math.pi / n
    half = theta + 0.5 * dth
    want = mob * np.sin(half) * math.sin(0.5 * dth) / (0.5 * dth)
    assert np.max(np.abs(vt - want[:, None])) < 1e-13


def _run(cp, mobility=None, steps=1, tol=1e-12):
    mob = cp.mobility if mobility is None else mobility
    U = [cp.electrons.u0.copy(), cp.holes.u0.copy()]
    out = []
    for k in range(steps):
        w = [np.array([1.0, 1.0]), np.array([1.0, 1.0])]
        U, phi, iters, change, ok = oc.gummel_step(
            cp.phi, [cp.electrons, cp.holes], U, cp.t[k], cp.t[k + 1], cp.theta_w, w,
            cp.w_phi, mob, cp.slots, tol, 60)
        assert ok
        out.append((U, phi, iters, change))
    return out


def _plain_step(prob, U, t0, t1, theta):
    L, B = po.operator(prob)
    f, g = po.source_w(prob, [1.0])
    return po.step(L, B, U, t1 - t0, theta, f, g, f, g)


def test_gummel_zero_mobility_decouples():
    cp = pi.coupled_pair(m=10, n=20)
    (U, phi, iters, change), = _run(cp, mobility=(0.0, 0.0))
    for c, prob in enumerate((cp.electrons, cp.holes)):
        want = _plain_step(prob, prob.u0, cp.t[0], cp.t[1], cp.theta_w)
        assert np.max(np.abs(U[c] - want)) / np.max(np.abs(want)) < 1e-14
    # the potential of the final densities, and no change once they are fixed
    src = [U[0], U[1], cp.phi.src[2]]
    assert np.max(np.abs(phi - oc.steady(replace(cp.phi, src=src), cp.w_phi))) < 1e-14
    assert iters == 3 and change == 0.0


def test_gummel_symmetric_pair_has_no_field():
    # identical carriers, opposite drift signs, no doping and phi = 0 on the rim: the
    # net charge p - n vanishes, so does phi, and both carriers take a plain step
    cp = pi.coupled_pair(m=10, n=20)
    N = cp.phi.N
    holes = replace(cp.electrons, name="holes")
    phi = replace(cp.phi, src=[np.zeros(N), np.zeros(N), np.zeros(N)],
                  bnd=[np.zeros(cp.phi.n)] * 3)
    cp = replace(cp, phi=phi, holes=holes)
    (U, phi_k, iters, _), = _run(cp, mobility=(-1.5, 1.5))
    assert np.max(np.abs(phi_k)) < 1e-15
    want = _plain_step(cp.electrons, cp.electrons.u0, cp.t[0], cp.t[1], cp.theta_w)
    for c in range(2):
        assert np.max(np.abs(U[c] - want)) / np.max(np.abs(want)) < 1e-14


def _inner_mass(prob, U, radius):
    geo = po.Geometry(prob.r, prob.theta)
    R, _ = node_coords(prob.r, prob.theta)
    return float(np.sum((geo.V * U)[R < radius]))


def test_gummel_drift_directions():
    # positive net charge in the centre (doping bump, phi = 0 on the rim) raises phi
    # there: electrons (v = +mu grad phi) gather toward the centre, holes (v = -mu grad
    # phi) leave it, relative to no field
    cp = pi.coupled_pair(m=16, n=32, scale=2.0)
    cp = replace(cp, phi=replace(cp.phi, bnd=[np.zeros(cp.phi.n)] * 3))
    (U, phi, _, _), = _run(cp)
    (U0, _, _, _), = _run(cp, mobility=(0.0, 0.0))
    R, _ = node_coords(cp.phi.r, cp.phi.theta)
    assert phi[0] > np.max(phi[R > 0.9])
    assert _inner_mass(cp.electrons, U[0], 0.5) > _inner_mass(cp.electrons, U0[0], 0.5)
    assert _inner_mass(cp.holes, U[1], 0.5) < _inner_mass(cp.holes, U0[1], 0.5)


def test_gummel_result_is_a_fixed_point():
    cp = pi.coupled_pair(m=12, n=24)
    (U, phi, iters, change), = _run(cp, tol=1e-13)
    assert iters >= 3 and change <= 1e-13
    # one more map from the converged potential changes the densities by about tol
    g_phi = po.source_w(cp.phi, cp.w_phi)[1]
    for c, prob in enumerate((cp.electrons, cp.holes)):
        vr, vt = oc.face_drift(prob.r, prob.theta, phi, g_phi, cp.mobility[c])
        again = _plain_step(replace(prob, v_rface=vr, v_tface=vt), prob.u0, cp.t[0], cp.t[1],
                            cp.theta_w)
        assert np.max(np.abs(again - U[c])) / np.max(np.abs(U[c])) < 1e-11


def test_anderson_gamma_is_the_least_squares_solution():
    rng = np.random.default_rng(5)
    cols = [rng.standard_normal(200) for _ in range(3)]
    f = rng.standard_normal(200)
    gam, kept = oc.anderson_gamma(cols, f)
    want, *_ = np.linalg.lstsq(np.stack(cols, 1), f, rcond=None)
    assert kept == 3 and np.max(np.abs(gam - want)) < 1e-12
    # a column that repeats an older one makes the Gram matrix singular: the oldest goes
    gam, kept = oc.anderson_gamma([cols[0], cols[1], cols[0].copy()], f)
    want, *_ = np.linalg.lstsq(np.stack([cols[1], cols[0]], 1), f, rcond=None)
    assert kept == 2 and np.max(np.abs(gam - want)) < 1e-12


def _step(cp, depth, tol=1e-12, max_iter=60):
    w = [np.array([1.0, 1.0]), np.array([1.0, 1.0])]
    return oc.gummel_step(cp.phi, [cp.electrons, cp.holes], [cp.electrons.u0, cp.holes.u0],
                          cp.t[0], cp.t[1], cp.theta_w, w, cp.w_phi, cp.mobility, cp.slots,
                          tol, max_iter, depth=depth)


@pytest.mark.parametrize("scale", [1.0, 4.0])
def test_anderson_reaches_the_plain_fixed_point(scale):
    cp = pi.coupled_pair(m=16, n=32, scale=scale)
    U0, phi0, it0, _, ok0 = _step(cp, 0)
    U3, phi3, it3, _, ok3 = _step(cp, 3)
    assert ok0 and ok3 and it3 < it0
    assert np.max(np.abs(phi3 - phi0)) / np.max(np.abs(phi0)) < 1e-11
    for a, b in zip(U3, U0):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-11


def test_anderson_converges_where_plain_gummel_does_not():
    cp = pi.coupled_pair(m=16, n=32, scale=8.0)
    assert not _step(cp, 0)[4]
    U, phi, it, change, ok = _step(cp, 3)
    assert ok and change <= 1e-12
    g_phi = po.source_w(cp.phi, cp.w_phi)[1]
    for c, prob in enumerate((cp.electrons, cp.holes)):   # a fixed point of the map
        vr, vt = oc.face_drift(prob.r, prob.theta, phi, g_phi, cp.mobility[c])
        again = _plain_step(replace(prob, v_rface=vr, v_tface=vt), prob.u0, cp.t[0], cp.t[1],
                            cp.theta_w)
        assert np.max(np.abs(again - U[c])) / np.max(np.abs(U[c])) < 1e-10
