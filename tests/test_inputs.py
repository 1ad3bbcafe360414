"""Input generators: SplitMix64 known answers and mesh invariants (Sections 2.1, 3.1)."""
import math
import os

import numpy as np
import pytest

import polar_inputs as pi
from polar_inputs import meshes
from polar_inputs.rng import SplitMix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_values():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for seed, *expect in rows:
        g = SplitMix64(seed)
        assert [g.next_u64() for _ in expect] == expect


@pytest.mark.parametrize("gen", [
    lambda: meshes.uniform_r(17), lambda: meshes.sine_stretch(17, 1.0),
    lambda: meshes.sine_stretch(17, 0.1), lambda: meshes.zhang_stretch(17, 0.6),
    lambda: meshes.capped_geometric(33, 1.03, True), lambda: meshes.capped_geometric(33, 1.03, False),
    lambda: meshes.capped_geometric(2048, 1.03, True)])
def test_radial_mesh_endpoints_monotone(gen):
    r = gen()
    assert r[0] == 0.0 and r[-1] == 1.0            # v(0) = 0, v(1) = 1 (Section 2.1)
    assert np.all(np.diff(r) > 0)


def test_capped_geometric_ratio():
    r = meshes.capped_geometric(200, 1.03, True)
    h = np.diff(r)
    ratios = h[1:] / h[:-1]
    assert np.isclose(ratios[0], 1.03) and np.isclose(ratios[-1], 1 / 1.03)
    assert np.isclose(h[0], h[-1])                  # symmetric grading
    graded = ratios[np.abs(ratios - 1.0) > 1e-3]
    assert np.allclose(np.maximum(graded, 1 / graded), 1.03, rtol=1e-12)


def test_angular_and_time_stretch_endpoints():
    th = meshes.angular_stretch(50, 1.9)
    assert th[0] == 0.0 and np.all(np.diff(th) > 0) and th[-1] < 2 * math.pi
    t = meshes.time_stretch(0.1, 1.5, 10)
    assert t[0] == 0.0 and t[-1] == 0.1 and np.all(np.diff(t) > 0)
    assert np.isclose(t[5], 0.1 * math.sin(0.5 ** 1.5 * math.pi / 2))


def test_density_theta_equidistributes():
    th0 = 1.234
    th = meshes.density_theta(256, th0)
    F = th + 0.5 * (np.sin(th - th0) + math.sin(th0))
    assert np.max(np.abs(F - 2 * math.pi * np.arange(256) / 256)) < 1e-13
    # local spacing ~ 1 / density
    mid = 0.5 * (th[1:] + th[:-1])
    dens = 1 + 0.5 * np.cos(mid - th0)
    sp = np.diff(th) * dens
    assert np.allclose(sp, 2 * math.pi / 256, rtol=1e-3)


def test_geometric_time():
    t = meshes.geometric_time(1e-4, 1.01, 1000)
    assert np.isclose(t[-1], 1e-4 * (1.01 ** 1000 - 1) / 0.01, rtol=1e-12)


def test_manufactured_sources_satisfy_pde_numerically():
    """The continuity source is n_t + L_c n for the continuous operator: check by
    finite differences of the closed-form fields at interior points."""
    prob = pi.continuity_problem(8, 16, 4, 123, phi_scale=0.7, delta=0.3)
    F = pi.problems._ContinuityFields(123, 1.0, 0.3)
    F.phi_scale = 0.7
    rng = np.random.default_rng(0)
    pts = rng.uniform(-0.5, 0.5, size=(20, 2))
    x, y = pts[:, 0], pts[:, 1]
    e = 1e-4

    def nstar(t, x, y):
        (A, *_), (B, *_) = F.parts(x, y)
        return math.exp(-t) * A + B

    def flux(t, x, y):
        D, _, _ = F.D(x, y)
        vx, vy, _ = F.vel(x, y)
        nx = (nstar(t, x + e, y) - nstar(t, x - e, y)) / (2 * e)
        ny = (nstar(t, x, y + e) - nstar(t, x, y - e)) / (2 * e)
        nn = nstar(t, x, y)
        return -D * nx + vx * nn, -D * ny + vy * nn

    t = 0.3
    fx1, _ = flux(t, x + e, y)
    fx0, _ = flux(t, x - e, y)
    _, fy1 = flux(t, x, y + e)
    _, fy0 = flux(t, x, y - e)
    div = (fx1 - fx0) / (2 * e) + (fy1 - fy0) / (2 * e)
    nt = (nstar(t + e, x, y) - nstar(t - e, x, y)) / (2 * e)
    f_expected = nt + div + 1.0 * nstar(t, x, y)
    # evaluate the separable source at the same points
    Dn, Dx, Dy = F.gradD(x, y)
    vx, vy, divv = F.vel(x, y)
    (A, Ax, Ay, lA), (B, Bx, By, lB) = F.parts(x, y)
    L = lambda P, Px, Py, lP: -(Dx * Px + Dy * Py) - Dn * lP + P * divv + vx * Px + vy * Py + P
    f = math.exp(-t) * (-A + L(A, Ax, Ay, lA)) + L(B, Bx, By, lB)
    assert np.allclose(f, f_expected, rtol=1e-5, atol=1e-5)


def test_chunked_field_evaluation_matches_whole_arrays():
    """Large workloads evaluate their fields in chunks on a thread pool; the values agree with
    one evaluation over the whole arrays to the rounding of the 8-term mode sums (the BLAS
    products may order them differently), ragged last chunk included."""
    from polar_inputs.problems import _chunked, _ContinuityFields
    F = _ContinuityFields(15879002, 1.3, 0.05)
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, 1, 1001), rng.uniform(-1, 1, 1001)
    whole = F.D(x, y)[0]
    assert np.allclose(_chunked(lambda a, b: F.D(a, b)[0], x, y, chunk=64), whole,
                       rtol=1e-14, atol=0)
    vx, vy, dv = F.vel(x, y)
    got = _chunked(lambda a, b: F.vel(a, b), x, y, nout=3, chunk=100)
    for g_, w_ in zip(got, (vx, vy, dv)):
        assert np.allclose(g_, w_, rtol=1e-13, atol=1e-13 * np.max(np.abs(w_)))


def test_coupled_pair_is_seeded_and_consistent():
    a, b = pi.coupled_pair(m=12, n=24), pi.coupled_pair(m=12, n=24)
    for pa, pb in ((a.phi, b.phi), (a.electrons, b.electrons), (a.holes, b.holes)):
        assert np.array_equal(pa.d_rface, pb.d_rface) and np.array_equal(pa.u0, pb.u0)
        assert pa.m == 12 and pa.n == 24 and np.array_equal(pa.r, a.phi.r)
        assert np.array_equal(pa.theta, a.phi.theta)
    c = pi.coupled_pair(m=12, n=24, seed=7)
    assert not np.array_equal(c.electrons.d_rface, a.electrons.d_rface)
    # the potential's source weights put the densities in with opposite signs and the
    # carriers' drift signs are opposite
    assert a.w_phi[a.slots[0]] == -a.w_phi[a.slots[1]]
    assert a.mobility[0] * a.mobility[1] < 0
    assert np.all(a.electrons.u0 > 0) and np.all(a.holes.u0 > 0)
