"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

* printed error tables of the paper's manufactured examples (Tables 2.1 and 3.1);
* exactness of the scheme on u = alpha t + beta (1 - r^2) on a uniform radial mesh;
* equality of the two operator forms where the paper's stencils coincide;
* discrete mass balance and the M-matrix sign/column-sum structure (Section 2.2);
* second-order convergence of Crank-Nicolson on a smooth solution (Theorem 2.1);
* a separable direct solve (Fourier in theta, tridiagonal in r, origin coupled to the
  mean mode only) for uniform angles.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import polar_inputs as pi
from polar_inputs import meshes
from oracle import polar_oracle as po

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return {int(l.split()[0]): list(map(float, l.split()[1:]))
                for l in f if l.strip() and not l.startswith("#")}


# ------------------------------------------------------------------------------ Table 2.1
@pytest.mark.parametrize("m", [19, 39])
def test_table_2_1_parabolic(m):
    """Section 2.3: literal stencil of Section 2.1, a = 0.4, dt = 0.01, t = 0.1.  The
    maximum error (origin included) reproduces the printed column of stretch (2.4)
    to 1.5 % and the uniform-radius column to 0.5 %."""
    tab = _table("table_2_1.txt")[m]
    for radial, col, tol in (("sine", 0, 0.015), ("uniform", 1, 0.005), ("zhang", 2, 0.06)):
        p = pi.paper_parabolic_e1(m, radial=radial)
        U = po.run(p)
        err = po.max_error(U, p.exact(p.t[-1]), include_origin=True)
        assert abs(err / tab[col] - 1.0) < tol, (radial, err, tab[col])


# ------------------------------------------------------------------------------ Table 3.1
@pytest.mark.parametrize("m", [19, 39])
def test_table_3_1_continuity(m):
    """Section 3.3: literal stencils of Sections 3.2.1/3.2.2 with D = E = r, the printed
    GR, a = 0.5, p = 0.1, q = 1.9, l = 1.5.  Maximum error over the non-origin nodes
    reproduces "Radius Non-adaptation" to 0.5 % and "Uniform Adaptation" to 2.5 %."""
    tab = _table("table_3_1.txt")[m]
    for radial_adaptive, col, tol in ((True, 0, 0.025), (False, 1, 0.005)):
        p = pi.paper_continuity_e3(m, radial_adaptive=radial_adaptive)
        U = po.run(p)
        err = po.max_error(U, p.exact(p.t[-1]), include_origin=False)
        assert abs(err / tab[col] - 1.0) < tol, (radial_adaptive, err, tab[col])


# ------------------------------------------------------------------------------ exactness
def _quadratic_problem(scheme, theta_mesh, th, alpha=0.7, beta=1.3, m=9, K=6, dt=0.05):
    r = meshes.uniform_r(m)
    n = len(theta_mesh)
    R, TH = pi.problems.node_coords(r, theta_mesh)
    return pi.Problem(
        name="quad", r=r, theta=theta_mesh, t=meshes.uniform_time(dt, K), theta_w=th,
        scheme=scheme, d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
        src=[np.full(m * n + 1, alpha + 4 * beta)], bnd=[np.zeros(n), np.ones(n)],
        u0=beta * (1 - R ** 2),
        weights=lambda tt: np.array([1.0, alpha * tt]), b_const=0.0, d0=1.0,
        exact=lambda tt: alpha * tt + beta * (1 - R ** 2))


@pytest.mark.parametrize("scheme", [po.CONSERVATIVE, po.PAPER])
@pytest.mark.parametrize("th", [0.5, 1.0, 0.3])
def test_exact_for_quadratic_in_r(scheme, th):
    """u = alpha t + beta (1 - r^2), f = alpha + 4 beta: the radial stencil and the
    origin row are exact for r^2 on a uniform radial mesh, the angular terms vanish
    and the theta-scheme is exact for u linear in t, so U equals u to rounding."""
    for theta_mesh in (meshes.uniform_theta(12), meshes.density_theta(12, 0.4)):
        p = _quadratic_problem(scheme, theta_mesh, th)
        U = po.run(p)
        assert np.max(np.abs(U - p.exact(p.t[-1]))) < 1e-11


# ------------------------------------------------------------------------------ operator equality
def test_conservative_equals_paper_where_stencils_coincide():
    """With v = 0 the face-flux form reproduces the printed ring rows of Section 3.2.1
    for any D and any angles, and the printed origin row when the angles are uniform
    and D at the origin faces equals D_0."""
    m, n = 7, 11
    r = meshes.sine_stretch(m, 0.7)
    for theta_mesh, uniform in ((meshes.angular_stretch(n, 1.6), False), (meshes.uniform_theta(n), True)):
        rng = np.random.default_rng(5)
        d_r = rng.uniform(0.5, 2.0, (m + 1) * n)
        if uniform:
            d_r.reshape(n, m + 1)[:, 0] = 1.7
        d_t = rng.uniform(0.5, 2.0, m * n)
        b = rng.uniform(0, 1, m * n + 1)
        base = dict(name="x", r=r, theta=theta_mesh, t=np.array([0, 1.0]), theta_w=0.5,
                    d_rface=d_r, d_tface=d_t, src=[], bnd=[], u0=np.zeros(m * n + 1),
                    weights=lambda t: np.zeros(0), b=b, d0=1.7)
        Lc, Bc = po.conservative_operator(pi.Problem(scheme=po.CONSERVATIVE, **base))
        Lp, Bp = po.paper_operator(pi.Problem(scheme=po.PAPER, **base))
        scale = abs(Lc).max()
        rows = slice(0 if uniform else 1, None)
        assert abs(Lc[rows] - Lp[rows]).max() < 1e-13 * scale
        assert abs(Bc - Bp).max() < 1e-13 * scale


# ------------------------------------------------------------------------------ mass balance
def _drift_problem(m=10, n=14, K=5, seed=7, pe=6.0):
    return pi.continuity_problem(m, n, K, seed, theta_w=0.6, pe_target=pe, d_amp=1.3, delta=0.2)


def test_discrete_mass_balance():
    """Control-volume bookkeeping: M^{k+1} - M^k = dt [th (S - F - R)^{k+1} +
    (1-th)(S - F - R)^k] with S = sum V f, F = outflow through r = 1, R = sum V b U."""
    p = _drift_problem()
    g = po.Geometry(p.r, p.theta)
    L, B = po.conservative_operator(p)
    U = p.u0.copy()
    th = p.theta_w
    for k in range(len(p.t) - 1):
        dt = p.t[k + 1] - p.t[k]
        fo, go = po.source(p, p.t[k])
        fn, gn = po.source(p, p.t[k + 1])
        Un = po.step(L, B, U, dt, th, fo, go, fn, gn)
        bal = lambda Uv, f, gb: g.V @ f - po.boundary_outflow(p, Uv, gb) - p.b_const * (g.V @ Uv)
        lhs = po.mass(p, Un) - po.mass(p, U)
        rhs = dt * (th * bal(Un, fn, gn) + (1 - th) * bal(U, fo, go))
        scale = dt * (abs(g.V @ fn) + abs(po.boundary_outflow(p, Un, gn)) + abs(g.V @ Un))
        assert abs(lhs - rhs) < 1e-13 * scale
        U = Un


def test_m_matrix_structure():
    """I/dt + th L (CONSERVATIVE, upwinded drift, Pe up to 20): non-positive
    off-diagonals, positive diagonal, and V-weighted column sums equal to
    V (1/dt + th b) except for ring-m columns, which also lose the boundary flux."""
    p = _drift_problem(pe=20.0)
    g = po.Geometry(p.r, p.theta)
    L, _ = po.conservative_operator(p)
    dt, th = 0.01, 0.6
    A = po.system_matrix(L, dt, th).tocsr()
    off = A - sp.diags(A.diagonal())
    assert off.max() <= 0.0
    assert A.diagonal().min() > 0
    col = (sp.diags(g.V) @ A).sum(axis=0).A1
    target = g.V * (1 / dt + th * p.b_const)
    ring_m = np.zeros(g.N, dtype=bool)
    ring_m[1:] = (np.arange(g.N - 1) % g.m) == g.m - 1
    assert np.allclose(col[~ring_m], target[~ring_m], rtol=1e-12)
    assert np.all(col[ring_m] >= target[ring_m] * (1 - 1e-12))


# ------------------------------------------------------------------------------ convergence
def test_crank_nicolson_second_order():
    """Smooth solution u = e^{-t}(1 - r^2)(1 + r cos theta), th = 0.5: halving h, mu and
    dt together divides the maximum error by about four (Theorem 2.1)."""
    errs = []
    for m in (16, 32, 64):
        n = 2 * m
        K = m // 2
        p = pi.parabolic_problem(meshes.uniform_r(m), meshes.uniform_theta(n),
                                 meshes.uniform_time(0.5 / K, K), 0.5)
        U = po.run(p)
        errs.append(po.max_error(U, p.exact(p.t[-1])))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.75 and rates[-1] > 1.85, (errs, rates)


def test_backward_euler_first_order_in_time():
    """th = 1: at a fixed fine mesh the time error halves with dt."""
    errs = []
    for K in (4, 8, 16):
        p = pi.parabolic_problem(meshes.uniform_r(48), meshes.uniform_theta(96),
                                 meshes.uniform_time(0.8 / K, K), 1.0)
        U = po.run(p)
        errs.append(po.max_error(U, p.exact(p.t[-1])))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 0.85 < min(rates) and max(rates) < 1.2, (errs, rates)


def test_drift_diffusion_converges():
    """Variable D, drift v = -grad(phi) fixed under refinement, b = 1: the upwinded
    scheme converges to the manufactured solution (at least first order)."""
    errs = []
    for m in (8, 16, 32):
        p = pi.continuity_problem(m, 2 * m, m, 11, theta_w=0.5, phi_scale=0.3, delta=0.3)
        p.t = meshes.uniform_time(0.25 / m, m)
        U = po.run(p)
        errs.append(po.max_error(U, p.exact(p.t[-1])))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 0.9, (errs, rates)


# ------------------------------------------------------------------------------ separable solve
def test_separable_fourier_solve_matches_sparse_step():
    """Uniform angles, D = 1, v = 0, constant b: the angular operator is diagonal in the
    discrete Fourier basis (eigenvalues 4 sin^2(k mu / 2) / mu^2), so each mode is a
    radial tridiagonal system; the origin row sees only the mean mode.  One step of
    this solve equals the sparse LU step to rounding."""
    m, n, dt, th, bc = 12, 16, 0.03, 0.55, 0.4
    r = meshes.sine_stretch(m, 1.2)
    theta = meshes.uniform_theta(n)
    rng = np.random.default_rng(3)
    p = pi.Problem(name="sep", r=r, theta=theta, t=np.array([0, dt]), theta_w=th,
                   scheme=po.CONSERVATIVE, d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
                   src=[], bnd=[], u0=np.zeros(m * n + 1), weights=lambda t: np.zeros(0),
                   b_const=bc)
    L, B = po.conservative_operator(p)
    e = rng.standard_normal(m * n + 1)
    U_lu = po.system_matrix(L, dt, th).tocsc()
    import scipy.sparse.linalg as spla
    x_ref = spla.spsolve(U_lu, e)

    # independent solve
    h = np.diff(r)
    ri = r[1:m + 1]
    rp = 0.5 * (r[1:m + 1] + r[2:m + 2])
    rm = 0.5 * (r[0:m] + r[1:m + 1])
    hi, hi1 = h[:m], h[1:m + 1]
    mu = 2 * math.pi / n
    lw = -2 * rm / (ri * hi * (hi + hi1))
    le = -2 * rp / (ri * hi1 * (hi + hi1))
    ldiag = -(lw + le)
    E = e[1:].reshape(n, m)
    Ehat = np.fft.fft(E, axis=0)                                  # modes along theta
    lam = 4 * np.sin(np.arange(n) * mu / 2) ** 2 / mu ** 2
    X = np.zeros((n, m), dtype=complex)
    e0 = e[0]
    h1 = h[0]
    for k in range(n):
        T = np.diag(1 / dt + th * (ldiag + lam[k] / ri ** 2 + bc))
        T += np.diag(th * lw[1:], -1) + np.diag(th * le[:-1], 1)
        rhs = Ehat[k].copy()
        if k == 0:
            # unknowns (x0, mean-mode line); origin row 1/dt x0 + th(4/h1^2 (x0 - mean) + b x0)
            M = np.zeros((m + 1, m + 1))
            M[1:, 1:] = T
            M[1, 0] = th * lw[0] * n                               # line row 1 couples to n * x0
            M[0, 0] = 1 / dt + th * (4 / h1 ** 2 + bc)
            M[0, 1] = -th * 4 / h1 ** 2 / n                         # mean = (mode 0) / n
            sol = np.linalg.solve(M, np.concatenate([[e0], rhs.real]))
            x0 = sol[0]
            X[0] = sol[1:]
        else:
            X[k] = np.linalg.solve(T, rhs)
    x = np.concatenate([[x0], np.fft.ifft(X, axis=0).real.ravel()])
    assert np.max(np.abs(x - x_ref)) < 1e-12 * np.max(np.abs(x_ref))


def test_paper_origin_row_matches_control_volume_balance():
    """Section 3.2.2: the origin row is the control-volume balance
    dn0/dt = 4 D0 (n1 - n0)/dr^2 - (2 E0 / dr) (n0 + n1)/2 + GR with n1 the angle mean
    of ring 1 and dr = h_1; so L U at the origin equals minus that flux part (+ b n0)."""
    m, n = 6, 9
    r = meshes.sine_stretch(m, 0.8)
    theta = meshes.uniform_theta(n)
    rng = np.random.default_rng(2)
    E = rng.uniform(0.2, 1.0, m * n + 1)
    p = pi.Problem(name="o", r=r, theta=theta, t=np.array([0, 1.0]), theta_w=0.5,
                   scheme=po.PAPER, d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
                   src=[], bnd=[], u0=np.zeros(m * n + 1), weights=lambda t: np.zeros(0),
                   e_node=E, b_const=0.3, d0=1.4)
    L, _ = po.paper_operator(p)
    U = rng.standard_normal(m * n + 1)
    h1 = r[1]
    n0, n1 = U[0], U[1:].reshape(n, m)[:, 0].mean()
    balance = 4 * 1.4 * (n1 - n0) / h1 ** 2 - (2 * E[0] / h1) * (n0 + n1) / 2
    assert abs((L @ U)[0] - (-balance + 0.3 * n0)) < 1e-12 * abs(balance)


# ------------------------------------------------------------------------------ sampled rows
def test_sampled_rows_equal_full_assembly():
    """conservative_operator restricted to a set of rows (origin, first and last rings,
    random cells) returns exactly those rows of the full assembly."""
    for p in (_drift_problem(m=17, n=23), pi.config2(m=21, n=30, K=2)):
        L, B = po.conservative_operator(p)
        rng = np.random.default_rng(5)
        for rows in (np.unique(np.concatenate([[0, 1, 2, p.m, p.N - 1],
                                               rng.integers(0, p.N, 40)])),
                     np.unique(rng.integers(1, p.N, 25))):
            Ls, Bs = po.conservative_operator(p, rows)
            assert (Ls != L[rows]).nnz == 0 and (Bs != B[rows]).nnz == 0


def test_step_residual_detects_a_perturbation():
    """The oracle's own step has a Jacobi-scaled residual at rounding level; moving one
    value by d shows up as -d in that row and as the coupling ratio in its neighbours."""
    p = _drift_problem(m=12, n=18, K=2)
    L, B = po.conservative_operator(p)
    dt, th = p.t[1] - p.t[0], p.theta_w
    fo, go = po.source(p, p.t[0])
    fn, gn = po.source(p, p.t[1])
    U1 = po.step(L, B, p.u0, dt, th, fo, go, fn, gn)
    res = po.step_residual(L, B, p.u0, U1, dt, th, fo, go, fn, gn)
    assert np.max(np.abs(res)) < 1e-15 * np.max(np.abs(U1))
    q, d = 1 + 5 * p.m + 7, 1e-6
    U2 = U1.copy()
    U2[q] += d
    res2 = po.step_residual(L, B, p.u0, U2, dt, th, fo, go, fn, gn)
    assert abs(res2[q] + d) < 1e-12
    A = po.system_matrix(L, dt, th).tocsr()
    col = A[:, q].toarray().ravel()
    expect = -col * d / A.diagonal()
    assert np.allclose(res2, expect, atol=1e-15)
    rows = np.array([0, q - 1, q, q + 1, p.N - 1])
    Ls, Bs = po.conservative_operator(p, rows)
    assert np.allclose(po.step_residual(Ls, Bs, p.u0, U2, dt, th, fo, go, fn, gn, rows),
                       res2[rows], rtol=0, atol=1e-18)
