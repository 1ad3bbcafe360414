"""Pin P4 of the oracle: whole theta-steps on tiny meshes against a dense direct solve.

The N x N matrix of each step is assembled here node by node, in plain Python loops,
straight from the printed formulas -- the control-volume balance of every cell (face
fluxes shared by the two cells of a face, Section 3.2.1 with the origin cell of
Section 3.2.2) and the printed stencils of Sections 2.1 / 3.2.1 / 3.2.2 -- without
calling the oracle's sparse assembly (conservative_operator / paper_operator).  The step
(Eq. 2.11 with the implicit weight th = 1 - a, Dirichlet data at both levels) is then
solved with LAPACK's dense LU (numpy.linalg.solve) and compared with the oracle's
sparse step, m in {3, 4, 6}, n in {5, 8}, both schemes, with and without drift.

A dropped face, a transposed neighbour, a wrong spacing or a sign slip in either
assembly moves the two solutions apart by far more than the 1e-13 allowed here.
"""
import math

import numpy as np
import pytest

import polar_inputs as pi
from polar_inputs import meshes
from oracle import polar_oracle as po


# ----------------------------------------------------------------------------- inputs
def _small_problem(m, n, scheme, drift, uniform_angles, seed):
    """Random coefficients, sources, Dirichlet data and state on a stretched mesh."""
    rng = np.random.default_rng(seed)
    r = meshes.sine_stretch(m, 0.8)
    theta = meshes.uniform_theta(n) if uniform_angles else meshes.angular_stretch(n, 1.4)
    N = m * n + 1
    d_r = rng.uniform(0.5, 2.0, (m + 1) * n)
    d_t = rng.uniform(0.5, 2.0, m * n)
    kw = {}
    if scheme == po.CONSERVATIVE and drift:
        kw["v_rface"] = rng.uniform(-4.0, 4.0, (m + 1) * n)
        kw["v_tface"] = rng.uniform(-4.0, 4.0, m * n)
    if scheme == po.PAPER and drift:
        kw["e_node"] = rng.uniform(0.0, 2.0, N)
    src = [rng.standard_normal(N), rng.standard_normal(N)]
    bnd = [rng.standard_normal(n), rng.standard_normal(n)]
    return pi.Problem(
        name="dense", r=r, theta=theta, t=np.array([0.0, 0.03, 0.07]), theta_w=0.5,
        scheme=scheme, d_rface=d_r, d_tface=d_t, src=src, bnd=bnd,
        u0=rng.standard_normal(N),
        weights=lambda tt: np.array([math.exp(-tt), 1.0 + tt]),
        b=rng.uniform(0.0, 1.5, N), d0=1.3, **kw)


# ----------------------------------------------------------------------------- mesh
class _Mesh:
    """Mesh quantities of Sections 2.1 / 3.1 with the paper's indices (1-based h, mu)."""

    def __init__(self, prob):
        self.m, self.n = m, n = prob.m, prob.n
        self.r = [float(v) for v in prob.r]                       # r_0 .. r_{m+1}
        self.h = [None] + [self.r[i] - self.r[i - 1] for i in range(1, m + 2)]
        th = [float(v) for v in prob.theta]
        self.mu = [None] * (n + 1)                                # mu_1 .. mu_n
        for j in range(1, n):
            self.mu[j] = th[j] - th[j - 1]
        self.mu[n] = 2.0 * math.pi + th[0] - th[n - 1]
        self.mu[0] = self.mu[n]

    def rh(self, i):          # r_{i+1/2}
        return 0.5 * (self.r[i] + self.r[i + 1])

    def mu_(self, j):         # mu_j with the periodic wrap
        return self.mu[j % self.n] if j % self.n else self.mu[self.n]

    def wcell(self, j):       # angular width of cell j: (mu_j + mu_{j+1}) / 2
        return 0.5 * (self.mu_(j) + self.mu_(j + 1))

    def kcell(self, i):       # radial width of ring i: (h_i + h_{i+1}) / 2
        return 0.5 * (self.h[i] + self.h[i + 1])

    def vol(self, i, j):
        return math.pi * self.h[1] ** 2 / 4.0 if i == 0 else self.r[i] * self.kcell(i) * self.wcell(j)

    def col(self, i, j):      # unknown index (Eq. 2.12 order); None on the Dirichlet ring
        if i == 0:
            return 0
        if i == self.m + 1:
            return None
        return 1 + (j % self.n) * self.m + (i - 1)


def _face(arr, n_per_line, j, i):
    return float(arr[j * n_per_line + i])


# ----------------------------------------------------------------------------- assembly
def _dense_conservative(prob):
    """L (N x N) and the Dirichlet map B (N x n) of the control-volume scheme, cell by cell:
    row(cell) = (sum of the fluxes out of the cell through its faces) / V_cell + b U_cell.
    Flux through a radial face (i+1/2, j), outward (toward larger r):
        w_j r_{i+1/2} [ D (U_{i,j} - U_{i+1,j}) / h_{i+1} + v+ U_{i,j} - v- U_{i+1,j} ],
    through an angular face (i, j+1/2), toward larger theta:
        k_i [ D (U_{i,j} - U_{i,j+1}) / (r_i mu_{j+1}) + w+ U_{i,j} - w- U_{i,j+1} ]."""
    g = _Mesh(prob)
    m, n = g.m, g.n
    N = m * n + 1
    L = np.zeros((N, N))
    B = np.zeros((N, n))
    vr = prob.v_rface
    vt = prob.v_tface
    b = np.full(N, prob.b_const) if prob.b is None else np.asarray(prob.b)

    def put(row, i, j, coef):
        c = g.col(i, j)
        if c is None:
            B[row, j % n] += coef
        else:
            L[row, c] += coef

    def radial_flux(row, sign, i, j):
        """sign * (flux through face (i+1/2, j)) / V added to `row`."""
        D = _face(prob.d_rface, m + 1, j, i)
        v = 0.0 if vr is None else _face(vr, m + 1, j, i)
        length = g.wcell(j) * g.rh(i)
        cond = D / g.h[i + 1]
        put(row, i, j, sign * length * (cond + max(v, 0.0)))
        put(row, i + 1, j, -sign * length * (cond + max(-v, 0.0)))

    def angular_flux(row, sign, i, j):
        """sign * (flux through face (i, j+1/2)) added to `row` (face of angles j, j+1)."""
        jj = j % n
        D = _face(prob.d_tface, m, jj, i - 1)
        w = 0.0 if vt is None else _face(vt, m, jj, i - 1)
        length = g.kcell(i)
        cond = D / (g.r[i] * g.mu_(jj + 1))
        put(row, i, jj, sign * length * (cond + max(w, 0.0)))
        put(row, i, jj + 1, -sign * length * (cond + max(-w, 0.0)))

    for j in range(n):
        for i in range(1, m + 1):
            row = g.col(i, j)
            V = g.vol(i, j)
            radial_flux(row, +1.0, i, j)            # east face, out of the cell
            radial_flux(row, -1.0, i - 1, j)        # west face, into the cell
            angular_flux(row, +1.0, i, j)           # north face
            angular_flux(row, -1.0, i, j - 1)       # south face
            L[row] /= V
            B[row] /= V
            L[row, row] += b[row]
    # origin cell: the n radial faces (1/2, j), all outward
    for j in range(n):
        radial_flux(0, +1.0, 0, j)
    L[0] /= g.vol(0, 0)
    B[0] /= g.vol(0, 0)
    L[0, 0] += b[0]
    return L, B


def _dense_paper(prob):
    """L and B of the printed stencils: ring rows of Section 3.2.1 (D at faces, E at nodes,
    forward differences) and the origin row of Section 3.2.2, each plus b U."""
    g = _Mesh(prob)
    m, n = g.m, g.n
    N = m * n + 1
    L = np.zeros((N, N))
    B = np.zeros((N, n))
    E = np.zeros(N) if prob.e_node is None else np.asarray(prob.e_node)
    b = np.full(N, prob.b_const) if prob.b is None else np.asarray(prob.b)
    for j in range(n):
        for i in range(1, m + 1):
            row = g.col(i, j)
            ri, hi, hi1 = g.r[i], g.h[i], g.h[i + 1]
            rm, rp = g.rh(i - 1), g.rh(i)
            Dm = _face(prob.d_rface, m + 1, j, i - 1)
            Dp = _face(prob.d_rface, m + 1, j, i)
            Dn = _face(prob.d_tface, m, j, i - 1)
            Ds = _face(prob.d_tface, m, (j - 1) % n, i - 1)
            mj, mj1 = g.mu_(j), g.mu_(j + 1)
            e = E[row]
            diag = (2.0 / (ri * (hi + hi1)) * (rp * Dp / hi1 + rm * Dm / hi)
                    + 2.0 / (ri * ri * (mj + mj1)) * (Dn / mj1 + Ds / mj)
                    + e * (1.0 / (ri * mj1) + 1.0 / hi1))
            L[row, row] += diag + b[row]
            L[row, g.col(i - 1, j)] += -2.0 * rm * Dm / (ri * hi * (hi + hi1))
            east = -(2.0 * rp * Dp / (ri * hi1 * (hi + hi1)) + e / hi1)
            if i == m:
                B[row, j] += east
            else:
                L[row, g.col(i + 1, j)] += east
            L[row, g.col(i, j - 1)] += -2.0 * Ds / (ri * ri * mj * (mj + mj1))
            L[row, g.col(i, j + 1)] += -(2.0 * Dn / (ri * ri * mj1 * (mj + mj1)) + e / (ri * mj1))
    h1, D0, E0 = g.h[1], prob.d0, E[0]
    L[0, 0] += 4.0 * D0 / h1 ** 2 + E0 / h1 + b[0]
    for j in range(n):
        L[0, g.col(1, j)] += -(4.0 * D0 / (n * h1 ** 2) - E0 / (n * h1))
    return L, B


def _dense_steps(prob, L, B, K):
    """K theta-steps of Eq. 2.11 (implicit weight th = 1 - a) by dense LU."""
    th = prob.theta_w
    U = np.asarray(prob.u0, dtype=np.float64).copy()
    I = np.eye(L.shape[0])
    out = []
    for k in range(K):
        t0, t1 = prob.t[k], prob.t[k + 1]
        dt = t1 - t0
        w0, w1 = prob.weights(t0), prob.weights(t1)
        f0 = sum(w0[q] * prob.src[q] for q in range(len(prob.src)))
        f1 = sum(w1[q] * prob.src[q] for q in range(len(prob.src)))
        g0 = sum(w0[q] * prob.bnd[q] for q in range(len(prob.bnd)))
        g1 = sum(w1[q] * prob.bnd[q] for q in range(len(prob.bnd)))
        rhs = ((I / dt - (1.0 - th) * L) @ U - (1.0 - th) * (B @ g0) - th * (B @ g1)
               + (1.0 - th) * f0 + th * f1)
        U = np.linalg.solve(I / dt + th * L, rhs)
        out.append(U.copy())
    return out


CASES = [(m, n, scheme, drift)
         for m in (3, 4, 6) for n in (5, 8)
         for scheme in (po.CONSERVATIVE, po.PAPER) for drift in (False, True)]


@pytest.mark.parametrize("m,n,scheme,drift", CASES)
def test_dense_assembly_equals_oracle_operator(m, n, scheme, drift):
    """The oracle's sparse L and B equal the node-by-node dense assembly entry by entry,
    on non-uniform angles (and, for the printed origin row, on uniform ones)."""
    for uniform in (False, True):
        prob = _small_problem(m, n, scheme, drift, uniform, seed=100 * m + n)
        Ld, Bd = (_dense_conservative if scheme == po.CONSERVATIVE else _dense_paper)(prob)
        Ls, Bs = po.operator(prob)
        scale = np.abs(Ld).max()
        assert np.abs(Ls.toarray() - Ld).max() <= 1e-14 * scale
        assert np.abs(Bs.toarray() - Bd).max() <= 1e-14 * scale


@pytest.mark.parametrize("m,n,scheme,drift", CASES)
def test_dense_solve_equals_oracle_step(m, n, scheme, drift):
    """Two variable-dt theta-steps (Crank-Nicolson and theta = 0.6): the oracle's sparse
    step (LU + extended-precision refinement) equals the dense LAPACK solve of the
    dense-assembled system to 1e-13 relative in the max norm."""
    for th in (0.5, 0.6):
        prob = _small_problem(m, n, scheme, drift, uniform_angles=(n == 8), seed=7 * m + n)
        prob.theta_w = th
        Ld, Bd = (_dense_conservative if scheme == po.CONSERVATIVE else _dense_paper)(prob)
        dense = _dense_steps(prob, Ld, Bd, 2)
        got = []
        po.run(prob, 2, callback=lambda k, U: got.append(U.copy()))
        for k in range(2):
            rel = np.max(np.abs(got[k] - dense[k])) / np.max(np.abs(dense[k]))
            assert rel <= 1e-13, (k, th, rel)


def test_dense_parabolic_row_of_section_2_1():
    """With D = 1, E = 0, b = 0 and uniform angles the printed stencil of Section 2.1
    (diagonal 2/(r_i (h_i + h_{i+1})) (r_{i+1/2}/h_{i+1} + r_{i-1/2}/h_i) + 2/(r_i mu)^2,
    angular neighbours -1/(r_i mu)^2, origin 4/h_1^2 and -4/(n h_1^2)) is what both dense
    assemblies give."""
    m, n = 5, 8
    r = meshes.sine_stretch(m, 0.7)
    theta = meshes.uniform_theta(n)
    N = m * n + 1
    prob = pi.Problem(name="p21", r=r, theta=theta, t=np.array([0.0, 0.1]), theta_w=0.6,
                      scheme=po.PAPER, d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
                      src=[], bnd=[], u0=np.zeros(N), weights=lambda tt: np.zeros(0),
                      b_const=0.0, d0=1.0)
    g = _Mesh(prob)
    mu = 2.0 * math.pi / n
    L21 = np.zeros((N, N))
    for j in range(n):
        for i in range(1, m + 1):
            row = g.col(i, j)
            ri, hi, hi1 = g.r[i], g.h[i], g.h[i + 1]
            L21[row, row] = (2.0 / (ri * (hi + hi1)) * (g.rh(i) / hi1 + g.rh(i - 1) / hi)
                             + 2.0 / (ri * ri * mu * mu))
            L21[row, g.col(i - 1, j)] = -2.0 * g.rh(i - 1) / (ri * hi * (hi + hi1))
            if i < m:
                L21[row, g.col(i + 1, j)] = -2.0 * g.rh(i) / (ri * hi1 * (hi + hi1))
            L21[row, g.col(i, j - 1)] += -1.0 / (ri * ri * mu * mu)
            L21[row, g.col(i, j + 1)] += -1.0 / (ri * ri * mu * mu)
    L21[0, 0] = 4.0 / g.h[1] ** 2
    for j in range(n):
        L21[0, g.col(1, j)] = -4.0 / (n * g.h[1] ** 2)
    scale = np.abs(L21).max()
    for dense in (_dense_paper(prob)[0], _dense_conservative(
            pi.Problem(**{**prob.__dict__, "scheme": po.CONSERVATIVE}))[0]):
        assert np.abs(dense - L21).max() <= 1e-13 * scale
