"""FP64 CPU oracle for the implicit theta-weighted step on the polar mesh.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this module.  It shares no code with the
CUDA library: it assembles the discrete operator as a sparse matrix straight from the
paper's formulas and solves every time step with a sparse direct factorisation.

Vector order (Eq. 2.12): index 0 = origin, index 1 + j*m + (i-1) = node (r_i, theta_j).

Notation
--------
h_i = r_i - r_{i-1} (i = 1..m+1), r_{i+1/2} = (r_i + r_{i+1})/2            (Section 2.1)
mu_j = theta_j - theta_{j-1} (j = 1..n-1), mu_0 = mu_n = 2 pi - theta_{n-1} (Section 3.1)
k_i = (h_i + h_{i+1})/2,  w_j = (mu_j + mu_{j+1})/2                          (cell widths)
V_ij = r_i k_i w_j,  V_0 = pi h_1^2 / 4 (the disk of radius h_1/2 of Section 3.2.2).

Two spatial operators L (the equation is u_t + L u = f):

* CONSERVATIVE (``conservative_operator``): cell-centred control volumes with face
  fluxes shared by both neighbours.  Flux out of a cell through a face =
  face length * ( D (U_in - U_out) / spacing + upwinded v U ).  With v = 0 the ring
  rows reduce to the stencil of Section 3.2.1 (and to Section 2.1's with D = 1) and
  the origin row to the control-volume row of Section 3.2.2 (Swarztrauber-Sweet row of
  Section 2.1 when D = 1); the angle mean is weighted by w_j / (2 pi) and the drift
  through the origin faces is upwinded face by face.
* PAPER (``paper_operator``): the printed stencils verbatim -- ring rows of
  Section 3.2.1 with scalar E at nodes and forward differences, the origin row of
  Section 3.2.2 (unweighted angle mean 1/n with D_0, E_0), plus b U.

Time step (Eq. 2.5 / 2.11 with the implicit weight th = 1 - a):
  (I/dt + th L) U^{k+1} = (I/dt - (1-th) L) U^k - (1-th) B g^k - th B g^{k+1}
                          + (1-th) f^k + th f^{k+1},
where B maps the Dirichlet ring values g_j = U_{m+1,j} (Eq. 2.9) into the rows of
ring m.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

CONSERVATIVE = 0
PAPER = 1


class Geometry:
    """Mesh metrics of Section 2.1 / 3.1 for nodes r[0..m+1] and angles theta[0..n-1]."""

    def __init__(self, r, theta):
        r = np.asarray(r, dtype=np.float64)
        theta = np.asarray(theta, dtype=np.float64)
        self.m = m = len(r) - 2
        self.n = n = len(theta)
        self.r = r
        self.theta = theta
        self.h = np.diff(r)                                    # h[i-1] = h_i, i = 1..m+1
        self.rh = 0.5 * (r[:-1] + r[1:])                       # rh[i] = r_{i+1/2}, i = 0..m
        mu = np.empty(n + 1)                                   # mu[j] = mu_j, j = 0..n
        mu[1:n] = np.diff(theta)
        mu[n] = 2.0 * math.pi - theta[n - 1] + theta[0]
        mu[0] = mu[n]
        self.mu = mu
        self.w = 0.5 * (mu[:n] + mu[1:])                       # w[j] = (mu_j + mu_{j+1})/2
        self.k = 0.5 * (self.h[:m] + self.h[1:])               # k[i-1] = (h_i + h_{i+1})/2
        ri = r[1:m + 1]
        self.V = np.empty(m * n + 1)
        self.V[0] = math.pi * self.h[0] ** 2 / 4.0
        self.V[1:] = np.outer(self.w, ri * self.k).ravel()     # [j, i-1]
        self.N = m * n + 1

    def idx(self, i, j):
        """Vector index of node (r_i, theta_j), i >= 1 (arrays broadcast)."""
        return 1 + j * self.m + (i - 1)


def conservative_operator(prob, rows=None):
    """Sparse L and boundary map B of the CONSERVATIVE scheme: N x N and N x n, or, when
    ``rows`` (sorted distinct vector indices) is given, only those rows (len(rows) x N and
    len(rows) x n), built from the faces of those cells alone.

    Radial face (i+1/2, j), i = 0..m: length w_j r_{i+1/2}, spacing h_{i+1},
      flux = w_j r_{i+1/2} [ (D/h_{i+1} + v+) U_in - (D/h_{i+1} + v-) U_out ],
      U_in = U_0 for i = 0, U_out = g_j for i = m.
    Angular face (i, j+1/2), i = 1..m: length k_i, spacing r_i mu_{j+1},
      flux = k_i [ (D/(r_i mu_{j+1}) + w+) U_{i,j} - (D/(r_i mu_{j+1}) + w-) U_{i,j+1} ].
    Row of a cell = (sum of outward fluxes) / V + b U.
    """
    g = Geometry(prob.r, prob.theta)
    m, n, N = g.m, g.n, g.N
    rows_, cols, vals = [], [], []
    brow, bcol, bval = [], [], []

    def add(rw, cl, v):
        rows_.append(np.ravel(rw)); cols.append(np.ravel(cl)); vals.append(np.ravel(v))

    # faces to visit: all of them, or those of the requested cells
    if rows is None:
        J, I = np.meshgrid(np.arange(n), np.arange(m + 1), indexing="ij")
        Jr, Ir = J.ravel(), I.ravel()                                      # radial faces
        J, I = np.meshgrid(np.arange(n), np.arange(1, m + 1), indexing="ij")
        Jt, It = J.ravel(), I.ravel()                                      # angular faces
    else:
        rows = np.asarray(rows, dtype=np.int64)
        cell = rows[rows > 0] - 1
        ci, cj = cell % m + 1, cell // m                                   # ring, angle
        fr = [np.stack([cj, ci - 1]), np.stack([cj, ci])]                  # faces i -+ 1/2
        if rows[0] == 0:
            fr.append(np.stack([np.arange(n), np.zeros(n, dtype=np.int64)]))
        fr = np.unique(np.concatenate(fr, axis=1), axis=1)
        Jr, Ir = fr[0], fr[1]
        ft = np.unique(np.concatenate([np.stack([cj, ci]), np.stack([(cj - 1) % n, ci])],
                                      axis=1), axis=1)                     # faces j -+ 1/2
        Jt, It = ft[0], ft[1]

    # radial faces
    D = np.asarray(prob.d_rface, dtype=np.float64).reshape(n, m + 1)[Jr, Ir]
    v = (np.zeros_like(D) if prob.v_rface is None
         else np.asarray(prob.v_rface, dtype=np.float64).reshape(n, m + 1)[Jr, Ir])
    length = g.w[Jr] * g.rh[Ir]
    cond = D / g.h[Ir]                                                      # h[i] = h_{i+1}
    c_in = length * (cond + np.maximum(v, 0.0))
    c_out = length * (cond + np.maximum(-v, 0.0))
    inner = np.where(Ir == 0, 0, g.idx(np.maximum(Ir, 1), Jr))
    outer_is_bnd = Ir == m
    outer = np.where(outer_is_bnd, -1, g.idx(np.minimum(Ir + 1, m), Jr))
    V_in = g.V[inner]
    # row of the inner cell: + flux / V_in
    add(inner, inner, c_in / V_in)
    nb = ~outer_is_bnd
    add(inner[nb], outer[nb], -c_out[nb] / V_in[nb])
    brow.append(inner[outer_is_bnd]); bcol.append(Jr[outer_is_bnd])
    bval.append(-c_out[outer_is_bnd] / V_in[outer_is_bnd])
    # row of the outer cell: - flux / V_out
    V_out = g.V[outer[nb]]
    add(outer[nb], inner[nb], -c_in[nb] / V_out)
    add(outer[nb], outer[nb], c_out[nb] / V_out)

    # angular faces
    D = np.asarray(prob.d_tface, dtype=np.float64).reshape(n, m)[Jt, It - 1]
    wv = (np.zeros_like(D) if prob.v_tface is None
          else np.asarray(prob.v_tface, dtype=np.float64).reshape(n, m)[Jt, It - 1])
    ri = g.r[It]
    mu_next = g.mu[Jt + 1]                                                  # mu_{j+1}
    length = g.k[It - 1]
    cond = D / (ri * mu_next)
    c_in = length * (cond + np.maximum(wv, 0.0))
    c_out = length * (cond + np.maximum(-wv, 0.0))
    left = g.idx(It, Jt)
    right = g.idx(It, (Jt + 1) % n)
    add(left, left, c_in / g.V[left])
    add(left, right, -c_out / g.V[left])
    add(right, left, -c_in / g.V[right])
    add(right, right, c_out / g.V[right])

    # reaction
    diag = np.arange(N) if rows is None else rows
    b = (np.full(len(diag), prob.b_const) if prob.b is None
         else np.asarray(prob.b, dtype=np.float64)[diag])
    add(diag, diag, b)

    R, C, X = np.concatenate(rows_), np.concatenate(cols), np.concatenate(vals)
    Rb, Cb, Xb = np.concatenate(brow), np.concatenate(bcol), np.concatenate(bval)
    nrow = N
    if rows is not None:   # keep the entries of the requested rows, renumbered 0..len-1
        pos = np.searchsorted(rows, R).clip(0, len(rows) - 1)
        keep = rows[pos] == R
        R, C, X = pos[keep], C[keep], X[keep]
        pos = np.searchsorted(rows, Rb).clip(0, len(rows) - 1)
        keep = rows[pos] == Rb
        Rb, Cb, Xb = pos[keep], Cb[keep], Xb[keep]
        nrow = len(rows)
    L = sp.coo_matrix((X, (R, C)), shape=(nrow, N)).tocsr()
    B = sp.coo_matrix((Xb, (Rb, Cb)), shape=(nrow, n)).tocsr()
    return L, B


def paper_operator(prob):
    """Sparse L and B of the printed stencils (Section 3.2.1 ring rows, Section 3.2.2
    origin row; Section 2.1 when D = 1, E = 0 and the angles are uniform), plus b U."""
    g = Geometry(prob.r, prob.theta)
    m, n, N = g.m, g.n, g.N
    J, I = np.meshgrid(np.arange(n), np.arange(1, m + 1), indexing="ij")    # [j, i-1]
    Dr = np.asarray(prob.d_rface, dtype=np.float64).reshape(n, m + 1)
    Dt = np.asarray(prob.d_tface, dtype=np.float64).reshape(n, m)
    E = (np.zeros(N) if prob.e_node is None else np.asarray(prob.e_node, dtype=np.float64))
    Eij = E[1:].reshape(n, m)
    ri = g.r[1:m + 1][None, :]
    hi = g.h[:m][None, :]                     # h_i
    hi1 = g.h[1:m + 1][None, :]               # h_{i+1}
    rm = g.rh[:m][None, :]                    # r_{i-1/2}
    rp = g.rh[1:m + 1][None, :]               # r_{i+1/2}
    Dm = Dr[:, :m]                            # D_{i-1/2,j}
    Dp = Dr[:, 1:m + 1]                       # D_{i+1/2,j}
    mu_j = g.mu[:n][:, None]                  # mu_j
    mu_j1 = g.mu[1:n + 1][:, None]            # mu_{j+1}
    Dn = Dt                                   # D_{i,j+1/2}
    Ds = np.roll(Dt, 1, axis=0)               # D_{i,j-1/2}
    b = np.full(N, prob.b_const) if prob.b is None else np.asarray(prob.b, dtype=np.float64)

    west = -2.0 * rm * Dm / (ri * hi * (hi + hi1))
    east = -(2.0 * rp * Dp / (ri * hi1 * (hi + hi1)) + Eij / hi1)
    south = -2.0 * Ds / (ri ** 2 * mu_j * (mu_j + mu_j1))
    north = -(2.0 * Dn / (ri ** 2 * mu_j1 * (mu_j + mu_j1)) + Eij / (ri * mu_j1))
    diag = (2.0 / (ri * (hi + hi1)) * (rp * Dp / hi1 + rm * Dm / hi)
            + 2.0 / (ri ** 2 * (mu_j + mu_j1)) * (Dn / mu_j1 + Ds / mu_j)
            + Eij * (1.0 / (ri * mu_j1) + 1.0 / hi1)) + b[1:].reshape(n, m)

    me = g.idx(I, J)
    rows, cols, vals = [me], [me], [diag]
    w_idx = np.where(I == 1, 0, g.idx(np.maximum(I - 1, 1), J))
    rows.append(me); cols.append(w_idx); vals.append(west)
    inner = I < m
    rows.append(me[inner]); cols.append(g.idx(I + 1, J)[inner]); vals.append(east[inner])
    rows.append(me); cols.append(g.idx(I, (J - 1) % n)); vals.append(south)
    rows.append(me); cols.append(g.idx(I, (J + 1) % n)); vals.append(north)
    # origin row, Section 3.2.2
    h1 = g.h[0]
    D0, E0 = prob.d0, E[0]
    rows.append(np.array([0])); cols.append(np.array([0]))
    vals.append(np.array([4.0 * D0 / h1 ** 2 + E0 / h1 + b[0]]))
    j = np.arange(n)
    rows.append(np.zeros(n, dtype=int)); cols.append(g.idx(1, j))
    vals.append(np.full(n, -(4.0 * D0 / (n * h1 ** 2) - E0 / (n * h1))))
    L = sp.coo_matrix((np.concatenate([np.ravel(v) for v in vals]),
                       (np.concatenate([np.ravel(x) for x in rows]),
                        np.concatenate([np.ravel(x) for x in cols]))), shape=(N, N)).tocsr()
    bnd = I == m
    B = sp.coo_matrix((east[bnd], (me[bnd], J[bnd])), shape=(N, n)).tocsr()
    return L, B


def operator(prob):
    return paper_operator(prob) if prob.scheme == PAPER else conservative_operator(prob)


def source(prob, tk):
    """f(t_k) and g(t_k) from the separable terms: sum_q w_q(t_k) S_q, sum_q w_q(t_k) G_q."""
    w = np.asarray(prob.weights(tk), dtype=np.float64)
    f = sum(w[q] * np.asarray(prob.src[q], dtype=np.float64) for q in range(len(prob.src)))
    gb = sum(w[q] * np.asarray(prob.bnd[q], dtype=np.float64) for q in range(len(prob.bnd)))
    return f, gb


def source_w(prob, w):
    """f and g for an explicit weight vector w (as passed to the library)."""
    w = np.asarray(w, dtype=np.float64)
    f = sum(w[q] * np.asarray(prob.src[q], dtype=np.float64) for q in range(len(prob.src)))
    gb = sum(w[q] * np.asarray(prob.bnd[q], dtype=np.float64) for q in range(len(prob.bnd)))
    return f, gb


def rhs(L, B, U, dt, th, f_old, g_old, f_new, g_new):
    """Right-hand side of Eq. (2.11) with th = 1 - a."""
    return (U / dt - (1.0 - th) * (L @ U + B @ g_old) - th * (B @ g_new)
            + (1.0 - th) * f_old + th * f_new)


def system_matrix(L, dt, th):
    """I/dt + th L, the matrix of Eq. (2.12) divided by dt."""
    return (sp.identity(L.shape[0], format="csr") / dt + th * L).tocsc()


def residual_extended(A, x, e):
    """e - A x accumulated in extended precision (numpy longdouble), rounded to FP64."""
    A = A.tocsr()
    prod = A.data.astype(np.longdouble) * x.astype(np.longdouble)[A.indices]
    rows = np.add.reduceat(prod, A.indptr[:-1])
    return (e.astype(np.longdouble) - rows).astype(np.float64)


def step(L, B, U, dt, th, f_old, g_old, f_new, g_new, lu=None, A=None):
    """One theta-step (Eq. 2.11): sparse LU solve followed by one step of iterative
    refinement whose residual is accumulated in extended precision, so the result is
    the discrete solution to rounding rather than to (condition number) x rounding."""
    e = rhs(L, B, U, dt, th, f_old, g_old, f_new, g_new)
    if A is None:
        A = system_matrix(L, dt, th)
    if lu is None:
        lu = spla.splu(A.tocsc())
    x = lu.solve(e)
    return x + lu.solve(residual_extended(A, x, e))


def _matvec_ext(M, x):
    """M x with products and sums in numpy longdouble (empty rows give 0)."""
    M = M.tocsr()
    out = np.zeros(M.shape[0], dtype=np.longdouble)
    if M.nnz == 0:
        return out
    prod = M.data.astype(np.longdouble) * x[M.indices].astype(np.longdouble)
    full = M.indptr[1:] > M.indptr[:-1]
    out[full] = np.add.reduceat(prod, M.indptr[:-1][full])
    return out


def step_residual(L, B, U_old, U_new, dt, th, f_old, g_old, f_new, g_new, rows=None):
    """Jacobi-scaled residual (e - A U_new)_i / A_ii of the theta-step (Eq. 2.11,
    A = I/dt + th L) for a candidate new level U_new, accumulated in extended precision.
    With ``rows``, L and B hold only those rows (conservative_operator(prob, rows)) and
    the residual is returned for them alone; U and f are full vectors either way."""
    sel = np.arange(L.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    ld = np.longdouble
    inv_dt = ld(1.0) / ld(dt)
    th = ld(th)
    e = (U_old[sel].astype(ld) * inv_dt
         - (1 - th) * (_matvec_ext(L, U_old) + _matvec_ext(B, g_old))
         - th * _matvec_ext(B, g_new)
         + (1 - th) * f_old[sel].astype(ld) + th * f_new[sel].astype(ld))
    AU = U_new[sel].astype(ld) * inv_dt + th * _matvec_ext(L, U_new)
    Lc = L.tocsr()
    diag = np.asarray(Lc[np.arange(len(sel)), sel]).ravel().astype(ld)
    return ((e - AU) / (inv_dt + th * diag)).astype(np.float64)


def run(prob, nsteps=None, callback=None):
    """Advance prob.u0 over prob.t[0..nsteps]; returns U at t[nsteps].
    ``callback(k, U)`` is called after each step k = 1..nsteps."""
    L, B = operator(prob)
    t = prob.t
    K = len(t) - 1 if nsteps is None else nsteps
    U = np.asarray(prob.u0, dtype=np.float64).copy()
    f_old, g_old = source(prob, t[0])
    lu, lu_dt, A = None, None, None
    for k in range(K):
        dt = t[k + 1] - t[k]
        if lu is None or abs(dt - lu_dt) > 1e-15 * dt:
            A = system_matrix(L, dt, prob.theta_w)
            lu, lu_dt = spla.splu(A), dt
        f_new, g_new = source(prob, t[k + 1])
        U = step(L, B, U, dt, prob.theta_w, f_old, g_old, f_new, g_new, lu, A)
        f_old, g_old = f_new, g_new
        if callback is not None:
            callback(k + 1, U)
    return U


# ---------------------------------------------------------------------------------------
# diagnostics

def mass(prob, U):
    """Discrete mass sum V U over all control volumes (V_0 = pi h_1^2 / 4)."""
    return float(Geometry(prob.r, prob.theta).V @ U)


def boundary_outflow(prob, U, gb):
    """Total CONSERVATIVE flux through the faces i = m+1/2 into the Dirichlet ring."""
    g = Geometry(prob.r, prob.theta)
    m, n = g.m, g.n
    D = np.asarray(prob.d_rface, dtype=np.float64).reshape(n, m + 1)[:, m]
    v = (np.zeros(n) if prob.v_rface is None
         else np.asarray(prob.v_rface, dtype=np.float64).reshape(n, m + 1)[:, m])
    length = g.w * g.rh[m]
    cond = D / g.h[m]
    Um = U[1:].reshape(n, m)[:, m - 1]
    return float(np.sum(length * ((cond + np.maximum(v, 0)) * Um - (cond + np.maximum(-v, 0)) * gb)))


def max_error(U, exact, include_origin=True):
    d = np.abs(U - exact)
    return float(d.max() if include_origin else d[1:].max())


def mean_error(U, exact, include_origin=True):
    d = np.abs(U - exact)
    return float(d.mean() if include_origin else d[1:].mean())
