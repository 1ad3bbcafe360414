"""FP64 CPU oracle for the electron-hole pair coupled to a potential.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this module.  It shares no code with the CUDA
library; it builds on ``polar_oracle`` (sparse assembly from the paper's formulas and
sparse direct solves).

The system (Section 3.1: the continuity equation Eq. 3.1 for each carrier; the field
from a Poisson equation as in the outlook of Section 4):

    n_t = div(D_n grad n - v_n n) - b_n n + f_n,     v_n = -s_n grad phi
    p_t = div(D_p grad p - v_p p) - b_p p + f_p,     v_p = -s_p grad phi
    -div(eps grad phi) = sum_q w_q S_q               (two of the S_q are n and p)

with Dirichlet data on r = 1 for all three; s_c is the signed mobility (s_n = -mu_n for
electrons, which drift up the potential gradient; s_p = +mu_p for holes).

Discrete drift (the face quantities the conservative scheme's fluxes use): the radial
component at radial face (i+1/2, j) is -s (phi_{i+1,j} - phi_{i,j}) / h_{i+1}, with
phi_{0,j} the origin value and phi_{m+1,j} the Dirichlet value; the angular component at
angular face (i, j+1/2) is -s (phi_{i,j+1} - phi_{i,j}) / (r_i mu_{j+1}), periodic in j.

Gummel's iteration for one theta-step t0 -> t1 (the drift held over the step), as a
fixed-point map G on the potential, G(x) = Poisson(densities advanced with the drift of x):
    x_0 = Poisson(n^k, p^k)
    for j = 0, 1, ...:
        g_j = G(x_j), f_j = g_j - x_j
        stop when max|f_j| / max|g_j| <= tol (the absolute change when g_j = 0); phi = g_j
        x_{j+1} = g_j                                   (depth 0: plain Gummel)
        x_{j+1} = g_j - sum_a gamma_a (dX_a + dF_a)     (Anderson acceleration, depth d)
where dX_a, dF_a are the last min(d, j) differences of consecutive x and f, and gamma
minimises |f_j - dF gamma|_2 through the normal equations (dF^T dF) gamma = dF^T f_j by
Cholesky; if a pivot is not above 1e-13 times the largest diagonal entry the oldest
difference is dropped and the solve repeated (Anderson 1965; Walker and Ni 2011 for the
form with g).
"""
from dataclasses import replace

import numpy as np
import scipy.sparse.linalg as spla

from . import polar_oracle as po


def steady(prob, w):
    """U with L U + B g = f (Eq. 2.1 / 3.1 without the time derivative), f and g the
    sources and Dirichlet fields weighted by w: sparse LU and one step of refinement
    with an extended-precision residual."""
    L, B = po.operator(prob)
    f, g = po.source_w(prob, w)
    e = f - B @ g
    A = L.tocsc()
    lu = spla.splu(A)
    x = lu.solve(e)
    return x + lu.solve(po.residual_extended(A, x, e))


def face_drift(r, theta, u, g, mobility):
    """(v_rface, v_tface) = -mobility grad u at the faces (layouts j (m+1) + i and
    j m + i - 1), u in the vector order of polar_oracle, g the values on r = 1."""
    geo = po.Geometry(r, theta)
    m, n = geo.m, geo.n
    full = np.empty((n, m + 2))
    full[:, 0] = u[0]
    full[:, 1:m + 1] = np.asarray(u[1:], dtype=np.float64).reshape(n, m)
    full[:, m + 1] = g
    vr = -mobility * (full[:, 1:] - full[:, :-1]) / geo.h[None, :]
    ri = geo.r[1:m + 1]
    ring = full[:, 1:m + 1]
    nxt = np.roll(ring, -1, axis=0)                       # row j holds phi_{i, j+1}
    vt = -mobility * (nxt - ring) / (ri[None, :] * geo.mu[1:n + 1][:, None])
    return vr.ravel(), vt.ravel()


def anderson_gamma(dF, f):
    """gamma of the Anderson step: the normal equations (dF^T dF) gamma = dF^T f by
    Cholesky, the oldest column dropped while a pivot is not above 1e-13 times the largest
    diagonal entry.  dF: list of columns, oldest first.  Returns (gamma, columns kept)."""
    cols = list(dF)
    while cols:
        A = np.array([[float(a @ b) for b in cols] for a in cols])
        rhs = np.array([float(a @ f) for a in cols])
        k = len(cols)
        Lc = np.zeros((k, k))
        ok = True
        top = max(A[i, i] for i in range(k))
        for i in range(k):
            for j in range(i + 1):
                acc = A[i, j] - sum(Lc[i, q] * Lc[j, q] for q in range(j))
                if i == j:
                    if not acc > 1e-13 * top:
                        ok = False
                        break
                    Lc[i, i] = np.sqrt(acc)
                else:
                    Lc[i, j] = acc / Lc[j, j]
            if not ok:
                break
        if ok:
            y = np.zeros(k)
            for i in range(k):
                y[i] = (rhs[i] - sum(Lc[i, q] * y[q] for q in range(i))) / Lc[i, i]
            gam = np.zeros(k)
            for i in reversed(range(k)):
                gam[i] = (y[i] - sum(Lc[q, i] * gam[q] for q in range(i + 1, k))) / Lc[i, i]
            return gam, len(cols)
        cols = cols[1:]
    return np.zeros(0), 0


def gummel_step(phi_prob, car_probs, U_car, t0, t1, theta, w_car, w_phi, mobility, slots,
                tol, max_iter, depth=0):
    """One coupled theta-step.  car_probs / U_car / w_car / mobility: electrons then
    holes (w_car[c] = weights at t0 followed by those at t1); slots: the potential's
    source slots that receive the electron and the hole densities; depth: Anderson depth
    (0: plain Gummel).  Returns (densities, phi, potential solves, last change,
    converged)."""
    g_phi = po.source_w(phi_prob, w_phi)[1]
    start = [np.asarray(u, dtype=np.float64).copy() for u in U_car]
    U = [u.copy() for u in start]
    phi_prev, change = None, 0.0
    dX, dF, x_last, f_last = [], [], None, None      # Anderson histories
    for it in range(max_iter):
        src = list(phi_prob.src)
        src[slots[0]], src[slots[1]] = U[0], U[1]
        phi = steady(replace(phi_prob, src=src), w_phi)
        if it > 0:
            diff, size = float(np.max(np.abs(phi - phi_prev))), float(np.max(np.abs(phi)))
            change = diff / size if size > 0 else diff     # phi = 0: the absolute change
            if change <= tol:
                return U, phi, it + 1, change, True
            if depth > 0:
                f = phi - phi_prev
                if f_last is not None:
                    dF = (dF + [f - f_last])[-depth:]
                    dX = (dX + [phi_prev - x_last])[-depth:]
                x_last, f_last = phi_prev, f
                gam, kept = anderson_gamma(dF, f)
                x = phi.copy()
                for a, ga in enumerate(gam):
                    col = len(dF) - kept + a
                    x = x - ga * (dX[col] + dF[col])
                phi = x
        phi_prev = phi
        for c in range(2):
            vr, vt = face_drift(phi_prob.r, phi_prob.theta, phi, g_phi, mobility[c])
            pc = replace(car_probs[c], v_rface=vr, v_tface=vt)
            L, B = po.operator(pc)
            Q = len(pc.src)
            f_old, g_old = po.source_w(pc, np.asarray(w_car[c][:Q]))
            f_new, g_new = po.source_w(pc, np.asarray(w_car[c][Q:2 * Q]))
            U[c] = po.step(L, B, start[c], t1 - t0, theta, f_old, g_old, f_new, g_new)
    return U, phi, max_iter, change, False
