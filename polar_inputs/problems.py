"""Synthetic problems: meshes, coefficients, separable sources, boundary data,
initial state and time schedule, for the paper's manufactured examples and for the
five benchmark workloads.  Nothing here discretises the equation: every field is a
closed-form function of (t, r, theta) sampled at nodes or face centres.

Vector layout (the paper's ordering of Eq. (2.12)): index 0 is the origin node,
index 1 + j*m + (i-1) is node (r_i, theta_j), i = 1..m, j = 0..n-1 -- radial lines
are contiguous.  Face arrays:

* ``d_rface``/``v_rface``: (m+1)*n values at radial faces (r_{i+1/2}, theta_j),
  i = 0..m, index j*(m+1) + i (i = 0 is the face of the origin cell).
* ``d_tface``/``v_tface``: m*n values at angular faces (r_i, theta_{j+1/2}),
  i = 1..m, index j*m + (i-1); theta_{n-1/2} = (theta_{n-1} + 2 pi)/2.

Sources and Dirichlet data are separable in time: f(t) = sum_q w_q(t) S_q and
g(t) = sum_q w_q(t) G_q with the same weights w_q(t).
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import meshes
from .rng import SplitMix64

SCHEME_CONSERVATIVE = 0
SCHEME_PAPER = 1

SEED_BASE = 15879000


@dataclass
class Problem:
    name: str
    r: np.ndarray
    theta: np.ndarray
    t: np.ndarray
    theta_w: float                       # implicit weight = 1 - a  (a weights the old level, Eq. 2.5)
    scheme: int
    d_rface: np.ndarray
    d_tface: np.ndarray
    src: List[np.ndarray]
    bnd: List[np.ndarray]
    u0: np.ndarray
    weights: Callable[[float], np.ndarray]
    v_rface: Optional[np.ndarray] = None
    v_tface: Optional[np.ndarray] = None
    e_node: Optional[np.ndarray] = None  # scalar E at nodes (paper's continuity stencil only)
    b: Optional[np.ndarray] = None
    b_const: float = 0.0
    d0: float = 1.0                      # D at the origin (paper's origin row only)
    exact: Optional[Callable[[float], np.ndarray]] = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return len(self.r) - 2

    @property
    def n(self) -> int:
        return len(self.theta)

    @property
    def N(self) -> int:
        return self.m * self.n + 1

    def weight_table(self) -> np.ndarray:
        """(K+1) x Q array of w_q(t_k)."""
        return np.array([self.weights(tk) for tk in self.t], dtype=np.float64).reshape(len(self.t), -1)


# ----------------------------------------------------------------------------------------
# node / face coordinates

def node_coords(r, theta):
    """(R, TH) of every unknown in vector order; the origin is (0, 0)."""
    m, n = len(r) - 2, len(theta)
    R = np.empty(m * n + 1)
    TH = np.empty(m * n + 1)
    R[0], TH[0] = 0.0, 0.0
    R[1:] = np.tile(r[1:m + 1], n)
    TH[1:] = np.repeat(theta, m)
    return R, TH


def rface_coords(r, theta):
    m, n = len(r) - 2, len(theta)
    rh = 0.5 * (r[:-1] + r[1:])                      # r_{i+1/2}, i = 0..m
    return np.tile(rh, n), np.repeat(theta, m + 1)


def tface_coords(r, theta):
    m, n = len(r) - 2, len(theta)
    th_next = np.concatenate([theta[1:], [2.0 * math.pi]])
    th_half = 0.5 * (theta + th_next)               # theta_{j+1/2}, j = 0..n-1
    return np.tile(r[1:m + 1], n), np.repeat(th_half, m)



# ----------------------------------------------------------------------------------------
# the paper's manufactured examples (used to pin the oracle against its printed tables)

def paper_parabolic_e1(m: int, radial: str = "sine", p: float = 1.0, ptilde: float = 0.6,
                       a: float = 0.4, dt: float = 0.01, T: float = 0.1) -> Problem:
    """Section 2.3, Numerical Experiment 1: u = e^{-t} r^2 + r^2 sqrt(1-r), b = 0,
    f as printed, u = e^{-t} on r = 1, n = floor(2 m pi), uniform angles, uniform dt.
    ``radial`` selects Eq. (2.4) ('sine', parameter p), Eq. (2.13) ('zhang', p~) or
    a uniform mesh ('uniform')."""
    n = int(math.floor(2 * m * math.pi))
    r = {"sine": lambda: meshes.sine_stretch(m, p),
         "zhang": lambda: meshes.zhang_stretch(m, ptilde),
         "uniform": lambda: meshes.uniform_r(m)}[radial]()
    theta = meshes.uniform_theta(n)
    K = int(round(T / dt))
    t = meshes.uniform_time(dt, K)
    R, TH = node_coords(r, theta)
    sq = np.sqrt(1.0 - R)
    S1 = -R ** 2 - 4.0
    S2 = -4.0 * sq + 5.0 * R / (2.0 * sq) + R ** 2 / (4.0 * sq ** 3)
    return Problem(
        name=f"paper_e1_{radial}_m{m}", r=r, theta=theta, t=t, theta_w=1.0 - a,
        scheme=SCHEME_PAPER,
        d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
        src=[S1, S2], bnd=[np.ones(n), np.zeros(n)],
        u0=R ** 2 + R ** 2 * sq,
        weights=lambda tt: np.array([math.exp(-tt), 1.0]),
        b_const=0.0, d0=1.0,
        exact=lambda tt: math.exp(-tt) * R ** 2 + R ** 2 * sq,
        meta=dict(table="2.1", a=a, radial=radial))


def paper_continuity_e3(m: int, radial_adaptive: bool = True, angle_adaptive: bool = True,
                        time_adaptive: bool = True, p: float = 0.1, q: float = 1.9,
                        l: float = 1.5, a: float = 0.5, T: float = 0.1, dtt: float = 0.01) -> Problem:
    """Section 3.3, Numerical Experiment 1 of the continuity equation: D = E = r,
    n = e^{-t} r + r sqrt(1-r) + r sin^2(theta), GR as printed, n = e^{-t} + sin^2(theta)
    on r = 1; radial (2.4) with p, angular stretch with q, time stretch with l."""
    n = int(math.floor(2 * m * math.pi))
    r = meshes.sine_stretch(m, p) if radial_adaptive else meshes.uniform_r(m)
    theta = meshes.angular_stretch(n, q) if angle_adaptive else meshes.uniform_theta(n)
    K = int(round(T / dtt))
    t = meshes.time_stretch(T, l, K) if time_adaptive else meshes.uniform_time(T / K, K)
    R, TH = node_coords(r, theta)
    sq = np.sqrt(1.0 - R)
    s2 = np.sin(TH) ** 2
    S1 = -R - 2.0 + 3.0 * R
    S2 = (-(2.0 * sq - 2.0 * R / sq + 0.25 * R ** 2 / sq ** 3 + 2.0 * s2 + 2.0 * np.cos(2 * TH))
          + 3.0 * R * sq - 0.5 * R ** 2 / sq + 3.0 * R * s2 + np.sin(2 * TH) * R)
    rr, _ = rface_coords(r, theta)
    tr, _ = tface_coords(r, theta)
    return Problem(
        name=f"paper_e3_m{m}", r=r, theta=theta, t=t, theta_w=1.0 - a, scheme=SCHEME_PAPER,
        d_rface=rr.copy(), d_tface=tr.copy(),
        src=[S1, S2], bnd=[np.ones(n), np.sin(theta) ** 2],
        u0=R + R * sq + R * s2,
        weights=lambda tt: np.array([math.exp(-tt), 1.0]),
        e_node=R.copy(), b_const=0.0, d0=0.0,
        exact=lambda tt: math.exp(-tt) * R + R * sq + R * s2,
        meta=dict(table="3.1", a=a))


# ----------------------------------------------------------------------------------------
# benchmark workloads

def parabolic_problem(r, theta, t, theta_w=0.5, name="parabolic") -> Problem:
    """u_t = Lap(u) + f with u = e^{-t} (1 - r^2)(1 + r cos theta), b = 0, g = 0;
    f = e^{-t} [4 + 8 r cos theta - (1 - r^2)(1 + r cos theta)] (Q = 1)."""
    m, n = len(r) - 2, len(theta)
    R, TH = node_coords(r, theta)
    shape = (1.0 - R ** 2) * (1.0 + R * np.cos(TH))
    S1 = 4.0 + 8.0 * R * np.cos(TH) - shape
    return Problem(
        name=name, r=r, theta=theta, t=t, theta_w=theta_w, scheme=SCHEME_CONSERVATIVE,
        d_rface=np.ones((m + 1) * n), d_tface=np.ones(m * n),
        src=[S1], bnd=[np.zeros(n)], u0=shape.copy(),
        weights=lambda tt: np.array([math.exp(-tt)]),
        b_const=0.0, d0=1.0,
        exact=lambda tt: math.exp(-tt) * shape)


def config1() -> Problem:
    """Uniform mesh m = 32, n = 64, Crank-Nicolson, dt = 0.01, 100 steps to T = 1."""
    return parabolic_problem(meshes.uniform_r(32), meshes.uniform_theta(64),
                             meshes.uniform_time(0.01, 100), 0.5, name="C1_parabolic_32x64")


def config2(m: int = 512, n: int = 1024, K: int = 1000, seed: int = SEED_BASE + 1) -> Problem:
    """Adaptive mesh: two-sided capped geometric r (ratio 1.03), angles with density
    1 + 0.5 cos(theta - theta0), dt_k = 1e-4 * 1.01^k, Crank-Nicolson."""
    rng = SplitMix64(seed)
    theta0 = 2.0 * math.pi * rng.uniform()
    p = parabolic_problem(meshes.capped_geometric(m, 1.03, True), meshes.density_theta(n, theta0),
                          meshes.geometric_time(1e-4, 1.01, K), 0.5,
                          name=f"C2_parabolic_{m}x{n}")
    p.meta.update(theta0=theta0, seed=seed)
    return p


def _fourier_modes(rng: SplitMix64, count: int = 8):
    amps, ks, phases = [], [], []
    for _ in range(count):
        amps.append(rng.uniform_in(-1.0, 1.0))
        mag = rng.uniform_in(1.0, 4.0 * math.pi)
        ang = rng.uniform_in(0.0, 2.0 * math.pi)
        ks.append((mag * math.cos(ang), mag * math.sin(ang)))
        phases.append(rng.uniform_in(0.0, 2.0 * math.pi))
    return np.array(amps), np.array(ks), np.array(phases)


class _ContinuityFields:
    """Closed-form D = A_D exp(ln2 s), phi, manufactured n*, and derivatives."""

    def __init__(self, seed: int, d_amp: float, delta: float):
        rng = SplitMix64(seed)
        a, self.ka, self.pa = _fourier_modes(rng)
        self.a = a / np.abs(a).sum()                      # sum |a_k| = 1 -> s in [-1, 1]
        self.c, self.kc, self.pc = _fourier_modes(rng)
        self.theta0 = 2.0 * math.pi * rng.uniform()
        self.d_amp = d_amp
        self.delta = delta
        self.phi_scale = 1.0

    def D(self, x, y):
        arg = np.outer(x, self.ka[:, 0]) + np.outer(y, self.ka[:, 1]) + self.pa
        s = np.cos(arg) @ self.a
        ds = -(np.sin(arg) * self.a)
        return (self.d_amp * np.exp(math.log(2.0) * s),
                ds @ self.ka[:, 0], ds @ self.ka[:, 1])

    def gradD(self, x, y):
        Dv, sx, sy = self.D(x, y)
        return Dv, math.log(2.0) * Dv * sx, math.log(2.0) * Dv * sy

    def vel(self, x, y):
        """v = -grad(phi) and div v = -Lap(phi)."""
        arg = np.outer(x, self.kc[:, 0]) + np.outer(y, self.kc[:, 1]) + self.pc
        cs = np.cos(arg) * self.c * self.phi_scale
        sn = np.sin(arg) * self.c * self.phi_scale
        vx = -(cs @ self.kc[:, 0])
        vy = -(cs @ self.kc[:, 1])
        k2 = self.kc[:, 0] ** 2 + self.kc[:, 1] ** 2
        divv = sn @ k2
        return vx, vy, divv

    def parts(self, x, y):
        """n* = e^{-t} A + B, A = 1 + x/2, B = (1 + y/2) exp(-(1 - r^2)/delta)."""
        d = self.delta
        A = 1.0 + 0.5 * x
        Ax, Ay, lapA = 0.5 * np.ones_like(x), np.zeros_like(x), np.zeros_like(x)
        E = np.exp(-(1.0 - x * x - y * y) / d)
        Ex, Ey = E * 2.0 * x / d, E * 2.0 * y / d
        lapE = E * (4.0 * (x * x + y * y) / d ** 2 + 4.0 / d)
        f = 1.0 + 0.5 * y
        B = f * E
        Bx, By = f * Ex, f * Ey + 0.5 * E
        lapB = f * lapE + Ey
        return (A, Ax, Ay, lapA), (B, Bx, By, lapB)


def _chunked(fn, *arrays, nout=1, chunk=1 << 20):
    """fn applied to consecutive slices of the (equal-length) arrays on a thread pool
    (numpy releases the GIL in its loops), outputs concatenated: one call on the whole
    arrays up to the summation order of the BLAS products inside fn, with temporaries
    bounded by the chunk size.  The chunking is fixed, so a workload's arrays are
    reproducible."""
    size = len(arrays[0])
    if size <= chunk:
        return fn(*arrays)
    starts = range(0, size, chunk)
    outs = [np.empty(size) for _ in range(nout)]

    def run(a):
        res = fn(*(x[a:a + chunk] for x in arrays))
        res = (res,) if nout == 1 else res
        for o, v in zip(outs, res):
            o[a:a + chunk] = v

    with ThreadPoolExecutor(min(32, os.cpu_count() or 1)) as ex:
        list(ex.map(run, starts))
    return outs[0] if nout == 1 else tuple(outs)


def continuity_problem(m: int, n: int, K: int, seed: int, theta_w: float = 0.5,
                       two_sided: bool = True, pe_target: float = 10.0, d_amp: float = 1.0,
                       b_const: float = 1.0, delta: float = 0.02, name: str = "continuity",
                       phi_scale: Optional[float] = None) -> Problem:
    """n_t = div(D grad n - v n) - b n + G on the unit disk (v = mu E = -grad phi),
    D = d_amp exp(ln2 sum_k a_k cos(kappa_k.x + psi_k)) (8 seeded modes, sum|a_k| = 1),
    phi = sum_k c_k sin(kappa'_k.x + psi'_k) rescaled so the largest face cell Peclet
    number |v| Delta / D equals ``pe_target`` (or by ``phi_scale`` when given, which
    keeps v fixed under mesh refinement); b = 1/tau; manufactured
    n* = e^{-t}(1 + x/2) + (1 + y/2) exp(-(1 - r^2)/delta) (sharp layer at r = 1).
    Mesh: capped geometric r (ratio 1.03), density-equidistributed angles, time
    stretch t_k = sin((k/K)^1.5 pi/2), T = 1."""
    F = _ContinuityFields(seed, d_amp, delta)
    r = meshes.capped_geometric(m, 1.03, two_sided)
    theta = meshes.density_theta(n, F.theta0)
    t = meshes.time_stretch(1.0, 1.5, K)
    # faces
    rr, rth = rface_coords(r, theta)
    tr, tth = tface_coords(r, theta)

    def face_d(rad, ang):
        return F.D(rad * np.cos(ang), rad * np.sin(ang))[0]

    def face_vr(rad, ang):       # radial component of v at radial faces
        c, s = np.cos(ang), np.sin(ang)
        vx, vy, _ = F.vel(rad * c, rad * s)
        return vx * c + vy * s

    def face_vt(rad, ang):       # angular component of v at angular faces
        c, s = np.cos(ang), np.sin(ang)
        vx, vy, _ = F.vel(rad * c, rad * s)
        return -vx * s + vy * c

    d_r = _chunked(face_d, rr, rth)
    d_t = _chunked(face_d, tr, tth)
    vr, vt = _chunked(face_vr, rr, rth), _chunked(face_vt, tr, tth)
    h = np.diff(r)                                        # h_{i+1} for face i+1/2, i = 0..m
    th_next = np.concatenate([theta[1:], [2.0 * math.pi]])
    mu_next = th_next - theta                             # mu_{j+1}
    pe_r = np.abs(vr) * np.tile(h, n) / d_r
    pe_t = np.abs(vt) * tr * np.repeat(mu_next, m) / d_t
    pe = max(pe_r.max(), pe_t.max())
    del pe_r, pe_t
    if phi_scale is not None:
        F.phi_scale = phi_scale
    else:
        F.phi_scale = pe_target / pe if pe > 0 else 0.0
    vr, vt = _chunked(face_vr, rr, rth), _chunked(face_vt, tr, tth)
    del rr, rth, tr, tth

    # sources: S1 = -A + Lc(A), S2 = Lc(B), Lc(P) = -div(D grad P) + div(v P) + b P
    def node_fields(rad, ang):
        x, y = rad * np.cos(ang), rad * np.sin(ang)
        Dn, Dx, Dy = F.gradD(x, y)
        vx, vy, divv = F.vel(x, y)
        (A, Ax, Ay, lapA), (B, Bx, By, lapB) = F.parts(x, y)

        def Lc(P, Px, Py, lapP):
            return -(Dx * Px + Dy * Py) - Dn * lapP + P * divv + vx * Px + vy * Py + b_const * P

        return -A + Lc(A, Ax, Ay, lapA), Lc(B, Bx, By, lapB), A, B

    R, TH = node_coords(r, theta)
    S1, S2, A, B = _chunked(node_fields, R, TH, nout=4)
    del R, TH
    G1 = 1.0 + 0.5 * np.cos(theta)
    G2 = 1.0 + 0.5 * np.sin(theta)
    return Problem(
        name=name, r=r, theta=theta, t=t, theta_w=theta_w, scheme=SCHEME_CONSERVATIVE,
        d_rface=d_r, d_tface=d_t, v_rface=vr, v_tface=vt,
        src=[S1, S2], bnd=[G1, G2], u0=A + B,
        weights=lambda tt: np.array([math.exp(-tt), 1.0]),
        b_const=b_const, d0=float(F.D(np.zeros(1), np.zeros(1))[0][0]),
        exact=lambda tt: math.exp(-tt) * A + B,
        meta=dict(seed=seed, pe_target=pe_target, d_amp=d_amp, theta0=F.theta0))


def config3(m: int = 2048, n: int = 4096, K: int = 2000) -> Problem:
    return continuity_problem(m, n, K, SEED_BASE + 2, theta_w=0.5, two_sided=True,
                              name=f"C3_continuity_{m}x{n}")


def config4_instance(i: int, K: int = 500, scale: float = 1.0) -> Problem:
    """Instance i of the 256-instance sweep: m log-uniform in [64, 1024], n log-uniform
    in [128, 2048], D amplitude log-uniform in [0.2, 5], Peclet log-uniform in [0.1, 20].
    ``scale`` shrinks m and n (for tests)."""
    seed = SEED_BASE + 3 * 1000 + i
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    m = int(round(math.exp(rng.uniform_in(math.log(64), math.log(1024))) * scale))
    n = int(round(math.exp(rng.uniform_in(math.log(128), math.log(2048))) * scale))
    d_amp = math.exp(rng.uniform_in(math.log(0.2), math.log(5.0)))
    pe = math.exp(rng.uniform_in(math.log(0.1), math.log(20.0)))
    return continuity_problem(max(m, 4), max(n, 8), K, seed, theta_w=0.5, two_sided=True,
                              pe_target=pe, d_amp=d_amp, name=f"C4_instance{i}")


def config5(m: int = 8192, n: int = 16384, K: int = 200) -> Problem:
    return continuity_problem(m, n, K, SEED_BASE + 4, theta_w=0.6, two_sided=False,
                              name=f"C5_continuity_{m}x{n}")


# ----------------------------------------------------------------------------------------
# electron-hole pair with a self-consistent potential

@dataclass
class CoupledPair:
    """Three problems on one mesh -- the potential, the electrons, the holes -- and the
    coupling data: signed mobilities (drift v_c = -mobility[c] grad phi), the potential's
    source slots that receive the densities, its source weights, the time levels and the
    carriers' implicit weight."""
    phi: Problem
    electrons: Problem
    holes: Problem
    mobility: tuple
    slots: tuple
    w_phi: np.ndarray
    t: np.ndarray
    theta_w: float


def coupled_pair(m: int = 24, n: int = 48, K: int = 3, seed: int = SEED_BASE + 31,
                 scale: float = 1.0, mobility=(-2.0, 1.5)) -> CoupledPair:
    """A drift-diffusion pair on a stretched adaptive mesh: the potential solves
    -div(0.5 grad phi) = scale (p - n + C) with a doping bump C = 1.5 exp(-8 r^2) - 0.3
    and phi = 0.3 scale cos(theta - theta1) on r = 1 (Gummel's iteration contracts by
    about 0.2 per sweep at scale 1 and stops converging near scale 8 at this dt); the
    carriers have face diffusivities drawn in [0.5, 2] and [0.3, 1.5], recombination rates
    1 and 0.5, smooth generation and boundary densities, smooth positive initial
    densities, dt = 0.02, theta = 0.5."""
    rng = SplitMix64(seed)
    theta0 = 2.0 * math.pi * rng.uniform()
    theta1 = 2.0 * math.pi * rng.uniform()
    r = meshes.sine_stretch(m, 0.8)
    theta = meshes.density_theta(n, theta0)
    t = meshes.uniform_time(0.02, K)
    N = m * n + 1
    R, TH = node_coords(r, theta)
    nrf, ntf = (m + 1) * n, m * n

    def draw(count, lo, hi):
        return np.array([lo + (hi - lo) * rng.uniform() for _ in range(count)])

    doping = 1.5 * np.exp(-8.0 * R ** 2) - 0.3
    phi = Problem(
        name=f"coupled_phi_{m}x{n}", r=r, theta=theta, t=t, theta_w=1.0,
        scheme=SCHEME_CONSERVATIVE, d_rface=np.full(nrf, 0.5), d_tface=np.full(ntf, 0.5),
        src=[np.zeros(N), np.zeros(N), doping],
        bnd=[np.zeros(n), np.zeros(n), 0.3 * np.cos(theta - theta1)],
        u0=np.zeros(N), weights=lambda tt: np.array([-scale, scale, scale]))

    def carrier(name, dlo, dhi, b, g_amp, bnd_val, phase):
        return Problem(
            name=f"coupled_{name}_{m}x{n}", r=r, theta=theta, t=t, theta_w=0.5,
            scheme=SCHEME_CONSERVATIVE, d_rface=draw(nrf, dlo, dhi), d_tface=draw(ntf, dlo, dhi),
            src=[0.5 + g_amp * R ** 2 * np.cos(TH - phase)],
            bnd=[bnd_val + 0.2 * np.sin(theta - phase)],
            u0=bnd_val + 0.3 * (1.0 - R ** 2) * (1.0 + 0.5 * np.cos(TH - phase)),
            weights=lambda tt: np.array([1.0]), b_const=b, b=np.full(N, b))

    electrons = carrier("electrons", 0.5, 2.0, 1.0, 0.5, 1.0, theta0)
    holes = carrier("holes", 0.3, 1.5, 0.5, 0.3, 0.8, theta1)
    return CoupledPair(phi=phi, electrons=electrons, holes=holes, mobility=tuple(mobility),
                       slots=(0, 1), w_phi=np.array([-scale, scale, scale]), t=t, theta_w=0.5)
