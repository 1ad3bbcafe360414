"""Mesh and time-schedule generators (inputs to the solver, not part of it).

The library takes the radial nodes r[0..m+1], the angles theta[0..n-1] and the time
levels t[0..K] as plain arrays; these functions produce them.

* ``sine_stretch``      — radial stretch v(s) = sin(s^p pi/2), Eq. (2.4).
* ``zhang_stretch``     — comparison stretch phi(s) = 1 - (1-s)^(p~+1), Eq. (2.13).
* ``angular_stretch``   — theta_j = 2 pi sin(((j mu~)/(2 pi))^q pi/2), Section 3.1.
* ``time_stretch``      — t_k = T sin((k/K)^l pi/2), Section 3.1.
* ``capped_geometric``  — spacing growing by a fixed ratio away from r=0 and/or r=1,
                          with the growth capped (the paper gives a ratio but no cap).
* ``density_theta``     — angles equidistributed for node density 1 + 0.5 cos(theta - theta0).
"""
import math

import numpy as np


def uniform_r(m: int) -> np.ndarray:
    """r_i = i/(m+1), i = 0..m+1 (Section 2.1 with p = 1 and no stretch)."""
    r = np.arange(m + 2, dtype=np.float64) / (m + 1)
    r[-1] = 1.0
    return r


def sine_stretch(m: int, p: float) -> np.ndarray:
    """r_i = sin((i h)^p pi/2), h = 1/(m+1), Eq. (2.4)."""
    s = np.arange(m + 2, dtype=np.float64) / (m + 1)
    r = np.sin(s ** p * (math.pi / 2))
    r[0], r[-1] = 0.0, 1.0
    return r


def zhang_stretch(m: int, ptilde: float) -> np.ndarray:
    """r_i = 1 - (1 - i h)^(p~+1), Eq. (2.13)."""
    s = np.arange(m + 2, dtype=np.float64) / (m + 1)
    r = 1.0 - (1.0 - s) ** (ptilde + 1.0)
    r[0], r[-1] = 0.0, 1.0
    return r


def capped_geometric(m: int, ratio: float = 1.03, two_sided: bool = True) -> np.ndarray:
    """Radial nodes whose spacing grows geometrically away from the graded end(s).

    There are M = m+1 intervals k = 0..M-1 with widths c * ratio^e_k, where
    e_k = min(k, M-1-k, G) (two-sided: finest at r=0 and r=1) or min(M-1-k, G)
    (one-sided: finest at r=1), G = min(floor(M/4), 128) caps the growth, and c
    normalises the widths to sum to one.
    """
    M = m + 1
    G = min(M // 4, 128)
    k = np.arange(M)
    if two_sided:
        e = np.minimum(np.minimum(k, M - 1 - k), G)
    else:
        e = np.minimum(M - 1 - k, G)
    w = ratio ** e.astype(np.float64)
    w /= w.sum()
    r = np.concatenate([[0.0], np.cumsum(w)])
    r[-1] = 1.0
    return r


def uniform_theta(n: int) -> np.ndarray:
    """theta_j = 2 pi j / n, j = 0..n-1 (Section 2.1)."""
    return 2.0 * math.pi * np.arange(n, dtype=np.float64) / n


def angular_stretch(n: int, q: float) -> np.ndarray:
    """theta_j = v(j mu~) with v(iota) = 2 pi sin((iota/2pi)^q pi/2), mu~ = 2pi/n
    (Section 3.1); j = 0..n-1 (theta_n = 2 pi is the periodic image of theta_0)."""
    s = np.arange(n, dtype=np.float64) / n
    th = 2.0 * math.pi * np.sin(s ** q * (math.pi / 2))
    th[0] = 0.0
    return th


def density_theta(n: int, theta0: float) -> np.ndarray:
    """Angles with node density proportional to 1 + 0.5 cos(theta - theta0).

    theta_j solves F(theta_j) = 2 pi j / n where
    F(theta) = theta + 0.5 (sin(theta - theta0) + sin(theta0)) is the normalised
    cumulative density (F(0) = 0, F(2 pi) = 2 pi, F' >= 1/2).  Newton's method
    inside a bisection bracket, to full double precision.
    """
    th = np.empty(n, dtype=np.float64)
    th[0] = 0.0
    for j in range(1, n):
        target = 2.0 * math.pi * j / n
        lo, hi = 0.0, 2.0 * math.pi
        x = target
        for _ in range(200):
            fx = x + 0.5 * (math.sin(x - theta0) + math.sin(theta0)) - target
            if fx > 0:
                hi = x
            else:
                lo = x
            dfx = 1.0 + 0.5 * math.cos(x - theta0)
            xn = x - fx / dfx
            if not (lo < xn < hi):
                xn = 0.5 * (lo + hi)
            if abs(xn - x) <= 1e-16 * max(1.0, abs(x)):
                x = xn
                break
            x = xn
        th[j] = x
    return th


def time_stretch(T: float, l: float, K: int) -> np.ndarray:
    """t_k = V(k dt~), V(t) = T sin((t/T)^l pi/2), dt~ = T/K (Section 3.1)."""
    s = np.arange(K + 1, dtype=np.float64) / K
    t = T * np.sin(s ** l * (math.pi / 2))
    t[0], t[-1] = 0.0, T
    return t


def uniform_time(dt: float, K: int) -> np.ndarray:
    """t_k = k dt (Section 2.1)."""
    return dt * np.arange(K + 1, dtype=np.float64)


def geometric_time(dt0: float, growth: float, K: int) -> np.ndarray:
    """t_0 = 0, t_{k+1} = t_k + dt0 growth^k."""
    t = np.zeros(K + 1, dtype=np.float64)
    dt = dt0
    for k in range(K):
        t[k + 1] = t[k] + dt
        dt *= growth
    return t
