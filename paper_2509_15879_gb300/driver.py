"""Convenience layer over the C ABI: loads a problem description (mesh, coefficient
arrays, separable sources, initial state, time levels) into a context and advances it.

A problem is any object with the attributes r, theta, t, theta_w, scheme, d_rface,
d_tface, v_rface, v_tface, e_node, b, b_const, d0, src, bnd, u0 and weight_table()
(face and node layouts of include/polar.h).  This module only moves arrays.
"""
import numpy as np

from . import _native as P


def _const(a):
    """Returns the common value if every entry of a equals it, else None."""
    if a is None:
        return None
    a = np.asarray(a)
    return float(a.flat[0]) if a.size and np.all(a == a.flat[0]) else None


def default_allocator():
    """PyTorch's caching allocator when torch sees a GPU (the library then takes its
    device memory from torch's pool), else None (the library's own cudaMalloc)."""
    try:
        import torch
        return "torch" if torch.cuda.is_available() else None
    except ImportError:
        return None


def create(problem, precision=P.POLAR_FP64, stream=None, compact_d=True, allocator="auto"):
    if allocator == "auto":
        allocator = default_allocator()
    ctx = P.polar_mesh_create(problem.r, problem.theta, problem.scheme, precision, stream,
                              allocator)
    load_coeffs(ctx, problem, compact_d=compact_d)
    P.polar_set_state(ctx, problem.u0, problem.t[0])
    return ctx


def load_coeffs(ctx, problem, compact_d=True):
    d_r, d_t, d_const = problem.d_rface, problem.d_tface, 1.0
    if compact_d:
        cr, ct = _const(d_r), _const(d_t)
        if cr is not None and cr == ct:
            d_r, d_t, d_const = None, None, cr
    P.polar_set_coeffs(ctx, d_rface=d_r, d_tface=d_t, v_rface=problem.v_rface,
                       v_tface=problem.v_tface, e_node=problem.e_node, b=problem.b,
                       d_const=d_const, b_const=problem.b_const, d0=problem.d0,
                       src=list(problem.src), bnd=list(problem.bnd))


def advance(ctx, problem, k0=0, k1=None, opts=None):
    """Advances over the time levels t[k0..k1] of the problem."""
    t = np.asarray(problem.t, dtype=np.float64)
    k1 = len(t) - 1 if k1 is None else k1
    w = problem.weight_table()[k0:k1 + 1]
    stats, _ = P.polar_advance(ctx, t[k0:k1 + 1], problem.theta_w, w, opts)
    return stats


def batch_advance(batch, problems, k0=0, k1=None, opts=None, check=True):
    """Advances every instance of a polar_batch over time levels t[k0..k1] of its problem."""
    ts, ws = [], []
    for p in problems:
        t = np.asarray(p.t, dtype=np.float64)
        kk = len(t) - 1 if k1 is None else k1
        ts.append(t[k0:kk + 1])
        ws.append(p.weight_table()[k0:kk + 1])
    return P.polar_batch_advance(batch, ts, [p.theta_w for p in problems], ws, opts, check)


def sweep(problems, precision=P.POLAR_FP64, stream=None, opts=None):
    """Advances every problem over its whole schedule together: one polar_batch whose
    CUDA graph holds a step of every instance per launch (parameter sweeps, mesh-tuning
    studies).  The problems must have the same number of steps.  Returns the final
    states and the per-instance step statistics."""
    K = len(problems[0].t) - 1
    if any(len(p.t) - 1 != K for p in problems):
        raise ValueError("every problem of a sweep needs the same number of steps")
    ctxs = [create(p, precision, stream) for p in problems]
    batch = P.polar_batch_create(ctxs, stream)
    stats, _ = batch_advance(batch, problems, 0, K, opts)
    states = [P.polar_get_state(c)[0] for c in ctxs]
    P.polar_batch_destroy(batch)
    return states, stats
