"""A first-order solver on the same objective, for comparison with DEAM.

DEAM (Sec. 2.3) minimises the I-divergence of Eq. (5) by majorise-minimise
steps that need no step size.  The solver here minimises the same F(c) with
plain gradient descent: the gradient b^ - b~ comes from ``deam_gradient`` (one
recomputation of the per-ray terms and one gather backprojection, the same
kernels a DEAM iteration runs), and the step length from the Barzilai-Borwein
rule (Barzilai and Borwein, IMA J. Numer. Anal. 8, 1988: alpha = s.s / s.y with
s the last step and y the change of gradient), kept monotone by halving alpha
until F does not increase.  With ``precondition=True`` the step direction is
the gradient scaled per voxel by 1/(Z b~_i(x)), the diagonal preconditioner of
which the DEAM c-step -(1/Z) log1p(delta / b~) is the exact-surrogate version
(the two agree to first order at alpha = 1); gradients and b~ then come from
``deam_backprojected_sums`` at the same cost, and the BB rule is taken in the
preconditioner's metric (alpha = s.D s / s.y with D = Z b~).  Only the step's
vector arithmetic (axpy, dot products) runs as PyTorch operations; it is a
small fraction of a step.
"""
from __future__ import annotations

import time

import numpy as np


def gradient_descent(deam, c, n_steps, alpha0=None, max_halvings=30, precondition=False):
    """n_steps monotone Barzilai-Borwein gradient steps on F(c), in place on
    the CUDA image c ([nz, ny, nx, 2] float32).

    Returns a dict with ``objective`` (F before each step and after the last,
    up to n_steps + 1 values), ``evaluations`` (gradient evaluations used after
    each step, cumulative) and ``seconds`` (wall time after each step,
    cumulative, synchronised).  alpha0 defaults to 1 when preconditioned (the
    DEAM-sized step) and otherwise to a step that moves c by 1e-3 of its norm
    along the first gradient.  Stops early when no halving decreases F."""
    import torch

    def evaluate(x):
        if not precondition:
            g, F = deam.gradient(x)
            return g, None, F
        sums, F, Z = deam.backprojected_sums(x)
        bt = sums[..., :2]
        D = Z * bt                                   # inverse preconditioner
        P = torch.where(bt > 0, 1.0 / torch.where(bt > 0, D, torch.ones_like(D)), torch.zeros_like(D))
        return sums[..., 2:].contiguous(), (P, D), F

    torch.cuda.synchronize(c.device)
    t0 = time.perf_counter()
    g, pre, F = evaluate(c)
    evals = 1
    out = {"objective": [F], "evaluations": [], "seconds": []}
    alpha = alpha0
    if alpha is None:
        if precondition:
            alpha = 1.0
        else:
            gn = float(torch.linalg.vector_norm(g))
            alpha = 1e-3 * float(torch.linalg.vector_norm(c)) / max(gn, 1e-300)
    c_new = torch.empty_like(c)
    for _ in range(n_steps):
        d = g if pre is None else pre[0] * g
        for _h in range(max_halvings + 1):
            torch.add(c, d, alpha=-alpha, out=c_new)
            g_new, pre_new, F_new = evaluate(c_new)
            evals += 1
            if F_new <= F:
                break
            alpha *= 0.5
        else:
            break  # no decrease at any tried step: stationary to FP32 resolution
        s = (c_new - c).reshape(-1).double()
        yv = (g_new - g).reshape(-1).double()
        sy = float(torch.dot(s, yv))
        sDs = float(torch.dot(s, s if pre is None else pre[1].reshape(-1).double() * s))
        c.copy_(c_new)
        g, pre, F = g_new, pre_new, F_new
        alpha = sDs / sy if sy > 0 else 2.0 * alpha
        torch.cuda.synchronize(c.device)
        out["objective"].append(F)
        out["evaluations"].append(evals)
        out["seconds"].append(time.perf_counter() - t0)
    out["objective"] = np.asarray(out["objective"])
    return out
