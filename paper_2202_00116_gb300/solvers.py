"""A first-order solver on the same objective, for comparison with DEAM.

DEAM (Sec. 2.3) minimises the I-divergence of Eq. (5) by majorise-minimise
steps that need no step size.  The solver here minimises the same F(c) with
plain gradient descent: the gradient b^ - b~ comes from ``deam_gradient`` (one
recomputation of the per-ray terms and one gather backprojection, the same
kernels a DEAM iteration runs), and the step length from the Barzilai-Borwein
rule (Barzilai and Borwein, IMA J. Numer. Anal. 8, 1988: alpha = s.s / s.y with
s the last step and y the change of gradient), kept monotone by halving alpha
until F does not increase.  Only the step's vector arithmetic (one axpy, two
dot products) runs as PyTorch operations; it is a small fraction of a step.
"""
from __future__ import annotations

import time

import numpy as np


def gradient_descent(deam, c, n_steps, alpha0=None, max_halvings=30):
    """n_steps monotone Barzilai-Borwein gradient steps on F(c), in place on
    the CUDA image c ([nz, ny, nx, 2] float32).

    Returns a dict with ``objective`` (F before each step and after the last,
    n_steps + 1 values), ``evaluations`` (gradient/objective evaluations used
    after each step, cumulative) and ``seconds`` (wall time after each step,
    cumulative, synchronised).  alpha0 defaults to a step that moves c by 1e-3
    of its norm along the first gradient."""
    import torch
    torch.cuda.synchronize(c.device)
    t0 = time.perf_counter()
    g, F = deam.gradient(c)
    g = g.clone()
    evals = 1
    out = {"objective": [F], "evaluations": [], "seconds": []}
    alpha = alpha0
    if alpha is None:
        gn = float(torch.linalg.vector_norm(g))
        alpha = 1e-3 * float(torch.linalg.vector_norm(c)) / max(gn, 1e-300)
    c_new = torch.empty_like(c)
    for _ in range(n_steps):
        for _h in range(max_halvings + 1):
            torch.add(c, g, alpha=-alpha, out=c_new)
            g_new, F_new = deam.gradient(c_new)
            evals += 1
            if F_new <= F:
                break
            alpha *= 0.5
        else:
            break  # no decrease at any tried step: stationary to FP32 resolution
        s = c_new - c
        yv = g_new - g
        sy = float(torch.dot(s.reshape(-1).double(), yv.reshape(-1).double()))
        ss = float(torch.dot(s.reshape(-1).double(), s.reshape(-1).double()))
        c.copy_(c_new)
        g.copy_(g_new)
        F = F_new
        alpha = ss / sy if sy > 0 else 2.0 * alpha
        torch.cuda.synchronize(c.device)
        out["objective"].append(F)
        out["evaluations"].append(evals)
        out["seconds"].append(time.perf_counter() - t0)
    out["objective"] = np.asarray(out["objective"])
    return out
