"""Training of the learned preconditioner correction on solver-generated data.

The corrected preconditioner T(r) = T0 r + K_A F3^H g(F3 K_A^H r / |k|^2) / |k|^2
(pcx_cnn_precond; T0 the curl-sandwich approximate inverse, g the gated
convolution net acting next to eps on the real-space field) is trained on
pairs (r, e = Op^{-1} r): r are residual columns that the mixed
precision eigensolver itself produces (pcx_solve's residual dump), e comes
from the preconditioned conjugate gradient solve pcx_cg_solve, and the loss
on the part the correction can reach, sum_v ||g(U_v) - F3 K_A^H (e_v - T0 r_v)||^2
/ ||K_A^H e_v||^2, is minimised by Adam.  Every device step
runs in libpcx kernels through the C ABI; this module only sequences the
calls and holds the tensors.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import pcx


@dataclass
class Sample:
    """Training pairs of one structure: real-space inputs U, targets T and
    per-vector loss weights w = 1 / (count ||e_v||^2)."""
    ctx: object
    k: np.ndarray
    U: object
    T: object
    w: np.ndarray


FORM = pcx.PCX_CNN_HERMITIAN | pcx.PCX_CNN_BF16   # the correction's form used for training and solves


def collect(ctx, k, n_pairs=16, nev=12, block=16, dump_every=3, cg_tol=1e-3, cg_maxit=300, seed=0, form=FORM):
    """Residuals from an FP32-phase solve at k, their PCG targets and the
    training pairs; the context is set to the correction's form (see
    pcx_set_cnn_form).  Returns a Sample, or None if no residual was dumped."""
    import torch
    pcx.pcx_set_cnn_form(ctx, form)
    n = ctx.n
    R = torch.empty((n_pairs, 3, n, n, n), dtype=torch.complex64, device="cuda")
    stats = pcx.pcx_solve_stats()
    pcx.pcx_solve(ctx, [k], nev, 1e-4, block=block, precision=pcx.PCX_FP32, stats=stats, raise_on_noconv=False,
                  dump_R=R, dump_every=dump_every, seed=seed)
    m = stats.dumped
    if m == 0:
        return None
    R = R[:m].contiguous()
    E = torch.empty_like(R)
    pcx.pcx_cg_solve(ctx, k, R, E, tol=cg_tol, maxit=cg_maxit)
    U = torch.empty_like(R)
    T = torch.empty_like(R)
    en2 = pcx.pcx_cnn_pairs(ctx, k, R, E, U, T)
    return Sample(ctx, np.asarray(k, dtype=np.float64), U, T, 1.0 / (m * en2))


def train(samples, steps=200, lr=3e-3, seed=1, params=None):
    """Adam on the samples in turn; returns (params, losses)."""
    import torch
    P = params
    if P is None:
        P = torch.empty(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
        pcx.pcx_cnn_init(seed, P)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.zeros_like(P)
    losses = []
    for step in range(1, steps + 1):
        s = samples[(step - 1) % len(samples)]
        losses.append(pcx.pcx_cnn_grad(s.ctx, P, s.U, s.T, s.w, grad))
        pcx.pcx_cnn_adam(P, grad, m, v, step, lr)
    return P, losses


def relative_error(samples, params):
    """Mean over samples of sum_v w_v ||T(r_v) - e_v||^2 with the given
    parameters (the training loss without an update)."""
    import torch
    grad = torch.zeros(pcx.PCX_CNN_NPARAMS, dtype=torch.float32, device="cuda")
    return float(np.mean([pcx.pcx_cnn_grad(s.ctx, params, s.U, s.T, s.w, grad) for s in samples]))
