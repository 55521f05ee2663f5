"""torch.autograd.Function over rw_solve / rw_solve_adjoint.

Forward: x = rw_solve(g, seeds; beta) on a batch of volumes (g: normalised
intensities, stored in FP32 so that gradients are defined).  Only x is saved
(no CG iterates).  Backward: one adjoint PCG solve on the same symmetric
system, then the per-edge gradient kernel gives dl/dg and dl/dbeta.
"""
from __future__ import annotations

import torch

from . import Opts, RW_STORE_F32, rw_solve, rw_solve_adjoint


class RWSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, beta, code, value, opts_kw=None):
        kw = dict(opts_kw or {})
        kw["beta"] = float(beta)
        opts = Opts(**kw)
        x, _ = rw_solve(g.detach(), code, value, opts, storage=RW_STORE_F32)
        ctx.save_for_backward(g.detach(), code, x)
        ctx.opts_kw = kw
        return x

    @staticmethod
    def backward(ctx, dx):
        g, code, x = ctx.saved_tensors
        opts = Opts(**ctx.opts_kw)
        dg, dbeta, _ = rw_solve_adjoint(g, code, x, dx.contiguous(), opts, storage=RW_STORE_F32)
        db = torch.tensor(float(dbeta.sum()), dtype=torch.float32, device=g.device)
        return dg, db, None, None, None
