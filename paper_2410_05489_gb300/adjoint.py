"""torch.autograd wrappers of the hand-written adjoint kernels (argument marshalling and
checkpoint bookkeeping only; every arithmetic step runs in the library's kernels).

residual(solver, W, sx, sy) -> (L, sx_out, sy_out)
    One residual evaluation (Sec. 2.1 Eq. 2.3 with the reconstruction of Sec. 3 and the
    flux of Sec. 2.3); its backward is ase_df_residual_adjoint.

rollout(solver, W0, nsteps, dt, every=10) -> W_final
    sigma^0 = prime(W0) (the sigma of a residual with sigma_in = 0), then nsteps SSP-RK3
    steps of fixed dt (Sec. 2.3), each stage consuming the sigma of the stage before.
    The forward keeps (W, sigma) every `every` steps.  The backward walks the segments
    in reverse: it recomputes the segment's step states from its checkpoint
    (ase_df_step; the forward is deterministic, so they are bit-identical), runs
    ase_df_step_adjoint back through them, and ends with the adjoint of the priming
    residual.  Memory: one state per checkpoint plus one segment of states.

The positivity repair of the stage updates is not differentiated: a rollout whose
forward needed it raises RuntimeError.
"""
from __future__ import annotations

import torch

from . import ase_df as A


def _contig(t):
    return None if t is None else t.contiguous()


class ResidualFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W, sx, sy, solver):
        L, sxo, syo = solver.residual(W, sx, sy)
        ctx.save_for_backward(W, sx, sy)
        ctx.solver = solver
        return L, sxo, syo

    @staticmethod
    def backward(ctx, gL, gsx, gsy):
        W, sx, sy = ctx.saved_tensors
        s = ctx.solver
        Wbar = torch.zeros_like(W)
        sxb = torch.zeros_like(sx)
        syb = torch.zeros_like(sy)
        A.ase_df_residual_adjoint(s.ctx, W, sx, s._sy(sy), _contig(gL), _contig(gsx), s._sy(_contig(gsy)), Wbar, sxb,
                                  s._sy(syb))
        return Wbar, sxb, syb, None


def residual(solver, W, sx, sy):
    return ResidualFunction.apply(W, sx, sy, solver)


class RolloutFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W0, solver, nsteps: int, dt: float, every: int):
        if not (dt > 0.0):
            raise ValueError("the rollout adjoint needs a fixed dt > 0")
        if every < 1:
            raise ValueError("every must be >= 1")
        pb = solver.pb
        c = solver.ctx
        W = W0.detach().clone().contiguous()
        sx = torch.zeros(pb.sx_shape, dtype=torch.float64, device=W.device)
        sy = torch.zeros(pb.sy_shape, dtype=torch.float64, device=W.device)
        A.ase_df_prime_sigma(c, W, sx, solver._sy(sy))
        _, marked0, _ = A.ase_df_get_repair_stats(c)
        ckpts = []
        k = 0
        while k < nsteps:
            ckpts.append((k, W.clone(), sx.clone(), sy.clone()))
            n = min(every, nsteps - k)
            A.ase_df_run(c, W, sx, solver._sy(sy), dt, n)
            k += n
        _, marked1, _ = A.ase_df_get_repair_stats(c)
        if marked1 != marked0:
            raise RuntimeError("the rollout needed the positivity repair, which the adjoint does not differentiate")
        ctx.save_for_backward(W0)
        ctx.ckpts = ckpts
        ctx.solver = solver
        ctx.nsteps, ctx.dt, ctx.every = nsteps, dt, every
        return W

    @staticmethod
    def backward(ctx, gW):
        (W0,) = ctx.saved_tensors
        s = ctx.solver
        c = s.ctx
        pb = s.pb
        Wbar = gW.detach().to(torch.float64).contiguous().clone()
        sxb = torch.zeros(pb.sx_shape, dtype=torch.float64, device=Wbar.device)
        syb = torch.zeros(pb.sy_shape, dtype=torch.float64, device=Wbar.device)
        for k0, Wc, sxc, syc in reversed(ctx.ckpts):
            k1 = min(k0 + ctx.every, ctx.nsteps)
            W, sx, sy = Wc.clone(), sxc.clone(), syc.clone()
            states = []
            for k in range(k0, k1):
                states.append((W.clone(), sx.clone(), sy.clone()))
                if k < k1 - 1:
                    A.ase_df_step(c, W, sx, s._sy(sy), ctx.dt)
            for Ws, sxs, sys_ in reversed(states):
                A.ase_df_step_adjoint(c, Ws, sxs, s._sy(sys_), ctx.dt, Wbar, sxb, s._sy(syb))
        # sigma^0 = sigma_out(W0, sigma_in = 0)
        zx = torch.zeros_like(sxb)
        zy = torch.zeros_like(syb)
        A.ase_df_residual_adjoint(c, W0.detach().contiguous(), zx, s._sy(zy), None, sxb, s._sy(syb), Wbar, None, None)
        return Wbar, None, None, None, None


def rollout(solver, W0, nsteps: int, dt: float, every: int = 10):
    return RolloutFunction.apply(W0, solver, int(nsteps), float(dt), int(every))
