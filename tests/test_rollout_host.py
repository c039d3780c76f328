"""Host logic of the checkpointed rollout adjoint (adjoint.RolloutFunction) with stand-in
library calls, no device.  The stand-in step is the nonlinear map W <- W + dt sin(W), so its
adjoint needs the exact pre-step state: the rollout must keep a checkpoint every `every` steps,
recompute each segment's states from it (the last segment ragged) and apply the step adjoints
in reverse order.  The gradient is checked against the chain rule written out."""
import types

import pytest
import torch

from paper_2410_05489_gb300 import adjoint as AD


class _Fakes:
    def __init__(self):
        self.steps = 0
        self.adjoint_steps = 0

    def step(self, c, W, sx, sy, dt):
        W += dt * torch.sin(W)
        self.steps += 1

    def run(self, c, W, sx, sy, dt, n):
        for _ in range(n):
            self.step(c, W, sx, sy, dt)

    def step_adjoint(self, c, W, sx, sy, dt, Wbar, sxb, syb):
        Wbar *= 1.0 + dt * torch.cos(W)  # the transpose of the step's Jacobian at its input
        self.adjoint_steps += 1


@pytest.mark.parametrize("nsteps, every", [(23, 10), (20, 10), (7, 1), (5, 9)])
def test_rollout_adjoint_bookkeeping(monkeypatch, nsteps, every):
    f = _Fakes()
    A = AD.A
    monkeypatch.setattr(A, "ase_df_prime_sigma", lambda c, W, sx, sy: sx.zero_())
    monkeypatch.setattr(A, "ase_df_get_repair_stats", lambda c: (0, 0, 0))
    monkeypatch.setattr(A, "ase_df_run", f.run)
    monkeypatch.setattr(A, "ase_df_step", f.step)
    monkeypatch.setattr(A, "ase_df_step_adjoint", f.step_adjoint)
    monkeypatch.setattr(A, "ase_df_residual_adjoint", lambda *a: None)
    pb = types.SimpleNamespace(sx_shape=(2, 3), sy_shape=(3, 2))
    solver = types.SimpleNamespace(pb=pb, ctx=None, _sy=lambda sy: sy)

    dt = 0.3
    W0 = torch.linspace(-2.0, 2.0, 7, dtype=torch.float64)
    gW = torch.linspace(0.5, 1.5, 7, dtype=torch.float64)
    W0r = W0.clone().requires_grad_(True)
    WT = AD.rollout(solver, W0r, nsteps, dt, every)
    assert f.steps == nsteps
    (grad,) = torch.autograd.grad(WT, W0r, gW)

    # the chain rule, written out
    W, states = W0.clone(), []
    for _ in range(nsteps):
        states.append(W.clone())
        W = W + dt * torch.sin(W)
    assert torch.equal(WT.detach(), W)
    g = gW.clone()
    for Wk in reversed(states):
        g = g * (1.0 + dt * torch.cos(Wk))
    assert torch.allclose(grad, g, rtol=0, atol=1e-14)
    assert f.adjoint_steps == nsteps
    segments = -(-nsteps // every)
    assert f.steps == nsteps + (nsteps - segments)  # the backward recomputes all but each segment's last step
