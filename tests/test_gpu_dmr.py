"""The double Mach reflection (Sec. 4.3 Example 4, reading G32) on the GPU: the split bottom
and the moving-shock top in the face kernels of both flux solvers and in the positivity
repair, each stage at its own time, against the CPU oracle.

Tolerances as test_gpu_parity.py (residual 1e-12 with the flux floor; sigma 1e-12 (1 + |s|) +
1e-13 s^2; steps 1e-9); the full run to t = 0.2 is compared in L1 (1e-6 of the mean density),
the paper shows this problem as a figure only."""
import numpy as np
import pytest

from parity_report import check
from paper_2410_05489_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_05489_gb300 import build

    build.build()
    from paper_2410_05489_gb300 import ase_df

    return ase_df


def dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def comp_err(gpu, cpu, floor):
    return max(np.abs(gpu[c] - cpu[c]).max() / max(np.abs(cpu[c]).max(), floor[c]) for c in range(cpu.shape[0]))


def floor_of(pb, Fx, Fy):
    inv = 1.0 / pb.dx + 1.0 / pb.dy
    return [1e-2 * inv * max(np.abs(Fx[c]).max(), np.abs(Fy[c]).max()) for c in range(pb.ncomp)]


def sigma_ok(g, c):
    return np.all(np.abs(g - c) <= 1e-12 * (1 + np.abs(c)) + 1e-13 * c * c)


def perturbed(pb, W, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(W * (1.0 + 0.02 * rng.uniform(-1.0, 1.0, W.shape)))


@pytest.mark.parametrize("r", [5, 9])
def test_residual_parity_at_several_times(A, oracle, r):
    import torch

    pb, W0 = P.double_mach_reflection(64, r)
    W = perturbed(pb, W0, r)
    rng = np.random.default_rng(7)
    sx, sy = rng.uniform(0.0, 0.6, pb.sx_shape), rng.uniform(0.0, 0.6, pb.sy_shape)
    s = A.Solver(pb)
    try:
        for t in (0.0, 0.0123, 0.05, 0.2):
            L, sxo, syo, Fx, Fy, _ = oracle.residual(pb, W, sx, sy, t=t)
            s.set_time(t)
            Lg, sxg, syg = s.residual(dev(W), dev(sx), dev(sy))
            torch.cuda.synchronize()
            check("L", comp_err(Lg.cpu().numpy(), L, floor_of(pb, Fx, Fy)), 1e-12)
            assert sigma_ok(sxg.cpu().numpy(), sxo) and sigma_ok(syg.cpu().numpy(), syo)
            # the gas-kinetic face kernel sees the same boundaries
            dt = 0.5 * oracle.cfl_dt(pb, W)
            Lk, Ltk, *_ = oracle.gks_residual(pb, W, sx, sy, dt, t=t)
            Lkg, Ltkg, _, _ = s.gks_residual(dt, dev(W), dev(sx), dev(sy))
            fl = floor_of(pb, Fx, Fy)
            check("L (GKS)", comp_err(Lkg.cpu().numpy(), Lk, fl), 1e-11)
            check("L_t (GKS)", comp_err(Ltkg.cpu().numpy(), Ltk, [f / dt for f in fl]), 1e-11)
    finally:
        s.close()


def test_steps_see_the_boundary_at_their_stage_times(A, oracle):
    """Fixed-dt steps from a time at which the shock passes a ghost centre inside the step:
    both flux solvers against the oracle, whose stage times are pinned separately."""
    import torch

    pb, W0 = P.double_mach_reflection(64, 5)
    dt = 0.5 * oracle.cfl_dt(pb, W0)
    i = 40
    t0 = (pb.x0 + (i + 0.5) * pb.dx - pb.shock_x0) / pb.shock_speed - 0.75 * dt
    sx, sy = oracle.prime_sigma(pb, W0)
    for gks in (False, True):
        Wc, sxc, syc, t = W0, sx, sy, t0
        s = A.Solver(pb)
        try:
            s.W.copy_(dev(W0))
            s.sx.copy_(dev(sx))
            s.sy.copy_(dev(sy))
            s.set_time(t0)
            for _ in range(6):
                if gks:
                    Wc, sxc, syc, h = oracle.gks_step(pb, Wc, sxc, syc, dt, t=t)
                    s.gks_step(dt)
                else:
                    Wc, sxc, syc, h = oracle.step(pb, Wc, sxc, syc, dt, t=t)
                    s.step(dt)
                assert h > 0
                t += dt
            torch.cuda.synchronize()
            flags, _, tg = s.status()
            assert flags & 1 == 0 and abs(tg - t) <= 1e-14 * t
            err = np.abs(s.W.cpu().numpy() - Wc).max() / np.abs(Wc).max()
            check("W after steps", err, 1e-11, gks)
        finally:
            s.close()


def run_gpu(A, pb, W0, t_end, gks=False):
    import torch

    s = A.Solver(pb, W0, t_end=t_end)
    try:
        for _ in range(100000):
            for _ in range(25):
                s.gks_step() if gks else s.step()
            flags, _, t = s.status()
            if t >= t_end * (1 - 1e-12) or flags & 1:
                break
        torch.cuda.synchronize()
        return s.W.cpu().numpy(), flags, t
    finally:
        s.close()


def test_lax_friedrichs_run_to_t02_matches_the_oracle(A, oracle):
    pb, W0 = P.double_mach_reflection(96, 5)
    W, flags, t = run_gpu(A, pb, W0, 0.2)
    assert abs(t - 0.2) < 1e-12 and flags & 1 == 0
    rho = W[0]
    assert rho.min() > 1.0 and 8.0 < rho.max() < 30.0  # pre-shock 1.4; Mach stem and jet above 8
    Wc, *_ = oracle.run(pb, W0, t_end=0.2)
    check("rho L1 end state", np.abs(rho - Wc[0]).mean() / np.abs(Wc[0]).mean(), 1e-6)


def test_gas_kinetic_run_matches_the_oracle(A, oracle):
    pb, W0 = P.double_mach_reflection(64, 5)
    W, flags, t = run_gpu(A, pb, W0, 0.03, gks=True)
    assert abs(t - 0.03) < 1e-12 and flags & 1 == 0
    Wc, *_ = oracle.gks_run(pb, W0, t_end=0.03)
    check("rho L1 end state", np.abs(W[0] - Wc[0]).mean() / np.abs(Wc[0]).mean(), 1e-6)


@pytest.mark.parametrize("gks", [False, True])
def test_paper_resolution_run_stays_physical(A, gks):
    """960 x 240 at order 9 to t = 0.2 (the paper's figure): no non-physical cell average,
    density within the physical range of the problem, and the incident shock in the top rows
    at the exact position x = 1/6 + (y + 20 t) / sqrt(3) within two cells."""
    pb, W0 = P.double_mach_reflection(960, 9)
    W, flags, t = run_gpu(A, pb, W0, 0.2, gks=gks)
    assert abs(t - 0.2) < 1e-12 and flags & 1 == 0
    rho = W[0]
    assert rho.min() > 1.3 and rho.max() < 30.0
    xs = pb.x0 + (np.arange(pb.nx) + 0.5) * pb.dx
    for j in (pb.ny - 1, pb.ny - 5):
        y = pb.y0 + (j + 0.5) * pb.dy
        k = int(np.argmax((rho[j] < 4.7) & (xs > 2.0)))
        assert abs(xs[k] - (1.0 / 6.0 + (y + 20.0 * t) / np.sqrt(3.0))) <= 2 * pb.dx
