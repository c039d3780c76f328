"""GPU adjoint: the hand-written residual and step adjoints (through the C ABI and the
torch.autograd wrappers) against the oracle's reverse mode and central differences.

Tolerances:
  * residual adjoint vs the oracle tape: per component c of Wbar,
    max|gpu - cpu| <= 1e-10 max|cpu_c|; sigma_in adjoints likewise against their max.
    Both sides differentiate the same piecewise function on the same branches (the
    branch choice comes from the same sigma_in); what remains is rounding of sums with
    cancellation (the flux difference, the WENO weight derivatives).  Scales have the
    floor 1e-4 max|Lbar| (1/dx + 1/dy): where the exact adjoint vanishes (a one-cell
    periodic grid, whose residual is identically zero) both sides give rounding noise.
  * rollout adjoint vs the oracle tape (few steps, small grids): 1e-9 of the max.
  * rollout adjoint vs central differences of J = sum rho_final^2 with h = 1e-6 on unit
    directions: |fd - ad| <= 1e-6 |ad| + 1e-9 |grad J|; the difference of J is formed
    as sum (rho_+ - rho_-)(rho_+ + rho_-) so that it does not cancel.
"""
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


def rel_err(gpu, cpu, floor=0.0):
    errs = []
    for c in range(cpu.shape[0]):
        scale = max(np.abs(cpu[c]).max(), floor)
        d = np.abs(gpu[c] - cpu[c]).max()
        errs.append(d / scale if scale > 0 else d)
    return max(errs)


def residual_case(name):
    if name == "2d_r9_periodic_37x45":
        pb, _ = P.isentropic_vortex(37, 9, ny=45)
        W = P.smooth_random(pb, 3)
        return pb, W, P.random_sigma(pb, 5, pb.sigma_thres / 2)
    if name == "2d_r7_outflow_40x33":
        pb = P.Problem(ndim=2, nx=40, ny=33, order=7)
        return pb, P.smooth_random(pb, 4), P.random_sigma(pb, 6, pb.sigma_thres / 2)
    if name == "2d_r5_mixed_bc_35x20":
        pb = P.Problem(ndim=2, nx=35, ny=20, order=5, bc=("periodic", "periodic", "outflow", "outflow"))
        return pb, P.smooth_random(pb, 7), P.random_sigma(pb, 8, pb.sigma_thres / 2)
    if name == "2d_r3_periodic_19x17":
        pb = P.Problem(ndim=2, nx=19, ny=17, order=3, bc=("periodic",) * 4)
        return pb, P.smooth_random(pb, 11), P.random_sigma(pb, 12, pb.sigma_thres)
    if name == "1d_r9_noise_300":
        pb = P.Problem(ndim=1, nx=300, order=9)
        return pb, P.white_noise(pb, 9), P.random_sigma(pb, 10, pb.sigma_thres / 2)
    if name == "1d_r5_noise_periodic_1":
        pb = P.Problem(ndim=1, nx=1, order=5, bc=("periodic", "periodic", "outflow", "outflow"))
        return pb, P.white_noise(pb, 13), P.random_sigma(pb, 14, pb.sigma_thres / 2)
    if name == "2d_r9_periodic_3x2":
        pb = P.Problem(ndim=2, nx=3, ny=2, order=9, bc=("periodic",) * 4)
        return pb, P.smooth_random(pb, 15), P.random_sigma(pb, 16, pb.sigma_thres / 2)
    if name == "2d_r9_jet_inflow_40x24":
        pb, _ = P.high_mach_jet(40, 24, 9)
        return pb, P.smooth_random(pb, 17), P.zero_sigma(pb)
    if name == "2d_r7_noise_20x18":
        pb = P.Problem(ndim=2, nx=20, ny=18, order=7)
        return pb, P.white_noise(pb, 18), P.random_sigma(pb, 19, pb.sigma_thres / 2)
    raise KeyError(name)


RESIDUAL_CASES = ["2d_r9_periodic_37x45", "2d_r7_outflow_40x33", "2d_r5_mixed_bc_35x20", "2d_r3_periodic_19x17",
                  "1d_r9_noise_300", "1d_r5_noise_periodic_1", "2d_r9_periodic_3x2", "2d_r9_jet_inflow_40x24",
                  "2d_r7_noise_20x18"]


@pytest.mark.parametrize("name", RESIDUAL_CASES)
def test_residual_adjoint_matches_oracle_tape(A, oracle, name):
    import torch

    from paper_2410_05489_gb300.adjoint import residual

    pb, W, (sx, sy) = residual_case(name)
    rng = np.random.default_rng(100)
    Lbar = rng.standard_normal(pb.state_shape)
    sxb = rng.standard_normal(pb.sx_shape)
    syb = rng.standard_normal(pb.sy_shape) if pb.ndim == 2 else np.zeros(pb.sy_shape)
    Wb_cpu, sxi_cpu, syi_cpu = oracle.residual_vjp(pb, W, sx, sy, Lbar, sxb, syb if pb.ndim == 2 else None)
    s = A.Solver(pb)
    try:
        # through the C ABI
        Wb, sxi, syi = s.residual_adjoint(dev(W), dev(sx), dev(sy), dev(Lbar), dev(sxb), dev(syb))
        torch.cuda.synchronize()
        floor = 1e-4 * np.abs(Lbar).max() * (1.0 / pb.dx + (1.0 / pb.dy if pb.ndim == 2 else 0.0))
        check("Wbar", rel_err(Wb.cpu().numpy(), Wb_cpu, floor), 1e-10)
        assert np.abs(sxi.cpu().numpy() - sxi_cpu).max() <= 1e-10 * max(np.abs(sxi_cpu).max(), floor)
        if pb.ndim == 2:
            assert np.abs(syi.cpu().numpy() - syi_cpu).max() <= 1e-10 * max(np.abs(syi_cpu).max(), floor)
        # through torch.autograd
        Wt = dev(W).requires_grad_(True)
        sxt = dev(sx).requires_grad_(True)
        syt = dev(sy).requires_grad_(True)
        L, sxo, syo = residual(s, Wt, sxt, syt)
        J = (L * dev(Lbar)).sum() + (sxo * dev(sxb)).sum() + ((syo * dev(syb)).sum() if pb.ndim == 2 else 0.0)
        gW, gsx = torch.autograd.grad(J, [Wt, sxt])
        assert torch.equal(gW, Wb) and torch.equal(gsx, sxi)
    finally:
        s.close()


def test_residual_adjoint_accumulates_and_is_deterministic(A):
    import torch

    pb, W, (sx, sy) = residual_case("2d_r7_noise_20x18")
    rng = np.random.default_rng(2)
    Lbar = dev(rng.standard_normal(pb.state_shape))
    s = A.Solver(pb)
    try:
        Wd, sxd, syd = dev(W), dev(sx), dev(sy)
        w1, x1, y1 = s.residual_adjoint(Wd, sxd, syd, Lbar)
        w2, x2, y2 = s.residual_adjoint(Wd, sxd, syd, Lbar)
        assert torch.equal(w1, w2) and torch.equal(x1, x2) and torch.equal(y1, y2)
        base = dev(rng.standard_normal(pb.state_shape))
        acc = base.clone()
        s.residual_adjoint(Wd, sxd, syd, Lbar, Wbar=acc)
        # accumulated per sweep direction: (base + x part) + y part
        assert torch.allclose(acc, base + w1, rtol=1e-14, atol=1e-14 * float(w1.abs().max()))
    finally:
        s.close()


@pytest.mark.parametrize("name", ["2d_r7_noise_20x18", "2d_r5_mixed_bc_35x20", "2d_r9_jet_inflow_40x24"])
def test_fused_gathers_equal_the_per_direction_gathers(A, name):
    """In 2D the gathers of both directions into W-bar and the sigma_in adjoints run as one
    launch; with kernel timing on they run per direction, in series. Both add the x-direction's
    sums before the y-direction's, so the results are equal bit for bit, also when they
    accumulate into nonzero outputs with nonzero sigma_out adjoints."""
    import torch

    pb, W, (sx, sy) = residual_case(name)
    rng = np.random.default_rng(5)
    Lbar = dev(rng.standard_normal(pb.state_shape))
    sxo, syo = dev(rng.standard_normal(sx.shape)), dev(rng.standard_normal(sy.shape))
    base = [dev(rng.standard_normal(a.shape)) for a in (W, sx, sy)]
    out = []
    s = A.Solver(pb)
    try:
        Wd, sxd, syd = dev(W), dev(sx), dev(sy)
        for timing in (False, True):
            A.ase_df_profile_enable(s.ctx, timing)
            acc = [b.clone() for b in base]
            s.residual_adjoint(Wd, sxd, syd, Lbar, sxo, syo, *acc)
            torch.cuda.synchronize()
            out.append(acc)
        A.ase_df_profile_enable(s.ctx, False)
    finally:
        s.close()
    for fused, serial in zip(*out):
        assert torch.equal(fused, serial), float((fused - serial).abs().max())


def perturbed_vortex(n, order, seed=1, ny=None):
    pb, W0 = P.isentropic_vortex(n, order, ny=ny)
    rng = np.random.default_rng(seed)
    W0 = W0.copy()
    W0[0] = W0[0] * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, W0[0].shape))
    return pb, W0


@pytest.mark.parametrize("case", ["vortex_r7_24x20", "vortex_r9_24x17", "sod_r5_80", "riemann2d_r5_24"])
def test_rollout_adjoint_matches_oracle_tape(A, oracle, case):
    import torch

    from paper_2410_05489_gb300.adjoint import rollout

    if case == "vortex_r7_24x20":
        pb, W0 = perturbed_vortex(24, 7, ny=20)
        nsteps, every = 5, 2
    elif case == "vortex_r9_24x17":
        pb, W0 = perturbed_vortex(24, 9, ny=17)
        nsteps, every = 2, 1
    elif case == "sod_r5_80":
        pb, W0 = P.sod(80, 5)
        nsteps, every = 4, 3
    else:
        pb, W0 = P.riemann_2d(24, 5, seed=3)
        nsteps, every = 3, 1
    dt = 0.5 * oracle.cfl_dt(pb, W0)
    Wf = oracle.run(pb, W0, nsteps=nsteps, dt=dt)[0]
    Wbf = np.zeros_like(Wf)
    Wbf[0] = 2.0 * Wf[0]
    G_cpu = oracle.run_vjp(pb, W0, nsteps, dt, Wbf)
    s = A.Solver(pb)
    try:
        W0t = dev(W0).requires_grad_(True)
        Wft = rollout(s, W0t, nsteps, dt, every=every)
        check("W final", rel_err(Wft.detach().cpu().numpy(), Wf), 1e-12)
        J = (Wft[0] ** 2).sum()
        (G,) = torch.autograd.grad(J, [W0t])
        G = G.cpu().numpy()
        check("gradient", rel_err(G, G_cpu), 1e-9)
    finally:
        s.close()


def test_adjoint_workload_vs_central_differences(A, oracle):
    """The adjoint workload: isentropic vortex on a 256^2 periodic grid, density times
    (1 + 0.01 xi), xi ~ U[-1, 1] per cell (seed 1), order 7, 50 SSP-RK3 steps at the t = 0
    CFL dt, checkpoints every 10 steps, J = sum of the final density squared; central
    differences with h = 1e-6 on 32 normalised Gaussian directions (seeds 100..131)."""
    import torch

    from paper_2410_05489_gb300.adjoint import rollout

    pb, W0 = perturbed_vortex(256, 7, seed=1)
    dt = oracle.cfl_dt(pb, W0)
    nsteps = 50
    s = A.Solver(pb)
    try:
        W0t = dev(W0).requires_grad_(True)
        Wf = rollout(s, W0t, nsteps, dt, every=10)
        J = (Wf[0] ** 2).sum()
        (G,) = torch.autograd.grad(J, [W0t])
        _, marked, _ = A.ase_df_get_repair_stats(s.ctx)
        assert marked == 0
        gnorm = float(torch.linalg.vector_norm(G))
        h = 1e-6
        worst = 0.0
        W0d = dev(W0)
        with torch.no_grad():
            for k in range(32):
                d = np.random.default_rng(100 + k).standard_normal(pb.state_shape)
                d = dev(d / np.linalg.norm(d))
                rp = rollout(s, W0d + h * d, nsteps, dt)[0]
                rm = rollout(s, W0d - h * d, nsteps, dt)[0]
                fd = float(((rp - rm) * (rp + rm)).sum()) / (2 * h)
                ad = float((G * d).sum())
                err = abs(fd - ad)
                worst = max(worst, err / (abs(ad) + 1e-3 * gnorm))
                assert err <= 1e-6 * abs(ad) + 1e-9 * gnorm, (k, fd, ad)
        print("adjoint workload: |grad J| = %.6e, worst relative FD mismatch %.3e" % (gnorm, worst))
    finally:
        s.close()
