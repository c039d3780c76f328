"""GPU parity of the gas-kinetic path (Sec. 2.2 with Appendix A): face kernel, L and L_t,
sigma_out, S2O4 steps, and the printed Table 1 errors reproduced on the GPU.

Tolerances:
  * L: per component, max|L_gpu - L_cpu| <= 1e-11 max(max|L_cpu|, floor), floor as in the
    Lax-Friedrichs parity (1e-3 max|F| (1/dx + 1/dy)): the flux adds erfc and exp (CUDA's
    and the C library's differ by an ulp) and a closed-form slope solve against the
    oracle's Gaussian elimination.
  * L_t: the same, with the floor 1e-3 max|F| (1/dx + 1/dy) / dt: F_t is formed as
    4 (F(dt) - 2 F(dt/2)) / dt^2 from flux integrals of size dt |F|, so its rounding is
    ~eps |F| / dt.
  * sigma_out: 1e-12 (1 + |s|) + 1e-14 s^2 elementwise (as the Lax-Friedrichs path).
  * S2O4 steps: max|W_gpu - W_cpu| <= 1e-10 max|W_cpu| after 5-10 steps.
"""
import math

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
    return max(np.abs(gpu[c] - cpu[c]).max() / max(np.abs(cpu[c]).max(), floor) for c in range(cpu.shape[0]))


def case(name):
    if name == "2d_r9_periodic_37x45":
        pb, _ = P.isentropic_vortex(37, 9, ny=45)
        return pb, P.smooth_random(pb, 3), P.random_sigma(pb, 5, pb.sigma_thres / 2)
    if name == "2d_r7_outflow_40x33":
        pb = P.Problem(ndim=2, nx=40, ny=33, order=7)
        return pb, P.smooth_random(pb, 4), P.random_sigma(pb, 6, pb.sigma_thres / 2)
    if name == "2d_r5_mixed_35x20":
        pb = P.Problem(ndim=2, nx=35, ny=20, order=5, bc=("periodic", "periodic", "outflow", "outflow"))
        return pb, P.smooth_random(pb, 7), P.random_sigma(pb, 8, pb.sigma_thres / 2)
    if name == "2d_r3_periodic_19x17":
        pb = P.Problem(ndim=2, nx=19, ny=17, order=3, bc=("periodic",) * 4)
        return pb, P.smooth_random(pb, 11), P.random_sigma(pb, 12, pb.sigma_thres)
    if name == "1d_r9_noise_300":
        pb = P.Problem(ndim=1, nx=300, order=9)
        return pb, P.white_noise(pb, 9), P.random_sigma(pb, 10, pb.sigma_thres / 2)
    if name == "1d_r5_sod_primed":
        pb, W = P.sod(200, 5)
        return pb, W, None
    if name == "2d_r9_riemann_40x36":
        pb, W = P.riemann_2d(40, 9, seed=3, ny=36)
        return pb, W, None
    if name == "2d_r9_jet_40x24":
        pb, _ = P.high_mach_jet(40, 24, 9)
        return pb, P.smooth_random(pb, 17), P.zero_sigma(pb)
    raise KeyError(name)


CASES = ["2d_r9_periodic_37x45", "2d_r7_outflow_40x33", "2d_r5_mixed_35x20", "2d_r3_periodic_19x17",
         "1d_r9_noise_300", "1d_r5_sod_primed", "2d_r9_riemann_40x36", "2d_r9_jet_40x24"]


@pytest.mark.parametrize("name", CASES)
def test_gks_residual_matches_oracle(A, oracle, name):
    import torch

    pb, W, sig = case(name)
    sx, sy = oracle.prime_sigma(pb, W) if sig is None else sig
    dt = 0.5 * oracle.cfl_dt(pb, W)
    L, Lt, sxo, syo, hist = oracle.gks_residual(pb, W, sx, sy, dt)
    s = A.Solver(pb)
    try:
        Lg, Ltg, sxg, syg = s.gks_residual(dt, dev(W), dev(sx), dev(sy))
        torch.cuda.synchronize()
        _, _, _, Fx, Fy, _ = oracle.residual(pb, W, sx, sy)  # the flux scale (Lax-Friedrichs)
        inv = 1.0 / pb.dx + (1.0 / pb.dy if pb.ndim == 2 else 0.0)
        Fmax = max(np.abs(Fx).max(), np.abs(Fy).max() if Fy is not None else 0.0)
        check("L (GKS)", comp_err(Lg.cpu().numpy(), L, 1e-3 * Fmax * inv), 1e-11)
        check("L_t (GKS)", comp_err(Ltg.cpu().numpy(), Lt, 1e-3 * Fmax * inv / dt), 1e-11)
        for a, b in ((sxg.cpu().numpy(), sxo), (syg.cpu().numpy(), syo)):
            if pb.ndim == 1 and b is syo:
                continue
            assert np.all(np.abs(a - b) <= 1e-12 * (1 + np.abs(b)) + 1e-14 * b * b)
    finally:
        s.close()


@pytest.mark.parametrize("name,nsteps", [("sod_r5", 10), ("vortex_r9_32", 5), ("riemann2d_r7_30", 5)])
def test_gks_steps_match_oracle(A, oracle, name, nsteps):
    import torch

    if name == "sod_r5":
        pb, W0 = P.sod(200, 5)
    elif name == "vortex_r9_32":
        pb, W0 = P.isentropic_vortex(32, 9)
    else:
        pb, W0 = P.riemann_2d(30, 7, seed=5)
    Wc, sxc, syc, t, n = oracle.gks_run(pb, W0, nsteps=nsteps)
    s = A.Solver(pb, W0)
    try:
        for _ in range(nsteps):
            s.gks_step()
        flags, last_dt, tg = s.status()
        torch.cuda.synchronize()
        assert flags & 1 == 0
        assert abs(tg - t) <= 1e-11 * t  # CFL dt from sqrt and division on both sides
        check("W after steps", comp_err(s.W.cpu().numpy(), Wc, 0.0), 1e-10)
    finally:
        s.close()


def test_gks_reproduces_table1_on_gpu(A, golden):
    """Sec. 4.2 Table 1, order 9, N = 40: dt = dx^(9/4), 1692 S2O4 steps to t = 2."""
    import torch

    tab = golden("sin_wave_accuracy_tables.json")["table1_1d"]["r9"]
    pb, W = P.sin_wave_1d(40, 9)
    pb = pb.replace(gks_c1=0.001)  # the accuracy runs' C1
    n = int(math.ceil(2.0 / pb.dx ** (9 / 4.0)))
    s = A.Solver(pb, W)
    try:
        for _ in range(n):
            s.gks_step(2.0 / n)
        torch.cuda.synchronize()
        ex = P.sin_wave_1d_exact(pb, 2.0)
        e = np.abs(s.W.cpu().numpy()[0] - ex[0]).sum() * pb.dx / 2.0
        assert abs(e / tab["err"][1] - 1.0) < 0.01, (e, tab["err"][1])
    finally:
        s.close()
