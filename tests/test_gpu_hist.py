"""The device branch histogram (ase_df_hist_*) against the oracle's: per face and side the
branch of Algorithm 1 taken by the normal and (2D) the tangential reconstruction, and the
Gauss points that took first-order states (reading G21). Both sides decide from the same
sigma with the same association, so the counts are equal exactly."""
import numpy as np
import pytest

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


def gpu_hist(A, pb, W, sx, sy):
    import torch

    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    ctx = A.ase_df_init(A.params_from_problem(pb))
    try:
        Wd, sxd, syd = dev(W), dev(sx), dev(sy)
        L = torch.empty_like(Wd)
        sxo, syo = torch.empty_like(sxd), torch.empty_like(syd)
        two = pb.ndim == 2
        A.ase_df_residual(ctx, Wd, sxd, syd if two else None, L, sxo, syo if two else None)
        assert A.ase_df_hist_read(ctx) == [0] * 7  # counting is off by default
        A.ase_df_hist_enable(ctx, True)
        A.ase_df_residual(ctx, Wd, sxd, syd if two else None, L, sxo, syo if two else None)
        h = A.ase_df_hist_read(ctx)
        assert A.ase_df_hist_read(ctx) == [0] * 7  # reading clears
        return np.array(h)
    finally:
        A.ase_df_destroy(ctx)


@pytest.mark.parametrize("order", [3, 5, 7, 9])
@pytest.mark.parametrize("ndim", [1, 2])
def test_branch_histogram_equals_oracle(A, oracle, ndim, order):
    if ndim == 2:
        pb = P.Problem(ndim=2, nx=83, ny=70, order=order, bc=("outflow", "outflow", "periodic", "periodic"))
    else:
        pb = P.Problem(ndim=1, nx=3000, order=order, bc=("outflow",) * 4)
    W = P.white_noise(pb, 60 + order)
    sx, sy = P.random_sigma(pb, 61 + order, 2.0 if order == 3 else 1.0)
    hc = oracle.residual(pb, W, sx, sy)[-1][:7]
    hg = gpu_hist(A, pb, W, sx, sy)
    np.testing.assert_array_equal(hg, hc)
    # every branch the order has is taken, and white noise sends some Gauss points to first order
    expect = {3: [4, 5], 5: [2, 3], 7: [1, 2, 3], 9: [0, 1, 2, 3]}[order]
    assert all(hg[k] > 0 for k in expect), hg
    assert hg[6] > 0


def test_branch_histogram_of_a_graph_run(A, oracle):
    """Counting inside the captured step graph (ase_df_run): the 2D Riemann quadrants, 3 steps
    with CFL time steps, against the oracle's counts of the same steps."""
    pb, W0 = P.riemann_2d(96, 9, 2, ny=64)
    hc = np.zeros(len(oracle.BRANCHES), dtype=np.int64)
    sx, sy = oracle.prime_sigma(pb, W0)
    W, t = W0, 0.0
    for _ in range(3):
        W, sx, sy, dt = oracle.step(pb, W, sx, sy, oracle.cfl_dt(pb, W), hc, t=t)
        t += dt
    s = A.Solver(pb, W0)
    try:
        A.ase_df_hist_enable(s.ctx, True)
        s.run(3)
        hg = np.array(A.ase_df_hist_read(s.ctx))
    finally:
        s.close()
    np.testing.assert_array_equal(hg, hc[:7])
    assert hg[3] > 0  # the fallback took part
