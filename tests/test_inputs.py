"""The seeded input generators (paper_2410_05489_gb300/problems.py) against the recipe they
state: ranges and distributions of the random states, the batched workload's mix, and
determinism per seed.  No method arithmetic is involved; both the oracle and the GPU path
take these inputs."""
import numpy as np

from paper_2410_05489_gb300 import problems as P


def _primitives(pb, W):
    g = pb.gamma
    rho = W[0]
    u = W[1] / rho
    v = W[2] / rho if pb.ndim == 2 else 0.0 * u
    p = (g - 1.0) * (W[-1] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def test_white_noise_follows_its_recipe():
    for ndim in (1, 2):
        pb = P.Problem(ndim=ndim, nx=200, ny=150 if ndim == 2 else 1, order=9)
        W = P.white_noise(pb, 3)
        assert W.shape == pb.state_shape and W.flags["C_CONTIGUOUS"]
        rho, u, v, p = _primitives(pb, W)
        tol = 1e-9
        assert rho.min() >= 0.1 - tol and rho.max() <= 10.0 + tol
        assert p.min() >= 0.1 - tol and p.max() <= 10.0 + tol
        assert np.abs(u).max() <= 2.0 + tol and np.abs(v).max() <= 2.0 + tol
        # log-uniform: log10(rho) spreads over [-1, 1] with mean ~0
        assert abs(np.log10(rho).mean()) < 0.02 and np.log10(rho).std() > 0.5
        assert np.array_equal(W, P.white_noise(pb, 3))
        assert not np.array_equal(W, P.white_noise(pb, 4))


def test_random_sigma_range_and_periodic_faces():
    pb = P.Problem(ndim=2, nx=30, ny=20, order=7, bc=("periodic",) * 4)
    sx, sy = P.random_sigma(pb, 1, 0.5)
    assert sx.shape == pb.sx_shape and sy.shape == pb.sy_shape
    assert sx.min() >= 0.0 and sx.max() < 0.5 and sy.min() >= 0.0 and sy.max() < 0.5
    assert np.array_equal(sx[:, -1], sx[:, 0]) and np.array_equal(sy[-1, :], sy[0, :])


def test_isentropic_vortex_is_symmetric_and_physical():
    pb, W = P.isentropic_vortex(64, 9)
    rho, u, v, p = _primitives(pb, W)
    assert rho.min() > 0 and p.min() > 0
    # rho depends on the distance to the centre only: symmetric under x <-> y
    assert np.abs(rho - rho.T).max() < 1e-13
    # the far field is the free stream (1, 1, 1, 1)
    assert abs(rho[0, 0] - 1.0) < 1e-6 and abs(u[0, 0] - 1.0) < 1e-5 and abs(p[0, 0] - 1.0) < 1e-6


def test_batched_workload_follows_its_recipe():
    probs = P.batched_problems()
    assert len(probs) == 512
    one, two = probs[:256], probs[256:]
    assert all(pb.ndim == 1 for pb, _ in one) and all(pb.ndim == 2 for pb, _ in two)
    assert all(128 <= pb.nx <= 16384 for pb, _ in one)
    assert all(64 <= pb.nx <= 512 and pb.ny == pb.nx for pb, _ in two)
    orders = [pb.order for pb, _ in probs]
    assert set(orders) == {3, 5, 7, 9} and min(orders.count(r) for r in (3, 5, 7, 9)) > 90
    assert all(pb.bc == ("outflow",) * 4 for pb, _ in probs)
    assert sum(pb.ncells for pb, _ in probs) == 18025229
    # log-uniform sizes: the median of the 1D sizes lies near the geometric mean of the range
    med = np.median([pb.nx for pb, _ in one])
    assert 0.6 * np.sqrt(128 * 16384) < med < 1.6 * np.sqrt(128 * 16384)
    # every problem is physical and piecewise constant (two 1D states, four 2D quadrants)
    for pb, W in probs[::37]:
        rho, u, v, p = _primitives(pb, W)
        assert rho.min() >= 0.1 - 1e-9 and rho.max() <= 10 + 1e-9 and p.min() >= 0.1 - 1e-9
        assert len(np.unique(rho)) <= (2 if pb.ndim == 1 else 4)
    again = P.batched_problems()
    assert all(np.array_equal(a[1], b[1]) for a, b in zip(probs[:8], again[:8]))


def test_jet_configuration():
    """The Mach-20000 jet (a re-scaled Sec. 4.3, Example 6): [0,1] x [-0.25,0.25] at 1600 x 800,
    gamma 5/3, ambient (0.5, 0, 0, 0.4127) at rest, inflow band |y| < 0.05 at x = 0 with
    rho = 5, p = 0.4127 and u = 20000 sqrt(gamma p / rho); the band edges fall on cell faces."""
    pb, W = P.high_mach_jet(1600, 800, 9)
    assert (pb.nx, pb.ny, pb.x0, pb.x1, pb.y0, pb.y1) == (1600, 800, 0.0, 1.0, -0.25, 0.25)
    assert abs(pb.gamma - 5.0 / 3.0) < 1e-15 and pb.bc == ("inflow", "outflow", "outflow", "outflow")
    rho_in, u_in, v_in, p_in = pb.inflow
    assert (rho_in, v_in, p_in) == (5.0, 0.0, 0.4127)
    assert abs(u_in / np.sqrt(pb.gamma * p_in / rho_in) - 20000.0) < 1e-6
    assert abs(u_in - 7417.996) < 1e-3
    for edge in (pb.inflow_lo, pb.inflow_hi):
        k = (edge - pb.y0) / pb.dy
        assert abs(k - round(k)) < 1e-9  # 80 cells on each side of y = 0
    rho, u, v, p = _primitives(pb, W)
    assert np.all(rho == 0.5) and np.all(u == 0.0) and np.allclose(p, 0.4127, rtol=0, atol=1e-15)
