"""Pins of the oracle's gas-kinetic flux and S2O4 stepping (Sec. 2.2, Appendix A).

* A uniform state: the GKS flux is the Euler flux and its time derivative vanishes.
* Continuous data (the same state and slopes on both sides): the flux is the Euler flux
  of that state and F_t the Cauchy-Kowalewski time derivative F'(W) W_t with
  W_t = -(F'(W) W_x + G'(W) W_y) -- the kinetic moments, the M a = b solves and the
  compatibility condition together must reproduce that exactly (Jacobians here by
  central differences of the closed-form Euler fluxes, independent of kinetic theory).
* Mirror symmetry of a Riemann-type point (x -> -x).
* Tables 1 and 2 of Sec. 4.2 (sin-waves, GKS + S2O4, dt = dx^(r/4), C1 = 0.001): the
  printed L1 errors are reproduced -- 1-D at N = 20 and 40 for orders 5, 7, 9 to 1 % (0.2 %
  observed), and the 2-D diagonal wave at N = 20, order 7, to 2 %.  (With the C1 = 0.05 of
  the paper's shock-case captions the 1-D errors come out 2 % higher; C1 = 0.001 is the
  reading for the accuracy runs.)
* Conservation on a periodic grid.
"""
import math

import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P


def cons(g, rho, u, v, p, dim=2):
    if dim == 1:
        return np.array([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])
    return np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])


def euler_fluxes(g, W):
    if len(W) == 3:
        rho, m, E = W
        u = m / rho
        p = (g - 1) * (E - 0.5 * rho * u * u)
        return np.array([m, m * u + p, u * (E + p)]), None
    rho, mu, mv, E = W
    u, v = mu / rho, mv / rho
    p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
    return np.array([mu, mu * u + p, mu * v, u * (E + p)]), np.array([mv, mv * u, mv * v + p, v * (E + p)])


def jacobian(f, W, h=1e-6):
    n = len(W)
    J = np.zeros((n, n))
    for k in range(n):
        d = np.zeros(n)
        d[k] = h * max(1.0, abs(W[k]))
        J[:, k] = (f(W + d) - f(W - d)) / (2 * d[k])
    return J


@pytest.mark.parametrize("dim", [1, 2])
def test_uniform_state_gives_the_euler_flux(oracle, dim):
    rng = np.random.default_rng(dim)
    for g in (1.4, 5.0 / 3.0):
        for _ in range(5):
            W = cons(g, rng.uniform(0.1, 5), rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(0.1, 5), dim)
            F, Ft = oracle.gks_point(dim, g, W, None, None, W, None, None, rng.uniform(1e-4, 1e-1))
            np.testing.assert_allclose(F, euler_fluxes(g, W)[0], rtol=1e-13, atol=1e-13 * np.abs(W).max())
            assert np.abs(Ft).max() <= 1e-10 * np.abs(W).max()


@pytest.mark.parametrize("dim", [1, 2])
def test_continuous_data_gives_flux_and_its_cauchy_kowalewski_derivative(oracle, dim):
    rng = np.random.default_rng(10 + dim)
    g = 1.4
    for _ in range(5):
        W = cons(g, rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.5, 2), dim)
        Wx = 0.3 * rng.standard_normal(len(W))
        Wy = 0.3 * rng.standard_normal(len(W)) if dim == 2 else np.zeros(len(W))
        F, Ft = oracle.gks_point(dim, g, W, Wx, Wy, W, Wx, Wy, rng.uniform(1e-4, 1e-2))
        Fx = lambda w: euler_fluxes(g, w)[0]  # noqa: E731
        A = jacobian(Fx, W)
        Wt = -A @ Wx
        if dim == 2:
            B = jacobian(lambda w: euler_fluxes(g, w)[1], W)
            Wt = Wt - B @ Wy
        np.testing.assert_allclose(F, Fx(W), rtol=1e-12, atol=1e-12 * np.abs(Fx(W)).max())
        np.testing.assert_allclose(Ft, A @ Wt, rtol=2e-7, atol=2e-7 * np.abs(A @ Wt).max())


def test_mirror_symmetry(oracle):
    """x -> -x maps (W_l, W_r) to (mirror W_r, mirror W_l) with flipped normal momentum
    and normal slopes of the same sign; the flux of mass and energy flips, that of
    normal momentum does not."""
    g = 1.4
    rng = np.random.default_rng(3)
    Wl = cons(g, 1.0, 0.3, 0.2, 1.0)
    Wr = cons(g, 0.4, -0.2, -0.1, 0.35)
    Wlx, Wrx = 0.2 * rng.standard_normal(4), 0.2 * rng.standard_normal(4)
    Wly, Wry = 0.2 * rng.standard_normal(4), 0.2 * rng.standard_normal(4)
    m = np.array([1.0, -1.0, 1.0, 1.0])  # flip the normal momentum
    F, Ft = oracle.gks_point(2, g, Wl, Wlx, Wly, Wr, Wrx, Wry, 1e-2)
    # mirrored: left <- mirror(right); d/dx flips sign, and so does the normal momentum
    G, Gt = oracle.gks_point(2, g, m * Wr, -m * Wrx, m * Wry, m * Wl, -m * Wlx, m * Wly, 1e-2)
    np.testing.assert_allclose(G, -m * F, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Gt, -m * Ft, rtol=1e-10, atol=1e-11)


def run_sin_wave_1d(oracle, N, r):
    pb, W = P.sin_wave_1d(N, r)
    pb = pb.replace(gks_c1=0.001)  # reading G24: the accuracy runs' C1 (not printed)
    n = int(math.ceil(2.0 / pb.dx ** (r / 4.0)))  # dt = dx^(r/s), s = 4 (S2O4), reading G28
    Wn, *_ = oracle.gks_run(pb, W, nsteps=n, dt=2.0 / n)
    ex = P.sin_wave_1d_exact(pb, 2.0)
    return np.abs(Wn[0] - ex[0]).sum() * pb.dx / 2.0


@pytest.mark.parametrize("r", [5, 7, 9])
def test_sin_wave_1d_reproduces_table1(oracle, golden, r):
    tab = golden("sin_wave_accuracy_tables.json")["table1_1d"]["r%d" % r]
    for k, N in enumerate((20, 40)):
        e = run_sin_wave_1d(oracle, N, r)
        assert abs(e / tab["err"][k] - 1.0) < 0.01, (N, e, tab["err"][k])


def test_sin_wave_2d_reproduces_table2(oracle, golden):
    """The diagonal wave at N = 20, order 7 (dt = dx^(7/4), below the CFL limit)."""
    tab = golden("sin_wave_accuracy_tables.json")["table2_2d"]["r7"]
    pb, W = P.sin_wave_2d_diag(20, 7)
    pb = pb.replace(gks_c1=0.001)
    n = int(math.ceil(2.0 / pb.dx ** (7 / 4.0)))
    Wn, *_ = oracle.gks_run(pb, W, nsteps=n, dt=2.0 / n)
    ex = P.sin_wave_2d_diag_exact(pb, 2.0)
    e = np.abs(Wn[0] - ex[0]).sum() * pb.dx * pb.dy / 4.0
    assert abs(e / tab["err"][0] - 1.0) < 0.02, (e, tab["err"][0])


def test_periodic_conservation(oracle):
    pb, _ = P.isentropic_vortex(12, 7, ny=10)
    W = P.smooth_random(pb, 5)
    sx, sy = P.random_sigma(pb, 6, pb.sigma_thres / 2)
    L, Lt, _, _, hist = oracle.gks_residual(pb, W, sx, sy, 1e-3)
    assert hist[oracle.BRANCHES.index("weno_df")] > 0
    for c in range(4):
        assert abs(L[c].sum()) <= 1e-12 * np.abs(L[c]).sum()
        assert abs(Lt[c].sum()) <= 1e-12 * np.abs(Lt[c]).sum()


def test_s2o4_is_fourth_order_in_time(oracle):
    """S2O4 (Sec. 2.2) on a fixed grid: the 1D sine wave on 40 cells at r = 9 with the
    gas-kinetic flux, marched to t = 0.4 with dt = 0.02 .. 0.0025 against 1280 steps of the same
    scheme.  The time error falls by 2^4 per halving of dt.  (At r = 5 the same runs show order 1:
    the flux terms proportional to the collision time tau = C1 dt + ..., which multiply the
    mismatch of the two reconstructed sides at a face, O(dx^(r-1)), are first order in dt and
    dominate there; at r = 9 they stay below the S2O4 error.)"""
    pb, W0 = P.sin_wave_1d(40, 9)
    T = 0.4
    ref = oracle.gks_run(pb, W0, nsteps=1280, dt=T / 1280)[0]
    errs = [np.abs(oracle.gks_run(pb, W0, nsteps=n, dt=T / n)[0] - ref).max() for n in (20, 40, 80, 160)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(3.9 < q < 4.1 for q in orders), orders
