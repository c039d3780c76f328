"""Pins of the oracle's flux, residual and time stepping (Sec. 2 and 4 of the paper)
against closed forms, invariants, a textbook first-order scheme, the exact Riemann
solution and the paper's printed convergence orders."""
import math

import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P


# ----------------------------------------------------------------------------------
# Lax-Friedrichs flux and sigma at a Gauss point (Sec. 2.3 and Sec. 3.1)
# ----------------------------------------------------------------------------------
def cons2(rho, u, v, p, g):
    return np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])


def test_lf_flux_consistency_and_sigma_closed_form(oracle):
    g = 1.4
    # rho = 1.4, p = 1 -> c = 1 exactly
    qL = cons2(1.4, 2.0, -0.5, 1.0, g)
    F, s, fb = oracle.lf_flux(qL, qL, g)
    E = qL[3]
    assert not fb and s == 0.0
    np.testing.assert_allclose(F, [1.4 * 2, 1.4 * 4 + 1, 1.4 * 2 * -0.5, 2 * (E + 1)], rtol=1e-15)
    # rho = 5.6, p = 4 -> c = 1; sigma = |dp|/pL + |dp|/pR + (dMa_n)^2 + (dMa_t)^2
    qR = cons2(5.6, 0.5, 1.5, 4.0, g)
    F, s, fb = oracle.lf_flux(qL, qR, g)
    assert not fb
    assert abs(s - (3 / 1 + 3 / 4 + (2 - 0.5) ** 2 + (-0.5 - 1.5) ** 2)) < 1e-14
    # Rusanov dissipation: lambda = max(|u|+c) = 3
    FL = np.array([2.8, 6.6, -1.4, 2 * (qL[3] + 1)])
    FR = np.array([5.6 * 0.5, 5.6 * 0.25 + 4, 5.6 * 0.5 * 1.5, 0.5 * (qR[3] + 4)])
    np.testing.assert_allclose(F, 0.5 * (FL + FR) - 0.5 * 3.0 * (qR - qL), rtol=1e-14)


def test_lf_positivity_fallback(oracle):
    """Reading G21: a non-physical reconstructed state -> the cell averages' flux and
    sigma = 1e30."""
    g = 1.4
    cL = cons2(1.0, 0.1, 0.0, 1.0, g)
    cR = cons2(0.5, 0.0, 0.2, 0.4, g)
    bad = cL.copy(); bad[0] = -0.1
    F, s, fb = oracle.lf_flux(bad, cR, g, cL, cR)
    F2, s2, fb2 = oracle.lf_flux(cL, cR, g)
    assert fb and not fb2 and s == 1e30
    np.testing.assert_array_equal(F, F2)
    bad = cR.copy(); bad[3] = 0.5 * (bad[1] ** 2 + bad[2] ** 2) / bad[0]  # p = 0
    F, s, fb = oracle.lf_flux(cL, bad, g, cL, cR)
    assert fb and s == 1e30


# ----------------------------------------------------------------------------------
# residual invariants
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("r", [3, 5, 7, 9])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_free_stream_is_exact(oracle, ndim, r, bc):
    pb = P.Problem(ndim=ndim, nx=13, ny=11, order=r, bc=(bc,) * 4)
    prim = (1.3, 0.7, -0.4, 2.1) if ndim == 2 else (1.3, 0.7, 2.1)
    U = P.conservative([np.full((pb.nyc, pb.nx), v) for v in prim], pb.gamma, ndim)
    L, sx, sy, *_ = oracle.residual(pb, U, *P.zero_sigma(pb))
    assert np.all(L == 0.0) and np.all(sx == 0.0) and np.all(sy == 0.0)


@pytest.mark.parametrize("r", [3, 5, 7, 9])
def test_conservation_periodic(oracle, r):
    """Telescoping of the face fluxes: sum of L over a periodic grid is round-off."""
    pb = P.Problem(ndim=2, nx=17, ny=14, order=r, bc=("periodic",) * 4)
    for seed, W in ((0, P.smooth_random(pb, 0)), (1, P.white_noise(pb, 1))):
        sx, sy = P.random_sigma(pb, seed, 0.5)
        L, _, _, Fx, Fy, _ = oracle.residual(pb, W, sx, sy)
        tot = L.sum(axis=(1, 2)) * pb.dx * pb.dy
        scale = max(np.abs(Fx).max(), np.abs(Fy).max()) * (pb.nx + pb.ny)
        assert np.all(np.abs(tot) < 1e-13 * scale), tot
        # faces 0 and nx (0 and ny) are the same periodic face
        np.testing.assert_array_equal(Fx[:, :, 0], Fx[:, :, -1])
        np.testing.assert_array_equal(Fy[:, 0, :], Fy[:, -1, :])


def _rough_share(hist, r):
    """Share of reconstructions that left the linear branches: the WENOZ-AO(5,3)+DF fallback
    (order 3: the DF-damped quadratic)."""
    return hist[5 if r == 3 else 3] / hist[:6].sum()


@pytest.mark.parametrize("r", [5, 9])
@pytest.mark.parametrize("sigma_scale", [0.5, 1.0])
def test_transpose_symmetry(oracle, r, sigma_scale):
    """Swapping x <-> y together with u <-> v transposes the residual. With face strengths
    up to 1.0 the 4-face sums straddle sigma_thres = 2, so a large share of the
    reconstructions take the WENOZ-AO(5,3)+DF fallback."""
    pb = P.Problem(ndim=2, nx=12, ny=12, order=r, bc=("periodic", "periodic", "outflow", "outflow"))
    pbt = pb.replace(bc=("outflow", "outflow", "periodic", "periodic"))
    W = P.white_noise(pb, 7)
    sx, sy = P.random_sigma(pb, 7, sigma_scale)
    sy[-1, :] = sy[0, :]  # periodic in y for pbt's x
    Wt = np.ascontiguousarray(W[[0, 2, 1, 3]].transpose(0, 2, 1))
    L, sxo, syo, *_, hist = oracle.residual(pb, W, sx, sy)
    if sigma_scale == 1.0:
        assert _rough_share(hist, r) > 0.3
    Lt, sxt, syt, *_ = oracle.residual(pbt, Wt, np.ascontiguousarray(sy.T), np.ascontiguousarray(sx.T))
    np.testing.assert_allclose(Lt, L[[0, 2, 1, 3]].transpose(0, 2, 1), rtol=0, atol=1e-12 * np.abs(L).max())
    np.testing.assert_allclose(sxt, syo.T, rtol=1e-12, atol=0)


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("r", [3, 5, 9])
@pytest.mark.parametrize("sigma_scale", [0.45, 1.0])
def test_mirror_symmetry(oracle, ndim, r, sigma_scale):
    """x -> -x with u -> -u mirrors the residual (the right state is the mirror image of
    the left one). In 2D the mirror also reverses the tangential reconstruction of the
    y-faces, which the oracle evaluates at the Gauss points directly (not through a mirrored
    stencil); with face strengths up to 1.0 a large share of it takes the WENOZ-AO(5,3)+DF
    fallback, whose weights are then pinned to treat beta3_{-1} and beta3_1 alike (reading
    G5)."""
    pb = P.Problem(ndim=ndim, nx=15 if ndim == 2 else 64, ny=9, order=r, bc=("outflow",) * 4)
    W = P.white_noise(pb, 11)
    # order 3 sums two faces: strengths up to 2.0 straddle sigma_thres there
    sx, sy = P.random_sigma(pb, 11, sigma_scale * (2.0 if r == 3 and sigma_scale == 1.0 else 1.0))
    Wm = W[:, :, ::-1].copy()
    Wm[1] *= -1
    L, sxo, syo, *_, hist = oracle.residual(pb, W, sx, sy)
    if sigma_scale == 1.0:
        assert _rough_share(hist, r) > 0.3
    Lm, sxm, sym_, *_ = oracle.residual(pb, Wm, np.ascontiguousarray(sx[:, ::-1]), np.ascontiguousarray(sy[:, ::-1]))
    Lref = L[:, :, ::-1].copy()
    Lref[1] *= -1
    for c in range(pb.ncomp):
        np.testing.assert_allclose(Lm[c], Lref[c], rtol=0, atol=1e-12 * np.abs(L[c]).max())
    np.testing.assert_allclose(sxm, sxo[:, ::-1], rtol=1e-11, atol=1e-12)


# ----------------------------------------------------------------------------------
# the DF limits (Remark 1 / Remark 4)
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("r", [5, 7, 9])
def test_df_recovers_linear_scheme_on_smooth_data(oracle, r):
    """On the smooth vortex the primed sigma stays below the threshold everywhere, so the
    residual equals the all-linear r-th order residual bit for bit."""
    pb, W = P.isentropic_vortex(32, r)
    s0 = P.zero_sigma(pb)
    sx, sy = oracle.prime_sigma(pb, W)
    assert max(sx.max(), sy.max()) < 0.25
    L1, *_, h1 = oracle.residual(pb, W, sx, sy)
    L0, *_, h0 = oracle.residual(pb, W, *s0)
    np.testing.assert_array_equal(L1, L0)
    lin = {5: 2, 7: 1, 9: 0}[r]
    assert h1[lin] == h1.sum()


def rusanov_first_order(pb, W):
    """Textbook first-order local Lax-Friedrichs (Rusanov) residual, 2D, periodic."""
    g = pb.gamma

    def flux(U, axis):
        rho = U[0]
        u, v = U[1] / rho, U[2] / rho
        p = (g - 1) * (U[3] - 0.5 * rho * (u * u + v * v))
        c = np.sqrt(g * p / rho)
        un = u if axis == 2 else v
        F = np.stack([rho * un, U[1] * un, U[2] * un, un * (U[3] + p)])
        F[1 if axis == 2 else 2] += p
        return F, np.abs(un) + c

    L = np.zeros_like(W)
    for axis, h in ((2, pb.dx), (1, pb.dy)):
        Ur = np.roll(W, -1, axis=axis)
        FL, aL = flux(W, axis)
        FR, aR = flux(Ur, axis)
        lam = np.maximum(aL, aR)
        Fh = 0.5 * (FL + FR) - 0.5 * lam * (Ur - W)  # flux at the +1/2 face
        L -= (Fh - np.roll(Fh, 1, axis=axis)) / h
    return L


@pytest.mark.parametrize("r", [5, 9])
def test_df_first_order_limit(oracle, r):
    """Remark 4: sigma >> sigma_thres drives every alpha to ~0, and the scheme becomes the
    first-order local Lax-Friedrichs scheme."""
    pb = P.Problem(ndim=2, nx=10, ny=8, order=r, bc=("periodic",) * 4)
    W = P.white_noise(pb, 5)
    sx = np.full(pb.sx_shape, 1e28)
    sy = np.full(pb.sy_shape, 1e28)
    L, *_ = oracle.residual(pb, W, sx, sy)
    Lref = rusanov_first_order(pb, W)
    for c in range(4):
        np.testing.assert_allclose(L[c], Lref[c], rtol=0, atol=1e-12 * np.abs(Lref[c]).max())


# ----------------------------------------------------------------------------------
# accuracy (Sec. 4.2)
# ----------------------------------------------------------------------------------
def sinwave2d_exact_rate(pb):
    """Exact d/dt of the cell averages of rho for the 2D sin-wave at t = 0:
    rho_t = -(rho_x + rho_y) with rho = 1 + 0.2 sin(pi x) sin(pi y); its cell average is
    -(1/(dx dy)) [ (F(x+) - F(x-)) * Y + X * (G(y+) - G(y-)) ] in closed form."""
    x = pb.x0 + np.arange(pb.nx + 1) * pb.dx
    y = pb.y0 + np.arange(pb.ny + 1) * pb.dy
    sx_ = np.sin(np.pi * x)
    sy_ = np.sin(np.pi * y)
    cx = -np.cos(np.pi * x) / np.pi  # antiderivative of sin
    cy = -np.cos(np.pi * y) / np.pi
    Ix = np.diff(cx)  # int sin(pi x) over cells
    Iy = np.diff(cy)
    dx_term = np.outer(Iy, np.diff(sx_))  # int_y sin(pi y) * [sin(pi x)]_{x-}^{x+}
    dy_term = np.outer(np.diff(sy_), Ix)
    return -0.2 * (dx_term + dy_term) / (pb.dx * pb.dy)


@pytest.mark.parametrize("r,min_order", [(5, 4.5), (7, 6.5), (9, 8.3)])
def test_residual_truncation_order_2d(oracle, r, min_order):
    """Space-only order of the 2D residual on exact cell averages of the sin-wave.  The
    (r-1)/2-point face quadrature of Sec. 2.1 bounds the formal 2D order by r-1, but its
    error constant is small: at these resolutions the observed order is ~r (4.96 / 6.94 /
    8.82 measured), and at least r - 1/2 is required."""
    errs = []
    Ns = (10, 20) if r == 9 else (16, 32)
    for N in Ns:
        pb, W = P.sin_wave_2d(N, r)
        L, *_ = oracle.residual(pb, W, *P.zero_sigma(pb))
        errs.append(np.abs(L[0] - sinwave2d_exact_rate(pb)).mean())
    order = math.log(errs[0] / errs[1], 2)
    assert order > min_order, (errs, order)


def run_sin_wave_1d(oracle, N, r):
    pb, W = P.sin_wave_1d(N, r)
    dt_cfl = oracle.cfl_dt(pb, W)
    dt = min(dt_cfl, pb.dx ** (r / 3.0))  # dt = dx^(r/s) with s = 3 (Sec. 4.2)
    nsteps = int(math.ceil(2.0 / dt))
    Wn, *_ = oracle.run(pb, W, nsteps=nsteps, dt=2.0 / nsteps)
    ex = P.sin_wave_1d_exact(pb, 2.0)
    return np.abs(Wn[0] - ex[0]).sum() * pb.dx / 2.0


@pytest.mark.parametrize("r", [5, 7, 9])
def test_sin_wave_1d_orders_match_table1(oracle, golden, r):
    """Sec. 4.2, Table 1: observed L1 orders at N = 20 -> 40 agree with the printed ones
    (4.95 / 6.96 / 8.97) within 0.35."""
    tab = golden("sin_wave_accuracy_tables.json")["table1_1d"]["r%d" % r]
    e20 = run_sin_wave_1d(oracle, 20, r)
    e40 = run_sin_wave_1d(oracle, 40, r)
    order = math.log(e20 / e40, 2)
    assert abs(order - tab["order"][1]) < 0.35, (e20, e40, order)


# ----------------------------------------------------------------------------------
# shock tube against the exact Riemann solution
# ----------------------------------------------------------------------------------
def test_exact_riemann_solver_sod_star_state(golden):
    from oracle import riemann_exact as R

    ref = golden("sod_star_state.json")
    ps, us = R.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - ref["p_star"]) < 1e-5 and abs(us - ref["u_star"]) < 1e-5
    rl = R.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), us - 1e-9)[0]
    rr = R.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), us + 1e-9)[0]
    assert abs(rl - ref["rho_star_left"]) < 1e-5 and abs(rr - ref["rho_star_right"]) < 1e-5
    # Rankine-Hugoniot across the right shock: mass flux continuity in the shock frame
    g = 1.4
    S = 0.0 + math.sqrt(g * 0.1 / 0.125) * math.sqrt((g + 1) / (2 * g) * ps / 0.1 + (g - 1) / (2 * g))
    assert abs(rr * (us - S) - 0.125 * (0.0 - S)) < 1e-12


@pytest.mark.slow
def test_sod_converges_to_exact_solution(oracle):
    from oracle import riemann_exact as R

    errs = []
    for n in (100, 200, 400):
        pb, W = P.sod(n, 5)
        Wn, _, _, t, _ = oracle.run(pb, W, t_end=0.2)
        assert abs(t - 0.2) < 1e-12
        rho = Wn[0, 0]
        u = Wn[1, 0] / rho
        p = (pb.gamma - 1) * (Wn[2, 0] - 0.5 * rho * u * u)
        assert rho.min() > 0 and p.min() > 0
        ex = R.cell_averages((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.0, 1.0, n, 0.5, 0.2, sub=16)
        errs.append(np.abs(rho - ex[0]).mean())
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 0.01


def test_jet_positivity_small(oracle):
    """Sec. 4.3, Example 6 (Ma ~ 20000, L-F solver): density and pressure stay positive on
    a coarse copy of the jet over its first steps."""
    pb, W = P.high_mach_jet(64, 32, 9)
    Wn, sx, sy, t, n = oracle.run(pb, W, nsteps=20)
    rho = Wn[0]
    p = (pb.gamma - 1) * (Wn[3] - 0.5 * (Wn[1] ** 2 + Wn[2] ** 2) / rho)
    assert np.all(np.isfinite(Wn)) and rho.min() > 0 and p.min() > 0
    # the inflow has entered: some cells next to the band carry x-momentum
    assert Wn[1, 12:20, 0].max() > 1.0


def near_vacuum_1d(n=100, r=9):
    """Two streams leaving each other at Mach ~40 on a periodic line: a near-vacuum
    rarefaction at x = 1/2 and a strong collision at x = 0."""
    pb = P.Problem(ndim=1, nx=n, order=r, bc=("periodic",) * 4)
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    prim = (np.ones(n), np.where(left, -6.0, 6.0), np.full(n, 0.02))
    return pb, np.ascontiguousarray(P.conservative(prim, pb.gamma, 1)[:, None, :])


def test_positivity_repair_is_conservative(oracle):
    """Reading G21b: where the high-order stage update would leave a cell non-physical,
    the first-order repair keeps every cell physical, and because repaired faces are
    shared by both of their cells the periodic totals stay conserved to rounding."""
    pb, W = near_vacuum_1d()
    tot0 = W.sum(axis=(1, 2))
    sx, sy = oracle.prime_sigma(pb, W)
    hist = np.zeros(len(oracle.BRANCHES), dtype=np.int64)
    for _ in range(30):
        W, sx, sy, dt = oracle.step(pb, W, sx, sy, 0.0, hist)
        assert dt > 0
    assert hist[oracle.BRANCHES.index("repaired")] > 0
    rho = W[0, 0]
    p = (pb.gamma - 1) * (W[2, 0] - 0.5 * W[1, 0] ** 2 / rho)
    assert rho.min() > 0 and p.min() > 0
    assert np.all(np.abs(W.sum(axis=(1, 2)) - tot0) <= 1e-13 * np.abs(W).sum(axis=(1, 2)))


@pytest.mark.parametrize("order", [5, 9])
def test_jet_reaches_t_end_with_repair(oracle, order):
    """Sec. 4.3, Example 6: the coarse Ma-20000 jet reaches t = 1e-5 with every cell
    physical at every step (order 5 needs the stage repair from the first step on)."""
    pb, W = P.high_mach_jet(80, 40, order)
    Wn, sx, sy, t, n = oracle.run(pb, W, t_end=1e-5)
    rho = Wn[0]
    p = (pb.gamma - 1) * (Wn[3] - 0.5 * (Wn[1] ** 2 + Wn[2] ** 2) / rho)
    assert abs(t - 1e-5) < 1e-15 and rho.min() > 0 and p.min() > 0



@pytest.mark.parametrize("r,min_order", [(5, 4.5), (7, 6.0)])
def test_vortex_convergence_order(oracle, r, min_order):
    """Measured convergence on the smooth isentropic vortex (strength 5 on (1,1,1,1),
    periodic [0,10]^2): the vortex is advected unchanged, so the exact solution at t is the
    initial field shifted by (t, t).  40^2 and 80^2 cells to t = 0.2 with dt = min(CFL dt,
    dx^(r/3)) (the SSP-RK3 time error then scales as dx^r): L1 error of the density falls
    at order >= 4.5 (r = 5, observed 4.72) and >= 6.0 (r = 7, observed 6.18; 40^2 cells
    resolve the vortex core with 4 cells per unit, still pre-asymptotic for the high orders).
    The GPU path's orders on 32^2 .. 256^2 to t = 2 are in tests/test_gpu_convergence.py."""
    T = 0.2
    errs = []
    for n in (40, 80):
        pb, W0 = P.isentropic_vortex(n, r)
        h = min(oracle.cfl_dt(pb, W0), pb.dx ** (r / 3.0))
        nsteps = int(np.ceil(T / h))
        W, *_ = oracle.run(pb, W0, nsteps=nsteps, dt=T / nsteps)
        errs.append(np.abs(W[0] - P.vortex_exact(pb, T)[0]).mean())
    assert np.log2(errs[0] / errs[1]) >= min_order, errs


def test_ssp_rk3_is_third_order_in_time(oracle):
    """SSP-RK3 (Sec. 2.3) on a fixed grid: the 1D sine wave on 40 cells at r = 9 (smooth,
    so the linear branch throughout), marched to t = 0.4 with dt = 0.02, 0.01, 0.005 and
    0.0025 (CFL 0.93 down to 0.12) against 1280 steps of the same scheme.  The spatial error
    is common to all runs, so the differences are the time error.  They fall by 2^3 per
    halving of dt; a wrong stage weight would leave the scheme first or second order."""
    pb, W0 = P.sin_wave_1d(40, 9)
    T = 0.4
    ref = oracle.run(pb, W0, nsteps=1280, dt=T / 1280)[0]
    errs = [np.abs(oracle.run(pb, W0, nsteps=n, dt=T / n)[0] - ref).max() for n in (20, 40, 80, 160)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(2.9 < q < 3.1 for q in orders), orders
