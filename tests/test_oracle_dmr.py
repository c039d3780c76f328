"""Pins of the double Mach reflection boundaries (Sec. 4.3 Example 4, reading G32) in the
oracle: the split bottom (the post-shock state below x < 1/6, a slip wall after) and the top
that follows the exact shock position x_s(t) = 1/6 + (1 + 20 t) / sqrt(3).

The ghost-cell rules are checked against an independent construction: the same grid
extended by G rows, the extra rows filled with what the rule prescribes, gives the same
residual on the original rows.  The stage times of SSP-RK3 (t, t + dt, t + dt/2) are checked
against a step composed by hand from residuals, and the moving boundary against the exact
position of a Rankine-Hugoniot shock."""
import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P

S3 = np.sqrt(3.0)


def dmr(nx, order, **kw):
    pb, W = P.double_mach_reflection(nx, order)
    return pb.replace(**kw), W


def xc(pb, i):
    return pb.x0 + (np.asarray(i, dtype=float) + 0.5) * pb.dx


def noise_sigma(pb, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 0.6, pb.sx_shape), rng.uniform(0.0, 0.6, pb.sy_shape)


def test_free_stream_is_kept_by_every_boundary_part(oracle):
    rest = (1.4, 0.0, 0.0, 1.0)
    for r in (5, 9):
        pb, _ = dmr(48, r, inflow=rest, state_b=rest)
        W = np.ascontiguousarray(np.broadcast_to(P.conservative(tuple(np.full((pb.ny, pb.nx), v) for v in rest),
                                                                pb.gamma, 2), pb.state_shape))
        for t in (0.0, 0.1):
            L, *_ = oracle.residual(pb, W, *noise_sigma(pb, 1), t=t)
            assert np.abs(L).max() <= 1e-12 * 1.0 / pb.dx


@pytest.mark.parametrize("r", [5, 9])
def test_split_bottom_equals_explicit_ghost_rows(oracle, r):
    """Bottom: ghost cells of columns with centre x < wall_x hold the post-shock state, the
    others mirror the rows above with v negated; sigma of the ghost faces clamps before the
    wall and mirrors after it."""
    K = (r - 1) // 2
    G = 2 * K + 4
    pb, W = dmr(48, r, bc=("outflow", "outflow", "wall_after", "outflow"))
    W = W.copy()
    W[:, :, :] += 0.05 * np.random.default_rng(3).standard_normal(W.shape) * np.abs(W)
    sx, sy = noise_sigma(pb, 2)
    L, sxo, syo, *_ = oracle.residual(pb, W, sx, sy)
    # the extended grid: rows -G .. -1 explicit
    ext = pb.replace(ny=pb.ny + G, y0=pb.y0 - G * pb.dy, bc=("outflow",) * 4)
    before = xc(pb, np.arange(pb.nx)) < pb.wall_x
    post = P.conservative(tuple(np.full(pb.nx, v) for v in pb.inflow), pb.gamma, 2)  # [4, nx]
    We = np.empty(ext.state_shape)
    We[:, G:, :] = W
    for g in range(1, G + 1):  # ghost row -g mirrors row g-1
        m = W[:, g - 1, :].copy()
        m[2] *= -1.0
        We[:, G - g, :] = np.where(before[None, :], post, m)
    sxe = np.empty(ext.sx_shape)
    sxe[G:, :] = sx
    before_f = xc(pb, np.arange(pb.nx + 1)) < pb.wall_x  # x-face f: the column right of it
    for g in range(1, G + 1):
        sxe[G - g, :] = np.where(before_f, sx[0, :], sx[g - 1, :])
    sye = np.empty(ext.sy_shape)
    sye[G:, :] = sy
    for g in range(1, G + 1):  # ghost face -g mirrors face g; before the wall face 0
        sye[G - g, :] = np.where(before, sy[0, :], sy[g, :])
    Le, sxoe, syoe, *_ = oracle.residual(ext, np.ascontiguousarray(We), sxe, sye)
    np.testing.assert_allclose(L, Le[:, G:, :], rtol=1e-13, atol=1e-13 * np.abs(L).max())
    np.testing.assert_allclose(sxo, sxoe[G:, :], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(syo, syoe[G:, :], rtol=1e-13, atol=1e-14)
    # and the split matters: a plain wall differs before x = 1/6 only
    Lw, *_ = oracle.residual(pb.replace(bc=("outflow", "outflow", "reflect", "outflow")), W, sx, sy)
    d = np.abs(Lw - L).max(axis=(0, 1))
    i_wall = int(np.sum(before))
    assert d[: i_wall].max() > 1e-6 * np.abs(L).max()
    assert d[i_wall + K + 3:].max() == 0.0


@pytest.mark.parametrize("r", [5, 9])
def test_moving_shock_top_equals_explicit_ghost_rows(oracle, r):
    K = (r - 1) // 2
    G = 2 * K + 4
    pb, W = dmr(48, r, bc=("outflow", "outflow", "outflow", "moving_shock"))
    sx, sy = noise_sigma(pb, 5)
    for t in (0.0, 0.013, 0.07):
        L, sxo, syo, *_ = oracle.residual(pb, W, sx, sy, t=t)
        ext = pb.replace(ny=pb.ny + G, y1=pb.y1 + G * pb.dy, bc=("outflow",) * 4)
        left = xc(pb, np.arange(pb.nx)) < pb.shock_x0 + pb.shock_speed * t
        post = P.conservative(tuple(np.full(pb.nx, v) for v in pb.inflow), pb.gamma, 2)
        pre = P.conservative(tuple(np.full(pb.nx, v) for v in pb.state_b), pb.gamma, 2)
        We = np.empty(ext.state_shape)
        We[:, : pb.ny, :] = W
        We[:, pb.ny:, :] = np.where(left, post, pre)[:, None, :]
        sxe = np.empty(ext.sx_shape)
        sxe[: pb.ny] = sx
        sxe[pb.ny:] = sx[-1]
        sye = np.empty(ext.sy_shape)
        sye[: pb.ny + 1] = sy
        sye[pb.ny + 1:] = sy[-1]
        Le, sxoe, syoe, *_ = oracle.residual(ext, np.ascontiguousarray(We), sxe, sye)
        np.testing.assert_allclose(L, Le[:, : pb.ny, :], rtol=1e-13, atol=1e-13 * np.abs(L).max())
        np.testing.assert_allclose(syo, syoe[: pb.ny + 1], rtol=1e-13, atol=1e-14)
    # the boundary moves: two times on either side of a column centre differ near it only
    i = 30
    tc = (xc(pb, i) - pb.shock_x0) / pb.shock_speed
    La, *_ = oracle.residual(pb, W, sx, sy, t=tc - 1e-9)
    Lb, *_ = oracle.residual(pb, W, sx, sy, t=tc + 1e-9)
    d = np.abs(La - Lb).max(axis=0)
    assert d[:, i].max() > 0.0
    cols = np.nonzero(d.max(axis=0))[0]
    rows = np.nonzero(d.max(axis=1))[0]
    assert cols.min() >= i - K - 2 and cols.max() <= i + K + 2
    assert rows.min() >= pb.ny - K - 2


def test_ssp_rk3_stages_see_the_boundary_at_their_own_times(oracle):
    """A step from t equals the step composed by hand from residuals at t, t + dt and
    t + dt/2 (with the sigma feedback); choosing t so that the shock passes a ghost centre
    between t + dt/2 and t + dt makes a wrong stage time visible."""
    pb, W = dmr(48, 5)
    sx, sy = oracle.prime_sigma(pb, W)
    dt = oracle.cfl_dt(pb, W)
    i = 25
    t = (xc(pb, i) - pb.shock_x0) / pb.shock_speed - 0.75 * dt
    W1s, sx1, sy1, dt_used = oracle.step(pb, W, sx, sy, dt, t=t)
    assert dt_used == dt

    def manual(times):
        L1, sa, sb, *_ = oracle.residual(pb, W, sx, sy, t=times[0])
        W1 = W + dt * L1
        L2, sc, sd, *_ = oracle.residual(pb, W1, sa, sb, t=times[1])
        W2 = 0.75 * W + 0.25 * W1 + 0.25 * dt * L2
        L3, se, sf, *_ = oracle.residual(pb, W2, sc, sd, t=times[2])
        return 1.0 / 3.0 * W + 2.0 / 3.0 * W2 + 2.0 / 3.0 * dt * L3, se, sf

    Wm, sxm, sym = manual((t, t + dt, t + 0.5 * dt))
    scale = np.abs(W).max()
    assert np.abs(W1s - Wm).max() <= 1e-13 * scale
    np.testing.assert_allclose(sx1, sxm, rtol=1e-13, atol=1e-14)
    Wx, _, _ = manual((t, t + dt, t + dt))  # stage 3 at the wrong time
    assert np.abs(Wx - Wm).max() > 1e-6 * scale


def test_top_boundary_moves_with_the_exact_shock(oracle):
    """With the Rankine-Hugoniot post-shock state of a Mach 10 shock in the gas at rest
    (rho 8, speed 8.25 at -30 degrees, p 116.5) the shock in the top rows stays within a
    cell of x = 1/6 + (y + 20 t) / sqrt(3)."""
    post = (8.0, 8.25 * np.cos(np.pi / 6), -8.25 * np.sin(np.pi / 6), 116.5)
    pb, W0 = P.double_mach_reflection(128, 5, post=post)
    W, _, _, t, _ = oracle.run(pb, W0, t_end=0.06)
    xs = xc(pb, np.arange(pb.nx))
    for j in range(pb.ny - 4, pb.ny):
        y = pb.y0 + (j + 0.5) * pb.dy
        rho = W[0, j]
        k = int(np.argmax(rho < 0.5 * (1.4 + 8.0)))
        # linear interpolation of the midpoint crossing
        x_num = xs[k - 1] + (rho[k - 1] - 4.7) / (rho[k - 1] - rho[k]) * pb.dx
        assert abs(x_num - (1.0 / 6.0 + (y + 20.0 * t) / S3)) <= pb.dx
