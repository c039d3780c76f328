"""Pins of the oracle's reverse mode (the tape build) against central finite differences.

The residual's Jacobian is the derivative of the scheme as defined: linear branches
with constant weights, the WENO-Z weights of Sec. 3.2 (|.| taken piecewise), the DF
factor alpha = sigma_thres / A of Eq. (3.2) where A >= sigma_thres, the Lax-Friedrichs
flux of Sec. 2.3 (max taken piecewise) and sigma of Sec. 3.1.  Branch decisions are
piecewise constant in sigma_in, so a central difference of small step agrees with the
reverse mode to O(h^2) plus rounding."""
import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P


def _objective(oracle, pb, W, sx, sy, Lbar, sxb, syb):
    L, sxo, syo, _, _, hist = oracle.residual(pb, W, sx, sy)
    J = float(np.sum(Lbar * L) + np.sum(sxb * sxo))
    if pb.ndim == 2:
        J += float(np.sum(syb * syo))
    return J, hist


def _case(name):
    if name == "smooth2d_r9":
        pb, _ = P.isentropic_vortex(11, 9, ny=10)
        W = P.smooth_random(pb, 3)
        return pb, W, P.random_sigma(pb, 5, pb.sigma_thres / 2)
    if name == "smooth2d_r7_outflow":
        pb = P.Problem(ndim=2, nx=10, ny=12, order=7)
        W = P.smooth_random(pb, 4)
        return pb, W, P.random_sigma(pb, 6, pb.sigma_thres / 2)
    if name == "smooth2d_r5":
        pb, _ = P.isentropic_vortex(9, 5, ny=11)
        W = P.smooth_random(pb, 7)
        return pb, W, P.random_sigma(pb, 8, pb.sigma_thres / 2)
    if name == "noise1d_r9":
        pb = P.Problem(ndim=1, nx=23, order=9)
        W = P.white_noise(pb, 9)
        return pb, W, P.random_sigma(pb, 10, pb.sigma_thres / 2)
    if name == "smooth2d_r3":
        pb = P.Problem(ndim=2, nx=8, ny=7, order=3, bc=("periodic",) * 4)
        W = P.smooth_random(pb, 11)
        return pb, W, P.random_sigma(pb, 12, pb.sigma_thres)
    raise KeyError(name)


CASES = ["smooth2d_r9", "smooth2d_r7_outflow", "smooth2d_r5", "noise1d_r9", "smooth2d_r3"]


@pytest.mark.parametrize("name", CASES)
def test_residual_vjp_matches_central_differences(oracle, name):
    pb, W, (sx, sy) = _case(name)
    rng = np.random.default_rng(100)
    Lbar = rng.standard_normal(pb.state_shape)
    sxb = rng.standard_normal(pb.sx_shape)
    syb = rng.standard_normal(pb.sy_shape) if pb.ndim == 2 else np.zeros(pb.sy_shape)
    # faces whose Gauss points took the first-order states carry the constant 1e30
    _, sxo, syo, _, _, _ = oracle.residual(pb, W, sx, sy)
    sxb[sxo >= 1e29] = 0.0
    syb[syo >= 1e29] = 0.0
    Wbar, sxbar_in, sybar_in = oracle.residual_vjp(pb, W, sx, sy, Lbar, sxb, syb if pb.ndim == 2 else None)
    J0, hist = _objective(oracle, pb, W, sx, sy, Lbar, sxb, syb)
    # the case exercises more than the linear branches
    assert hist[oracle.BRANCHES.index("weno_df")] + hist[oracle.BRANCHES.index("df3")] > 0
    for k in range(3):
        dW = W * rng.uniform(-1.0, 1.0, W.shape)
        # WENO-Z weights vary on the scale of eps = 1e-6 in beta where the data is smooth,
        # so the central difference needs a step well below that
        h = 1e-7
        Jp, hp = _objective(oracle, pb, W + h * dW, sx, sy, Lbar, sxb, syb)
        Jm, hm = _objective(oracle, pb, W - h * dW, sx, sy, Lbar, sxb, syb)
        np.testing.assert_array_equal(hp[:5], hist[:5])
        fd = (Jp - Jm) / (2 * h)
        ad = float(np.sum(Wbar * dW))
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-8 * np.sum(np.abs(Wbar * dW)), (k, fd, ad)
    # sigma_in direction: only alpha = sigma_thres / A depends on it
    dsx = rng.uniform(0.0, 1.0, sx.shape) * sx
    dsy = rng.uniform(0.0, 1.0, sy.shape) * sy
    if "periodic" in pb.bc[:2]:
        dsx[:, -1] = dsx[:, 0]
    h = 1e-5
    Jp, hp = _objective(oracle, pb, W, sx + h * dsx, sy + h * dsy, Lbar, sxb, syb)
    Jm, hm = _objective(oracle, pb, W, sx - h * dsx, sy - h * dsy, Lbar, sxb, syb)
    np.testing.assert_array_equal(hp[:6], hist[:6])
    np.testing.assert_array_equal(hm[:6], hist[:6])
    fd = (Jp - Jm) / (2 * h)
    ad = float(np.sum(sxbar_in * dsx) + (np.sum(sybar_in * dsy) if pb.ndim == 2 else 0.0))
    assert ad != 0.0
    assert abs(fd - ad) <= 1e-6 * (abs(fd) + 1e-3 * np.sum(np.abs(sxbar_in * dsx))), (fd, ad)


def test_residual_vjp_smooth_data_has_no_sigma_gradient(oracle):
    """On the linear branches (every A < sigma_thres) alpha is the constant 1, so the
    gradient with respect to sigma_in vanishes identically."""
    pb, W = P.isentropic_vortex(12, 7)
    sx, sy = P.zero_sigma(pb)
    rng = np.random.default_rng(1)
    Lbar = rng.standard_normal(pb.state_shape)
    Wbar, sxb, syb = oracle.residual_vjp(pb, W, sx, sy, Lbar)
    assert np.all(sxb == 0.0) and np.all(syb == 0.0)
    assert np.all(np.isfinite(Wbar)) and np.abs(Wbar).max() > 0.0


def test_residual_vjp_is_linear_in_the_seed(oracle):
    """A VJP is linear in (Lbar, sigma_bar_out): the tape must give u^T J for u = a u1 + b u2."""
    pb, W, (sx, sy) = _case("smooth2d_r5")
    rng = np.random.default_rng(3)
    L1, L2 = rng.standard_normal((2,) + pb.state_shape)
    a, b = 0.75, -2.5
    W1, s1x, s1y = oracle.residual_vjp(pb, W, sx, sy, L1)
    W2, s2x, s2y = oracle.residual_vjp(pb, W, sx, sy, L2)
    W3, s3x, s3y = oracle.residual_vjp(pb, W, sx, sy, a * L1 + b * L2)
    np.testing.assert_allclose(W3, a * W1 + b * W2, rtol=1e-12, atol=1e-12 * np.abs(W3).max())
    np.testing.assert_allclose(s3x, a * s1x + b * s2x, rtol=1e-12, atol=1e-12 * (np.abs(s3x).max() + 1e-300))


@pytest.mark.parametrize("r", [7, 9])
def test_run_vjp_matches_central_differences(oracle, r):
    """Reverse mode through sigma^0 = prime(W^0) and 3 SSP-RK3 steps of fixed dt, with
    J = sum of the final density squared (the objective of the adjoint workload)."""
    pb, W0 = P.isentropic_vortex(12, r, ny=10)
    rng = np.random.default_rng(r)
    W0 = W0.copy()
    W0[0] *= 1.0 + 0.01 * rng.uniform(-1.0, 1.0, W0[0].shape)
    dt = 0.5 * oracle.cfl_dt(pb, W0)
    nsteps = 3

    def J(W):
        Wf = oracle.run(pb, W, nsteps=nsteps, dt=dt)[0]
        return float(np.sum(Wf[0] ** 2)), Wf

    J0, Wf = J(W0)
    Wbf = np.zeros_like(Wf)
    Wbf[0] = 2.0 * Wf[0]
    G = oracle.run_vjp(pb, W0, nsteps, dt, Wbf)
    for k in range(2):
        d = rng.standard_normal(W0.shape)
        d /= np.linalg.norm(d)
        h = 1e-6
        fd = (J(W0 + h * d)[0] - J(W0 - h * d)[0]) / (2 * h)
        ad = float(np.sum(G * d))
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-9, (k, fd, ad)


def test_kinks_take_the_symmetric_subgradient(oracle):
    """Reading G23.  On the Sod tube at t = 0 the velocity is exactly zero and the
    Gauss-point pressures of the constant regions agree to rounding, so |u| in the
    Lax-Friedrichs speed and |p_L - p_R| in sigma sit on their kinks; a central
    difference sees the symmetric subgradient (0) there, and so must the tape."""
    pb, W = P.sod(80, 5)
    sx, sy = oracle.prime_sigma(pb, W)
    rng = np.random.default_rng(7)
    Lbar = rng.standard_normal(pb.state_shape)
    _, sxo, _, _, _, _ = oracle.residual(pb, W, sx, sy)
    sxb = np.where(sxo < 1e29, rng.standard_normal(pb.sx_shape), 0.0)
    Wbar, _, _ = oracle.residual_vjp(pb, W, sx, sy, Lbar, sxb)
    for k in range(3):
        dW = W * rng.uniform(-1.0, 1.0, W.shape)
        h = 1e-7
        Jp, _ = _objective(oracle, pb, W + h * dW, sx, sy, Lbar, sxb, np.zeros(pb.sy_shape))
        Jm, _ = _objective(oracle, pb, W - h * dW, sx, sy, Lbar, sxb, np.zeros(pb.sy_shape))
        fd = (Jp - Jm) / (2 * h)
        ad = float(np.sum(Wbar * dW))
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-8 * np.sum(np.abs(Wbar * dW)), (k, fd, ad)
