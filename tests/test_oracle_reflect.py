"""Pins of the reflecting-wall boundary (ghost cells mirrored about the wall face with the
normal momentum negated): a reflecting domain gives the same residual as the matching half of
the mirror-symmetric periodic domain twice its size, and mass and energy are conserved
exactly while momentum changes only by the wall pressure."""
import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P


def mirror_1d(W):
    """[0,1] -> [-1,1]: W(-x) = W(x) with the momentum negated."""
    M = W[:, :, ::-1].copy()
    M[1] *= -1.0
    return np.concatenate([M, W], axis=2)


@pytest.mark.parametrize("r", [5, 9])
def test_reflecting_1d_equals_mirrored_periodic(oracle, r):
    n = 24
    pb = P.Problem(ndim=1, nx=n, order=r, bc=("reflect", "reflect", "outflow", "outflow"))
    W = P.white_noise(pb, 3)
    # the doubled periodic domain [-1, 1] (so the mirror of x-hi wraps onto x-lo too)
    pb2 = P.Problem(ndim=1, nx=2 * n, x0=-1.0, x1=1.0, order=r, bc=("periodic",) * 4)
    W2 = mirror_1d(W)
    L, sxo, _, _, _, _ = oracle.residual(pb, W, *P.zero_sigma(pb))
    L2, sxo2, _, _, _, _ = oracle.residual(pb2, W2, *P.zero_sigma(pb2))
    np.testing.assert_allclose(L, L2[:, :, n:], rtol=1e-13, atol=1e-13 * np.abs(L).max())
    np.testing.assert_allclose(sxo, sxo2[:, n:], rtol=1e-13, atol=1e-14)


def test_reflecting_2d_x_walls_equal_mirrored_periodic(oracle):
    n, m = 18, 14
    pb = P.Problem(ndim=2, nx=n, ny=m, order=7, bc=("reflect", "reflect", "periodic", "periodic"))
    W = P.smooth_random(pb, 4)
    pb2 = P.Problem(ndim=2, nx=2 * n, ny=m, x0=-1.0, x1=1.0, order=7, bc=("periodic",) * 4)
    M = W[:, :, ::-1].copy()
    M[1] *= -1.0
    W2 = np.concatenate([M, W], axis=2)
    L, _, _, _, _, _ = oracle.residual(pb, W, *P.zero_sigma(pb))
    L2, _, _, _, _, _ = oracle.residual(pb2, W2, *P.zero_sigma(pb2))
    np.testing.assert_allclose(L, L2[:, :, n:], rtol=1e-12, atol=1e-12 * np.abs(L).max())


def test_walls_conserve_mass_and_energy(oracle):
    pb = P.Problem(ndim=2, nx=16, ny=12, order=9, bc=("reflect",) * 4)
    W = P.white_noise(pb, 5)
    sx, sy = P.random_sigma(pb, 6, pb.sigma_thres / 2)
    L, *_ = oracle.residual(pb, W, sx, sy)
    for c in (0, 3):
        assert abs(L[c].sum()) <= 1e-12 * np.abs(L[c]).sum()
    # the GKS path too
    Lg, Ltg, *_ = oracle.gks_residual(pb, W, sx, sy, 1e-4)
    for c in (0, 3):
        assert abs(Lg[c].sum()) <= 1e-11 * np.abs(Lg[c]).sum()
