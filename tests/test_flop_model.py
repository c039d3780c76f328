"""The roofline's flop model against the oracle's operation counter.

bench.py counts, per Gauss point, both sides' primitives, the Lax-Friedrichs flux
1/2 (F_L + F_R - lambda (q_R - q_L)) and sigma (Sec. 2.3, Sec. 3.1).  The oracle's op-counting
build performs the same steps but scales both halves of the flux by 1/2, one multiplication
per component more; its count of one point is data-independent on physical states."""
import numpy as np
import pytest

import bench
from oracle import oracle as O


def _count_point(C, qL, qR):
    import ctypes

    lib = O._lib(True)
    F = np.empty(C)
    s = np.empty(1)
    lib.oracle_reset_op_counts()
    fb = lib.oracle_lf_flux(C, 1.4, O._ptr(qL), O._ptr(qR), O._ptr(qL), O._ptr(qR), O._ptr(F), O._ptr(s))
    assert fb == 0  # physical states: no first-order fallback
    out = (ctypes.c_longlong * 4)()
    lib.oracle_op_counts(out)
    return sum(out)


@pytest.mark.parametrize("ndim", [1, 2])
def test_gauss_point_flops_are_the_oracles_count_less_one_half_per_component(ndim):
    C = 4 if ndim == 2 else 3
    rng = np.random.default_rng(7)
    counts = set()
    for _ in range(5):
        rho = rng.uniform(0.5, 2.0, 2)
        p = rng.uniform(0.5, 2.0, 2)
        u = rng.uniform(-1.0, 1.0, (2, C - 2))
        q = [np.concatenate(([rho[k]], rho[k] * u[k], [p[k] / 0.4 + 0.5 * rho[k] * np.sum(u[k] ** 2)]))
             for k in range(2)]
        counts.add(_count_point(C, q[0], q[1]))
    assert len(counts) == 1
    assert bench.GAUSS_POINT_FLOPS[ndim] == counts.pop() - C


def test_face_flops_of_the_roofline():
    # 2D, per face of one sweep: 2 C (2r-1) + 2 C G (2r-1) + G (70 + 2 C + 1) + 1
    assert [bench.algorithmic_flops_per_face(2, r) for r in (3, 5, 7, 9)] == [160, 375, 654, 997]


@pytest.mark.parametrize("r", [5, 7, 9])
def test_vjp_edges_per_operation_of_the_adjoint_model(r):
    """The residual adjoint's flop model scales the forward's algorithmic flops by
    1 + 2 e, e the edges per operation of the reverse-mode graph (one multiply-add per edge in
    the reverse sweep); e is the oracle tape's on smooth 2D data."""
    from paper_2410_05489_gb300 import problems as P

    pb = P.Problem(ndim=2, nx=32, ny=32, order=r, bc=("periodic",) * 4, x1=2.0, y1=2.0)
    W = P.smooth_random(pb, 3)
    sx, sy = P.zero_sigma(pb)
    O.residual_vjp(pb, W, sx, sy, np.random.default_rng(1).normal(size=W.shape))
    edges = O.last_vjp_edges()
    ops = sum(O.op_counts_residual(pb, W, sx, sy))
    assert abs(bench.VJP_EDGES_PER_OP[r] - edges / ops) < 1e-3 * bench.VJP_EDGES_PER_OP[r]
