"""The plain oracle's optional host threads (one block of lines per thread in the face
loops) give the serial results bit for bit: every face is computed by the same code from
the same inputs whatever the split."""
import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P


@pytest.mark.parametrize("ndim,r", [(1, 9), (2, 3), (2, 5), (2, 9)])
def test_threaded_residual_and_steps_equal_serial(oracle, ndim, r):
    pb = P.Problem(ndim=ndim, nx=37, ny=23, order=r, bc=("outflow", "outflow", "periodic", "periodic"))
    W = P.white_noise(pb, 40 + r)
    sx, sy = P.random_sigma(pb, 41 + r, 1.0)
    ref = oracle.residual(pb, W, sx, sy)
    ref_steps = oracle.run(pb, W, nsteps=3)
    for n in (2, 5, 64):
        with oracle.threads(n):
            got = oracle.residual(pb, W, sx, sy)
            got_steps = oracle.run(pb, W, nsteps=3)
        for a, b in zip(got, ref):
            if a is not None:
                np.testing.assert_array_equal(a, b)
        for a, b in zip(got_steps[:3], ref_steps[:3]):
            np.testing.assert_array_equal(a, b)
        assert got_steps[3] == ref_steps[3]
    assert oracle.set_threads(1) == 1  # the context manager restored the default
