"""Checkpoint / resume and failure reporting on the GPU.

* A run saved after k steps and resumed in a fresh context continues bit for bit (the path
  has no floating-point atomics, so it is deterministic).
* A non-finite cell average planted on the host is reported by the device status word
  (ASE_DF_FLAG_NONPHYSICAL) after the next step, on both flux solvers, and the context stays
  usable; a bad configuration is refused before any device work.
"""
import os
import tempfile

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


@pytest.mark.parametrize("gks", [False, True])
def test_checkpoint_resume_is_bit_identical(A, gks):
    import torch

    pb, W0 = P.riemann_2d(48, 7, seed=2)
    s = A.Solver(pb, W0)
    for _ in range(20):
        s.gks_step() if gks else s.step()
    ref = s.W.cpu().numpy().copy()
    ref_t = s.status()[2]
    s.close()
    s = A.Solver(pb, W0)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ckpt.npz")
        for _ in range(8):
            s.gks_step() if gks else s.step()
        s.save(path)
        s.close()
        s = A.Solver(pb)
        s.load(path)
    for _ in range(12):
        s.gks_step() if gks else s.step()
    torch.cuda.synchronize()
    assert np.array_equal(s.W.cpu().numpy(), ref)
    assert s.status()[2] == ref_t
    s.close()


@pytest.mark.parametrize("gks", [False, True])
def test_nonfinite_cell_is_reported(A, gks):
    pb, W0 = P.isentropic_vortex(32, 5)
    s = A.Solver(pb, W0)
    try:
        s.step()
        flags, _, _ = s.status()
        assert flags & A.FLAG_NONPHYSICAL == 0
        W = s.W.cpu().numpy()
        W[0, 16, 16] = np.nan
        s.W.copy_(__import__("torch").as_tensor(W))
        s.gks_step() if gks else s.step()
        flags, _, _ = s.status()
        assert flags & A.FLAG_NONPHYSICAL
        with pytest.raises(A.AseDfError) as ei:
            A._check(s.ctx, A._load().ase_df_get_status(s.ctx, None, None, None))
        assert ei.value.status == 4
        # the context stays usable: a fresh state steps cleanly after a reset
        s.set_state(W0)
        s.step()
        assert s.status()[0] & A.FLAG_NONPHYSICAL == 0
    finally:
        s.close()


def test_bad_configuration_is_refused(A):
    with pytest.raises(A.AseDfError) as ei:
        A.Solver(P.Problem(ndim=2, nx=3, ny=8, order=9, bc=("reflect", "reflect", "outflow", "outflow")))
    assert ei.value.status == 1


def test_bounded_wait_runs_out_and_reports_timeout(A):
    """Failure detection without a GPU fault: a grid barrier that can never complete (it waits
    for one CTA more than its grid has) gives up after its poll limit, raises FLAG_SYNC and
    returns. ase_df_get_status then reports ASE_DF_E_TIMEOUT and the context stays usable: after
    a reset, steps whose positivity repair runs its passes through the same barrier complete
    without the flag, as before."""
    import time

    import torch
    from test_oracle_scheme import near_vacuum_1d

    pb, W0 = near_vacuum_1d()
    s = A.Solver(pb, W0)
    try:
        t0 = time.perf_counter()
        A.ase_df_selftest_wait(s.ctx)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        flags, _, _ = s.status()
        assert flags & A.FLAG_SYNC
        assert A._load().ase_df_get_status(s.ctx, None, None, None) == 5  # ASE_DF_E_TIMEOUT
        assert waited < 30.0, waited
        s.set_state(W0)  # ase_df_reset: clears the status word and the barrier's counters
        for _ in range(30):
            s.step()
        flags, _, _ = s.status()
        assert not flags & (A.FLAG_SYNC | A.FLAG_NONPHYSICAL), flags
        _, repaired, _ = A.ase_df_get_repair_stats(s.ctx)
        assert repaired > 0  # the repair's passes ran through the barrier
    finally:
        s.close()
