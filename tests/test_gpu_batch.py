"""Batched solves (one persistent launch per sweep direction over many problems of mixed
dimension and order): same results as the one-problem path and as the oracle."""
import numpy as np
import pytest

from parity_report import check
from paper_2410_05489_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_05489_gb300 import build

    build.build()
    from paper_2410_05489_gb300 import ase_df, batch

    return ase_df, batch


def mixed_set():
    out = [P.riemann_1d(300, 3, 1), P.riemann_1d(517, 9, 2), P.sod(200, 5), P.riemann_2d(40, 7, 3, ny=33),
           P.riemann_2d(37, 5, 4), P.isentropic_vortex(48, 9), P.high_mach_jet(64, 32, 9),
           P.riemann_2d(20, 3, 5, ny=50), P.riemann_1d(129, 7, 6)]
    pb, W = P.sin_wave_2d(24, 9)
    out.append((pb, W))
    # reflecting walls: the 1D blast wave and a 2D Riemann problem in a closed box
    out.append(P.blast_wave(160, 5))
    pb, W = P.riemann_2d(26, 9, 8, ny=21)
    out.append((pb.replace(bc=("reflect",) * 4), W))
    return out


def comp_err(a, b):
    return max(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300) for c in range(b.shape[0]))


def test_batch_matches_one_problem_path(B):
    A, Bt = B
    probs = mixed_set()
    bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
    try:
        for i, (pb, W) in enumerate(probs):  # primed sigma
            s = A.Solver(pb, W)
            sx, sy = bt.sigma(i)
            assert np.array_equal(sx, s.sx.cpu().numpy())
            if pb.ndim == 2:
                assert np.array_equal(sy, s.sy.cpu().numpy())
            s.close()
        bt.run(3)
        flags, t, dt = bt.status()
        for i, (pb, W) in enumerate(probs):
            s = A.Solver(pb, W)
            for _ in range(3):
                s.step()
            f1, dt1, t1 = s.status()
            assert abs(t[i] - t1) <= 1e-15 * t1 and flags[i] == f1
            check("W vs single", comp_err(bt.state(i), s.W.cpu().numpy()), 1e-13, i)
            s.close()
    finally:
        bt.close()


def test_batch_matches_oracle(B, oracle):
    A, Bt = B
    probs = [P.riemann_1d(200, 9, 11), P.riemann_2d(30, 7, 12), P.isentropic_vortex(32, 5)]
    bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
    try:
        for _ in range(5):
            bt.step()
        flags, t, _ = bt.status()
        for i, (pb, W) in enumerate(probs):
            Wc, _, _, tc, _ = oracle.run(pb, W, nsteps=5)
            assert abs(t[i] - tc) <= 1e-12 * tc
            check("W vs oracle", comp_err(bt.state(i), Wc), 1e-9, i)
    finally:
        bt.close()


def test_schedules_do_not_change_results(B):
    """Schedules and 2D tile shapes (8 x 64 or 8 x 32 faces per tile, per order) change the
    work assignment only: the results are the same bit for bit."""
    A, Bt = B
    probs = mixed_set()
    ref = None
    for sched, tiles in (((2, True, 4096), (64, 64, 64, 64)), ((1, False, 65536), (32, 32, 32, 32)),
                         ((2, False, 256), (32, 64, 32, 64))):
        bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
        try:
            bt.set_schedule(*sched)
            bt.set_tiles(tiles)
            for _ in range(2):
                bt.step()
            got = bt.W.cpu().numpy()
            if ref is None:
                ref = got
            else:
                assert np.array_equal(got, ref)
        finally:
            bt.close()


def test_autotune_restores_state_and_caches(B, tmp_path):
    A, Bt = B
    probs = mixed_set()
    bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
    try:
        W0 = bt.W.clone()
        cache = str(tmp_path / "sched.json")
        entry = Bt.autotune(bt, steps=1, cache=cache, candidates=[(2, True, 16384), (1, True, 4096)])
        assert len(entry["ms_per_step"]) == 2
        assert len(entry["tiles_ms_per_step"]) == 4  # orders 3, 5, 7, 9 all have 2D problems here
        assert all(v in (32, 64) for v in entry["tiles"])
        assert bool((bt.W == W0).all())
        again = Bt.autotune(bt, steps=1, cache=cache)
        assert again["schedule"] == entry["schedule"] and again["tiles"] == entry["tiles"]
    finally:
        bt.close()


def test_full_batched_workload_sampled_problems(B, oracle):
    """The batched workload at its full size (512 problems, 18.0 M cells), as the benchmark
    runs it (graph replays): the smallest 1D and 2D problems against the oracle (1e-9, the
    step tolerance of the parity tests) and a spread of the others, the largest included,
    against the one-problem path (1e-13)."""
    A, Bt = B
    probs = P.batched_problems()
    bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
    try:
        bt.set_schedule(2, True, 4096)
        bt.run(2)
        flags, t, _ = bt.status()
        assert not np.any(flags & 1)
        size = np.array([p.ncells for p, _ in probs])
        one_d = [i for i, (p, _) in enumerate(probs) if p.ndim == 1]
        two_d = [i for i, (p, _) in enumerate(probs) if p.ndim == 2]
        small = sorted(one_d, key=lambda i: size[i])[:3] + sorted(two_d, key=lambda i: size[i])[:2]
        for i in small:
            pb, W = probs[i]
            Wc, _, _, tc, _ = oracle.run(pb, W, nsteps=2)
            assert abs(t[i] - tc) <= 1e-12 * tc
            check("W vs oracle", comp_err(bt.state(i), Wc), 1e-9, i)
        rng = np.random.default_rng(5)
        spread = list(rng.choice(len(probs), 6, replace=False)) + [int(np.argmax(size))]
        for i in spread:
            pb, W = probs[i]
            s = A.Solver(pb, W)
            for _ in range(2):
                s.step()
            check("W vs single", comp_err(bt.state(i), s.W.cpu().numpy()), 1e-13, i)
            s.close()
    finally:
        bt.close()
