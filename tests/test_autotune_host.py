"""Host logic of the batched-solve autotuner (batch.autotune) with a stand-in batch and
timer, no device: it takes the fastest of the 12 schedules, keeps the 8 x 32 tile for a 2D
order only where that is more than 1 % faster, restores the batch state, and caches the
choice per device name and batch signature (a second call times nothing)."""
import json

import torch

from paper_2410_05489_gb300 import batch as B
from paper_2410_05489_gb300.problems import Problem


class FakeBatch:
    def __init__(self, problems):
        self.problems = problems
        self.W = torch.arange(6, dtype=torch.float64)
        self.sx = torch.ones(3, dtype=torch.float64)
        self.sy = torch.zeros(2, dtype=torch.float64)
        self.schedule = None
        self.tiles = None

    def set_schedule(self, c, o, k):
        self.schedule = (c, o, k)

    def set_tiles(self, tiles):
        self.tiles = list(tiles)


def _fake_timer(ms_of):
    calls = []

    def timer(batch, saved, steps):
        batch.W.copy_(saved[0])
        batch.W += 1.0  # a "step" changes the state; autotune must restore it
        calls.append((batch.schedule, tuple(batch.tiles)))
        return ms_of(batch.schedule, batch.tiles)

    return timer, calls


def test_autotune_picks_the_fastest_schedule_and_tiles_and_caches(tmp_path, monkeypatch):
    problems = [Problem(ndim=1, nx=300, order=9), Problem(ndim=2, nx=64, ny=64, order=5),
                Problem(ndim=2, nx=96, ny=80, order=9)]
    fb = FakeBatch(problems)
    W0 = fb.W.clone()
    best_schedule = (1, False, 16384)

    def ms_of(schedule, tiles):
        ms = 10.0 if schedule == best_schedule else 12.0 + 0.1 * schedule[0] + schedule[2] / 1e5
        # order 5 gains 2 % from the 8 x 32 tile (kept), order 9 gains 0.5 % (refused); order 7
        # is absent from the batch and must not be tried
        if tiles[1] == 32:
            ms *= 0.98
        if tiles[3] == 32:
            ms *= 0.995
        assert tiles[0] == 64 and tiles[2] == 64
        return ms

    timer, calls = _fake_timer(ms_of)
    monkeypatch.setattr(B, "_time_steps", timer)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "Fake GPU")
    cache = str(tmp_path / "sched.json")

    entry = B.autotune(fb, cache=cache)
    assert tuple(entry["schedule"]) == best_schedule and fb.schedule == best_schedule
    assert entry["tiles"] == [64, 32, 64, 64] and fb.tiles == [64, 32, 64, 64]
    assert len(calls) == len(B.CANDIDATES) + 2  # every schedule, then one trial per 2D order present
    assert {c[0] for c in calls[:len(B.CANDIDATES)]} == set(B.CANDIDATES)
    assert calls[-2][1] == (64, 32, 64, 64) and calls[-1][1] == (64, 32, 64, 32)
    assert torch.equal(fb.W, W0)  # state restored
    with open(cache) as f:
        table = json.load(f)
    (key,) = table
    assert key.startswith("Fake GPU|")

    # cached: a fresh batch of the same problems gets the choice without any timing
    fb2 = FakeBatch(problems)
    n_before = len(calls)
    entry2 = B.autotune(fb2, cache=cache)
    assert len(calls) == n_before
    assert fb2.schedule == best_schedule and fb2.tiles == [64, 32, 64, 64]
    assert entry2["tiles"] == entry["tiles"]

    # another batch signature is tuned afresh
    fb3 = FakeBatch(problems[:2])
    B.autotune(fb3, cache=cache)
    assert len(calls) == n_before + len(B.CANDIDATES) + 1
