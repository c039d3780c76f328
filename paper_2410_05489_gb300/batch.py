"""Batched solves through the C ABI (ase_df_batch_*) and the schedule autotuner.

Batch packs many independent problems (1D/2D, mixed orders) into three device arrays
and advances them together, one persistent launch per sweep direction and RK stage.
autotune() times the schedule candidates (persistent CTAs per SM, work ordering, chunk
size), then the tile shape of each 2D order present (8 x 64 faces, two per thread, or
8 x 32, one per thread), on a copy of the state and caches the fastest per device and batch
shape in ~/.cache/ase_df/batch_schedule.json.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import ase_df as A
from .problems import Problem

_c = ctypes
_VP = _c.c_void_p


def _setup():
    lib = A._load()
    if getattr(lib, "_batch_ready", False):
        return lib
    P = _c.POINTER(A.ase_df_params)
    I64 = _c.POINTER(_c.c_int64)
    sig = {
        "ase_df_batch_init": ([P, _c.c_int32, _c.POINTER(_VP)], _c.c_int),
        "ase_df_batch_destroy": ([_VP], None),
        "ase_df_batch_layout": ([_VP, I64, I64, I64], _c.c_int),
        "ase_df_batch_prime_sigma": ([_VP, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_batch_step": ([_VP, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_batch_run": ([_VP, _VP, _VP, _VP, _c.c_int32, _VP], _c.c_int),
        "ase_df_batch_get_status": ([_VP, _c.POINTER(_c.c_uint32), _c.POINTER(_c.c_double),
                                     _c.POINTER(_c.c_double)], _c.c_int),
        "ase_df_batch_set_schedule": ([_VP, _c.c_int32, _c.c_int32, _c.c_int32], _c.c_int),
        "ase_df_batch_set_tiles": ([_VP, _c.POINTER(_c.c_int32)], _c.c_int),
        "ase_df_batch_last_error": ([_VP], _c.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    lib._batch_ready = True
    return lib


def _check(b, st):
    if st != 0:
        msg = _setup().ase_df_batch_last_error(b)
        raise A.AseDfError(st, msg.decode() if msg else "")


def _ptr(t):
    return _c.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return _c.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------------
# C ABI, one function per entry point
# ----------------------------------------------------------------------------------
def ase_df_batch_init(params: Sequence[A.ase_df_params]):
    lib = _setup()
    arr = (A.ase_df_params * len(params))(*params)
    b = _VP()
    _check(None, lib.ase_df_batch_init(arr, len(params), _c.byref(b)))
    return b


def ase_df_batch_destroy(b) -> None:
    _setup().ase_df_batch_destroy(b)


def ase_df_batch_layout(b, n: int):
    w = (_c.c_int64 * (n + 1))()
    x = (_c.c_int64 * (n + 1))()
    y = (_c.c_int64 * (n + 1))()
    _check(b, _setup().ase_df_batch_layout(b, w, x, y))
    return list(w), list(x), list(y)


def ase_df_batch_prime_sigma(b, W, sx, sy, stream=None) -> None:
    _check(b, _setup().ase_df_batch_prime_sigma(b, _ptr(W), _ptr(sx), _ptr(sy), _stream(stream)))


def ase_df_batch_step(b, W, sx, sy, stream=None) -> None:
    _check(b, _setup().ase_df_batch_step(b, _ptr(W), _ptr(sx), _ptr(sy), _stream(stream)))


def ase_df_batch_run(b, W, sx, sy, nsteps: int, stream=None) -> None:
    _check(b, _setup().ase_df_batch_run(b, _ptr(W), _ptr(sx), _ptr(sy), int(nsteps), _stream(stream)))


def ase_df_batch_get_status(b, n: int):
    f = (_c.c_uint32 * n)()
    t = (_c.c_double * n)()
    dt = (_c.c_double * n)()
    st = _setup().ase_df_batch_get_status(b, f, t, dt)
    if st not in (0, 4):
        _check(b, st)
    return np.array(f, dtype=np.uint32), np.array(t), np.array(dt)


def ase_df_batch_set_schedule(b, ctas_per_sm: int, order_by_cost: bool, chunk_cells: int) -> None:
    _check(b, _setup().ase_df_batch_set_schedule(b, int(ctas_per_sm), int(bool(order_by_cost)), int(chunk_cells)))


def ase_df_batch_set_tiles(b, lines: Sequence[int]) -> None:
    """Lines of the 2D sweep tiles of orders 3, 5, 7, 9 (each 32 or 64)."""
    arr = (_c.c_int32 * 4)(*[int(v) for v in lines])
    _check(b, _setup().ase_df_batch_set_tiles(b, arr))


# ----------------------------------------------------------------------------------
# convenience wrapper
# ----------------------------------------------------------------------------------
class Batch:
    """Problems and their packed device state (W, sx, sy)."""

    def __init__(self, problems: Sequence[Problem], states: Sequence[np.ndarray] | None = None,
                 t_end: float = 0.0):
        if not torch.cuda.is_available():
            raise RuntimeError("the ASE-DF library needs a CUDA device")
        self.problems = list(problems)
        self.n = len(self.problems)
        self.b = ase_df_batch_init([A.params_from_problem(p, t_end) for p in self.problems])
        self.w_off, self.sx_off, self.sy_off = ase_df_batch_layout(self.b, self.n)
        dev = "cuda"
        self.W = torch.zeros(max(1, self.w_off[-1]), dtype=torch.float64, device=dev)
        self.sx = torch.zeros(max(1, self.sx_off[-1]), dtype=torch.float64, device=dev)
        self.sy = torch.zeros(max(1, self.sy_off[-1]), dtype=torch.float64, device=dev)
        if states is not None:
            self.set_states(states)

    @property
    def ncells(self) -> int:
        return sum(p.ncells for p in self.problems)

    def set_states(self, states: Sequence[np.ndarray], prime: bool = True) -> None:
        host = np.concatenate([np.ascontiguousarray(s, dtype=np.float64).ravel() for s in states])
        assert host.size == self.w_off[-1]
        self.W.copy_(torch.from_numpy(host))
        if prime:
            ase_df_batch_prime_sigma(self.b, self.W, self.sx, self.sy)

    def state(self, i: int) -> np.ndarray:
        pb = self.problems[i]
        return self.W[self.w_off[i]:self.w_off[i + 1]].cpu().numpy().reshape(pb.state_shape)

    def sigma(self, i: int):
        pb = self.problems[i]
        sx = self.sx[self.sx_off[i]:self.sx_off[i + 1]].cpu().numpy().reshape(pb.sx_shape)
        sy = (self.sy[self.sy_off[i]:self.sy_off[i + 1]].cpu().numpy().reshape(pb.sy_shape)
              if pb.ndim == 2 else np.zeros((1, 1)))
        return sx, sy

    def step(self) -> None:
        ase_df_batch_step(self.b, self.W, self.sx, self.sy)

    def run(self, nsteps: int) -> None:
        ase_df_batch_run(self.b, self.W, self.sx, self.sy, nsteps)

    def status(self):
        return ase_df_batch_get_status(self.b, self.n)

    def set_schedule(self, ctas_per_sm: int, order_by_cost: bool, chunk_cells: int) -> None:
        ase_df_batch_set_schedule(self.b, ctas_per_sm, order_by_cost, chunk_cells)

    def set_tiles(self, lines: Sequence[int]) -> None:
        ase_df_batch_set_tiles(self.b, lines)

    def close(self) -> None:
        if getattr(self, "b", None) is not None:
            ase_df_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CANDIDATES: List[Tuple[int, bool, int]] = [
    (c, o, k) for c in (2, 1) for o in (True, False) for k in (4096, 16384, 65536)
]


def _signature(batch: Batch) -> str:
    h = hashlib.sha1()
    for p in batch.problems:
        h.update(("%d:%d:%d:%d;" % (p.ndim, p.order, p.nx, p.nyc)).encode())
    return h.hexdigest()[:16]


def _time_steps(batch: Batch, saved, steps: int) -> float:
    batch.W.copy_(saved[0]); batch.sx.copy_(saved[1]); batch.sy.copy_(saved[2])
    batch.step()  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        batch.step()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def autotune(batch: Batch, steps: int = 2, cache: str | None = None, candidates=CANDIDATES):
    """Times each schedule on a copy of the batch state (the state is restored) and sets
    the fastest; then, per 2D order present, the tile shape (8 x 32 faces instead of 8 x 64
    where that is faster by more than 1 %).  The choice is cached per device name and batch
    signature."""
    cache = cache or os.path.join(os.path.expanduser("~"), ".cache", "ase_df", "batch_schedule.json")
    dev = torch.cuda.get_device_name()
    key = "%s|%s" % (dev, _signature(batch))
    table = {}
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table and "tiles" in table[key]:
        c, o, k = table[key]["schedule"]
        batch.set_schedule(c, o, k)
        batch.set_tiles(table[key]["tiles"])
        return table[key]
    saved = (batch.W.clone(), batch.sx.clone(), batch.sy.clone())
    tiles = [64, 64, 64, 64]
    batch.set_tiles(tiles)
    timings = {}
    for cand in candidates:
        batch.set_schedule(*cand)
        timings[str(cand)] = _time_steps(batch, saved, steps)
    best = min(candidates, key=lambda c: timings[str(c)])
    batch.set_schedule(*best)
    best_ms = timings[str(best)]
    tile_timings = {}
    for r in sorted({p.order for p in batch.problems if p.ndim == 2}):
        trial = list(tiles)
        trial[(r - 3) // 2] = 32
        batch.set_tiles(trial)
        ms = _time_steps(batch, saved, steps)
        tile_timings[str(trial)] = ms
        if ms < 0.99 * best_ms:
            tiles, best_ms = trial, ms
    batch.set_tiles(tiles)
    batch.W.copy_(saved[0]); batch.sx.copy_(saved[1]); batch.sy.copy_(saved[2])
    entry = {"schedule": list(best), "tiles": tiles, "ms_per_step": timings, "tiles_ms_per_step": tile_timings}
    table[key] = entry
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    except OSError:
        pass
    return entry
