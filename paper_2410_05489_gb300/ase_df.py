"""Thin Python binding of the C ABI in include/ase_df.h (ctypes, argument marshalling only).

Every function of the C ABI has a function of the same name here taking torch CUDA
tensors (FP64, contiguous) and an optional torch stream; all computation runs in the
library's CUDA kernels.  Importing this module loads libasedf.so and fails loudly when it
is missing or no CUDA device is present: there is no CPU fallback.

The Solver class bundles a context with its problem and device tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import torch

from .problems import Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libasedf.so")

ASE_DF_OK = 0
STATUS_NAMES = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_NONPHYSICAL", 5: "E_TIMEOUT", 6: "E_BOUNDS"}
FLAG_NONPHYSICAL = 0x1
FLAG_POSITIVITY = 0x2
FLAG_DT = 0x4
FLAG_FROZEN = 0x8
FLAG_SYNC = 0x10


class AseDfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ase_df_params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("order", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("sigma_thres", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("inflow_state", ctypes.c_double * 4),
        ("inflow_lo", ctypes.c_double), ("inflow_hi", ctypes.c_double),
        ("t_end", ctypes.c_double),
        ("gks_c1", ctypes.c_double), ("gks_c2", ctypes.c_double),
        ("state_b", ctypes.c_double * 4), ("wall_x", ctypes.c_double),
        ("shock_x0", ctypes.c_double), ("shock_speed", ctypes.c_double),
    ]


_c = ctypes
_VP = _c.c_void_p
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libasedf.so is not built (%s); run paper_2410_05489_gb300.build.build()" % LIB_PATH)
    lib = _c.CDLL(LIB_PATH)
    P = _c.POINTER(ase_df_params)
    CTX = _c.c_void_p
    sig = {
        "ase_df_init": ([P, _c.POINTER(CTX)], _c.c_int),
        "ase_df_destroy": ([CTX], None),
        "ase_df_prime_sigma": ([CTX, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_residual": ([CTX, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_copy_face_fluxes": ([CTX, _VP, _VP, _VP], _c.c_int),
        "ase_df_step": ([CTX, _VP, _VP, _VP, _c.c_double, _VP], _c.c_int),
        "ase_df_run": ([CTX, _VP, _VP, _VP, _c.c_double, _c.c_int32, _VP], _c.c_int),
        "ase_df_residual_adjoint": ([CTX, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_step_adjoint": ([CTX, _VP, _VP, _VP, _c.c_double, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_gks_residual": ([CTX, _VP, _VP, _VP, _c.c_double, _VP, _VP, _VP, _VP, _VP], _c.c_int),
        "ase_df_gks_step": ([CTX, _VP, _VP, _VP, _c.c_double, _VP], _c.c_int),
        "ase_df_get_status": ([CTX, _c.POINTER(_c.c_uint32), _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)], _c.c_int),
        "ase_df_reset": ([CTX, _c.c_double, _VP], _c.c_int),
        "ase_df_selftest_wait": ([CTX, _VP], _c.c_int),
        "ase_df_get_repair_stats": ([CTX, _c.POINTER(_c.c_uint32), _c.POINTER(_c.c_uint64),
                                     _c.POINTER(_c.c_uint64)], _c.c_int),
        "ase_df_last_error": ([CTX], _c.c_char_p),
        "ase_df_fp64_fma_rate": ([_c.POINTER(_c.c_double)], _c.c_int),
        "ase_df_check_recip": ([_VP, _VP, _c.c_int64, _VP], _c.c_int),
        "ase_df_profile_enable": ([CTX, _c.c_int32], _c.c_int),
        "ase_df_profile_read": ([CTX, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int64)], _c.c_int),
        "ase_df_hist_enable": ([CTX, _c.c_int32], _c.c_int),
        "ase_df_hist_read": ([CTX, _c.POINTER(_c.c_uint64)], _c.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def params_from_problem(pb: Problem, t_end: float = 0.0) -> ase_df_params:
    p = ase_df_params()
    p.ndim, p.order = pb.ndim, pb.order
    p.nx, p.ny = pb.nx, pb.nyc
    p.x0, p.x1, p.y0, p.y1 = pb.x0, pb.x1, pb.y0, pb.y1
    p.gamma, p.sigma_thres, p.cfl = pb.gamma, pb.sigma_thres, pb.cfl
    for i, c in enumerate(pb.bc_codes()):
        p.bc[i] = c
    for i in range(4):
        p.inflow_state[i] = pb.inflow[i]
    p.inflow_lo, p.inflow_hi = pb.inflow_lo, pb.inflow_hi
    p.t_end = t_end
    p.gks_c1, p.gks_c2 = pb.gks_c1, pb.gks_c2
    for i in range(4):
        p.state_b[i] = pb.state_b[i]
    p.wall_x, p.shock_x0, p.shock_speed = pb.wall_x, pb.shock_x0, pb.shock_speed
    return p


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return _c.c_void_p(t.data_ptr())


def _stream(stream) -> _c.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return _c.c_void_p(s.cuda_stream)


def _check(ctx, status: int):
    if status != ASE_DF_OK:
        msg = _load().ase_df_last_error(ctx)
        raise AseDfError(status, msg.decode() if msg else "")


# ----------------------------------------------------------------------------------
# the C ABI, one function per entry point
# ----------------------------------------------------------------------------------
def ase_df_init(params: ase_df_params):
    lib = _load()
    ctx = _c.c_void_p()
    st = lib.ase_df_init(_c.byref(params), _c.byref(ctx))
    _check(None, st)
    return ctx


def ase_df_destroy(ctx) -> None:
    _load().ase_df_destroy(ctx)


def ase_df_prime_sigma(ctx, W, sx, sy, stream=None) -> None:
    _check(ctx, _load().ase_df_prime_sigma(ctx, _ptr(W), _ptr(sx), _ptr(sy), _stream(stream)))


def ase_df_residual(ctx, W, sx_in, sy_in, L, sx_out, sy_out, stream=None) -> None:
    _check(ctx, _load().ase_df_residual(ctx, _ptr(W), _ptr(sx_in), _ptr(sy_in), _ptr(L), _ptr(sx_out),
                                        _ptr(sy_out), _stream(stream)))


def ase_df_copy_face_fluxes(ctx, Fx, Fy, stream=None) -> None:
    _check(ctx, _load().ase_df_copy_face_fluxes(ctx, _ptr(Fx), _ptr(Fy), _stream(stream)))


def ase_df_step(ctx, W, sx, sy, dt: float = 0.0, stream=None) -> None:
    _check(ctx, _load().ase_df_step(ctx, _ptr(W), _ptr(sx), _ptr(sy), float(dt), _stream(stream)))


def ase_df_run(ctx, W, sx, sy, dt: float, nsteps: int, stream=None) -> None:
    _check(ctx, _load().ase_df_run(ctx, _ptr(W), _ptr(sx), _ptr(sy), float(dt), int(nsteps), _stream(stream)))


def ase_df_residual_adjoint(ctx, W, sx_in, sy_in, Lbar, sxbar_out, sybar_out, Wbar, sxbar_in, sybar_in,
                            stream=None) -> None:
    _check(ctx, _load().ase_df_residual_adjoint(ctx, _ptr(W), _ptr(sx_in), _ptr(sy_in), _ptr(Lbar), _ptr(sxbar_out),
                                                _ptr(sybar_out), _ptr(Wbar), _ptr(sxbar_in), _ptr(sybar_in),
                                                _stream(stream)))


def ase_df_step_adjoint(ctx, W, sx, sy, dt: float, Wbar, sxbar, sybar, stream=None) -> None:
    _check(ctx, _load().ase_df_step_adjoint(ctx, _ptr(W), _ptr(sx), _ptr(sy), float(dt), _ptr(Wbar), _ptr(sxbar),
                                            _ptr(sybar), _stream(stream)))


def ase_df_gks_residual(ctx, W, sx_in, sy_in, dt: float, L, Lt, sx_out, sy_out, stream=None) -> None:
    _check(ctx, _load().ase_df_gks_residual(ctx, _ptr(W), _ptr(sx_in), _ptr(sy_in), float(dt), _ptr(L), _ptr(Lt),
                                            _ptr(sx_out), _ptr(sy_out), _stream(stream)))


def ase_df_gks_step(ctx, W, sx, sy, dt: float = 0.0, stream=None) -> None:
    _check(ctx, _load().ase_df_gks_step(ctx, _ptr(W), _ptr(sx), _ptr(sy), float(dt), _stream(stream)))


def ase_df_get_status(ctx) -> Tuple[int, float, float]:
    flags = _c.c_uint32()
    dt = _c.c_double()
    t = _c.c_double()
    st = _load().ase_df_get_status(ctx, _c.byref(flags), _c.byref(dt), _c.byref(t))
    if st not in (ASE_DF_OK, 4, 5):  # non-physical and timeout are reported through the flags
        _check(ctx, st)
    return int(flags.value), float(dt.value), float(t.value)


def ase_df_selftest_wait(ctx, stream=None) -> None:
    """A device wait that runs out (about a second): raises FLAG_SYNC in the status word."""
    _check(ctx, _load().ase_df_selftest_wait(ctx, _stream(stream)))


def ase_df_get_repair_stats(ctx):
    """-> (last_stage counts [18], cells marked since the last reset, cells frozen)."""
    arr = (_c.c_uint32 * 18)()
    tot = _c.c_uint64()
    frz = _c.c_uint64()
    _check(ctx, _load().ase_df_get_repair_stats(ctx, arr, _c.byref(tot), _c.byref(frz)))
    return list(arr), int(tot.value), int(frz.value)


def ase_df_reset(ctx, t: float = 0.0, stream=None) -> None:
    _check(ctx, _load().ase_df_reset(ctx, float(t), _stream(stream)))


def ase_df_last_error(ctx) -> str:
    m = _load().ase_df_last_error(ctx)
    return m.decode() if m else ""


def ase_df_profile_enable(ctx, enable: bool) -> None:
    _check(ctx, _load().ase_df_profile_enable(ctx, int(bool(enable))))


def ase_df_profile_read(ctx):
    """-> (ms[5], n[5]) per kernel kind: x-sweep, y-sweep, combine, wave-speed, repair."""
    ms = (_c.c_double * 5)()
    n = (_c.c_int64 * 5)()
    _check(ctx, _load().ase_df_profile_read(ctx, ms, n))
    return list(ms), list(n)


BRANCH_SLOTS = ("lin9", "lin7", "lin5", "weno_df", "lin3", "df3", "first_order")


def ase_df_hist_enable(ctx, enable: bool) -> None:
    _check(ctx, _load().ase_df_hist_enable(ctx, int(bool(enable))))


def ase_df_hist_read(ctx):
    """-> branch counts since the last read, in BRANCH_SLOTS order (then cleared)."""
    arr = (_c.c_uint64 * 7)()
    _check(ctx, _load().ase_df_hist_read(ctx, arr))
    return list(arr)


def ase_df_check_recip(x, out, stream=None) -> None:
    _check(None, _load().ase_df_check_recip(_ptr(x), _ptr(out), int(x.numel()), _stream(stream)))


def ase_df_fp64_fma_rate() -> float:
    r = _c.c_double()
    _check(None, _load().ase_df_fp64_fma_rate(_c.byref(r)))
    return float(r.value)


# ----------------------------------------------------------------------------------
# convenience wrapper
# ----------------------------------------------------------------------------------
class Solver:
    """A context plus the device state of one problem.

    W, sx, sy are FP64 CUDA tensors of shapes pb.state_shape, pb.sx_shape, pb.sy_shape.
    """

    def __init__(self, pb: Problem, W0=None, t_end: float = 0.0, device: str = "cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("the ASE-DF library needs a CUDA device")
        self.pb = pb
        self.device = torch.device(device)
        self.ctx = ase_df_init(params_from_problem(pb, t_end))
        self.W = torch.zeros(pb.state_shape, dtype=torch.float64, device=self.device)
        self.sx = torch.zeros(pb.sx_shape, dtype=torch.float64, device=self.device)
        self.sy = torch.zeros(pb.sy_shape, dtype=torch.float64, device=self.device)
        if W0 is not None:
            self.set_state(W0)

    def _sy(self, t):
        return t if self.pb.ndim == 2 else None

    def set_state(self, W0, prime: bool = True) -> None:
        self.W.copy_(torch.as_tensor(W0, dtype=torch.float64))
        if prime:
            self.prime()
        ase_df_reset(self.ctx, 0.0)

    def set_time(self, t: float) -> None:
        """Sets the device time t (and clears the status word); time-dependent boundaries
        are evaluated at it."""
        ase_df_reset(self.ctx, t)

    def prime(self) -> None:
        ase_df_prime_sigma(self.ctx, self.W, self.sx, self._sy(self.sy))

    def residual(self, W=None, sx=None, sy=None):
        W = self.W if W is None else W
        sx = self.sx if sx is None else sx
        sy = self.sy if sy is None else sy
        L = torch.empty_like(W)
        sxo = torch.empty_like(sx)
        syo = torch.empty_like(sy)
        ase_df_residual(self.ctx, W, sx, self._sy(sy), L, sxo, self._sy(syo))
        return L, sxo, syo

    def residual_adjoint(self, W, sx, sy, Lbar=None, sxbar_out=None, sybar_out=None, Wbar=None, sxbar_in=None,
                         sybar_in=None):
        """Accumulates the residual's vector-Jacobian product into Wbar, sxbar_in, sybar_in
        (zero tensors are made for the ones not given) and returns them."""
        Wbar = torch.zeros_like(W) if Wbar is None else Wbar
        sxbar_in = torch.zeros_like(sx) if sxbar_in is None else sxbar_in
        sybar_in = torch.zeros_like(sy) if sybar_in is None else sybar_in
        ase_df_residual_adjoint(self.ctx, W, sx, self._sy(sy), Lbar, sxbar_out, self._sy(sybar_out), Wbar, sxbar_in,
                                self._sy(sybar_in))
        return Wbar, sxbar_in, sybar_in

    def step_adjoint(self, W, sx, sy, dt: float, Wbar, sxbar, sybar) -> None:
        """In place: (Wbar, sxbar, sybar) from the adjoint of W^{n+1}, sigma^{n+1} to that
        of W^n, sigma^n for the step of fixed dt from (W, sx, sy)."""
        ase_df_step_adjoint(self.ctx, W, sx, self._sy(sy), dt, Wbar, sxbar, self._sy(sybar))

    def gks_residual(self, dt: float, W=None, sx=None, sy=None):
        """Gas-kinetic L and L_t for step size dt: -> (L, Lt, sx_out, sy_out)."""
        W = self.W if W is None else W
        sx = self.sx if sx is None else sx
        sy = self.sy if sy is None else sy
        L = torch.empty_like(W)
        Lt = torch.empty_like(W)
        sxo = torch.empty_like(sx)
        syo = torch.empty_like(sy)
        ase_df_gks_residual(self.ctx, W, sx, self._sy(sy), dt, L, Lt, sxo, self._sy(syo))
        return L, Lt, sxo, syo

    def gks_step(self, dt: float = 0.0) -> None:
        ase_df_gks_step(self.ctx, self.W, self.sx, self._sy(self.sy), dt)

    def face_fluxes(self):
        pb = self.pb
        Fx = torch.empty((pb.ncomp, pb.nyc, pb.nx + 1), dtype=torch.float64, device=self.device)
        Fy = torch.empty((pb.ncomp, pb.ny + 1, pb.nx), dtype=torch.float64, device=self.device) if pb.ndim == 2 else None
        ase_df_copy_face_fluxes(self.ctx, Fx, Fy)
        return Fx, Fy

    def step(self, dt: float = 0.0) -> None:
        ase_df_step(self.ctx, self.W, self.sx, self._sy(self.sy), dt)

    def run(self, nsteps: int, dt: float = 0.0) -> None:
        ase_df_run(self.ctx, self.W, self.sx, self._sy(self.sy), dt, nsteps)

    def status(self):
        return ase_df_get_status(self.ctx)

    def save(self, path: str) -> None:
        """Checkpoint: the state W, sigma and the device time t (one .npz file)."""
        import numpy as np

        flags, last_dt, t = self.status()
        np.savez(path, W=self.W.cpu().numpy(), sx=self.sx.cpu().numpy(), sy=self.sy.cpu().numpy(),
                 t=np.float64(t), last_dt=np.float64(last_dt), flags=np.uint32(flags))

    def load(self, path: str) -> None:
        """Resume from save(): the run continues bit for bit as if it had not stopped."""
        import numpy as np

        d = np.load(path)
        if tuple(d["W"].shape) != tuple(self.W.shape):
            raise ValueError("checkpoint of a different problem size")
        self.W.copy_(torch.as_tensor(d["W"]))
        self.sx.copy_(torch.as_tensor(d["sx"]))
        self.sy.copy_(torch.as_tensor(d["sy"]))
        ase_df_reset(self.ctx, float(d["t"]))

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None:
            ase_df_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
