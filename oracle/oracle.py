"""ORACLE -- test infrastructure only.

Python wrapper (ctypes) of the plain serial FP64 C++ oracle in ase_df_oracle.cpp.  It is
the reference the CUDA library is checked against and shares no code with it.  Only
tests/, __graft_entry__.smoke() and bench.py's CPU baseline / reference arm may import
it.  build() compiles the shared library with g++ (-O2 -ffp-contract=off) into
oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ase_df_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libasedf_oracle.so")
_LIB_COUNT = os.path.join(_BUILD, "libasedf_oracle_count.so")
_LIB_TAPE = os.path.join(_BUILD, "libasedf_oracle_tape.so")
_lock = threading.Lock()

BRANCHES = ("lin9", "lin7", "lin5", "weno_df", "lin3", "df3", "first_order", "repaired", "frozen")


def _compile(out: str, extra=()) -> None:
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           *extra, _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> None:
    """Compile the oracle libraries (plain and op-counting) if missing or stale."""
    with _lock:
        for out, extra in ((_LIB, ()), (_LIB_COUNT, ("-DORACLE_COUNT_OPS",)), (_LIB_TAPE, ("-DORACLE_TAPE",))):
            if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
                _compile(out, extra)


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32), ("order", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("sigma_thres", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("inflow", ctypes.c_double * 4),
        ("inflow_lo", ctypes.c_double), ("inflow_hi", ctypes.c_double),
        ("gks_c1", ctypes.c_double), ("gks_c2", ctypes.c_double),
        ("t", ctypes.c_double), ("state_b", ctypes.c_double * 4), ("wall_x", ctypes.c_double),
        ("shock_x0", ctypes.c_double), ("shock_speed", ctypes.c_double),
    ]


_P = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_libs = {}


def _setup(lib):
    lib.oracle_residual.argtypes = [ctypes.POINTER(_Params), _P, _P, _P, _P, _P, _P, _P, _P, _I64]
    lib.oracle_residual.restype = ctypes.c_int
    lib.oracle_residual_rows.argtypes = [ctypes.POINTER(_Params), _P, _P, _P, _P, _P, _P, ctypes.c_int64,
                                         ctypes.c_int64]
    lib.oracle_residual_rows.restype = ctypes.c_int
    lib.oracle_cfl_dt.argtypes = [ctypes.POINTER(_Params), _P]
    lib.oracle_cfl_dt.restype = ctypes.c_double
    lib.oracle_step.argtypes = [ctypes.POINTER(_Params), _P, _P, _P, ctypes.c_double, _I64]
    lib.oracle_step.restype = ctypes.c_double
    lib.oracle_prime_sigma.argtypes = [ctypes.POINTER(_Params), _P, _P, _P]
    lib.oracle_reconstruct.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P]
    lib.oracle_reconstruct.restype = ctypes.c_int
    lib.oracle_weno_ao53.argtypes = [_P, _P, ctypes.c_int, _P, _P, ctypes.c_int, _P]
    lib.oracle_weno_ao53.restype = None
    lib.oracle_coef_table.argtypes = [ctypes.c_int, _P, _P]
    lib.oracle_coef_table.restype = ctypes.c_int
    lib.oracle_zq.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.oracle_zq.restype = ctypes.c_double
    lib.oracle_gauss01.argtypes = [ctypes.c_int, _P, _P]
    lib.oracle_gauss01.restype = None
    lib.oracle_lf_flux.argtypes = [ctypes.c_int, ctypes.c_double, _P, _P, _P, _P, _P, _P]
    lib.oracle_lf_flux.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    return lib


def _lib(counting: bool = False, tape: bool = False):
    key = "count" if counting else ("tape" if tape else "plain")
    if key not in _libs:
        build()
        lib = _setup(ctypes.CDLL(_LIB_COUNT if counting else (_LIB_TAPE if tape else _LIB)))
        if counting:
            lib.oracle_op_counts.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
            lib.oracle_reset_op_counts.argtypes = []
        if key == "plain":
            lib.oracle_gks_point.argtypes = ([ctypes.c_int32, ctypes.c_double] + [_P] * 6 +
                                             [ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P])
            lib.oracle_gks_point.restype = None
            lib.oracle_gks_residual.argtypes = [ctypes.POINTER(_Params), _P, _P, _P, ctypes.c_double, _P, _P, _P,
                                                _P, _I64]
            lib.oracle_gks_residual.restype = None
            lib.oracle_gks_step.argtypes = [ctypes.POINTER(_Params), _P, _P, _P, ctypes.c_double, _I64]
            lib.oracle_gks_step.restype = ctypes.c_double
        if tape:
            lib.oracle_residual_vjp.argtypes = [ctypes.POINTER(_Params)] + [_P] * 9
            lib.oracle_residual_vjp.restype = ctypes.c_int64
            lib.oracle_run_vjp.argtypes = [ctypes.POINTER(_Params), _P, ctypes.c_int32, ctypes.c_double, _P, _P]
            lib.oracle_run_vjp.restype = ctypes.c_int64
            lib.oracle_last_vjp_edges.argtypes = []
            lib.oracle_last_vjp_edges.restype = ctypes.c_int64
        _libs[key] = lib
    return _libs[key]


def _params(pb, t: float = 0.0) -> _Params:
    """The problem's parameters; t is the time of the evaluation (the moving-shock boundary
    depends on it)."""
    p = _Params()
    p.ndim, p.order = pb.ndim, pb.order
    p.nx, p.ny = pb.nx, pb.nyc
    p.x0, p.x1, p.y0, p.y1 = pb.x0, pb.x1, pb.y0, pb.y1
    p.gamma, p.sigma_thres, p.cfl = pb.gamma, pb.sigma_thres, pb.cfl
    for i, c in enumerate(pb.bc_codes()):
        p.bc[i] = c
    for i in range(4):
        p.inflow[i] = pb.inflow[i]
    p.inflow_lo, p.inflow_hi = pb.inflow_lo, pb.inflow_hi
    p.gks_c1, p.gks_c2 = pb.gks_c1, pb.gks_c2
    p.t = float(t)
    for i in range(4):
        p.state_b[i] = pb.state_b[i]
    p.wall_x, p.shock_x0, p.shock_speed = pb.wall_x, pb.shock_x0, pb.shock_speed
    return p


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> int:
    """Host threads for the face loops of the plain build (default 1; the results do not
    depend on it).  Returns the previous setting."""
    return _lib().oracle_set_threads(int(n))


class threads:
    """Context manager: run the plain oracle's face loops on n host threads."""

    def __init__(self, n: int):
        self.n = n

    def __enter__(self):
        self.old = set_threads(self.n)
        return self

    def __exit__(self, *exc):
        set_threads(self.old)


def residual(pb, W, sx, sy, counting: bool = False, t: float = 0.0):
    """One residual evaluation L(W; sigma_in) at time t -> (L, sx_out, sy_out, Fx, Fy, hist)."""
    W, sx, sy = _f64(W), _f64(sx), _f64(sy)
    assert W.shape == pb.state_shape and sx.shape == pb.sx_shape and sy.shape == pb.sy_shape
    L = np.empty_like(W)
    sxo = np.empty(pb.sx_shape)
    syo = np.zeros(pb.sy_shape)
    Fx = np.empty((pb.ncomp, pb.nyc, pb.nx + 1))
    Fy = np.empty((pb.ncomp, pb.ny + 1, pb.nx)) if pb.ndim == 2 else None
    hist = np.zeros(len(BRANCHES), dtype=np.int64)
    p = _params(pb, t)
    _lib(counting).oracle_residual(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), _ptr(L), _ptr(sxo),
                                   _ptr(syo), _ptr(Fx), _ptr(Fy), hist.ctypes.data_as(_I64))
    return L, sxo, syo, Fx, Fy, hist


def residual_rows(pb, W, sx, sy, row_lo: int, row_hi: int):
    """Rows row_lo..row_hi of L, sigma_x_out (same rows) and sigma_y_out (faces row_lo..
    row_hi+1) of one residual evaluation; the oracle computes only what those rows need."""
    W, sx, sy = _f64(W), _f64(sx), _f64(sy)
    L = np.full(pb.state_shape, np.nan)
    sxo = np.full(pb.sx_shape, np.nan)
    syo = np.full(pb.sy_shape, np.nan)
    p = _params(pb)
    rc = _lib().oracle_residual_rows(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), _ptr(L), _ptr(sxo), _ptr(syo),
                                     row_lo, row_hi)
    if rc != 0:
        raise ValueError("bad row range")
    return (L[:, row_lo:row_hi + 1], sxo[row_lo:row_hi + 1],
            syo[row_lo:row_hi + 2] if pb.ndim == 2 else None)


def prime_sigma(pb, W) -> Tuple[np.ndarray, np.ndarray]:
    """sigma^0: the sigma of a residual evaluated with sigma_in = 0."""
    W = _f64(W)
    sx = np.empty(pb.sx_shape)
    sy = np.zeros(pb.sy_shape)
    p = _params(pb)
    _lib().oracle_prime_sigma(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy))
    return sx, sy


def cfl_dt(pb, W) -> float:
    p = _params(pb)
    return _lib().oracle_cfl_dt(ctypes.byref(p), _ptr(_f64(W)))


def step(pb, W, sx, sy, dt: float = 0.0, hist: Optional[np.ndarray] = None, t: float = 0.0):
    """One SSP-RK3 step from time t; returns (W_new, sx_new, sy_new, dt_used)."""
    W, sx, sy = _f64(W).copy(), _f64(sx).copy(), _f64(sy).copy()
    h = hist if hist is not None else np.zeros(len(BRANCHES), dtype=np.int64)
    p = _params(pb, t)
    dt_used = _lib().oracle_step(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), float(dt),
                                 h.ctypes.data_as(_I64))
    return W, sx, sy, dt_used


def run(pb, W, t_end: float = 0.0, nsteps: int = 0, dt: float = 0.0, sigma=None):
    """March with SSP-RK3 to t_end (CFL steps, the last one shortened) or for nsteps steps
    of size dt (CFL when dt <= 0).  sigma^0 is primed unless given."""
    sx, sy = prime_sigma(pb, W) if sigma is None else sigma
    t = 0.0
    n = 0
    W = _f64(W)
    while True:
        if nsteps and n >= nsteps:
            break
        if t_end and t >= t_end * (1 - 1e-14):
            break
        h = dt if dt > 0 else cfl_dt(pb, W)
        if h <= 0:
            raise FloatingPointError("non-physical state at t=%g" % t)
        if t_end and t + h > t_end:
            h = t_end - t
        W, sx, sy, h = step(pb, W, sx, sy, h, t=t)
        if h < 0:
            raise FloatingPointError("non-physical state after the step at t=%g" % t)
        t += h
        n += 1
    return W, sx, sy, t, n


def reconstruct(r: int, vals, sig, thres: float = 2.0, xi=(0.0,)) -> Tuple[np.ndarray, int]:
    """ASE-DF reconstruction of one cell (Algorithm 1 capped at r) at points xi of [-1, 0]."""
    vals, sig, xi = _f64(vals), _f64(sig), _f64(xi)
    k = (r - 1) // 2
    assert vals.shape == (2 * k + 1,) and sig.shape == (2 * k,)
    out = np.empty(len(xi))
    br = _lib().oracle_reconstruct(r, _ptr(vals), _ptr(sig), thres, len(xi), _ptr(xi), _ptr(out))
    return out, br


def weno_ao53(vals, alpha, xi=(0.0,), force_linear_weights=False):
    """WENOZ-AO(5,3) with explicit DF factors; returns (values, (beta_-1, beta_0, beta_1,
    beta5_bar, tau_Z))."""
    vals, alpha, xi = _f64(vals), _f64(alpha), _f64(xi)
    out = np.empty(len(xi))
    beta = np.empty(5)
    _lib().oracle_weno_ao53(_ptr(vals), _ptr(alpha), len(xi), _ptr(xi), _ptr(out),
                            int(bool(force_linear_weights)), _ptr(beta))
    return out, beta


def coef_table(stencil: int):
    """Printed coefficient table: stencil 0..2 = S3_-1, S3_0, S3_1; 5, 7, 9."""
    num = np.zeros(8 * 9)
    den = np.zeros(8)
    n = _lib().oracle_coef_table(stencil, _ptr(num), _ptr(den))
    return num[: n * 9].reshape(n, 9), den[:n]


def zq(q: int, xi: float) -> float:
    return _lib().oracle_zq(q, xi)


def gauss01(G: int):
    t = np.empty(G)
    w = np.empty(G)
    _lib().oracle_gauss01(G, _ptr(t), _ptr(w))
    return t, w


def lf_flux(qL, qR, gamma: float, cL=None, cR=None):
    """Lax-Friedrichs flux of one Gauss point in the face frame -> (F, sigma, fallback)."""
    qL, qR = _f64(qL), _f64(qR)
    cL = qL if cL is None else _f64(cL)
    cR = qR if cR is None else _f64(cR)
    C = len(qL)
    F = np.empty(C)
    s = np.empty(1)
    fb = _lib().oracle_lf_flux(C, gamma, _ptr(qL), _ptr(qR), _ptr(cL), _ptr(cR), _ptr(F), _ptr(s))
    return F, float(s[0]), bool(fb)


def op_counts_residual(pb, W, sx, sy):
    """FP64 operations (add, mul, div, sqrt) the oracle performs for one residual."""
    lib = _lib(True)
    lib.oracle_reset_op_counts()
    residual(pb, W, sx, sy, counting=True)
    out = (ctypes.c_longlong * 4)()
    lib.oracle_op_counts(out)
    return tuple(int(v) for v in out)


def last_vjp_edges() -> int:
    """Edges (operation, non-constant operand) of the graph of the last residual_vjp."""
    return int(_lib(tape=True).oracle_last_vjp_edges())


def residual_vjp(pb, W, sx, sy, Lbar, sxbar_out=None, sybar_out=None):
    """Reverse-mode VJP of (L, sigma_out) = R(W, sigma_in) by the oracle's tape:
    -> (Wbar, sxbar_in, sybar_in)."""
    W, sx, sy, Lbar = _f64(W), _f64(sx), _f64(sy), _f64(Lbar)
    Wbar = np.zeros(pb.state_shape)
    sxb = np.zeros(pb.sx_shape)
    syb = np.zeros(pb.sy_shape)
    sxo = None if sxbar_out is None else _f64(sxbar_out)
    syo = None if sybar_out is None else _f64(sybar_out)
    p = _params(pb)
    _lib(tape=True).oracle_residual_vjp(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), _ptr(Lbar), _ptr(sxo),
                                        _ptr(syo), _ptr(Wbar), _ptr(sxb), _ptr(syb))
    return Wbar, sxb, syb


def run_vjp(pb, W0, nsteps: int, dt: float, Wbar_final):
    """Reverse mode through sigma^0 = prime(W0) and nsteps fixed-dt SSP-RK3 steps:
    -> dJ/dW0 for J with dJ/dW_final = Wbar_final."""
    W0, Wbf = _f64(W0), _f64(Wbar_final)
    Wbar0 = np.zeros(pb.state_shape)
    p = _params(pb)
    n = _lib(tape=True).oracle_run_vjp(ctypes.byref(p), _ptr(W0), int(nsteps), float(dt), _ptr(Wbf), _ptr(Wbar0))
    if n < 0:
        raise FloatingPointError("non-physical state in the taped run")
    return Wbar0


# ----------------------------------------------------------------------------------
# gas-kinetic flux and S2O4 (Sec. 2.2)
# ----------------------------------------------------------------------------------
def gks_point(dim: int, gamma: float, Wl, Wlx, Wly, Wr, Wrx, Wry, dt: float, c1: float = 0.05, c2: float = 1.0):
    """GKS flux at one Gauss point, face frame: -> (F, F_t)."""
    n = dim + 2
    arrs = [_f64(np.asarray(a, dtype=np.float64).reshape(-1)[:n]) if a is not None else np.zeros(n)
            for a in (Wl, Wlx, Wly, Wr, Wrx, Wry)]
    F = np.zeros(n)
    Ft = np.zeros(n)
    _lib().oracle_gks_point(int(dim), float(gamma), *[_ptr(a) for a in arrs], float(dt), float(c1), float(c2),
                            _ptr(F), _ptr(Ft))
    return F, Ft


def gks_residual(pb, W, sx, sy, dt: float, t: float = 0.0):
    """One GKS evaluation at time t: -> (L, L_t, sx_out, sy_out, hist)."""
    W, sx, sy = _f64(W), _f64(sx), _f64(sy)
    L = np.empty_like(W)
    Lt = np.empty_like(W)
    sxo = np.empty(pb.sx_shape)
    syo = np.zeros(pb.sy_shape)
    hist = np.zeros(len(BRANCHES), dtype=np.int64)
    p = _params(pb, t)
    _lib().oracle_gks_residual(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), float(dt), _ptr(L), _ptr(Lt),
                               _ptr(sxo), _ptr(syo), hist.ctypes.data_as(_I64))
    return L, Lt, sxo, syo, hist


def gks_step(pb, W, sx, sy, dt: float = 0.0, hist: Optional[np.ndarray] = None, t: float = 0.0):
    """One S2O4 step from time t (CFL when dt <= 0): -> (W, sx, sy, dt used; negative if
    non-physical)."""
    W, sx, sy = _f64(W).copy(), _f64(sx).copy(), _f64(sy).copy()
    h = np.zeros(len(BRANCHES), dtype=np.int64) if hist is None else hist
    p = _params(pb, t)
    d = _lib().oracle_gks_step(ctypes.byref(p), _ptr(W), _ptr(sx), _ptr(sy), float(dt), h.ctypes.data_as(_I64))
    return W, sx, sy, d


def gks_run(pb, W, t_end: float = 0.0, nsteps: int = 0, dt: float = 0.0, dt_cap: float = 0.0):
    """S2O4 march to t_end (CFL steps, capped by dt_cap if > 0, the last one shortened) or
    nsteps steps of dt; sigma^0 is primed.  -> (W, sx, sy, t, n)."""
    sx, sy = prime_sigma(pb, W)
    W = _f64(W)
    t, n = 0.0, 0
    while True:
        if nsteps and n >= nsteps:
            break
        if t_end and t >= t_end * (1 - 1e-14):
            break
        h = dt if dt > 0 else cfl_dt(pb, W)
        if h <= 0:
            raise FloatingPointError("non-physical state at t=%g" % t)
        if dt_cap > 0:
            h = min(h, dt_cap)
        if t_end and t + h > t_end:
            h = t_end - t
        W, sx, sy, h2 = gks_step(pb, W, sx, sy, h, t=t)
        if h2 < 0:
            raise FloatingPointError("non-physical state after the step at t=%g" % t)
        t += h
        n += 1
    return W, sx, sy, t, n
