"""The no-allocation residual entry point, for callers that cannot allocate device
memory: code inside another library's CUDA graph capture (cudaMalloc would break the
capture), real-time loops that must not synchronise the device (cudaFree does), and
frameworks that own every device byte through their own pool.

It is called here through the C ABI with ctypes. It runs the same kernels on the same
inputs as the context-based ase_df_residual, with tables from the same builder and a
problem described by the same setup code, so its residual and sigma_out must equal
ase_df_residual's bit for bit. Each case makes two calls in a row on different data
(the second call reuses the fixed scratch array the first one left behind), checks that
a call changes the device's free memory by nothing, and that a call captured into a CUDA
graph after a first, uncaptured call replays to the same result. This file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_05489_gb300 import problems as P

pytestmark = pytest.mark.gpu

E_INVAL, E_BOUNDS = 1, 6


@pytest.fixture(scope="module")
def lib_and_binding():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2410_05489_gb300 import build

    build.build()
    from paper_2410_05489_gb300 import ase_df as A

    lib = A._load()
    f = lib.ase_df_residual_noalloc
    f.argtypes = [ctypes.POINTER(A.ase_df_params)] + [ctypes.c_void_p] * 7
    f.restype = ctypes.c_int
    return f, A


def _dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _reference(A, pb, W, sx, sy):
    import torch

    ctx = A.ase_df_init(A.params_from_problem(pb))
    try:
        L = torch.empty_like(W)
        sxo = torch.empty_like(sx)
        syo = torch.empty_like(sy)
        two = pb.ndim == 2
        A.ase_df_residual(ctx, W, sx, sy if two else None, L, sxo, syo if two else None)
        torch.cuda.synchronize()
        return L.cpu().numpy(), sxo.cpu().numpy(), syo.cpu().numpy()
    finally:
        A.ase_df_destroy(ctx)


class _Call:
    """Output buffers (allocated by the test, as a caller's pool would) and one call."""

    def __init__(self, f, A, pb, W, sx, sy):
        import torch

        self.f, self.pb = f, pb
        self.W, self.sx, self.sy = W, sx, sy
        self.L = torch.full_like(W, np.nan)
        self.sxo = torch.full_like(sx, np.nan)
        self.syo = torch.full_like(sy, np.nan)
        self.params = A.params_from_problem(pb)

    def __call__(self):
        import torch

        two = self.pb.ndim == 2
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return self.f(ctypes.byref(self.params), _p(self.W), _p(self.sx), _p(self.sy) if two else None,
                      _p(self.L), _p(self.sxo), _p(self.syo) if two else None, stream)

    def results(self):
        import torch

        torch.cuda.synchronize()
        return self.L.cpu().numpy(), self.sxo.cpu().numpy(), self.syo.cpu().numpy()


def _equal(got, ref, ndim):
    Ln, sxn, syn = got
    Lr, sxr, syr = ref
    assert not np.isnan(Ln).any()
    assert np.array_equal(Ln, Lr), np.abs(Ln - Lr).max()
    assert np.array_equal(sxn, sxr), np.abs(sxn - sxr).max()
    if ndim == 2:
        assert np.array_equal(syn, syr), np.abs(syn - syr).max()


def _dmr_fixed_top(nx, order):
    """The double Mach reflection's inflow and split-wall boundaries with an outflow top
    (the moving shock needs the solver time, which the entry point does not take)."""
    pb, W = P.double_mach_reflection(nx, order)
    return pb.replace(bc=("inflow", "outflow", "wall_after", "outflow")), W


CASES = {
    "vortex_2d_r9": lambda: P.isentropic_vortex(96, 9, ny=80),
    "vortex_2d_r5": lambda: P.isentropic_vortex(96, 5, ny=80),
    "riemann_2d_r3": lambda: P.riemann_2d(70, 3, 4, ny=45),
    "riemann_1d_r7": lambda: P.riemann_1d(700, 7, 3),
    "jet_inflow_band_r9": lambda: P.high_mach_jet(120, 60, 9),
    "blast_walls_1d_r5": lambda: P.blast_wave(300, 5),
    "dmr_wall_after_r7": lambda: _dmr_fixed_top(160, 7),
    "largest_accepted_511_r9": lambda: P.riemann_2d(511, 9, 5),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_equals_context_residual(lib_and_binding, case):
    import torch

    f, A = lib_and_binding
    pb, W0 = CASES[case]()
    cases = [(W0, P.random_sigma(pb, 1, 1.0)), (P.white_noise(pb, 2), P.random_sigma(pb, 2, 0.6))]
    for k, (W, (sx, sy)) in enumerate(cases):  # two calls in a row on different data
        Wd, sxd, syd = _dev(W), _dev(sx), _dev(sy)
        ref = _reference(A, pb, Wd, sxd, syd)
        call = _Call(f, A, pb, Wd, sxd, syd)
        assert call() == 0, A._load().ase_df_last_error(None)
        _equal(call.results(), ref, pb.ndim)
        if k == 1:
            # the same call again allocates nothing: the device's free memory is unchanged
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            assert call() == 0
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free1 == free0, (free0, free1)
            _equal(call.results(), ref, pb.ndim)


@pytest.mark.parametrize("case", ["vortex_2d_r9", "riemann_1d_r7"])
def test_noalloc_inside_a_graph_capture(lib_and_binding, case):
    """Allocation is off limits inside a stream capture: a call made there after a first,
    uncaptured call (which found the scratch address) is recorded into the graph, and
    the replay gives the context residual of the data in the captured buffers."""
    import torch

    f, A = lib_and_binding
    pb, W0 = CASES[case]()
    sx, sy = P.random_sigma(pb, 3, 1.0)
    Wd, sxd, syd = _dev(W0), _dev(sx), _dev(sy)
    call = _Call(f, A, pb, Wd, sxd, syd)
    assert call() == 0  # outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = call()
    assert st == 0, A._load().ase_df_last_error(None)
    W2 = P.white_noise(pb, 4)
    sx2, sy2 = P.random_sigma(pb, 4, 0.8)
    for W, s_x, s_y in ((W0, sx, sy), (W2, sx2, sy2)):
        Wd.copy_(_dev(W))
        sxd.copy_(_dev(s_x))
        syd.copy_(_dev(s_y))
        call.L.fill_(np.nan)
        graph.replay()
        _equal(call.results(), _reference(A, pb, _dev(W), _dev(s_x), _dev(s_y)), pb.ndim)


def test_noalloc_rejects_what_it_cannot_do(lib_and_binding):
    import torch

    f, A = lib_and_binding
    last_error = A._load().ase_df_last_error
    # a grid beyond the fixed scratch
    pb = P.Problem(ndim=2, nx=512, ny=512, order=5, bc=("periodic",) * 4)
    W = torch.zeros(pb.state_shape, dtype=torch.float64, device="cuda")
    sx = torch.zeros(pb.sx_shape, dtype=torch.float64, device="cuda")
    sy = torch.zeros(pb.sy_shape, dtype=torch.float64, device="cuda")
    L = torch.empty_like(W)
    params = A.params_from_problem(pb)
    st = f(ctypes.byref(params), _p(W), _p(sx), _p(sy), _p(L), _p(torch.empty_like(sx)), _p(torch.empty_like(sy)),
           None)
    assert st == E_BOUNDS
    assert b"fixed scratch" in last_error(None)
    # the moving-shock boundary needs the solver time
    pb, _ = P.double_mach_reflection(64, 5)
    params = A.params_from_problem(pb)
    W = torch.zeros(pb.state_shape, dtype=torch.float64, device="cuda")
    sx = torch.zeros(pb.sx_shape, dtype=torch.float64, device="cuda")
    sy = torch.zeros(pb.sy_shape, dtype=torch.float64, device="cuda")
    st = f(ctypes.byref(params), _p(W), _p(sx), _p(sy), _p(torch.empty_like(W)), _p(torch.empty_like(sx)),
           _p(torch.empty_like(sy)), None)
    assert st == E_INVAL
    assert b"moving-shock" in last_error(None)
    # validation is ase_df_init's: a reflecting wall needs (r + 1) / 2 cells
    pb = P.Problem(ndim=1, nx=3, order=9, bc=("reflect", "reflect", "outflow", "outflow"))
    params = A.params_from_problem(pb)
    W = torch.zeros(pb.state_shape, dtype=torch.float64, device="cuda")
    sx = torch.zeros(pb.sx_shape, dtype=torch.float64, device="cuda")
    st = f(ctypes.byref(params), _p(W), _p(sx), None, _p(torch.empty_like(W)), _p(torch.empty_like(sx)), None, None)
    assert st == E_INVAL
    assert b"reflecting x-wall" in last_error(None)
