"""The C-ABI library builds, loads and exports every entry point include/ase_df.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(ase_df_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_05489_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for n in ("ase_df_init", "ase_df_destroy", "ase_df_residual", "ase_df_step", "ase_df_prime_sigma",
              "ase_df_get_status", "ase_df_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_layout_matches_header():
    """The ctypes mirror of ase_df_params has the C layout (offsets of the last fields)."""
    from paper_2410_05489_gb300.ase_df import ase_df_params

    assert ase_df_params.bc.offset == 80
    assert ase_df_params.inflow_state.offset == 96
    assert ase_df_params.t_end.offset == 144
    assert ase_df_params.gks_c1.offset == 152 and ase_df_params.gks_c2.offset == 160
    assert ase_df_params.state_b.offset == 168 and ase_df_params.wall_x.offset == 200
    assert ase_df_params.shock_x0.offset == 208 and ase_df_params.shock_speed.offset == 216
    assert ctypes.sizeof(ase_df_params) == 224


def test_init_rejects_bad_parameters_without_a_device(lib):
    """Validation happens before any CUDA call, so it works on a CPU-only host."""
    from paper_2410_05489_gb300 import ase_df as A
    from paper_2410_05489_gb300.problems import Problem

    for bad in (dict(order=4), dict(nx=0), dict(gamma=1.0), dict(ndim=3), dict(cfl=0.0)):
        kw = dict(ndim=2, nx=8, ny=8, order=5)
        kw.update(bad)
        pb = Problem(**kw)
        with pytest.raises(A.AseDfError) as ei:
            A.ase_df_init(A.params_from_problem(pb))
        assert ei.value.status == 1
    pb = Problem(ndim=2, nx=8, ny=8, bc=("periodic", "outflow", "outflow", "outflow"))
    with pytest.raises(A.AseDfError):
        A.ase_df_init(A.params_from_problem(pb))
    pb = Problem(ndim=2, nx=1 << 21, ny=8)
    with pytest.raises(A.AseDfError) as ei:
        A.ase_df_init(A.params_from_problem(pb))
    assert ei.value.status == 6
    # the double Mach reflection boundaries: the split wall on y-lo and the moving shock on
    # y-hi of a 2D grid only, with physical states and finite positions
    good = dict(ndim=2, nx=16, ny=8, order=5, bc=("inflow", "outflow", "wall_after", "moving_shock"),
                inflow=(8.0, 7.1, -4.1, 116.0), inflow_lo=-1.0, inflow_hi=2.0, state_b=(1.4, 0.0, 0.0, 1.0),
                wall_x=0.2, shock_x0=0.5, shock_speed=11.0)
    for bad in (dict(bc=("wall_after", "outflow", "outflow", "outflow")),
                dict(bc=("outflow", "outflow", "moving_shock", "outflow")),
                dict(ndim=1, bc=("outflow", "outflow", "wall_after", "outflow")),
                dict(state_b=(1.4, 0.0, 0.0, -1.0)), dict(inflow=(0.0, 0.0, 0.0, 1.0)),
                dict(wall_x=float("nan")), dict(shock_speed=float("inf")), dict(ny=2, order=9)):
        kw = dict(good)
        kw.update(bad)
        with pytest.raises(A.AseDfError) as ei:
            A.ase_df_init(A.params_from_problem(Problem(**kw)))
        assert ei.value.status == 1


def test_batch_init_rejects_bad_sets_without_a_device(lib):
    """An empty batch, a batch with an invalid problem and one with a problem too large for
    its 32-bit offsets are refused before any CUDA call."""
    from paper_2410_05489_gb300 import ase_df as A
    from paper_2410_05489_gb300 import batch as B
    from paper_2410_05489_gb300.problems import Problem

    with pytest.raises(A.AseDfError) as ei:
        B.ase_df_batch_init([])
    assert ei.value.status == 1
    ok = A.params_from_problem(Problem(ndim=2, nx=8, ny=8, order=5))
    for bad, status in ((Problem(ndim=2, nx=0, ny=8, order=5), 1), (Problem(ndim=2, nx=8, ny=8, order=6), 1),
                        (Problem(ndim=2, nx=1 << 20, ny=1 << 12, order=5), 6)):
        with pytest.raises(A.AseDfError) as ei:
            B.ase_df_batch_init([ok, A.params_from_problem(bad)])
        assert ei.value.status == status
