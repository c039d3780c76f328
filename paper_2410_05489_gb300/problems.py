"""Problem descriptions and seeded synthetic initial data.

This module states problems (grid, boundary conditions, gas constant, scheme order) and
builds their initial cell averages.  It holds none of the reconstruction, flux or time
stepping of the method: it is the one module that both the CUDA path and the CPU
oracle are fed from.  It imports neither torch nor any compiled library.

Initial data are cell averages computed by tensor Gauss-Legendre quadrature (10 points
per direction by default) of closed-form primitive fields converted to conservative
variables; point values would cap the accuracy of a high-order scheme at 2nd order.

Workloads (the paper's section in brackets; the others are synthetic stand-ins):
  * 1D sin-wave, 2D sin-wave            (Sec. 4.2, accuracy tests)
  * Sod shock tube                      (a textbook Riemann problem)
  * isentropic vortex                   (a textbook smooth 2D Euler solution)
  * high-Mach jet, Ma ~ 20000           (Sec. 4.3, Example 6, re-scaled domain)
  * 2D Riemann data of Configuration-3 shape, random states   (Sec. 4.1, Example 2)
  * random smooth Fourier fields, random Riemann data, per-cell white noise (parity)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Sequence, Tuple

import numpy as np

BC_NAMES = {"periodic": 0, "outflow": 1, "inflow": 2, "reflect": 3, "wall_after": 4, "moving_shock": 5}


@dataclasses.dataclass
class Problem:
    """A 1D or 2D Euler problem on a uniform Cartesian grid.

    bc is (x-lo, x-hi, y-lo, y-hi), each "periodic", "outflow", "reflect" (a wall: mirrored
    ghost cells with the normal momentum negated) or (x-lo only) "inflow": the inflow band
    inflow_lo < y < inflow_hi of the x-lo boundary takes the fixed primitive state
    inflow = (rho, u, v, p); outside the band it is outflow.  Two more for the double Mach
    reflection: (y-lo only) "wall_after": ghost cells whose centre x is below wall_x take the
    inflow state, the rest a reflecting wall; (y-hi only) "moving_shock": ghost cells take
    the inflow state where their centre x is below shock_x0 + shock_speed t, and state_b
    beyond.
    """

    ndim: int
    nx: int
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    order: int = 5
    gamma: float = 1.4
    sigma_thres: float = 2.0
    cfl: float = 0.5
    bc: Tuple[str, str, str, str] = ("outflow", "outflow", "outflow", "outflow")
    inflow: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    inflow_lo: float = 0.0
    inflow_hi: float = 0.0
    gks_c1: float = 0.05   # tau_n constants of the gas-kinetic path (Sec. 2.2; the paper's
    gks_c2: float = 1.0    # captions give 0.05 and 1.0, and c2 = 5.0 for the blast wave)
    state_b: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    wall_x: float = 0.0
    shock_x0: float = 0.0
    shock_speed: float = 0.0

    @property
    def ncomp(self) -> int:
        return 3 if self.ndim == 1 else 4

    @property
    def nyc(self) -> int:
        return 1 if self.ndim == 1 else self.ny

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return 1.0 if self.ndim == 1 else (self.y1 - self.y0) / self.ny

    @property
    def ncells(self) -> int:
        return self.nx * self.nyc

    @property
    def state_shape(self) -> Tuple[int, int, int]:
        return (self.ncomp, self.nyc, self.nx)

    @property
    def sx_shape(self) -> Tuple[int, int]:
        return (self.nyc, self.nx + 1)

    @property
    def sy_shape(self) -> Tuple[int, int]:
        return (self.ny + 1, self.nx) if self.ndim == 2 else (1, 1)

    def bc_codes(self) -> Tuple[int, int, int, int]:
        return tuple(BC_NAMES[b] for b in self.bc)  # type: ignore[return-value]

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------------
# primitive -> conservative and cell averaging
# ----------------------------------------------------------------------------------
def conservative(prim: Sequence[np.ndarray], gamma: float, ndim: int) -> np.ndarray:
    """(rho, u, [v], p) -> (rho, rho u, [rho v], E) with E = p/(gamma-1) + rho|u|^2/2."""
    if ndim == 1:
        rho, u, p = prim
        return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
    rho, u, v, p = prim
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def _leggauss01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def cell_average(pb: Problem, prim_fn: Callable, npts: int = 10) -> np.ndarray:
    """Cell averages of the conservative variables of prim_fn(x[, y]) -> primitives."""
    t, w = _leggauss01(npts)
    xs = pb.x0 + (np.arange(pb.nx)[:, None] + t[None, :]) * pb.dx  # [nx, npts]
    if pb.ndim == 1:
        U = conservative(prim_fn(xs), pb.gamma, 1)  # [3, nx, npts]
        return np.ascontiguousarray((U * w).sum(-1)[:, None, :])
    ys = pb.y0 + (np.arange(pb.ny)[:, None] + t[None, :]) * pb.dy  # [ny, npts]
    X = xs[None, :, None, :]  # [1, nx, 1, q]
    Y = ys[:, None, :, None]  # [ny, 1, q, 1]
    X, Y = np.broadcast_arrays(X, Y)  # [ny, nx, qy, qx]
    U = conservative(prim_fn(X, Y), pb.gamma, 2)  # [4, ny, nx, qy, qx]
    ww = w[:, None] * w[None, :]
    return np.ascontiguousarray((U * ww).sum((-1, -2)))


# ----------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------
def sod(n: int = 200, order: int = 5) -> Tuple[Problem, np.ndarray]:
    """Sod tube on [0,1]: (1,0,1) | (0.125,0,0.1) at x = 0.5, gamma 1.4, outflow."""
    pb = Problem(ndim=1, nx=n, order=order, gamma=1.4, bc=("outflow",) * 4)

    def prim(x):
        left = x < 0.5
        return (np.where(left, 1.0, 0.125), np.zeros_like(x), np.where(left, 1.0, 0.1))

    return pb, cell_average(pb, prim)


def sin_wave_1d(n: int, order: int) -> Tuple[Problem, np.ndarray]:
    """Sec. 4.2: rho = 1 + 0.2 sin(pi x), u = p = 1 on [0,2], periodic."""
    pb = Problem(ndim=1, nx=n, x0=0.0, x1=2.0, order=order, gamma=1.4, bc=("periodic",) * 4)
    return pb, cell_average(pb, lambda x: (1.0 + 0.2 * np.sin(np.pi * x), np.ones_like(x), np.ones_like(x)))


def sin_wave_1d_exact(pb: Problem, t: float) -> np.ndarray:
    return cell_average(pb, lambda x: (1.0 + 0.2 * np.sin(np.pi * (x - t)), np.ones_like(x), np.ones_like(x)))


def sin_wave_2d(n: int, order: int) -> Tuple[Problem, np.ndarray]:
    """Sec. 4.2: rho = 1 + 0.2 sin(pi x) sin(pi y), u = v = p = 1 on [0,2]^2, periodic."""
    pb = Problem(ndim=2, nx=n, ny=n, x0=0.0, x1=2.0, y0=0.0, y1=2.0, order=order, gamma=1.4,
                 bc=("periodic",) * 4)
    return pb, sin_wave_2d_exact(pb, 0.0)


def sin_wave_2d_diag(n: int, order: int) -> Tuple[Problem, np.ndarray]:
    """The 2-D sin-wave of Table 2 (Sec. 4.2): rho = 1 + 0.2 sin(pi (x + y)), u = v = p = 1 on
    [0,2]^2, periodic (the diagonal wave reproduces the printed Table 2 errors)."""
    pb = Problem(ndim=2, nx=n, ny=n, x0=0.0, x1=2.0, y0=0.0, y1=2.0, order=order, gamma=1.4,
                 bc=("periodic",) * 4)
    return pb, sin_wave_2d_diag_exact(pb, 0.0)


def sin_wave_2d_diag_exact(pb: Problem, t: float) -> np.ndarray:
    def prim(x, y):
        one = np.ones_like(x)
        return (1.0 + 0.2 * np.sin(np.pi * (x + y - 2.0 * t)), one, one, one)

    return cell_average(pb, prim)


def sin_wave_2d_exact(pb: Problem, t: float) -> np.ndarray:
    def prim(x, y):
        one = np.ones_like(x)
        return (1.0 + 0.2 * np.sin(np.pi * (x - t)) * np.sin(np.pi * (y - t)), one, one, one)

    return cell_average(pb, prim)


def isentropic_vortex(n: int, order: int, strength: float = 5.0, gamma: float = 1.4,
                      ny: int | None = None) -> Tuple[Problem, np.ndarray]:
    """Isentropic vortex of strength 5 on the free stream (1,1,1,1), periodic [0,10]^2."""
    pb = Problem(ndim=2, nx=n, ny=ny or n, x0=0.0, x1=10.0, y0=0.0, y1=10.0, order=order,
                 gamma=gamma, bc=("periodic",) * 4)
    return pb, vortex_exact(pb, 0.0, strength)


def vortex_exact(pb: Problem, t: float, strength: float = 5.0) -> np.ndarray:
    g = pb.gamma
    eps = strength

    def prim(x, y):
        # centre advected with the free stream (1, 1), wrapped to the periodic box
        xc = 5.0 + t
        yc = 5.0 + t
        dxv = (x - xc + 5.0) % 10.0 - 5.0
        dyv = (y - yc + 5.0) % 10.0 - 5.0
        r2 = dxv * dxv + dyv * dyv
        e = np.exp(0.5 * (1.0 - r2))
        u = 1.0 - eps / (2.0 * np.pi) * e * dyv
        v = 1.0 + eps / (2.0 * np.pi) * e * dxv
        T = 1.0 - (g - 1.0) * eps * eps / (8.0 * g * np.pi * np.pi) * e * e
        rho = T ** (1.0 / (g - 1.0))
        return rho, u, v, rho * T

    return cell_average(pb, prim)


JET_U = 20000.0 * math.sqrt((5.0 / 3.0) * 0.4127 / 5.0)


def high_mach_jet(nx: int = 1600, ny: int = 800, order: int = 9) -> Tuple[Problem, np.ndarray]:
    """Ma ~ 20000 jet: [0,1] x [-0.25,0.25], gamma 5/3, ambient (0.5, 0, 0, 0.4127) at rest,
    inflow band |y| < 0.05 at x = 0 with rho = 5, p = 0.4127, u = 20000 sqrt(gamma p / rho);
    outflow elsewhere.  A re-scaled variant of Sec. 4.3, Example 6."""
    pb = Problem(ndim=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=-0.25, y1=0.25, order=order,
                 gamma=5.0 / 3.0, bc=("inflow", "outflow", "outflow", "outflow"),
                 inflow=(5.0, JET_U, 0.0, 0.4127), inflow_lo=-0.05, inflow_hi=0.05)
    rho = np.full((ny, nx), 0.5)
    p = np.full((ny, nx), 0.4127)
    z = np.zeros((ny, nx))
    return pb, np.ascontiguousarray(conservative((rho, z, z, p), pb.gamma, 2))


def riemann_1d(n: int, order: int, seed: int) -> Tuple[Problem, np.ndarray]:
    """Two random states split at a random x in [0.3, 0.7]; rho, p log-uniform [0.1, 10],
    u uniform [-2, 2]; outflow; [0,1]."""
    rng = np.random.default_rng(seed)
    pb = Problem(ndim=1, nx=n, order=order, gamma=1.4)
    rho = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 2))
    p = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 2))
    u = rng.uniform(-2.0, 2.0, 2)
    xs = rng.uniform(0.3, 0.7)
    x = pb.x0 + (np.arange(n) + 0.5) * pb.dx
    side = (x >= xs).astype(int)
    return pb, np.ascontiguousarray(conservative((rho[side], u[side], p[side]), pb.gamma, 1)[:, None, :])


def riemann_2d(n: int, order: int, seed: int, ny: int | None = None, x1: float = 1.0) -> Tuple[Problem, np.ndarray]:
    """Four random quadrant states split at (x1/2, 0.5) on [0,x1] x [0,1] (the shape of
    Configuration 3, Sec. 4.1); rho, p log-uniform [0.1, 10], u, v uniform [-2, 2]."""
    rng = np.random.default_rng(seed)
    ny = ny or n
    pb = Problem(ndim=2, nx=n, ny=ny, x1=x1, order=order, gamma=1.4)
    rho = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    p = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 4))
    u = rng.uniform(-2.0, 2.0, 4)
    v = rng.uniform(-2.0, 2.0, 4)
    x = (np.arange(n) + 0.5) * pb.dx
    y = (np.arange(ny) + 0.5) * pb.dy
    X, Y = np.meshgrid(x, y)
    q = (X >= 0.5 * x1).astype(int) + 2 * (Y >= 0.5).astype(int)
    return pb, np.ascontiguousarray(conservative((rho[q], u[q], v[q], p[q]), pb.gamma, 2))


def blast_wave(n: int = 400, order: int = 5, gks_c2: float = 5.0) -> Tuple[Problem, np.ndarray]:
    """Blast wave of Sec. 4.3 (Example 1): [0,1], reflecting walls, gamma 1.4, rho = 1, u = 0,
    p = 1000 (x < 0.1), 0.01, 100 (x > 0.9); run to t = 0.038 (the printed "t = 3.8" read as
    0.038, the time of the standard problem); c2 = 5.0 as in the paper's GKS runs."""
    pb = Problem(ndim=1, nx=n, order=order, gamma=1.4, bc=("reflect", "reflect", "outflow", "outflow"),
                 gks_c2=gks_c2)
    x = (np.arange(n) + 0.5) * pb.dx
    p = np.where(x < 0.1, 1000.0, np.where(x > 0.9, 100.0, 0.01))
    one = np.ones(n)
    return pb, np.ascontiguousarray(conservative((one, 0.0 * one, p), pb.gamma, 1)[:, None, :])


def shu_osher(n: int = 200, order: int = 5) -> Tuple[Problem, np.ndarray]:
    """Shu-Osher problem as Sec. 4.3 prints it: [0,10], (rho, u, p) = (3.857134, 2.629369,
    10.33333) for x < 1, (1 + 0.2 sin(5x), 0, 1) elsewhere, gamma 1.4, outflow; run to t = 1.8."""
    pb = Problem(ndim=1, nx=n, x0=0.0, x1=10.0, order=order, gamma=1.4)

    def prim(x):
        left = x < 1.0
        return (np.where(left, 3.857134, 1.0 + 0.2 * np.sin(5.0 * x)), np.where(left, 2.629369, 0.0),
                np.where(left, 10.33333, 1.0))

    return pb, cell_average(pb, prim)


def configuration3(n: int, order: int, gks_c1: float = 0.05, gks_c2: float = 1.0,
                   ny: int | None = None) -> Tuple[Problem, np.ndarray]:
    """Configuration 3 of Sec. 4.3 (Example 2): [0,1]^2 with n x ny cells (ny = n by default),
    quadrant states split at (0.7, 0.7), outflow, gamma 1.4; the workload of the paper's
    timing table (Table 4)."""
    ny = ny or n
    pb = Problem(ndim=2, nx=n, ny=ny, order=order, gamma=1.4, gks_c1=gks_c1, gks_c2=gks_c2)
    x = (np.arange(n) + 0.5) * pb.dx
    y = (np.arange(ny) + 0.5) * pb.dy
    X, Y = np.meshgrid(x, y)
    lo_x, lo_y = X < 0.7, Y < 0.7
    rho = np.where(lo_x & lo_y, 0.138, np.where(~lo_x & lo_y, 0.5323, np.where(~lo_x & ~lo_y, 1.5, 0.5323)))
    u = np.where(lo_x & lo_y, 1.206, np.where(~lo_x & lo_y, 0.0, np.where(~lo_x & ~lo_y, 0.0, 1.206)))
    v = np.where(lo_x & lo_y, 1.206, np.where(~lo_x & lo_y, 1.206, np.where(~lo_x & ~lo_y, 0.0, 0.0)))
    p = np.where(lo_x & lo_y, 0.129, np.where(~lo_x & lo_y, 0.3, np.where(~lo_x & ~lo_y, 1.5, 0.3)))
    return pb, np.ascontiguousarray(conservative((rho, u, v, p), pb.gamma, 2))


DMR_PRE = (1.4, 0.0, 0.0, 1.0)
DMR_POST = (8.0, 7.145, -4.125, 116.8333)


def double_mach_reflection(nx: int, order: int, gks_c1: float = 0.05, gks_c2: float = 1.0,
                           post: Tuple[float, float, float, float] = DMR_POST) -> Tuple[Problem, np.ndarray]:
    """Double Mach reflection, Sec. 4.3 Example 4 (reading G32): [0,4] x [0,1] with nx x nx/4
    cells, gamma 1.4; a Mach 10 shock at 60 degrees to the x-axis through (1/6, 0), the
    pre-shock state (1.4, 0, 0, 1) below y = sqrt(3) (x - 1/6) and the post-shock state
    (8, 7.145, -4.125, 116.8333) above; x-lo the post-shock inflow, x-hi outflow, y-lo the
    post-shock state for x < 1/6 and a slip wall after, y-hi the exact shock position
    x = 1/6 + (1 + 20 t) / sqrt(3).  Cell averages by 8 x 8 Gauss points."""
    s3 = np.sqrt(3.0)
    pb = Problem(ndim=2, nx=nx, ny=nx // 4, x0=0.0, x1=4.0, y0=0.0, y1=1.0, order=order, gamma=1.4,
                 bc=("inflow", "outflow", "wall_after", "moving_shock"), inflow=tuple(post),
                 inflow_lo=-1.0, inflow_hi=2.0, state_b=DMR_PRE, wall_x=1.0 / 6.0,
                 shock_x0=1.0 / 6.0 + 1.0 / s3, shock_speed=20.0 / s3, gks_c1=gks_c1, gks_c2=gks_c2)

    def prim(x, y):
        pre = y < s3 * (x - 1.0 / 6.0)
        return tuple(np.where(pre, a, b) for a, b in zip(DMR_PRE, post))

    return pb, cell_average(pb, prim, npts=8)


def smooth_random(pb: Problem, seed: int, nmodes: int = 3) -> np.ndarray:
    """Random smooth periodic Fourier field with O(1) relative variation."""
    rng = np.random.default_rng(seed)
    L = (pb.x1 - pb.x0, pb.y1 - pb.y0)

    def field(base, amp, *X):
        f = np.full_like(X[0], base)
        for _ in range(nmodes):
            k = rng.integers(1, 4, size=len(X))
            ph = rng.uniform(0, 2 * np.pi, size=len(X))
            a = rng.uniform(-amp, amp)
            term = np.ones_like(X[0])
            for d, x in enumerate(X):
                term = term * np.sin(2 * np.pi * k[d] * (x - (pb.x0 if d == 0 else pb.y0)) / L[d] + ph[d])
            f = f + a * term
        return f

    if pb.ndim == 1:
        def prim(x):
            return field(1.0, 0.15, x), field(0.5, 0.3, x), field(1.0, 0.15, x)
    else:
        def prim(x, y):
            return field(1.0, 0.15, x, y), field(0.5, 0.3, x, y), field(-0.3, 0.3, x, y), field(1.0, 0.15, x, y)
    return cell_average(pb, prim, npts=6)


def white_noise(pb: Problem, seed: int) -> np.ndarray:
    """Per-cell independent states: rho, p log-uniform [0.1, 10], velocities uniform [-2, 2]."""
    rng = np.random.default_rng(seed)
    shape = (pb.nyc, pb.nx)
    rho = np.exp(rng.uniform(np.log(0.1), np.log(10.0), shape))
    p = np.exp(rng.uniform(np.log(0.1), np.log(10.0), shape))
    u = rng.uniform(-2.0, 2.0, shape)
    if pb.ndim == 1:
        return np.ascontiguousarray(conservative((rho, u, p), pb.gamma, 1))
    v = rng.uniform(-2.0, 2.0, shape)
    return np.ascontiguousarray(conservative((rho, u, v, p), pb.gamma, 2))


def random_sigma(pb: Problem, seed: int, scale: float) -> Tuple[np.ndarray, np.ndarray]:
    """Random face strengths uniform in [0, scale) (scale ~ sigma_thres / 4 straddles the
    threshold in the 4..8-face stencil sums)."""
    rng = np.random.default_rng(seed)
    sx = rng.uniform(0.0, scale, pb.sx_shape)
    sy = rng.uniform(0.0, scale, pb.sy_shape) if pb.ndim == 2 else np.zeros((1, 1))
    if "periodic" in pb.bc[:2]:
        sx[:, -1] = sx[:, 0]  # x-faces 0 and nx are the same face
    if pb.ndim == 2 and "periodic" in pb.bc[2:]:
        sy[-1, :] = sy[0, :]
    return np.ascontiguousarray(sx), np.ascontiguousarray(sy)


def zero_sigma(pb: Problem) -> Tuple[np.ndarray, np.ndarray]:
    return np.zeros(pb.sx_shape), np.zeros(pb.sy_shape)


def batched_problems(seed: int = 20241008, n1: int = 256, n2: int = 256,
                     n1_range=(128, 16384), n2_range=(64, 512)):
    """The batched workload: n1 1D problems with N log-uniform in n1_range and n2 2D N x N
    problems with N log-uniform in n2_range; random Riemann data (rho, p log-uniform
    [0.1, 10], velocities uniform [-2, 2]; 1D: two states split at a random x in
    [0.3, 0.7]; 2D: four quadrants split at (0.5, 0.5)); orders uniform over {3,5,7,9};
    outflow boundaries; CFL 0.5.  Returns a list of (Problem, W)."""
    rng = np.random.default_rng(seed)
    out = []
    for kind, count, (lo, hi) in ((1, n1, n1_range), (2, n2, n2_range)):
        for _ in range(count):
            n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
            order = int(rng.choice([3, 5, 7, 9]))
            sub = int(rng.integers(0, 2 ** 31 - 1))
            if kind == 1:
                out.append(riemann_1d(n, order, sub))
            else:
                out.append(riemann_2d(n, order, sub))
    return out
