"""The roofline's flop model against the oracle's operation counter.

bench.py counts, per Gauss point, both sides' primitives, the Lax-Friedrichs flux
1/2 (F_L + F_R - lambda (q_R - q_L)) and sigma (Sec. 2.3, Sec. 3.1).  The oracle's op-counting
build performs the same steps but scales both halves of the flux by 1/2, one multiplication
per component more; its count of one point is data-independent on physical states."""
import numpy as np
import pytest

import bench
from oracle import oracle as O


def _count_point(C, qL, qR):
    import ctypes

    lib = O._lib(True)
    F = np.empty(C)
    s = np.empty(1)
    lib.oracle_reset_op_counts()
    fb = lib.oracle_lf_flux(C, 1.4, O._ptr(qL), O._ptr(qR), O._ptr(qL), O._ptr(qR), O._ptr(F), O._ptr(s))
    assert fb == 0  # physical states: no first-order fallback
    out = (ctypes.c_longlong * 4)()
    lib.oracle_op_counts(out)
    return sum(out)


@pytest.mark.parametrize("ndim", [1, 2])
def test_gauss_point_flops_are_the_oracles_count_less_one_half_per_component(ndim):
    C = 4 if ndim == 2 else 3
    rng = np.random.default_rng(7)
    counts = set()
    for _ in range(5):
        rho = rng.uniform(0.5, 2.0, 2)
        p = rng.uniform(0.5, 2.0, 2)
        u = rng.uniform(-1.0, 1.0, (2, C - 2))
        q = [np.concatenate(([rho[k]], rho[k] * u[k], [p[k] / 0.4 + 0.5 * rho[k] * np.sum(u[k] ** 2)]))
             for k in range(2)]
        counts.add(_count_point(C, q[0], q[1]))
    assert len(counts) == 1
    assert bench.GAUSS_POINT_FLOPS[ndim] == counts.pop() - C


def test_face_flops_of_the_roofline():
    # 2D, per face of one sweep: 2 C (2r-1) + 2 C G (2r-1) + G (70 + 2 C + 1) + 1
    assert [bench.algorithmic_flops_per_face(2, r) for r in (3, 5, 7, 9)] == [160, 375, 654, 997]


def test_gks_face_flops_of_the_roofline():
    # 2D, per face of one sweep: 4 C (2r-1) + 2 C + 2 C G (3 (2r-1) + 1) + G (1365 + 43 + 4 C + 1) + 1
    assert [bench.gks_flops_per_face(2, r) for r in (3, 5, 7, 9)] == [1642, 3451, 5452, 7645]
    # 1D: 4 C (2r-1) + 2 C + 598 + 32 + 4 C + 1 + 1
    assert [bench.gks_flops_per_face(1, r) for r in (3, 5, 7, 9)] == [710, 758, 806, 854]


@pytest.mark.parametrize("r", [5, 7, 9])
def test_vjp_edges_per_operation_of_the_adjoint_model(r):
    """The residual adjoint's flop model scales the forward's algorithmic flops by
    1 + 2 e, e the edges per operation of the reverse-mode graph (one multiply-add per edge in
    the reverse sweep); e is the oracle tape's on smooth 2D data."""
    from paper_2410_05489_gb300 import problems as P

    pb = P.Problem(ndim=2, nx=32, ny=32, order=r, bc=("periodic",) * 4, x1=2.0, y1=2.0)
    W = P.smooth_random(pb, 3)
    sx, sy = P.zero_sigma(pb)
    O.residual_vjp(pb, W, sx, sy, np.random.default_rng(1).normal(size=W.shape))
    edges = O.last_vjp_edges()
    ops = sum(O.op_counts_residual(pb, W, sx, sy))
    assert abs(bench.VJP_EDGES_PER_OP[r] - edges / ops) < 1e-3 * bench.VJP_EDGES_PER_OP[r]


# ----------------------------------------------------------------------------------
# Gas-kinetic Gauss point (Sec. 2.2, Appendix A)
# ----------------------------------------------------------------------------------
class _Op:
    """A float that counts the FP64 operations done on it (add, sub, mul, div: 1 each;
    sqrt, exp, erfc: 1 each). Operations with a literal 0 or 1 are free (a compiler folds them),
    and so are those between literals (per-launch constants such as gamma, dt, C1)."""

    n = 0

    def __init__(self, v):
        self.v = float(v)

    @staticmethod
    def _v(x):
        return x.v if isinstance(x, _Op) else float(x)

    def _bin(self, o, f, ident_l, ident_r):
        if not isinstance(o, _Op):
            if o in ident_r:
                return ident_r[o](self)
        _Op.n += 1
        return _Op(f(self.v, _Op._v(o)))

    def __add__(self, o):
        return self._bin(o, lambda a, b: a + b, None, {0.0: lambda s: s})

    def __radd__(self, o):
        return self.__add__(o)

    def __sub__(self, o):
        return self._bin(o, lambda a, b: a - b, None, {0.0: lambda s: s})

    def __rsub__(self, o):
        if o == 0.0:
            return -self
        _Op.n += 1
        return _Op(float(o) - self.v)

    def __mul__(self, o):
        return self._bin(o, lambda a, b: a * b, None, {1.0: lambda s: s, 0.0: lambda s: 0.0})

    def __rmul__(self, o):
        return self.__mul__(o)

    def __truediv__(self, o):
        return self._bin(o, lambda a, b: a / b, None, {1.0: lambda s: s})

    def __rtruediv__(self, o):
        _Op.n += 1
        return _Op(float(o) / self.v)

    def __neg__(self):
        return _Op(-self.v)

    def __abs__(self):
        return _Op(abs(self.v))


def _fn(f):
    def g(x):
        if not isinstance(x, _Op):
            return f(x)
        _Op.n += 1
        return _Op(f(x.v))
    return g


_sqrt, _exp = _fn(np.sqrt), _fn(np.exp)
_erfc = _fn(lambda x: float(__import__("math").erfc(x)))


def _maxwellian(W, dim, gamma, K):
    """Moments of the Maxwellian of W (Appendix A): <u^n> (n <= 6), <v^n> (n <= 5), <xi^(2l)>."""
    rho = W[0]
    ir = 1.0 / rho
    U = W[1] * ir
    V = W[2] * ir if dim == 2 else 0.0
    p = (gamma - 1.0) * (W[dim + 1] - 0.5 * rho * (U * U + V * V))
    h = p * ir  # 1 / (2 lambda)
    m = {"rho": rho, "ir": ir, "U": U, "V": V, "h": h, "lam": 0.5 / h}
    mu = [1.0, U]
    for n in range(5):
        mu.append(U * mu[n + 1] + ((n + 1) * h) * mu[n])
    mv = [1.0, V] + [0.0] * 4
    if dim == 2:
        for n in range(4):
            mv[n + 2] = V * mv[n + 1] + ((n + 1) * h) * mv[n]
    m["mu"], m["mv"] = mu, mv
    m["mx"] = [1.0, K * h, (K + 2.0) * h * (K * h)]
    m["dx4"] = 2.0 * K * h * h
    return m


def _half(m, pos):
    """<u^n> of the Maxwellian over u > 0 (pos) or u < 0, n <= 6."""
    lam, U, h = m["lam"], m["U"], m["h"]
    isl = 1.0 / _sqrt(lam)
    sl = lam * isl
    e = 0.28209479177387814 * _exp(-(lam * U * U)) * isl
    mh = [0.5 * _erfc(-(sl * U) if pos else sl * U)]
    mh.append(U * mh[0] + e if pos else U * mh[0] - e)
    for n in range(5):
        mh.append(U * mh[n + 1] + ((n + 1) * h) * mh[n])
    return mh


def _mom1(i, s, t, mu, m, dim):
    """<u^s v^t psi_i> with the u moments mu."""
    mv, mx = m["mv"], m["mx"]

    def M(a, b, l):
        return mu[a] * mv[b] * mx[l]

    if dim == 2:
        return [lambda: M(s, t, 0), lambda: M(s + 1, t, 0), lambda: M(s, t + 1, 0),
                lambda: 0.5 * (M(s + 2, t, 0) + M(s, t + 2, 0) + M(s, t, 1))][i]()
    return [lambda: M(s, 0, 0), lambda: M(s + 1, 0, 0), lambda: 0.5 * (M(s + 2, 0, 0) + M(s, 0, 1))][i]()


def _slope_moments(a, s, t, mu, m, dim):
    """rho <u^s v^t psi (psi . a)>, the u, v and xi moments factored."""
    mv, mx, rho = m["mv"], m["mx"], m["rho"]
    if dim == 2:
        a3h = 0.5 * a[3]
        a0p = a3h * mx[1] + a[0]
        A = [a3h * mu[s + k + 2] + (a[1] * mu[s + k + 1] + a0p * mu[s + k]) for k in range(3)]
        B = [a3h * mv[t + k + 2] + a[2] * mv[t + k + 1] for k in range(3)]
        P00 = mv[t] * A[0] + mu[s] * B[0]
        P10 = mv[t] * A[1] + mu[s + 1] * B[0]
        P01 = mv[t + 1] * A[0] + mu[s] * B[1]
        P20 = mv[t] * A[2] + mu[s + 2] * B[0]
        P02 = mv[t + 2] * A[0] + mu[s] * B[2]
        Px = mx[1] * P00 + a3h * m["dx4"] * (mu[s] * mv[t])
        return [rho * P00, rho * P10, rho * P01, 0.5 * rho * (P20 + P02 + Px)]
    a2h = 0.5 * a[2]
    a0p = a2h * mx[1] + a[0]
    A = [a2h * mu[s + k + 2] + (a[1] * mu[s + k + 1] + a0p * mu[s + k]) for k in range(3)]
    Px = mx[1] * A[0] + a2h * m["dx4"] * mu[s]
    return [rho * A[0], rho * A[1], 0.5 * rho * (A[2] + Px)]


def _solve_slope(m, D, b, dim):
    """a with <psi psi^T> a = b, closed form (Appendix A)."""
    l, U, V = m["lam"], m["U"], m["V"]
    i4D = 4.0 / D
    if dim == 2:
        q = U * U + V * V + D * m["h"]
        R4, R3, R2 = 2.0 * b[3] - q * b[0], b[2] - V * b[0], b[1] - U * b[0]
        a3 = i4D * l * l * (R4 - 2.0 * U * R2 - 2.0 * V * R3)
        a2 = 2.0 * l * R3 - V * a3
        a1 = 2.0 * l * R2 - U * a3
        return [b[0] - U * a1 - V * a2 - 0.5 * a3 * q, a1, a2, a3]
    q = U * U + D * m["h"]
    R3, R2 = 2.0 * b[2] - q * b[0], b[1] - U * b[0]
    a2 = i4D * l * l * (R3 - 2.0 * U * R2)
    a1 = 2.0 * l * R2 - U * a2
    return [b[0] - U * a1 - 0.5 * a2 * q, a1, a2]


def _gks_point_closed_form(dim, gamma, Wl, Wlx, Wly, Wr, Wrx, Wry, dt, C1, C2):
    """The gas-kinetic flux of one Gauss point (face frame), F and F_t, in closed form."""
    n = dim + 2
    K = (4.0 - 2.0 * gamma) / (gamma - 1.0) if dim == 2 else (3.0 - gamma) / (gamma - 1.0)
    D = K + dim
    gl, gr = _maxwellian(Wl, dim, gamma, K), _maxwellian(Wr, dim, gamma, K)
    alx = _solve_slope(gl, D, [Wlx[i] * gl["ir"] for i in range(n)], dim)
    arx = _solve_slope(gr, D, [Wrx[i] * gr["ir"] for i in range(n)], dim)
    if dim == 2:
        aly = _solve_slope(gl, D, [Wly[i] * gl["ir"] for i in range(n)], dim)
        ary = _solve_slope(gr, D, [Wry[i] * gr["ir"] for i in range(n)], dim)
    mlp, mrn = _half(gl, True), _half(gr, False)
    Wc = [gl["rho"] * _mom1(i, 0, 0, mlp, gl, dim) + gr["rho"] * _mom1(i, 0, 0, mrn, gr, dim) for i in range(n)]
    t1, t2 = _slope_moments(alx, 0, 0, mlp, gl, dim), _slope_moments(arx, 0, 0, mrn, gr, dim)
    Wcx = [t1[i] + t2[i] for i in range(n)]
    if dim == 2:
        t1, t2 = _slope_moments(aly, 0, 0, mlp, gl, dim), _slope_moments(ary, 0, 0, mrn, gr, dim)
        Wcy = [t1[i] + t2[i] for i in range(n)]
    gc = _maxwellian(Wc, dim, gamma, K)
    acx = _solve_slope(gc, D, [Wcx[i] * gc["ir"] for i in range(n)], dim)
    if dim == 2:
        acy = _solve_slope(gc, D, [Wcy[i] * gc["ir"] for i in range(n)], dim)
    t1 = _slope_moments(acx, 1, 0, gc["mu"], gc, dim)
    if dim == 2:
        t2 = _slope_moments(acy, 0, 1, gc["mu"], gc, dim)
        b = [-(t1[i] + t2[i]) * gc["ir"] for i in range(n)]
    else:
        b = [-t1[i] * gc["ir"] for i in range(n)]
    Ac = _solve_slope(gc, D, b, dim)
    T0 = [gc["rho"] * _mom1(i, 1, 0, gc["mu"], gc, dim) for i in range(n)]
    T3 = [gl["rho"] * _mom1(i, 1, 0, mlp, gl, dim) + gr["rho"] * _mom1(i, 1, 0, mrn, gr, dim) for i in range(n)]
    T1 = _slope_moments(acx, 2, 0, gc["mu"], gc, dim)
    T2 = _slope_moments(Ac, 1, 0, gc["mu"], gc, dim)
    t1, t2 = _slope_moments(alx, 2, 0, mlp, gl, dim), _slope_moments(arx, 2, 0, mrn, gr, dim)
    T4 = [t1[i] + t2[i] for i in range(n)]
    if dim == 2:
        t1 = _slope_moments(acy, 1, 1, gc["mu"], gc, dim)
        T1 = [T1[i] + t1[i] for i in range(n)]
        t1, t2 = _slope_moments(aly, 1, 1, mlp, gl, dim), _slope_moments(ary, 1, 1, mrn, gr, dim)
        T4 = [T4[i] + (t1[i] + t2[i]) for i in range(n)]
    pl, pr = gl["rho"] * gl["h"], gr["rho"] * gr["h"]
    taun = C1 * dt + C2 * (abs(pl - pr) / (pl + pr)) * dt
    eh = _exp(-((0.5 * dt) / taun))
    Fd = []
    for k in range(2):
        d = dt if k == 0 else 0.5 * dt
        e = eh * eh if k == 0 else eh
        ome = 1.0 - e
        c1 = d - taun * ome
        c2 = taun * taun * ome - taun * d * e
        c3 = 0.5 * d * d
        c4 = taun * ome
        Fd.append([c1 * T0[i] + c2 * (T1[i] - T4[i]) + c3 * T2[i] + c4 * T3[i] for i in range(n)])
    idt = 1.0 / dt
    F = [(4.0 * Fd[1][i] - Fd[0][i]) * idt for i in range(n)]
    Ft = [4.0 * (Fd[0][i] - 2.0 * Fd[1][i]) * idt * idt for i in range(n)]
    return F, Ft


def _sigma_point(qa, qb, gamma, C):
    """sigma of one Gauss point (Sec. 3.1) from the two conservative states (face frame)."""
    ia, ib = 1.0 / qa[0], 1.0 / qb[0]
    ua, ub = qa[1] * ia, qb[1] * ib
    wa, wb = (qa[2] * ia, qb[2] * ib) if C == 4 else (0.0, 0.0)
    pa = (gamma - 1.0) * (qa[C - 1] - 0.5 * qa[0] * (ua * ua + wa * wa))
    pb = (gamma - 1.0) * (qb[C - 1] - 0.5 * qb[0] * (ub * ub + wb * wb))
    ica, icb = 1.0 / _sqrt(gamma * pa * ia), 1.0 / _sqrt(gamma * pb * ib)
    dmn = ua * ica - ub * icb
    s = abs(pa - pb) * (1.0 / pa + 1.0 / pb) + dmn * dmn
    if C == 4:
        dmt = wa * ica - wb * icb
        s = s + dmt * dmt
    return s


def _gks_inputs(rng, dim):
    n = dim + 2
    states = []
    for _ in range(2):
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        u = rng.uniform(-1.0, 1.0, dim)
        W = np.concatenate(([rho], rho * u, [p / 0.4 + 0.5 * rho * np.sum(u ** 2)]))
        states.append((W, rng.normal(0.0, 0.3, n), rng.normal(0.0, 0.3, n) if dim == 2 else np.zeros(n)))
    return states


@pytest.mark.parametrize("dim", [1, 2])
def test_gks_point_flops_count_a_closed_form_that_gives_the_oracles_flux(dim):
    """bench.GKS_POINT_FLOPS counts one closed-form evaluation of the gas-kinetic Gauss point.
    That evaluation gives the oracle's F and F_t (which solves the slope systems by elimination
    and integrates generic moment polynomials), and its count is data-independent."""
    rng = np.random.default_rng(11)
    counts = set()
    for _ in range(5):
        (Wl, Wlx, Wly), (Wr, Wrx, Wry) = _gks_inputs(rng, dim)
        dt = 1e-3
        F_ref, Ft_ref = O.gks_point(dim, 1.4, Wl, Wlx, Wly, Wr, Wrx, Wry, dt)
        _Op.n = 0
        wrap = [[_Op(x) for x in a] for a in (Wl, Wlx, Wly, Wr, Wrx, Wry)]
        F, Ft = _gks_point_closed_form(dim, 1.4, *wrap, dt, 0.05, 1.0)
        counts.add(_Op.n)
        F, Ft = np.array([f.v for f in F]), np.array([f.v for f in Ft])
        assert np.allclose(F, F_ref, rtol=1e-10, atol=1e-10 * np.abs(F_ref).max())
        assert np.allclose(Ft, Ft_ref, rtol=1e-8, atol=1e-8 * np.abs(Ft_ref).max())
    assert len(counts) == 1
    assert bench.GKS_POINT_FLOPS[dim] == counts.pop()


@pytest.mark.parametrize("dim", [1, 2])
def test_sigma_point_flops_count_the_oracles_sigma(dim):
    """bench.SIGMA_POINT_FLOPS counts sigma of one Gauss point (Sec. 3.1) from the two
    conservative states; the value is the oracle's (which returns it with the L-F flux)."""
    C = dim + 2
    rng = np.random.default_rng(12)
    counts = set()
    for _ in range(5):
        (qa, _, _), (qb, _, _) = _gks_inputs(rng, dim)
        F = np.empty(C)
        s_ref = np.empty(1)
        O._lib().oracle_lf_flux(C, 1.4, O._ptr(qa), O._ptr(qb), O._ptr(qa), O._ptr(qb), O._ptr(F), O._ptr(s_ref))
        _Op.n = 0
        s = _sigma_point([_Op(x) for x in qa], [_Op(x) for x in qb], 1.4, C)
        counts.add(_Op.n)
        assert abs(s.v - s_ref[0]) <= 1e-13 * abs(s_ref[0])
    assert len(counts) == 1
    assert bench.SIGMA_POINT_FLOPS[dim] == counts.pop()
