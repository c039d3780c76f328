"""Pins of the oracle's reconstruction (Sec. 3 of the paper) against what the paper and
the mathematics fix: the cell-average interpolation problem its coefficient tables
solve, exact reproduction of polynomials, the branch predicates of Eq. (3.2) /
Algorithm 1, the AO identity, the smoothness-indicator definition and Remark 3/4."""
from fractions import Fraction as Fr

import numpy as np
import pytest

pytestmark = []


# ----------------------------------------------------------------------------------
# exact helpers (rational arithmetic; independent of the oracle)
# ----------------------------------------------------------------------------------
def cell_avg_monomial(q, m):
    """Exact mean of xi^q over the stencil cell m = [m-1, m]."""
    return (Fr(m) ** (q + 1) - Fr(m - 1) ** (q + 1)) / (q + 1)


def zero_mean_avg(q, m):
    """Exact mean of Z_q over cell m, with Z_q zero-mean on [-1, 0]."""
    return cell_avg_monomial(q, m) - cell_avg_monomial(q, 0)


STENCIL_CELLS = {0: [-2, -1, 0], 1: [-1, 0, 1], 2: [0, 1, 2], 5: list(range(-2, 3)),
                 7: list(range(-3, 4)), 9: list(range(-4, 5))}


@pytest.mark.parametrize("stencil", [0, 1, 2, 5, 7, 9])
def test_coefficient_tables_solve_cell_average_problem(oracle, stencil):
    """Sec. 3.2-3.4: each printed table (readings G1 basis, G2 '2f_3' = 2W_3) makes
    W_0 + sum_q W_xq Z_q reproduce the cell average of every stencil cell, exactly."""
    num, den = oracle.coef_table(stencil)
    cells = STENCIL_CELLS[stencil]
    assert num.shape[0] == len(cells) - 1
    for t in cells:  # unit data: W_t = 1, others 0
        for m in cells:
            avg = Fr(1 if t == 0 else 0)  # W_0 Z_0
            for q in range(1, len(cells)):
                wxq = Fr(int(num[q - 1, t + 4])) / Fr(int(den[q - 1]))
                avg += wxq * zero_mean_avg(q, m)
            assert avg == Fr(1 if m == t else 0), (stencil, t, m)
    # cells outside the stencil carry no weight
    for q in range(num.shape[0]):
        for t in range(-4, 5):
            if t not in cells:
                assert num[q, t + 4] == 0


def test_zero_mean_basis(oracle):
    x, w = np.polynomial.legendre.leggauss(12)
    xi = 0.5 * (x - 1.0)  # nodes on [-1, 0]
    for q in range(1, 9):
        vals = np.array([oracle.zq(q, v) for v in xi])
        assert abs(np.dot(0.5 * w, vals)) < 1e-15
        # Z_q - xi^q is a constant
        d = vals - xi ** q
        assert np.ptp(d) < 1e-15


@pytest.mark.parametrize("G", [1, 2, 3, 4])
def test_gauss_points_match_legendre(oracle, G):
    t, w = oracle.gauss01(G)
    x, ww = np.polynomial.legendre.leggauss(G)
    np.testing.assert_allclose(t, 0.5 * (x + 1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * ww, rtol=0, atol=1e-15)


def poly_cell_avgs(coeffs, k):
    """Exact cell averages over cells m=-k..k of p(xi) = sum c_q xi^q (Fractions)."""
    return [sum(Fr(c) * cell_avg_monomial(q, m) for q, c in enumerate(coeffs)) for m in range(-k, k + 1)]


def poly_eval(coeffs, x):
    return sum(c * x ** q for q, c in enumerate(coeffs))


GAUSS = {1: [0.5], 2: [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)]}


@pytest.mark.parametrize("r", [3, 5, 7, 9])
def test_linear_branch_reproduces_polynomials(oracle, r):
    """sigma = 0 -> linear r-th order branch: degree r-1 polynomials are reproduced
    exactly at the face (xi = 0), the other face (xi = -1) and interior points."""
    k = (r - 1) // 2
    rng = np.random.default_rng(r)
    xi = np.array([0.0, -1.0, -0.5, -0.2113248654051871, -0.7886751345948129, -0.93])
    for trial in range(5):
        coeffs = [int(c) for c in rng.integers(-9, 10, size=r)]
        vals = np.array([float(v) for v in poly_cell_avgs(coeffs, k)])
        out, br = oracle.reconstruct(r, vals, np.zeros(2 * k), 2.0, xi)
        assert br == {3: 4, 5: 2, 7: 1, 9: 0}[r]
        exact = np.array([poly_eval(coeffs, x) for x in xi])
        scale = max(1.0, np.abs(vals).max())
        np.testing.assert_allclose(out, exact, rtol=0, atol=2e-13 * scale)
    # one degree higher is NOT reproduced (the order is exactly r)
    coeffs = [0] * r + [1]
    vals = np.array([float(v) for v in poly_cell_avgs(coeffs, k)])
    out, _ = oracle.reconstruct(r, vals, np.zeros(2 * k), 2.0, [0.0])
    assert abs(out[0] - 0.0) > 1e-6


def test_branch_selection_follows_algorithm1(oracle):
    """Eq. (3.2) with the predicate A < sigma_thres (G12) and Algorithm 1 capped at r=9
    (G13): place face strengths so that exactly the wanted stencil sum crosses 2.0."""
    r, k = 9, 4
    rng = np.random.default_rng(0)
    coeffs = [int(c) for c in rng.integers(-5, 6, size=9)]
    vals = np.array([float(v) for v in poly_cell_avgs(coeffs, k)])
    # faces m-1/2 for m = -3..4 -> index m+3
    # outermost faces -7/2 (m=-3 -> idx 0) and 7/2 (m=4 -> idx 7) only reach S9
    s = np.zeros(8); s[0] = 1.0; s[7] = 1.0          # A9 = 2.0 exactly -> not smooth
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 1  # lin7
    s = np.zeros(8); s[0] = 0.999; s[7] = 1.0          # A9 < 2 -> lin9
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 0
    s = np.zeros(8); s[1] = 1.0; s[6] = 1.0            # faces -5/2, 5/2: A7 = 2 -> lin5
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 2
    s = np.zeros(8); s[3] = 2.0                         # face -1/2 in S5 -> WENO
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 3
    s = np.zeros(8); s[2] = 1.0; s[5] = 0.999999        # A5 just below 2, nothing else
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 0  # -> the extension reaches lin9
    s[1] = 0.5                                          # now A7 > 2 -> stops at lin5
    assert oracle.reconstruct(r, vals, s, 2.0)[1] == 2
    # order 7 never selects lin9, order 5 never lin7
    s = np.zeros(6)
    assert oracle.reconstruct(7, vals[1:-1], s, 2.0)[1] == 1
    assert oracle.reconstruct(5, vals[2:-2], np.zeros(4), 2.0)[1] == 2
    # order 3 (G20): smooth -> lin3, else DF-damped
    assert oracle.reconstruct(3, vals[3:6], np.zeros(2), 2.0)[1] == 4
    assert oracle.reconstruct(3, vals[3:6], np.array([1.0, 1.0]), 2.0)[1] == 5


def test_lower_branches_reproduce_their_degree(oracle):
    """The lin7 / lin5 branches of the 9th-order scheme use the 7 / 5 centre cells only."""
    k = 4
    for deg, s_idx, br in ((6, (0, 7), 1), (4, (1, 6), 2)):
        coeffs = [1, -2, 3, 1, -1, 2, 1][: deg + 1]
        vals = np.array([float(v) for v in poly_cell_avgs(coeffs, k)])
        vals[0] += 1e3 if deg == 4 else 0.0  # outer cells must not matter
        vals[-1] -= 1e3 if deg == 4 else 0.0
        s = np.zeros(8); s[s_idx[0]] = 1.5; s[s_idx[1]] = 1.5
        out, b = oracle.reconstruct(9, vals, s, 2.0, [0.0, -1.0])
        assert b == br
        np.testing.assert_allclose(out, [poly_eval(coeffs, 0.0), poly_eval(coeffs, -1.0)], atol=1e-12)


def test_weno_ao_identity(oracle):
    """Sec. 3.2: with the nonlinear weights replaced by the linear ones and alpha = 1 the
    AO combination is exactly the 5th-order polynomial."""
    rng = np.random.default_rng(3)
    xi = [0.0, -1.0, -0.3]
    for _ in range(10):
        v = rng.normal(size=5)
        out, _ = oracle.weno_ao53(v, [1, 1, 1, 1], xi, force_linear_weights=True)
        ref, br = oracle.reconstruct(5, v, np.zeros(4), 2.0, xi)
        assert br == 2
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14 * max(1, np.abs(v).max()))


def test_weno_limits(oracle):
    """Remark 4: alpha -> 0 gives the first-order value W_0; constant data gives W_0 for
    any alpha; linear data (equal betas, tau = 0) keeps the linear weights and is exact."""
    rng = np.random.default_rng(4)
    for _ in range(10):
        v = rng.normal(size=5)
        out, _ = oracle.weno_ao53(v, [1e-300] * 4, [0.0, -1.0, -0.5])
        np.testing.assert_allclose(out, v[2], rtol=0, atol=1e-14)
        c = rng.normal()
        out, beta = oracle.weno_ao53([c] * 5, rng.uniform(0.01, 1, 4), [0.0, -0.4])
        np.testing.assert_allclose(out, c, rtol=0, atol=1e-15 * max(1, abs(c)))
        assert np.all(np.abs(beta) <= 1e-28 * max(1.0, c * c))
    # linear data: cell averages of a + b xi are a + b (m - 1/2)
    a, b = 0.7, -1.3
    v = np.array([a + b * (m - 0.5) for m in range(-2, 3)])
    out, beta = oracle.weno_ao53(v, [1, 1, 1, 1], [0.0, -1.0])
    np.testing.assert_allclose(beta[:4], b * b, rtol=1e-14)
    assert beta[4] < 1e-14
    np.testing.assert_allclose(out, [a, a - b], rtol=1e-14)


def test_weno_picks_smooth_substencil_at_a_jump(oracle):
    """The WENO-Z weights make the AO polynomial follow the one smooth 3-cell
    sub-stencil next to a jump (the essentially non-oscillatory property)."""
    out, beta = oracle.weno_ao53([0, 0, 0, 1, 1], [1, 1, 1, 1], [0.0])
    assert beta[0] == 0.0 and beta[1] > 1 and beta[2] > 1
    assert abs(out[0]) < 1e-9
    out, beta = oracle.weno_ao53([1, 1, 0, 0, 0], [1, 1, 1, 1], [0.0])
    assert beta[2] == 0.0
    assert abs(out[0]) < 1e-9


def beta_by_definition(a1, a2):
    """Eq. (LocalSmoothnessIndicator) for P = W_0 + a1 Z_1 + a2 Z_2 in the local
    coordinate: int_{-1}^{0} (P')^2 + (P'')^2, integrated with Gauss-Legendre."""
    x, w = np.polynomial.legendre.leggauss(8)
    xi = 0.5 * (x - 1.0)
    d1 = a1 + 2.0 * a2 * xi
    return float(np.dot(0.5 * w, d1 * d1)) + (2.0 * a2) ** 2


def test_beta_matches_its_definition(oracle):
    rng = np.random.default_rng(5)
    for _ in range(20):
        v = rng.normal(size=5)
        _, beta = oracle.weno_ao53(v, [1, 1, 1, 1], [0.0])
        for k, s in enumerate((0, 1, 2)):
            num, den = oracle.coef_table(s)
            a1 = float(np.dot(num[0, 2:7], v)) / den[0]
            a2 = float(np.dot(num[1, 2:7], v)) / den[1]
            assert abs(beta[k] - beta_by_definition(a1, a2)) < 1e-12 * max(1, beta[k])
        # the simple 5-cell indicator and tau_Z as defined in Sec. 3.2 (reading G5)
        b = beta[:3]
        b5 = (b[0] + 4 * b[1] + b[2]) / 6 + abs(b[0] - b[2])
        assert abs(beta[3] - b5) < 1e-13 * max(1, b5)
        tau = (abs(b5 - b[0]) + abs(b5 - b[1]) + abs(b5 - b[2])) / 3
        assert abs(beta[4] - tau) < 1e-13 * max(1, b5)


def test_beta_remark3_leading_terms(oracle):
    """Remark 3: beta3_k = W'^2 dx^2 + 13/12 W''^2 dx^4 + ...; for a quadratic centred on
    the cell (W' = 0 there) every beta3_k and beta5_bar is exactly 13/12 W''^2 dx^4."""
    for h in (0.1, 0.05):
        A = 3.0  # W = A (x - x_c)^2, W'' = 2A
        # cell m (width h) centred at (m - 1/2) h relative to cell 0's centre at -h/2
        v = np.array([A * (((m - 0.5) * h + 0.5 * h) ** 2 + h * h / 12.0) for m in range(-2, 3)])
        _, beta = oracle.weno_ao53(v, [1, 1, 1, 1], [0.0])
        np.testing.assert_allclose(beta[:4], 13.0 / 12.0 * (2 * A) ** 2 * h ** 4, rtol=1e-12)
    # smooth data: beta / dx^2 -> W'^2 with an O(dx^2) error
    errs = []
    for h in (0.02, 0.01):
        xc = 0.3
        v = np.array([(np.cos(xc + (m - 1) * h) - np.cos(xc + m * h)) / h for m in range(-2, 3)])
        # cell averages of sin over [(m-1)h, mh] shifted so cell 0 is centred at xc - h/2
        _, beta = oracle.weno_ao53(v, [1, 1, 1, 1], [0.0])
        wp = np.cos(xc - 0.5 * h)
        errs.append(abs(beta[1] / h ** 2 - wp ** 2))
    assert errs[1] < errs[0] / 3.0


def test_weno_reconstruction_is_mirror_equivariant(oracle):
    """The reflection x -> -x maps cell 0 = [-1, 0] onto itself (xi -> -1 - xi), reverses
    the stencil and swaps the DF factors of S3_{-1} and S3_1. A reconstruction has no
    preferred direction, so the WENOZ-AO(5,3)+DF value must commute with it. With the linear
    weights d3_{-1} = d3_1 this holds only if the global indicator tau_Z treats beta3_{-1}
    and beta3_1 alike (reading G5); the printed form, with |beta5 - beta3_1| twice and no
    beta3_0 term, breaks it by O(1) on rough data."""
    rng = np.random.default_rng(12)
    xi = np.array([0.0, -1.0, -0.3, -0.5, -0.8873])
    cases = [rng.normal(size=5) for _ in range(150)]
    cases += [np.array([0, 0, 0, 1, 1.0]), np.array([1, 2, 2, 2, 7.0]), np.array([0.1, 10, 0.1, 0.1, 0.2])]
    cases += [rng.lognormal(size=5) * rng.choice([1e-3, 1.0, 1e3]) for _ in range(50)]
    swapped = 0
    for v in cases:
        alpha = rng.uniform(0.02, 1.0, 4)
        if rng.uniform() < 0.3:
            alpha[:] = 1.0
        out, beta = oracle.weno_ao53(v, alpha, xi)
        outm, betam = oracle.weno_ao53(v[::-1].copy(), alpha[[2, 1, 0, 3]].copy(), -1.0 - xi)
        scale = np.abs(v).max()
        # the indicators are mirror images of each other (beta3_{-1} <-> beta3_1)
        np.testing.assert_allclose(betam[[2, 1, 0, 3, 4]], beta, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(outm, out, rtol=0, atol=1e-13 * scale)
        swapped += abs(beta[0] - beta[2]) > 0.1 * max(beta[0], beta[2])
    assert swapped > 100  # most cases have clearly different beta3_{-1} and beta3_1


def _sine_averages(F, x0, h):
    """Cell averages over the five cells [x0 + (m-1)h, x0 + m h], m = -2..2, of f = F';
    cell 0 is [x0 - h, x0] and its right face is x0."""
    return np.array([(F(x0 + m * h) - F(x0 + (m - 1) * h)) / h for m in range(-2, 3)])


@pytest.mark.parametrize("profile", ["monotone", "extremum_at_face", "extremum_inside_stencil"])
def test_weno_fallback_is_fifth_order_on_smooth_data(oracle, profile):
    """Sec. 3.2: the WENOZ-AO(5,3) combination with alpha = 1 reaches fifth order at the
    face in smooth regions, also next to a critical point (f' = 0), where a global indicator
    tau_Z that is not a difference of the betas, or weights that react to beta3_k alone,
    fall back to third order."""
    f, F, x0 = {
        "monotone": (np.sin, lambda x: -np.cos(x), 0.3),
        "extremum_at_face": (np.cos, np.sin, 0.0),
        "extremum_inside_stencil": (np.cos, np.sin, 0.05),
    }[profile]
    hs = np.array([0.2, 0.1, 0.05, 0.025, 0.0125])
    errs = []
    for h in hs:
        out, _ = oracle.weno_ao53(_sine_averages(F, x0, h), [1, 1, 1, 1], [0.0])
        errs.append(abs(out[0] - f(x0)))
    # error / h^5 stays bounded (third order would grow it 256-fold from h = 0.2 to 0.0125);
    # a fitted slope is not used because the error changes sign near the extremum
    ratio = np.array(errs) / hs ** 5
    assert ratio[2:].max() <= 4.0 * ratio[:2].max(), ratio
    assert errs[-1] < 1e-11


def test_weno_epsilon_sets_the_linear_amplitude(oracle):
    """The absolute epsilon = 1e-6 of the WENO-Z weights (Sec. 3.2, reading G22) fixes the
    amplitude below which the fallback stays on the linear weights: a step of height delta
    has beta ~ delta^2, so for delta = 1e-4 (beta ~ 1e-8, far below epsilon) the value is the
    linear fifth-order one, 0.4 delta above the base (weights (2, -13, 47, 27, -3)/60 on
    (0, 0, 0, 1, 1)), while for delta = 1e-2 (beta ~ 1e-4, far above epsilon) the weights are
    non-oscillatory and the value stays on the smooth side of the step. A much smaller
    epsilon makes both non-oscillatory; a much larger one makes both linear."""
    base = 2.5
    step = np.array([0, 0, 0, 1, 1.0])
    for delta, expect, tol in ((1e-4, 0.4, 1e-3), (1e-5, 0.4, 1e-5), (1e-2, 0.0, 2e-3), (1.0, 0.0, 1e-9)):
        out, beta = oracle.weno_ao53(base + delta * step, [1, 1, 1, 1], [0.0])
        assert abs((out[0] - base) / delta - expect) < tol, (delta, (out[0] - base) / delta)
