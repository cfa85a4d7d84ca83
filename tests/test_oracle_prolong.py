"""Pins of the oracle's prolongations (Section 3.1, 3.2).

Pi (new extrapolation): the printed 1-D and 2-D cases, and exactness on the
error model the extrapolation assumes (u^{l-1} = U + C h^2, u^{l-2} = U +
C (2h)^2 with C bilinear gives U + C (h/2)^2 at every level-(l-1) node; this
is what pins the cell-centre value, which the paper does not print).
P (quadratic interpolation): exact on biquadratic polynomials; P(Pi(.))
reproduces the paper's expanded 1-D quarter-point formulas.
L (Eq. 15): the four printed cases.
"""
import numpy as np
import pytest


def grid_sizes(orc, h, w, L=3):
    return orc.level_sizes(h, w, L)


def test_pi_printed_one_dimensional_cases(orc):
    """1-D (a one-row image): coarse nodes (5u2 - u1)/4, midpoints u2 + ((u2-u1)_i + (u2-u1)_{i+1})/8."""
    rng = np.random.default_rng(20)
    n2 = 9  # level l-1 (the paper's G_2), 2^3 + 1 nodes
    n1 = 5  # level l-2 (G_1)
    u2 = rng.uniform(0, 255, (1, n2))
    u1 = rng.uniform(0, 255, (1, n1))
    out = orc.extrapolate(u2, u1)
    for i in range(n1):
        assert out[0, 2 * i] == pytest.approx((5 * u2[0, 2 * i] - u1[0, i]) / 4, rel=1e-15)
    for i in range(n1 - 1):
        exp = u2[0, 2 * i + 1] + ((u2[0, 2 * i] - u1[0, i]) + (u2[0, 2 * i + 2] - u1[0, i + 1])) / 8
        assert out[0, 2 * i + 1] == pytest.approx(exp, rel=1e-14)


def test_pi_printed_two_dimensional_cases(orc):
    rng = np.random.default_rng(21)
    h1, w1, h2, w2 = 9, 17, 5, 9
    u1 = rng.uniform(0, 255, (h1, w1))  # u^{l-1}
    u2 = rng.uniform(0, 255, (h2, w2))  # u^{l-2}
    out = orc.extrapolate(u1, u2)
    d = lambda A, B: u1[2 * A, 2 * B] - u2[A, B]
    for A in range(h2):
        for B in range(w2):
            assert out[2 * A, 2 * B] == pytest.approx((5 * u1[2 * A, 2 * B] - u2[A, B]) / 4, rel=1e-14)
            if B + 1 < w2:  # (i, j + 1/2)
                exp = u1[2 * A, 2 * B + 1] + (d(A, B) + d(A, B + 1)) / 8
                assert out[2 * A, 2 * B + 1] == pytest.approx(exp, rel=1e-14)
            if A + 1 < h2:  # (i + 1/2, j)
                exp = u1[2 * A + 1, 2 * B] + (d(A, B) + d(A + 1, B)) / 8
                assert out[2 * A + 1, 2 * B] == pytest.approx(exp, rel=1e-14)


@pytest.mark.parametrize("h1,w1", [(9, 9), (17, 9), (5, 33)])
def test_pi_exact_on_its_error_model(orc, h1, w1):
    """u1 = U + C h^2 and u2 = U + 4 C h^2 (C bilinear) give U + C h^2 / 4 at all level-(l-1) nodes."""
    rng = np.random.default_rng(22)
    h2, w2 = (h1 + 1) // 2, (w1 + 1) // 2
    a, b, c, e = rng.uniform(-1, 1, 4)
    yy, xx = np.indices((h1, w1)).astype(float)
    C1 = a + b * yy + c * xx + e * yy * xx        # C at level-(l-1) nodes
    C2 = C1[::2, ::2]                             # C at level-(l-2) nodes (same points)
    U1 = rng.uniform(0, 255, (h1, w1))
    hsq = 0.37
    u1 = U1 + C1 * hsq
    u2 = U1[::2, ::2] + C2 * 4 * hsq
    out = orc.extrapolate(u1, u2)
    assert np.allclose(out, U1 + C1 * hsq / 4, rtol=0, atol=1e-12)


@pytest.mark.parametrize("h,w", [(17, 17), (33, 9), (9, 65)])
def test_quadratic_exact_on_biquadratics(orc, h, w):
    """x^a y^b (a, b <= 2) sampled at level-(l-1) nodes are reproduced at every level-l pixel."""
    h1, w1 = (h + 1) // 2, (w + 1) // 2
    yy1, xx1 = np.indices((h1, w1)).astype(float) * 2.0  # node a sits at fine coordinate 2a
    yy, xx = np.indices((h, w)).astype(float)
    for pa in range(3):
        for pb in range(3):
            f1 = (yy1 ** pa) * (xx1 ** pb)
            f = (yy ** pa) * (xx ** pb)
            out = orc.quadratic(f1, h, w)
            assert np.allclose(out, f, rtol=1e-13, atol=1e-9), (pa, pb)


def test_quadratic_printed_weights(orc):
    """Section 3.2: quarter points 3/8, 3/4, -1/8 and mirror; nodes copied."""
    rng = np.random.default_rng(23)
    ut = rng.uniform(0, 255, (1, 5))  # triplets (0,1,2), (2,3,4)
    out = orc.quadratic(ut, 1, 9)
    for A in range(2):
        i, m, j = ut[0, 2 * A], ut[0, 2 * A + 1], ut[0, 2 * A + 2]
        assert out[0, 4 * A] == i
        assert out[0, 4 * A + 2] == m
        assert out[0, 4 * A + 1] == pytest.approx(3 / 8 * i + 3 / 4 * m - 1 / 8 * j, rel=1e-14)
        assert out[0, 4 * A + 3] == pytest.approx(-1 / 8 * i + 3 / 4 * m + 3 / 8 * j, rel=1e-14)
    assert out[0, 8] == ut[0, 4]


def test_pi_then_p_matches_printed_expanded_form(orc):
    """Section 3.2 (1-D): u^3_{i+1/4} = (1/16)[(9u^2_i + 12u^2_{i+1/2} - u^2_{i+1}) - (3u^1_i + u^1_{i+1})].

    The expanded form uses the un-extrapolated level-(l-1) midpoint value, so
    this also checks the reading that P acts on Pi's output.
    """
    rng = np.random.default_rng(24)
    u2 = rng.uniform(0, 255, (1, 9))
    u1 = rng.uniform(0, 255, (1, 5))
    out = orc.quadratic(orc.extrapolate(u2, u1), 1, 17)
    for i in range(4):
        a, m, b = u2[0, 2 * i], u2[0, 2 * i + 1], u2[0, 2 * i + 2]
        c0, c1 = u1[0, i], u1[0, i + 1]
        q1 = ((9 * a + 12 * m - b) - (3 * c0 + c1)) / 16
        q3 = ((9 * b + 12 * m - a) - (3 * c1 + c0)) / 16
        assert out[0, 4 * i + 1] == pytest.approx(q1, rel=1e-13)
        assert out[0, 4 * i + 3] == pytest.approx(q3, rel=1e-13)


def test_pi_then_p_matches_printed_two_dimensional_rows(orc):
    """Section 3.2 (2-D), row direction (i, j + 1/4) and (i, j + 3/4), with the 1-D reading of the midpoint."""
    rng = np.random.default_rng(25)
    u1 = rng.uniform(0, 255, (5, 9))   # u^{l-1}
    u2 = rng.uniform(0, 255, (3, 5))   # u^{l-2}
    out = orc.quadratic(orc.extrapolate(u1, u2), 9, 17)
    for A in range(3):
        for B in range(4):
            a, m, b = u1[2 * A, 2 * B], u1[2 * A, 2 * B + 1], u1[2 * A, 2 * B + 2]
            c0, c1 = u2[A, B], u2[A, B + 1]
            assert out[4 * A, 4 * B + 1] == pytest.approx(((9 * a + 12 * m - b) - (3 * c0 + c1)) / 16, rel=1e-13)
            assert out[4 * A, 4 * B + 3] == pytest.approx(((9 * b + 12 * m - a) - (3 * c1 + c0)) / 16, rel=1e-13)


def test_linear_prolongation_printed_cases(orc):
    """Eq. 15 in 1-based indices, checked literally."""
    rng = np.random.default_rng(26)
    hc, wc = 4, 5
    uc = rng.uniform(0, 255, (hc, wc))
    h, w = 2 * hc - 1, 2 * wc - 1
    out = orc.linear(uc, h, w)
    U = lambda i, j: uc[i - 1, j - 1]  # 1-based access
    for i in range(1, h + 1):
        for j in range(1, w + 1):
            if i % 2 and j % 2:
                exp = U((i + 1) // 2, (j + 1) // 2)
            elif i % 2:
                exp = 0.5 * (U((i + 1) // 2, j // 2) + U((i + 1) // 2, j // 2 + 1))
            elif j % 2:
                exp = 0.5 * (U(i // 2, (j + 1) // 2) + U(i // 2 + 1, (j + 1) // 2))
            else:
                exp = 0.5 * (U(i // 2, j // 2) + U(i // 2 + 1, j // 2 + 1))
            assert out[i - 1, j - 1] == pytest.approx(exp, rel=1e-15)


def test_clamped_edges_stay_finite_and_constant_preserving(orc):
    """Even sizes leave a partial last cell; clamping keeps constants constant."""
    for (h, w) in [(64, 64), (30, 14), (7, 6)]:
        h1, w1 = (h + 1) // 2, (w + 1) // 2
        h2, w2 = (h1 + 1) // 2, (w1 + 1) // 2
        ue = orc.extrapolate(np.full((h1, w1), 3.5), np.full((h2, w2), 3.5))
        assert np.all(ue == 3.5)
        assert np.allclose(orc.quadratic(ue, h, w), 3.5, rtol=1e-15)
        assert np.allclose(orc.linear(np.full((h1, w1), 2.0), h, w), 2.0)
