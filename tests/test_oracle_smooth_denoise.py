"""Pins of the local smoothing S_l (Section 3.3) and PM denoising D_l (Section 4).

S: per pixel, the weighted least-squares problem of Eq. 19 with the weights
of Eq. 18, solved here independently with numpy's least squares; constant
and affine images are unchanged; an isolated bright pixel is kept.
D: the dense matrix A(u) of Eq. 26 built from the diffusivity of Eq. 21;
conservation of the sum (zero flux); constants unchanged; the k -> infinity
limit is the linear 5-point step; the discrete maximum principle for
tau <= 1/4.
"""
import numpy as np
import pytest


def smooth_lstsq(u, scale=1.0):
    """Eq. 19 per pixel via numpy lstsq on sqrt(w)-weighted rows [1, s, t]."""
    h, w = u.shape
    out = np.zeros_like(u)
    for i in range(h):
        for j in range(w):
            rows, vals, wts = [], [], []
            for s in (-1, 0, 1):
                for t in (-1, 0, 1):
                    if 0 <= i + s < h and 0 <= j + t < w:
                        v = u[i + s, j + t]
                        wts.append(np.exp(-(scale * (u[i, j] - v)) ** 2))
                        rows.append([1.0, s, t])
                        vals.append(v)
            sw = np.sqrt(np.array(wts))
            A = np.array(rows) * sw[:, None]
            b = np.array(vals) * sw
            coef, *_ = np.linalg.lstsq(A, b, rcond=1e-10)
            out[i, j] = coef[0]
    return out


def test_smooth_matches_weighted_least_squares(orc):
    rng = np.random.default_rng(30)
    # values within a few grey levels so that weights are not degenerate
    u = rng.uniform(0, 2.5, (9, 11))
    assert np.allclose(orc.smooth(u), smooth_lstsq(u), rtol=1e-10, atol=1e-10)
    u2 = rng.uniform(0, 40, (7, 8))
    assert np.allclose(orc.smooth(u2, 0.1), smooth_lstsq(u2, 0.1), rtol=1e-9, atol=1e-9)


def test_smooth_constant_and_affine_unchanged(orc):
    u = np.full((8, 9), 123.25)
    assert np.array_equal(orc.smooth(u), u)
    yy, xx = np.indices((10, 12)).astype(float)
    for (a, b, c) in [(10.0, 0.3, -0.2), (100.0, 1.0, 0.5), (5.0, 0.0, 40.0)]:
        plane = a + b * yy + c * xx
        assert np.allclose(orc.smooth(plane), plane, rtol=0, atol=1e-9)
    # Steep plane: at the border a neighbour of weight exp(-16) ~ 1.1e-7 spans
    # a direction whose moment eigenvalue falls under the 1e-6 W cut, so the
    # fit drops that slope; the error is bounded by slope * (dropped weight).
    plane = 100.0 + 7.0 * yy + 3.0 * xx
    err = np.abs(orc.smooth(plane) - plane)
    assert err[1:-1, 1:-1].max() <= 1e-9
    assert err.max() <= 7.0 * 1e-6


def test_smooth_isolated_bright_pixel_is_kept(orc):
    """All neighbour weights underflow: the fit has only the centre, a0 = u."""
    u = np.full((7, 7), 50.0)
    u[3, 3] = 250.0
    out = orc.smooth(u)
    assert out[3, 3] == 250.0
    assert np.allclose(np.delete(out.ravel(), 3 * 7 + 3), 50.0)


def dense_A(u, k):
    """A(u) of Eq. 26 with c from Eq. 21 (central differences, out-of-image -> centre)."""
    h, w = u.shape
    up = np.pad(u, 1, mode="edge")  # replacing the missing neighbour by the centre value
    gx = 0.5 * (up[1:-1, 2:] - up[1:-1, :-2])
    gy = 0.5 * (up[2:, 1:-1] - up[:-2, 1:-1])
    c = 1.0 / (1.0 + (gx ** 2 + gy ** 2) / k ** 2)
    N = h * w
    A = np.zeros((N, N))
    for i in range(h):
        for j in range(w):
            for (a, b) in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)):
                if 0 <= a < h and 0 <= b < w:
                    coef = 0.5 * (c[i, j] + c[a, b])
                    A[i * w + j, a * w + b] = coef
                    A[i * w + j, i * w + j] -= coef
    return A


@pytest.mark.parametrize("shape", [(5, 5), (6, 9), (1, 7)])
def test_denoise_equals_dense_matrix_form(orc, shape):
    """Eq. 25: u^{n+1} = u^n + tau A(u^n) u^n."""
    rng = np.random.default_rng(31)
    u = rng.uniform(0, 255, shape)
    tau, k = 0.2, 10.0
    exp = u.ravel() + tau * dense_A(u, k) @ u.ravel()
    assert np.allclose(orc.denoise(u, tau, k).ravel(), exp, rtol=1e-13, atol=1e-10)


def test_denoise_invariants(orc):
    rng = np.random.default_rng(32)
    u = rng.uniform(0, 255, (16, 13))
    out = orc.denoise(u, 0.25, 10.0)
    assert abs(out.sum() - u.sum()) <= 1e-12 * u.sum()            # zero flux
    assert out.min() >= u.min() - 1e-9 and out.max() <= u.max() + 1e-9  # max principle
    cst = np.full((6, 7), 42.0)
    assert np.array_equal(orc.denoise(cst, 0.2, 10.0), cst)


def test_denoise_large_k_is_linear_diffusion(orc):
    """c -> 1: one explicit heat step with zero-flux boundary."""
    rng = np.random.default_rng(33)
    u = rng.uniform(0, 255, (8, 10))
    up = np.pad(u, 1, mode="edge")
    lap = (up[2:, 1:-1] + up[:-2, 1:-1] + up[1:-1, 2:] + up[1:-1, :-2] - 4 * u)
    assert np.allclose(orc.denoise(u, 0.2, 1e30), u + 0.2 * lap, rtol=1e-13, atol=1e-10)
