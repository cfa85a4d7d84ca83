"""Pins of the oracle's RMS norm (Eq. 10) and PSNR (Section 5) against hand-computed values.

Both functions sit on each side of every stopping decision and every PSNR
comparison, so each is pinned here by numbers worked out by hand, not by the
oracle itself:
  * Eq. 10: ||V|| = ((1/m) sum v_i^2)^(1/2).  [3, 4] gives sqrt(12.5); n equal
    entries c give |c| for every n (dropping the 1/m would give |c| sqrt(n));
    the shape (1 x N, N x 1, h x w) does not matter.
  * Section 5: PSNR = 20 log10(255 / ||u - u_hat||) with the same norm.  A
    constant error of 255 / 10^k gives exactly 20 k dB at any image size (the
    Euclidean norm would give 20 k - 10 log10(N) dB); an error of 255 gives
    0 dB; the value is symmetric in its two arguments.
  * The residual norms the level solvers report are the RMS of g - H u
    recomputed here with numpy from the returned iterate.
"""
import math

import numpy as np
import pytest


def test_rms_of_hand_computed_vectors(orc):
    assert orc.rms(np.array([[3.0, 4.0]])) == pytest.approx(math.sqrt(12.5), rel=1e-15)
    assert orc.rms(np.array([[3.0], [4.0]])) == pytest.approx(math.sqrt(12.5), rel=1e-15)
    assert orc.rms(np.array([[1.0, -1.0, 1.0, -1.0]])) == pytest.approx(1.0, rel=1e-15)
    # [1, 2, 2] -> sqrt(9 / 3) = sqrt(3)
    assert orc.rms(np.array([[1.0, 2.0, 2.0]])) == pytest.approx(math.sqrt(3.0), rel=1e-15)


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (17, 1), (5, 9), (64, 64)])
def test_rms_of_a_constant_is_its_magnitude_at_every_size(orc, shape):
    for c in (2.5, -7.0):
        assert orc.rms(np.full(shape, c)) == pytest.approx(abs(c), rel=1e-14)


def test_rms_is_not_the_euclidean_norm(orc):
    x = np.full((10, 10), 3.0)
    assert orc.rms(x) == pytest.approx(3.0, rel=1e-15)
    assert abs(orc.rms(x) - float(np.linalg.norm(x))) > 20.0


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (7, 13), (128, 96)])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_psnr_of_a_constant_error(orc, shape, k):
    rng = np.random.default_rng(3 + k)
    u = rng.uniform(0.0, 255.0, shape)
    err = 255.0 / 10.0 ** k
    for sign in (1.0, -1.0):
        assert orc.psnr(u, u + sign * err) == pytest.approx(20.0 * k, abs=1e-9)


def test_psnr_with_a_half_and_half_error(orc):
    # errors +a on half the pixels and -a on the other half: RMS a, so 20 log10(255 / a)
    u = np.zeros((4, 6))
    e = np.where(np.arange(24).reshape(4, 6) % 2 == 0, 5.1, -5.1)
    assert orc.psnr(u, u + e) == pytest.approx(20.0 * math.log10(50.0), abs=1e-12)
    # one pixel of error 255 among N = 100: RMS 255 / sqrt(N), PSNR 10 log10(N) = 20 dB
    v = np.zeros((10, 10))
    v[3, 4] = 255.0
    assert orc.psnr(np.zeros((10, 10)), v) == pytest.approx(20.0, abs=1e-12)


def test_psnr_is_symmetric(orc):
    rng = np.random.default_rng(9)
    a, b = rng.uniform(0, 255, (20, 30)), rng.uniform(0, 255, (20, 30))
    assert orc.psnr(a, b) == pytest.approx(orc.psnr(b, a), rel=1e-15)


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_solver_residual_norm_is_the_rms_of_the_residual(orc, solver):
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(21)
    K = synth.gaussian_psf(1.5, 4)
    g = rng.uniform(0.0, 255.0, (19, 23))
    for m in (0, 1, 3):
        u, it, res = getattr(orc, solver)(K, g, None, m)
        r = g - orc.apply_H(K, u)
        assert res == pytest.approx(math.sqrt(float(np.mean(r * r))), rel=1e-10), m
