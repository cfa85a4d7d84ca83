"""Pins of the oracle's operators against what the paper and mathematics fix.

H (Eqs. 1, 7; block-Toeplitz = zero boundary), H^T, the coarse operator of
Eq. 14, restriction (Eqs. 12-13), level sizes and the economy schedule of
Section 2.  Every check builds its expectation independently of the oracle:
dense matrices written out entry by entry, Kronecker products, delta
responses and hand-evaluated schedule values.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def dense_conv(K, h, w):
    """Dense matrix of zero-boundary convolution: H[(i,j),(i2,j2)] = K(i-i2, j-j2)."""
    ry, rx = K.shape[0] // 2, K.shape[1] // 2
    H = np.zeros((h * w, h * w))
    for i in range(h):
        for j in range(w):
            for i2 in range(max(0, i - ry), min(h, i + ry + 1)):
                for j2 in range(max(0, j - rx), min(w, j + rx + 1)):
                    H[i * w + j, i2 * w + j2] = K[i - i2 + ry, j - j2 + rx]
    return H


def toeplitz_1d(k, n):
    """T[i, i2] = k(i - i2) for a centred odd 1-D kernel k."""
    r = len(k) // 2
    T = np.zeros((n, n))
    for i in range(n):
        for i2 in range(n):
            if abs(i - i2) <= r:
                T[i, i2] = k[i - i2 + r]
    return T


@pytest.mark.parametrize("shape", [(7, 9), (1, 5), (6, 1), (12, 11)])
@pytest.mark.parametrize("ks", [(3, 5), (5, 3), (1, 1), (7, 7)])
def test_delta_response_is_psf(orc, shape, ks):
    """H applied to a delta image places the PSF at the delta, cropped at the borders."""
    rng = np.random.default_rng(1)
    h, w = shape
    K = rng.uniform(-1, 1, ks)
    ry, rx = ks[0] // 2, ks[1] // 2
    for (i0, j0) in [(0, 0), (h - 1, w - 1), (h // 2, w // 2), (0, w - 1)]:
        x = np.zeros(shape)
        x[i0, j0] = 1.0
        y = orc.apply_H(K, x)
        exp = np.zeros(shape)
        for p in range(-ry, ry + 1):
            for q in range(-rx, rx + 1):
                if 0 <= i0 + p < h and 0 <= j0 + q < w:
                    exp[i0 + p, j0 + q] = K[p + ry, q + rx]
        assert np.array_equal(y, exp)


def test_identity_psf(orc):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 255, (9, 13))
    assert np.array_equal(orc.apply_H(np.ones((1, 1)), x), x)
    K = np.zeros((5, 5))
    K[2, 2] = 1.0
    assert np.array_equal(orc.apply_H(K, x), x)
    assert np.array_equal(orc.apply_HT(K, x), x)


@pytest.mark.parametrize("shape", [(8, 8), (7, 10), (13, 5)])
def test_adjoint_brute_force(orc, shape):
    """<H x, y> = <x, H^T y> for a non-symmetric PSF and random x, y."""
    rng = np.random.default_rng(3)
    K = rng.uniform(-1, 1, (5, 7))
    for _ in range(3):
        x = rng.standard_normal(shape)
        y = rng.standard_normal(shape)
        lhs = np.sum(orc.apply_H(K, x) * y)
        rhs = np.sum(x * orc.apply_HT(K, y))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))


@pytest.mark.parametrize("shape", [(6, 7), (10, 4)])
def test_dense_matrix_equals_entrywise_definition(orc, shape):
    """Every column of H and H^T matches the dense definition."""
    rng = np.random.default_rng(4)
    h, w = shape
    K = rng.uniform(-1, 1, (3, 5))
    D = dense_conv(K, h, w)
    x = rng.standard_normal(shape)
    assert np.allclose(orc.apply_H(K, x).ravel(), D @ x.ravel(), rtol=0, atol=1e-12)
    assert np.allclose(orc.apply_HT(K, x).ravel(), D.T @ x.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [8, 11])
def test_separable_psf_is_kronecker(orc, n):
    """Section 5: H = h (x) h for the Gaussian PSF; also with distinct row/column kernels."""
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(5)
    psf = synth.gaussian_psf(1.5, 3)
    h1 = psf.sum(axis=1)  # the normalised 1-D kernel (outer product rows)
    T = toeplitz_1d(h1, n)
    x = rng.standard_normal((n, n))
    assert np.allclose(orc.apply_H(psf, x).ravel(), np.kron(T, T) @ x.ravel(), atol=1e-13)
    ky = rng.uniform(0, 1, 5)
    kx = rng.uniform(0, 1, 3)
    K = np.outer(ky, kx)
    x = rng.standard_normal((n, n + 2))
    exp = np.kron(toeplitz_1d(ky, n), toeplitz_1d(kx, n + 2)) @ x.ravel()
    assert np.allclose(orc.apply_H(K, x).ravel(), exp, atol=1e-13)


@pytest.mark.parametrize("hf,wf", [(8, 8), (9, 7), (6, 11), (13, 10)])
def test_coarse_operator_is_galerkin_product(orc, hf, wf):
    """Eq. 14: H_l = R_l H_{l+1} R_l^*, R = injection of even pixels, R^* the RMS adjoint.

    R^* is built from its defining identity <R x, y>_l = <x, R^* y>_{l+1} under
    the inner product of the RMS norm (Eq. 10).
    """
    rng = np.random.default_rng(6)
    K = rng.uniform(-1, 1, (7, 5))
    hs, ws = orc.level_sizes(hf, wf, 2)
    hc, wc = hs[0], ws[0]
    Nf, Nc = hf * wf, hc * wc
    R = np.zeros((Nc, Nf))
    for a in range(hc):
        for b in range(wc):
            R[a * wc + b, (2 * a) * wf + 2 * b] = 1.0
    # <Rx, y>_c = (1/Nc) (Rx).y ; <x, R* y>_f = (1/Nf) x.(R* y)  =>  R* = (Nf/Nc) R^T
    Rstar = (Nf / Nc) * R.T
    x = rng.standard_normal(Nf)
    y = rng.standard_normal(Nc)
    assert abs((R @ x) @ y / Nc - x @ (Rstar @ y) / Nf) < 1e-12
    Hc_dense = R @ dense_conv(K, hf, wf) @ Rstar
    Kc = orc.coarse_psf(K, Nf / Nc)
    assert Kc.shape == (2 * (3 // 2) + 1, 2 * (2 // 2) + 1)
    assert np.allclose(dense_conv(Kc, hc, wc), Hc_dense, rtol=0, atol=1e-13)
    xc = rng.standard_normal((hc, wc))
    assert np.allclose(orc.apply_H(Kc, xc).ravel(), Hc_dense @ xc.ravel(), atol=1e-12)


def test_coarse_psf_of_separable_stays_separable(orc):
    from paper_2311_03010_gb300 import synth

    psf = synth.gaussian_psf(3.0, 10)
    Kc = orc.coarse_psf(psf, 4.0)
    assert Kc.shape == (11, 11)
    s = np.linalg.svd(Kc, compute_uv=False)
    assert s[1] < 1e-14 * s[0]


def test_level_sizes(orc):
    """Section 2: next coarser side is (n+1)/2 for odd n and n/2 for even n."""
    assert orc.level_sizes(64, 64, 3) == ([16, 32, 64], [16, 32, 64])
    assert orc.level_sizes(33, 65, 4) == ([5, 9, 17, 33], [9, 17, 33, 65])
    assert orc.level_sizes(100, 75, 5) == ([7, 13, 25, 50, 100], [5, 10, 19, 38, 75])
    assert orc.level_sizes(1, 1, 3) == ([1, 1, 1], [1, 1, 1])


def test_restriction_is_injection_of_odd_one_based_pixels(orc):
    """Eq. 12: coarse k = fine 2k-1 (1-based) per dimension = fine 2a (0-based)."""
    for (hf, wf) in [(8, 8), (9, 7), (1, 6)]:
        ii, jj = np.indices((hf, wf))
        fine = 1000.0 * ii + jj
        hs, ws = orc.level_sizes(hf, wf, 2)
        c = orc.restrict(fine, hs[0], ws[0])
        for a in range(hs[0]):
            for b in range(ws[0]):
                # 1-based coarse (a+1, b+1) comes from 1-based fine (2(a+1)-1, 2(b+1)-1)
                i1, j1 = 2 * (a + 1) - 1, 2 * (b + 1) - 1
                assert c[a, b] == 1000.0 * (i1 - 1) + (j1 - 1)


def test_schedule_hand_values(orc):
    """Section 2 schedule with L_0 = L/2, m_0 = m_* = 1, beta = 4, eps_0 = 1/2.

    Hand evaluation, L = 5: l=1: (5-1.5)*1 = 3.5 -> 4; l=2: (5-3)*4 = 8;
    l=3: 2.5^2 * 4^2 = 100; l=4: 6.25*4 = 25; l=5: 6.25 -> 7.
    """
    assert orc.schedule(3) == [2, 9, 3]
    assert orc.schedule(4) == [3, 4, 16, 4]
    assert orc.schedule(5) == [4, 8, 100, 25, 7]
    assert orc.schedule(6) == [5, 12, 24, 144, 36, 9]
    assert orc.schedule(1) == [1]
    assert orc.schedule(2) == [1, 1]
