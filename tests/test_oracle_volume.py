"""Pins of the oracle's volume functions (the method carried over to 3-D).

The paper names volumes as the method's next application without writing
the 3-D operators out; the oracle treats the slice axis exactly like the row
and column axes.  Two families of pins tie every volume function to
something other than itself:
  * one slice with a one-slice PSF reduces each volume function to its 2-D
    counterpart, whose own pins live in the other oracle test files;
  * permuting the three axes of the input (and of the PSF) permutes the
    output in the same way, so the slice axis behaves like the two pinned
    axes.
Independent checks on top: scipy's zero-fill convolution for H, the dense
Galerkin product of Eq. 14 for the coarse PSF, exactness of P on
triquadratics, Pi's cases on its error model, numpy's weighted lstsq for S,
conservation and constants for D, and the cascade returning the data for a
delta PSF.
"""
import itertools

import numpy as np
import pytest

PERMS = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (1, 2, 0), (2, 0, 1)]


def slab(a):
    """A 2-D array as a one-slice volume."""
    return a[None, :, :]


# ------------------------------------------------------------ one slice


def test_one_slice_operators_equal_2d(orc):
    rng = np.random.default_rng(100)
    x = rng.uniform(0, 255, (11, 13))
    K = rng.uniform(-1, 1, (5, 3))
    assert np.array_equal(orc.apply_H3(slab(K), slab(x))[0], orc.apply_H(K, x))
    assert np.array_equal(orc.apply_HT3(slab(K), slab(x))[0], orc.apply_HT(K, x))
    assert np.array_equal(orc.restrict3(slab(x), 1, 6, 7)[0], orc.restrict(x, 6, 7))
    Kf = rng.uniform(0, 1, (9, 5))
    assert np.array_equal(orc.coarse_psf3(slab(Kf), 3.5)[0], orc.coarse_psf(Kf, 3.5))
    u1 = rng.uniform(0, 255, (11, 13))
    u2 = rng.uniform(0, 255, (6, 7))
    # each corner difference is counted twice along the one slice: rounding only
    assert np.allclose(orc.extrapolate3(slab(u1), slab(u2))[0], orc.extrapolate(u1, u2),
                       rtol=1e-15, atol=1e-12)
    assert np.array_equal(orc.quadratic3(slab(u1), 1, 21, 25)[0], orc.quadratic(u1, 21, 25))
    assert np.array_equal(orc.denoise3(slab(x), 0.2, 10.0)[0], orc.denoise(x, 0.2, 10.0))
    # S: the slice offsets have no spread, so the moment matrix's slice row is
    # zero and the fit is the 2-D one (different eigen-solver: rounding only)
    xs = rng.uniform(0, 3, (9, 10))
    assert np.allclose(orc.smooth3(slab(xs))[0], orc.smooth(xs), rtol=0, atol=1e-10)
    assert np.allclose(orc.smooth3(slab(x))[0], orc.smooth(x), rtol=0, atol=1e-9)


def test_one_slice_level_sizes_and_mr2_equal_2d(orc):
    assert orc.level_sizes3(1, 33, 65, 4) == ([1, 1, 1, 1],) + orc.level_sizes(33, 65, 4)
    assert orc.level_sizes3(9, 8, 5, 3) == ([3, 5, 9], [2, 4, 8], [2, 3, 5])
    rng = np.random.default_rng(101)
    K = rng.uniform(0, 1, (5, 5))
    K = 0.5 * (K + K[::-1, ::-1])
    g = rng.uniform(0, 255, (12, 14))
    u0 = rng.uniform(0, 255, (12, 14))
    for m, tol in [(1, 0.0), (4, 0.0), (9, 3.0)]:
        a = orc.mr2_3(slab(K), slab(g), slab(u0), m, tol, 1e-9)
        b = orc.mr2(K, g, u0, m, tol, 1e-9)
        assert np.array_equal(a[0][0], b[0]) and a[1:] == b[1:]


@pytest.mark.parametrize("coarse_op", ["rms", "renorm"])
def test_one_slice_cascade_equals_2d(orc, coarse_op):
    from paper_2311_03010_gb300 import synth

    p = synth.make_problem(40, 36, 102, synth.gaussian_psf(1.5, 3), 0.01)
    a = orc.cascade3(slab(p.g), 4, slab(p.psf), delta=p.delta, coarse_op=coarse_op)
    b = orc.cascade(p.g, 4, p.psf, delta=p.delta, coarse_op=coarse_op)
    assert a[1] == b[1]
    assert np.allclose(a[0][0], b[0], rtol=0, atol=1e-7)


# ------------------------------------------------------------ axis permutations


def _perm_cases():
    rng = np.random.default_rng(103)
    x = rng.uniform(0, 255, (5, 7, 6))
    K = rng.uniform(-1, 1, (3, 5, 1))
    return rng, x, K


@pytest.mark.parametrize("perm", PERMS[1:])
def test_operators_commute_with_axis_permutations(orc, perm):
    rng, x, K = _perm_cases()
    T = lambda a: np.ascontiguousarray(np.transpose(a, perm))
    assert np.allclose(orc.apply_H3(T(K), T(x)), T(orc.apply_H3(K, x)), rtol=1e-14, atol=1e-11)
    assert np.allclose(orc.apply_HT3(T(K), T(x)), T(orc.apply_HT3(K, x)), rtol=1e-14, atol=1e-11)
    ds, hs, ws = orc.level_sizes3(*x.shape, 2)
    cs = (ds[0], hs[0], ws[0])
    assert np.array_equal(orc.restrict3(T(x), *[cs[i] for i in perm]), T(orc.restrict3(x, *cs)))
    Kf = rng.uniform(0, 1, (5, 9, 3))
    assert np.array_equal(orc.coarse_psf3(T(Kf), 7.0), T(orc.coarse_psf3(Kf, 7.0)))
    u2 = rng.uniform(0, 255, cs)
    assert np.allclose(orc.extrapolate3(T(x), T(u2)), T(orc.extrapolate3(x, u2)),
                       rtol=0, atol=1e-12)
    fs = (9, 14, 11)
    assert np.allclose(orc.quadratic3(T(x), *[fs[i] for i in perm]),
                       T(orc.quadratic3(x, *fs)), rtol=0, atol=1e-11)
    xs = rng.uniform(0, 3, x.shape)
    assert np.allclose(orc.smooth3(T(xs)), T(orc.smooth3(xs)), rtol=0, atol=1e-10)
    assert np.allclose(orc.smooth3(T(x)), T(orc.smooth3(x)), rtol=0, atol=1e-8)
    assert np.allclose(orc.denoise3(T(x), 0.15, 8.0), T(orc.denoise3(x, 0.15, 8.0)),
                       rtol=0, atol=1e-11)


@pytest.mark.parametrize("perm", [(2, 1, 0), (1, 2, 0)])
def test_solver_and_cascade_commute_with_axis_permutations(orc, perm):
    from paper_2311_03010_gb300 import synth

    T = lambda a: np.ascontiguousarray(np.transpose(a, perm))
    v = synth.make_volume_problem(12, 18, 10, 104, synth.gaussian_psf3(1.2, 2), 0.01)
    a = orc.mr2_3(v.psf, v.g, None, 6)
    b = orc.mr2_3(T(v.psf), T(v.g), None, 6)
    assert a[1] == b[1] and np.allclose(b[0], T(a[0]), rtol=0, atol=1e-8)
    a = orc.cascade3(v.g, 3, v.psf, delta=v.delta)
    b = orc.cascade3(T(v.g), 3, T(v.psf), delta=v.delta)
    assert a[1] == b[1] and np.allclose(b[0], T(a[0]), rtol=0, atol=1e-7)


# ------------------------------------------------------------ independent checks


@pytest.mark.parametrize("shape,ks", [((6, 7, 8), (3, 5, 3)), ((1, 9, 4), (5, 1, 3)),
                                      ((8, 3, 5), (7, 7, 1))])
def test_H3_is_zero_fill_convolution(orc, shape, ks):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(105)
    x = rng.standard_normal(shape)
    K = rng.standard_normal(ks)
    exp = ndi.convolve(x, K, mode="constant", cval=0.0)
    assert np.allclose(orc.apply_H3(K, x), exp, rtol=0, atol=1e-12)
    exp_t = ndi.correlate(x, K, mode="constant", cval=0.0)
    assert np.allclose(orc.apply_HT3(K, x), exp_t, rtol=0, atol=1e-12)
    y = rng.standard_normal(shape)
    assert abs(np.vdot(orc.apply_H3(K, x), y) - np.vdot(x, orc.apply_HT3(K, y))) < 1e-10


def test_coarse_psf3_is_galerkin_product(orc):
    """Eq. 14 with R = injection of even voxels and R^* its RMS adjoint (N_f/N_c) R^T."""
    rng = np.random.default_rng(106)
    K = rng.uniform(-1, 1, (5, 3, 7))
    df, hf, wf = 7, 6, 9
    ds, hs, ws = orc.level_sizes3(df, hf, wf, 2)
    dc, hc, wc = ds[0], hs[0], ws[0]
    Nf, Nc = df * hf * wf, dc * hc * wc
    R = np.zeros((Nc, Nf))
    for a, b, c in itertools.product(range(dc), range(hc), range(wc)):
        R[(a * hc + b) * wc + c, ((2 * a) * hf + 2 * b) * wf + 2 * c] = 1.0
    Hf = np.zeros((Nf, Nf))
    for j in range(Nf):
        e = np.zeros(Nf)
        e[j] = 1.0
        Hf[:, j] = orc.apply_H3(K, e.reshape(df, hf, wf)).ravel()
    Hc = R @ Hf @ ((Nf / Nc) * R.T)
    Kc = orc.coarse_psf3(K, Nf / Nc)
    assert Kc.shape == (3, 1, 3)
    xc = rng.standard_normal((dc, hc, wc))
    assert np.allclose(orc.apply_H3(Kc, xc).ravel(), Hc @ xc.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("d1,h1,w1", [(5, 7, 9), (9, 5, 7)])
def test_quadratic3_exact_on_triquadratics(orc, d1, h1, w1):
    """P interpolates a quadratic in each axis exactly where no index is clamped."""
    rng = np.random.default_rng(107)
    cz, cy, cx = rng.standard_normal(3), rng.standard_normal(3), rng.standard_normal(3)
    f = lambda z, y, x: ((cz[0] + cz[1] * z + cz[2] * z * z) * (cy[0] + cy[1] * y + cy[2] * y * y)
                         * (cx[0] + cx[1] * x + cx[2] * x * x))
    zz, yy, xx = np.indices((d1, h1, w1)).astype(float)
    ut = f(zz, yy, xx)
    d, h, w = 2 * d1 - 1, 2 * h1 - 1, 2 * w1 - 1
    out = orc.quadratic3(ut, d, h, w)
    Z, Y, X = np.indices((d, h, w)).astype(float)
    exp = f(Z / 2.0, Y / 2.0, X / 2.0)
    # fine index y lies in the coarse cell starting at 2*(y//4); clamping only
    # touches cells whose three nodes run past the last coarse node
    ok = ((2 * (np.indices((d, h, w))[0] // 4) + 2 <= d1 - 1)
          & (2 * (np.indices((d, h, w))[1] // 4) + 2 <= h1 - 1)
          & (2 * (np.indices((d, h, w))[2] // 4) + 2 <= w1 - 1))
    assert ok.sum() > 0.4 * ok.size
    assert np.allclose(out[ok], exp[ok], rtol=1e-12, atol=1e-9)


def test_extrapolate3_cases(orc):
    """Pi: coarse nodes get (5 u1 - u2)/4; consistent levels (d = 0) give u1 back;
    an edge midpoint gets 1/8 of the sum of its two node differences."""
    rng = np.random.default_rng(108)
    u1 = rng.uniform(0, 255, (7, 9, 5))
    u2 = u1[::2, ::2, ::2].copy()
    assert np.array_equal(orc.extrapolate3(u1, u2), u1)
    u2 = rng.uniform(0, 255, (4, 5, 3))
    out = orc.extrapolate3(u1, u2)
    for (C, A, B) in [(0, 0, 0), (3, 4, 2), (1, 2, 1)]:
        assert np.isclose(out[2 * C, 2 * A, 2 * B], (5 * u1[2 * C, 2 * A, 2 * B] - u2[C, A, B]) / 4,
                          rtol=1e-15, atol=1e-12)
    d = u1[::2, ::2, ::2] - u2
    assert np.isclose(out[3, 4, 2], u1[3, 4, 2] + (d[1, 2, 1] + d[2, 2, 1]) / 8, rtol=1e-15,
                      atol=1e-12)
    assert np.isclose(out[1, 1, 1], u1[1, 1, 1] + d[0:2, 0:2, 0:2].sum() / 32, rtol=1e-15,
                      atol=1e-12)


def smooth3_lstsq(u, scale=1.0):
    """Per voxel: numpy lstsq on sqrt(w)-weighted rows [1, r, s, t] (Eqs. 18-19 in 3-D)."""
    d, h, w = u.shape
    out = np.zeros_like(u)
    for k, i, j in itertools.product(range(d), range(h), range(w)):
        rows, vals, wts = [], [], []
        for r, s, t in itertools.product((-1, 0, 1), repeat=3):
            if 0 <= k + r < d and 0 <= i + s < h and 0 <= j + t < w:
                v = u[k + r, i + s, j + t]
                wts.append(np.exp(-(scale * (u[k, i, j] - v)) ** 2))
                rows.append([1.0, r, s, t])
                vals.append(v)
        sw = np.sqrt(np.array(wts))
        coef, *_ = np.linalg.lstsq(np.array(rows) * sw[:, None], np.array(vals) * sw,
                                   rcond=1e-10)
        out[k, i, j] = coef[0]
    return out


def test_smooth3_matches_weighted_least_squares(orc):
    rng = np.random.default_rng(109)
    u = rng.uniform(0, 2.5, (4, 5, 6))
    assert np.allclose(orc.smooth3(u), smooth3_lstsq(u), rtol=1e-10, atol=1e-10)
    u2 = rng.uniform(0, 40, (3, 6, 4))
    assert np.allclose(orc.smooth3(u2, 0.1), smooth3_lstsq(u2, 0.1), rtol=1e-9, atol=1e-9)


def test_smooth3_constant_and_affine_unchanged(orc):
    u = np.full((4, 5, 6), 77.5)
    assert np.array_equal(orc.smooth3(u), u)
    zz, yy, xx = np.indices((5, 6, 7)).astype(float)
    for (a, b, c, e) in [(10.0, 0.3, -0.2, 0.1), (100.0, 1.0, 0.5, -0.7)]:
        plane = a + b * zz + c * yy + e * xx
        assert np.allclose(orc.smooth3(plane), plane, rtol=0, atol=1e-9)


def test_denoise3_invariants(orc):
    rng = np.random.default_rng(110)
    u = rng.uniform(0, 255, (5, 6, 7))
    out = orc.denoise3(u, 1.0 / 6.0, 10.0)
    assert np.isclose(out.sum(), u.sum(), rtol=1e-13)
    assert out.max() <= u.max() + 1e-9 and out.min() >= u.min() - 1e-9
    c = np.full((3, 4, 5), 12.0)
    assert np.array_equal(orc.denoise3(c, 0.2, 5.0), c)
    # k -> infinity: c = 1 everywhere, the linear 7-point step with zero flux
    lin = u.copy()
    for ax in range(3):
        f = np.diff(u, axis=ax)
        pad_lo = [(0, 0)] * 3
        pad_lo[ax] = (1, 0)
        pad_hi = [(0, 0)] * 3
        pad_hi[ax] = (0, 1)
        lin += 0.1 * (np.pad(f, pad_hi) - np.pad(f, pad_lo))
    assert np.allclose(orc.denoise3(u, 0.1, 1e12), lin, rtol=0, atol=1e-9)


def test_cascade3_delta_psf_returns_data(orc):
    rng = np.random.default_rng(111)
    g = rng.uniform(0, 255, (9, 12, 10))
    K = np.zeros((3, 3, 3))
    K[1, 1, 1] = 1.0
    u, it, res = orc.cascade3(g, 3, K, stop="fixed", iters=[1, 1, 1], diffusion_steps=0)
    assert np.allclose(u, g, rtol=0, atol=1e-9)


def test_cascade3_rejects_other_smoothers(orc):
    with pytest.raises(ValueError):
        orc.cascade3(np.zeros((3, 3, 3)), 2, np.ones((2, 3, 3)))


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 4), (2, 5, 3)])
def test_mr2_3_is_krylov_minimiser(orc, shape):
    """MR-II on a volume: the k-th iterate is the least-squares minimiser of
    ||g - H u|| over u0 + span{H r0, ..., H^k r0}, with H built densely from the
    scipy zero-fill convolution (independent of the oracle's own H)."""
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(120)
    K = rng.uniform(0, 1, (3, 3, 3))
    K = 0.5 * (K + K[::-1, ::-1, ::-1])
    K[1, 1, 1] += 1.5 * K.sum()  # diagonally dominant: well conditioned
    K /= K.sum()
    N = int(np.prod(shape))
    Hd = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        Hd[:, j] = ndi.convolve(e.reshape(shape), K, mode="constant", cval=0.0).ravel()
    assert np.allclose(Hd, Hd.T)
    g = rng.uniform(0, 255, shape)
    u0 = rng.uniform(0, 255, shape)
    r0 = g.ravel() - Hd @ u0.ravel()
    for k in range(1, 6):
        V = np.stack([np.linalg.matrix_power(Hd, j) @ r0 for j in range(1, k + 1)], axis=1)
        Q, _ = np.linalg.qr(V)
        Q, _ = np.linalg.qr(Q)
        y, *_ = np.linalg.lstsq(Hd @ Q, r0, rcond=None)
        exp = u0.ravel() + Q @ y
        u, it, _ = orc.mr2_3(K, g, u0, k)
        assert it == k
        assert np.linalg.norm(u.ravel() - exp) <= 1e-9 * np.linalg.norm(exp)
