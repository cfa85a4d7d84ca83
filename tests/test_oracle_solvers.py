"""Pins of the oracle's level smoothers (Section 2, "CG" and "MR").

Readings: "MR" = MR-II (minimal residual over u0 + K_k(H, H r0), H
symmetric) and "CG" = CGLS (minimal residual over u0 + K_k(H^T H, H^T r0)).
Both are pinned by brute force: the k-th iterate must equal the explicit
least-squares minimiser over the Krylov space, built here from dense
matrices with an orthonormal basis; at k = N with a well-conditioned PSF the
iterate is the dense solution; residual norms never increase.
"""
import numpy as np
import pytest

from test_oracle_operators import dense_conv


def centro_psf(rng, n):
    K = rng.uniform(0, 1, (n, n))
    K = 0.5 * (K + K[::-1, ::-1])
    K[n // 2, n // 2] += 1.5 * K.sum()  # diagonally dominant: well conditioned
    return K / K.sum()


def krylov_ls(Hd, g, u0, basis_vecs):
    """argmin_{u in u0 + span(basis)} ||g - H u||, via an orthonormal basis (QR, twice)."""
    V = np.stack(basis_vecs, axis=1)
    Q, _ = np.linalg.qr(V)
    Q, _ = np.linalg.qr(Q)
    r0 = g - Hd @ u0
    y, *_ = np.linalg.lstsq(Hd @ Q, r0, rcond=None)
    return u0 + Q @ y


@pytest.mark.parametrize("shape", [(6, 6), (5, 7), (8, 8)])
def test_mr2_is_krylov_minimiser(orc, shape):
    rng = np.random.default_rng(10)
    h, w = shape
    K = centro_psf(rng, 3)
    Hd = dense_conv(K, h, w)
    assert np.allclose(Hd, Hd.T)
    g = rng.uniform(0, 255, shape)
    u0 = rng.uniform(0, 255, shape)
    r0 = g.ravel() - Hd @ u0.ravel()
    for k in range(1, 7):
        basis = [np.linalg.matrix_power(Hd, j) @ r0 for j in range(1, k + 1)]
        exp = krylov_ls(Hd, g.ravel(), u0.ravel(), basis)
        u, it, _ = orc.mr2(K, g, u0, k)
        assert it == k
        assert np.linalg.norm(u.ravel() - exp) <= 1e-9 * np.linalg.norm(exp)


@pytest.mark.parametrize("shape", [(6, 6), (7, 5)])
def test_cgls_is_krylov_minimiser(orc, shape):
    rng = np.random.default_rng(11)
    h, w = shape
    K = rng.uniform(0, 1, (3, 5))
    K[1, 2] += 2 * K.sum()  # non-symmetric, well conditioned
    Hd = dense_conv(K, h, w)
    g = rng.uniform(0, 255, shape)
    u0 = rng.uniform(0, 255, shape)
    r0 = g.ravel() - Hd @ u0.ravel()
    s0 = Hd.T @ r0
    HtH = Hd.T @ Hd
    for k in range(1, 7):
        basis = [np.linalg.matrix_power(HtH, j) @ s0 for j in range(k)]
        exp = krylov_ls(Hd, g.ravel(), u0.ravel(), basis)
        u, it, _ = orc.cgls(K, g, u0, k)
        assert it == k
        assert np.linalg.norm(u.ravel() - exp) <= 1e-9 * np.linalg.norm(exp)


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_full_dimension_iterate_is_the_solution(orc, solver):
    """With k = N iterations (or an exact breakdown before), H u = g."""
    rng = np.random.default_rng(12)
    K = np.full((3, 3), 0.05)
    K[1, 1] = 0.6
    h, w = 4, 4
    g = rng.uniform(0, 255, (h, w))
    u, it, res = getattr(orc, solver)(K, g, None, h * w, conv_tol=1e-12)
    exp = np.linalg.solve(dense_conv(K, h, w), g.ravel())
    assert np.linalg.norm(u.ravel() - exp) <= 1e-8 * np.linalg.norm(exp)
    assert res <= 1e-8 * np.sqrt(np.mean(g * g))


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_residuals_never_increase(orc, solver):
    """Both methods minimise ||r|| over nested spaces."""
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(13)
    K = synth.gaussian_psf(2.0, 5)
    g = rng.uniform(0, 255, (24, 20))
    prev = np.inf
    for m in range(0, 12):
        _, it, res = getattr(orc, solver)(K, g, None, m)
        assert it == m
        assert res <= prev * (1 + 1e-12)
        prev = res


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_discrepancy_rule_stops_at_first_small_residual(orc, solver):
    """Section 2: stop when ||g - H u_k|| <= c delta (checked before each iteration)."""
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(14)
    K = synth.gaussian_psf(1.5, 4)
    g = rng.uniform(0, 255, (20, 20))
    fixed = [getattr(orc, solver)(K, g, None, m)[2] for m in range(0, 15)]
    tol = 0.5 * (fixed[3] + fixed[4])  # between the 3rd and 4th residual
    u, it, res = getattr(orc, solver)(K, g, None, 14, stop_tol=tol)
    k_first = next(k for k, r in enumerate(fixed) if r <= tol)
    assert it == k_first
    assert res == pytest.approx(fixed[k_first], rel=1e-12)


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_identity_operator_one_step(orc, solver):
    """H = I: the first iterate is g and the method stops on an exact breakdown."""
    rng = np.random.default_rng(15)
    g = rng.uniform(0, 255, (9, 11))
    u0 = rng.uniform(0, 255, (9, 11))
    u, it, res = getattr(orc, solver)(np.ones((1, 1)), g, u0, 5)
    assert it == 1
    assert np.allclose(u, g, rtol=1e-14, atol=1e-12)


def test_mr2_zero_residual_takes_no_step(orc):
    rng = np.random.default_rng(16)
    K = centro_psf(rng, 3)
    u0 = rng.uniform(0, 255, (6, 6))
    g = orc.apply_H(K, u0)
    u, it, res = orc.mr2(K, g, u0, 5)
    assert it <= 1
    assert np.allclose(u, u0, rtol=1e-12)


def test_convergence_stop_keeps_the_converged_iterate(orc):
    """Past exact convergence the literal recurrence drifts; the convergence stop does not.

    On a 4 x 4 grid the Krylov space is exhausted after about 10 MR-II
    steps.  Without the stop, extra steps follow rounding noise and the
    iterate leaves the solution while the recursive residual stays tiny;
    with it, the iterate stays at the dense solution.
    """
    rng = np.random.default_rng(12)
    K = np.full((3, 3), 0.05)
    K[1, 1] = 0.6
    g = rng.uniform(0, 255, (4, 4))
    exp = np.linalg.solve(dense_conv(K, 4, 4), g.ravel())
    u, it, _ = orc.mr2(K, g, None, 19, conv_tol=1e-10)
    assert it < 19
    assert np.linalg.norm(u.ravel() - exp) <= 1e-9 * np.linalg.norm(exp)
    u_lit, it_lit, res_lit = orc.mr2(K, g, None, 19)
    assert it_lit == 19 and res_lit < 1e-10
    assert np.linalg.norm(u_lit.ravel() - exp) > 1e-6 * np.linalg.norm(exp)


@pytest.mark.parametrize("solver", ["mr2", "cgls"])
def test_convergence_stop_rule(orc, solver):
    """The level stops before the first iteration whose residual is <= conv_tol ||g||."""
    rng = np.random.default_rng(17)
    K = np.full((3, 3), 0.04)
    K[1, 1] = 0.68
    g = rng.uniform(0, 255, (10, 12))
    gn = np.linalg.norm(g)
    fixed = []
    for m in range(0, 12):
        u, it, res = getattr(orc, solver)(K, g, None, m)
        fixed.append(res * np.sqrt(g.size))  # Euclidean norm of the residual
    tol = 0.5 * (fixed[5] + fixed[6]) / gn
    u, it, _ = getattr(orc, solver)(K, g, None, 11, conv_tol=tol)
    assert it == next(k for k, r in enumerate(fixed) if r <= tol * gn)


def mr2_lanczos_givens(Hd, g, u0, m):
    """MR-II by the Lanczos process on H started at H r0 and Givens QR of the
    (k+1) x k tridiagonal least-squares problem with right-hand side <w_j, r0>."""
    r0 = g - Hd @ u0
    v = Hd @ r0
    W = [v / np.linalg.norm(v)]
    alphas, betas = [], []
    u = u0.copy()
    for k in range(m):
        z = Hd @ W[k]
        a = z @ W[k]
        z = z - a * W[k] - (betas[-1] * W[k - 1] if k else 0.0)
        b = np.linalg.norm(z)
        alphas.append(a)
        betas.append(b)
        W.append(z / b)
        T = np.zeros((k + 2, k + 1))
        for j in range(k + 1):
            T[j, j] = alphas[j]
            T[j + 1, j] = betas[j]
            if j:
                T[j - 1, j] = betas[j - 1]
        c = np.array([w @ r0 for w in W])
        y, *_ = np.linalg.lstsq(T, c, rcond=None)
        u = u0 + np.stack(W[:k + 1], axis=1) @ y
    return u


def test_mr2_recurrence_equals_lanczos_form(orc):
    """Two formulations of MR-II give the same iterates (FP64, ill-conditioned H).

    k stays at or below 15 on this 168-pixel grid: beyond that both FP64
    formulations lose Lanczos orthogonality and part (1.5e-5 at k = 25).
    """
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(18)
    K = synth.gaussian_psf(1.5, 4)
    h, w = 12, 14
    Hd = dense_conv(K, h, w)
    g = rng.uniform(0, 255, (h, w))
    u0 = rng.uniform(0, 255, (h, w))
    for m in (3, 10, 15):
        exp = mr2_lanczos_givens(Hd, g.ravel(), u0.ravel(), m)
        u, it, _ = orc.mr2(K, g, u0, m)
        assert it == m
        assert np.linalg.norm(u.ravel() - exp) <= 1e-10 * np.linalg.norm(exp), m
