"""GPU parity of the per-level operators (C ABI) against the FP64 oracle.

H and H^T (Eqs. 1, 7, 14), restriction (Eqs. 12-13), the nonlinear
prolongation Pi + P (Section 3.2), P and L alone (Algorithm 1, Eq. 15), S
(Section 3.3) and D (Section 4).  Shapes span one to several 32 x 64 tiles
with ragged edges, and the degenerate 1 x 1 and 2 x 3 images.

Tolerances (FP32 path vs FP64 oracle on identical FP32 inputs):
  H, H^T:  max |diff| <= 2e-5 * sum|K| * max|x|   (FP32 taps and a sum of at
           most 625 FP32 products; worst-case rounding bound n * 2^-24)
  Pi + P, P, L:  max |diff| <= 2e-6 * max|u| + 1e-5 (a few FP32 operations)
  S, D:    max |diff| <= 1e-3 grey levels and rel-L2 <= 1e-6 (FP32 exp and
           the 1e-6 W eigenvalue cut of the local fit)
  restriction: bit-exact.
"""
import numpy as np
import pytest

from gpu_helpers import dev, host, oracle_pyramid, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (2, 3), (7, 5), (16, 16), (17, 17), (33, 65), (100, 130), (64, 200)]


def psf_cases():
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(50)
    c5 = rng.uniform(0, 1, (5, 5))
    c5 = 0.5 * (c5 + c5[::-1, ::-1])
    ns = rng.uniform(0, 1, (3, 7))
    return {
        "gauss1.5": (synth.gaussian_psf(1.5, 4), "mr2"),
        "gauss3": (synth.gaussian_psf(3.0, 10), "mr2"),
        "gauss4max": (synth.gaussian_psf(4.0, 12), "mr2"),
        "motion15": (synth.motion_psf(15, 30.0), "mr2"),
        "motion21": (synth.motion_psf(21, 100.0), "mr2"),
        "centro5": (c5 / c5.sum(), "mr2"),
        "nonsym3x7": (ns / ns.sum(), "cgls"),
    }


@pytest.fixture(scope="module")
def gpu():
    return require_gpu()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", list(psf_cases().keys()))
def test_apply_H_and_HT(gpu, orc, shape, name):
    torch, E = gpu
    psf, smo = psf_cases()[name]
    h, w = shape
    rng = np.random.default_rng([h, w, sum(map(ord, name))])
    x = rng.uniform(0, 255, shape).astype(np.float32)
    plan = E.Plan(w, h, 1, psf, smoother=smo)
    xd = dev(torch, x)
    yd = torch.empty_like(xd)
    bound = 2e-5 * np.abs(psf).sum() * np.abs(x).max() + 1e-6
    for tr, ref in ((0, orc.apply_H), (1, orc.apply_HT)):
        E.eecmg_apply_H(plan.handle, 0, xd, yd, tr)
        d = np.abs(host(yd) - ref(psf, x.astype(np.float64))).max()
        assert d <= bound, (tr, d, bound)
    plan.close()


def test_coarse_level_operators(gpu, orc):
    """Every level's H_l is the Galerkin coarse operator of Eq. 14 (both readings)."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    for coarse_op in ("rms", "renorm"):
        for psf in (synth.gaussian_psf(3.0, 10), synth.motion_psf(17, 60.0)):
            h, w, L = 150, 201, 5
            hs, ws, Ks = oracle_pyramid(orc, h, w, L, psf, coarse_op)
            plan = E.Plan(w, h, L, psf, coarse_op=coarse_op)
            info = plan.info
            assert info["h"] == hs and info["w"] == ws
            assert info["iters"] == orc.schedule(L)
            rng = np.random.default_rng(51)
            for l in range(L):
                x = rng.uniform(0, 255, (hs[l], ws[l])).astype(np.float32)
                xd = dev(torch, x)
                yd = torch.empty_like(xd)
                E.eecmg_apply_H(plan.handle, l, xd, yd, 0)
                ref = orc.apply_H(Ks[l], x.astype(np.float64))
                assert np.abs(host(yd) - ref).max() <= 2e-5 * np.abs(Ks[l]).sum() * 255 + 1e-6
            plan.close()


@pytest.mark.parametrize("name", ["gauss3", "motion15", "nonsym3x7"])
def test_delta_response_is_psf(gpu, name):
    torch, E = gpu
    psf, smo = psf_cases()[name]
    h, w = 40, 70
    plan = E.Plan(w, h, 1, psf, smoother=smo)
    ry, rx = psf.shape[0] // 2, psf.shape[1] // 2
    for (i0, j0) in [(0, 0), (20, 35), (39, 69), (3, 66)]:
        x = np.zeros((h, w), np.float32)
        x[i0, j0] = 1.0
        xd = dev(torch, x)
        yd = torch.empty_like(xd)
        E.eecmg_apply_H(plan.handle, 0, xd, yd, 0)
        y = host(yd)
        exp = np.zeros((h, w))
        for p in range(-ry, ry + 1):
            for q in range(-rx, rx + 1):
                if 0 <= i0 + p < h and 0 <= j0 + q < w:
                    exp[i0 + p, j0 + q] = psf[p + ry, q + rx]
        assert np.abs(y - exp).max() <= 3e-7 * np.abs(psf).max()
    plan.close()


def test_adjoint_on_gpu(gpu):
    torch, E = gpu
    psf, _ = psf_cases()["nonsym3x7"]
    rng = np.random.default_rng(52)
    h, w = 77, 131
    plan = E.Plan(w, h, 1, psf, smoother="cgls")
    x = rng.standard_normal((h, w)).astype(np.float32)
    y = rng.standard_normal((h, w)).astype(np.float32)
    hx, hty = torch.empty(h, w, device="cuda"), torch.empty(h, w, device="cuda")
    E.eecmg_apply_H(plan.handle, 0, dev(torch, x), hx, 0)
    E.eecmg_apply_H(plan.handle, 0, dev(torch, y), hty, 1)
    lhs = float(np.sum(host(hx) * y))
    rhs = float(np.sum(x * host(hty)))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(x) * np.linalg.norm(y)
    plan.close()


def test_restrict_bitexact(gpu, orc):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    for (h, w) in [(64, 64), (45, 70), (9, 7), (2, 3)]:
        plan = E.Plan(w, h, 3, synth.gaussian_psf(1.0, 2))
        hs, ws = orc.level_sizes(h, w, 3)
        f = np.random.default_rng(53).uniform(0, 255, (h, w)).astype(np.float32)
        c = torch.empty(hs[1], ws[1], device="cuda")
        E.eecmg_restrict(plan.handle, 1, dev(torch, f), c)
        assert np.array_equal(host(c), orc.restrict(f.astype(np.float64), hs[1], ws[1]))
        plan.close()


@pytest.mark.parametrize("shape", [(64, 64), (65, 65), (45, 70), (30, 14), (7, 6), (5, 5)])
def test_prolong_pi_then_p(gpu, orc, shape):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    h, w = shape
    plan = E.Plan(w, h, 3, synth.gaussian_psf(1.0, 2))
    hs, ws = orc.level_sizes(h, w, 3)
    rng = np.random.default_rng(54)
    u1 = rng.uniform(0, 255, (hs[1], ws[1])).astype(np.float32)
    u2 = (u1[::2, ::2] + rng.uniform(-3, 3, (hs[0], ws[0]))).astype(np.float32)
    out = torch.empty(h, w, device="cuda")
    E.eecmg_prolong(plan.handle, 2, dev(torch, u1), dev(torch, u2), out)
    ref = orc.quadratic(orc.extrapolate(u1.astype(np.float64), u2.astype(np.float64)), h, w)
    assert np.abs(host(out) - ref).max() <= 2e-6 * np.abs(ref).max() + 1e-5
    for quad, fn in ((1, lambda a: orc.quadratic(a, h, w)), (0, lambda a: orc.linear(a, h, w))):
        E.eecmg_prolong_single(plan.handle, 2, dev(torch, u1), out, quad)
        ref = fn(u1.astype(np.float64))
        assert np.abs(host(out) - ref).max() <= 2e-6 * np.abs(ref).max() + 1e-5
    plan.close()


def _smooth_inputs():
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(55)
    imgs = [rng.uniform(0, 3, (33, 65)), synth.synthetic_image(100, 130, 7),
            rng.uniform(0, 255, (17, 17)), np.full((5, 9), 77.0)]
    p = synth.make_problem(96, 96, 8, synth.gaussian_psf(2.0, 6), 0.02)
    imgs.append(p.g.astype(np.float64))
    return [a.astype(np.float32) for a in imgs]


def test_smooth_matches_oracle(gpu, orc):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    for u in _smooth_inputs():
        h, w = u.shape
        for scale in (1.0, 0.2):
            plan = E.Plan(w, h, 1, synth.gaussian_psf(1.0, 1), s_scale=scale)
            out = torch.empty(h, w, device="cuda")
            E.eecmg_smooth(plan.handle, 0, dev(torch, u), out)
            ref = orc.smooth(u.astype(np.float64), scale)
            got = host(out)
            assert np.abs(got - ref).max() <= 1e-3
            assert rel_l2(got, ref) <= 1e-6
            plan.close()


def test_denoise_matches_oracle(gpu, orc):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    for u in _smooth_inputs():
        h, w = u.shape
        for (tau, k) in ((0.2, 10.0), (0.25, 3.0), (0.1, 50.0)):
            plan = E.Plan(w, h, 1, synth.gaussian_psf(1.0, 1), alpha=tau, k=k)
            out = torch.empty(h, w, device="cuda")
            E.eecmg_denoise(plan.handle, 0, dev(torch, u), out)
            ref = orc.denoise(u.astype(np.float64), tau, k)
            got = host(out)
            assert np.abs(got - ref).max() <= 1e-3
            assert rel_l2(got, ref) <= 1e-6
            plan.close()


@pytest.mark.parametrize("shape", [(64, 64), (65, 65), (45, 70), (130, 200), (33, 700), (7, 6), (5, 5)])
def test_start_level_is_the_operator_chain(gpu, orc, shape):
    """The fused start of a prolonged level, D(S(P(Pi(u1, u2)))) in one pass over 32 x 64 tiles
    with shared-memory halos, equals eecmg_prolong, eecmg_smooth and eecmg_denoise in sequence
    bitwise (partial tiles, tiles narrower than the halo, one-tile images) and the FP64 oracle's
    chain within the operators' FP32 bar."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    h, w = shape
    plan = E.Plan(w, h, 3, synth.gaussian_psf(1.0, 2))
    hs, ws = orc.level_sizes(h, w, 3)
    rng = np.random.default_rng(56)
    u1 = synth.synthetic_image(hs[1], ws[1], 57).astype(np.float32)
    u2 = (u1[::2, ::2] + rng.uniform(-3, 3, (hs[0], ws[0]))).astype(np.float32)
    d1, d2 = dev(torch, u1), dev(torch, u2)
    fused = torch.full((h, w), float("nan"), device="cuda")
    E.eecmg_start_level(plan.handle, 2, d1, d2, fused)
    p, s, d = (torch.empty(h, w, device="cuda") for _ in range(3))
    E.eecmg_prolong(plan.handle, 2, d1, d2, p)
    E.eecmg_smooth(plan.handle, 2, p, s)
    E.eecmg_denoise(plan.handle, 2, s, d)
    assert np.array_equal(host(fused), host(d))
    ref = orc.denoise(orc.smooth(orc.quadratic(orc.extrapolate(u1.astype(np.float64),
                                                               u2.astype(np.float64)), h, w), 1.0),
                      0.2, 10.0)
    assert np.abs(host(fused) - ref).max() <= 1e-3
    assert rel_l2(host(fused), ref) <= 1e-6
    plan.close()
