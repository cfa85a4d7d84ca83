"""GPU parity of the volume path (C ABI) against the oracle's volume functions.

The volume cascade carries Algorithm 2 to 3-D (slice axis treated like the
row and column axes).  Each operator of the CUDA path is compared element by
element with the FP64 oracle on the same FP32 inputs, over shapes from one
voxel to several 8 x 8 x 32 tiles with ragged edges; level solves and whole
cascades are compared on iteration counts (equal) and on the result.

Tolerances (FP32 path vs FP64 oracle):
  H, H^T:     max |diff| <= 2e-5 * sum|K| * max|x|  (FP32 taps, <= 2197 products)
  restriction: bit-exact
  Pi, P:      max |diff| <= 2e-6 * max|u| + 1e-5
  S, D, start: max |diff| <= 1e-3 grey levels, rel-L2 <= 1e-6 (FP32 exp and the
              1e-6 W eigenvalue cut of the fit)
  solve, cascade: equal iteration counts, rel-L2 <= 1e-4 (as for images);
              residual norms within 1e-4 relative or 1e-5 max|g| (the FP32
              floor a converged coarse level ends at)
"""
import numpy as np
import pytest

from gpu_helpers import dev, host, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

SHAPES3 = [(1, 1, 1), (3, 5, 2), (8, 8, 32), (9, 17, 33), (20, 24, 70), (17, 9, 40)]


def psf3_cases():
    from paper_2311_03010_gb300 import synth

    rng = np.random.default_rng(300)
    ns = rng.uniform(0, 1, (3, 3, 5))
    ns = 0.5 * (ns + ns[::-1, ::-1, ::-1])
    i = np.arange(-3, 4, dtype=float)
    hz = np.exp(-i[2:5] ** 2 / 2.0)
    hy = np.exp(-i[1:6] ** 2 / 3.0)
    hx = np.exp(-i ** 2 / 5.0)
    an = hz[:, None, None] * hy[None, :, None] * hx[None, None, :]
    return {
        "gauss1.2": synth.gaussian_psf3(1.2, 2),
        "gauss1.5": synth.gaussian_psf3(1.5, 3),
        "gauss1.8r4": synth.gaussian_psf3(1.8, 4),
        "gauss1.8r5": synth.gaussian_psf3(1.8, 5),
        "gauss2max": synth.gaussian_psf3(2.0, 6),
        "aniso3x5x7": an / an.sum(),
        "nonsep3x3x5": ns / ns.sum(),
    }


@pytest.fixture(scope="module")
def gpu():
    return require_gpu()


def oracle_pyramid3(orc, d, h, w, L, psf, coarse_op="rms"):
    ds, hs, ws = orc.level_sizes3(d, h, w, L)
    Ks = [None] * L
    Ks[-1] = np.asarray(psf, dtype=np.float64)
    for l in range(L - 1, 0, -1):
        rho = ds[l] * hs[l] * ws[l] / (ds[l - 1] * hs[l - 1] * ws[l - 1])
        Ks[l - 1] = orc.coarse_psf3(Ks[l], rho)
        if coarse_op == "renorm":
            Ks[l - 1] *= Ks[-1].sum() / Ks[l - 1].sum()
    return ds, hs, ws, Ks


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("name", list(psf3_cases().keys()))
def test_apply_H_every_level(gpu, orc, shape, name):
    torch, E = gpu
    psf = psf3_cases()[name]
    d, h, w = shape
    L = 3
    plan = E.VolumePlan(w, h, d, L, psf)
    try:
        ds, hs, ws, Ks = oracle_pyramid3(orc, d, h, w, L, psf)
        assert plan.info["d"] == ds and plan.info["h"] == hs and plan.info["w"] == ws
        rng = np.random.default_rng(301)
        for l in range(L):
            x = rng.uniform(0, 255, (ds[l], hs[l], ws[l])).astype(np.float32)
            xd, yd = dev(torch, x), torch.empty(x.shape, device="cuda")
            bound = 2e-5 * np.abs(Ks[l]).sum() * 255.0
            for tr, fn in ((0, orc.apply_H3), (1, orc.apply_HT3)):
                E.eecmg_vol_apply_H(plan.h, l, xd, yd, tr)
                ref = fn(Ks[l], x.astype(np.float64))
                assert np.abs(host(yd) - ref).max() <= bound + 1e-6, (l, tr)
    finally:
        plan.close()


def test_delta_response_is_the_psf(gpu):
    torch, E = gpu
    psf = psf3_cases()["aniso3x5x7"]
    plan = E.VolumePlan(16, 12, 9, 1, psf)
    try:
        x = np.zeros((9, 12, 16), np.float32)
        x[4, 6, 8] = 1.0
        yd = torch.empty(x.shape, device="cuda")
        E.eecmg_vol_apply_H(plan.h, 0, dev(torch, x), yd, 0)
        y = host(yd)
        exp = np.zeros(x.shape)
        exp[3:6, 4:9, 5:12] = psf
        assert np.allclose(y, exp, rtol=1e-6, atol=1e-9)
    finally:
        plan.close()


def test_restriction_bitexact(gpu, orc):
    torch, E = gpu
    plan = E.VolumePlan(33, 17, 9, 2, psf3_cases()["gauss1.2"])
    try:
        x = np.random.default_rng(302).uniform(0, 255, (9, 17, 33)).astype(np.float32)
        c = torch.empty((5, 9, 17), device="cuda")
        E.eecmg_vol_restrict(plan.h, 0, dev(torch, x), c)
        assert np.array_equal(host(c), orc.restrict3(x.astype(np.float64), 5, 9, 17))
    finally:
        plan.close()


def smooth_volume(shape, seed):
    from paper_2311_03010_gb300 import synth

    d, h, w = shape
    v = synth.synthetic_volume(d, h, w, seed)
    rng = np.random.default_rng(seed + 1)
    return (v + rng.normal(0, 2.0, v.shape)).astype(np.float32)


@pytest.mark.parametrize("shape", [(5, 9, 12), (17, 20, 44), (33, 33, 33), (40, 9, 70)])
@pytest.mark.parametrize("steps", [1, 0, 2])
def test_start_level_matches_oracle(gpu, orc, shape, steps):
    torch, E = gpu
    d, h, w = shape
    L = 3
    plan = E.VolumePlan(w, h, d, L, psf3_cases()["gauss1.2"], alpha=0.15, k=8.0,
                        diffusion_steps=steps)
    try:
        ds, hs, ws = orc.level_sizes3(d, h, w, L)
        u1 = smooth_volume((ds[1], hs[1], ws[1]), 303)
        u2 = smooth_volume((ds[0], hs[0], ws[0]), 305)
        out = torch.empty((d, h, w), device="cuda")
        E.eecmg_vol_start_level(plan.h, 2, dev(torch, u1), dev(torch, u2), out)
        ue = orc.extrapolate3(u1.astype(np.float64), u2.astype(np.float64))
        ref = orc.smooth3(orc.quadratic3(ue, d, h, w))
        for _ in range(steps):
            ref = orc.denoise3(ref, 0.15, 8.0)
        got = host(out)
        assert np.abs(got - ref).max() <= 1e-3
        assert rel_l2(got, ref) <= 1e-6
    finally:
        plan.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (9, 17, 33), (24, 30, 41)])
def test_smooth_and_denoise_match_oracle(gpu, orc, shape):
    torch, E = gpu
    d, h, w = shape
    plan = E.VolumePlan(w, h, d, 1, psf3_cases()["gauss1.2"], alpha=1.0 / 6.0, k=5.0)
    try:
        x = smooth_volume(shape, 306)
        y = torch.empty(shape, device="cuda")
        E.eecmg_vol_smooth(plan.h, 0, dev(torch, x), y)
        ref = orc.smooth3(x.astype(np.float64))
        assert np.abs(host(y) - ref).max() <= 1e-3 and rel_l2(host(y), ref) <= 1e-6
        E.eecmg_vol_denoise(plan.h, 0, dev(torch, x), y)
        ref = orc.denoise3(x.astype(np.float64), 1.0 / 6.0, 5.0)
        assert np.abs(host(y) - ref).max() <= 1e-3 and rel_l2(host(y), ref) <= 1e-6
    finally:
        plan.close()


@pytest.mark.parametrize("shape,name", [((20, 24, 70), "gauss1.5"), ((9, 17, 33), "nonsep3x3x5"),
                                        ((32, 32, 32), "gauss2max")])
@pytest.mark.parametrize("m,stop", [(1, "fixed"), (6, "fixed"), (12, "discrepancy")])
def test_level_solve_matches_oracle(gpu, orc, shape, name, m, stop):
    from paper_2311_03010_gb300 import synth

    torch, E = gpu
    d, h, w = shape
    psf = psf3_cases()[name]
    p = synth.make_volume_problem(d, h, w, 307, psf, 0.01)
    u0 = smooth_volume(shape, 308)
    plan = E.VolumePlan(w, h, d, 1, psf, stop=stop, delta=p.delta)
    try:
        ud = dev(torch, u0)
        E.eecmg_vol_level_solve(plan.h, 0, dev(torch, p.g), ud, m)
        it, res = plan.stats()
        tol = 1.1 * p.delta if stop == "discrepancy" else 0.0
        ref, k, rres = orc.mr2_3(psf, p.g.astype(np.float64), u0.astype(np.float64), m, tol, 1e-5)
        assert it[0] == k
        assert rel_l2(host(ud), ref) <= 1e-4
        assert abs(res[0] - rres) <= 1e-4 * max(rres, 1.0)
    finally:
        plan.close()


CASCADES = [
    # (d, h, w), L, psf, v, options
    ((20, 24, 70), 3, "gauss1.5", 0.01, {}),
    ((33, 40, 37), 4, "gauss1.5", 0.01, {}),
    ((33, 40, 37), 4, "gauss1.5", 0.05, {}),
    ((48, 48, 48), 4, "gauss1.2", 0.01, {"coarse_op": "renorm"}),
    ((30, 34, 28), 3, "gauss1.5", 0.01, {"diffusion_steps": 0}),
    ((30, 34, 28), 3, "gauss1.5", 0.01, {"diffusion_steps": 2}),
    ((25, 31, 29), 3, "nonsep3x3x5", 0.01, {}),
    ((40, 40, 40), 4, "aniso3x5x7", 0.02, {}),
    ((26, 26, 26), 4, "gauss1.5", 0.01, {"stop": "fixed", "iters": [1, 1, 2, 2]}),
]


@pytest.mark.parametrize("case", range(len(CASCADES)))
def test_cascade_matches_oracle(gpu, orc, case):
    from paper_2311_03010_gb300 import synth

    torch, E = gpu
    (d, h, w), L, name, v, opts = CASCADES[case]
    opts = dict(opts)
    iters = opts.pop("iters", None)
    psf = psf3_cases()[name]
    p = synth.make_volume_problem(d, h, w, 310 + case, psf, v)
    plan = E.VolumePlan(w, h, d, L, psf, iters=iters, delta=p.delta, **opts)
    try:
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        plan.restore(gd, ud)
        it, res = plan.stats()
        ref, rit, rres = orc.cascade3(p.g.astype(np.float64), L, psf, iters=iters,
                                      delta=p.delta, **opts)
        assert it == rit
        assert rel_l2(host(ud), ref) <= 1e-4
        # a converged coarse level ends at the FP32 floor of its data
        assert np.allclose(res, rres, rtol=1e-4, atol=1e-5 * np.abs(p.g).max())
        # a second restoration replays the graph: bitwise the same
        ud2 = torch.empty_like(gd)
        plan.restore(gd, ud2)
        assert torch.equal(ud, ud2)
    finally:
        plan.close()


def test_graph_and_plain_launches_agree_and_host_entry(gpu):
    from paper_2311_03010_gb300 import synth

    torch, E = gpu
    psf = psf3_cases()["gauss1.5"]
    p = synth.make_volume_problem(24, 36, 52, 320, psf, 0.01)
    a = E.VolumePlan(52, 36, 24, 4, psf, delta=p.delta)
    b = E.VolumePlan(52, 36, 24, 4, psf, delta=p.delta, use_graph=0)
    try:
        gd = dev(torch, p.g)
        ua, ub = torch.empty_like(gd), torch.empty_like(gd)
        a.restore(gd, ua)
        b.restore(gd, ub)
        assert torch.equal(ua, ub)
        uh = np.empty_like(p.g)
        E.eecmg_vol_restore_host(a.h, np.ascontiguousarray(p.g), uh)
        assert np.array_equal(uh, host(ua).astype(np.float32))
        # aliased buffers: restore in place
        gi = gd.clone()
        a.restore(gi, gi)
        assert torch.equal(gi, ua)
    finally:
        a.close()
        b.close()


def test_128_cube_matches_oracle(gpu, orc):
    from paper_2311_03010_gb300 import synth

    torch, E = gpu
    psf = synth.gaussian_psf3(1.5, 3)
    p = synth.make_volume_problem(128, 128, 128, 330, psf, 0.01)
    plan = E.VolumePlan(128, 128, 128, 4, psf, delta=p.delta)
    try:
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        plan.restore(gd, ud)
        it, res = plan.stats()
        ref, rit, rres = orc.cascade3(p.g.astype(np.float64), 4, psf, delta=p.delta)
        assert it == rit
        assert rel_l2(host(ud), ref) <= 1e-4
    finally:
        plan.close()


def test_256_cube_properties(gpu, orc):
    """The full-size volume workload: the oracle is too slow for the whole
    cascade, so check what holds at any size: every level either met the
    discrepancy rule or ran its cap, the reported residual equals ||g - H u||
    recomputed by the oracle on the finest level, and the restoration gains
    PSNR over the data."""
    from paper_2311_03010_gb300 import synth

    torch, E = gpu
    psf = synth.gaussian_psf3(1.5, 3)
    n = 256
    p = synth.make_volume_problem(n, n, n, 340, psf, 0.01)
    plan = E.VolumePlan(n, n, n, 4, psf, delta=p.delta)
    try:
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        plan.restore(gd, ud)
        it, res = plan.stats()
        caps = plan.info["iters"]
        for l in range(4):
            assert it[l] == caps[l] or res[l] <= 1.1 * p.delta * (1 + 1e-6)
        u = host(ud)
        r = p.g.astype(np.float64) - orc.apply_H3(psf, u)
        assert abs(np.sqrt(np.mean(r * r)) - res[-1]) <= 1e-4 * res[-1]
        assert orc.psnr(u.reshape(n, -1), p.u.reshape(n, -1)) > orc.psnr(
            p.g.astype(np.float64).reshape(n, -1), p.u.reshape(n, -1)) + 5.0
    finally:
        plan.close()
