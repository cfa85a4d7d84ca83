"""Pins of the oracle's cascade (Algorithm 2, EECMG; Algorithm 1, IECMG).

PSF = delta makes H_L the identity, so the finest level's first iteration
returns its data exactly and the whole cascade outputs g, for any schedule
and either smoother; with the re-normalised coarse operators every level is
the identity and every u_l equals g_l.  L = 1 is the standalone smoother.
The oracle is deterministic and thread-count invariant.  The stored golden
values are regression pins of the oracle written by tests/golden/make_golden.py.
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cascade_small.json")


@pytest.mark.parametrize("smoother", ["mr2", "cgls"])
@pytest.mark.parametrize("coarse_op", ["rms", "renorm"])
@pytest.mark.parametrize("shape,L", [((64, 64), 3), ((37, 50), 4), ((20, 9), 3)])
def test_delta_psf_returns_data(orc, smoother, coarse_op, shape, L):
    rng = np.random.default_rng(40)
    g = rng.uniform(0, 255, shape)
    psf = np.zeros((5, 5))
    psf[2, 2] = 1.0
    u, it, res = orc.cascade(g, L, psf, smoother=smoother, coarse_op=coarse_op)
    assert np.allclose(u, g, rtol=1e-13, atol=1e-11)
    assert it[-1] == 1


def test_delta_psf_renorm_levels_are_restrictions(orc):
    """GALERKIN_RENORM with PSF = delta: every H_l = I, u_l = g_l, d = 0, so the
    finest start is P(g_{L-1}); with m_L = 0 iterations the output shows it."""
    rng = np.random.default_rng(41)
    g = rng.uniform(0, 255, (33, 33))
    psf = np.ones((1, 1))
    hs, ws = orc.level_sizes(33, 33, 3)
    g1 = orc.restrict(g, hs[1], ws[1])
    u, it, _ = orc.cascade(g, 3, psf, coarse_op="renorm", iters=[3, 3, 0])
    start = orc.denoise(orc.smooth(orc.quadratic(g1, 33, 33)), 0.2, 10.0)
    assert np.allclose(u, start, rtol=1e-14, atol=1e-11)
    assert it == [1, 1, 0]


@pytest.mark.parametrize("smoother", ["mr2", "cgls"])
def test_single_level_is_standalone_solver(orc, smoother):
    from paper_2311_03010_gb300 import synth

    p = synth.make_problem(40, 48, 5, synth.gaussian_psf(1.5, 4), 0.02, texture=False)
    g = p.g.astype(np.float64)
    u, it, res = orc.cascade(g, 1, p.psf, smoother=smoother, iters=[4])
    u2, k2, r2 = getattr(orc, smoother)(p.psf, g, None, 4, conv_tol=orc.CONV_TOL)
    assert np.array_equal(u, u2) and it == [k2]


def test_deterministic_and_thread_invariant(orc):
    from paper_2311_03010_gb300 import synth

    p = synth.make_problem(96, 80, 9, synth.gaussian_psf(2.0, 6), 0.01)
    g = p.g.astype(np.float64)
    orc.set_threads(1)
    a, _, _ = orc.cascade(g, 4, p.psf)
    b, _, _ = orc.cascade(g, 4, p.psf)
    orc.set_threads(4)
    c, _, _ = orc.cascade(g, 4, p.psf)
    orc.set_threads(1)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_iecmg_variants_run_and_differ(orc):
    from paper_2311_03010_gb300 import synth

    p = synth.make_problem(64, 64, 1000, synth.gaussian_psf(1.5, 4), 0.01, texture=False)
    g = p.g.astype(np.float64)
    outs = {}
    for pr in ("eecmg", "iecmg_p", "iecmg_l"):
        u, it, _ = orc.cascade(g, 3, p.psf, prolong=pr)
        assert np.all(np.isfinite(u))
        outs[pr] = u
    assert not np.array_equal(outs["eecmg"], outs["iecmg_p"])
    assert not np.array_equal(outs["iecmg_p"], outs["iecmg_l"])


def test_invalid_arguments(orc):
    with pytest.raises(ValueError):
        orc.cascade(np.zeros((8, 8)), 3, np.ones((2, 2)))


def test_golden_regression(orc):
    """Values written by tests/golden/make_golden.py (oracle only)."""
    import sys

    sys.path.insert(0, os.path.dirname(GOLDEN))
    from make_golden import run_case

    data = json.load(open(GOLDEN))["cases"]
    for name, c in data.items():
        p, u, it, res = run_case(c["h"], c["w"], c["L"], tuple(c["psf"]), c["v"], c["seed"],
                                 c["smoother"])
        assert it == c["iters"], name
        assert np.allclose(res, c["res_rms"], rtol=1e-8), name
        assert orc.psnr(p.u, u) == pytest.approx(c["psnr"], rel=1e-10)
        assert float(u.sum()) == pytest.approx(c["sum"], rel=1e-10)
        for (i, j, val) in c["samples"]:
            assert u[i, j] == pytest.approx(val, rel=1e-9, abs=1e-9)
