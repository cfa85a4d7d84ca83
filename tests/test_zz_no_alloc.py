"""The residual entry point that allocates no device memory, against the plan path.

eecmg_residual_noalloc serves callers that cannot call cudaMalloc: a
serving process that allows no device allocation once it is running (an
allocation can stall the device in the middle of a request), or code whose
framework allocator already holds the GPU's memory.  It keeps its scratch in
a fixed device array instead of a plan's workspace.  Here its output must
match the existing plan-based entry points on the same inputs: r against
g - eecmg_apply_H(u), and ||r|| against the residual that eecmg_level_solve
(0 iterations: only the residual step) reports, within the tolerances of
the operator tests, on two calls in a row with different inputs.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test.
"""
import gc

import numpy as np
import pytest

from gpu_helpers import dev, host, require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_plan_entry_points():
    torch, E = require_gpu()
    from paper_2311_03010_gb300 import synth

    h, w = 300, 411
    for psf in (synth.gaussian_psf(2.0, 6), synth.motion_psf(11, 40.0)):
        plan = E.Plan(w, h, 1, psf)
        rng = np.random.default_rng(90)
        for call in range(2):
            g = rng.uniform(0, 255, (h, w)).astype(np.float32)
            u = rng.uniform(0, 255, (h, w)).astype(np.float32)
            gd, ud = dev(torch, g), dev(torch, u)
            r = torch.empty_like(gd)
            norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
            E.eecmg_residual_noalloc(w, h, psf, gd, ud, r, norms)
            hu = torch.empty_like(gd)
            E.eecmg_apply_H(plan.handle, 0, ud, hu, 0)
            r_ref = g.astype(np.float64) - host(hu)
            bound = 2e-5 * np.abs(psf).sum() * 255.0 + 1e-6
            assert np.abs(host(r) - r_ref).max() <= bound, call
            u2 = ud.clone()
            E.eecmg_level_solve(plan.handle, 0, gd, u2, 0)
            _, res = plan.stats()
            nrm = norms.cpu().numpy()
            assert np.sqrt(nrm[0] / (h * w)) == pytest.approx(res[0], rel=1e-5), call
            assert nrm[1] == pytest.approx(float(np.sum(g.astype(np.float64) ** 2)), rel=1e-6)
        plan.close()


def test_noalloc_calls_after_the_warm_up_allocate_nothing():
    """The first call (at start-up) reserves the fixed scratch array with the library's device
    code; every later call leaves the device's free memory and torch's allocator untouched."""
    torch, E = require_gpu()
    from paper_2311_03010_gb300 import synth

    h, w = 257, 333
    psf = synth.gaussian_psf(1.5, 4)
    rng = np.random.default_rng(91)
    gd = dev(torch, rng.uniform(0, 255, (h, w)))
    ud = dev(torch, rng.uniform(0, 255, (h, w)))
    r = torch.empty_like(gd)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    E.eecmg_residual_noalloc(w, h, psf, gd, ud, r, norms)  # warm-up
    first = torch.empty((h, w), dtype=torch.float32)  # host copies: no device allocation
    again = torch.empty((h, w), dtype=torch.float32)
    first.copy_(r)
    gc.collect()  # garbage of earlier tests must not be freed inside the measurement
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        r.fill_(float("nan"))
        E.eecmg_residual_noalloc(w, h, psf, gd, ud, r, norms)
        again.copy_(r)
        assert torch.equal(again, first)
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversized_images():
    torch, E = require_gpu()
    x = torch.zeros(1, device="cuda")
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_residual_noalloc(4097, 8, np.ones((3, 3)) / 9, x, x.clone(), x.clone(), norms)
    assert ei.value.status == 1
