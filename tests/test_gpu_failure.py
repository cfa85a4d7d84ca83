"""Failure path on the GPU without a fault: bounded waits give up and report.

Every wait inside a level solve is bounded by a clock limit.  A barrier
whose arrival count can never be reached (one block waiting for two) must
give up, flag the job and return; the call reports EECMG_ERR_TIMEOUT and the
context stays usable for a normal restoration afterwards.
"""
import numpy as np
import pytest

from gpu_helpers import dev, host, require_gpu

pytestmark = pytest.mark.gpu

EECMG_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def gpu():
    return require_gpu()


@pytest.mark.parametrize("cluster", [0, 1])
def test_unreachable_barrier_times_out(gpu, cluster):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    assert E.eecmg_selftest_bounded_wait(cluster) == EECMG_ERR_TIMEOUT
    # the context is still usable
    p = synth.make_problem(64, 64, 1000, synth.gaussian_psf(1.5, 4), 0.01, texture=False)
    plan = E.Plan(64, 64, 3, p.psf)
    gd = dev(torch, p.g)
    ud = torch.empty_like(gd)
    plan.restore(gd, ud)
    torch.cuda.synchronize()
    assert np.isfinite(host(ud)).all()
    plan.close()
