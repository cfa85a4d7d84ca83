"""Partition parameters and the autotuner.

The parameters are process-wide and may change only while no plan owns a
workspace (BUSY otherwise), so that every solve is partitioned the same way
alone, batched or served.  The autotuner times candidates on description-only
plans and keeps the fastest; results under any partition stay within the
FP32 bar of the FP64 oracle, and batched results stay bitwise the plans' own.
"""
import gc

import numpy as np
import pytest

from gpu_helpers import dev, host, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

EECMG_ERR_INVALID_ARG, EECMG_ERR_BUSY = 1, 7


@pytest.fixture(scope="module")
def gpu():
    return require_gpu()


@pytest.fixture()
def restore_default_tuning(gpu):
    _, E = gpu
    gc.collect()
    before = E.eecmg_get_tuning()
    yield
    gc.collect()
    E.eecmg_set_tuning(**before)


def test_set_tuning_is_refused_while_a_plan_owns_a_workspace(gpu, restore_default_tuning):
    _, E = gpu
    from paper_2311_03010_gb300 import synth

    t = E.eecmg_get_tuning()
    plan = E.Plan(64, 64, 3, synth.gaussian_psf(1.5, 4))
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_set_tuning(**t)
    assert ei.value.status == EECMG_ERR_BUSY
    plan.close()
    desc = E.Plan(64, 64, 3, synth.gaussian_psf(1.5, 4), workspace=0)  # holds no device memory
    E.eecmg_set_tuning(**t)
    desc.close()
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_set_tuning(t["cluster_max_px"], 512, t["blocks_per_sm"])
    assert ei.value.status == EECMG_ERR_INVALID_ARG
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_set_tuning(t["cluster_max_px"], t["px_per_block"], t["blocks_per_sm"], 33)
    assert ei.value.status == EECMG_ERR_INVALID_ARG
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_set_tuning(t["cluster_max_px"], t["px_per_block"], t["blocks_per_sm"], 32, 24)
    assert ei.value.status == EECMG_ERR_INVALID_ARG


@pytest.mark.parametrize("tuning", [(0, 1024, 2, 0, 32), (262144, 4096, 1, 8, 16), (65536, 2048, 3, 32, 32),
                                    (16384, 2048, 2, 0, 16)])
def test_other_partitions_match_the_oracle_and_stay_bitwise_batched(gpu, orc, restore_default_tuning,
                                                                   tuning):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    E.eecmg_set_tuning(*tuning)
    cases = [synth.make_problem(256, 192, 91, synth.gaussian_psf(2.0, 6), 0.02),
             synth.make_problem(130, 97, 92, synth.motion_psf(9, 60.0), 0.02)]
    plans, gs, singles = [], [], []
    for p in cases:
        h, w = p.g.shape
        pl = E.Plan(w, h, 4, p.psf)
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        pl.restore(gd, ud)
        singles.append(host(ud))
        plans.append(pl)
        gs.append(gd)
    us = [torch.empty_like(g) for g in gs]
    E.eecmg_restore_batched([pl.handle for pl in plans], gs, us)
    for s_, u in zip(singles, us):
        assert np.array_equal(s_, host(u))
    for p, u in zip(cases, singles):
        ref, _, _ = orc.cascade(p.g.astype(np.float64), 4, p.psf)
        assert rel_l2(u, ref) <= 1e-4
    for pl in plans:
        pl.close()


def test_autotune_picks_a_valid_partition(gpu, restore_default_tuning):
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    probs = [synth.make_problem(512, 384, 93, synth.gaussian_psf(2.5, 7), 0.01),
             synth.make_problem(200, 300, 94, synth.motion_psf(11, 20.0), 0.02)]
    descs = [E.Plan(p.g.shape[1], p.g.shape[0], 5, p.psf, workspace=0) for p in probs]
    gs = [dev(torch, p.g) for p in probs]
    best = E.eecmg_autotune(descs, gs, reps=3)
    assert best == E.eecmg_get_tuning()
    assert best["cluster_max_px"] in (0, 4096, 16384, 65536, 262144)
    assert best["px_per_block"] in (1024, 2048, 4096) and best["blocks_per_sm"] in (1, 2, 3)
    assert best["resident_max_tiles"] in (0, 16, 32) and best["psd_tile_h"] in (16, 32)
    # with a plan alive the tuner refuses
    full = E.Plan(64, 64, 3, synth.gaussian_psf(1.5, 4))
    with pytest.raises(E.EecmgError) as ei:
        E.eecmg_autotune(descs, gs, reps=1)
    assert ei.value.status == EECMG_ERR_BUSY
    full.close()
    for d in descs:
        d.close()


@pytest.mark.parametrize("shape", [(512, 384), (97, 131), (45, 700)])
def test_fused_start_tile_height_changes_nothing(gpu, restore_default_tuning, shape):
    """The fused level start on 16-row tiles gives bitwise the result of 32-row tiles, alone
    (eecmg_start_level) and in whole restorations, alone and batched."""
    torch, E = gpu
    from paper_2311_03010_gb300 import synth

    h, w = shape
    p = synth.make_problem(h, w, 95, synth.gaussian_psf(2.0, 6), 0.02)
    out = {}
    for th in (32, 16):
        t = E.eecmg_get_tuning()
        t["psd_tile_h"] = th
        E.eecmg_set_tuning(**t)
        plan = E.Plan(w, h, 4, p.psf, delta=p.delta)
        hs, ws = plan.info["h"], plan.info["w"]
        rng = np.random.default_rng(96)
        u1 = synth.synthetic_image(hs[2], ws[2], 97).astype(np.float32)
        u2 = (u1[::2, ::2] + rng.uniform(-3, 3, (hs[1], ws[1]))).astype(np.float32)
        start = torch.empty(hs[3], ws[3], device="cuda")
        E.eecmg_start_level(plan.handle, 3, dev(torch, u1), dev(torch, u2), start)
        gd = dev(torch, p.g)
        ud = torch.empty_like(gd)
        plan.restore(gd, ud)
        ub = torch.empty_like(gd)
        E.eecmg_restore_batched([plan.handle], [gd], [ub])
        out[th] = (host(start), host(ud), host(ub))
        plan.close()
    for a, b in zip(out[32], out[16]):
        assert np.array_equal(a, b)

