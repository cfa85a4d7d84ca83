"""The C-ABI library builds, loads without a GPU, and exports every declared entry point.

Also checks the host-side argument validation of eecmg_plan, which runs
before any CUDA call (so it is testable on a machine without a GPU).
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eecmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eecmg_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_03010_gb300 import build_lib, eecmg

    build_lib.build()
    return eecmg


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    assert set(names) == set(lib._SIGS), set(names) ^ set(lib._SIGS)


def test_version_and_defaults(lib):
    assert "sm_103a" in lib.eecmg_version()
    o = lib.eecmg_default_options()
    assert (o.smoother, o.coarse_op, o.storage, o.stop) == (0, 0, 0, 1)  # stop: discrepancy rule
    assert (o.c, o.delta, o.diffusion_steps, o.s_scale) == (1.1, 0.0, 1, 1.0)
    assert o.conv_tol == 1e-5 and o.prolong == 0 and o.use_graph == 1 and o.persistent == 1
    assert o.precise_conv == -1  # resolved per plan: compensated where a level can run long
    assert o.workspace == 1 and o.fuse_start == 0 and o.early_check == 1


@pytest.mark.parametrize("args,status", [
    (dict(width=0), 1), (dict(height=-1), 1), (dict(levels=0), 1),
    (dict(psf=np.ones((2, 3))), 1), (dict(psf=np.ones((27, 27))), 1),
    (dict(psf=-np.ones((3, 3))), 1), (dict(psf=np.full((3, 3), np.nan)), 1),
    (dict(alpha=0.3), 1), (dict(alpha=-0.1), 1), (dict(k=0.0), 1),
    (dict(iters=[1, -1, 2]), 1),
    (dict(psf=np.tri(5)), 2),            # MR-II needs a centrosymmetric PSF
    (dict(storage="bf16", persistent=0), 2),  # BF16 storage needs the persistent solve
    (dict(early_check=3), 1), (dict(fuse_start=2), 1),
])
def test_plan_validation_without_gpu(lib, args, status):
    kw = dict(width=64, height=64, levels=3, psf=np.ones((3, 3)) / 9, alpha=0.2, k=10.0)
    kw.update(args)
    opts = {k: kw.pop(k) for k in ("storage", "persistent", "early_check", "fuse_start") if k in kw}
    with pytest.raises(lib.EecmgError) as ei:
        lib.eecmg_plan(kw["width"], kw["height"], kw["levels"], kw["psf"], kw["alpha"], kw["k"],
                       kw.get("iters"), **opts)
    assert ei.value.status == status
    assert lib.eecmg_last_error()


def test_null_handles_rejected(lib):
    for fn, args in [(lib.eecmg_plan_info, (None,)), (lib.eecmg_restore, (None, 1, 1)),
                     (lib.eecmg_smooth, (None, 0, 1, 2))]:
        with pytest.raises(lib.EecmgError) as ei:
            fn(*args)
        assert ei.value.status == 1


def test_server_arguments_checked_before_any_device_call(lib):
    for fn, args in [(lib.eecmg_server_create, (0, 4)), (lib.eecmg_server_create, (1 << 20, 0)),
                     (lib.eecmg_server_create, (1 << 20, 5000)),
                     (lib.eecmg_server_submit, (None, None, 1, 1)),
                     (lib.eecmg_server_poll, (None, 1)), (lib.eecmg_server_drain, (None,))]:
        with pytest.raises(lib.EecmgError) as ei:
            fn(*args)
        assert ei.value.status == 1
    lib.eecmg_server_destroy(None)  # NULL is a no-op


def test_volume_plan_validation(lib):
    """eecmg_vol_plan checks sizes, PSF and options on the host, before any CUDA call."""
    from paper_2311_03010_gb300 import synth

    g = synth.gaussian_psf3(1.5, 3)
    def code(**kw):
        args = dict(width=16, height=16, depth=16, levels=3, psf=g)
        args.update(kw)
        try:
            h = lib.eecmg_vol_plan(args.pop("width"), args.pop("height"), args.pop("depth"),
                                   args.pop("levels"), args.pop("psf"), **args)
        except lib.EecmgError as e:
            return e.status
        raise AssertionError(f"accepted {kw} ({h})")

    assert code(width=0) == 1
    assert code(levels=0) == 1
    assert code(psf=np.ones((2, 3, 3))) == 1                        # even side
    assert code(psf=synth.gaussian_psf3(2.0, 7)) == 1               # radius 7 > 6
    assert code(psf=-g) == 1                                        # non-positive sum
    assert code(alpha=0.3) == 1                                     # above 0.25
    assert code(k=0.0) == 1
    ns = np.random.default_rng(1).uniform(0, 1, (3, 3, 3))
    assert code(psf=ns) == 2                                        # MR-II, not centrosymmetric
    assert code(smoother="cgls") == 2
    assert code(prolong="iecmg_p") == 2
    assert code(storage="bf16") == 2
    assert code(iters=[1, -1, 1]) == 1
    assert code(c=1.0) == 1


def test_volume_entry_points_reject_a_null_plan(lib):
    """Every volume call checks its plan on the host before touching the device."""
    so = lib.load()
    null = None
    calls = [
        ("eecmg_vol_restore", (null, null, null, null)),
        ("eecmg_vol_restore_host", (null, null, null, null)),
        ("eecmg_vol_plan_stats", (null, null, null)),
        ("eecmg_vol_plan_info", (null, null, null, null, null, null, null)),
        ("eecmg_vol_apply_H", (null, 0, null, null, 0, null)),
        ("eecmg_vol_restrict", (null, 0, null, null, null)),
        ("eecmg_vol_start_level", (null, 2, null, null, null, null)),
        ("eecmg_vol_smooth", (null, 0, null, null, null)),
        ("eecmg_vol_denoise", (null, 0, null, null, null)),
        ("eecmg_vol_level_solve", (null, 0, null, null, 1, null)),
        ("eecmg_vol_plan_profile", (null, 1)),
        ("eecmg_vol_plan_profile_read", (null, null, null, null)),
    ]
    for name, args in calls:
        assert getattr(so, name)(*args) == 1, name
    assert so.eecmg_vol_plan_destroy(None) == 0
