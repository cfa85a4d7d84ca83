"""Shared helpers of the GPU parity tests (CUDA library vs FP64 oracle)."""
import os

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03010_gb300 import build_lib, eecmg

    build_lib.build()
    eecmg.load()
    return torch, eecmg


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def oracle_pyramid(orc, h, w, L, psf, coarse_op="rms"):
    """Level sizes and coarse PSFs (Eq. 14) from the oracle."""
    hs, ws = orc.level_sizes(h, w, L)
    Ks = [None] * L
    Ks[-1] = np.asarray(psf, dtype=np.float64)
    for l in range(L - 1, 0, -1):
        Ks[l - 1] = orc.coarse_psf(Ks[l], hs[l] * ws[l] / (hs[l - 1] * ws[l - 1]))
        if coarse_op == "renorm":
            Ks[l - 1] *= Ks[-1].sum() / Ks[l - 1].sum()
    return hs, ws, Ks


def oracle_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1
