"""Writes tests/golden/cascade_small.json from the FP64 oracle only.

The stored values are regression pins of the oracle itself (the paper
prints no worked example whose input is available).  Inputs come from the
seeded generator; every expected value is computed by ``oracle``.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2311_03010_gb300 import synth  # noqa: E402

CASES = [
    # name, h, w, L, psf (kind, a, b), v, seed, smoother
    ("cfg1_mr2", 64, 64, 3, ("gauss", 1.5, 4), 0.01, 1000, "mr2"),
    ("cfg1_cgls", 64, 64, 3, ("gauss", 1.5, 4), 0.01, 1000, "cgls"),
    ("rect_motion_cgls", 45, 70, 4, ("motion", 7, 30.0), 0.02, 77, "cgls"),
    ("rect_motion_mr2", 45, 70, 4, ("motion", 7, 30.0), 0.02, 77, "mr2"),
]


def run_case(h, w, L, psf_spec, v, seed, smoother):
    psf = synth.psf_from_spec(psf_spec)
    p = synth.make_problem(h, w, seed, psf, v, texture=(h * w > 4096))
    u, it, res = oracle.cascade(p.g.astype(np.float64), L, psf, smoother=smoother)
    return p, u, it, res


def main():
    out = {"note": "written by tests/golden/make_golden.py from the FP64 oracle", "cases": {}}
    for (name, h, w, L, spec, v, seed, smo) in CASES:
        p, u, it, res = run_case(h, w, L, spec, v, seed, smo)
        idx = [(0, 0), (h - 1, w - 1), (h // 2, w // 3), (h // 3, w - 2), (1, w // 2)]
        out["cases"][name] = {
            "h": h, "w": w, "L": L, "psf": list(spec), "v": v, "seed": seed, "smoother": smo,
            "iters": it, "res_rms": res, "psnr": oracle.psnr(p.u, u),
            "sum": float(u.sum()), "sumsq": float((u * u).sum()),
            "samples": [[i, j, float(u[i, j])] for (i, j) in idx],
        }
    with open(os.path.join(HERE, "cascade_small.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
