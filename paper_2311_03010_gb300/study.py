"""PSNR against work of the cascade's iteration schedules, on the GPU library.

The paper's conclusion claims that the economy schedule of Section 2 cuts
the work of the cascade; its Section 2 also gives the discrepancy rule
(||g^delta - H u_k|| <= c delta) as the smoothers' stopping test.  This study
restores seeded synthetic problems (the stand-ins for the paper's test image)
under several schedules and reports, per variant, the PSNR of the result
(Section 5, RMS norm, peak 255) against that of the data, the iterations each
level ran, the work in fine-grid-equivalent iterations (sum over levels of
m_l N_l / N_L) and the GPU time of one restoration:

  * eecmg-disc   Algorithm 2, each level stopped by the discrepancy rule with
                 the economy schedule as the cap: an adaptive m_l per level
                 (the library's default);
  * eecmg-fixed  Algorithm 2 with exactly the economy schedule's m_l;
  * eecmg-disc-uncapped  the discrepancy rule with caps of 1000 iterations;
  * iecmg-p / iecmg-l    Algorithm 1 (quadratic / linear prolongation), with
                 the discrepancy rule;
  * eecmg-disc-renorm  eecmg-disc with the coarse PSFs rescaled to the fine
                 PSF's sum instead of the RMS-adjoint Galerkin operators;
  * eecmg-disc-cgls    eecmg-disc with CGLS as the level smoother;
  * mr2-disc / cgls-disc  MR-II or CGLS on the finest grid alone, from zero,
                 stopped by the discrepancy rule (cap 1000: the standalone
                 smoothers of Table 1);
  * mr2-same-work  MR-II on the finest grid alone with the work eecmg-disc
                 spent (rounded up to whole iterations).

Every restoration runs through the C ABI (eecmg_plan / eecmg_restore); this
module only builds the inputs and measures.  Run as
``python -m paper_2311_03010_gb300.study`` (needs a GPU); it prints a
Markdown table.
"""
from __future__ import annotations

import argparse
import math

import numpy as np

CASES = {
    # name: (h, w, levels, psf spec, noise level, image seed, noise seed)
    "64x64-gauss1.5-1%": (64, 64, 3, ("gauss", 1.5, 4), 0.01, 1000, 1001),
    "512x512-gauss2.5-1%": (512, 512, 5, ("gauss", 2.5, 7), 0.01, 2000, 2001),
    "512x512-gauss2.5-5%": (512, 512, 5, ("gauss", 2.5, 7), 0.05, 2000, 2002),
    "2048x2048-gauss3-1%": (2048, 2048, 5, ("gauss", 3.0, 10), 0.01, 3000, 3001),
    "2048x2048-motion15-1%": (2048, 2048, 5, ("motion", 15, 30.0), 0.01, 3000, 3001),
    "4096x4096-gauss3-1%": (4096, 4096, 5, ("gauss", 3.0, 10), 0.01, 3001, 3002),
}


def psnr(u, ref) -> float:
    """Section 5: 20 log10(255 / ||u - ref||) with the RMS norm of Eq. 10."""
    d = np.asarray(u, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    return 20.0 * math.log10(255.0 / math.sqrt(float(np.mean(d * d))))


def _variants(levels, delta):
    big = [1000] * levels
    return [
        ("eecmg-disc", levels, None, dict(stop="discrepancy", delta=delta)),
        ("eecmg-fixed", levels, None, dict(stop="fixed")),
        ("eecmg-disc-uncapped", levels, big, dict(stop="discrepancy", delta=delta)),
        ("iecmg-p", levels, None, dict(stop="discrepancy", delta=delta, prolong="iecmg_p")),
        ("iecmg-l", levels, None, dict(stop="discrepancy", delta=delta, prolong="iecmg_l")),
        ("eecmg-disc-renorm", levels, None, dict(stop="discrepancy", delta=delta, coarse_op="renorm")),
        ("eecmg-disc-cgls", levels, None, dict(stop="discrepancy", delta=delta, smoother="cgls")),
        ("mr2-disc", 1, [1000], dict(stop="discrepancy", delta=delta)),
        ("cgls-disc", 1, [1000], dict(stop="discrepancy", delta=delta, smoother="cgls")),
    ]


def restore(torch, eecmg, g, psf, levels, iters, opts, reps=5):
    """(result, iterations per level, fine-equivalent work, ms per restoration)."""
    h, w = g.shape
    plan = eecmg.Plan(w, h, levels, psf, iters=iters, **opts)
    gd = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    ud = torch.empty_like(gd)
    plan.restore(gd, ud)  # first call captures the plan's CUDA graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        e0.record()
        plan.restore(gd, ud)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    it, _ = plan.stats()
    info = plan.info
    n_fine = float(h * w)
    work = sum(k * hh * ww / n_fine for k, hh, ww in zip(it, info["h"], info["w"]))
    u = ud.double().cpu().numpy()
    plan.close()
    return u, it, work, float(np.median(ms))


def run(cases=None):
    import torch

    from paper_2311_03010_gb300 import eecmg, synth

    eecmg.load()
    rows = []
    for name in cases or CASES:
        h, w, L, spec, v, seed, nseed = CASES[name]
        psf = synth.psf_from_spec(spec)
        p = synth.make_problem(h, w, seed, psf, v, noise_seed=nseed, texture=(h * w > 4096))
        smo = "mr2"
        pg = psnr(p.g, p.u)
        disc_work = None
        for (var, levels, iters, opts) in _variants(L, p.delta):
            u, it, work, ms = restore(torch, eecmg, p.g, psf, levels, iters, dict(dict(smoother=smo), **opts))
            if var == "eecmg-disc":
                disc_work = work
            rows.append((name, var, pg, psnr(u, p.u), it, work, ms))
        k = max(1, int(math.ceil(disc_work)))
        u, it, work, ms = restore(torch, eecmg, p.g, psf, 1, [k], dict(stop="fixed", smoother=smo))
        rows.append((name, "mr2-same-work", pg, psnr(u, p.u), it, work, ms))
    return rows


def table(rows) -> str:
    out = ["| case | variant | PSNR(g) dB | PSNR(u) dB | iterations per level | work (fine-eq. it.) | GPU ms |",
           "|---|---|---|---|---|---|---|"]
    for (name, var, pg, pu, it, work, ms) in rows:
        out.append(f"| {name} | {var} | {pg:.2f} | {pu:.2f} | {it} | {work:.2f} | {ms:.3f} |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--cases", nargs="*", default=None, choices=sorted(CASES))
    args = ap.parse_args()
    print(table(run(args.cases)))


if __name__ == "__main__":
    main()
