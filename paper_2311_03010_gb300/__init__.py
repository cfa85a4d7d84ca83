"""GB300 (sm_103a) implementation of EECMG image restoration.

Extrapolation Economy Cascadic Multigrid (Chu, Yan & Li): a coarse-to-fine
cascade of Krylov level solves (MR-II or CGLS) joined by a nonlinear
prolongation (new extrapolation + quadratic interpolation), local
weighted-least-squares smoothing and an explicit Perona-Malik step.

The compute path is the CUDA C-ABI library ``libeecmg.so`` (include/eecmg.h);
``eecmg`` is its Python binding and ``synth`` makes seeded test workloads.
"""
from . import eecmg  # noqa: F401
