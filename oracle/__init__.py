"""FP64 CPU oracle for EECMG image restoration (Chu, Yan & Li).

TEST INFRASTRUCTURE.  This package is the independent checker for the CUDA
library: a plain, slow, single-definition FP64 restatement of the paper's
operators and of Algorithm 2 (and Algorithm 1), in C (``eecmg_oracle.c``),
loaded here through ctypes.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import it; the product path never does.
It shares no code with the CUDA library.

Every function takes and returns float64 numpy arrays of shape (rows, cols).

Parity status per function (what pins it; see the tests under tests/):
  apply_H / apply_HT   pinned: delta response = PSF, brute-force adjoint,
                       dense Kronecker form h (x) h, PSF = delta gives I.
  coarse_psf           pinned: dense R H R^* product (Eq. 14) on tiny grids.
  schedule             pinned: hand evaluation of the Section 2 formulas.
  mr2 / cgls           pinned: explicit Krylov least squares (brute force),
                       dense LU solve at k = N, monotone residuals.
  extrapolate          pinned: the printed 1-D cases and exactness on the
                       extrapolation's error model.
  quadratic            pinned: exact on biquadratic polynomials; the two
                       printed 1-D forms agree.
  linear               pinned: Eq. 15 printed cases, exact on bilinear-free
                       planes a + b x + c y.
  smooth               pinned: per-pixel weighted lstsq (numpy), constants
                       and planes unchanged.
  denoise              pinned: dense A(u) of Eq. 26, conservation, k -> inf
                       limit, constants unchanged, max principle.
  cascade              pinned: PSF = delta returns g exactly; end-to-end
                       values against the paper are unpinned (the paper's
                       test image is not published).

The volume functions (suffix 3; arrays of shape (slices, rows, cols)) carry
the method to 3-D, which the paper names but does not write out.  Pinned:
with one slice and a one-slice PSF each equals its pinned 2-D function;
permuting the three axes of the input (and of the PSF) permutes the output
the same way, which ties the slice axis to the pinned row and column axes;
apply_H3 equals scipy.ndimage.convolve with zero fill; coarse_psf3 equals
the dense R H R^* product; quadratic3 is exact on triquadratics; smooth3
equals a per-voxel weighted lstsq (numpy) and keeps affine volumes;
denoise3 conserves the sum and keeps constants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eecmg_oracle.c")
_LIB = os.path.join(_HERE, "libeecmg_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile eecmg_oracle.c into libeecmg_oracle.so with gcc (OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Options(ctypes.Structure):
    _fields_ = [
        ("smoother", ctypes.c_int),
        ("coarse_op", ctypes.c_int),
        ("prolong", ctypes.c_int),
        ("stop", ctypes.c_int),
        ("c", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("diffusion_steps", ctypes.c_int),
        ("s_scale", ctypes.c_double),
        ("conv_tol", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_dot.restype = ctypes.c_double
            lib.or_rms.restype = ctypes.c_double
            lib.or_psnr.restype = ctypes.c_double
            lib.or_mr2.restype = ctypes.c_int
            lib.or_cgls.restype = ctypes.c_int
            lib.or_cascade.restype = ctypes.c_int
            lib.or_cascade3.restype = ctypes.c_int
            lib.or_mr2_3.restype = ctypes.c_int
            lib.or_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_max_threads())


def level_sizes(h: int, w: int, L: int):
    hs = (ctypes.c_int * L)()
    ws = (ctypes.c_int * L)()
    _load().or_level_sizes(h, w, L, hs, ws)
    return list(hs), list(ws)


def restrict(fine, hc: int, wc: int) -> np.ndarray:
    fine = _f64(fine)
    out = np.zeros((hc, wc))
    _load().or_restrict(_p(fine), fine.shape[0], fine.shape[1], _p(out), hc, wc)
    return out


def apply_H(K, x) -> np.ndarray:
    K, x = _f64(K), _f64(x)
    y = np.zeros_like(x)
    _load().or_apply_H(_p(K), K.shape[0], K.shape[1], _p(x), x.shape[0], x.shape[1], _p(y))
    return y


def apply_HT(K, x) -> np.ndarray:
    K, x = _f64(K), _f64(x)
    y = np.zeros_like(x)
    _load().or_apply_HT(_p(K), K.shape[0], K.shape[1], _p(x), x.shape[0], x.shape[1], _p(y))
    return y


def coarse_psf(K, rho: float) -> np.ndarray:
    K = _f64(K)
    ch = 2 * (K.shape[0] // 2 // 2) + 1
    cw = 2 * (K.shape[1] // 2 // 2) + 1
    out = np.zeros((ch, cw))
    a, b = ctypes.c_int(), ctypes.c_int()
    _load().or_coarse_psf(_p(K), K.shape[0], K.shape[1], ctypes.c_double(rho), _p(out),
                          ctypes.byref(a), ctypes.byref(b))
    assert (a.value, b.value) == (ch, cw)
    return out


def schedule(L: int):
    m = (ctypes.c_int * L)()
    _load().or_schedule(L, m)
    return list(m)


def dot(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return float(_load().or_dot(_p(x), _p(y), x.shape[0], x.shape[1]))


def rms(x) -> float:
    x = _f64(x)
    return float(_load().or_rms(_p(x), x.shape[0], x.shape[1]))


def _solver(fn, K, g, u0, m, stop_tol, conv_tol):
    K, g = _f64(K), _f64(g)
    u = _f64(u0).copy() if u0 is not None else np.zeros_like(g)
    res = ctypes.c_double()
    k = fn(_p(K), K.shape[0], K.shape[1], _p(g), g.shape[0], g.shape[1], _p(u), int(m),
           ctypes.c_double(stop_tol), ctypes.c_double(conv_tol), ctypes.byref(res))
    return u, int(k), float(res.value)


def mr2(K, g, u0=None, m=1, stop_tol=0.0, conv_tol=0.0):
    """MR-II for at most m iterations from u0; returns (u, iterations, ||r||_RMS)."""
    return _solver(_load().or_mr2, K, g, u0, m, stop_tol, conv_tol)


def cgls(K, g, u0=None, m=1, stop_tol=0.0, conv_tol=0.0):
    """CGLS for at most m iterations from u0; returns (u, iterations, ||r||_RMS)."""
    return _solver(_load().or_cgls, K, g, u0, m, stop_tol, conv_tol)


def extrapolate(u1, u2) -> np.ndarray:
    u1, u2 = _f64(u1), _f64(u2)
    out = np.zeros_like(u1)
    _load().or_extrapolate(_p(u1), u1.shape[0], u1.shape[1], _p(u2), u2.shape[0], u2.shape[1],
                           _p(out))
    return out


def quadratic(ut, h: int, w: int) -> np.ndarray:
    ut = _f64(ut)
    out = np.zeros((h, w))
    _load().or_quadratic(_p(ut), ut.shape[0], ut.shape[1], _p(out), h, w)
    return out


def linear(uc, h: int, w: int) -> np.ndarray:
    uc = _f64(uc)
    out = np.zeros((h, w))
    _load().or_linear(_p(uc), uc.shape[0], uc.shape[1], _p(out), h, w)
    return out


def smooth(u, scale: float = 1.0) -> np.ndarray:
    u = _f64(u)
    out = np.zeros_like(u)
    _load().or_smooth(_p(u), u.shape[0], u.shape[1], ctypes.c_double(scale), _p(out))
    return out


def denoise(u, tau: float, k: float) -> np.ndarray:
    u = _f64(u)
    out = np.zeros_like(u)
    _load().or_denoise(_p(u), u.shape[0], u.shape[1], ctypes.c_double(tau), ctypes.c_double(k),
                       _p(out))
    return out


# Default convergence stop of a level solve: ||r|| <= CONV_TOL * ||g_l||.
CONV_TOL = 1e-5

_SMOOTHERS = {"mr2": 0, "cgls": 1}
_COARSE = {"rms": 0, "renorm": 1}
_PROLONG = {"eecmg": 0, "iecmg_p": 1, "iecmg_l": 2}


def cascade(g, L: int, psf, tau: float = 0.2, k: float = 10.0, iters=None,
            smoother: str = "mr2", coarse_op: str = "rms", prolong: str = "eecmg",
            stop: str = "discrepancy", c: float = 1.1, delta: float = 0.0,
            diffusion_steps: int = 1, s_scale: float = 1.0, conv_tol: float = CONV_TOL):
    """Algorithm 2 (or Algorithm 1) on data g; returns (u, iterations, ||r||_RMS per level)."""
    g, psf = _f64(g), _f64(psf)
    h, w = g.shape
    o = _Options(_SMOOTHERS[smoother], _COARSE[coarse_op], _PROLONG[prolong],
                 1 if stop == "discrepancy" else 0, c, delta, diffusion_steps, s_scale,
                 conv_tol)
    u = np.zeros_like(g)
    it = (ctypes.c_int * L)()
    res = (ctypes.c_double * L)()
    it_arr = None
    if iters is not None:
        it_arr = (ctypes.c_int * L)(*[int(v) for v in iters])
    rc = _load().or_cascade(_p(g), h, w, int(L), _p(psf), psf.shape[0], psf.shape[1],
                            ctypes.c_double(tau), ctypes.c_double(k), it_arr,
                            ctypes.byref(o), _p(u), it, res)
    if rc != 0:
        raise ValueError("oracle cascade: invalid arguments")
    return u, list(it), list(res)


def psnr(u, uh) -> float:
    u, uh = _f64(u), _f64(uh)
    return float(_load().or_psnr(_p(u), _p(uh), u.shape[0], u.shape[1]))


# ---------------------------------------------------------------- volumes


def _shape3(a):
    assert a.ndim == 3, "volume functions take (slices, rows, cols) arrays"
    return a.shape


def level_sizes3(d: int, h: int, w: int, L: int):
    ds, hs, ws = (ctypes.c_int * L)(), (ctypes.c_int * L)(), (ctypes.c_int * L)()
    _load().or_level_sizes3(d, h, w, L, ds, hs, ws)
    return list(ds), list(hs), list(ws)


def restrict3(fine, dc: int, hc: int, wc: int) -> np.ndarray:
    fine = _f64(fine)
    out = np.zeros((dc, hc, wc))
    _load().or_restrict3(_p(fine), *_shape3(fine), _p(out), dc, hc, wc)
    return out


def apply_H3(K, x) -> np.ndarray:
    K, x = _f64(K), _f64(x)
    y = np.zeros_like(x)
    _load().or_apply_H3(_p(K), *_shape3(K), _p(x), *_shape3(x), _p(y))
    return y


def apply_HT3(K, x) -> np.ndarray:
    K, x = _f64(K), _f64(x)
    y = np.zeros_like(x)
    _load().or_apply_HT3(_p(K), *_shape3(K), _p(x), *_shape3(x), _p(y))
    return y


def coarse_psf3(K, rho: float) -> np.ndarray:
    K = _f64(K)
    cs = tuple(2 * (n // 2 // 2) + 1 for n in _shape3(K))
    out = np.zeros(cs)
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _load().or_coarse_psf3(_p(K), *K.shape, ctypes.c_double(rho), _p(out), ctypes.byref(a),
                           ctypes.byref(b), ctypes.byref(c))
    assert (a.value, b.value, c.value) == cs
    return out


def mr2_3(K, g, u0=None, m=1, stop_tol=0.0, conv_tol=0.0):
    """MR-II on a volume for at most m iterations; returns (u, iterations, ||r||_RMS)."""
    K, g = _f64(K), _f64(g)
    u = _f64(u0).copy() if u0 is not None else np.zeros_like(g)
    res = ctypes.c_double()
    k = _load().or_mr2_3(_p(K), *_shape3(K), _p(g), *_shape3(g), _p(u), int(m),
                         ctypes.c_double(stop_tol), ctypes.c_double(conv_tol), ctypes.byref(res))
    return u, int(k), float(res.value)


def extrapolate3(u1, u2) -> np.ndarray:
    u1, u2 = _f64(u1), _f64(u2)
    out = np.zeros_like(u1)
    _load().or_extrapolate3(_p(u1), *_shape3(u1), _p(u2), *_shape3(u2), _p(out))
    return out


def quadratic3(ut, d: int, h: int, w: int) -> np.ndarray:
    ut = _f64(ut)
    out = np.zeros((d, h, w))
    _load().or_quadratic3(_p(ut), *_shape3(ut), _p(out), d, h, w)
    return out


def smooth3(u, scale: float = 1.0) -> np.ndarray:
    u = _f64(u)
    out = np.zeros_like(u)
    _load().or_smooth3(_p(u), *_shape3(u), ctypes.c_double(scale), _p(out))
    return out


def denoise3(u, tau: float, k: float) -> np.ndarray:
    u = _f64(u)
    out = np.zeros_like(u)
    _load().or_denoise3(_p(u), *_shape3(u), ctypes.c_double(tau), ctypes.c_double(k), _p(out))
    return out


def cascade3(g, L: int, psf, tau: float = 0.2, k: float = 10.0, iters=None,
             coarse_op: str = "rms", stop: str = "discrepancy", c: float = 1.1,
             delta: float = 0.0, diffusion_steps: int = 1, s_scale: float = 1.0,
             conv_tol: float = CONV_TOL):
    """Algorithm 2 on a volume g (MR-II); returns (u, iterations, ||r||_RMS per level)."""
    g, psf = _f64(g), _f64(psf)
    o = _Options(0, _COARSE[coarse_op], 0, 1 if stop == "discrepancy" else 0, c, delta,
                 diffusion_steps, s_scale, conv_tol)
    u = np.zeros_like(g)
    it = (ctypes.c_int * L)()
    res = (ctypes.c_double * L)()
    it_arr = None
    if iters is not None:
        it_arr = (ctypes.c_int * L)(*[int(v) for v in iters])
    rc = _load().or_cascade3(_p(g), *_shape3(g), int(L), _p(psf), *_shape3(psf),
                             ctypes.c_double(tau), ctypes.c_double(k), it_arr, ctypes.byref(o),
                             _p(u), it, res)
    if rc != 0:
        raise ValueError("oracle cascade3: invalid arguments")
    return u, list(it), list(res)
