"""Python binding of the EECMG C ABI (include/eecmg.h), by ctypes.

Argument marshalling only: every step of the method runs in the CUDA
library ``libeecmg.so``.  Device buffers are passed as torch CUDA tensors
(float32, contiguous) or raw integer addresses; streams as
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or None (the
current torch stream when torch is loaded, else the legacy default stream).
Functions keep the C names; errors raise ``EecmgError``.

The library must have been built (``build_lib.build()``); if it is missing
this module raises at load time rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeecmg.so")

STATUS = {0: "EECMG_OK", 1: "EECMG_ERR_INVALID_ARG", 2: "EECMG_ERR_UNSUPPORTED",
          3: "EECMG_ERR_OOM", 4: "EECMG_ERR_CUDA", 5: "EECMG_ERR_NUMERIC",
          6: "EECMG_ERR_TIMEOUT", 7: "EECMG_ERR_BUSY"}

SMOOTHER = {"mr2": 0, "cgls": 1}
COARSE = {"rms": 0, "renorm": 1}
STORAGE = {"fp32": 0, "bf16": 1}
STOP = {"fixed": 0, "discrepancy": 1}
PROLONG = {"eecmg": 0, "iecmg_p": 1, "iecmg_l": 2}


class EecmgError(RuntimeError):
    def __init__(self, func, status, msg):
        super().__init__(f"{func}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class eecmg_options(ctypes.Structure):
    _fields_ = [
        ("smoother", ctypes.c_int),
        ("coarse_op", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("stop", ctypes.c_int),
        ("c", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("diffusion_steps", ctypes.c_int),
        ("s_scale", ctypes.c_double),
        ("conv_tol", ctypes.c_double),
        ("prolong", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("precise_conv", ctypes.c_int),
        ("persistent", ctypes.c_int),
        ("workspace", ctypes.c_int),
        ("fuse_start", ctypes.c_int),
        ("early_check", ctypes.c_int),
    ]


class eecmg_tuning(ctypes.Structure):
    _fields_ = [("cluster_max_px", ctypes.c_longlong), ("px_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("resident_max_tiles", ctypes.c_int),
                ("psd_tile_h", ctypes.c_int)]


class eecmg_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)

# name -> argtypes (all return eecmg_status unless listed in _RESTYPES)
_SIGS = {
    "eecmg_default_options": [ctypes.POINTER(eecmg_options)],
    "eecmg_plan": [_I, _I, _I, _PD, _I, _I, _D, _D, _PI, ctypes.POINTER(eecmg_options),
                   ctypes.POINTER(_VP)],
    "eecmg_plan_destroy": [_VP],
    "eecmg_plan_info": [_VP, _PI, _PI, _PI, _PI, ctypes.POINTER(ctypes.c_size_t)],
    "eecmg_restore": [_VP, _VP, _VP, _VP],
    "eecmg_restore_host": [_VP, _VP, _VP, _VP],
    "eecmg_restore_batched": [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I,
                              _VP],
    "eecmg_plan_stats": [_VP, _PI, _PD],
    "eecmg_batch_time_step": [ctypes.POINTER(_VP), _I, _I, _I],
    "eecmg_batch_step_time": [ctypes.POINTER(_VP), _I, ctypes.POINTER(ctypes.c_float), _PI, _PD],
    "eecmg_batch_info": [ctypes.POINTER(_VP), _I, _PI],
    "eecmg_restore_batched_host": [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I,
                                   _VP],
    "eecmg_restore_batched_host_async": [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                         _I, _VP],
    "eecmg_level_partition": [_VP, _I, _PI, _PI, _PI],
    "eecmg_plan_profile": [_VP, _I],
    "eecmg_plan_profile_read": [_VP, ctypes.POINTER(eecmg_kernel_stat), _I, _PI],
    "eecmg_apply_H": [_VP, _I, _VP, _VP, _I, _VP],
    "eecmg_restrict": [_VP, _I, _VP, _VP, _VP],
    "eecmg_prolong": [_VP, _I, _VP, _VP, _VP, _VP],
    "eecmg_prolong_single": [_VP, _I, _VP, _VP, _I, _VP],
    "eecmg_start_level": [_VP, _I, _VP, _VP, _VP, _VP],
    "eecmg_smooth": [_VP, _I, _VP, _VP, _VP],
    "eecmg_denoise": [_VP, _I, _VP, _VP, _VP],
    "eecmg_level_solve": [_VP, _I, _VP, _VP, _I, _VP],
    "eecmg_residual_noalloc": [_I, _I, _PD, _I, _I, _VP, _VP, _VP, _VP, _VP],
    "eecmg_selftest_bounded_wait": [_I, _VP],
    "eecmg_probe_fp32_fma": [_I, _VP, _PD],
    "eecmg_get_tuning": [ctypes.POINTER(eecmg_tuning)],
    "eecmg_set_tuning": [ctypes.POINTER(eecmg_tuning)],
    "eecmg_autotune": [ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _I, _VP,
                       ctypes.POINTER(eecmg_tuning)],
    "eecmg_server_create": [ctypes.c_size_t, _I, ctypes.POINTER(_VP)],
    "eecmg_server_submit": [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_uint64)],
    "eecmg_server_poll": [_VP, ctypes.c_uint64, _PI, _PD],
    "eecmg_server_drain": [_VP],
    "eecmg_server_destroy": [_VP],
    "eecmg_vol_plan": [_I, _I, _I, _I, _PD, _I, _I, _I, _D, _D, _PI, ctypes.POINTER(eecmg_options),
                       ctypes.POINTER(_VP)],
    "eecmg_vol_plan_destroy": [_VP],
    "eecmg_vol_plan_info": [_VP, _PI, _PI, _PI, _PI, _PI, ctypes.POINTER(ctypes.c_size_t)],
    "eecmg_vol_restore": [_VP, _VP, _VP, _VP],
    "eecmg_vol_restore_host": [_VP, _VP, _VP, _VP],
    "eecmg_vol_plan_stats": [_VP, _PI, _PD],
    "eecmg_vol_apply_H": [_VP, _I, _VP, _VP, _I, _VP],
    "eecmg_vol_restrict": [_VP, _I, _VP, _VP, _VP],
    "eecmg_vol_start_level": [_VP, _I, _VP, _VP, _VP, _VP],
    "eecmg_vol_smooth": [_VP, _I, _VP, _VP, _VP],
    "eecmg_vol_denoise": [_VP, _I, _VP, _VP, _VP],
    "eecmg_vol_level_solve": [_VP, _I, _VP, _VP, _I, _VP],
    "eecmg_vol_plan_profile": [_VP, _I],
    "eecmg_vol_plan_profile_read": [_VP, _PD, _PD, _PD],
    "eecmg_last_error": [],
    "eecmg_version": [],
}
_RESTYPES = {"eecmg_last_error": ctypes.c_char_p, "eecmg_version": ctypes.c_char_p}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libeecmg.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"EECMG CUDA library not built: {path} is missing "
                           "(run paper_2311_03010_gb300.build_lib.build())")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPES.get(name, ctypes.c_int)
    _lib = lib
    return lib


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise EecmgError(name, st, lib.eecmg_last_error().decode())


def _ptr(x):
    """Device (or host) address of a tensor / array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(x.dtype) != "torch.float32":
            raise ValueError("tensor must be float32")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous float32")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def eecmg_version() -> str:
    return load().eecmg_version().decode()


def eecmg_last_error() -> str:
    return load().eecmg_last_error().decode()


def eecmg_default_options(**kw) -> eecmg_options:
    o = eecmg_options()
    _call("eecmg_default_options", ctypes.byref(o))
    for k, v in kw.items():
        table = {"smoother": SMOOTHER, "coarse_op": COARSE, "storage": STORAGE, "stop": STOP,
                 "prolong": PROLONG}.get(k)
        setattr(o, k, table[v] if (table and isinstance(v, str)) else v)
    return o


def eecmg_plan(width, height, levels, psf, alpha=0.2, k=10.0, iters=None, opt=None, **kw):
    """Returns an opaque plan handle (int).  kw are option overrides."""
    psf = np.ascontiguousarray(psf, dtype=np.float64)
    if opt is None:
        opt = eecmg_default_options(**kw)
    it = None
    if iters is not None:
        it = (ctypes.c_int * levels)(*[int(v) for v in iters])
    h = _VP()
    _call("eecmg_plan", int(width), int(height), int(levels), psf.ctypes.data_as(_PD),
          psf.shape[1], psf.shape[0], float(alpha), float(k), it, ctypes.byref(opt),
          ctypes.byref(h))
    return h.value


def eecmg_plan_destroy(plan):
    _call("eecmg_plan_destroy", plan)


def eecmg_plan_info(plan):
    n = _I()
    _call("eecmg_plan_info", plan, ctypes.byref(n), None, None, None, None)
    L = n.value
    w = (_I * L)()
    hh = (_I * L)()
    m = (_I * L)()
    ws = ctypes.c_size_t()
    _call("eecmg_plan_info", plan, None, w, hh, m, ctypes.byref(ws))
    return {"levels": L, "w": list(w), "h": list(hh), "iters": list(m),
            "workspace_bytes": ws.value}


def eecmg_restore(plan, g, u, stream=None):
    _call("eecmg_restore", plan, _ptr(g), _ptr(u), _stream(stream))


def eecmg_restore_host(plan, g, u, stream=None):
    _call("eecmg_restore_host", plan, _ptr(g), _ptr(u), _stream(stream))


def eecmg_restore_batched(plans, gs, us, stream=None):
    n = len(plans)
    P = (_VP * n)(*plans)
    G = (_VP * n)(*[_ptr(x) for x in gs])
    U = (_VP * n)(*[_ptr(x) for x in us])
    _call("eecmg_restore_batched", P, G, U, n, _stream(stream))


def eecmg_plan_stats(plan):
    L = eecmg_plan_info(plan)["levels"]
    it = (_I * L)()
    res = (_D * L)()
    _call("eecmg_plan_stats", plan, it, res)
    return list(it), list(res)


def eecmg_level_partition(plan, level):
    """(cluster, blocks, resident) of the level's persistent solve."""
    c, b, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _call("eecmg_level_partition", plan, int(level), ctypes.byref(c), ctypes.byref(b), ctypes.byref(r))
    return c.value, b.value, r.value


def eecmg_plan_profile(plan, enable=1):
    _call("eecmg_plan_profile", plan, int(enable))


def eecmg_plan_profile_read(plan):
    """{class: {"launches", "ms", "bytes"}} accumulated since profiling was enabled."""
    n = _I()
    _call("eecmg_plan_profile_read", plan, None, 0, ctypes.byref(n))
    arr = (eecmg_kernel_stat * n.value)()
    _call("eecmg_plan_profile_read", plan, arr, n.value, ctypes.byref(n))
    return {a.name.decode(): {"launches": a.launches, "ms": a.ms, "bytes": a.bytes} for a in arr}


def eecmg_apply_H(plan, level, x, y, transpose=0, stream=None):
    _call("eecmg_apply_H", plan, int(level), _ptr(x), _ptr(y), int(transpose), _stream(stream))


def eecmg_restrict(plan, level, fine, coarse, stream=None):
    _call("eecmg_restrict", plan, int(level), _ptr(fine), _ptr(coarse), _stream(stream))


def eecmg_prolong(plan, level, u1, u2, out, stream=None):
    _call("eecmg_prolong", plan, int(level), _ptr(u1), _ptr(u2), _ptr(out), _stream(stream))


def eecmg_prolong_single(plan, level, u1, out, quadratic=1, stream=None):
    _call("eecmg_prolong_single", plan, int(level), _ptr(u1), _ptr(out), int(quadratic),
          _stream(stream))


def eecmg_start_level(plan, level, u1, u2, out, stream=None):
    _call("eecmg_start_level", plan, int(level), _ptr(u1), _ptr(u2), _ptr(out), _stream(stream))


def eecmg_smooth(plan, level, x, y, stream=None):
    _call("eecmg_smooth", plan, int(level), _ptr(x), _ptr(y), _stream(stream))


def eecmg_denoise(plan, level, x, y, stream=None):
    _call("eecmg_denoise", plan, int(level), _ptr(x), _ptr(y), _stream(stream))


def eecmg_level_solve(plan, level, g, u, m, stream=None):
    _call("eecmg_level_solve", plan, int(level), _ptr(g), _ptr(u), int(m), _stream(stream))


def eecmg_residual_noalloc(width, height, psf, g, u, r, norms, stream=None):
    """r = g - H u and norms[0:2] = (||r||^2, ||g||^2); allocates no device memory.

    norms is a device buffer of two float64 values (tensor or address).
    """
    psf = np.ascontiguousarray(psf, dtype=np.float64)
    if psf.ndim != 2 or psf.shape[0] % 2 != 1 or psf.shape[1] % 2 != 1:
        raise ValueError("psf must be a 2-D array with odd sides")
    if isinstance(norms, int):
        nptr = norms
    else:
        if str(norms.dtype) != "torch.float64" or not norms.is_contiguous() or norms.numel() < 2:
            raise ValueError("norms must be a contiguous float64 tensor of at least 2 elements")
        if not norms.is_cuda:
            raise ValueError("norms must be a device tensor")
        nptr = norms.data_ptr()
    _call("eecmg_residual_noalloc", int(width), int(height), psf.ctypes.data_as(_PD),
          psf.shape[1], psf.shape[0], _ptr(g), _ptr(u), _ptr(r), nptr, _stream(stream))


def _tuning_dict(t):
    return {"cluster_max_px": t.cluster_max_px, "px_per_block": t.px_per_block,
            "blocks_per_sm": t.blocks_per_sm, "resident_max_tiles": t.resident_max_tiles,
            "psd_tile_h": t.psd_tile_h}


def eecmg_restore_batched_host(plans, g_host, u_host, stream=None):
    """Host-buffer batched restoration (host pointers or numpy / pinned torch tensors)."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    hg = (_VP * n)(*[_ptr(x) for x in g_host])
    hu = (_VP * n)(*[_ptr(x) for x in u_host])
    _call("eecmg_restore_batched_host", hp, hg, hu, n, _stream(stream))


def eecmg_restore_batched_host_async(plans, g_host, u_host, stream=None):
    """As eecmg_restore_batched_host, queued on the stream without synchronising: the host
    buffers (pinned, for asynchronous copies) must stay alive until the stream passes it."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    hg = (_VP * n)(*[_ptr(x) for x in g_host])
    hu = (_VP * n)(*[_ptr(x) for x in u_host])
    _call("eecmg_restore_batched_host_async", hp, hg, hu, n, _stream(stream))


def eecmg_batch_info(plans):
    """Device launches (graph nodes) of one eecmg_restore_batched of these plans."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    k = _I()
    _call("eecmg_batch_info", hp, n, ctypes.byref(k))
    return k.value


def eecmg_batch_time_step(plans, step, enable=1):
    """Event pair inside the batched graph of these plans around cascade step `step`'s solves."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    _call("eecmg_batch_time_step", hp, n, int(step), int(enable))


def eecmg_batch_step_time(plans):
    """(ms, level-solve launches, algorithmic bytes) of the hooked step in the last replay."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    ms, k, b = ctypes.c_float(), _I(), _D()
    _call("eecmg_batch_step_time", hp, n, ctypes.byref(ms), ctypes.byref(k), ctypes.byref(b))
    return ms.value, k.value, b.value


def eecmg_get_tuning():
    t = eecmg_tuning()
    _call("eecmg_get_tuning", ctypes.byref(t))
    return _tuning_dict(t)


def eecmg_set_tuning(cluster_max_px, px_per_block, blocks_per_sm, resident_max_tiles=32, psd_tile_h=32):
    t = eecmg_tuning(int(cluster_max_px), int(px_per_block), int(blocks_per_sm), int(resident_max_tiles),
                     int(psd_tile_h))
    _call("eecmg_set_tuning", ctypes.byref(t))


def eecmg_autotune(plans, g, reps=10, stream=None):
    """plans: description-only plan handles (or Plan objects); g: their device inputs."""
    n = len(plans)
    hp = (_VP * n)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    hg = (_VP * n)(*[_ptr(x) for x in g])
    t = eecmg_tuning()
    _call("eecmg_autotune", hp, hg, n, int(reps), _stream(stream), ctypes.byref(t))
    return _tuning_dict(t)


def eecmg_selftest_bounded_wait(cluster, stream=None):
    """Returns the status code (EECMG_ERR_TIMEOUT = 6 is the designed outcome)."""
    lib = load()
    return lib.eecmg_selftest_bounded_wait(int(cluster), _stream(stream))


def eecmg_probe_fp32_fma(reps=5, stream=None):
    """Measured FP32 FMA rate of the current GPU in TFLOP/s (2 flops per FMA)."""
    t = _D()
    _call("eecmg_probe_fp32_fma", int(reps), _stream(stream), ctypes.byref(t))
    return t.value


def eecmg_server_create(mem_budget_bytes, max_slots):
    h = _VP()
    _call("eecmg_server_create", ctypes.c_size_t(int(mem_budget_bytes)), int(max_slots),
          ctypes.byref(h))
    return h.value


def eecmg_server_submit(srv, plan, g, u):
    t = ctypes.c_uint64()
    _call("eecmg_server_submit", srv, plan, _ptr(g), _ptr(u), ctypes.byref(t))
    return t.value


def eecmg_server_poll(srv, ticket):
    done = _I()
    lat = _D()
    _call("eecmg_server_poll", srv, ctypes.c_uint64(ticket), ctypes.byref(done),
          ctypes.byref(lat))
    return bool(done.value), lat.value


def eecmg_server_drain(srv):
    _call("eecmg_server_drain", srv)


def eecmg_server_destroy(srv):
    _call("eecmg_server_destroy", srv)


# ---------------------------------------------------------------- volumes


def eecmg_vol_plan(width, height, depth, levels, psf, alpha=0.2, k=10.0, iters=None, opt=None,
                   **kw):
    """Volume plan handle (int); psf is a (depth, rows, cols) FP64 array."""
    psf = np.ascontiguousarray(psf, dtype=np.float64)
    if psf.ndim != 3:
        raise ValueError("a volume PSF is a 3-D array (slices, rows, cols)")
    if opt is None:
        opt = eecmg_default_options(**kw)
    it = None
    if iters is not None:
        if len(iters) != levels:
            raise ValueError("iters needs one entry per level")
        it = (ctypes.c_int * levels)(*[int(v) for v in iters])
    h = _VP()
    _call("eecmg_vol_plan", int(width), int(height), int(depth), int(levels),
          psf.ctypes.data_as(_PD), psf.shape[2], psf.shape[1], psf.shape[0], float(alpha),
          float(k), it, ctypes.byref(opt), ctypes.byref(h))
    return h.value


def eecmg_vol_plan_destroy(plan):
    _call("eecmg_vol_plan_destroy", plan)


def eecmg_vol_plan_info(plan):
    n = _I()
    _call("eecmg_vol_plan_info", plan, ctypes.byref(n), None, None, None, None, None)
    L = n.value
    w, hh, dd, m = (_I * L)(), (_I * L)(), (_I * L)(), (_I * L)()
    ws = ctypes.c_size_t()
    _call("eecmg_vol_plan_info", plan, None, w, hh, dd, m, ctypes.byref(ws))
    return {"levels": L, "w": list(w), "h": list(hh), "d": list(dd), "iters": list(m),
            "workspace_bytes": ws.value}


def eecmg_vol_restore(plan, g, u, stream=None):
    _call("eecmg_vol_restore", plan, _ptr(g), _ptr(u), _stream(stream))


def eecmg_vol_restore_host(plan, g, u, stream=None):
    _call("eecmg_vol_restore_host", plan, _ptr(g), _ptr(u), _stream(stream))


def eecmg_vol_plan_stats(plan):
    L = eecmg_vol_plan_info(plan)["levels"]
    it = (_I * L)()
    res = (_D * L)()
    _call("eecmg_vol_plan_stats", plan, it, res)
    return list(it), list(res)


def eecmg_vol_plan_profile(plan, enable=1):
    _call("eecmg_vol_plan_profile", plan, int(enable))


def eecmg_vol_plan_profile_read(plan):
    """Per level: (start ms, solve ms, solve algorithmic bytes) of the last restoration."""
    L = eecmg_vol_plan_info(plan)["levels"]
    a, b, c = (_D * L)(), (_D * L)(), (_D * L)()
    _call("eecmg_vol_plan_profile_read", plan, a, b, c)
    return list(a), list(b), list(c)


def eecmg_vol_apply_H(plan, level, x, y, transpose=0, stream=None):
    _call("eecmg_vol_apply_H", plan, int(level), _ptr(x), _ptr(y), int(transpose), _stream(stream))


def eecmg_vol_restrict(plan, level, fine, coarse, stream=None):
    _call("eecmg_vol_restrict", plan, int(level), _ptr(fine), _ptr(coarse), _stream(stream))


def eecmg_vol_start_level(plan, level, u1, u2, out, stream=None):
    _call("eecmg_vol_start_level", plan, int(level), _ptr(u1), _ptr(u2), _ptr(out),
          _stream(stream))


def eecmg_vol_smooth(plan, level, x, y, stream=None):
    _call("eecmg_vol_smooth", plan, int(level), _ptr(x), _ptr(y), _stream(stream))


def eecmg_vol_denoise(plan, level, x, y, stream=None):
    _call("eecmg_vol_denoise", plan, int(level), _ptr(x), _ptr(y), _stream(stream))


def eecmg_vol_level_solve(plan, level, g, u, m, stream=None):
    _call("eecmg_vol_level_solve", plan, int(level), _ptr(g), _ptr(u), int(m), _stream(stream))


class VolumePlan:
    """Owning wrapper of a volume plan (eecmg_vol_plan / eecmg_vol_plan_destroy)."""

    def __init__(self, width, height, depth, levels, psf, alpha=0.2, k=10.0, iters=None, **opts):
        self.h = eecmg_vol_plan(width, height, depth, levels, psf, alpha, k, iters, **opts)
        self.info = eecmg_vol_plan_info(self.h)

    def close(self):
        if self.h:
            eecmg_vol_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def restore(self, g, u, stream=None):
        eecmg_vol_restore(self.h, g, u, stream)

    def stats(self):
        return eecmg_vol_plan_stats(self.h)


class Plan:
    """Owning wrapper of an eecmg_plan_t (destroyed with the object)."""

    def __init__(self, width, height, levels, psf, alpha=0.2, k=10.0, iters=None, **opts):
        self.width, self.height, self.levels = int(width), int(height), int(levels)
        self.handle = eecmg_plan(width, height, levels, psf, alpha, k, iters, **opts)
        self.info = eecmg_plan_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            eecmg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def restore(self, g, u, stream=None):
        eecmg_restore(self.handle, g, u, stream)

    def stats(self):
        return eecmg_plan_stats(self.handle)


class Server:
    """Owning wrapper of an eecmg_server_t (drained and destroyed on close)."""

    def __init__(self, mem_budget_bytes, max_slots):
        self.handle = eecmg_server_create(mem_budget_bytes, max_slots)

    def submit(self, plan, g, u):
        return eecmg_server_submit(self.handle, plan.handle if isinstance(plan, Plan) else plan, g, u)

    def poll(self, ticket):
        return eecmg_server_poll(self.handle, ticket)

    def drain(self):
        eecmg_server_drain(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            eecmg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
