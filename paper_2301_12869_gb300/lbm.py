"""Thin ctypes binding of liblbm (C ABI in include/lbm.h).

The functions below carry the ABI's names and only marshal arguments: every
step of the computation runs in the library's CUDA kernels. Buffers can be
given as numpy arrays (host), torch tensors (host or CUDA) or raw integer
addresses. PyTorch is used, when present, only to allocate device memory and to
pick the current CUDA stream (``Lattice``).

There is no fallback: if ``_lib/liblbm.so`` has not been built (``python -m
paper_2301_12869_gb300._build`` or ``__graft_entry__.build()``), loading fails
with an error.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblbm.so")

# ---- constants of include/lbm.h
LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENONPHYS, LBM_ETIMEOUT, LBM_ENOMEM = 0, -1, -2, -3, -4, -5
LBM_FP64, LBM_FP32, LBM_DOUBLE_FLOAT = 0, 1, 2
LBM_GRAVITY_RHO_G, LBM_GRAVITY_RHO_MINUS_MEAN_G = 1, 2
LBM_HOST, LBM_DEVICE = 0, 1
LBM_WALL_BOUNCE_BACK, LBM_WALL_ZOU_HE = 0, 1
(LBM_REDUCE_MASS, LBM_REDUCE_MEAN_RHO, LBM_REDUCE_RESIDUAL, LBM_REDUCE_MAX_U,
 LBM_REDUCE_INTERFACE_Y, LBM_REDUCE_RHO_LV) = range(6)

ERROR_NAMES = {
    LBM_EINVAL: "LBM_EINVAL", LBM_ECUDA: "LBM_ECUDA", LBM_ENONPHYS: "LBM_ENONPHYS",
    LBM_ETIMEOUT: "LBM_ETIMEOUT", LBM_ENOMEM: "LBM_ENOMEM",
}

#: every symbol include/lbm.h declares
EXPORTS = (
    "lbm_params_default", "lbm_workspace_bytes", "lbm_init", "lbm_step", "lbm_moments", "lbm_reduce",
    "lbm_get_state", "lbm_set_state", "lbm_set_params", "lbm_status", "lbm_destroy", "lbm_last_error",
    "lbm_critical_point", "lbm_coexistence", "lbm_launch_info", "lbm_step_noalloc",
    "lbm_autotune", "lbm_tile_variants", "lbm_set_tiling", "lbm_set_temperature", "lbm_get_temperature",
    "lbm_batch_init", "lbm_batch_run", "lbm_batch_run_stall", "lbm_batch_set_acceleration", "lbm_batch_results", "lbm_batch_moments", "lbm_batch_get_state", "lbm_batch_rest_state",
    "lbm_batch_convert", "lbm_batch_destroy", "lbm_batch_column_seconds",
    "lbm_batch_set_threads", "lbm_batch_autotune", "lbm_wait_bound_selftest",
    "lbm_mlp_create", "lbm_mlp_set_params", "lbm_mlp_get_params", "lbm_mlp_gradients", "lbm_mlp_train",
    "lbm_mlp_predict", "lbm_mlp_features", "lbm_mlp_warm_start", "lbm_mlp_gemm", "lbm_mlp_gemm_enqueue",
    "lbm_mlp_destroy", "lbm_slab_partials", "lbm_slab_init", "lbm_slab_mass", "lbm_slab_step",
)

MLP_WIDTH, MLP_INPUTS, MLP_IN_PAD = 128, 6, 16
#: packed parameter layout of the warm-start network: (name, shape) in order
MLP_LAYOUT = (("W1", (128, 16)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 128)),
              ("b3", (128,)), ("w4", (128,)), ("b4", (1,)))
MLP_NPARAMS = sum(int(np.prod(sh)) for _, sh in MLP_LAYOUT)


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32), ("precision", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double), ("T", ctypes.c_double),
        ("G", ctypes.c_double), ("sigma", ctypes.c_double),
        ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double), ("tau_varsigma", ctypes.c_double),
        ("tau_j", ctypes.c_double), ("tau_q", ctypes.c_double), ("tau_nu", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("gravity_form", ctypes.c_int32), ("thermal", ctypes.c_int32),
        ("rho_ref", ctypes.c_double), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
        ("c_v", ctypes.c_double), ("kappa", ctypes.c_double), ("T_bot", ctypes.c_double), ("T_top", ctypes.c_double),
        ("wall", ctypes.c_int32), ("reserved1", ctypes.c_int32),
    ]


class lbm_column(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("gravity_form", ctypes.c_int32), ("T", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double)]


class lbm_slab(ctypes.Structure):
    _fields_ = [("y0", ctypes.c_int32), ("ny_own", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("reserved2", ctypes.c_int32)]


LBM_SLAB_HALO = 2


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbm.so once; raises if it is missing (the CUDA path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblbm.so not built at {path}; run paper_2301_12869_gb300._build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, d, i32, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    sig = {
        "lbm_params_default": (None, [P(lbm_params)]),
        "lbm_workspace_bytes": (i32, [P(lbm_params), P(ctypes.c_uint64)]),
        "lbm_init": (i32, [P(lbm_params), vp, i32, vp, P(vp)]),
        "lbm_step": (i32, [vp, i64]),
        "lbm_moments": (i32, [vp, vp, vp, vp, i32]),
        "lbm_reduce": (i32, [vp, i32, P(d)]),
        "lbm_get_state": (i32, [vp, vp, i32, P(i64)]),
        "lbm_set_state": (i32, [vp, vp, i32, i64]),
        "lbm_set_params": (i32, [vp, P(lbm_params)]),
        "lbm_status": (i32, [vp]),
        "lbm_destroy": (i32, [vp]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_critical_point": (i32, [d, d, d, P(d), P(d), P(d)]),
        "lbm_coexistence": (i32, [d, d, d, d, P(d), P(d), P(d)]),
        "lbm_launch_info": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(i32), P(i32)]),
        "lbm_step_noalloc": (i32, [P(lbm_params), vp, vp, vp]),
        "lbm_autotune": (i32, [vp, i32, P(i32), P(d)]),
        "lbm_tile_variants": (i32, [i32]),
        "lbm_set_tiling": (i32, [vp, i32]),
        "lbm_set_temperature": (i32, [vp, vp, i32]),
        "lbm_get_temperature": (i32, [vp, vp, i32]),
        "lbm_batch_init": (i32, [P(lbm_params), P(lbm_column), i32, vp, i32, vp, P(vp)]),
        "lbm_batch_run": (i32, [vp, d, i64, i32, P(d)]),
        "lbm_batch_run_stall": (i32, [vp, d, i64, i32, i32, P(d)]),
        "lbm_batch_set_acceleration": (i32, [vp, i32]),
        "lbm_batch_set_threads": (i32, [vp, i32]),
        "lbm_wait_bound_selftest": (i32, [ctypes.c_longlong]),
        "lbm_batch_autotune": (i32, [vp, i32, vp, vp]),
        "lbm_batch_results": (i32, [vp, vp, vp, vp]),
        "lbm_batch_moments": (i32, [vp, vp, vp, vp, i32]),
        "lbm_batch_get_state": (i32, [vp, vp, i32]),
        "lbm_batch_rest_state": (i32, [vp]),
        "lbm_batch_convert": (i32, [vp, i32, P(vp)]),
        "lbm_batch_destroy": (i32, [vp]),
        "lbm_batch_column_seconds": (i32, [vp, vp]),
        "lbm_mlp_create": (i32, [vp, i32, vp, P(vp)]),
        "lbm_mlp_set_params": (i32, [vp, vp]),
        "lbm_mlp_get_params": (i32, [vp, vp]),
        "lbm_mlp_gradients": (i32, [vp, vp, vp, i32, vp, P(d)]),
        "lbm_mlp_train": (i32, [vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_ulonglong, vp]),
        "lbm_mlp_predict": (i32, [vp, vp, i64, vp]),
        "lbm_mlp_features": (i32, [vp, i32, i32, d, d, d, vp, vp, vp, vp, vp]),
        "lbm_mlp_warm_start": (i32, [vp, vp, i32, i32, d, d, d, vp, vp]),
        "lbm_mlp_gemm": (i32, [vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, i32, vp]),
        "lbm_mlp_gemm_enqueue": (i32, [vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, i32, vp, vp]),
        "lbm_mlp_destroy": (i32, [vp]),
        "lbm_slab_partials": (i32, [P(lbm_params), P(lbm_slab), P(i32)]),
        "lbm_slab_init": (i32, [P(lbm_params), P(lbm_slab), vp, vp, vp]),
        "lbm_slab_mass": (i32, [P(lbm_params), P(lbm_slab), vp, vp, i32, vp]),
        "lbm_slab_step": (i32, [P(lbm_params), P(lbm_slab), vp, vp, vp, i32, vp, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, h=None):
    if rc != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LbmError(rc, msg.decode() if msg else "")
    return rc


def _ptr(buf):
    """(address, where) of a numpy array, torch tensor or raw int (int = device address)."""
    if buf is None:
        return None, None
    if isinstance(buf, int):
        return buf, LBM_DEVICE
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous or buf.dtype != np.float64:
            raise ValueError("host buffers must be C-contiguous float64 arrays")
        return buf.ctypes.data, LBM_HOST
    if hasattr(buf, "data_ptr"):  # torch tensor
        if not buf.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return buf.data_ptr(), (LBM_DEVICE if buf.is_cuda else LBM_HOST)
    raise TypeError(f"unsupported buffer type {type(buf)}")


# ---------------------------------------------------------------- ABI functions
def lbm_params_default():
    p = lbm_params()
    load().lbm_params_default(ctypes.byref(p))
    return p


def lbm_workspace_bytes(p):
    n = ctypes.c_uint64()
    _check(load().lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def lbm_init(p, rho0, stream=None):
    addr, where = _ptr(rho0)
    h = ctypes.c_void_p()
    _check(load().lbm_init(ctypes.byref(p), addr, where, stream, ctypes.byref(h)))
    return h


def lbm_step(h, nsteps):
    _check(load().lbm_step(h, int(nsteps)), h)


def lbm_moments(h, rho=None, ux=None, uy=None):
    wheres = {w for _, w in map(_ptr, (rho, ux, uy)) if w is not None}
    if len(wheres) > 1:
        raise ValueError("moment outputs must all be host or all be device buffers")
    where = wheres.pop() if wheres else LBM_HOST
    _check(load().lbm_moments(h, _ptr(rho)[0], _ptr(ux)[0], _ptr(uy)[0], where), h)


def lbm_reduce(h, kind, check=True):
    out = (ctypes.c_double * 2)(math.nan, math.nan)
    rc = load().lbm_reduce(h, kind, out)
    if check:
        _check(rc, h)
    vals = [out[0], out[1]] if kind == LBM_REDUCE_RHO_LV else [out[0]]
    return (vals, rc) if not check else vals


def lbm_get_state(h, f):
    addr, where = _ptr(f)
    steps = ctypes.c_int64()
    _check(load().lbm_get_state(h, addr, where, ctypes.byref(steps)), h)
    return steps.value


def lbm_set_state(h, f, steps_done=0):
    addr, where = _ptr(f)
    _check(load().lbm_set_state(h, addr, where, int(steps_done)), h)


def lbm_set_temperature(h, T):
    addr, where = _ptr(T)
    _check(load().lbm_set_temperature(h, addr, where), h)


def lbm_get_temperature(h, T):
    addr, where = _ptr(T)
    _check(load().lbm_get_temperature(h, addr, where), h)


def lbm_set_params(h, p):
    _check(load().lbm_set_params(h, ctypes.byref(p)), h)


def lbm_status(h):
    return load().lbm_status(h)


def lbm_destroy(h):
    _check(load().lbm_destroy(h))


def lbm_last_error(h=None):
    msg = load().lbm_last_error(h)
    return msg.decode() if msg else ""


def lbm_critical_point(a, b, R):
    rc_, Tc, pc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_critical_point(a, b, R, ctypes.byref(rc_), ctypes.byref(Tc), ctypes.byref(pc)))
    return rc_.value, Tc.value, pc.value


def lbm_coexistence(a, b, R, T):
    rv, rl, ps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_coexistence(a, b, R, T, ctypes.byref(rv), ctypes.byref(rl), ctypes.byref(ps)))
    return rv.value, rl.value, ps.value


def lbm_launch_info(h):
    vals = [ctypes.c_int() for _ in range(6)]
    _check(load().lbm_launch_info(h, *[ctypes.byref(v) for v in vals]), h)
    keys = ("grid", "block", "smem_bytes", "band_width", "strip_rows", "stages")
    return {k: v.value for k, v in zip(keys, vals)}


def lbm_autotune(h, steps=20):
    """Times the fused kernel's tile variants on this lattice and keeps the fastest;
    returns (variant, ms per step)."""
    v, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().lbm_autotune(h, int(steps), ctypes.byref(v), ctypes.byref(ms)), h)
    return v.value, ms.value


def lbm_tile_variants(precision):
    n = load().lbm_tile_variants(int(precision))
    if n < 0:
        _check(n)
    return n


def lbm_set_tiling(h, variant):
    _check(load().lbm_set_tiling(h, int(variant)), h)


def _noalloc_buffer(t, name, p):
    """Address of a populations array for lbm_step_noalloc: a contiguous torch CUDA tensor
    on the current device, of the precision's real type, with 9 nx ny elements. The C side
    receives only a pointer, so a host array or a short / wrongly typed one is refused here
    before it can reach the kernel as a device address."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch CUDA tensor (got {type(t).__name__})")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must live on the current CUDA device (got {t.device})")
    want = torch.float32 if p.precision == LBM_FP32 else torch.float64
    if t.dtype != want:
        raise ValueError(f"{name} must be {want} for this precision (got {t.dtype})")
    if t.numel() != 9 * p.nx * p.ny:
        raise ValueError(f"{name} must hold 9 nx ny = {9 * p.nx * p.ny} values (got {t.numel()})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def lbm_step_noalloc(p, f_in, f_out, stream=None):
    """One step f_out = step(f_in) on caller-owned device arrays of deviations
    f_i - w_i rho_ref (real type of p.precision), with no device allocation."""
    a_in, a_out = _noalloc_buffer(f_in, "f_in", p), _noalloc_buffer(f_out, "f_out", p)
    _check(load().lbm_step_noalloc(ctypes.byref(p), a_in, a_out, stream))


def _slab_ptr(t, name):
    """Device address of a contiguous torch CUDA tensor (slab calls take device pointers only)."""
    if t is None:
        return None
    if not (hasattr(t, "data_ptr") and t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous torch CUDA tensor")
    return t.data_ptr()


def make_slab(y0, ny_own):
    s = lbm_slab()
    s.y0, s.ny_own = int(y0), int(ny_own)
    return s


def lbm_slab_partials(p, s):
    n = ctypes.c_int()
    _check(load().lbm_slab_partials(ctypes.byref(p), ctypes.byref(s), ctypes.byref(n)))
    return n.value


def lbm_slab_init(p, s, rho0, f, stream=None):
    """Own rows of the slab buffer f = rest equilibrium of rho0 (ny_own x nx, device FP64)."""
    _check(load().lbm_slab_init(ctypes.byref(p), ctypes.byref(s), _slab_ptr(rho0, "rho0"), _slab_ptr(f, "f"), stream))


def lbm_slab_mass(p, s, f, part, stream=None):
    """The FP64 mass partials of the slab's own rows into part (device, >= lbm_slab_partials)."""
    _check(load().lbm_slab_mass(ctypes.byref(p), ctypes.byref(s), _slab_ptr(f, "f"), _slab_ptr(part, "part"),
                                int(part.numel()), stream))


def lbm_slab_step(p, s, f_in, f_out, part_in, part_out, status, stream=None):
    """One step of the slab; part_in: the domain's partials of f_in (summed over slabs)."""
    _check(load().lbm_slab_step(ctypes.byref(p), ctypes.byref(s), _slab_ptr(f_in, "f_in"), _slab_ptr(f_out, "f_out"),
                                _slab_ptr(part_in, "part_in"), 0 if part_in is None else int(part_in.numel()),
                                _slab_ptr(part_out, "part_out"), int(part_out.numel()), _slab_ptr(status, "status"),
                                stream))


def lbm_batch_init(p, columns, rho0, stream=None):
    """columns: sequence of dicts with ny, gravity_form (or form), T, gx, gy."""
    arr = (lbm_column * len(columns))()
    for c, col in zip(arr, columns):
        c.ny = int(col["ny"])
        c.gravity_form = int(col.get("gravity_form", col.get("form", 1)))
        c.T = float(col["T"])
        c.gx = float(col.get("gx", 0.0))
        c.gy = float(col.get("gy", 0.0))
    addr, where = _ptr(rho0)
    b = ctypes.c_void_p()
    _check(load().lbm_batch_init(ctypes.byref(p), arr, len(columns), addr, where, stream, ctypes.byref(b)))
    return b


def lbm_batch_run(b, tol, max_steps, check_every=100):
    """Runs every column to its residual target or max_steps; returns the device seconds."""
    sec = ctypes.c_double()
    _check(load().lbm_batch_run(b, float(tol), int(max_steps), int(check_every), ctypes.byref(sec)))
    return sec.value


def lbm_batch_run_stall(b, tol, max_steps, check_every=100, stall_checks=10):
    """lbm_batch_run, with each column also stopping at its rounding floor (no 1 % gain in
    stall_checks consecutive checks); returns the device seconds."""
    sec = ctypes.c_double()
    _check(load().lbm_batch_run_stall(b, float(tol), int(max_steps), int(check_every), int(stall_checks),
                                      ctypes.byref(sec)))
    return sec.value


def lbm_batch_set_acceleration(b, checks):
    """Extrapolation every `checks` residual checks (0: off) for later runs of this batch."""
    _check(load().lbm_batch_set_acceleration(b, int(checks)))


def lbm_wait_bound_selftest(cycles=2_000_000):
    """The device-side bounded wait's failure path on purpose: returns LBM_ETIMEOUT's code
    when the wait gave up and its status came back (the expected outcome), else raises."""
    rc = load().lbm_wait_bound_selftest(int(cycles))
    if rc != LBM_ETIMEOUT:
        _check(rc if rc != LBM_OK else LBM_EINVAL)
    return rc


def lbm_batch_set_threads(b, threads):
    """Block size of the batched kernel: 128, 256 (default) or 512 threads per column CTA."""
    _check(load().lbm_batch_set_threads(b, int(threads)))


def lbm_batch_autotune(b, steps=200):
    """Times each block size on a copy of the batch's state and keeps the fastest; returns
    (threads kept, {threads: microseconds per step of the whole batch})."""
    th = (ctypes.c_int * 3)()
    us = (ctypes.c_double * 3)()
    _check(load().lbm_batch_autotune(b, int(steps), th, us))
    times = {int(th[i]): float(us[i]) for i in range(3)}
    return min(times, key=times.get), times


def batch_tuned_threads(b, cache_path, key, steps=200):
    """lbm_batch_autotune with its result cached in a JSON file: the block size stored under
    `key` (a string naming the GPU and the batch's shape) is applied without timing; else the
    batch is tuned and the choice and its timings are stored. Returns the block size."""
    import json

    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    if key in cache:
        lbm_batch_set_threads(b, cache[key]["threads"])
        return int(cache[key]["threads"])
    best, times = lbm_batch_autotune(b, steps)
    cache[key] = {"threads": best, "us_per_step": {str(k): v for k, v in times.items()}, "steps": int(steps)}
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return best


def lbm_batch_results(b, ncols, check=True):
    steps = np.zeros(ncols, dtype=np.int64)
    res = np.zeros(ncols)
    status = np.zeros(ncols, dtype=np.int32)
    rc = load().lbm_batch_results(b, steps.ctypes.data, res.ctypes.data, status.ctypes.data)
    if check and rc != LBM_ENONPHYS:
        _check(rc)
    return steps, res, status


def lbm_batch_column_seconds(b, ncols):
    """Per column: device seconds the persistent launches spent on it, summed over runs."""
    sec = np.empty(ncols)
    _check(load().lbm_batch_column_seconds(b, sec.ctypes.data))
    return sec


def lbm_batch_moments(b, rho=None, ux=None, uy=None):
    wheres = {w for _, w in map(_ptr, (rho, ux, uy)) if w is not None}
    where = wheres.pop() if wheres else LBM_HOST
    _check(load().lbm_batch_moments(b, _ptr(rho)[0], _ptr(ux)[0], _ptr(uy)[0], where))


def lbm_batch_rest_state(b):
    """Every column's populations become the rest state of its stored density field."""
    _check(load().lbm_batch_rest_state(b))


def lbm_batch_get_state(b, f):
    addr, where = _ptr(f)
    _check(load().lbm_batch_get_state(b, addr, where))


def lbm_batch_convert(b, precision):
    out = ctypes.c_void_p()
    _check(load().lbm_batch_convert(b, int(precision), ctypes.byref(out)))
    return out


def lbm_batch_destroy(b):
    _check(load().lbm_batch_destroy(b))


# ---------------------------------------------------------------- convenience
def make_params(nx, ny, T, precision="fp64", **kw):
    """lbm_params from the paper's defaults plus keyword overrides (names of the C struct;
    ``form`` is accepted for ``gravity_form`` and ``g`` for (gx, gy))."""
    p = lbm_params_default()
    p.nx, p.ny, p.T = int(nx), int(ny), float(T)
    prec = str(precision).lower()
    p.precision = (LBM_FP32 if prec in ("fp32", "float32", "1")
                   else LBM_DOUBLE_FLOAT if prec in ("dd", "double_float", "2") else LBM_FP64)
    if "form" in kw:
        p.gravity_form = int(kw.pop("form"))
    if "g" in kw:
        p.gx, p.gy = map(float, kw.pop("g"))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Lattice:
    """A handle whose workspace is a torch CUDA tensor and whose stream is torch's
    current stream. Outputs of ``moments`` are torch tensors on the device."""

    def __init__(self, params, rho0, device="cuda"):
        import torch

        self._torch = torch
        self.params = params
        nbytes = lbm_workspace_bytes(params)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self._ws.data_ptr()
        params.workspace = (base + 255) // 256 * 256
        params.workspace_bytes = nbytes
        self.stream = torch.cuda.current_stream(self._ws.device).cuda_stream
        self.h = lbm_init(params, rho0, self.stream)
        self.nx, self.ny = params.nx, params.ny

    def step(self, n):
        lbm_step(self.h, n)

    def moments(self):
        t = self._torch
        rho, ux, uy = (t.empty((self.ny, self.nx), dtype=t.float64, device=self._ws.device) for _ in range(3))
        lbm_moments(self.h, rho, ux, uy)
        return rho, ux, uy

    def reduce(self, kind):
        return lbm_reduce(self.h, kind)

    def get_state(self):
        f = np.empty((9, self.ny, self.nx))
        lbm_get_state(self.h, f)
        return f

    def set_state(self, f, steps_done=0):
        lbm_set_state(self.h, np.ascontiguousarray(f, dtype=np.float64), steps_done)

    def temperature(self):
        t = self._torch
        T = t.empty((self.ny, self.nx), dtype=t.float64, device=self._ws.device)
        lbm_get_temperature(self.h, T)
        return T

    def status(self):
        return lbm_status(self.h)

    def close(self):
        if self.h is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- warm-start network
def mlp_pack(params):
    """Packed FP32 parameter array from a dict of arrays (W1 may be 128 x 5: padded to 16)."""
    out = np.zeros(MLP_NPARAMS, dtype=np.float32)
    off = 0
    for name, shape in MLP_LAYOUT:
        n = int(np.prod(shape))
        a = np.zeros(shape)
        src = np.asarray(params[name], dtype=np.float64)
        a[tuple(slice(0, k) for k in src.shape)] = src
        out[off:off + n] = a.ravel()
        off += n
    return out


def mlp_unpack(packed):
    """Dict of FP64 arrays from a packed parameter array (W1 cut to its 5 used inputs)."""
    out, off = {}, 0
    for name, shape in MLP_LAYOUT:
        n = int(np.prod(shape))
        out[name] = np.asarray(packed[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    out["W1"] = out["W1"][:, :MLP_INPUTS].copy()
    return out


def mlp_initial_params(seed):
    """Initial packed parameters: every weight uniform in +-sqrt(6/(fan_in + fan_out)) from the
    seeded draws of the input module, biases zero."""
    from . import inputs

    u = inputs.mlp_draws(seed, MLP_WIDTH, MLP_INPUTS)
    fan = {"W1": (MLP_INPUTS, MLP_WIDTH), "W2": (MLP_WIDTH, MLP_WIDTH), "W3": (MLP_WIDTH, MLP_WIDTH),
           "w4": (MLP_WIDTH, 1)}
    P = {k: (2.0 * u[k] - 1.0) * np.sqrt(6.0 / sum(fan[k])) for k in fan}
    P.update(b1=np.zeros(MLP_WIDTH), b2=np.zeros(MLP_WIDTH), b3=np.zeros(MLP_WIDTH), b4=np.zeros(1))
    return mlp_pack(P)


def _dev(t):
    if not (hasattr(t, "data_ptr") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def lbm_mlp_create(packed, batch_capacity, stream=None):
    p = np.ascontiguousarray(packed, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(load().lbm_mlp_create(p.ctypes.data, int(batch_capacity), stream, ctypes.byref(h)))
    return h


def lbm_mlp_set_params(h, packed):
    p = np.ascontiguousarray(packed, dtype=np.float32)
    _check(load().lbm_mlp_set_params(h, p.ctypes.data))


def lbm_mlp_get_params(h):
    out = np.empty(MLP_NPARAMS, dtype=np.float32)
    _check(load().lbm_mlp_get_params(h, out.ctypes.data))
    return out


def lbm_mlp_gradients(h, x, t):
    """x: CUDA float32 tensor (n, 6); t: (n,). Returns (loss, packed gradient array)."""
    g = np.empty(MLP_NPARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(load().lbm_mlp_gradients(h, _dev(x), _dev(t), int(t.numel()), g.ctypes.data, ctypes.byref(loss)))
    return loss.value, g


def lbm_mlp_train(h, x, t, batch, iters, lr, seed, record=True):
    losses = np.empty(max(1, iters), dtype=np.float32) if record else None
    _check(load().lbm_mlp_train(h, _dev(x), _dev(t), int(t.numel()), int(batch), int(iters), float(lr),
                                int(seed) & 0xFFFFFFFFFFFFFFFF, losses.ctypes.data if record else None))
    return losses[:iters] if record else None


def lbm_mlp_predict(h, x, y):
    _check(load().lbm_mlp_predict(h, _dev(x), int(x.shape[0]), _dev(y)))


def _columns_array(cols):
    arr = (lbm_column * len(cols))()
    for i, c in enumerate(cols):
        arr[i].ny = int(c["ny"])
        arr[i].gravity_form = int(c.get("form", c.get("gravity_form", 1)))
        arr[i].T = float(c["T"])
        arr[i].gx = float(c.get("gx", 0.0))
        arr[i].gy = float(c.get("gy", 0.0))
    return arr


def lbm_mlp_features(cols, nx, a, b, R, x, t=None, rho=None, mean_rho=None, stream=None):
    arr = _columns_array(cols)
    mr = None if mean_rho is None else np.ascontiguousarray(mean_rho, dtype=np.float64)
    _check(load().lbm_mlp_features(arr, len(cols), int(nx), a, b, R, None if rho is None else _dev(rho),
                                   None if mr is None else mr.ctypes.data, _dev(x),
                                   None if t is None else _dev(t), stream))


def lbm_mlp_warm_start(h, cols, nx, a, b, R, mean_rho, rho0):
    arr = _columns_array(cols)
    mr = np.ascontiguousarray(mean_rho, dtype=np.float64)
    _check(load().lbm_mlp_warm_start(h, arr, len(cols), int(nx), a, b, R, mr.ctypes.data, _dev(rho0)))


def lbm_mlp_gemm(A, B, C, k_split=0, accumulate=False, stream=None):
    """C (+)= A B^T on the tensor cores; A (M, K), B (N, K): CUDA int16/uint16 tensors holding
    bfloat16 bit patterns (or torch.bfloat16); C (M, N) CUDA float32."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().lbm_mlp_gemm(_dev(A), A.stride(0), _dev(B), B.stride(0), _dev(C), C.stride(0), M, N, K,
                               int(k_split), 1 if accumulate else 0, stream))


def lbm_mlp_gemm_enqueue(A, B, C, status, k_split=0, accumulate=False, stream=None):
    """lbm_mlp_gemm enqueued on `stream` without waiting; status: a CUDA int32 tensor of one
    element that the kernel ORs a non-zero bit into on a tensor-core wait timeout."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().lbm_mlp_gemm_enqueue(_dev(A), A.stride(0), _dev(B), B.stride(0), _dev(C), C.stride(0), M, N, K,
                                       int(k_split), 1 if accumulate else 0, _dev(status), stream))


def lbm_mlp_destroy(h):
    _check(load().lbm_mlp_destroy(h))
