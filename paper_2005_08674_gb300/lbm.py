"""Thin ctypes binding of the C ABI declared in include/lbm.h.

Functions keep the C names and only marshal arguments; every step of the
simulation runs in the CUDA library.  PyTorch supplies device memory
(``Simulation`` binds torch-allocated buffers) and the CUDA stream.  There is
no CPU fallback: if ``liblbm.so`` is missing or fails to load, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_CHECKED=1 loads the bounds-checked build (build(check=True)) instead
CHECKED = os.environ.get("LBM_CHECKED") == "1"
LIB_PATH = os.path.join(_HERE, "liblbm_check.so" if CHECKED else "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2, 3
LBM_BGK, LBM_MRT = 0, 1
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_2005_08674_gb300.build.build() "
                      "(nvcc, sm_103a) first")

_L = ctypes.CDLL(LIB_PATH)
_vp, _dp, _i32, _dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double
_i32p = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "lbm_create": (_vp, [_i32, _i32, _dbl, _dbl, _dp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_set_nsbc": (ctypes.c_int, [_vp, _dbl, _dbl, _dbl, _i32, _i32]),
    "lbm_set_precision": (ctypes.c_int, [_vp, _i32]),
    "lbm_set_collision": (ctypes.c_int, [_vp, _i32, _dbl, _dbl, _dbl]),
    "lbm_set_edges": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_batch_set_edges": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbm_get_dims": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "lbm_buffer_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_scratch_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_bind": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_init": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_init_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_step": (ctypes.c_int, [_vp, _i32]),
    "lbm_steps_done": (ctypes.c_int64, [_vp]),
    "lbm_get_macros": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_get_macros_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_get_populations": (ctypes.c_int, [_vp, _vp]),
    "lbm_set_populations": (ctypes.c_int, [_vp, _vp]),
    "lbm_reduce": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _dp]),
    "lbm_save_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_load_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "lbm_state_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_set_launch": (ctypes.c_int, [_vp, _i32, _i32, _i32]),
    "lbm_autotune": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _dp]),
    "lbm_set_staged": (ctypes.c_int, [_vp, _i32]),
    "lbm_get_staged": (ctypes.c_int32, [_vp]),
    "lbm_set_fused": (ctypes.c_int, [_vp, _i32]),
    "lbm_get_fused": (ctypes.c_int32, [_vp]),
    "lbm_set_twostep": (ctypes.c_int, [_vp, _i32]),
    "lbm_get_twostep": (ctypes.c_int32, [_vp]),
    "lbm_status": (ctypes.c_int, [_vp]),
    "lbm_reduce_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _dp]),
    "lbm_set_tune_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "lbm_tune_cache_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_profile": (ctypes.c_int, [_vp, _i32]),
    "lbm_profile_read": (ctypes.c_int, [_vp, _dp]),
    "lbm_batch_create": (_vp, [_i32, _vp, _i32]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm_batch_set_nsbc": (ctypes.c_int, [_vp, _dbl, _dbl, _dbl, _i32, _i32]),
    "lbm_batch_set_collision": (ctypes.c_int, [_vp, _i32, _dbl, _dbl, _dbl]),
    "lbm_batch_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbm_batch_cells": (ctypes.c_int64, [_vp]),
    "lbm_batch_get_dims": (ctypes.c_int, [_vp, _i32, _i32p, _i32p]),
    "lbm_batch_buffer_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_batch_scratch_bytes": (ctypes.c_size_t, [_vp]),
    "lbm_batch_bind": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_batch_init": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "lbm_batch_step": (ctypes.c_int, [_vp, _i32]),
    "lbm_batch_steps_done": (ctypes.c_int64, [_vp]),
    "lbm_batch_get_macros": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "lbm_batch_unstable_nodes": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_batch_set_launch": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, _i32, _i32]),
    "lbm_batch_autotune": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _dp]),
    "lbm_batch_set_twostep": (ctypes.c_int, [_vp, _i32]),
    "lbm_batch_get_twostep": (ctypes.c_int32, [_vp]),
    "lbm_batch_status": (ctypes.c_int, [_vp]),
    "lbm_wait_selftest": (ctypes.c_int, [ctypes.c_int64]),
    "lbm_partition_instances": (ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_int64), _i32, _i32p]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_check_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64), _i32]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_L, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def lbm_last_error() -> str:
    return _L.lbm_last_error().decode()


def _check(rc: int) -> int:
    if rc != LBM_OK:
        raise LbmError(rc, lbm_last_error())
    return rc


def lbm_check_read(reset: bool = False):
    """(checked build?, rejected accesses, first rejected address) -- see lbm.h."""
    n, a = ctypes.c_int64(0), ctypes.c_uint64(0)
    rc = _L.lbm_check_read(ctypes.byref(n), ctypes.byref(a), int(reset))
    if rc < 0:
        raise LbmError(rc, lbm_last_error())
    return bool(rc), int(n.value), int(a.value)


def _host_in(a, shape, what: str) -> np.ndarray:
    """A C-contiguous float64 view (or copy) of an input field of `shape`."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != tuple(shape):
        raise LbmError(LBM_EINVAL, f"{what}: array of shape {a.shape}, expected {tuple(shape)}")
    return a


def _host_out(a, shape, what: str) -> np.ndarray:
    """An output array the library writes into: float64, C-contiguous,
    writeable and of `shape` (no copy is made, so nothing else will do)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable
            and a.shape == tuple(shape)):
        got = (a.shape, a.dtype) if isinstance(a, np.ndarray) else type(a).__name__
        raise LbmError(LBM_EINVAL, f"{what}: needs a writeable C-contiguous float64 array of shape "
                                   f"{tuple(shape)}, got {got}")
    return a


def _hp(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --- same-name wrappers ------------------------------------------------------

def lbm_create(nx, ny, tau, farfield_rho=1.0, farfield_u=(0.0, 0.0)):
    u = (ctypes.c_double * 2)(*farfield_u)
    h = _L.lbm_create(int(nx), int(ny), float(tau), float(farfield_rho), u)
    if not h:
        raise LbmError(LBM_EINVAL, lbm_last_error())
    return ctypes.c_void_p(h)


def lbm_destroy(h):
    _L.lbm_destroy(h)


def lbm_set_nsbc(h, gamma=0.6, beta=0.0, kappa=3.0, corner_mode=0, grad_order=1):
    return _check(_L.lbm_set_nsbc(h, gamma, beta, kappa, corner_mode, grad_order))


def lbm_set_precision(h, storage):
    return _check(_L.lbm_set_precision(h, STORAGE.get(storage, storage)))


def lbm_set_collision(h, model, omega_e=1.0, omega_eps=1.0, omega_q=1.0):
    m = {"bgk": LBM_BGK, "mrt": LBM_MRT}.get(model, model)
    return _check(_L.lbm_set_collision(h, m, omega_e, omega_eps, omega_q))


LBM_EDGE_NSBC, LBM_EDGE_PERIODIC, LBM_EDGE_VELOCITY = 0, 1, 2
_EDGE = {"nsbc": LBM_EDGE_NSBC, "periodic": LBM_EDGE_PERIODIC, "velocity": LBM_EDGE_VELOCITY}


def _edge_args(edges):
    """edges: 4 entries (left, right, bottom, top), each 'nsbc', 'periodic' or
    ('velocity', ux, uy)."""
    types = (ctypes.c_int32 * 4)()
    uw = (ctypes.c_double * 8)()
    for s, e in enumerate(edges):
        if isinstance(e, (tuple, list)):
            types[s] = _EDGE[e[0]]
            uw[2 * s], uw[2 * s + 1] = float(e[1]), float(e[2])
        else:
            types[s] = _EDGE[e]
    return ctypes.cast(types, ctypes.c_void_p), ctypes.cast(uw, ctypes.c_void_p), (types, uw)


def lbm_set_edges(h, edges):
    t, u, _keep = _edge_args(edges)
    return _check(_L.lbm_set_edges(h, t, u))


def lbm_batch_set_edges(b, edges):
    t, u, _keep = _edge_args(edges)
    return _check(_L.lbm_batch_set_edges(b, t, u))


def lbm_set_stream(h, stream_handle: int):
    return _check(_L.lbm_set_stream(h, ctypes.c_void_p(stream_handle)))


def lbm_buffer_bytes(h) -> int:
    return int(_L.lbm_buffer_bytes(h))


def lbm_scratch_bytes(h) -> int:
    return int(_L.lbm_scratch_bytes(h))


def lbm_bind(h, dev_a: int, dev_b: int, dev_scratch: int):
    return _check(_L.lbm_bind(h, ctypes.c_void_p(dev_a), ctypes.c_void_p(dev_b), ctypes.c_void_p(dev_scratch)))


def lbm_get_dims(h):
    """(nx, ny) of the domain."""
    nx, ny = ctypes.c_int32(), ctypes.c_int32()
    _check(_L.lbm_get_dims(h, ctypes.byref(nx), ctypes.byref(ny)))
    return nx.value, ny.value


def _shape(h):
    nx, ny = lbm_get_dims(h)
    return ny, nx


def lbm_init(h, rho, ux, uy):
    """Host fields [ny][nx] (numpy float64)."""
    shape = _shape(h)
    rho, ux, uy = (_host_in(a, shape, "lbm_init") for a in (rho, ux, uy))
    return _check(_L.lbm_init(h, _hp(rho), _hp(ux), _hp(uy)))


def lbm_init_device(h, d_rho: int, d_ux: int, d_uy: int):
    return _check(_L.lbm_init_device(h, ctypes.c_void_p(d_rho), ctypes.c_void_p(d_ux), ctypes.c_void_p(d_uy)))


def lbm_step(h, n: int):
    return _check(_L.lbm_step(h, int(n)))


def lbm_steps_done(h) -> int:
    return int(_L.lbm_steps_done(h))


def lbm_get_macros(h, rho: np.ndarray, ux: np.ndarray, uy: np.ndarray):
    shape = _shape(h)
    rho, ux, uy = (_host_out(a, shape, "lbm_get_macros") for a in (rho, ux, uy))
    return _check(_L.lbm_get_macros(h, _hp(rho), _hp(ux), _hp(uy)))


def lbm_get_macros_device(h, d_rho: int, d_ux: int, d_uy: int):
    return _check(_L.lbm_get_macros_device(h, ctypes.c_void_p(d_rho), ctypes.c_void_p(d_ux),
                                           ctypes.c_void_p(d_uy)))


def lbm_get_populations(h, f: np.ndarray):
    f = _host_out(f, (9,) + _shape(h), "lbm_get_populations")
    return _check(_L.lbm_get_populations(h, _hp(f)))


def lbm_set_populations(h, f):
    f = _host_in(f, (9,) + _shape(h), "lbm_set_populations")
    return _check(_L.lbm_set_populations(h, _hp(f)))


def lbm_reduce(h, ref_rho: int = 0, ref_ux: int = 0, ref_uy: int = 0, ref_pitch: int = 0,
               allow_unstable: bool = False):
    out = (ctypes.c_double * 4)()
    rc = _L.lbm_reduce(h, ctypes.c_void_p(ref_rho or None), ctypes.c_void_p(ref_ux or None),
                       ctypes.c_void_p(ref_uy or None), int(ref_pitch), out)
    if rc == LBM_EUNSTABLE and allow_unstable:
        return list(out)
    _check(rc)
    return list(out)


def lbm_state_bytes(h) -> int:
    return int(_L.lbm_state_bytes(h))


def lbm_save_state(h):
    """(checkpoint record as a numpy uint8 array, step count)."""
    buf = np.empty(lbm_state_bytes(h), dtype=np.uint8)
    steps = ctypes.c_int64()
    _check(_L.lbm_save_state(h, _hp(buf), buf.nbytes, ctypes.byref(steps)))
    return buf, steps.value


def lbm_load_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    return _check(_L.lbm_load_state(h, _hp(buf), buf.nbytes))


def lbm_reduce_noalloc(h, ref_rho: int = 0, ref_ux: int = 0, ref_uy: int = 0, ref_pitch: int = 0,
                       allow_unstable: bool = False):
    """lbm_reduce without any device allocation: for callers that cannot
    allocate device memory at that point (e.g. a hook inside another
    framework's step loop that owns the device memory).  Its partial sums use
    a fixed array inside the library, shared by every call on the device, so
    calls that overlap on the GPU race; at most 8192^2 nodes."""
    out = (ctypes.c_double * 4)()
    rc = _L.lbm_reduce_noalloc(h, ctypes.c_void_p(ref_rho or None), ctypes.c_void_p(ref_ux or None),
                               ctypes.c_void_p(ref_uy or None), int(ref_pitch), out)
    if rc == LBM_EUNSTABLE and allow_unstable:
        return list(out)
    _check(rc)
    return list(out)


def lbm_set_tune_cache(path):
    """Autotuner cache file (None turns it off); see lbm.h."""
    return _check(_L.lbm_set_tune_cache(None if path is None else os.fsencode(path)))


def lbm_tune_cache_stats():
    """(hits, misses) of the autotuner cache since the process started."""
    hits, misses = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_L.lbm_tune_cache_stats(ctypes.byref(hits), ctypes.byref(misses)))
    return hits.value, misses.value


def lbm_set_launch(h, threads_x: int, rows: int, prefetch_rows: int = 0):
    return _check(_L.lbm_set_launch(h, threads_x, rows, prefetch_rows))


def lbm_autotune(h):
    """(threads_x, rows, prefetch_rows, ms_per_step) of the fastest bulk launch."""
    bx, rows, pf, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(_L.lbm_autotune(h, ctypes.byref(bx), ctypes.byref(rows), ctypes.byref(pf), ctypes.byref(ms)))
    return bx.value, rows.value, pf.value, ms.value


def lbm_set_staged(h, stages: int):
    return _check(_L.lbm_set_staged(h, int(stages)))


def lbm_get_staged(h) -> int:
    return int(_L.lbm_get_staged(h))


def lbm_set_fused(h, enable: bool):
    return _check(_L.lbm_set_fused(h, int(bool(enable))))


def lbm_get_fused(h) -> int:
    return int(_L.lbm_get_fused(h))


def lbm_set_twostep(h, enable: bool):
    return _check(_L.lbm_set_twostep(h, int(bool(enable))))


def lbm_get_twostep(h) -> int:
    return int(_L.lbm_get_twostep(h))


def lbm_status(h):
    return _check(_L.lbm_status(h))


def lbm_profile(h, enable: bool):
    return _check(_L.lbm_profile(h, int(bool(enable))))


def lbm_profile_read(h):
    """(bulk_ms_total, bulk_launches, nsbc_ms_total, nsbc_launches)."""
    out = (ctypes.c_double * 4)()
    _check(_L.lbm_profile_read(h, out))
    return out[0], int(out[1]), out[2], int(out[3])


# --- convenience object over torch-owned memory --------------------------------

class Simulation:
    """One domain on the current CUDA device; torch allocates its memory."""

    def __init__(self, nx, ny, tau, farfield_rho=1.0, farfield_u=(0.0, 0.0), storage="f32",
                 gamma=0.6, beta=0.0, kappa=3.0, grad_order=1, stream=None, collision="bgk",
                 mrt_rates=(1.0, 1.0, 1.0), edges=None, corner_mode=0):
        import torch
        self.nx, self.ny, self.tau = nx, ny, tau
        self.storage = storage
        self.h = lbm_create(nx, ny, tau, farfield_rho, farfield_u)
        try:
            lbm_set_precision(self.h, storage)
            lbm_set_nsbc(self.h, gamma, beta, kappa, corner_mode, grad_order)
            lbm_set_collision(self.h, collision, *mrt_rates)
            if edges is not None:
                lbm_set_edges(self.h, edges)
            dev = torch.device("cuda", torch.cuda.current_device())
            self.stream = stream or torch.cuda.current_stream(dev)
            lbm_set_stream(self.h, self.stream.cuda_stream)
            bb, sb = lbm_buffer_bytes(self.h), lbm_scratch_bytes(self.h)
            self._a = torch.empty(bb, dtype=torch.uint8, device=dev)
            self._b = torch.empty(bb, dtype=torch.uint8, device=dev)
            self._s = torch.empty(sb, dtype=torch.uint8, device=dev)
            lbm_bind(self.h, self._a.data_ptr(), self._b.data_ptr(), self._s.data_ptr())
        except Exception:
            lbm_destroy(self.h)
            self.h = None
            raise

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_nsbc(self, gamma=0.6, beta=0.0, kappa=3.0, grad_order=1, corner_mode=0):
        lbm_set_nsbc(self.h, gamma, beta, kappa, corner_mode, grad_order)
        return self

    def init(self, rho, ux, uy):
        lbm_init(self.h, rho, ux, uy)
        return self

    def _device_dense(self, t, shape, what):
        """t must be a contiguous float64 tensor of `shape` on this domain's device."""
        import torch
        if not (isinstance(t, torch.Tensor) and t.device == self._a.device and t.dtype == torch.float64
                and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
            got = (tuple(t.shape), t.dtype, str(t.device)) if isinstance(t, torch.Tensor) else type(t).__name__
            raise LbmError(LBM_EINVAL, f"{what}: needs a contiguous float64 tensor of shape {tuple(shape)} "
                                       f"on {self._a.device}, got {got}")
        return t

    def init_device(self, rho, ux, uy):
        """torch float64 CUDA tensors [ny][nx]."""
        for t in (rho, ux, uy):
            self._device_dense(t, (self.ny, self.nx), "init_device")
        lbm_init_device(self.h, rho.data_ptr(), ux.data_ptr(), uy.data_ptr())
        return self

    def step(self, n=1):
        lbm_step(self.h, n)
        return self

    @property
    def steps(self):
        return lbm_steps_done(self.h)

    def macros(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        lbm_get_macros(self.h, rho, ux, uy)
        return rho, ux, uy

    def macros_device(self, out=None):
        import torch
        if out is None:
            out = torch.empty((3, self.ny, self.nx), dtype=torch.float64, device=self._a.device)
        self._device_dense(out, (3, self.ny, self.nx), "macros_device")
        lbm_get_macros_device(self.h, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        lbm_get_populations(self.h, f)
        return f

    def set_populations(self, f):
        lbm_set_populations(self.h, f)
        return self

    def reduce(self, ref=None, ref_pitch=None, allow_unstable=False):
        """ref: None or a float64 CUDA tensor [3, H, W] whose [:, 0, 0] lines up with node (0, 0)."""
        if ref is None:
            return lbm_reduce(self.h, allow_unstable=allow_unstable)
        import torch
        if not (isinstance(ref, torch.Tensor) and ref.device == self._a.device and ref.dtype == torch.float64
                and ref.dim() == 3 and ref.shape[0] >= 3 and ref.stride(-1) == 1):
            raise LbmError(LBM_EINVAL, "reduce: ref must be a float64 tensor [3, H, W] with unit stride along W "
                                       f"on {self._a.device}")
        if ref_pitch is None and (ref.shape[1] < self.ny or ref.shape[2] < self.nx):
            raise LbmError(LBM_EINVAL, f"reduce: ref of shape {tuple(ref.shape)} does not cover the "
                                       f"{self.ny} x {self.nx} domain")
        pitch = ref_pitch or ref.stride(-2)
        span = (self.ny - 1) * pitch + self.nx  # elements read from the start of each ref plane
        for c in range(3):
            avail = ref[c].untyped_storage().nbytes() // 8 - ref[c].storage_offset()
            if pitch < self.nx or avail < span:
                raise LbmError(LBM_EINVAL, f"reduce: ref plane {c} holds {avail} elements from its start, "
                                           f"{self.ny} rows of pitch {pitch} need {span} (pitch >= {self.nx})")
        return lbm_reduce(self.h, ref[0].data_ptr(), ref[1].data_ptr(), ref[2].data_ptr(), pitch,
                          allow_unstable=allow_unstable)

    def autotune(self):
        return lbm_autotune(self.h)

    def set_launch(self, threads_x, rows, prefetch_rows=0):
        lbm_set_launch(self.h, threads_x, rows, prefetch_rows)
        return self

    def set_staged(self, stages=3):
        """The staged producer/consumer step kernel (3 or 4 stages; 0 = bulk + NSBC kernel pair)."""
        lbm_set_staged(self.h, stages)
        return self

    @property
    def staged(self) -> int:
        return lbm_get_staged(self.h)

    def set_fused(self, enable=True):
        """Bulk grid of the current shape and NSBC quads in one launch per step."""
        lbm_set_fused(self.h, enable)
        return self

    @property
    def fused(self) -> bool:
        return lbm_get_fused(self.h) == 1

    def set_twostep(self, enable=True):
        """Two steps per launch, the step in between kept on chip (see lbm_set_twostep)."""
        lbm_set_twostep(self.h, enable)
        return self

    @property
    def twostep(self) -> bool:
        return lbm_get_twostep(self.h) == 1

    def status(self):
        """Raises LbmError(LBM_ETIMEOUT) if a bounded device-side wait gave up."""
        lbm_status(self.h)
        return self


# --- batched mode -----------------------------------------------------------------

class InstanceDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("farfield_rho", ctypes.c_double), ("farfield_ux", ctypes.c_double),
                ("farfield_uy", ctypes.c_double)]


def lbm_batch_create(descs, storage="f32"):
    """descs: iterable of (nx, ny, tau, farfield_rho, farfield_ux, farfield_uy)."""
    arr = (InstanceDesc * len(descs))(*[InstanceDesc(*d) for d in descs])
    b = _L.lbm_batch_create(len(descs), ctypes.cast(arr, ctypes.c_void_p), STORAGE.get(storage, storage))
    if not b:
        raise LbmError(LBM_EINVAL, lbm_last_error())
    return ctypes.c_void_p(b)


def lbm_batch_destroy(b):
    _L.lbm_batch_destroy(b)


def lbm_batch_set_nsbc(b, gamma=0.6, beta=0.0, kappa=3.0, corner_mode=0, grad_order=1):
    return _check(_L.lbm_batch_set_nsbc(b, gamma, beta, kappa, corner_mode, grad_order))


def lbm_batch_set_collision(b, model, omega_e=1.0, omega_eps=1.0, omega_q=1.0):
    m = {"bgk": LBM_BGK, "mrt": LBM_MRT}.get(model, model)
    return _check(_L.lbm_batch_set_collision(b, m, omega_e, omega_eps, omega_q))


def lbm_batch_set_stream(b, stream_handle: int):
    return _check(_L.lbm_batch_set_stream(b, ctypes.c_void_p(stream_handle)))


def lbm_batch_cells(b) -> int:
    return int(_L.lbm_batch_cells(b))


def lbm_batch_buffer_bytes(b) -> int:
    return int(_L.lbm_batch_buffer_bytes(b))


def lbm_batch_scratch_bytes(b) -> int:
    return int(_L.lbm_batch_scratch_bytes(b))


def lbm_batch_bind(b, dev_a: int, dev_b: int, dev_scratch: int):
    return _check(_L.lbm_batch_bind(b, ctypes.c_void_p(dev_a), ctypes.c_void_p(dev_b), ctypes.c_void_p(dev_scratch)))


def lbm_batch_get_dims(b, k):
    """(nx, ny) of instance k."""
    nx, ny = ctypes.c_int32(), ctypes.c_int32()
    _check(_L.lbm_batch_get_dims(b, int(k), ctypes.byref(nx), ctypes.byref(ny)))
    return nx.value, ny.value


def lbm_batch_init(b, k, rho, ux, uy):
    nx, ny = lbm_batch_get_dims(b, k)
    rho, ux, uy = (_host_in(a, (ny, nx), "lbm_batch_init") for a in (rho, ux, uy))
    return _check(_L.lbm_batch_init(b, int(k), _hp(rho), _hp(ux), _hp(uy)))


def lbm_batch_step(b, n: int):
    return _check(_L.lbm_batch_step(b, int(n)))


def lbm_batch_steps_done(b) -> int:
    return int(_L.lbm_batch_steps_done(b))


def lbm_batch_get_macros(b, k, rho, ux, uy):
    nx, ny = lbm_batch_get_dims(b, k)
    rho, ux, uy = (_host_out(a, (ny, nx), "lbm_batch_get_macros") for a in (rho, ux, uy))
    return _check(_L.lbm_batch_get_macros(b, int(k), _hp(rho), _hp(ux), _hp(uy)))


def lbm_batch_unstable_nodes(b, k) -> int:
    c = ctypes.c_int64()
    _check(_L.lbm_batch_unstable_nodes(b, int(k), ctypes.byref(c)))
    return c.value


def lbm_batch_set_launch(b, threads_x: int, rows: int, blocks: int = -1, prefetch_rows: int = 0,
                         split: int = 0, tma_tile: int = 0):
    return _check(_L.lbm_batch_set_launch(b, threads_x, rows, blocks, prefetch_rows, split, tma_tile))


def lbm_batch_autotune(b):
    """(threads_x, rows, blocks, prefetch_rows, split, tma_tile, ms_per_step) of the fastest batched launch."""
    v = [ctypes.c_int32() for _ in range(6)]
    ms = ctypes.c_double()
    _check(_L.lbm_batch_autotune(b, *[ctypes.byref(x) for x in v], ctypes.byref(ms)))
    return tuple(x.value for x in v) + (ms.value,)


def lbm_batch_status(b):
    return _check(_L.lbm_batch_status(b))


def lbm_batch_set_twostep(b, enable: bool):
    return _check(_L.lbm_batch_set_twostep(b, int(bool(enable))))


def lbm_batch_get_twostep(b) -> int:
    return int(_L.lbm_batch_get_twostep(b))


def lbm_partition_instances(cells, ranks: int):
    """Rank of each instance for a node-balanced split over `ranks` (see lbm.h)."""
    n = len(cells)
    c = (ctypes.c_int64 * max(n, 1))(*[int(v) for v in cells])
    out = (ctypes.c_int32 * max(n, 1))()
    _check(_L.lbm_partition_instances(n, c, int(ranks), out))
    return [int(out[k]) for k in range(n)]


def lbm_wait_selftest(budget_cycles: int) -> int:
    """Status code of the bounded-wait check (LBM_ETIMEOUT expected)."""
    return int(_L.lbm_wait_selftest(int(budget_cycles)))


class Batch:
    """Independent instances stepped by one launch per step; torch allocates the pools."""

    def __init__(self, workloads, storage="f32", collision="bgk", mrt_rates=(1.0, 1.0, 1.0),
                 gamma=0.6, beta=0.0, kappa=3.0, grad_order=1, stream=None, edges=None, corner_mode=0):
        import torch
        self.shapes = [(w.nx, w.ny) for w in workloads]
        descs = [(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u[0], w.farfield_u[1]) for w in workloads]
        self.b = lbm_batch_create(descs, storage)
        try:
            lbm_batch_set_nsbc(self.b, gamma, beta, kappa, corner_mode, grad_order)
            lbm_batch_set_collision(self.b, collision, *mrt_rates)
            if edges is not None:
                lbm_batch_set_edges(self.b, edges)
            dev = torch.device("cuda", torch.cuda.current_device())
            self.stream = stream or torch.cuda.current_stream(dev)
            lbm_batch_set_stream(self.b, self.stream.cuda_stream)
            pb, sb = lbm_batch_buffer_bytes(self.b), lbm_batch_scratch_bytes(self.b)
            self._a = torch.empty(pb, dtype=torch.uint8, device=dev)
            self._b = torch.empty(pb, dtype=torch.uint8, device=dev)
            self._s = torch.empty(sb, dtype=torch.uint8, device=dev)
            lbm_batch_bind(self.b, self._a.data_ptr(), self._b.data_ptr(), self._s.data_ptr())
        except Exception:
            lbm_batch_destroy(self.b)
            self.b = None
            raise

    @property
    def cells(self):
        return lbm_batch_cells(self.b)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, k, rho, ux, uy):
        lbm_batch_init(self.b, k, rho, ux, uy)
        return self

    def step(self, n=1):
        lbm_batch_step(self.b, n)
        return self

    def macros(self, k):
        nx, ny = self.shapes[k]
        rho = np.empty((ny, nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        lbm_batch_get_macros(self.b, k, rho, ux, uy)
        return rho, ux, uy

    def unstable_nodes(self, k):
        return lbm_batch_unstable_nodes(self.b, k)

    def autotune(self):
        return lbm_batch_autotune(self.b)

    def set_launch(self, threads_x, rows, blocks=-1, prefetch_rows=0, split=0, tma_tile=0):
        lbm_batch_set_launch(self.b, threads_x, rows, blocks, prefetch_rows, split, tma_tile)
        return self

    def status(self):
        return lbm_batch_status(self.b)

    def set_twostep(self, enable=True):
        """Two steps per pass for every instance (see lbm_batch_set_twostep)."""
        lbm_batch_set_twostep(self.b, enable)
        return self

    @property
    def twostep(self) -> bool:
        return lbm_batch_get_twostep(self.b) == 1
