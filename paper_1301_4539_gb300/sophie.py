"""ctypes binding of libsophie (include/sophie.h), argument marshalling only.

Every function has the C name and signature; a negative return code raises
SophieError carrying the code and sophie_last_error(). Arrays are numpy
arrays on the host. The library is loaded from this package directory; if it
is missing the import of a function fails loudly (there is no CPU fallback).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsophie.so")

OK, EINVAL, EUNSTABLE, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ETOOMANYMAT, ENOTSUP = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
EX, EY, EZ, HX, HY, HZ = range(6)
GAUSS_SINE, GAUSS = 0, 1
FP32, FP16, BF16, FP16HL, FP24 = 0, 1, 2, 3, 4
KERNEL_PLAIN, KERNEL_BLOCKED, KERNEL_ENERGY, KERNEL_ADJOINT = 0, 1, 2, 3

# Exported symbols with (restype, argtypes).
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong
SIGNATURES = {
    "sophie_version": (_I, []),
    "sophie_create_grid": (_I, [_I, _I, _I, _D, _D, ctypes.POINTER(_P)]),
    "sophie_destroy_grid": (_I, [_P]),
    "sophie_set_materials": (_I, [_P, _P, _P]),
    "sophie_add_source": (_I, [_P, _I, _I, _I, _I, _D, _D, _D, _D, _I]),
    "sophie_add_probe": (_I, [_P, _I, _I, _I, _I, ctypes.POINTER(_I)]),
    "sophie_step": (_I, [_P, _I]),
    "sophie_get_step": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_read_probe": (_I, [_P, _I, _P, _I, ctypes.POINTER(_I)]),
    "sophie_energy": (_I, [_P, ctypes.POINTER(_D)]),
    "sophie_energy_noalloc": (_I, [_P, _P]),
    "sophie_set_fields": (_I, [_P, _I, _P]),
    "sophie_get_fields": (_I, [_P, _I, _P]),
    "sophie_reset": (_I, [_P]),
    "sophie_set_stream": (_I, [_P, _P]),
    "sophie_sync": (_I, [_P]),
    "sophie_configure": (_I, [_P, _I, _I, _I, _I]),
    "sophie_set_storage_scale": (_I, [_P, _P]),
    "sophie_autotune": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "sophie_set_zero_skip": (_I, [_P, _I]),
    "sophie_set_spacing": (_I, [_P, _P, _P, _P]),
    "sophie_launch_count": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_launch_config": (_I, [_P, ctypes.POINTER(_I)]),
    "sophie_profile": (_I, [_P, _I]),
    "sophie_profile_read": (_I, [_P, _I, ctypes.POINTER(_LL), ctypes.POINTER(_D)]),
    "sophie_objective_forward": (_I, [_P, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_D)]),
    "sophie_objective_grad_eps": (_I, [_P, _I, _I, _I, _I, _I, _I, _P]),
    "sophie_objective_release": (_I, [_P]),
    "sophie_objective_set_design": (_I, [_P, _I, _I, _I, _I, _I, _I]),
    "sophie_batch_create": (_I, [_I, _P, _D, _D, ctypes.POINTER(_P)]),
    "sophie_batch_destroy": (_I, [_P]),
    "sophie_batch_set_materials": (_I, [_P, _P, _P]),
    "sophie_batch_add_source": (_I, [_P, _I, _I, _I, _I, _I, _D, _D, _D, _D, _I]),
    "sophie_batch_step": (_I, [_P, _I]),
    "sophie_batch_get_step": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_batch_energy": (_I, [_P, _P]),
    "sophie_batch_set_fields": (_I, [_P, _I, _I, _P]),
    "sophie_batch_get_fields": (_I, [_P, _I, _I, _P]),
    "sophie_batch_reset": (_I, [_P]),
    "sophie_batch_set_stream": (_I, [_P, _P]),
    "sophie_batch_configure": (_I, [_P, _I, _I, _I, _I]),
    "sophie_batch_autotune": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                   ctypes.POINTER(_D)]),
    "sophie_batch_info": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_I),
                               ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "sophie_batch_launch_count": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_batch_sync": (_I, [_P]),
    "sophie_batch_create_packed": (_I, [_I, _P, _D, _D, ctypes.POINTER(_P)]),
    "sophie_batch_pack_plan": (_I, [_I, _P, _P, _P]),
    "sophie_batch_layout": (_I, [_P, ctypes.POINTER(_I), _P, ctypes.POINTER(_I)]),
    "sophie_batch_cavity_origin": (_I, [_P, _I, _P]),
    "sophie_check_guards": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_batch_check_guards": (_I, [_P, ctypes.POINTER(_LL)]),
    "sophie_selftest_wait_timeout": (_I, [_P, ctypes.POINTER(_D)]),
    "sophie_debug_fail_alloc": (_I, [_I]),
    "sophie_debug_material_tables": (_I, [_I, _I, _I, _D, _D, _P, _P, _I, _P, _P, _P, _P, _P, _LL,
                                          ctypes.POINTER(_LL)]),
    "sophie_last_error": (ctypes.c_char_p, []),
}


class SophieError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsophie error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libsophie.so (building it first if absent and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        from . import build as _b
        _b.build()
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _chk(rc: int) -> int:
    if rc < 0:
        raise SophieError(rc, load().sophie_last_error().decode())
    return rc


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


# ---- the C API, one wrapper per function (same names) ----------------------
def sophie_version() -> int:
    return load().sophie_version()


def sophie_create_grid(nx: int, ny: int, nz: int, dx: float, dt: float) -> int:
    h = _P()
    _chk(load().sophie_create_grid(nx, ny, nz, dx, dt, ctypes.byref(h)))
    return h.value


def sophie_destroy_grid(g: int) -> None:
    _chk(load().sophie_destroy_grid(g))


def sophie_set_materials(g: int, eps_r: np.ndarray, sigma: np.ndarray) -> None:
    e, s = _f32(eps_r), _f32(sigma)
    _chk(load().sophie_set_materials(g, e.ctypes.data, s.ctypes.data))


def sophie_add_source(g: int, comp: int, i: int, j: int, k: int, amp: float, f0: float,
                      bw: float, t0: float, kind: int) -> None:
    _chk(load().sophie_add_source(g, comp, i, j, k, amp, f0, bw, t0, kind))


def sophie_add_probe(g: int, comp: int, i: int, j: int, k: int) -> int:
    pid = _I()
    _chk(load().sophie_add_probe(g, comp, i, j, k, ctypes.byref(pid)))
    return pid.value


def sophie_step(g: int, n: int) -> None:
    _chk(load().sophie_step(g, n))


def sophie_get_step(g: int) -> int:
    n = _LL()
    _chk(load().sophie_get_step(g, ctypes.byref(n)))
    return n.value


def sophie_read_probe(g: int, probe_id: int, cap: int) -> np.ndarray:
    out = np.zeros(max(cap, 0), np.float64)
    nw = _I()
    _chk(load().sophie_read_probe(g, probe_id, out.ctypes.data, cap, ctypes.byref(nw)))
    return out[: nw.value]


def sophie_energy(g: int) -> float:
    w = _D()
    _chk(load().sophie_energy(g, ctypes.byref(w)))
    return w.value


def sophie_energy_noalloc(g: int, W_dev: int) -> None:
    """Energy into caller-owned device memory (a double at address W_dev); no allocation."""
    _chk(load().sophie_energy_noalloc(g, W_dev))


def sophie_set_fields(g: int, comp: int, host: np.ndarray) -> None:
    a = _f32(host)
    _chk(load().sophie_set_fields(g, comp, a.ctypes.data))


def sophie_get_fields(g: int, comp: int, shape) -> np.ndarray:
    out = np.empty(shape, np.float32)
    _chk(load().sophie_get_fields(g, comp, out.ctypes.data))
    return out


def sophie_reset(g: int) -> None:
    _chk(load().sophie_reset(g))


def sophie_set_stream(g: int, cuda_stream: int) -> None:
    _chk(load().sophie_set_stream(g, cuda_stream))


def sophie_sync(g: int) -> None:
    _chk(load().sophie_sync(g))


def sophie_configure(g: int, temporal_k: int = 0, tile_x: int = 0, tile_y: int = 0,
                     precision: int = FP32) -> None:
    _chk(load().sophie_configure(g, temporal_k, tile_x, tile_y, precision))


def sophie_set_storage_scale(g: int, scale) -> None:
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    assert sc.size == 6
    _chk(load().sophie_set_storage_scale(g, sc.ctypes.data))


def sophie_autotune(g: int):
    """(chosen temporal_k, device ms per time step)."""
    k = _I()
    ms = _D()
    _chk(load().sophie_autotune(g, ctypes.byref(k), ctypes.byref(ms)))
    return k.value, ms.value


def sophie_set_zero_skip(g: int, enable: bool) -> None:
    _chk(load().sophie_set_zero_skip(g, 1 if enable else 0))


def sophie_set_spacing(g: int, wx, wy, wz) -> None:
    """Cell widths along x, y, z (metres; None = uniform dx on that axis)."""
    arrs = [None if w is None else np.ascontiguousarray(w, np.float64) for w in (wx, wy, wz)]
    ptrs = [None if a is None else a.ctypes.data for a in arrs]
    _chk(load().sophie_set_spacing(g, *ptrs))


def sophie_launch_config(g: int) -> dict:
    """The launch configuration of the next step (see include/sophie.h)."""
    out = (_I * 7)()
    _chk(load().sophie_launch_config(g, out))
    v = list(out)
    return {"k": v[0], "plain_zchunk": v[1], "plain_ctas": v[2], "blocked_ctas": v[3],
            "blocked_zsplit": v[4], "blocked_order": v[5], "blocked_rows": v[6]}


def sophie_launch_count(g: int) -> int:
    n = _LL()
    _chk(load().sophie_launch_count(g, ctypes.byref(n)))
    return n.value


def sophie_profile(g: int, enable: bool) -> None:
    _chk(load().sophie_profile(g, 1 if enable else 0))


def sophie_profile_read(g: int, kernel: int):
    n = _LL()
    ms = _D()
    _chk(load().sophie_profile_read(g, kernel, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def sophie_objective_forward(g: int, nsteps: int, comp: int, i: int, j: int, k: int,
                             checkpoint_every: int = 0) -> float:
    J = _D()
    _chk(load().sophie_objective_forward(g, nsteps, comp, i, j, k, checkpoint_every, ctypes.byref(J)))
    return J.value


def sophie_objective_grad_eps(g: int, i0: int, j0: int, k0: int, ni: int, nj: int, nk: int) -> np.ndarray:
    """dJ/d eps_r of the cell box, shape (nk, nj, ni)."""
    out = np.zeros((nk, nj, ni), np.float64)
    _chk(load().sophie_objective_grad_eps(g, i0, j0, k0, ni, nj, nk, out.ctypes.data))
    return out


def sophie_objective_set_design(g: int, i0: int = 0, j0: int = 0, k0: int = 0, ni: int = 0, nj: int = 0,
                                nk: int = 0) -> None:
    _chk(load().sophie_objective_set_design(g, i0, j0, k0, ni, nj, nk))


def sophie_objective_release(g: int) -> None:
    _chk(load().sophie_objective_release(g))


def sophie_last_error() -> str:
    return load().sophie_last_error().decode()


class Grid:
    """Owning handle: the same calls bound to one grid (marshalling only)."""

    def __init__(self, nx: int, ny: int, nz: int, dx: float, dt: float):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = sophie_create_grid(nx, ny, nz, dx, dt)

    @property
    def shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    def close(self):
        if self.h:
            sophie_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_materials(self, eps, sigma):
        sophie_set_materials(self.h, eps, sigma)

    def add_source(self, comp, i, j, k, amp, f0, bw, t0, kind):
        sophie_add_source(self.h, comp, i, j, k, amp, f0, bw, t0, kind)

    def add_probe(self, comp, i, j, k):
        return sophie_add_probe(self.h, comp, i, j, k)

    def step(self, n):
        sophie_step(self.h, n)

    @property
    def n(self):
        return sophie_get_step(self.h)

    def read_probe(self, pid, cap=None):
        return sophie_read_probe(self.h, pid, self.n if cap is None else cap)

    def energy(self):
        return sophie_energy(self.h)

    def set_field(self, comp, arr):
        sophie_set_fields(self.h, comp, arr)

    def get_field(self, comp):
        return sophie_get_fields(self.h, comp, self.shape)

    def fields(self):
        return [self.get_field(c) for c in range(6)]

    def reset(self):
        sophie_reset(self.h)

    def set_stream(self, s):
        sophie_set_stream(self.h, s)

    def sync(self):
        sophie_sync(self.h)

    def configure(self, temporal_k=0, tile_x=0, tile_y=0, precision=FP32):
        sophie_configure(self.h, temporal_k, tile_x, tile_y, precision)

    def set_storage_scale(self, scale):
        sophie_set_storage_scale(self.h, scale)

    def autotune(self):
        return sophie_autotune(self.h)

    def set_zero_skip(self, enable=True):
        sophie_set_zero_skip(self.h, enable)

    def set_spacing(self, wx=None, wy=None, wz=None):
        """Non-uniform mesh: cell widths (nx, ny, nz arrays, metres); all None = uniform."""
        for w, n in ((wx, self.nx), (wy, self.ny), (wz, self.nz)):
            if w is not None and np.shape(w) != (n,):
                raise ValueError(f"width array of shape {np.shape(w)}, expected ({n},)")
        sophie_set_spacing(self.h, wx, wy, wz)

    def launch_count(self):
        return sophie_launch_count(self.h)

    def launch_config(self):
        return sophie_launch_config(self.h)

    def profile(self, enable):
        sophie_profile(self.h, enable)

    def profile_read(self, kernel):
        return sophie_profile_read(self.h, kernel)

    def check_guards(self):
        return sophie_check_guards(self.h)

    def selftest_wait_timeout(self):
        return sophie_selftest_wait_timeout(self.h)

    def objective_forward(self, nsteps, comp, i, j, k, checkpoint_every=0):
        return sophie_objective_forward(self.h, nsteps, comp, i, j, k, checkpoint_every)

    def objective_grad_eps(self, i0, j0, k0, ni, nj, nk):
        return sophie_objective_grad_eps(self.h, i0, j0, k0, ni, nj, nk)

    def objective_set_design(self, i0=0, j0=0, k0=0, ni=0, nj=0, nk=0):
        sophie_objective_set_design(self.h, i0, j0, k0, ni, nj, nk)

    def objective_release(self):
        sophie_objective_release(self.h)


# ---- diagnostics -------------------------------------------------------------
def sophie_check_guards(g: int) -> int:
    n = _LL()
    _chk(load().sophie_check_guards(g, ctypes.byref(n)))
    return n.value


def sophie_batch_check_guards(b: int) -> int:
    n = _LL()
    _chk(load().sophie_batch_check_guards(b, ctypes.byref(n)))
    return n.value


def sophie_selftest_wait_timeout(g: int) -> float:
    ms = _D()
    _chk(load().sophie_selftest_wait_timeout(g, ctypes.byref(ms)))
    return ms.value


def sophie_debug_fail_alloc(n: int) -> None:
    _chk(load().sophie_debug_fail_alloc(n))


def sophie_debug_material_tables(eps, sig, dx: float, dt: float, nthreads: int = 1, exp_cap: int = 1 << 20):
    """Host material build without a GPU: (words, class_coef, class_eps,
    exp_coef, exp_eps) for per-cell eps_r / sigma of shape (nz, ny, nx)."""
    eps = np.ascontiguousarray(eps, np.float32)
    sig = np.ascontiguousarray(sig, np.float32)
    nz, ny, nx = eps.shape
    nxp = ((nx + 1) + 7) // 8 * 8
    words = np.zeros((nz + 1, ny + 1, nxp), np.uint32)
    ccoef = np.zeros((512, 2), np.float32)
    ceps = np.zeros(512, np.float64)
    ecoef = np.zeros((exp_cap, 3, 2), np.float32)
    eeps = np.zeros((exp_cap, 3), np.float64)
    n = _LL()
    _chk(load().sophie_debug_material_tables(nx, ny, nz, dx, dt, eps.ctypes.data, sig.ctypes.data, nthreads,
                                              words.ctypes.data, ccoef.ctypes.data, ceps.ctypes.data,
                                              ecoef.ctypes.data, eeps.ctypes.data, exp_cap, ctypes.byref(n)))
    k = min(n.value, exp_cap)
    return words, ccoef, ceps, ecoef[:k], eeps[:k]


# ---- batched cavities -------------------------------------------------------
def sophie_batch_create(dims, dx: float, dt: float) -> int:
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    h = _P()
    _chk(load().sophie_batch_create(len(d), d.ctypes.data, dx, dt, ctypes.byref(h)))
    return h.value


def sophie_batch_create_packed(dims, dx: float, dt: float) -> int:
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    h = _P()
    _chk(load().sophie_batch_create_packed(len(d), d.ctypes.data, dx, dt, ctypes.byref(h)))
    return h.value


def sophie_batch_pack_plan(dims):
    """(origins ncav x 3, extent 3) of the packed placement (host only)."""
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    org = np.zeros((len(d), 3), np.int32)
    ext = np.zeros(3, np.int32)
    _chk(load().sophie_batch_pack_plan(len(d), d.ctypes.data, org.ctypes.data, ext.ctypes.data))
    return org, ext


def sophie_batch_layout(b: int):
    packed, k = _I(), _I()
    ext = np.zeros(3, np.int32)
    _chk(load().sophie_batch_layout(b, ctypes.byref(packed), ext.ctypes.data, ctypes.byref(k)))
    return {"packed": bool(packed.value), "extent": tuple(int(v) for v in ext), "temporal_k": k.value}


def sophie_batch_cavity_origin(b: int, cav: int):
    o = np.zeros(3, np.int32)
    _chk(load().sophie_batch_cavity_origin(b, cav, o.ctypes.data))
    return tuple(int(v) for v in o)


def sophie_batch_destroy(b: int) -> None:
    _chk(load().sophie_batch_destroy(b))


def sophie_batch_set_materials(b: int, eps_r, sigma=None) -> None:
    e = None if eps_r is None else _f32(eps_r)
    s = None if sigma is None else _f32(sigma)
    _chk(load().sophie_batch_set_materials(b, None if e is None else e.ctypes.data,
                                           None if s is None else s.ctypes.data))


def sophie_batch_add_source(b: int, cav: int, comp: int, i: int, j: int, k: int, amp: float, f0: float,
                            bw: float, t0: float, kind: int) -> None:
    _chk(load().sophie_batch_add_source(b, cav, comp, i, j, k, amp, f0, bw, t0, kind))


def sophie_batch_step(b: int, n: int) -> None:
    _chk(load().sophie_batch_step(b, n))


def sophie_batch_get_step(b: int) -> int:
    n = _LL()
    _chk(load().sophie_batch_get_step(b, ctypes.byref(n)))
    return n.value


def sophie_batch_energy(b: int, ncav: int) -> np.ndarray:
    out = np.zeros(ncav, np.float64)
    _chk(load().sophie_batch_energy(b, out.ctypes.data))
    return out


def sophie_batch_set_fields(b: int, cav: int, comp: int, host: np.ndarray) -> None:
    a = _f32(host)
    _chk(load().sophie_batch_set_fields(b, cav, comp, a.ctypes.data))


def sophie_batch_get_fields(b: int, cav: int, comp: int, shape) -> np.ndarray:
    out = np.empty(shape, np.float32)
    _chk(load().sophie_batch_get_fields(b, cav, comp, out.ctypes.data))
    return out


def sophie_batch_reset(b: int) -> None:
    _chk(load().sophie_batch_reset(b))


def sophie_batch_set_stream(b: int, cuda_stream: int) -> None:
    _chk(load().sophie_batch_set_stream(b, cuda_stream))


def sophie_batch_configure(b: int, tile_x: int = 0, tile_y: int = 0, zchunk: int = 0,
                           use_graph: bool = True) -> None:
    _chk(load().sophie_batch_configure(b, tile_x, tile_y, zchunk, 1 if use_graph else 0))


def sophie_batch_autotune(b: int):
    """(tile_x, tile_y, zchunk, device ms per time step) of the fastest work split."""
    tx, ty, zc, ms = _I(), _I(), _I(), _D()
    _chk(load().sophie_batch_autotune(b, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(ms)))
    return tx.value, ty.value, zc.value, ms.value


def sophie_batch_info(b: int):
    cells, items, tx, ty, zc = _LL(), _LL(), _I(), _I(), _I()
    _chk(load().sophie_batch_info(b, ctypes.byref(cells), ctypes.byref(items), ctypes.byref(tx), ctypes.byref(ty),
                                  ctypes.byref(zc)))
    return {"cells": cells.value, "work_items": items.value, "tile_x": tx.value, "tile_y": ty.value,
            "zchunk": zc.value}


def sophie_batch_launch_count(b: int) -> int:
    n = _LL()
    _chk(load().sophie_batch_launch_count(b, ctypes.byref(n)))
    return n.value


def sophie_batch_sync(b: int) -> None:
    _chk(load().sophie_batch_sync(b))


class Batch:
    """Owning handle of a batch of cavities (marshalling only)."""

    def __init__(self, dims, dx: float, dt: float, packed: bool = False):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.h = (sophie_batch_create_packed if packed else sophie_batch_create)(self.dims, dx, dt)

    def close(self):
        if self.h:
            sophie_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, cav):
        nx, ny, nz = self.dims[cav]
        return (nz + 1, ny + 1, nx + 1)

    def set_materials(self, eps=None, sigma=None):
        sophie_batch_set_materials(self.h, eps, sigma)

    def add_source(self, cav, comp, i, j, k, amp, f0, bw, t0, kind):
        sophie_batch_add_source(self.h, cav, comp, i, j, k, amp, f0, bw, t0, kind)

    def step(self, n):
        sophie_batch_step(self.h, n)

    @property
    def n(self):
        return sophie_batch_get_step(self.h)

    def energy(self):
        return sophie_batch_energy(self.h, len(self.dims))

    def set_field(self, cav, comp, arr):
        sophie_batch_set_fields(self.h, cav, comp, arr)

    def get_field(self, cav, comp):
        return sophie_batch_get_fields(self.h, cav, comp, self.shape(cav))

    def fields(self, cav):
        return [self.get_field(cav, c) for c in range(6)]

    def reset(self):
        sophie_batch_reset(self.h)

    def set_stream(self, s):
        sophie_batch_set_stream(self.h, s)

    def configure(self, tile_x=0, tile_y=0, zchunk=0, use_graph=True):
        sophie_batch_configure(self.h, tile_x, tile_y, zchunk, use_graph)

    def autotune(self):
        return sophie_batch_autotune(self.h)

    def info(self):
        return sophie_batch_info(self.h)

    def launch_count(self):
        return sophie_batch_launch_count(self.h)

    def check_guards(self):
        return sophie_batch_check_guards(self.h)

    def sync(self):
        sophie_batch_sync(self.h)

    def layout(self):
        return sophie_batch_layout(self.h)

    def origin(self, cav):
        return sophie_batch_cavity_origin(self.h, cav)
