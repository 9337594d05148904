"""ctypes front end of the C oracle (``yee_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring). Each call follows the
paper's Sec. 2.1 scheme; the C file documents every step and its citation.

Arrays are numpy arrays of shape (nz+1, ny+1, nx+1) (x fastest) per component,
in the component order ex, ey, ez, hx, hy, hz.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

C0 = 299792458.0
EPS0 = 8.8541878128e-12

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "yee_oracle.c")
_GRAD = os.path.join(_HERE, "yee_oracle_grad.c")
_BODY = os.path.join(_HERE, "yee_oracle_body.h")
_LIB = os.path.join(_HERE, "_build", "libyee_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(p) for p in (_SRC, _GRAD, _BODY, __file__))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, _GRAD, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            D = ctypes.c_double
            F = ctypes.c_float
            for suf, R in (("f64", D), ("f32", F)):
                getattr(lib, f"oracle_coefs_{suf}").argtypes = [I, I, I, D, D, P, P] + [P] * 6 + [P] * 3
                getattr(lib, f"oracle_coefs_{suf}").restype = None
                getattr(lib, f"oracle_step_{suf}").argtypes = (
                    [I, I, I, R] + [P] * 6 + [P] * 6 + [I, P, P, L, I, P, P, L, I])
                getattr(lib, f"oracle_step_{suf}").restype = None
                getattr(lib, f"oracle_energy_{suf}").argtypes = [I, I, I, R, D] + [P] * 6 + [P] * 3
                getattr(lib, f"oracle_energy_{suf}").restype = D
            for suf, R in (("f64", D), ("f32", F)):
                getattr(lib, f"oracle_step_nu_{suf}").argtypes = (
                    [I, I, I, R] + [P] * 6 + [P] * 6 + [P] * 6 + [I, P, P, L, I, P, P, L, I])
                getattr(lib, f"oracle_step_nu_{suf}").restype = None
                getattr(lib, f"oracle_energy_nu_{suf}").argtypes = [I, I, I, R, D] + [P] * 6 + [P] * 3 + [P] * 6
                getattr(lib, f"oracle_energy_nu_{suf}").restype = D
            lib.oracle_grad_f64.argtypes = [I, I, I, D, D, P, P] + [P] * 6 + [I, P, P, I, I, I, I, I, I, P, P]
            lib.oracle_grad_f64.restype = D
            lib.oracle_waveform.argtypes = [I, D, D, D, D, D, L, L, P]
            lib.oracle_waveform.restype = None
            lib.oracle_round24_f32.argtypes = [P, L]
            lib.oracle_round24_f32.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def cfl_dt(dx: float, frac: float = 0.99) -> float:
    """dt = frac * dx / (c sqrt(3)): a fraction of the 3-D Courant limit."""
    return frac * dx / (C0 * math.sqrt(3.0))


def waveform(kind: int, amp: float, f0: float, bw: float, t0: float, dt: float,
             n0: int, n: int) -> np.ndarray:
    """amp * w((n0 + m + 1/2) dt) for m in [0, n), in float64."""
    out = np.empty(n, np.float64)
    load().oracle_waveform(int(kind), amp, f0, bw, t0, dt, int(n0), int(n), _ptr(out))
    return out


def round24(a: np.ndarray) -> np.ndarray:
    """The 24-bit storage form of a float32 array (yee_oracle.c,
    oracle_round24_f32): each value rounded to 16 significant bits by
    Veltkamp's splitting, then the low 8 bits of its pattern dropped."""
    out = np.ascontiguousarray(a, np.float32).copy()
    load().oracle_round24_f32(_ptr(out), out.size)
    return out


class OracleGrid:
    """State of one cavity advanced by the oracle.

    precision: "f64" or "f32". Materials are per-cell float32 arrays of shape
    (nz, ny, nx); the oracle turns them into per-edge coefficients (Ca, Cb).
    """

    COMPS = ("ex", "ey", "ez", "hx", "hy", "hz")

    def __init__(self, nx: int, ny: int, nz: int, dx: float, dt: float,
                 precision: str = "f64"):
        assert precision in ("f64", "f32")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dt = float(dx), float(dt)
        self.precision = precision
        self.dtype = np.float64 if precision == "f64" else np.float32
        self.S = self.dtype(C0 * dt / dx)
        shp = (nz + 1, ny + 1, nx + 1)
        self.f = [np.zeros(shp, self.dtype) for _ in range(6)]
        self.n = 0
        self.sources = []  # (comp, i, j, k, amp, f0, bw, t0, kind)
        self.probes = []   # (comp, i, j, k)
        self.probe_trace = []
        self.ratios = None  # non-uniform mesh: (rx, ry, rz, rxd, ryd, rzd)
        self.set_materials(np.ones((nz, ny, nx), np.float32), np.zeros((nz, ny, nx), np.float32))

    # -- inputs ---------------------------------------------------------------
    def set_materials(self, eps_cell: np.ndarray, sig_cell: np.ndarray) -> None:
        nx, ny, nz = self.nx, self.ny, self.nz
        eps_cell = np.ascontiguousarray(eps_cell, np.float32).reshape(nz, ny, nx)
        sig_cell = np.ascontiguousarray(sig_cell, np.float32).reshape(nz, ny, nx)
        shp = (nz + 1, ny + 1, nx + 1)
        self.eps_cell, self.sig_cell = eps_cell.copy(), sig_cell.copy()
        self.coef = [np.zeros(shp, self.dtype) for _ in range(6)]  # cax cbx cay cby caz cbz
        self.eps_edge = [np.zeros(shp, np.float64) for _ in range(3)]
        fn = getattr(load(), f"oracle_coefs_{self.precision}")
        fn(nx, ny, nz, self.dx, self.dt, _ptr(eps_cell), _ptr(sig_cell),
           *[_ptr(c) for c in self.coef], *[_ptr(e) for e in self.eps_edge])

    def set_spacing(self, wx=None, wy=None, wz=None) -> None:
        """Cell widths (metres) along x (nx), y (ny), z (nz); None = uniform dx.
        The update then scales every difference by dx / (width it spans):
        primary widths in the H update, dual (mean of the two adjacent cells)
        in the E update (yee_oracle_body.h, non-uniform mesh). At a wall node
        the dual width is the end cell's own width, as the uniform energy
        weights the wall faces by a whole cell; no update reads those two."""
        if wx is None and wy is None and wz is None:
            self.ratios = None
            return
        out = []
        for w, n in ((wx, self.nx), (wy, self.ny), (wz, self.nz)):
            w = np.full(n, self.dx) if w is None else np.asarray(w, np.float64)
            assert w.shape == (n,) and np.all(w > 0)
            prim = self.dx / w
            ext = np.concatenate([w[:1], w, w[-1:]])
            dual = self.dx / ((ext[:-1] + ext[1:]) / 2.0)
            out.append((prim.astype(self.dtype), dual.astype(self.dtype)))
        self.ratios = tuple(a for a, _ in out) + tuple(b for _, b in out)

    def set_field(self, comp: int, arr: np.ndarray) -> None:
        self.f[comp][...] = arr

    def add_source(self, comp: int, i: int, j: int, k: int, amp: float, f0: float,
                   bw: float, t0: float, kind: int) -> None:
        self.sources.append((comp, i, j, k, amp, f0, bw, t0, kind))

    def add_probe(self, comp: int, i: int, j: int, k: int) -> int:
        self.probes.append((comp, i, j, k))
        self.probe_trace.append([])
        return len(self.probes) - 1

    # -- stepping -------------------------------------------------------------
    def step(self, nsteps: int) -> None:
        if nsteps <= 0:
            return
        nsrc = len(self.sources)
        src = np.array([s[:4] for s in self.sources] or [[0, 0, 0, 0]], np.int32).reshape(-1)
        sval = np.zeros((max(nsrc, 1), nsteps), self.dtype)
        for q, s in enumerate(self.sources):
            w = waveform(s[8], s[4], s[5], s[6], s[7], self.dt, self.n, nsteps)
            sval[q] = w.astype(self.dtype)  # one rounding from the double value
        nprb = len(self.probes)
        prb = np.array(self.probes or [[0, 0, 0, 0]], np.int32).reshape(-1)
        pout = np.zeros((max(nprb, 1), nsteps), self.dtype)
        if self.ratios is None:
            fn = getattr(load(), f"oracle_step_{self.precision}")
            fn(self.nx, self.ny, self.nz, self.S, *[_ptr(a) for a in self.f],
               *[_ptr(c) for c in self.coef], nsrc, _ptr(src), _ptr(sval), nsteps,
               nprb, _ptr(prb), _ptr(pout), nsteps, nsteps)
        else:
            fn = getattr(load(), f"oracle_step_nu_{self.precision}")
            fn(self.nx, self.ny, self.nz, self.S, *[_ptr(a) for a in self.f],
               *[_ptr(c) for c in self.coef], *[_ptr(r) for r in self.ratios], nsrc, _ptr(src),
               _ptr(sval), nsteps, nprb, _ptr(prb), _ptr(pout), nsteps, nsteps)
        for q in range(nprb):
            self.probe_trace[q].extend(pout[q].astype(np.float64).tolist())
        self.n += nsteps

    def round_fields24(self) -> None:
        """Store every field value in the 24-bit form (float32 grids)."""
        assert self.precision == "f32"
        for a in self.f:
            load().oracle_round24_f32(_ptr(a), a.size)

    def step_stored24(self, nsteps: int, k: int) -> None:
        """nsteps steps with the fields held in the 24-bit form between
        launches: launches of k steps while k steps remain, then single steps,
        each launch computing in float and storing once at its end (the
        library's launch sequence for sophie_step(nsteps) at temporal_k = k).
        Probe samples are the unrounded values of every step."""
        m = 0
        while m < nsteps:
            adv = k if (k >= 2 and nsteps - m >= k) else 1
            self.step(adv)
            self.round_fields24()
            m += adv

    def _source_table(self, nsteps: int):
        nsrc = len(self.sources)
        src = np.array([s[:4] for s in self.sources] or [[0, 0, 0, 0]], np.int32).reshape(-1)
        sval = np.zeros((max(nsrc, 1), nsteps), self.dtype)
        for q, s in enumerate(self.sources):
            sval[q] = waveform(s[8], s[4], s[5], s[6], s[7], self.dt, self.n, nsteps).astype(self.dtype)
        return nsrc, src, sval

    def grad_eps(self, pcomp: int, pi: int, pj: int, pk: int, nsteps: int, cells) -> tuple:
        """Objective J = dt * sum over the next nsteps steps of (probe value)^2 and
        dJ/d eps_r of each listed cell (reverse-mode sweep, yee_oracle_grad.c).

        The probe is component pcomp at index (pi, pj, pk), sampled after every
        step. Advances the state by nsteps steps (float64 grids only).
        """
        assert self.precision == "f64" and self.ratios is None  # uniform meshes only
        cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 3)
        grad = np.zeros(len(cells), np.float64)
        nsrc, src, sval = self._source_table(nsteps)
        J = load().oracle_grad_f64(self.nx, self.ny, self.nz, self.dx, self.dt,
                                   _ptr(self.eps_cell), _ptr(self.sig_cell), *[_ptr(a) for a in self.f],
                                   nsrc, _ptr(src), _ptr(sval), pcomp, pi, pj, pk, nsteps,
                                   len(cells), _ptr(cells), _ptr(grad))
        if not math.isfinite(J):
            raise MemoryError("oracle gradient: allocation failed")
        self.n += nsteps
        return J, grad

    def energy(self) -> float:
        if self.ratios is not None:
            fn = getattr(load(), f"oracle_energy_nu_{self.precision}")
            return fn(self.nx, self.ny, self.nz, self.S, self.dx, *[_ptr(a) for a in self.f],
                      *[_ptr(e) for e in self.eps_edge], *[_ptr(r) for r in self.ratios])
        fn = getattr(load(), f"oracle_energy_{self.precision}")
        return fn(self.nx, self.ny, self.nz, self.S, self.dx, *[_ptr(a) for a in self.f],
                  *[_ptr(e) for e in self.eps_edge])

    def probe(self, q: int) -> np.ndarray:
        return np.asarray(self.probe_trace[q], np.float64)
