"""Helpers that run the same seeded case through the CUDA library and the oracle."""

from __future__ import annotations

import numpy as np

from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

DX = 1e-3


def make_pair(oracle_mod, nx, ny, nz, eps=None, sig=None, fields=None, sources=(), probes=(),
              temporal_k=1, prec="f32"):
    dt = wl.cfl_dt(DX)
    g = so.Grid(nx, ny, nz, DX, dt)
    g.configure(temporal_k=temporal_k)
    o = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, prec)
    if eps is not None:
        g.set_materials(eps, sig)
        o.set_materials(eps, sig)
    if fields is not None:
        for c in range(6):
            g.set_field(c, fields[c].astype(np.float32))
            o.set_field(c, fields[c].astype(o.dtype))
    for s in sources:
        g.add_source(*s)
        o.add_source(*s)
    for p in probes:
        g.add_probe(*p)
        o.add_probe(*p)
    return g, o


def assert_fields_equal(g, o, exact=True, tol=1e-5):
    from modes import rel_l2
    gf = g.fields()
    for c in range(6):
        if exact:
            bad = np.argwhere(gf[c] != o.f[c])
            assert bad.size == 0, (c, bad[:5], gf[c][tuple(bad[0])] if bad.size else None,
                                   o.f[c][tuple(bad[0])] if bad.size else None)
        else:
            assert rel_l2(gf[c], o.f[c]) <= tol, c
    return gf
