"""sophie_energy_noalloc: the energy for callers that cannot allocate.

Some applications reserve their whole device-memory budget up front (a
caching allocator that owns the heap, or a host that forbids allocation once
it runs), so a cudaMalloc at the point where they need the energy fails or is
not allowed; this entry point serves them by keeping its reduction scratch in
a static device array instead of allocating. Here it is called through the C ABI
and must give the same energy as sophie_energy (the allocating entry point),
within the 1e-12 relative tolerance the energy tests use, on two calls in a
row (the static scratch keeps the previous call's contents), on a uniform and
on a non-uniform mesh.
"""

import ctypes

import numpy as np
import pytest

from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DX = 1e-3


def _grid(graded=False):
    nx, ny, nz = 70, 45, 38
    widths = [wl.random_widths(n, seed=30 + a) for a, n in enumerate((nx, ny, nz))]
    g = so.Grid(nx, ny, nz, DX, wl.mesh_dt(*widths) if graded else wl.cfl_dt(DX))
    eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=6, seed=21, radius=(3, 10))
    g.set_materials(eps, sig)
    if graded:  # the volume-weighted energy of a non-uniform mesh
        g.set_spacing(*widths)
    f = wl.random_fields(nx, ny, nz, seed=22)
    for c in range(6):
        g.set_field(c, f[c])
    return g


@pytest.mark.parametrize("graded", [False, True])
def test_energy_noalloc_matches_energy(sophie, graded):
    import torch

    lib = so.load()
    g = _grid(graded)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")  # caller-owned result slots
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:
            g.step(7)
        ref = g.energy()
        rc = lib.sophie_energy_noalloc(ctypes.c_void_p(g.h), ctypes.c_void_p(out.data_ptr() + 8 * call))
        assert rc == 0, so.sophie_last_error()
        g.sync()
        got = float(out[call].item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
    # the same state twice in a row: the second call must not depend on the first's scratch
    rc1 = lib.sophie_energy_noalloc(ctypes.c_void_p(g.h), ctypes.c_void_p(out.data_ptr()))
    rc2 = lib.sophie_energy_noalloc(ctypes.c_void_p(g.h), ctypes.c_void_p(out.data_ptr() + 8))
    assert rc1 == 0 and rc2 == 0
    g.sync()
    a, b = out.cpu().numpy()
    assert a == b
    assert abs(a - g.energy()) <= 1e-12 * abs(a)
    g.close()


def test_energy_noalloc_rejects_null(sophie):
    lib = so.load()
    g = _grid()
    assert lib.sophie_energy_noalloc(ctypes.c_void_p(g.h), None) == so.EINVAL
    assert lib.sophie_energy_noalloc(None, None) == so.EINVAL
    g.close()
