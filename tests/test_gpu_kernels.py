"""Step kernels against each other and, at the benchmark's full size, against
the oracle.

* The TMA-staged kernel (64x16 tiles, persistent CTAs, z chunks) and the
  direct-load kernel (32x8 tiles) give bitwise identical fields on ragged grids
  that span several tiles, chunks and a partial last tile.
* The 256^3 sphere cavity (the benchmark workload) for the full 1000 steps in
  the launch configuration bench.py times: every field value and every probe
  sample equals the float32 oracle's.
"""

import numpy as np
import pytest

from gpu_helpers import DX, assert_fields_equal, make_pair
from modes import rel_l2
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n3,steps", [((130, 70, 50), 9), ((64, 16, 8), 5), ((65, 17, 33), 7),
                                      ((200, 3, 12), 4)])
def test_tma_kernel_equals_direct_kernel(sophie, n3, steps):
    nx, ny, nz = n3
    eps, sig = wl.random_materials(nx, ny, nz, seed=nx + ny, nmat=7, sigma=(0.0, 0.4))
    f = wl.random_fields(nx, ny, nz, seed=nz)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    src = (2, nx // 2, max(1, ny // 2), nz // 2, 20.0, f0, bw, 3e-12, 0)
    prbs = wl.probe_edges(nx, ny, nz, 5, seed=3) + [(3, 0, 0, 0), (5, nx - 1, ny - 1, nz)]
    out = []
    for tile_x in (64, 32):
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.configure(temporal_k=1, tile_x=tile_x)
        g.set_materials(eps, sig)
        for c in range(6):
            g.set_field(c, f[c])
        g.add_source(*src)
        for p in prbs:
            g.add_probe(*p)
        g.step(steps)
        out.append((g.fields(), [g.read_probe(q) for q in range(len(prbs))], g.energy()))
    for c in range(6):
        np.testing.assert_array_equal(out[0][0][c], out[1][0][c])
    for q in range(len(prbs)):
        np.testing.assert_array_equal(out[0][1][q], out[1][1][q])
    assert out[0][2] == out[1][2]


def test_full_size_sphere_cavity_1000_steps(oracle_mod, sophie):
    """Benchmark workload, full length, every kernel configuration the bench can time."""
    w = wl.sphere_cavity(256)
    n = w["nx"]
    o = oracle_mod.OracleGrid(n, n, n, w["dx"], w["dt"], "f32")
    o.set_materials(w["eps"], w["sigma"])
    for s in w["sources"]:
        o.add_source(*s)
    for p in w["probes"]:
        o.add_probe(*p)
    o.step(1000)
    Wo = o.energy()
    for K in (1, 2, 3, 4):
        g = so.Grid(n, n, n, w["dx"], w["dt"])
        g.configure(temporal_k=K)
        g.set_materials(w["eps"], w["sigma"])
        for s in w["sources"]:
            g.add_source(*s)
        for p in w["probes"]:
            g.add_probe(*p)
        g.step(1000)
        gf = assert_fields_equal(g, o)
        for c in range(6):
            assert rel_l2(gf[c], o.f[c]) <= 1e-5
        for q in range(len(w["probes"])):
            np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
        W = g.energy()
        assert abs(W - Wo) <= 1e-12 * abs(Wo)
        assert W > 0
        g.close()


def test_launches_with_and_without_programmatic_dependent_launch(tmp_path):
    """The step kernels wait for the previous kernel before any global access
    (programmatic dependent launch); SOPHIE_PDL=0 launches them plainly. A
    mixed sequence (plain and blocked steps, a precision change, probes, the
    energy) gives bitwise the same fields either way; each run is a fresh
    process, since the switch is read once."""
    import subprocess
    import sys

    code = r"""
import sys, numpy as np
from paper_1301_4539_gb300 import sophie as so, workloads as wl
nx, ny, nz = 150, 70, 60
eps, sig = wl.random_materials(nx, ny, nz, seed=5, nmat=6, sigma=(0.0, 0.3))
g = so.Grid(nx, ny, nz, 1e-3, wl.cfl_dt(1e-3))
g.set_materials(eps, sig)
amp, f0, bw, t0, kind = wl.gaussian_sine_source()
g.add_source(2, 75, 35, 30, 20.0, f0, bw, 3e-12, 0)
pid = g.add_probe(2, 80, 30, 31)
for k, n in ((1, 7), (2, 12), (3, 7), (0, 9)):
    g.configure(temporal_k=k)
    g.step(n)
g.configure(temporal_k=2, precision=so.FP24)
g.step(10)
W = g.energy()
np.savez(sys.argv[1], *[g.get_field(c) for c in range(6)], probe=g.read_probe(pid), W=np.array([W]))
"""
    outs = []
    for v in ("1", "0"):
        path = tmp_path / f"pdl{v}.npz"
        env = dict(__import__("os").environ, SOPHIE_PDL=v)
        root = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
        r = subprocess.run([sys.executable, "-c", code, str(path)], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(path))
    for key in outs[0].files:
        np.testing.assert_array_equal(outs[0][key], outs[1][key])
