"""Non-uniform mesh (per-axis cell widths): the CUDA path against the oracle.

* Random widths on every axis, lossy materials with conducting cells, random
  initial fields, a source and probes: fields and probe samples bitwise equal
  to the float oracle's, for the TMA-staged plain kernel, the direct-load
  kernel and the temporally blocked kernel at K = 2, 3, 4, on grids spanning
  several tiles with ragged tails; energy within 1e-12 of the oracle's.
* All widths equal to dx: bitwise the uniform run; clearing the widths
  returns to the uniform kernels.
* Lossless, sourceless graded mesh: the volume-weighted energy is conserved.
* Zero-field skipping on a graded mesh (plain, direct-load, K = 2, 3):
  bitwise the oracle.
* Split hi+lo half storage on a graded mesh stays within 1e-4 of float
  (K = 1, 2).
* The graded 256^3 sphere cavity (the non-uniform bench workload, its launch
  configuration): 300 steps, fields and probes bitwise equal to the float
  oracle, energy within the summation-order bound.
* Argument errors: bad widths, a time step above the mesh's Courant limit,
  probe objectives on this mesh.
"""

import numpy as np
import pytest

from gpu_helpers import DX, assert_fields_equal
from modes import rel_l2
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _graded_pair(oracle_mod, nx, ny, nz, seed, tile_x=64, lossy=True, fields=True, source=True, probes=True, K=1):
    wx, wy, wz = (wl.random_widths(n, seed + a) for a, n in enumerate((nx, ny, nz)))
    dt = wl.mesh_dt(wx, wy, wz)
    eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=6, sigma=(0.0, 0.4) if lossy else (0.0, 0.0))
    if lossy:
        eps = eps.copy()
        eps[np.random.default_rng(seed).random(eps.shape) < 0.01] = np.inf  # conducting cells
    g = so.Grid(nx, ny, nz, DX, dt)
    g.configure(temporal_k=K, tile_x=tile_x)
    o = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f32")
    for t in (g, o):
        t.set_materials(eps, sig)
        t.set_spacing(wx, wy, wz)
    if fields:
        f = wl.random_fields(nx, ny, nz, seed + 10)
        for c in range(6):
            g.set_field(c, f[c])
            o.set_field(c, f[c])
    prbs = []
    if source:
        amp, f0, bw, t0, kind = wl.gaussian_sine_source()
        src = (2, nx // 2, max(1, ny // 2), nz // 2, 20.0, f0, bw, 3e-12, kind)
        g.add_source(*src)
        o.add_source(*src)
    if probes:
        prbs = wl.probe_edges(nx, ny, nz, 5, seed=seed) + [(3, 0, 0, 0), (4, nx - 1, 1, nz - 1), (5, 1, ny - 1, 2)]
        for p in prbs:
            g.add_probe(*p)
            o.add_probe(*p)
    return g, o, prbs, (wx, wy, wz)


@pytest.mark.parametrize("kernel", ["plain", "direct", "k2", "k3", "k4", "k6", "k8"])
@pytest.mark.parametrize("n3,steps", [((70, 37, 19), 23), ((130, 21, 40), 11), ((64, 16, 8), 7), ((3, 90, 5), 9)])
def test_graded_mesh_equals_oracle(oracle_mod, sophie, kernel, n3, steps):
    tile_x = 32 if kernel == "direct" else 64
    K = int(kernel[1]) if kernel.startswith("k") else 1
    g, o, prbs, _ = _graded_pair(oracle_mod, *n3, seed=sum(n3), tile_x=tile_x, K=K)
    g.step(steps)
    o.step(steps)
    assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    Wo = o.energy()
    assert abs(g.energy() - Wo) <= 1e-12 * abs(Wo)


def test_unit_widths_are_the_uniform_mesh(sophie):
    nx, ny, nz = 90, 40, 33
    eps, sig = wl.random_materials(nx, ny, nz, 3, nmat=5, sigma=(0.0, 0.3))
    f = wl.random_fields(nx, ny, nz, 4)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    out = []
    for mode in ("uniform", "unit", "cleared"):
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.set_materials(eps, sig)
        for c in range(6):
            g.set_field(c, f[c])
        g.add_source(2, 40, 20, 16, 5.0, f0, bw, t0, kind)
        if mode != "uniform":
            g.set_spacing(np.full(nx, DX), np.full(ny, DX), np.full(nz, DX))
        if mode == "cleared":
            g.set_spacing()
        g.step(17)
        out.append((g.fields(), g.energy()))
        g.close()
    for m in (1, 2):
        for c in range(6):
            np.testing.assert_array_equal(out[m][0][c], out[0][0][c])
        assert abs(out[m][1] - out[0][1]) <= 1e-13 * out[0][1]


def test_energy_conserved_on_graded_mesh(oracle_mod, sophie):
    g, o, _, _ = _graded_pair(oracle_mod, 60, 50, 40, seed=21, lossy=False, source=False, probes=False)
    W0 = g.energy()
    assert abs(W0 - o.energy()) <= 1e-12 * abs(W0)
    drift = 0.0
    for _ in range(8):
        g.step(25)
        drift = max(drift, abs(g.energy() - W0) / W0)
    print(f"max relative energy drift over 200 steps: {drift:.3e}")
    assert drift < 5e-6


@pytest.mark.parametrize("tile_x,K", [(64, 1), (32, 1), (64, 2), (64, 3)])
def test_zero_skip_on_graded_mesh(oracle_mod, sophie, tile_x, K):
    g, o, prbs, _ = _graded_pair(oracle_mod, 150, 70, 60, seed=5, tile_x=tile_x, fields=False, K=K)
    g.set_zero_skip(True)
    done = 0
    for n in (3, 20, 45):
        g.step(n - done)
        o.step(n - done)
        done = n
        assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))


@pytest.mark.parametrize("K", [1, 2])
def test_fp16hl_storage_on_graded_mesh(oracle_mod, sophie, K):
    g, o, _, _ = _graded_pair(oracle_mod, 80, 48, 36, seed=8, fields=False)
    g.configure(temporal_k=K, precision=so.FP16HL)
    g.set_storage_scale([2.0 ** 6] * 6)
    g.step(150)
    o.step(150)
    gf = g.fields()
    for c in range(6):
        assert rel_l2(gf[c], o.f[c]) < 1e-4, c


def test_graded_sphere_cavity_full_size(oracle_mod, sophie):
    """The graded 256^3 sphere cavity in the bench's configuration (autotuned)."""
    w = wl.sphere_cavity_graded(256)
    n = w["nx"]
    steps = 300
    o = oracle_mod.OracleGrid(n, n, n, w["dx"], w["dt"], "f32")
    g = so.Grid(n, n, n, w["dx"], w["dt"])
    for t in (o, g):
        t.set_materials(w["eps"], w["sigma"])
        t.set_spacing(*w["widths"])
        for s in w["sources"]:
            t.add_source(*s)
        for p in w["probes"]:
            t.add_probe(*p)
    o.step(steps)
    g.step(steps)
    gf = assert_fields_equal(g, o)
    assert np.abs(gf[2]).max() > 0
    for q in range(len(w["probes"])):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    # Same float fields, different double summation orders (the oracle one
    # running sum, the GPU a block tree) of N ~ 1e8 terms, nearly all positive
    # (sum |t| ~ W): the worst-case bound of sequential summation is (N-1) u W
    # (measured 2.4e-11 relative).
    Wo = o.energy()
    nterms = 6 * (n + 1) ** 3
    assert Wo > 0 and abs(g.energy() - Wo) <= nterms * 2.0 ** -53 * Wo


def test_spacing_errors(sophie):
    nx, ny, nz = 20, 16, 12
    g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    with pytest.raises(ValueError):
        g.set_spacing(np.full(nx + 1, DX))
    for bad in (0.0, -DX, np.nan, np.inf):
        w = np.full(nx, DX)
        w[3] = bad
        with pytest.raises(so.SophieError) as e:
            g.set_spacing(w)
        assert e.value.code == so.EINVAL
    w = np.full(ny, DX)
    w[5] = 0.5 * DX  # dt is at the uniform limit: a finer cell is unstable
    with pytest.raises(so.SophieError) as e:
        g.set_spacing(None, w)
    assert e.value.code == so.EUNSTABLE
    g.set_spacing(np.full(nx, 2 * DX))  # coarser cells are fine
    g.configure(temporal_k=2)  # the blocked kernel takes the mesh too
    with pytest.raises(so.SophieError) as e:
        g.objective_forward(10, 2, 5, 5, 5)
    assert e.value.code == so.ENOTSUP
    g.close()
