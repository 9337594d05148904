"""CUDA path vs the CPU oracle, element by element, on seeded inputs.

Bar: the float32 fields and probe samples are bitwise equal to the oracle's
float32 run (both evaluate the same expression tree, one fused
multiply-add per update and every other operation rounded separately, and
the per-edge coefficients are the same double expression rounded once); relative L2 <= 1e-5 is the tolerance the method fixes, and is
also checked. The energy (double accumulation of the same float values)
agrees to 1e-12 relative.
"""

import math

import numpy as np
import pytest

from gpu_helpers import DX, assert_fields_equal, make_pair
from modes import CavityMode, rel_l2
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _tm110(oracle_mod):
    S = oracle_mod.C0 * wl.cfl_dt(DX) / DX
    m = CavityMode(32, 32, 32, 1, 1, 0, [0, 0, 1], S)
    st = m.state(0)
    return m, [a.astype(np.float32) for a in st]


def test_tm110_cavity(oracle_mod, sophie):
    m, st = _tm110(oracle_mod)
    g, o = make_pair(oracle_mod, 32, 32, 32, fields=st, probes=[(2, 9, 13, 5)])
    W0 = g.energy()
    assert abs(W0 - o.energy()) / W0 < 1e-12
    wmax = 0.0
    for _ in range(20):
        g.step(10)
        o.step(10)
        W = g.energy()
        assert abs(W - o.energy()) / W0 < 1e-12
        wmax = max(wmax, abs(W - W0) / W0)
    assert wmax < 1e-6
    gf = assert_fields_equal(g, o)
    ref = m.state(200)
    assert max(rel_l2(gf[c], ref[c]) for c in (2, 3, 4)) < 1e-5
    np.testing.assert_array_equal(g.read_probe(0), o.probe(0))


CASES = [
    (5, 6, 7, 30),
    (17, 33, 9, 25),
    (40, 21, 35, 20),
    (70, 9, 20, 15),
    (33, 65, 18, 12),
]


@pytest.mark.parametrize("nx,ny,nz,steps", CASES)
def test_random_lossy_with_source_and_probes(oracle_mod, sophie, nx, ny, nz, steps):
    eps, sig = wl.random_materials(nx, ny, nz, seed=nx * 7 + ny, nmat=6, sigma=(0.0, 0.5))
    f = wl.random_fields(nx, ny, nz, seed=nx + 1000 * ny)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, nx // 2 if nx > 1 else 0, max(1, ny // 2), nz // 2, 30.0, f0, bw, 5 * 1.9e-12, 0)]
    if nx > 2 and nz > 2:
        srcs.append((0, 0, max(1, ny // 3), max(1, nz // 3), 10.0, f0, bw, 8 * 1.9e-12, 1))
    prbs = [(c, min(1, nx - 1) if c in (1, 2) else 0, min(1, ny - 1), min(1, nz - 1)) for c in range(6)]
    prbs += wl.probe_edges(nx, ny, nz, 4, seed=nx)
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, srcs, prbs)
    g.step(steps)
    o.step(steps)
    assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    W, Wo = g.energy(), o.energy()
    assert abs(W - Wo) / abs(Wo) < 1e-12


@pytest.mark.parametrize("n3", [(1, 1, 1), (1, 1, 5), (2, 2, 2), (1, 7, 3), (3, 1, 9)])
def test_degenerate_grids(oracle_mod, sophie, n3):
    nx, ny, nz = n3
    f = wl.random_fields(nx, ny, nz, seed=7)
    g, o = make_pair(oracle_mod, nx, ny, nz, fields=f)
    g.step(5)
    o.step(5)
    assert_fields_equal(g, o)


def test_step_zero_and_counter(oracle_mod, sophie):
    g, o = make_pair(oracle_mod, 6, 5, 4, fields=wl.random_fields(6, 5, 4, 3))
    before = g.fields()
    g.step(0)
    assert g.n == 0
    after = g.fields()
    for c in range(6):
        np.testing.assert_array_equal(before[c], after[c])
    g.step(3)
    assert g.n == 3


def test_reset_and_rerun_is_deterministic(oracle_mod, sophie):
    nx, ny, nz = 24, 20, 18
    eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=5, seed=2, radius=(2, 5))
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g, _ = make_pair(oracle_mod, nx, ny, nz, eps, sig, sources=[(2, 12, 10, 9, amp, f0, bw, t0, 0)],
                     probes=[(2, 3, 4, 5)])
    g.step(40)
    a = g.fields()
    pa = g.read_probe(0)
    g.reset()
    assert g.n == 0
    g.step(40)
    b = g.fields()
    for c in range(6):
        np.testing.assert_array_equal(a[c], b[c])
    np.testing.assert_array_equal(pa, g.read_probe(0))


def test_pec_and_range_masking_on_set_fields(oracle_mod, sophie):
    nx, ny, nz = 6, 5, 4
    g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    ones = np.ones((nz + 1, ny + 1, nx + 1), np.float32)
    ref = wl.random_fields(nx, ny, nz, 0)
    for c in range(6):
        g.set_field(c, ones)
        got = g.get_field(c)
        np.testing.assert_array_equal(got != 0, ref[c] != 0)


def test_argument_errors_on_gpu(sophie):
    nx, ny, nz = 8, 8, 8
    g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    ones = np.ones((nz, ny, nx), np.float32)
    zeros = np.zeros((nz, ny, nx), np.float32)
    with pytest.raises(so.SophieError) as e:
        g.set_materials(ones * 0.5, zeros)
    assert e.value.code == so.EINVAL
    with pytest.raises(so.SophieError) as e:
        g.set_materials(ones, zeros - 1)
    assert e.value.code == so.EINVAL
    bad = ones.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(so.SophieError):
        g.set_materials(bad, zeros)
    with pytest.raises(so.SophieError):
        g.add_source(2, 0, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # ez on the x=0 wall: PEC
    with pytest.raises(so.SophieError):
        g.add_source(3, 3, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # H component
    with pytest.raises(so.SophieError):
        g.add_probe(0, nx, 3, 3)  # ex has no index nx
    with pytest.raises(so.SophieError):
        g.step(-1)
    with pytest.raises(so.SophieError) as e:
        g.configure(precision=7)
    assert e.value.code == so.ENOTSUP
    nan = np.zeros((nz + 1, ny + 1, nx + 1), np.float32)
    nan[2, 2, 2] = np.nan
    g.set_field(3, nan)
    with pytest.raises(so.SophieError) as e:
        g.energy()
    assert e.value.code == so.ENONFINITE


@pytest.mark.parametrize("K", [1, 2, 3])
def test_continuous_materials_explicit_points(oracle_mod, sophie, K):
    """Every cell its own (eps, sigma): far more edge materials than classes,
    so most points carry explicit coefficients; still bitwise = oracle."""
    nx, ny, nz = 23, 19, 14
    rng = np.random.default_rng(31)
    eps = rng.uniform(1.0, 12.0, size=(nz, ny, nx)).astype(np.float32)
    sig = rng.uniform(0.0, 0.5, size=(nz, ny, nx)).astype(np.float32)
    f = wl.random_fields(nx, ny, nz, 17)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, [(2, 11, 9, 7, 5.0, f0, bw, t0, kind)],
                     [(2, 4, 5, 6), (0, 3, 3, 3)], temporal_k=K)
    g.step(3 * K + 1)
    o.step(3 * K + 1)
    assert_fields_equal(g, o)
    for q in range(2):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    assert abs(g.energy() - o.energy()) <= 1e-12 * abs(o.energy())


@pytest.mark.parametrize("K", [1, 2])
def test_design_region_in_class_background(oracle_mod, sophie, K):
    """Sphere background (classes) with a random-eps design block (explicit points)."""
    n = 48
    eps, sig = wl.sphere_materials(n, n, n, nspheres=6, seed=3, radius=(3, 9))
    rng = np.random.default_rng(8)
    eps[16:32, 16:32, 16:32] = rng.uniform(1.0, 4.0, size=(16, 16, 16)).astype(np.float32)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g, o = make_pair(oracle_mod, n, n, n, eps, sig, None, [(2, 8, 24, 24, amp, f0, bw, t0, 1)],
                     [(2, 40, 24, 24)], temporal_k=K)
    g.step(30)
    o.step(30)
    assert_fields_equal(g, o)
    np.testing.assert_array_equal(g.read_probe(0), o.probe(0))


@pytest.mark.parametrize("K", [1, 2, 3])
def test_conducting_cells(oracle_mod, sophie, K):
    """Perfectly conducting cells (eps_r = +inf): scattered cells, a full layer
    splitting the grid, and 4^3-block random eps (explicit entries shared by
    points with the same three edge materials); bitwise = oracle."""
    nx, ny, nz = 41, 22, 17
    rng = np.random.default_rng(77)
    blocks = rng.uniform(1.0, 12.0, size=((nz + 3) // 4, (ny + 3) // 4, (nx + 3) // 4)).astype(np.float32)
    eps = np.repeat(np.repeat(np.repeat(blocks, 4, 0), 4, 1), 4, 2)[:nz, :ny, :nx].copy()
    eps[rng.random((nz, ny, nx)) < 0.03] = np.inf
    eps[:, :, 20] = np.inf
    sig = rng.uniform(0.0, 0.2, size=(nz, ny, nx)).astype(np.float32)
    f = wl.random_fields(nx, ny, nz, 5)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, [(2, 30, 11, 8, 3.0, f0, bw, t0, kind)],
                     [(2, 10, 10, 10), (2, 31, 11, 8)], temporal_k=K)
    g.step(4 * K + 1)
    o.step(4 * K + 1)
    assert_fields_equal(g, o)
    for q in range(2):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    assert abs(g.energy() - o.energy()) <= 1e-12 * abs(o.energy())
