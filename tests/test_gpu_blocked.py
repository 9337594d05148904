"""Temporally blocked kernel (K steps per launch) against K plain steps and the oracle.

Sec. 3.1: restructuring the loops changes no output value. The blocked
kernel evaluates the same float expressions, so fields and probe samples must
be bitwise equal to the plain kernel's and to the oracle's, for every K, on
grids that span several tiles, ragged tails, and z ranges split across CTAs
(small grids give each CTA a few planes, so the replay of 3K-2 planes before a
range start is exercised everywhere).
"""

import numpy as np
import pytest

from gpu_helpers import DX, assert_fields_equal, make_pair
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# (37, 116, 21) and (50, 200, 13): many y tiles, probes next to both y walls.
SIZES = [(5, 6, 7), (17, 33, 9), (40, 21, 35), (70, 9, 20), (130, 70, 50), (61, 29, 3), (37, 116, 21),
         (50, 200, 13)]


@pytest.mark.parametrize("K", [2, 3, 4, 6, 8])
@pytest.mark.parametrize("n3", SIZES)
def test_blocked_equals_oracle(oracle_mod, sophie, K, n3):
    nx, ny, nz = n3
    eps, sig = wl.random_materials(nx, ny, nz, seed=nx * 3 + nz, nmat=6, sigma=(0.0, 0.5))
    f = wl.random_fields(nx, ny, nz, seed=ny + 17)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, nx // 2 if nx > 1 else 0, max(1, ny // 2), nz // 2, 30.0, f0, bw, 4e-12, 0)]
    if nx > 2 and nz > 2:
        srcs.append((1, max(1, nx // 3), 0, max(1, nz // 2), 7.0, f0, bw, 6e-12, 1))
    prbs = wl.probe_edges(nx, ny, nz, 6, seed=nx + K) + [(3, 0, 0, 0), (4, nx - 1, ny, max(0, nz - 1)),
                                                         (5, 0, 0, nz)]
    if ny > 8 and nx > 2 and nz > 2:  # rows next to the y walls (inside the wall tiles)
        prbs += [(0, nx // 2, ny - 1, nz // 2), (2, nx // 2, ny - 2, nz // 2), (1, 1, 0, 1), (3, nx // 2, ny - 1, 1)]
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, srcs, prbs, temporal_k=K)
    steps = 3 * K + 2  # blocked launches plus a plain remainder
    g.step(steps)
    o.step(steps)
    assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    assert abs(g.energy() - o.energy()) <= 1e-12 * abs(o.energy())


@pytest.mark.parametrize("aligned", ["2", "3", "0"])
@pytest.mark.parametrize("K", [2, 3])
def test_blocked_many_tiles_several_units_per_cta(oracle_mod, sophie, monkeypatch, K, aligned):
    """More tiles than SMs: the aligned split gives each CTA several (z range,
    tile) units taken with a stride of the grid (700x420x40 at K=2: 180 tiles,
    2 ranges), tile-major (2) or range-major (3); the contiguous split (0)
    ranges that straddle tiles."""
    monkeypatch.setenv("SOPHIE_BLOCKED_ALIGNED", aligned)
    nx, ny, nz = 700, 420, 40
    eps, sig = wl.random_materials(nx, ny, nz, seed=71, nmat=6, sigma=(0.0, 0.5))
    f = wl.random_fields(nx, ny, nz, seed=72)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, 350, 210, 20, 30.0, f0, bw, 4e-12, 0)]
    prbs = wl.probe_edges(nx, ny, nz, 6, seed=73) + [(0, 599, 419, 39), (2, 61, 27, 0)]
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, srcs, prbs, temporal_k=K)
    steps = 2 * K + 1
    g.step(steps)
    o.step(steps)
    assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))


@pytest.mark.parametrize("K", [2, 3, 4, 6, 8])
def test_blocked_equals_plain_long(sophie, K):
    nx, ny, nz = 100, 90, 80
    eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=12, seed=9, radius=(3, 15))
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    src = (2, nx // 2, ny // 2, nz // 2, amp, f0, bw, t0, kind)
    prbs = wl.probe_edges(nx, ny, nz, 8, seed=77)
    res = []
    for k in (1, K):
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.configure(temporal_k=k)
        g.set_materials(eps, sig)
        g.add_source(*src)
        for p in prbs:
            g.add_probe(*p)
        g.step(200)
        res.append((g.fields(), [g.read_probe(q) for q in range(len(prbs))]))
    for c in range(6):
        np.testing.assert_array_equal(res[0][0][c], res[1][0][c])
    for q in range(len(prbs)):
        np.testing.assert_array_equal(res[0][1][q], res[1][1][q])


def test_unsupported_k(sophie):
    g = so.Grid(8, 8, 8, DX, wl.cfl_dt(DX))
    for k in (5, 7):
        with pytest.raises(so.SophieError) as e:
            g.configure(temporal_k=k)
        assert e.value.code == so.ENOTSUP
    # the deep forms are built for float storage only
    for prec in (so.FP16, so.BF16, so.FP16HL, so.FP24):
        with pytest.raises(so.SophieError) as e:
            g.configure(temporal_k=6, precision=prec)
        assert e.value.code == so.ENOTSUP
    g.configure(temporal_k=8)
    with pytest.raises(so.SophieError) as e:
        g.configure(temporal_k=8, precision=so.FP24)
    assert e.value.code == so.ENOTSUP
    with pytest.raises(so.SophieError):
        g.configure(temporal_k=9)


@pytest.mark.parametrize("zsplit", ["13", "20"])
@pytest.mark.parametrize("K", [2, 3, 4, 6, 8])
def test_blocked_short_units(oracle_mod, sophie, monkeypatch, K, zsplit):
    """Units of 2 to 3 planes (every tile's 40 planes cut into 13 or 20 z
    ranges): most units start within the first planes or replay 3K - 2 planes,
    and each starts its levels' state (carries and shared-memory seam rows)
    from zero. Lossy materials with explicit entries, sources and probes."""
    monkeypatch.setenv("SOPHIE_BLOCKED_ZSPLIT", zsplit)
    nx, ny, nz = 130, 21, 40
    eps, sig = wl.random_materials(nx, ny, nz, seed=11 * K, nmat=6, sigma=(0.0, 0.5))
    eps = eps.copy()
    eps[:, : ny // 3, : nx // 4] = np.random.default_rng(K).uniform(1, 9, size=(nz, ny // 3, nx // 4))
    f = wl.random_fields(nx, ny, nz, seed=K + 3)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, nx // 2, ny // 2, nz // 2, 25.0, f0, bw, 4e-12, 0), (0, nx // 3, ny // 3, 1, 3.0, f0, bw, 5e-12, 1)]
    prbs = wl.probe_edges(nx, ny, nz, 5, seed=nx) + [(3, nx // 2, ny // 2, 0), (5, 1, 1, nz)]
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, srcs, prbs, temporal_k=K)
    for n in (3 * K + 1, K + 2):
        g.step(n)
        o.step(n)
        assert_fields_equal(g, o)
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
