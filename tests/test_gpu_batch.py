"""Batching form: many cavities of uneven sizes advanced together.

* Every cavity of a batch equals, bitwise, the float oracle run of that cavity
  alone (and a single-grid run of the library), for lossy materials with
  explicit entries and conducting cells, random initial fields and sources,
  with and without graph replay, and after the autotuner changes the split.
* Energy of every lossless cavity is conserved once its source pulse is over
  (the discrete energy identity; float fields, double accumulation).
"""

import numpy as np
import pytest

from gpu_helpers import DX
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DIMS = [(16, 17, 18), (1, 1, 5), (40, 33, 21), (96, 20, 30), (5, 70, 9), (33, 8, 64), (2, 2, 2), (64, 64, 16)]


def _materials(dims, seed):
    rng = np.random.default_rng(seed)
    eps, sig = [], []
    for (nx, ny, nz) in dims:
        nb = [(n + 3) // 4 for n in (nz, ny, nx)]
        blocks = rng.uniform(1.0, 12.0, size=nb).astype(np.float32)
        e = np.repeat(np.repeat(np.repeat(blocks, 4, 0), 4, 1), 4, 2)[:nz, :ny, :nx].copy()
        e[rng.random((nz, ny, nx)) < 0.02] = np.inf
        eps.append(e)
        sig.append(rng.uniform(0.0, 0.3, size=(nz, ny, nx)).astype(np.float32))
    return eps, sig


def _sources(dims, seed):
    rng = np.random.default_rng(seed)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    out = []
    for c, (nx, ny, nz) in enumerate(dims):
        if nx < 2 or ny < 2:
            continue
        for q in range(1 + c % 2):
            out.append((c, 2, int(rng.integers(1, nx)), int(rng.integers(1, ny)), int(rng.integers(0, nz)),
                        float(rng.uniform(1, 20)), f0, bw, t0 * (1 + q), kind))
    return out


def test_batch_equals_oracle_and_single_grids(oracle_mod, sophie):
    dims = DIMS
    eps, sig = _materials(dims, 4)
    srcs = _sources(dims, 5)
    b = so.Batch(dims, DX, wl.cfl_dt(DX))
    b.set_materials(np.concatenate([e.ravel() for e in eps]), np.concatenate([s.ravel() for s in sig]))
    fields = [wl.random_fields(*d, seed=100 + c) for c, d in enumerate(dims)]
    for c in range(len(dims)):
        for comp in range(6):
            b.set_field(c, comp, fields[c][comp])
    for s in srcs:
        b.add_source(*s)
    N1, N2, N3 = 13, 10, 6
    b.step(N1)  # TMA-staged kernel, 64 x 16 tiles, graph replay
    b.configure(tile_x=32, tile_y=4, zchunk=5, use_graph=False)
    b.step(N2)  # direct-load kernel
    b.configure(tile_x=64, zchunk=3)
    b.step(N3)
    N2 += N3
    assert b.n == N1 + N2
    W = b.energy()
    for c, (nx, ny, nz) in enumerate(dims):
        o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f32")
        o.set_materials(eps[c], sig[c])
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.set_materials(eps[c], sig[c])
        for comp in range(6):
            o.set_field(comp, fields[c][comp])
            g.set_field(comp, fields[c][comp])
        for s in srcs:
            if s[0] == c:
                o.add_source(*s[1:])
                g.add_source(*s[1:])
        o.step(N1 + N2)
        g.step(N1 + N2)
        for comp in range(6):
            got = b.get_field(c, comp)
            np.testing.assert_array_equal(got, o.f[comp], err_msg=f"cavity {c} comp {comp}")
            np.testing.assert_array_equal(got, g.get_field(comp))
        assert abs(W[c] - o.energy()) <= 1e-12 * abs(o.energy())
        g.close()


def test_graph_replay_autotune_and_reset(sophie):
    dims = DIMS[:6]
    eps, sig = _materials(dims, 8)
    srcs = _sources(dims, 9)
    b = so.Batch(dims, DX, wl.cfl_dt(DX))
    b.set_materials(np.concatenate([e.ravel() for e in eps]), np.concatenate([s.ravel() for s in sig]))
    for s in srcs:
        b.add_source(*s)
    b.step(21)  # recorded into a graph
    ref = [b.fields(c) for c in range(len(dims))]
    b.reset()
    tx, ty, zc, ms = b.autotune()
    assert (tx, ty) in ((64, 16), (32, 4), (32, 8), (32, 16)) and zc >= 1 and ms > 0
    info = b.info()
    assert (info["tile_x"], info["tile_y"], info["zchunk"]) == (tx, ty, zc)
    assert info["cells"] == sum(x * y * z for x, y, z in dims)
    assert b.n == 0
    for c in range(len(dims)):
        for comp in range(6):
            assert not b.get_field(c, comp).any()  # the trial launches left the state alone
    b.step(21)
    b.reset()
    b.step(21)  # graph replay of the same run
    for c in range(len(dims)):
        got = b.fields(c)
        for comp in range(6):
            np.testing.assert_array_equal(got[comp], ref[c][comp])
    b.configure(use_graph=False)
    b.reset()
    b.step(21)
    for c in range(len(dims)):
        for comp in range(6):
            np.testing.assert_array_equal(b.get_field(c, comp), ref[c][comp])


def test_energy_conserved_after_pulse(sophie):
    """A small instance of the batching workload: 24 lossless cavities with
    4^3-block eps_r U(1,12) and a Gaussian-pulse Ez source each; after the
    pulse (2 t0) each cavity's energy stays constant."""
    dims, eps, srcs = wl.batch_cavities(ncav=24, size_range=(16, 40), seed=17)
    b = so.Batch(dims, DX, wl.cfl_dt(DX))
    b.set_materials(eps)
    for s in srcs:
        b.add_source(*s)
    t0 = srcs[0][8]
    n_off = int(np.ceil(2 * t0 / wl.cfl_dt(DX))) + 2
    b.step(n_off)
    W0 = b.energy()
    assert np.all(W0 > 0)
    b.step(250)
    W1 = b.energy()
    rel = np.abs(W1 - W0) / W0
    print(f"max relative energy change over 250 steps after the pulse: {rel.max():.3e}")
    assert rel.max() < 2e-6


def test_batch_errors(sophie):
    with pytest.raises(so.SophieError):
        so.Batch([(0, 4, 4)], DX, wl.cfl_dt(DX))
    with pytest.raises(so.SophieError) as e:
        so.Batch([(4, 4, 4)], DX, 2 * wl.cfl_dt(DX))
    assert e.value.code == so.EUNSTABLE
    b = so.Batch([(8, 8, 8), (9, 9, 9)], DX, wl.cfl_dt(DX))
    with pytest.raises(so.SophieError):
        b.add_source(2, 2, 3, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # no cavity 2
    with pytest.raises(so.SophieError):
        b.add_source(0, 2, 0, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # PEC edge
    for q in range(4):
        b.add_source(1, 2, 3, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)
    with pytest.raises(so.SophieError):
        b.add_source(1, 2, 3, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # a fifth source
    with pytest.raises(so.SophieError) as e:
        b.configure(tile_x=32, tile_y=5)
    assert e.value.code == so.ENOTSUP
    with pytest.raises(so.SophieError) as e:
        b.configure(tile_x=64, tile_y=8)
    assert e.value.code == so.ENOTSUP
    with pytest.raises(so.SophieError):
        b.set_materials(np.full(8 ** 3 + 9 ** 3, 0.5, np.float32))
    with pytest.raises(so.SophieError):
        so.sophie_batch_get_fields(b.h, 3, 0, (2, 2, 2))  # no cavity 3


def _batch_sample_vs_oracle(oracle_mod, b, dims, eps_all, srcs, sample, nsteps):
    """Cavities `sample` of batch b after nsteps steps, bitwise = FP32 oracle."""
    offs = np.concatenate([[0], np.cumsum([int(x) * int(y) * int(z) for x, y, z in dims])])
    for c in sample:
        nx, ny, nz = (int(v) for v in dims[c])
        o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f32")
        e = eps_all[offs[c]:offs[c + 1]].reshape(nz, ny, nx)
        o.set_materials(e, np.zeros_like(e))
        for s in srcs:
            if s[0] == c:
                o.add_source(*s[1:])
        o.step(nsteps)
        for comp in range(6):
            got = b.get_field(c, comp)
            bad = np.argwhere(got != o.f[comp])
            assert bad.size == 0, (f"cavity {c} {dims[c]} comp {comp}", bad[:4])


def test_full_size_work_list_equals_oracle(oracle_mod, sophie):
    """The batching workload's generator (sizes U{16..96} per axis, eps_r per
    4^3 block, one Gaussian-pulse source each) at 512 cavities: thousands of
    work items, many times the persistent CTAs (2 per SM), so every CTA walks
    many units -- the unit context double-buffered by parity, the cross-unit
    prefetch of explicit coefficients and the tuned z chunks all run. A seeded
    sample of 16 cavities, with the largest and the smallest, is compared with
    the float oracle bit for bit after 60 steps replayed from a CUDA graph,
    once with the autotuned split and once with 32-plane z chunks."""
    import torch
    dims, eps, srcs = wl.batch_cavities(ncav=512, seed=1304)
    vol = dims.prod(axis=1)
    rng = np.random.default_rng(1314)
    sample = sorted(set([int(vol.argmax()), int(vol.argmin())]) |
                    set(int(c) for c in rng.choice(len(dims), 14, replace=False)))
    assert len(sample) >= 16
    b = so.Batch(dims, DX, wl.cfl_dt(DX))
    b.set_materials(eps)
    for s in srcs:
        b.add_source(*s)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    tx, ty, zc, _ = b.autotune()
    for cfg in ((tx, ty, zc), (64, 16, 32)):
        b.configure(tile_x=cfg[0], tile_y=cfg[1], zchunk=cfg[2], use_graph=True)
        info = b.info()
        assert info["work_items"] > 4 * 2 * nsm, info
        b.reset()
        b.step(60)  # recorded into a graph
        b.reset()
        b.step(60)  # replay of the recorded graph
        assert b.n == 60
        _batch_sample_vs_oracle(oracle_mod, b, dims, eps, srcs, sample, 60)
    b.close()


def test_packed_batch_equals_oracle_and_work_list(oracle_mod, sophie):
    """Packed layout: every cavity of the batch, run inside one grid between
    conducting layers by the tuned (temporally blocked) kernels with graph
    replay, is bitwise equal to its float oracle run and to the work-list
    layout's, with lossy block materials, conducting cells, random fields and
    sources; energies per cavity within 1e-12 of the oracle's."""
    dims = DIMS
    eps, sig = _materials(dims, 6)
    srcs = _sources(dims, 7)
    fields = [wl.random_fields(*d, seed=200 + c) for c, d in enumerate(dims)]
    out = {}
    for packed in (True, False):
        b = so.Batch(dims, DX, wl.cfl_dt(DX), packed=packed)
        b.set_materials(np.concatenate([e.ravel() for e in eps]), np.concatenate([s.ravel() for s in sig]))
        for c in range(len(dims)):
            for comp in range(6):
                b.set_field(c, comp, fields[c][comp])
        for s in srcs:
            b.add_source(*s)
        b.step(11)
        b.step(11)  # a second recorded run
        lay = b.layout()
        assert lay["packed"] == packed
        if packed:
            assert lay["temporal_k"] >= 1 and min(lay["extent"]) >= 1
        out[packed] = ([b.fields(c) for c in range(len(dims))], b.energy())
        b.close()
    for c, (nx, ny, nz) in enumerate(dims):
        o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f32")
        o.set_materials(eps[c], sig[c])
        for comp in range(6):
            o.set_field(comp, fields[c][comp])
        for s in srcs:
            if s[0] == c:
                o.add_source(*s[1:])
        o.step(22)
        for comp in range(6):
            np.testing.assert_array_equal(out[True][0][c][comp], o.f[comp], err_msg=f"cavity {c} comp {comp}")
            np.testing.assert_array_equal(out[True][0][c][comp], out[False][0][c][comp])
        assert abs(out[True][1][c] - o.energy()) <= 1e-12 * abs(o.energy())


def test_packed_batch_workload_sample_equals_oracle(oracle_mod, sophie):
    """The batching workload's generator at 512 cavities in the packed layout:
    60 steps recorded and then replayed from a CUDA graph (autotuned k and
    tilings), a seeded sample of 16 cavities with the largest and the smallest
    bitwise equal to the float oracle; every cavity's energy conserved once
    its pulse is over is checked elsewhere, here the sample's energies match
    the oracle's within 1e-12."""
    dims, eps, srcs = wl.batch_cavities(ncav=512, seed=1304)
    vol = dims.prod(axis=1)
    rng = np.random.default_rng(1315)
    sample = sorted(set([int(vol.argmax()), int(vol.argmin())]) |
                    set(int(c) for c in rng.choice(len(dims), 14, replace=False)))
    b = so.Batch(dims, DX, wl.cfl_dt(DX), packed=True)
    b.set_materials(eps)
    for s in srcs:
        b.add_source(*s)
    tx, ty, zc, ms = b.autotune()
    assert ms > 0 and zc == 0
    b.step(60)
    b.reset()
    b.step(60)  # replay of the recorded graph
    assert b.n == 60
    _batch_sample_vs_oracle(oracle_mod, b, dims, eps, srcs, sample, 60)
    W = b.energy()
    offs = np.concatenate([[0], np.cumsum(vol)])
    for c in sample[:4]:
        nx, ny, nz = (int(v) for v in dims[c])
        o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f32")
        e = eps[offs[c]:offs[c + 1]].reshape(nz, ny, nx)
        o.set_materials(e, np.zeros_like(e))
        for s in srcs:
            if s[0] == c:
                o.add_source(*s[1:])
        o.step(60)
        assert abs(W[c] - o.energy()) <= 1e-12 * abs(o.energy())
    b.close()


def test_packed_batch_errors(sophie):
    b = so.Batch([(8, 8, 8), (9, 9, 9)], DX, wl.cfl_dt(DX), packed=True)
    with pytest.raises(so.SophieError) as e:
        b.configure(tile_x=64)
    assert e.value.code == so.ENOTSUP
    b.configure(use_graph=False)
    with pytest.raises(so.SophieError):
        b.add_source(0, 2, 0, 3, 3, 1.0, 1e10, 5e9, 1e-10, 0)  # PEC edge
    with pytest.raises(so.SophieError):
        b.origin(2)
    o0, o1 = b.origin(0), b.origin(1)
    assert o0 != o1
    w = so.Batch([(8, 8, 8)], DX, wl.cfl_dt(DX))
    with pytest.raises(so.SophieError) as e:
        w.origin(0)
    assert e.value.code == so.ENOTSUP
    assert not w.layout()["packed"]
    w.close()
    b.close()
