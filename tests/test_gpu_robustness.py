"""Bounds, failure and timeout behaviour on the GPU (no fault, no hang).

* Guards: every kernel form (plain, blocked K = 2..4, the 2-byte and hi+lo
  storage, the direct-load kernel, the objective record and reverse sweep,
  both batch kernels) leaves the guard bytes around the field buffers intact.
* Bounded waits: a kernel waits on an mbarrier that nothing completes; the
  wait gives up after its limit, the host sees SOPHIE_ETIMEOUT once, and the
  grid keeps producing the oracle's fields.
* Allocation failures (host-side hook): every allocation of grid creation,
  batch creation and the objective record can fail; the call returns ENOMEM,
  frees what it had, and later calls work.
* Double destroy and oversized grids are rejected.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import DX, assert_fields_equal, make_pair
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _grid(n3=(37, 29, 23), seed=3):
    nx, ny, nz = n3
    g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=5, sigma=(0.0, 0.5))
    g.set_materials(eps, sig)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g.add_source(2, nx // 2, ny // 2, nz // 2, amp, f0, bw, t0, kind)
    g.add_probe(2, 3, 4, 5)
    for c in range(6):
        g.set_field(c, wl.random_fields(nx, ny, nz, seed + 1)[c])
    return g


def test_guards_intact_after_every_kernel(sophie):
    g = _grid()
    assert g.check_guards() == 0
    for prec in (so.FP32, so.FP16, so.BF16, so.FP16HL):
        for k in (1, 2, 3, 4):
            g.configure(temporal_k=k, precision=prec)
            g.step(2 * k + 1)
            assert g.check_guards() == 0, (prec, k)
    g.configure(temporal_k=1, tile_x=32, precision=so.FP32)
    g.step(5)
    g.configure(temporal_k=0, tile_x=0)
    g.step(6)
    g.objective_forward(23, 2, 20, 14, 11, 7)
    g.objective_grad_eps(5, 5, 5, 8, 6, 4)
    assert g.check_guards() == 0
    dims = [(17, 12, 9), (65, 20, 33), (3, 40, 5)]
    b = so.Batch(dims, DX, wl.cfl_dt(DX))
    b.set_materials(np.concatenate([wl.random_materials(*d, seed=c)[0].ravel() for c, d in enumerate(dims)]))
    for c in range(len(dims)):
        for comp in range(6):
            b.set_field(c, comp, wl.random_fields(*dims[c], seed=40 + c)[comp])
    for tx, ty in ((64, 16), (32, 4), (32, 8), (32, 16)):
        b.configure(tile_x=tx, tile_y=ty, zchunk=7)
        b.step(3)
        assert b.check_guards() == 0, (tx, ty)


def test_bounded_wait_times_out_and_grid_recovers(oracle_mod, sophie):
    nx, ny, nz = 24, 20, 18
    eps, sig = wl.random_materials(nx, ny, nz, 9, nmat=4)
    f = wl.random_fields(nx, ny, nz, 10)
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, f, temporal_k=2)
    g.step(4)
    o.step(4)
    waited = g.selftest_wait_timeout()
    assert 900.0 <= waited <= 5000.0  # the 1 s limit, not a hang
    with pytest.raises(so.SophieError) as e:
        g.sync()
    assert e.value.code == so.ETIMEOUT
    g.sync()  # reported once, then cleared
    g.step(7)
    o.step(7)
    assert_fields_equal(g, o)


def _free_mib():
    free, _ = torch.cuda.mem_get_info()
    return free / 2 ** 20


def test_allocation_failures_return_enomem_and_clean_up(sophie):
    torch.cuda.synchronize()
    before = _free_mib()
    failed = 0
    for n in range(1, 40):
        so.sophie_debug_fail_alloc(n)
        try:
            g = so.Grid(33, 21, 17, DX, wl.cfl_dt(DX))
        except so.SophieError as e:
            assert e.code == so.ENOMEM
            failed += 1
            continue
        finally:
            so.sophie_debug_fail_alloc(0)
        g.step(3)
        g.close()
        break
    assert failed >= 5  # every allocation of creation was exercised
    failed_b = 0
    for n in range(1, 40):
        so.sophie_debug_fail_alloc(n)
        try:
            b = so.Batch([(9, 8, 7), (12, 5, 6)], DX, wl.cfl_dt(DX))
        except so.SophieError as e:
            assert e.code == so.ENOMEM
            failed_b += 1
            continue
        finally:
            so.sophie_debug_fail_alloc(0)
        b.step(2)
        b.close()
        break
    assert failed_b >= 5
    g = _grid((30, 22, 18))
    so.sophie_debug_fail_alloc(1)  # the first checkpoint
    with pytest.raises(so.SophieError) as e:
        g.objective_forward(120, 2, 20, 11, 9, 10)
    assert e.value.code == so.ENOMEM
    so.sophie_debug_fail_alloc(0)
    g.objective_forward(40, 2, 20, 11, 9, 10)  # works again
    g.objective_grad_eps(5, 5, 5, 4, 4, 4)
    g.close()
    torch.cuda.synchronize()
    assert _free_mib() > before - 64  # nothing of significant size leaked


def test_double_destroy_and_oversized_grids(sophie):
    h = so.sophie_create_grid(8, 8, 8, DX, wl.cfl_dt(DX))
    so.sophie_destroy_grid(h)
    with pytest.raises(so.SophieError) as e:
        so.sophie_destroy_grid(h)
    assert e.value.code == so.EINVAL
    hb = so.sophie_batch_create([(4, 4, 4)], DX, wl.cfl_dt(DX))
    so.sophie_batch_destroy(hb)
    with pytest.raises(so.SophieError) as e:
        so.sophie_batch_destroy(hb)
    assert e.value.code == so.EINVAL
    with pytest.raises(so.SophieError) as e:
        so.Grid(1 << 21, 4, 4, DX, wl.cfl_dt(DX))
    assert e.value.code == so.EINVAL
    with pytest.raises(so.SophieError) as e:
        so.Grid(8192, 8192, 8192, DX, wl.cfl_dt(DX))
    assert e.value.code == so.ENOMEM
