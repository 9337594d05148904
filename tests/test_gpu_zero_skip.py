"""Zero-field skipping (early-time sparsity): with it on, the step kernels skip
work units outside the box known to hold every nonzero value; fields, probe
samples and energies must be bitwise those of the oracle and of a run without
skipping, while the box is small, while it grows, after the caller writes
fields (skipping then covers the whole grid) and after a reset."""

import numpy as np
import pytest

from gpu_helpers import DX, assert_fields_equal, make_pair
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [0, 1, 2, 3, 8])
def test_skip_matches_oracle_while_the_box_grows(oracle_mod, sophie, K):
    """K = 0: autotuned, so the first step runs the tuner's trial launches
    (which write the spare buffer everywhere) with skipping already on."""
    nx, ny, nz = 150, 70, 60
    eps, sig = wl.random_materials(nx, ny, nz, seed=K + 1, nmat=5, sigma=(0.0, 0.3))
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, 12, 10, 8, 9.0, f0, bw, 0.0, kind)]  # strong from the first step
    prbs = [(2, 14, 10, 8), (2, 140, 60, 50), (0, 60, 30, 30), (4, 30, 10, 8)]
    g, o = make_pair(oracle_mod, nx, ny, nz, eps, sig, None, srcs, prbs, temporal_k=K)
    g.set_zero_skip(True)
    plain = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    plain.configure(temporal_k=1)
    plain.set_materials(eps, sig)
    plain.add_source(*srcs[0])
    done = 0
    for n in (2, 7, 24, 60, 130):
        g.step(n - done)
        o.step(n - done)
        plain.step(n - done)
        done = n
        assert_fields_equal(g, o)
        for c in range(6):
            np.testing.assert_array_equal(g.get_field(c), plain.get_field(c))
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    assert abs(g.energy() - o.energy()) <= 1e-12 * abs(o.energy())


def test_skip_with_caller_fields_and_after_reset(oracle_mod, sophie):
    nx, ny, nz = 80, 40, 30
    f = wl.random_fields(nx, ny, nz, 2)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    src = (2, 70, 30, 20, 5.0, f0, bw, 0.0, kind)
    g, o = make_pair(oracle_mod, nx, ny, nz, fields=f, sources=[src], temporal_k=2)
    g.set_zero_skip(True)
    g.step(9)
    o.step(9)
    assert_fields_equal(g, o)  # caller's fields: the whole grid is computed
    g.reset()
    o2 = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f32")
    o2.add_source(*src)
    g.step(15)
    o2.step(15)
    assert_fields_equal(g, o2)  # after the reset only the source's neighbourhood is live


def test_no_sources_no_work(sophie):
    g = so.Grid(64, 48, 40, DX, wl.cfl_dt(DX))
    g.set_zero_skip(True)
    g.step(10)
    for c in range(6):
        assert not g.get_field(c).any()
    assert g.energy() == 0.0
