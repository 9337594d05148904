"""Autotuner: trial launches leave the state untouched, the choice is a valid
configuration, and stepping with it gives the fields of the plain kernel
bitwise (float storage)."""

import numpy as np
import pytest

from gpu_helpers import DX
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n3", [(40, 36, 28), (96, 80, 72), (13, 9, 7)])
def test_autotune_keeps_state_and_results(sophie, n3):
    nx, ny, nz = n3
    eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=6, seed=1301, radius=(2, 6))
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    src = (2, nx // 2, ny // 2, nz // 2, amp, f0, bw, t0, kind)
    prb = (2, nx // 3, ny // 3, nz // 3)
    grids = []
    for tk in (1, 0):
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.configure(temporal_k=tk)
        g.set_materials(eps, sig)
        g.add_source(*src)
        g.add_probe(*prb)
        g.step(9)
        grids.append(g)
    plain, tuned = grids
    before = tuned.fields()
    k, ms = tuned.autotune()
    assert 1 <= k <= 4 and ms > 0
    assert tuned.n == 9
    for c in range(6):
        np.testing.assert_array_equal(tuned.get_field(c), before[c])
    np.testing.assert_array_equal(tuned.read_probe(0), plain.read_probe(0))
    plain.step(23)
    tuned.step(23)
    for c in range(6):
        np.testing.assert_array_equal(tuned.get_field(c), plain.get_field(c))
    np.testing.assert_array_equal(tuned.read_probe(0), plain.read_probe(0))


def test_autotune_half_storage_keeps_k2(sophie):
    g = so.Grid(48, 40, 32, DX, wl.cfl_dt(DX))
    g.configure(temporal_k=0, precision=so.FP16)
    k, ms = g.autotune()
    assert k == 2 and ms > 0


@pytest.mark.parametrize("tk", [0, 1, 2, 3])
def test_launch_config_reports_the_tuned_choice(sophie, tk):
    """sophie_launch_config: the k in use and a valid split for it, before the
    first step (the cost model's) and after it (the measured choice)."""
    g = so.Grid(96, 80, 72, DX, wl.cfl_dt(DX))
    g.configure(temporal_k=tk)
    for when in ("model", "tuned"):
        cfg = g.launch_config()
        assert cfg["plain_zchunk"] >= 1 and cfg["plain_ctas"] >= 1
        if tk:
            assert cfg["k"] == tk
        if cfg["k"] >= 2:
            assert cfg["blocked_ctas"] >= 1 and cfg["blocked_rows"] in (2, 4)
            assert cfg["blocked_zsplit"] >= 0 and cfg["blocked_order"] in (0, 1)
        else:
            assert cfg["blocked_ctas"] == cfg["blocked_zsplit"] == cfg["blocked_rows"] == 0
        if when == "model":
            g.step(max(tk, 1))
    if tk == 0:
        k, _ = g.autotune()
        assert g.launch_config()["k"] == k
