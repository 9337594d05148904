"""Placement of a packed batch (sophie_batch_pack_plan, host only, no GPU).

Every cavity must lie inside the packed grid and be separated from every other
cavity by at least one cell (the conducting layer): the closed boxes
[o, o + n] (each cavity's cells plus the cell after it on every axis) of two
cavities never meet. Checked by rasterising the closed boxes (a count above one
marks an overlap), plus a pairwise check on small sets; the plan is
deterministic and fills the grid densely on the batching workload's sizes.
"""

import numpy as np
import pytest

from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    try:
        so.load()
    except Exception as e:  # the library is built by the session's build step
        pytest.skip(f"libsophie not built: {e}")


def _check(dims, org, ext):
    dims = np.asarray(dims, np.int64)
    assert np.all(org >= 0)
    assert np.all(org + dims <= ext[None, :]), "cavity outside the grid"
    occ = np.zeros((ext[2] + 1, ext[1] + 1, ext[0] + 1), np.uint8)
    for (nx, ny, nz), (x, y, z) in zip(dims, org):
        occ[z:z + nz + 1, y:y + ny + 1, x:x + nx + 1] += 1
    assert occ.max() == 1, "two cavities closer than one conducting cell"


def test_plan_small_sets_pairwise(lib):
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(1, 40))
        dims = rng.integers(1, 30, size=(n, 3))
        org, ext = so.sophie_batch_pack_plan(dims)
        _check(dims, org, ext)
        lo, hi = org, org + dims
        for a in range(n):
            for b in range(a + 1, n):
                sep = (hi[a] < lo[b]) | (hi[b] < lo[a])  # a gap of at least one cell on some axis
                assert sep.any(), (trial, a, b)


def test_plan_batching_workload(lib):
    dims, _, _ = wl.batch_cavities(ncav=512, seed=1304)
    org, ext = so.sophie_batch_pack_plan(dims)
    _check(dims, org, ext)
    eff = dims.prod(axis=1).sum() / float(np.prod(ext))
    assert eff > 0.7, eff
    org2, ext2 = so.sophie_batch_pack_plan(dims)
    assert np.array_equal(org, org2) and np.array_equal(ext, ext2)
    full, _, _ = wl.batch_cavities(ncav=4096, seed=1304)
    _, extf = so.sophie_batch_pack_plan(full)
    print("4096-cavity workload packed into", extf, "fill", full.prod(axis=1).sum() / float(np.prod(extf)))
    assert full.prod(axis=1).sum() / float(np.prod(extf)) > 0.75


def test_plan_errors(lib):
    with pytest.raises(so.SophieError):
        so.sophie_batch_pack_plan(np.array([[0, 4, 4]]))
    with pytest.raises(so.SophieError):
        so.sophie_batch_pack_plan(np.array([[5000, 4, 4]]))
