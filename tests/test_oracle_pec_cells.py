"""Pins of perfectly conducting cells (eps_r = +inf) in the oracle.

A PEC cell makes every edge it touches a PEC edge, like the outer walls
(Sec. 2.1 scheme with the wall condition of the paper's cavities). A layer of
PEC cells therefore splits a grid into cavities that evolve independently:
each one must follow its own closed-form discrete eigenmode, and equal, value
for value, a separate run of that cavity alone. This is how many cavities are
batched side by side.
"""

import math

import numpy as np

from modes import CavityMode, rel_l2

DX = 1e-3


def _embed(big_shape, sub, i_off):
    out = np.zeros(big_shape)
    nzp, nyp, nxp = sub.shape
    out[:nzp, :nyp, i_off:i_off + nxp] = sub
    return out


def test_pec_layer_splits_into_independent_eigenmode_cavities(oracle_mod):
    nx, ny, nz = 21, 12, 10
    wall = 9  # cells i = 9 are PEC: left cavity i in [0,9), right cavity i in [10,21)
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    left = CavityMode(9, ny, nz, 1, 1, 0, [0, 0, 1], S)
    right = CavityMode.transverse(11, ny, nz, 2, 1, 1, [0.3, -0.2, 1.0], S)
    eps = np.ones((nz, ny, nx), np.float32)
    eps[:, :, wall] = np.inf
    sig = np.zeros_like(eps)
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), "f64")
    g.set_materials(eps, sig)
    shape = (nz + 1, ny + 1, nx + 1)
    sl, sr = left.state(0), right.state(0)
    for c in range(6):
        g.set_field(c, _embed(shape, sl[c], 0) + _embed(shape, sr[c], wall + 1))
    solo = []
    for m, st in ((left, sl), (right, sr)):
        o = oracle_mod.OracleGrid(m.nx, m.ny, m.nz, DX, oracle_mod.cfl_dt(DX), "f64")
        for c in range(6):
            o.set_field(c, st[c])
        solo.append(o)
    W0 = g.energy()
    assert abs(W0 - (solo[0].energy() + solo[1].energy())) <= 1e-13 * W0
    N = 150
    g.step(N)
    for o in solo:
        o.step(N)
    for c in range(6):
        # the embedded cavities equal the separate runs exactly
        np.testing.assert_array_equal(g.f[c][:, :, :wall + 1], solo[0].f[c])
        np.testing.assert_array_equal(g.f[c][:, :, wall + 1:], solo[1].f[c])
    for m, o in zip((left, right), solo):
        ref = m.state(N)
        for c in range(6):
            if np.abs(ref[c]).max() > 0:
                assert rel_l2(o.f[c], ref[c]) < 1e-12
    assert abs(g.energy() - W0) <= 1e-12 * W0


def test_pec_cell_edges_have_zero_coefficients(oracle_mod):
    nx, ny, nz = 6, 5, 4
    eps = np.full((nz, ny, nx), 2.0, np.float32)
    eps[2, 1, 3] = np.inf
    sig = np.full_like(eps, 0.01)
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), "f64")
    g.set_materials(eps, sig)
    cax, cbx, cay, cby, caz, cbz = g.coef
    i, j, k = 3, 1, 2
    # the 12 edges of cell (3,1,2)
    for a in (0, 1):
        for b in (0, 1):
            assert cax[k + b, j + a, i] == 0 and cbx[k + b, j + a, i] == 0
            assert cay[k + b, j, i + a] == 0 and cby[k + b, j, i + a] == 0
            assert caz[k, j + b, i + a] == 0 and cbz[k, j + b, i + a] == 0
            assert g.eps_edge[0][k + b, j + a, i] == 0
    # an interior edge not touching it keeps the lossy coefficients
    beta = 0.01 * g.dt / (2 * oracle_mod.EPS0 * 2.0)
    S = oracle_mod.C0 * g.dt / DX
    assert math.isclose(cbx[1, 1, 1], (S / 2.0) / (1 + beta), rel_tol=1e-6)
    assert math.isclose(cax[1, 1, 1], (1 - beta) / (1 + beta), rel_tol=1e-6)
