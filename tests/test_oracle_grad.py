"""Pins of the oracle's reverse-mode gradient dJ/d eps_r (yee_oracle_grad.c).

J = dt * sum_{n=1..N} (probe value after step n)^2. The gradient is checked
against brute force: central finite differences of J, where each J comes from
the pinned forward oracle (OracleGrid.step with a probe), not from the code
under test. Cell perturbations are powers of two, exact in float32 for the
eps_r values used, so the difference quotient has an exact denominator.

The cases are chosen so that a plausible slip fails: a non-cubic grid with
random lossy materials (sigma large enough that the dCa/deps term matters),
random initial fields (every coupling active from step 0), a source on an edge
of listed cells (the source term of the stored bracket), every cell of the grid
listed (wall-adjacent cells with PEC edges included), and an H-component probe.
"""

import numpy as np
import pytest

from paper_1301_4539_gb300 import workloads as wl

DX = 1e-3


def _J_forward(oracle_mod, n3, eps, sig, fields, src, probe, nsteps):
    nx, ny, nz = n3
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), "f64")
    g.set_materials(eps, sig)
    for c in range(6):
        g.set_field(c, fields[c])
    if src is not None:
        g.add_source(*src)
    q = g.add_probe(*probe)
    g.step(nsteps)
    p = g.probe(q)
    return g.dt * float(np.sum(p * p)), g


def _grad(oracle_mod, n3, eps, sig, fields, src, probe, nsteps, cells):
    nx, ny, nz = n3
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), "f64")
    g.set_materials(eps, sig)
    for c in range(6):
        g.set_field(c, fields[c])
    if src is not None:
        g.add_source(*src)
    return g.grad_eps(*probe, nsteps, cells)


def _fd(oracle_mod, n3, eps, sig, fields, src, probe, nsteps, cells, h=2.0 ** -14):
    nx, ny, nz = n3
    out = []
    for (i, j, k) in cells:
        ep = eps.copy()
        em = eps.copy()
        ep[k, j, i] += np.float32(h)
        em[k, j, i] -= np.float32(h)
        assert float(ep[k, j, i]) - float(em[k, j, i]) == 2 * h
        jp, _ = _J_forward(oracle_mod, n3, ep, sig, fields, src, probe, nsteps)
        jm, _ = _J_forward(oracle_mod, n3, em, sig, fields, src, probe, nsteps)
        out.append((jp - jm) / (2 * h))
    return np.array(out)


def _case(seed, n3, sigma):
    nx, ny, nz = n3
    eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=6, eps=(1.0, 4.0), sigma=sigma)
    fields = [f.astype(np.float64) for f in wl.random_fields(nx, ny, nz, seed + 7)]
    return eps, sig, fields


@pytest.mark.parametrize("sigma", [(0.0, 0.0), (0.0, 6.0)])
def test_grad_matches_central_differences_all_cells(oracle_mod, sigma):
    n3 = (7, 6, 5)
    nx, ny, nz = n3
    eps, sig, fields = _case(11, n3, sigma)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source(f0=60e9, bw=40e9)
    src = (1, 3, 2, 2, amp, f0, bw, t0, kind)
    probe = (2, 4, 3, 2)
    cells = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    nsteps = 24
    J, g = _grad(oracle_mod, n3, eps, sig, fields, src, probe, nsteps, cells)
    J0, _ = _J_forward(oracle_mod, n3, eps, sig, fields, src, probe, nsteps)
    assert abs(J - J0) <= 1e-13 * abs(J0)
    fd = _fd(oracle_mod, n3, eps, sig, fields, src, probe, nsteps, cells)
    scale = np.max(np.abs(fd))
    assert scale > 0
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * scale + 1e-6 * np.abs(fd)), (np.max(err) / scale)
    # every cell matters here: a dropped edge would show
    assert np.count_nonzero(np.abs(fd) > 1e-3 * scale) > 0.8 * len(cells)


def test_grad_h_probe_and_source_edge_cells(oracle_mod):
    n3 = (6, 7, 6)
    eps, sig, fields = _case(23, n3, (0.0, 10.0))
    amp, f0, bw, t0, kind = wl.gaussian_pulse_source(bw=50e9)
    src = (0, 2, 3, 3, amp * 3.0, f0, bw, t0, kind)
    probe = (4, 3, 3, 2)  # hy face
    # the four cells around the source edge ex(2,3,3), plus two others
    cells = [(2, 2, 2), (2, 3, 2), (2, 2, 3), (2, 3, 3), (0, 0, 0), (5, 6, 5)]
    J, g = _grad(oracle_mod, n3, eps, sig, fields, src, probe, 20, cells)
    fd = _fd(oracle_mod, n3, eps, sig, fields, src, probe, 20, cells)
    scale = np.max(np.abs(fd))
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * scale)


def test_grad_zero_outside_domain_of_influence(oracle_mod):
    """From zero fields, a cell whose edges the source cannot reach and whose
    perturbation cannot reach the probe within N steps has exactly zero gradient:
    the Yee stencil moves information one cell per half step at most."""
    n3 = (24, 6, 6)
    nx, ny, nz = n3
    eps, sig = wl.random_materials(nx, ny, nz, 5, nmat=4, eps=(1.0, 4.0), sigma=(0.0, 1.0))
    zero = [np.zeros((nz + 1, ny + 1, nx + 1)) for _ in range(6)]
    amp, f0, bw, t0, kind = wl.gaussian_pulse_source(bw=80e9)
    src = (2, 3, 3, 2, amp, f0, bw, t0, kind)
    probe = (2, 4, 3, 2)
    N = 6
    far = [(20, 2, 2), (23, 5, 5), (17, 3, 3)]
    near = [(3, 2, 2), (4, 3, 1)]
    _, g = _grad(oracle_mod, n3, eps, sig, zero, src, probe, N, far + near)
    assert np.all(g[:3] == 0.0)
    assert np.all(g[3:] != 0.0)
    fd = _fd(oracle_mod, n3, eps, sig, zero, src, probe, N, near)
    np.testing.assert_allclose(g[3:], fd, rtol=1e-6)


def test_design_workload_generator():
    w = wl.design_cavity(n=32, design=(12, 20), ncells=16)
    lo = 12
    assert w["eps"].shape == (32, 32, 32)
    d = w["eps"][12:20, 12:20, 12:20]
    assert d.min() >= 1.0 and d.max() <= 4.0 and d.std() > 0.3
    e = w["eps"].copy()
    e[12:20, 12:20, 12:20] = 1.0
    assert np.all(e == 1.0) and np.all(w["sigma"] == 0)
    assert len(set(w["cells"])) == 16
    assert all(lo <= c < 20 for cell in w["cells"] for c in cell)
    assert w["probe"] == (2, 23, 16, 16) and w["sources"][0][:4] == (2, 8, 16, 16)
    assert w["sources"][0][8] == 1
