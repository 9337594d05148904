"""Pins of the oracle against exact discrete cavity modes (Sec. 2.1 scheme).

The closed forms live in tests/modes.py and are derived from the scheme on
paper, not from any implementation. A dropped term, a wrong sign or a wrong
index in any of the six update loops changes the mode and fails here.
"""

import math

import numpy as np
import pytest

from modes import CavityMode, lossy_mode_amplitudes, rel_l2


DX = 1e-3


def _run(oracle_mod, prec, mode, nsteps, eps=None, sig=None):
    nx, ny, nz = mode.nx, mode.ny, mode.nz
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), prec)
    if eps is not None:
        g.set_materials(eps, sig)
    st = mode.state(0)
    for c in range(6):
        g.set_field(c, st[c])
    return g


def test_tm110_32_dispersion_numbers(oracle_mod):
    """32^3 at 0.99 CFL: sin(w dt/2) and w dt of the TM110 mode."""
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    m = CavityMode(32, 32, 32, 1, 1, 0, [0, 0, 1], S)
    # sin^2(w dt/2)/(c dt)^2 = sum sin^2(k dx/2)/dx^2 with k = pi/(32 dx)
    lhs = m.half ** 2 / (S * DX) ** 2
    rhs = 2 * math.sin(math.pi / 64) ** 2 / DX ** 2
    assert abs(lhs - rhs) / rhs < 1e-14
    assert abs(m.half - 0.039662952) < 5e-9
    assert abs(m.wdt - 0.079346718) < 5e-9


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_tm110_cavity_200_steps(oracle_mod, prec, tol):
    """TM110 in a 32^3 PEC vacuum cavity, amplitude 1, 200 steps."""
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    m = CavityMode(32, 32, 32, 1, 1, 0, [0, 0, 1], S)
    g = _run(oracle_mod, prec, m, 200)
    W0 = g.energy()
    Wmax = 0.0
    for _ in range(20):
        g.step(10)
        Wmax = max(Wmax, abs(g.energy() - W0) / W0)
    ref = m.state(200)
    errs = [rel_l2(g.f[c], ref[c]) for c in (2, 3, 4)]
    assert max(errs) < tol, errs
    for c in (0, 1, 5):
        assert np.abs(g.f[c]).max() == 0.0
    assert Wmax < (1e-12 if prec == "f64" else 1e-6), Wmax
    assert abs(math.cos(200 * m.wdt) - (-0.98700642)) < 1e-7


def test_tm110_probe_frequency(oracle_mod):
    """The Ez trace at an interior edge oscillates at the discrete w to 1e-6."""
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    m = CavityMode(32, 32, 32, 1, 1, 0, [0, 0, 1], S)
    g = _run(oracle_mod, "f64", m, 0)
    q = g.add_probe(2, 9, 13, 5)
    g.step(400)
    tr = g.probe(q)
    amp0 = math.sin(m.kx * 9) * math.sin(m.ky * 13)
    n = np.arange(1, 401)
    # fit w by least squares on cos(w n): scan a fine grid then refine
    ws = np.linspace(m.wdt * 0.99, m.wdt * 1.01, 2001)
    res = [np.sum((tr - amp0 * np.cos(w * n)) ** 2) for w in ws]
    w0 = ws[int(np.argmin(res))]
    ws = np.linspace(w0 - 2e-5 * w0, w0 + 2e-5 * w0, 2001)
    res = [np.sum((tr - amp0 * np.cos(w * n)) ** 2) for w in ws]
    wfit = ws[int(np.argmin(res))]
    assert abs(wfit - m.wdt) / m.wdt < 1e-6


@pytest.mark.parametrize("mnp,vec,dims,transverse", [
    ((1, 2, 1), (0.3, -0.7, 0.2), (12, 10, 14), True),
    ((2, 1, 3), (1.0, 0.5, -0.25), (9, 11, 13), True),
    ((0, 1, 1), (1.0, 0.0, 0.0), (8, 12, 10), False),   # Ex-polarised, axis-permuted TM110
    ((1, 0, 1), (0.0, 1.0, 0.0), (10, 8, 12), False),   # Ey-polarised
])
def test_general_modes_f64(oracle_mod, mnp, vec, dims, transverse):
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    nx, ny, nz = dims
    if transverse:
        m = CavityMode.transverse(nx, ny, nz, *mnp, vec, S)
    else:
        m = CavityMode(nx, ny, nz, *mnp, vec, S)
    g = _run(oracle_mod, "f64", m, 0)
    g.step(150)
    ref = m.state(150)
    nonzero = 0
    for c in range(6):
        if np.abs(ref[c]).max() > 1e-12:
            nonzero += 1
            assert rel_l2(g.f[c], ref[c]) < 1e-11, c
        else:
            assert np.abs(g.f[c]).max() < 1e-12, c
    assert nonzero >= 3


def test_uniform_dielectric_mode(oracle_mod):
    """eps_r = 4 everywhere: dispersion sin^2(w dt/2) = S^2|sig|^2/(4 eps_r), so Cb = S/eps_r."""
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    nx, ny, nz = 10, 12, 8
    m = CavityMode.transverse(nx, ny, nz, 1, 1, 1, (0.2, 0.9, -0.4), S, eps_r=4.0)
    eps = np.full((nz, ny, nx), 4.0, np.float32)
    sig = np.zeros((nz, ny, nx), np.float32)
    g = _run(oracle_mod, "f64", m, 0, eps, sig)
    g.step(120)
    ref = m.state(120)
    assert max(rel_l2(g.f[c], ref[c]) for c in range(6)) < 1e-11


def test_lossy_mode_recurrence(oracle_mod):
    """Uniform eps_r, sigma > 0: e^n = a_n E with the scalar recurrence of modes.py.

    Pins Ca = (1-beta)/(1+beta), Cb = (S/eps_r)/(1+beta), beta = sigma dt/(2 eps0 eps_r).
    """
    S = oracle_mod.C0 * oracle_mod.cfl_dt(DX) / DX
    nx, ny, nz = 10, 9, 11
    er, sg = 2.5, 0.8
    dt = oracle_mod.cfl_dt(DX)
    m = CavityMode.transverse(nx, ny, nz, 1, 2, 1, (0.5, -0.1, 0.7), S, eps_r=er)
    eps = np.full((nz, ny, nx), er, np.float32)
    sig = np.full((nz, ny, nx), sg, np.float32)
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f64")
    g.set_materials(eps, sig)
    es = m.e_shapes()
    for c in range(3):
        g.set_field(c, m.E[c] * es[c])
    beta = float(np.float32(sg)) * dt / (2 * oracle_mod.EPS0 * float(np.float32(er)))
    q = S * S * float(m.sig @ m.sig) / float(np.float32(er))
    a = lossy_mode_amplitudes(q, beta, 80)
    g.step(80)
    ref = [a[80] * m.E[c] * es[c] for c in range(3)]
    for c in range(3):
        if np.abs(ref[c]).max() > 0:
            assert rel_l2(g.f[c], ref[c]) < 1e-11
    assert a[80] ** 2 < 0.9  # the mode really decays
