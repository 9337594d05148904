"""Pins of the oracle against identities the scheme fixes (Sec. 2.1-2.2).

* Energy balance: with W^n = 1/2 eps0 dV [sum eps_r e^2 + sum h^{n-1/2} h^{n+1/2}],
    W^{n+1} - W^n = -(dt dV / 4) sum_edges sigma (e^{n+1}+e^n)^2
                    + 1/2 eps0 dV S (e_s^{n+1}+e_s^n) s^{n+1/2}
  exactly, because the two discrete curls are mutual adjoints (the discrete
  antisymmetry the paper requires for stability, Sec. 2.1).
* Node divergence of eps_r e is invariant without loss and sources.
* Antisymmetry itself: <h, A e> = -<e, B h> with A the H-update curl and B
  the E-update curl.
* Edge material = mean of the four cells sharing the edge (2x2 box filter).
* Source waveform: the envelope's amplitude spectrum has the stated FWHM and
  the modulated spectrum peaks at f0.
"""

import math

import numpy as np
import pytest

from modes import rel_l2
from paper_1301_4539_gb300 import workloads as wl

DX = 1e-3


def _grid(oracle_mod, n3, prec="f64", seed=3, lossy=True, nmat=4):
    nx, ny, nz = n3
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), prec)
    eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=nmat,
                                   sigma=(0.0, 0.5) if lossy else (0.0, 0.0))
    g.set_materials(eps, sig)
    f = wl.random_fields(nx, ny, nz, seed + 100)
    for c in range(6):
        g.set_field(c, f[c].astype(g.dtype))
    return g, eps, sig


def _sigma_edges(sig, nx, ny, nz):
    """Mean sigma per interior edge via a 2x2 box filter over the transverse axes."""
    s = sig.astype(np.float64)
    out = [np.zeros((nz + 1, ny + 1, nx + 1)) for _ in range(3)]
    # ex(i,j,k), j in [1,ny), k in [1,nz): cells (i, j-1..j, k-1..k)
    out[0][1:nz, 1:ny, 0:nx] = 0.25 * (s[:-1, :-1, :] + s[:-1, 1:, :] + s[1:, :-1, :] + s[1:, 1:, :])
    out[1][1:nz, 0:ny, 1:nx] = 0.25 * (s[:-1, :, :-1] + s[:-1, :, 1:] + s[1:, :, :-1] + s[1:, :, 1:])
    out[2][0:nz, 1:ny, 1:nx] = 0.25 * (s[:, :-1, :-1] + s[:, :-1, 1:] + s[:, 1:, :-1] + s[:, 1:, 1:])
    return out


def test_edge_average_is_box_filter(oracle_mod):
    from scipy.ndimage import uniform_filter
    nx, ny, nz = 7, 6, 5
    g, eps, _ = _grid(oracle_mod, (nx, ny, nz))
    e = eps.astype(np.float64)
    # ex edges average over (k, j) 2x2 windows at fixed i
    box_yz = uniform_filter(e, size=(2, 2, 1), origin=(0, 0, 0), mode="constant")
    # uniform_filter with size 2 centres the window on [idx-1, idx]
    np.testing.assert_allclose(g.eps_edge[0][1:nz, 1:ny, 0:nx], box_yz[1:nz, 1:ny, :], rtol=1e-15)
    box_xz = uniform_filter(e, size=(2, 1, 2), mode="constant")
    np.testing.assert_allclose(g.eps_edge[1][1:nz, 0:ny, 1:nx], box_xz[1:nz, :, 1:nx], rtol=1e-15)
    box_xy = uniform_filter(e, size=(1, 2, 2), mode="constant")
    np.testing.assert_allclose(g.eps_edge[2][0:nz, 1:ny, 1:nx], box_xy[:, 1:ny, 1:nx], rtol=1e-15)
    # walls carry no coefficients (PEC)
    assert g.coef[0][0].max() == 0 and g.coef[2][:, :, 0].max() == 0 and g.coef[5][:, 0, :].max() == 0


@pytest.mark.parametrize("n3", [(9, 8, 7), (5, 6, 7)])
def test_energy_balance_lossy_with_source(oracle_mod, n3):
    nx, ny, nz = n3
    g, eps, sig = _grid(oracle_mod, n3)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    si, sj, sk = nx // 2, ny // 2, nz // 2
    g.add_source(2, si, sj, sk, 50.0, f0, bw, 20 * g.dt, kind)
    sig_e = _sigma_edges(sig, nx, ny, nz)
    dV = DX ** 3
    S = float(g.S)
    sval = oracle_mod.waveform(kind, 50.0, f0, bw, 20 * g.dt, g.dt, 0, 60)
    worst = 0.0
    W = g.energy()
    for n in range(60):
        e_old = [g.f[c].copy() for c in range(3)]
        g.step(1)
        W1 = g.energy()
        loss = sum(float((sig_e[c] * (g.f[c] + e_old[c]) ** 2).sum()) for c in range(3))
        src = 0.5 * oracle_mod.EPS0 * dV * S * float(g.f[2][sk, sj, si] + e_old[2][sk, sj, si]) * sval[n]
        pred = W - (g.dt * dV / 4.0) * loss + src
        worst = max(worst, abs(W1 - pred) / W)
        W = W1
    assert worst < 1e-12, worst


def test_energy_constant_lossless(oracle_mod):
    g, _, _ = _grid(oracle_mod, (10, 9, 8), lossy=False)
    W0 = g.energy()
    g.step(100)
    assert abs(g.energy() - W0) / W0 < 1e-12


def _node_div(g, eps_e):
    nx, ny, nz = g.nx, g.ny, g.nz
    ex, ey, ez = [g.f[c].astype(np.float64) * eps_e[c] for c in range(3)]
    # interior nodes i in [1,nx-1], j in [1,ny-1], k in [1,nz-1]
    d = (ex[1:nz, 1:ny, 1:nx] - ex[1:nz, 1:ny, 0:nx - 1]
         + ey[1:nz, 1:ny, 1:nx] - ey[1:nz, 0:ny - 1, 1:nx]
         + ez[1:nz, 1:ny, 1:nx] - ez[0:nz - 1, 1:ny, 1:nx])
    return d


def test_divergence_invariant(oracle_mod):
    g, _, _ = _grid(oracle_mod, (9, 10, 8), lossy=False)
    d0 = _node_div(g, g.eps_edge)
    g.step(50)
    d1 = _node_div(g, g.eps_edge)
    scale = np.abs(d0).max()
    assert np.abs(d1 - d0).max() < 1e-12 * max(scale, 1.0) * 10


def test_divergence_source_changes_only_its_two_nodes(oracle_mod):
    nx, ny, nz = 9, 9, 9
    g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), "f64")
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    g.add_source(2, 4, 5, 3, 1.0, f0, bw, 10 * g.dt, kind)
    g.step(40)
    d = _node_div(g, g.eps_edge)
    nz_idx = np.argwhere(np.abs(d) > 1e-12)
    # interior node (i,j,k) maps to d[k-1, j-1, i-1]; the edge ez(4,5,3) joins nodes k=3 and k=4
    got = sorted(tuple(int(v) for v in x) for x in nz_idx)
    assert got == [(2, 4, 3), (3, 4, 3)], got


def test_curls_are_antisymmetric(oracle_mod):
    nx, ny, nz = 7, 6, 8
    dt = oracle_mod.cfl_dt(DX)
    S = oracle_mod.C0 * dt / DX
    fr = wl.random_fields(nx, ny, nz, 11)
    # run 1: e random, h = 0 -> after one step, h = S A e
    g1 = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f64")
    for c in range(3):
        g1.set_field(c, fr[c])
    g1.step(1)
    Ae = [g1.f[3 + c] / S for c in range(3)]
    # run 2: e = 0, h random -> after one step, e = S B h (vacuum: Ca = 1, Cb = S)
    g2 = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f64")
    for c in range(3):
        g2.set_field(3 + c, fr[3 + c])
    g2.step(1)
    Bh = [g2.f[c] / S for c in range(3)]
    lhs = sum(float((fr[3 + c].astype(np.float64) * Ae[c]).sum()) for c in range(3))
    rhs = -sum(float((fr[c].astype(np.float64) * Bh[c]).sum()) for c in range(3))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)
    assert abs(lhs) > 1.0


def test_waveform_bandwidth_and_centre(oracle_mod):
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    dt = 1e-12
    n = 1 << 15
    env = oracle_mod.waveform(1, 1.0, f0, bw, t0 + 8000 * dt, dt, 0, n)
    spec = np.abs(np.fft.rfft(env))
    freqs = np.fft.rfftfreq(n, dt)
    half = spec.max() / 2
    b = int(np.nonzero(spec >= half)[0].max())  # last bin above half maximum
    fc = freqs[b] + (spec[b] - half) / (spec[b] - spec[b + 1]) * (freqs[b + 1] - freqs[b])
    fwhm = 2 * fc  # the envelope's spectrum is centred at 0
    assert abs(fwhm - bw) / bw < 2e-3
    mod = oracle_mod.waveform(0, 1.0, f0, bw, t0 + 8000 * dt, dt, 0, n)
    spec_m = np.abs(np.fft.rfft(mod))
    assert abs(freqs[int(np.argmax(spec_m))] - f0) / f0 < 2e-3
    # closed-form values at the pulse centre and one period later (kind 0 crosses zero)
    v = oracle_mod.waveform(1, 2.0, f0, bw, 0.5 * dt, dt, 0, 1)
    assert v[0] == 2.0


def test_fp32_tracks_fp64(oracle_mod):
    nx, ny, nz = 24, 20, 16
    eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=6, seed=5, radius=(2, 6))
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    gs = []
    for prec in ("f64", "f32"):
        g = oracle_mod.OracleGrid(nx, ny, nz, DX, oracle_mod.cfl_dt(DX), prec)
        g.set_materials(eps, sig)
        g.add_source(2, nx // 2, ny // 2, nz // 2, amp, f0, bw, t0, kind)
        g.add_probe(2, 5, 7, 9)
        g.step(300)
        gs.append(g)
    errs = [rel_l2(gs[1].f[c], gs[0].f[c]) for c in range(6)]
    assert max(errs) < 1e-5, errs
    assert rel_l2(gs[1].probe(0), gs[0].probe(0)) < 1e-5
