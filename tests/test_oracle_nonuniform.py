"""Pins of the oracle's non-uniform mesh (1-D width arrays per axis).

* All widths equal to dx: the non-uniform expressions reduce to the uniform
  ones exactly (ratios 1), so the fields and the energy must equal the
  uniform oracle's bit for bit, in double and in float.
* Uniform refinement: widths dx/2 everywhere is a uniform grid of step dx/2;
  a TM110 mode follows the closed form of that grid (S' = 2 S).
* Graded mesh: the volume-weighted discrete energy is conserved without loss
  or source (the weighted brackets stay mutual negative transposes).
* Brute force on 4x4x4 with random widths on every axis: every value computed
  point by point (doubled coordinates, exact FMA emulation) equals the
  oracle's bit for bit; this pins which width (primary or dual, which axis)
  scales which difference.
"""

import numpy as np
import pytest

from modes import CavityMode, rel_l2
from paper_1301_4539_gb300 import workloads as wl
from test_oracle_bruteforce import Box, e_dir, edge_coefficients, fma, h_dir, on_wall, positions, shift

DX = 1e-3


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unit_ratios_equal_uniform_bitwise(oracle_mod, prec):
    nx, ny, nz = 11, 9, 8
    eps, sig = wl.random_materials(nx, ny, nz, 5, nmat=4, sigma=(0.0, 2.0))
    f = wl.random_fields(nx, ny, nz, 6)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    src = (2, 5, 4, 3, 3.0, f0, bw, t0, kind)
    grids = []
    for nonuni in (False, True):
        o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), prec)
        o.set_materials(eps, sig)
        for c in range(6):
            o.set_field(c, f[c].astype(o.dtype))
        o.add_source(*src)
        q = o.add_probe(2, 3, 3, 3)
        if nonuni:
            o.set_spacing(np.full(nx, DX), np.full(ny, DX), np.full(nz, DX))
        o.step(17)
        grids.append(o)
    for c in range(6):
        np.testing.assert_array_equal(grids[0].f[c], grids[1].f[c])
    np.testing.assert_array_equal(grids[0].probe(q), grids[1].probe(q))
    assert grids[0].energy() == grids[1].energy()  # same terms, unit weights, same order


def test_uniform_refinement_follows_the_closed_form(oracle_mod):
    n = 24
    dt = wl.cfl_dt(DX / 2)  # stable for the refined step
    S_half = oracle_mod.C0 * dt / (DX / 2)
    m = CavityMode(n, n, n, 1, 1, 0, [0, 0, 1], S_half)
    o = oracle_mod.OracleGrid(n, n, n, DX, dt, "f64")
    o.set_spacing(np.full(n, DX / 2), np.full(n, DX / 2), np.full(n, DX / 2))
    st = m.state(0)
    for c in range(6):
        o.set_field(c, st[c])
    o.step(120)
    ref = m.state(120)
    for c in (2, 3, 4):
        assert rel_l2(o.f[c], ref[c]) < 1e-12


def test_graded_mesh_conserves_energy(oracle_mod):
    nx, ny, nz = 14, 12, 10
    rng = np.random.default_rng(7)
    wx = DX * rng.uniform(0.6, 1.5, nx)
    wy = DX * rng.uniform(0.6, 1.5, ny)
    wz = DX * rng.uniform(0.6, 1.5, nz)
    wmin = min(wx.min(), wy.min(), wz.min())
    dt = 0.95 / (oracle_mod.C0 * np.sqrt(1 / wx.min() ** 2 + 1 / wy.min() ** 2 + 1 / wz.min() ** 2))
    assert dt < wmin / oracle_mod.C0
    eps, _ = wl.random_materials(nx, ny, nz, 8, nmat=4, eps=(1.0, 5.0))
    o = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f64")
    o.set_materials(eps, np.zeros_like(eps))
    o.set_spacing(wx, wy, wz)
    f = wl.random_fields(nx, ny, nz, 9)
    for c in range(6):
        o.set_field(c, f[c].astype(np.float64))
    W0 = o.energy()
    drift = 0.0
    for _ in range(10):
        o.step(20)
        drift = max(drift, abs(o.energy() - W0) / W0)
    assert drift < 1e-12, drift
    # without the volume weights the same run does not conserve: the weights matter
    o.set_spacing()
    Wu0 = o.energy()
    o.set_spacing(wx, wy, wz)
    o.step(20)
    o.set_spacing()
    assert abs(o.energy() - Wu0) / Wu0 > 1e-6


def _brute_nu(n, eps, sig, fields, src, svals, nsteps, r):
    """The brute force of test_oracle_bruteforce with width ratios: r = (rx, ry, rz, rxd, ryd, rzd)."""
    dt = wl.cfl_dt(DX)
    S = 299792458.0 * dt / DX
    prim, dual = r[:3], r[3:]
    E, H = Box(n), Box(n)
    for p in positions(n, "e"):
        i, j, k = (v // 2 for v in p)
        E.v[p] = float(fields[e_dir(p)][k, j, i])
    for p in positions(n, "h"):
        i, j, k = (v // 2 for v in p)
        H.v[p] = float(fields[3 + h_dir(p)][k, j, i])
    coef = {p: edge_coefficients(p, eps, sig, dt, S) for p in positions(n, "e") if not on_wall(p, n)}
    sc, si, sj, sk = src
    src_pos = tuple(2 * v + (1 if a == sc else 0) for a, v in enumerate((si, sj, sk)))

    def ratio(kind, axis, p):
        # primary: the width of the cell the face spans along `axis` (odd coordinate);
        # dual: the dual width at the node the edge sits on along `axis` (even coordinate)
        idx = p[axis] // 2
        return float(prim[axis][idx]) if kind == "p" else float(dual[axis][idx])

    for m in range(nsteps):
        newH = {}
        for p in positions(n, "h"):
            c = h_dir(p)
            a1, a2 = (c + 1) % 3, (c + 2) % 3
            pa, ma = shift(p, a2, 1), shift(p, a2, -1)
            pb, mb = shift(p, a1, 1), shift(p, a1, -1)
            ea1 = E.get(pa) if E.inside(pa) and e_dir(pa) == a1 else 0.0
            ea0 = E.get(ma) if E.inside(ma) and e_dir(ma) == a1 else 0.0
            eb1 = E.get(pb) if E.inside(pb) and e_dir(pb) == a2 else 0.0
            eb0 = E.get(mb) if E.inside(mb) and e_dir(mb) == a2 else 0.0
            br = fma(ratio("p", a2, p), ea1 - ea0, -(ratio("p", a1, p) * (eb1 - eb0)))
            newH[p] = fma(S, br, H.get(p))
        H.v = newH
        newE = dict(E.v)
        for p, (ca, cb) in coef.items():
            c = e_dir(p)
            a1, a2 = (c + 1) % 3, (c + 2) % 3
            pa, ma = shift(p, a1, 1), shift(p, a1, -1)
            pb, mb = shift(p, a2, 1), shift(p, a2, -1)
            ha1 = H.get(pa) if h_dir(pa) == a2 else 0.0
            ha0 = H.get(ma) if h_dir(ma) == a2 else 0.0
            hb1 = H.get(pb) if h_dir(pb) == a1 else 0.0
            hb0 = H.get(mb) if h_dir(mb) == a1 else 0.0
            br = fma(ratio("d", a1, p), ha1 - ha0, -(ratio("d", a2, p) * (hb1 - hb0)))
            if p == src_pos:
                br = br + svals[m]
            newE[p] = fma(cb, br, ca * E.get(p))
        E.v = newE
    out = [np.zeros((n[2] + 1, n[1] + 1, n[0] + 1)) for _ in range(6)]
    for p, v in E.v.items():
        i, j, k = (q // 2 for q in p)
        out[e_dir(p)][k, j, i] = v
    for p, v in H.v.items():
        i, j, k = (q // 2 for q in p)
        out[3 + h_dir(p)][k, j, i] = v
    return out


def test_bruteforce_graded_4cubed(oracle_mod):
    n = (4, 4, 4)
    rng = np.random.default_rng(44)
    eps, sig = wl.random_materials(*n, seed=414, nmat=4, eps=(1.0, 6.0), sigma=(0.0, 20.0))
    fields = [f.astype(np.float64) for f in wl.random_fields(*n, seed=415)]
    amp, f0, bw, t0, kind = wl.gaussian_sine_source(f0=80e9, bw=60e9)
    src = (0, 1, 2, 2)
    o = oracle_mod.OracleGrid(*n, DX, wl.cfl_dt(DX), "f64")
    o.set_materials(eps, sig)
    o.set_spacing(*(DX * rng.uniform(1.0, 2.0, 4) for _ in range(3)))
    for c in range(6):
        o.set_field(c, fields[c])
    o.add_source(*src, 5.0, f0, bw, t0, kind)
    svals = oracle_mod.waveform(kind, 5.0, f0, bw, t0, o.dt, 0, 3)
    ratios = o.ratios
    o.step(3)
    ref = _brute_nu(n, eps, sig, fields, src, svals, 3, ratios)
    for c in range(6):
        np.testing.assert_array_equal(o.f[c], ref[c], err_msg=f"component {c}")
