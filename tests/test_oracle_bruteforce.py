"""Brute-force pin of the oracle: steps on a 4x4x4 grid computed point by
point in plain Python and compared exactly (FP64) with the oracle.

The brute force is an independent formulation of the Sec. 2.1 leapfrog:
every field value lives at a position in doubled integer coordinates (an E
edge has exactly one odd coordinate, along its direction; an H face exactly
two, the even one is its normal), values outside the box are zero, and the
curls are taken from the axis structure,

    h_c += S * [ (E_{c+1}(p + e_{c+2}) - E_{c+1}(p - e_{c+2}))
               - (E_{c+2}(p + e_{c+1}) - E_{c+2}(p - e_{c+1})) ]
    e_c  = Ca*e_c + Cb * [ (H_{c+2}(p + e_{c+1}) - H_{c+2}(p - e_{c+1}))
                         - (H_{c+1}(p + e_{c+2}) - H_{c+1}(p - e_{c+2})) + s ]

with every face inside the box updated and every edge not lying on a wall
updated. The evaluation follows the reading of the paper's scheme used
throughout (one fused multiply-add per update, every other operation rounded
separately); the fused operations are emulated exactly with rationals, so the
comparison is bit for bit. Edge materials are the mean of the four cells
around the edge (C-3), with the loss coefficients of the semi-implicit form.
"""

import math
from fractions import Fraction

import numpy as np

from paper_1301_4539_gb300 import workloads as wl

DX = 1e-3
C0 = 299792458.0
EPS0 = 8.8541878128e-12
N = (4, 4, 4)


def fma(a: float, b: float, c: float) -> float:
    """Correctly rounded a*b + c (exact rational, one rounding)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


class Box:
    """Field values keyed by doubled coordinates (X, Y, Z)."""

    def __init__(self, n):
        self.n = n
        self.v = {}

    def inside(self, p):
        return all(0 <= p[a] <= 2 * self.n[a] for a in range(3))

    def get(self, p):
        return self.v.get(p, 0.0)


def e_dir(p):
    odd = [a for a in range(3) if p[a] % 2]
    return odd[0] if len(odd) == 1 else None


def h_dir(p):
    even = [a for a in range(3) if p[a] % 2 == 0]
    return even[0] if len(even) == 1 else None


def shift(p, axis, d):
    q = list(p)
    q[axis] += d
    return tuple(q)


def positions(n, kind):
    out = []
    for X in range(2 * n[0] + 1):
        for Y in range(2 * n[1] + 1):
            for Z in range(2 * n[2] + 1):
                p = (X, Y, Z)
                if (kind == "e" and e_dir(p) is not None) or (kind == "h" and h_dir(p) is not None):
                    out.append(p)
    return out


def on_wall(p, n):
    """An E edge lies on a wall if one of its transverse coordinates is 0 or 2n."""
    c = e_dir(p)
    return any(p[a] in (0, 2 * n[a]) for a in range(3) if a != c)


def edge_coefficients(p, eps, sig, dt, S):
    """(Ca, Cb) of the E edge at p from its four cells (C-3, C-4)."""
    c = e_dir(p)
    t = [a for a in range(3) if a != c]
    cells = []
    # the four cells around the edge, order (-,-), (+,-), (-,+), (+,+) of the
    # two transverse axes in increasing axis order
    for db in (-1, 1):
        for da in (-1, 1):
            q = list(p)
            q[t[0]] += da
            q[t[1]] += db
            cells.append(tuple(v // 2 for v in q))  # cell index (i, j, k)
    e4 = ((float(eps[cells[0][2], cells[0][1], cells[0][0]]) + float(eps[cells[1][2], cells[1][1], cells[1][0]]))
          + float(eps[cells[2][2], cells[2][1], cells[2][0]])) + float(eps[cells[3][2], cells[3][1], cells[3][0]])
    s4 = ((float(sig[cells[0][2], cells[0][1], cells[0][0]]) + float(sig[cells[1][2], cells[1][1], cells[1][0]]))
          + float(sig[cells[2][2], cells[2][1], cells[2][0]])) + float(sig[cells[3][2], cells[3][1], cells[3][0]])
    e, s = e4 * 0.25, s4 * 0.25
    beta = (s * dt) / (2.0 * EPS0 * e)
    return (1.0 - beta) / (1.0 + beta), (S / e) / (1.0 + beta)


def brute_steps(n, eps, sig, fields, src, svals, nsteps):
    dt = wl.cfl_dt(DX)
    S = C0 * dt / DX
    E, H = Box(n), Box(n)
    # load the arrays: component c at index (i, j, k) sits at doubled coordinates
    for p in positions(n, "e"):
        c = e_dir(p)
        i, j, k = (v // 2 for v in p)
        E.v[p] = float(fields[c][k, j, i])
    for p in positions(n, "h"):
        c = h_dir(p)
        i, j, k = (v // 2 for v in p)
        H.v[p] = float(fields[3 + c][k, j, i])
    coef = {p: edge_coefficients(p, eps, sig, dt, S) for p in positions(n, "e") if not on_wall(p, n)}
    sc, si, sj, sk = src
    src_pos = tuple(2 * v + (1 if a == sc else 0) for a, v in enumerate((si, sj, sk)))
    for m in range(nsteps):
        newH = {}
        for p in positions(n, "h"):
            c = h_dir(p)
            a1, a2 = (c + 1) % 3, (c + 2) % 3
            # E_{c+1} differenced along c+2, E_{c+2} along c+1
            pa, ma = shift(p, a2, 1), shift(p, a2, -1)
            pb, mb = shift(p, a1, 1), shift(p, a1, -1)
            ea1 = E.get(pa) if E.inside(pa) and e_dir(pa) == a1 else 0.0
            ea0 = E.get(ma) if E.inside(ma) and e_dir(ma) == a1 else 0.0
            eb1 = E.get(pb) if E.inside(pb) and e_dir(pb) == a2 else 0.0
            eb0 = E.get(mb) if E.inside(mb) and e_dir(mb) == a2 else 0.0
            br = (ea1 - ea0) - (eb1 - eb0)
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
            br = (ha1 - ha0) - (hb1 - hb0)
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


def test_three_steps_on_4cubed_match_oracle_exactly(oracle_mod):
    n = N
    eps, sig = wl.random_materials(*n, seed=404, nmat=4, eps=(1.0, 6.0), sigma=(0.0, 30.0))
    fields = [f.astype(np.float64) for f in wl.random_fields(*n, seed=405)]
    amp, f0, bw, t0, kind = wl.gaussian_sine_source(f0=80e9, bw=60e9)
    src = (1, 2, 1, 2)
    o = oracle_mod.OracleGrid(*n, DX, wl.cfl_dt(DX), "f64")
    o.set_materials(eps, sig)
    for c in range(6):
        o.set_field(c, fields[c])
    o.add_source(*src, 7.0, f0, bw, t0, kind)
    nsteps = 3
    svals = oracle_mod.waveform(kind, 7.0, f0, bw, t0, o.dt, 0, nsteps)
    assert np.all(svals != 0)
    o.step(nsteps)
    ref = brute_steps(n, eps, sig, fields, src, svals, nsteps)
    for c in range(6):
        np.testing.assert_array_equal(o.f[c], ref[c], err_msg=f"component {c}")
    assert max(np.abs(ref[c]).max() for c in range(6)) > 0


def test_fma_emulation():
    a, b, c = 0.1, 10.0, -1.0
    assert fma(a, b, c) == float(Fraction(0.1) * 10 - 1)
    assert fma(a, b, c) != a * b + c or math.isclose(fma(a, b, c), a * b + c)
