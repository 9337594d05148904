"""Pins of the oracle's 24-bit storage rounding (oracle.round24) and of the
24-bit storage form's accuracy.

The storage form keeps the upper 24 bits of each float (sign, exponent, 15
mantissa bits). The oracle rounds a value by Veltkamp's splitting in float
arithmetic; that is pinned here against an independent integer computation
of round-to-nearest-even to 16 significant bits on the float's bit pattern
(exact for normal floats: within a binade the patterns are evenly spaced and a
carry out of the mantissa moves to the next binade), which a dropped term or
a wrong split constant would fail.
"""

import numpy as np

import oracle
from paper_1301_4539_gb300 import workloads as wl


def _rne24_int(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even of float32 values to 16 significant bits, on the
    bit pattern of the magnitude (independent of the oracle's float split)."""
    u = x.view(np.uint32)
    m = (u & 0x7FFFFFFF).astype(np.int64)
    low = m & 0xFF
    down = m - low
    up = down + 0x100
    keep_up = (low > 0x80) | ((low == 0x80) & (((down >> 8) & 1) == 1))
    r = np.where(keep_up, up, down).astype(np.uint32) | (u & 0x80000000)
    return r.view(np.float32)


def test_round24_is_round_to_nearest_even_on_16_bits():
    rng = np.random.default_rng(24)
    # normal floats whose split does not overflow (|v| * 257 finite)
    u = rng.integers(0x00800000, 0x7A000000, size=400_000, dtype=np.uint64).astype(np.uint32)
    u[::3] = (u[::3] & 0xFFFFFF00) | 0x80  # exact ties
    u[1::7] = u[1::7] | 0xFF               # just below a carry into the next binade
    x = u.view(np.float32) * np.where(rng.random(u.size) < 0.5, -1, 1).astype(np.float32)
    r = oracle.round24(x)
    np.testing.assert_array_equal(r.view(np.uint32), _rne24_int(x).view(np.uint32))
    assert np.all((r.view(np.uint32) & 0xFF) == 0)
    # the error bound of 16 significant bits, and idempotence
    rel = np.abs(r.astype(np.float64) - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -16
    np.testing.assert_array_equal(oracle.round24(r).view(np.uint32), r.view(np.uint32))


def test_round24_special_values():
    x = np.array([0.0, -0.0, 1.0, 1 + 2 ** -16, 1 + 3 * 2 ** -16, 2 - 2 ** -23, 1e-40, -3e-39], np.float32)
    r = oracle.round24(x)
    bits = r.view(np.uint32)
    assert bits[0] == 0 and bits[1] == 0                # -0 comes out as +0 (c + (v - c) = -0 + +0)
    assert r[2] == 1.0
    assert r[3] == 1.0                                  # tie -> even (down)
    assert r[4] == np.float32(1 + 2 ** -14)             # tie -> even (up)
    assert r[5] == 2.0                                  # carry into the next binade
    assert np.all(bits[6:] & 0xFF == 0)                 # subnormals: low byte dropped
    assert abs(float(r[6]) - 1e-40) < 2 ** -126 * 2 ** -14


def test_storage_form_meets_the_bar_in_emulation():
    """The 24-bit storage form against the FP64 oracle on the sphere
    generator at 64^3 x 400 steps (fields held in the form between launches of
    one and of two steps): relative L2 well below the 1e-3 bar, and the float
    form far below it."""
    n, T = 64, 400
    w = wl.sphere_cavity(n)

    def grid(prec):
        g = oracle.OracleGrid(n, n, n, w["dx"], w["dt"], prec)
        g.set_materials(w["eps"], w["sigma"])
        for s in w["sources"]:
            g.add_source(*s)
        return g

    ref = grid("f64")
    ref.step(T)
    den = sum(float(np.sum(a ** 2)) for a in ref.f)
    errs = {}
    for k in (1, 2):
        g = grid("f32")
        g.step_stored24(T, k)
        errs[k] = (sum(float(np.sum((g.f[c].astype(np.float64) - ref.f[c]) ** 2)) for c in range(6)) / den) ** 0.5
    print("24-bit storage form vs FP64 oracle, 64^3 x 400 steps:", errs)
    assert errs[1] < 1e-3 and errs[2] < 1e-3
    assert errs[2] < errs[1] * 1.2 + 1e-7
