"""Storage-precision forms (float / half / bfloat16 fields, float arithmetic).

* Round trips: values representable in the storage format come back exactly,
  with per-component power-of-two scales; switching the format converts the
  fields.
* Accuracy: each form against the FP64 oracle on a seeded sphere cavity, as
  relative L2 over all six fields and over the probe traces. Float storage must
  stay within the 1e-5 bar, the hi+lo half split within 1e-4 and the 24-bit
  form within the stated 1e-3 bar; the 2-byte forms are held to loose bounds
  here (to catch defects) and their measured errors are printed.
* The 24-bit form is bitwise equal to the float oracle run with the same
  storage rounding between launches (oracle.round24 / step_stored24), for
  every K, with sources, probes, lossy materials and explicit entries.
"""

import numpy as np
import pytest

from gpu_helpers import DX
from modes import rel_l2
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_roundtrip_and_conversion(sophie):
    nx, ny, nz = 20, 12, 9
    g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
    rng = np.random.default_rng(5)
    # k/32 with |k| < 128: at most 7 significant bits, exact in half and bfloat16
    f = [rng.integers(-127, 128, size=(nz + 1, ny + 1, nx + 1)).astype(np.float32) / 32 for _ in range(6)]
    ref = wl.random_fields(nx, ny, nz, 0)
    masked = [np.where(ref[c] != 0, f[c], 0).astype(np.float32) for c in range(6)]
    for c in range(6):
        g.set_field(c, f[c])
    for prec in (so.FP16, so.BF16, so.FP32, so.FP16HL, so.FP24, so.FP16, so.FP24, so.FP32):
        g.configure(temporal_k=1, precision=prec)
        for c in range(6):
            np.testing.assert_array_equal(g.get_field(c), masked[c])
    g.set_storage_scale([2.0 ** 4, 2.0 ** -3, 1.0, 2.0, 2.0 ** 10, 0.5])
    for c in range(6):
        np.testing.assert_array_equal(g.get_field(c), masked[c])
    with pytest.raises(so.SophieError):
        g.set_storage_scale([3.0, 1, 1, 1, 1, 1])
    with pytest.raises(so.SophieError):
        g.configure(tile_x=32, precision=so.FP16)


def _run_modes(oracle_mod, n, steps, modes, full_generator=False):
    nx = ny = nz = n
    if full_generator:
        w = wl.sphere_cavity(n)
        eps, sig, src, prbs = w["eps"], w["sigma"], w["sources"][0], w["probes"]
    else:
        eps, sig = wl.sphere_materials(nx, ny, nz, nspheres=10, seed=1301, radius=(2, 8))
        amp, f0, bw, t0, kind = wl.gaussian_sine_source()
        src = (2, nx // 2, ny // 2, nz // 2, amp, f0, bw, t0, kind)
        prbs = wl.probe_edges(nx, ny, nz, 8, seed=1302)
    o = oracle_mod.OracleGrid(nx, ny, nz, DX, wl.cfl_dt(DX), "f64")
    o.set_materials(eps, sig)
    o.add_source(*src)
    for p in prbs:
        o.add_probe(*p)
    o.step(steps)
    ref = np.concatenate([a.ravel() for a in o.f])
    pref = np.concatenate([o.probe(q) for q in range(len(prbs))])
    out = {}
    for name, prec, k, scale in modes:
        g = so.Grid(nx, ny, nz, DX, wl.cfl_dt(DX))
        g.configure(temporal_k=k, precision=prec)
        if scale is not None:
            g.set_storage_scale([scale] * 6)
        g.set_materials(eps, sig)
        g.add_source(*src)
        for p in prbs:
            g.add_probe(*p)
        g.step(steps)
        got = np.concatenate([g.get_field(c).astype(np.float64).ravel() for c in range(6)])
        pgot = np.concatenate([g.read_probe(q) for q in range(len(prbs))])
        out[name] = (rel_l2(got, ref), rel_l2(pgot, pref))
        g.close()
    return out


def test_precision_forms_vs_fp64_oracle(oracle_mod, sophie):
    modes = [("fp32_k1", so.FP32, 1, None), ("fp32_k2", so.FP32, 2, None),
             ("fp16_k1", so.FP16, 1, 2.0 ** 10), ("fp16_k2", so.FP16, 2, 2.0 ** 10),
             ("bf16_k1", so.BF16, 1, None), ("bf16_k2", so.BF16, 2, None),
             ("fp16hl_k1", so.FP16HL, 1, 2.0 ** 10), ("fp16hl_k2", so.FP16HL, 2, 2.0 ** 10),
             ("fp24_k1", so.FP24, 1, None), ("fp24_k2", so.FP24, 2, None)]
    out = _run_modes(oracle_mod, 64, 400, modes)
    for k, v in out.items():
        print(f"precision 64^3 x 400 steps {k}: fields rel-L2 {v[0]:.3e}, probes rel-L2 {v[1]:.3e}")
    assert out["fp32_k1"][0] < 1e-5 and out["fp32_k2"][0] < 1e-5
    assert out["fp32_k1"] == out["fp32_k2"]
    assert out["fp16_k1"][0] < 5e-2 and out["fp16_k2"][0] < 5e-2
    assert out["bf16_k1"][0] < 5e-1 and out["bf16_k2"][0] < 5e-1
    # two steps per rounding cannot be worse than one by much
    assert out["fp16_k2"][0] < 1.5 * out["fp16_k1"][0] + 1e-6
    # the hi+lo split meets the 1e-3 bar with a wide margin
    assert out["fp16hl_k1"][0] < 1e-4 and out["fp16hl_k2"][0] < 1e-4
    assert out["fp16hl_k1"][1] < 1e-4 and out["fp16hl_k2"][1] < 1e-4
    # the 24-bit form meets the 1e-3 bar
    for k in ("fp24_k1", "fp24_k2"):
        assert out[k][0] < 1e-3 and out[k][1] < 1e-3, (k, out[k])


@pytest.mark.slow
def test_precision_forms_256_2000_steps(oracle_mod, sophie):
    """The precision protocol at 256^3: 2000 steps against the FP64 oracle."""
    modes = [("fp32_k2", so.FP32, 2, None), ("fp16_k1", so.FP16, 1, 2.0 ** 10),
             ("fp16_k2", so.FP16, 2, 2.0 ** 10), ("bf16_k2", so.BF16, 2, None),
             ("fp16hl_k2", so.FP16HL, 2, 2.0 ** 10), ("fp24_k1", so.FP24, 1, None),
             ("fp24_k2", so.FP24, 2, None), ("fp24_k3", so.FP24, 3, None), ("fp24_k4", so.FP24, 4, None)]
    out = _run_modes(oracle_mod, 256, 2000, modes, full_generator=True)
    for k, v in out.items():
        print(f"precision 256^3 x 2000 steps {k}: fields rel-L2 {v[0]:.3e}, probes rel-L2 {v[1]:.3e}")
    assert out["fp32_k2"][0] < 1e-5
    assert out["fp16hl_k2"][0] < 1e-3 and out["fp16hl_k2"][1] < 1e-3
    for k in ("fp24_k1", "fp24_k2", "fp24_k3", "fp24_k4"):
        assert out[k][0] < 1e-3 and out[k][1] < 1e-3, (k, out[k])


@pytest.mark.parametrize("zsplit", [None, "13"])
@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("n3", [(70, 37, 19), (33, 65, 18), (130, 21, 40)])
def test_fp24_equals_oracle_with_storage_rounding(oracle_mod, sophie, monkeypatch, K, n3, zsplit):
    """Fields, probe samples and energy of the 24-bit form, bitwise equal to
    the float oracle whose fields are held in the same form between launches
    (K steps per launch, single steps for the remainder). zsplit = 13: every
    tile's planes cut into 13 z ranges of about 3 planes, so most units start
    near plane 0 or replay their levels' history (the blocked kernel once read
    stale shared-memory seam rows in such units)."""
    if zsplit:
        if K == 1:
            pytest.skip("the z split is a blocked-kernel knob")
        monkeypatch.setenv("SOPHIE_BLOCKED_ZSPLIT", zsplit)
    nx, ny, nz = n3
    eps, sig = wl.random_materials(nx, ny, nz, seed=nx + 7 * K, nmat=6, sigma=(0.0, 0.5))
    eps = eps.copy()
    eps[:, : ny // 3, : nx // 4] = np.random.default_rng(K).uniform(1, 9, size=(nz, ny // 3, nx // 4))  # explicit entries
    f = wl.random_fields(nx, ny, nz, seed=ny + K)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source()
    srcs = [(2, nx // 2, ny // 2, nz // 2, 25.0, f0, bw, 4e-12, 0), (0, nx // 3, ny // 3, nz // 3, 3.0, f0, bw, 5e-12, 1)]
    prbs = wl.probe_edges(nx, ny, nz, 5, seed=nx) + [(3, nx // 2, ny // 2, nz // 2), (5, 1, 1, nz)]
    dt = wl.cfl_dt(DX)
    g = so.Grid(nx, ny, nz, DX, dt)
    g.configure(temporal_k=K, precision=so.FP24)
    g.set_materials(eps, sig)
    o = oracle_mod.OracleGrid(nx, ny, nz, DX, dt, "f32")
    o.set_materials(eps, sig)
    for c in range(6):
        g.set_field(c, f[c])
    for c in range(6):
        o.set_field(c, g.get_field(c))  # the stored (masked, rounded) initial state
        np.testing.assert_array_equal(o.f[c], np.where(o.f[c] != 0, oracle_mod.round24(f[c]), 0))
    for s in srcs:
        g.add_source(*s)
        o.add_source(*s)
    for p in prbs:
        g.add_probe(*p)
        o.add_probe(*p)
    for n in (3 * K + 1, K + 2):
        g.step(n)
        o.step_stored24(n, K)
        for c in range(6):
            got = g.get_field(c)
            bad = np.argwhere(got != o.f[c])
            assert bad.size == 0, (K, c, bad[:4])
    for q in range(len(prbs)):
        np.testing.assert_array_equal(g.read_probe(q), o.probe(q))
    assert abs(g.energy() - o.energy()) <= 1e-12 * abs(o.energy())
    g.close()
