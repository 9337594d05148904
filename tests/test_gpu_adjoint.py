"""Differentiation form: gradients of a probe objective w.r.t. eps_r through
the C ABI (sophie_objective_forward / sophie_objective_grad_eps) and the
torch.autograd.Function, against the FP64 oracle's reverse-mode gradient and
against central finite differences of the FP64 oracle's forward run.

J = dt * sum_{n=1..N} (probe value after step n)^2. The library differentiates
its float steps; the oracle differentiates the double ones. The two agree to
float accuracy; the bars below are stated per test.
"""

import numpy as np
import pytest

from gpu_helpers import DX
from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _small_case(seed=41):
    nx, ny, nz = 40, 36, 28
    eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=5, eps=(1.0, 6.0), sigma=(0.0, 2.0))
    rng = np.random.default_rng(seed)
    box = (10, 8, 6, 12, 12, 8)  # i0, j0, k0, ni, nj, nk
    i0, j0, k0, ni, nj, nk = box
    eps[k0:k0 + nk, j0:j0 + nj, i0:i0 + ni] = rng.uniform(1.0, 4.0, (nk, nj, ni)).astype(np.float32)
    amp, f0, bw, t0, kind = wl.gaussian_sine_source(f0=40e9, bw=30e9)
    src = (2, 6, 18, 14, amp, f0, bw, t0, kind)
    probe = (2, 30, 17, 13)
    return (nx, ny, nz), eps, sig, src, probe, box


def _gpu_grad(n3, eps, sig, src, probe, box, nsteps, K=0, temporal_k=2, fields=None, traced=False):
    g = so.Grid(*n3, DX, wl.cfl_dt(DX))
    g.configure(temporal_k=temporal_k)
    g.set_materials(eps, sig)
    if fields is not None:
        for c in range(6):
            g.set_field(c, fields[c])
    g.add_source(*src)
    if traced:
        g.objective_set_design(*box)
    J = g.objective_forward(nsteps, *probe, K)
    grad = g.objective_grad_eps(*box)
    return g, J, grad


def _oracle_grad(oracle_mod, n3, eps, sig, src, probe, cells, nsteps, fields=None):
    o = oracle_mod.OracleGrid(*n3, DX, wl.cfl_dt(DX), "f64")
    o.set_materials(eps, sig)
    if fields is not None:
        for c in range(6):
            o.set_field(c, fields[c].astype(np.float64))
    o.add_source(*src)
    return o.grad_eps(*probe, nsteps, cells)


def _box_cells(box):
    i0, j0, k0, ni, nj, nk = box
    return [(i0 + i, j0 + j, k0 + k) for k in range(nk) for j in range(nj) for i in range(ni)]


@pytest.mark.parametrize("form", ["default", "direct"])
@pytest.mark.parametrize("probe_comp", [2, 4])
def test_grad_matches_fp64_oracle_gradient(oracle_mod, sophie, monkeypatch, form, probe_comp):
    """Both forms of the reverse sweep (forward step kernel on u = Cb l_e,
    mu = -S l_h; literal transposed step on l_e, l_h), for an E and an H
    objective, against the FP64 oracle's gradient over every design cell."""
    if form == "direct":
        monkeypatch.setenv("SOPHIE_ADJOINT", "direct")
    n3, eps, sig, src, probe, box = _small_case()
    probe = (probe_comp,) + probe[1:]
    N = 130  # segments 50, 50, 30
    g, J, grad = _gpu_grad(n3, eps, sig, src, probe, box, N)
    Jo, go = _oracle_grad(oracle_mod, n3, eps, sig, src, probe, _box_cells(box), N)
    go = go.reshape(grad.shape)
    print(f"[{form}, comp {probe_comp}] J gpu {J:.9e} oracle {Jo:.9e}")
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    scale = np.max(np.abs(go))
    rel = np.linalg.norm(grad - go) / np.linalg.norm(go)
    worst = np.max(np.abs(grad - go)) / scale
    print(f"[{form}, comp {probe_comp}] gradient vs FP64 oracle: rel-L2 {rel:.3e}, max |diff|/max|g| {worst:.3e}")
    assert rel <= 1e-4 and worst <= 1e-4
    assert g.n == N


def test_grad_independent_of_checkpoint_interval_and_step_kernel(sophie):
    n3, eps, sig, src, probe, box = _small_case(seed=7)
    N = 77
    ref = None
    for K, tk in ((0, 2), (7, 1), (1, 3), (77, 2), (200, 4)):
        _, J, grad = _gpu_grad(n3, eps, sig, src, probe, box, N, K=K, temporal_k=tk)
        if ref is None:
            ref = (J, grad)
        else:
            assert J == ref[0]
            np.testing.assert_array_equal(grad, ref[1])


def test_traced_record_equals_checkpointed(sophie):
    """A design box registered before the forward pass: the traces of every
    step are gathered during it and the reverse sweep recomputes nothing; the
    gradient is bitwise the checkpointed record's (the same float values are
    gathered), for an E and an H objective. A traced record keeps no
    checkpoints, so another box is refused; after clearing the box the next
    record is checkpointed again and serves any box."""
    n3, eps, sig, src, probe, box = _small_case(seed=11)
    N = 90
    for pc in (2, 3):
        pr = (pc,) + probe[1:]
        _, J0, g0 = _gpu_grad(n3, eps, sig, src, pr, box, N, K=30)
        g1, J1, gr1 = _gpu_grad(n3, eps, sig, src, pr, box, N, K=30, traced=True)
        assert J0 == J1
        np.testing.assert_array_equal(gr1, g0)
        # the forward state is that of plain steps either way
        g2 = so.Grid(*n3, DX, wl.cfl_dt(DX))
        g2.set_materials(eps, sig)
        g2.add_source(*src)
        g2.step(N)
        for c in range(6):
            np.testing.assert_array_equal(g1.get_field(c), g2.get_field(c))
        other = (box[0] + 1, box[1], box[2], box[3] - 2, box[4], box[5])
        with pytest.raises(so.SophieError):
            g1.objective_grad_eps(*other)
        g1.objective_set_design()  # cleared: the next record is checkpointed again
        g1.reset()
        J3 = g1.objective_forward(N, *pr, 30)
        np.testing.assert_array_equal(g1.objective_grad_eps(*box), g0)
        assert J3 == J0 and g1.objective_grad_eps(*other).shape == (other[5], other[4], other[3])
    with pytest.raises(so.SophieError):
        g1.objective_set_design(0, 0, 0, n3[0] + 1, 1, 1)


def test_forward_state_equals_plain_steps_and_probes_unaffected(sophie):
    n3, eps, sig, src, probe, box = _small_case(seed=3)
    N = 64
    a = so.Grid(*n3, DX, wl.cfl_dt(DX))
    b = so.Grid(*n3, DX, wl.cfl_dt(DX))
    for g in (a, b):
        g.set_materials(eps, sig)
        g.add_source(*src)
        g.add_probe(2, 20, 20, 20)
    pa = a.add_probe(*probe)
    a.objective_forward(N, *probe, 10)
    b.step(N)
    for c in range(6):
        np.testing.assert_array_equal(a.get_field(c), b.get_field(c))
    np.testing.assert_array_equal(a.read_probe(0), b.read_probe(0))
    # the objective is the sum of squares of the same samples a probe records
    f = a.read_probe(pa)
    J = a.objective_forward(1, *probe)  # one more step; compare the first record below
    a2 = so.Grid(*n3, DX, wl.cfl_dt(DX))
    a2.set_materials(eps, sig)
    a2.add_source(*src)
    J64 = a2.objective_forward(N, *probe)
    assert abs(J64 - wl.cfl_dt(DX) * float(np.sum(f * f))) <= 1e-12 * J64
    assert J > 0
    # a probe added after an objective record starts clean
    q = a.add_probe(*probe)
    a.step(3)
    tr = a.read_probe(q)
    assert np.all(tr[: N + 1] == 0) and np.all(tr[N + 1:] == a.read_probe(pa)[N + 1:])


def test_objective_errors(sophie):
    n3, eps, sig, src, probe, box = _small_case()
    g = so.Grid(*n3, DX, wl.cfl_dt(DX))
    g.set_materials(eps, sig)
    g.add_source(*src)
    with pytest.raises(so.SophieError) as e:
        g.objective_grad_eps(*box)
    assert e.value.code == so.EINVAL
    g.objective_forward(10, *probe)
    g.objective_grad_eps(*box)
    g.step(1)  # the record is stale now
    with pytest.raises(so.SophieError) as e:
        g.objective_grad_eps(*box)
    assert e.value.code == so.EINVAL
    g.objective_forward(10, *probe)
    with pytest.raises(so.SophieError):
        g.objective_grad_eps(0, 0, 0, n3[0] + 1, 1, 1)
    with pytest.raises(so.SophieError):
        g.objective_forward(0, *probe)
    with pytest.raises(so.SophieError):
        g.objective_forward(5, 2, 3, 3, n3[2])  # ez has no k = nz
    with pytest.raises(so.SophieError):
        g.objective_forward(5, 3, n3[0], 3, 3)  # hx on the plane i = nx
    g.configure(precision=so.FP16)
    with pytest.raises(so.SophieError) as e:
        g.objective_forward(5, *probe)
    assert e.value.code == so.ENOTSUP
    g.configure(precision=so.FP32)
    g.objective_release()
    with pytest.raises(so.SophieError):
        g.objective_grad_eps(*box)


def test_autograd_function(sophie):
    import torch
    from paper_1301_4539_gb300.autograd import probe_objective
    n3, eps, sig, src, probe, box = _small_case(seed=9)
    i0, j0, k0, ni, nj, nk = box
    g = so.Grid(*n3, DX, wl.cfl_dt(DX))
    g.add_source(*src)
    d = torch.tensor(eps[k0:k0 + nk, j0:j0 + nj, i0:i0 + ni], dtype=torch.float64, requires_grad=True)
    J = probe_objective(d, g, eps, sig, box, probe, 90, 25)
    (3.0 * J).backward()
    _, J2, grad = _gpu_grad(n3, eps, sig, src, probe, box, 90, K=25)
    assert float(J.detach()) == J2
    np.testing.assert_array_equal(d.grad.numpy(), 3.0 * grad)
    # a second evaluation at other eps values resets the grid first
    d2 = (d.detach() * 1.01).requires_grad_(True)
    J3 = probe_objective(d2, g, eps, sig, box, probe, 90, 25)
    assert float(J3.detach()) != float(J.detach())


def test_design_cavity_vs_central_differences(oracle_mod, sophie):
    """The differentiation workload: 128^3 vacuum cavity, 32^3 design region
    with eps_r U(1,4), Gaussian-pulse Ez source 8 cells inside a face, Ez probe,
    800 steps, checkpoints every 50. dJ/deps_r on 16 seeded design cells against
    central differences (h = 1e-3) of the FP64 oracle's J, to 1e-3 relative,
    and against the FP64 oracle's reverse-mode gradient."""
    w = wl.design_cavity()
    n3 = (w["nx"], w["ny"], w["nz"])
    eps, sig, src, probe = w["eps"], w["sigma"], w["sources"][0], w["probe"]
    N = 800
    g, J, grad = _gpu_grad(n3, eps, sig, src, probe, w["design"], N, K=50, traced=True)
    lo = w["design"][0]
    gc = np.array([grad[k - lo, j - lo, i - lo] for (i, j, k) in w["cells"]])
    Jo, go = _oracle_grad(oracle_mod, n3, eps, sig, src, probe, w["cells"], N)
    print(f"design cavity: J gpu {J:.9e} oracle {Jo:.9e}")
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    fd = []
    for (i, j, k) in w["cells"]:
        vals = []
        for sgn in (1, -1):
            e = eps.copy()
            e[k, j, i] = np.float32(float(eps[k, j, i]) + sgn * 1e-3)
            o = oracle_mod.OracleGrid(*n3, DX, wl.cfl_dt(DX), "f64")
            o.set_materials(e, sig)
            o.add_source(*src)
            q = o.add_probe(*probe)
            o.step(N)
            p = o.probe(q)
            vals.append((o.dt * float(np.sum(p * p)), float(e[k, j, i])))
        fd.append((vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1]))
    fd = np.array(fd)
    rel_fd = np.abs(gc - fd) / np.abs(fd)
    rel_or = np.abs(gc - go) / np.abs(go)
    for q, (i, j, k) in enumerate(w["cells"]):
        print(f"cell ({i},{j},{k}): gpu {gc[q]:+.6e} oracle {go[q]:+.6e} fd {fd[q]:+.6e} "
              f"rel vs fd {rel_fd[q]:.2e} vs oracle {rel_or[q]:.2e}")
    assert np.all(rel_fd <= 1e-3)
    # float steps against double steps: an absolute floor set by the largest
    # gradient (cells with small gradients lose relative digits to it)
    assert np.max(np.abs(gc - go)) <= 3e-5 * np.max(np.abs(go))
    # the oracle's own gradient against its central differences (h = 1e-3)
    assert np.all(np.abs(go - fd) <= 1e-5 * np.abs(fd))
