"""Host half of sophie_set_materials, checked on the CPU (no GPU needed).

The library turns per-cell eps_r / sigma into one 32-bit word per index point
plus coefficient tables. Here every word is decoded and compared with an
independent NumPy computation of the scheme's edge materials: the mean of the
four cells sharing the edge, summed in double in the order (-,-), (+,-),
(-,+), (+,+) of the two transverse offsets; a conducting cell (eps_r = +inf)
makes the edge PEC, Ca = Cb = 0; otherwise beta = sigma dt / (2 eps0 eps),
Ca = (1 - beta)/(1 + beta), Cb = (S/eps)/(1 + beta), rounded once to float.
Bit for bit, for every edge, through the class table and through explicit
entries (more distinct edge materials than 511 classes). Also: the result
does not depend on the number of host threads, the classes are the most
frequent edge materials, and the words carry nothing on the padding columns.
"""

import numpy as np
import pytest

from paper_1301_4539_gb300 import sophie as so
from paper_1301_4539_gb300 import workloads as wl

C0 = 299792458.0
EPS0 = 8.8541878128e-12
DX = 1e-3
SHIFT = (3, 12, 21)


def edge_means(eps, sig):
    """(E, S): arrays (3, nz+1, ny+1, nx+1) of each component's edge eps and
    sigma means; NaN where the index is not an interior edge of it."""
    nz, ny, nx = eps.shape
    e, s = eps.astype(np.float64), sig.astype(np.float64)
    E = np.full((3, nz + 1, ny + 1, nx + 1), np.nan)
    S = np.full_like(E, np.nan)
    for a, A in ((e, E), (s, S)):
        # ex(i, j, k): cells (i, j-1, k-1), (i, j, k-1), (i, j-1, k), (i, j, k)
        A[0, 1:nz, 1:ny, 0:nx] = (((a[:-1, :-1, :] + a[:-1, 1:, :]) + a[1:, :-1, :]) + a[1:, 1:, :]) * 0.25
        # ey(i, j, k): cells (i-1, j, k-1), (i, j, k-1), (i-1, j, k), (i, j, k)
        A[1, 1:nz, 0:ny, 1:nx] = (((a[:-1, :, :-1] + a[:-1, :, 1:]) + a[1:, :, :-1]) + a[1:, :, 1:]) * 0.25
        # ez(i, j, k): cells (i-1, j-1, k), (i, j-1, k), (i-1, j, k), (i, j, k)
        A[2, 0:nz, 1:ny, 1:nx] = (((a[:, :-1, :-1] + a[:, :-1, 1:]) + a[:, 1:, :-1]) + a[:, 1:, 1:]) * 0.25
    return E, S


def coefficients(E, S, dt):
    """Expected float (Ca, Cb) per edge; (0, 0) for PEC edges and non-edges."""
    Sc = C0 * dt / DX
    with np.errstate(invalid="ignore", divide="ignore"):
        beta = (S * dt) / (2.0 * EPS0 * E)
        ca = ((1.0 - beta) / (1.0 + beta)).astype(np.float32)
        cb = ((Sc / E) / (1.0 + beta)).astype(np.float32)
    dead = ~np.isfinite(E)
    ca[dead] = 0.0
    cb[dead] = 0.0
    return ca, cb


def decode(words, ccoef, ceps, ecoef, eeps):
    """(Ca, Cb, eps) per component and index point, as the kernels read them."""
    shp = (3,) + words.shape
    ca, cb, ep = np.zeros(shp, np.float32), np.zeros(shp, np.float32), np.zeros(shp)
    expl = (words & 4) != 0
    q = (words >> 3).astype(np.int64)
    for c in range(3):
        cls = ((words >> SHIFT[c]) & 511).astype(np.int64)
        ca[c] = np.where(expl, ecoef[np.where(expl, q, 0), c, 0] if len(ecoef) else 0, ccoef[cls, 0])
        cb[c] = np.where(expl, ecoef[np.where(expl, q, 0), c, 1] if len(ecoef) else 0, ccoef[cls, 1])
        ep[c] = np.where(expl, eeps[np.where(expl, q, 0), c] if len(eeps) else 0, ceps[cls])
    return ca, cb, ep


def _materials(n3, seed, continuous):
    nx, ny, nz = n3
    rng = np.random.default_rng(seed)
    if continuous:  # more distinct edge materials than classes: explicit entries
        eps = rng.uniform(1.0, 12.0, (nz, ny, nx)).astype(np.float32)
        sig = rng.uniform(0.0, 0.4, (nz, ny, nx)).astype(np.float32)
    else:
        eps, sig = wl.random_materials(nx, ny, nz, seed, nmat=6, sigma=(0.0, 0.4))
        eps = eps.copy()
    eps[rng.random(eps.shape) < 0.03] = np.inf  # conducting cells
    return eps, sig


@pytest.mark.parametrize("continuous", [False, True])
@pytest.mark.parametrize("n3", [(13, 11, 9), (40, 7, 20), (1, 6, 5)])
def test_words_decode_to_the_edge_coefficients(n3, continuous):
    nx, ny, nz = n3
    eps, sig = _materials(n3, sum(n3) + continuous, continuous)
    dt = wl.cfl_dt(DX)
    words, ccoef, ceps, ecoef, eeps = so.sophie_debug_material_tables(eps, sig, DX, dt, nthreads=1)
    E, S = edge_means(eps, sig)
    want_ca, want_cb = coefficients(E, S, dt)
    got_ca, got_cb, got_eps = decode(words[:, :, : nx + 1], ccoef, ceps, ecoef, eeps)
    np.testing.assert_array_equal(got_ca, want_ca)
    np.testing.assert_array_equal(got_cb, want_cb)
    live = np.isfinite(E)
    np.testing.assert_array_equal(got_eps[live], E[live])  # eps_r(edge) in double, for the energy
    assert not words[:, :, nx + 1:].any()  # padding columns carry nothing
    assert (words & 3).max() == 0  # no source or probe flags from the host build
    ndistinct = len(np.unique(np.stack([E[live], S[live]], axis=1), axis=0))
    assert (len(ecoef) > 0) == (ndistinct > 511)  # explicit entries exactly when the classes run out
    if continuous and nx > 1:
        assert ndistinct > 511
    assert ccoef[0].tolist() == [0.0, 0.0]  # class 0: PEC / no edge


@pytest.mark.parametrize("continuous", [False, True])
def test_thread_count_does_not_change_the_tables(continuous):
    eps, sig = _materials((37, 23, 70), 5, continuous)
    dt = wl.cfl_dt(DX)
    a = so.sophie_debug_material_tables(eps, sig, DX, dt, nthreads=1)
    b = so.sophie_debug_material_tables(eps, sig, DX, dt, nthreads=3)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_classes_are_the_most_frequent_edge_materials():
    eps, sig = _materials((30, 30, 30), 9, True)
    dt = wl.cfl_dt(DX)
    _, ccoef, ceps, _, _ = so.sophie_debug_material_tables(eps, sig, DX, dt, nthreads=2)
    E, S = edge_means(eps, sig)
    live = np.isfinite(E)
    pairs, counts = np.unique(np.stack([E[live], S[live]], axis=1), axis=0, return_counts=True)
    freq = {(p[0], p[1]): c for p, c in zip(pairs, counts)}
    assert len(freq) > 511
    # a class is identified by its table row (eps_r in double, (Ca, Cb) in
    # float); a point with any edge outside the classes is explicit as a whole,
    # so the words alone do not show which materials are classes
    table = {(ceps[q], ccoef[q, 0], ccoef[q, 1]) for q in range(1, 512)}
    assert len(table) == 511
    mats = np.array(list(freq), np.float64)
    ca, cb = coefficients(mats[:, 0], mats[:, 1], dt)
    in_class = np.array([(m[0], a, b) in table for m, a, b in zip(mats, ca, cb)])
    f = np.array([freq[(m[0], m[1])] for m in mats])
    assert in_class.sum() == 511  # every class row is one of the materials
    assert f[in_class].min() >= f[~in_class].max()  # and the classes are the most frequent ones


def test_bad_materials_are_rejected():
    eps = np.full((4, 4, 4), 2.0, np.float32)
    sig = np.zeros_like(eps)
    eps[1, 2, 3] = 0.5
    with pytest.raises(so.SophieError) as e:
        so.sophie_debug_material_tables(eps, sig, DX, wl.cfl_dt(DX))
    assert e.value.code == so.EINVAL
    eps[1, 2, 3] = 2.0
    sig[0, 0, 1] = np.nan
    with pytest.raises(so.SophieError) as e:
        so.sophie_debug_material_tables(eps, sig, DX, wl.cfl_dt(DX))
    assert e.value.code == so.EINVAL
