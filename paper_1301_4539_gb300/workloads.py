"""Seeded synthetic inputs shaped like the paper's cavity workloads.

This module only draws inputs (materials, source and probe placement, random
initial fields). It holds none of the Yee update arithmetic, so both the CUDA
path and the CPU oracle can be fed from it.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition; a double in [0, 1) is (x >> 11) * 2**-53.

Workloads (the paper's Sophie cavities, Sec. 4.2, are not available; these
stand in for them):
  * TM110 cavity: 32^3, vacuum, no source (initial state from the exact mode).
  * Sphere cavity: n^3 PEC box with 64 random dielectric spheres (radius
    U(4,24) cells, eps_r U(1,12), sigma U(0,0.05) S/m), later spheres overwrite
    earlier ones, a Gaussian-modulated-sine Ez source at the centre (10 GHz,
    5 GHz bandwidth) and 16 random interior Ez probes.
  * Graded sphere cavity: the same on a non-uniform mesh refined towards the
    centre along every axis (widths dx down to dx/2, Gaussian profile).
"""

from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1

C0 = 299792458.0
DX_DEFAULT = 1e-3


class SplitMix64:
    """splitmix64 sequence generator (published constants)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (2.0 ** -53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi)."""
        return lo + int(self.uniform() * (hi - lo))


def cfl_dt(dx: float = DX_DEFAULT, frac: float = 0.99) -> float:
    """Time step at a fraction of the 3-D Courant limit dx / (c sqrt 3)."""
    return frac * dx / (C0 * math.sqrt(3.0))


def sphere_list(nx: int, ny: int, nz: int, nspheres: int = 64, seed: int = 1301,
                radius=(4.0, 24.0), eps=(1.0, 12.0), sigma=(0.0, 0.05)):
    """Sphere parameters (cx, cy, cz, r, eps_r, sigma) in generation order."""
    g = SplitMix64(seed)
    out = []
    for _ in range(nspheres):
        cx = g.uniform(0.0, nx)
        cy = g.uniform(0.0, ny)
        cz = g.uniform(0.0, nz)
        r = g.uniform(*radius)
        e = g.uniform(*eps)
        s = g.uniform(*sigma)
        out.append((cx, cy, cz, r, e, s))
    return out


def sphere_materials(nx: int, ny: int, nz: int, nspheres: int = 64, seed: int = 1301,
                     radius=(4.0, 24.0), eps=(1.0, 12.0), sigma=(0.0, 0.05)):
    """Per-cell (eps_r, sigma) arrays of shape (nz, ny, nx), float32.

    A cell belongs to a sphere if its centre (i+1/2, j+1/2, k+1/2) lies within
    r of the sphere centre; later spheres overwrite earlier ones. Background is
    vacuum (eps_r = 1, sigma = 0).
    """
    eps_a = np.ones((nz, ny, nx), np.float32)
    sig_a = np.zeros((nz, ny, nx), np.float32)
    for cx, cy, cz, r, e, s in sphere_list(nx, ny, nz, nspheres, seed, radius, eps, sigma):
        i0, i1 = max(0, int(math.floor(cx - r - 1))), min(nx, int(math.ceil(cx + r + 1)))
        j0, j1 = max(0, int(math.floor(cy - r - 1))), min(ny, int(math.ceil(cy + r + 1)))
        k0, k1 = max(0, int(math.floor(cz - r - 1))), min(nz, int(math.ceil(cz + r + 1)))
        if i0 >= i1 or j0 >= j1 or k0 >= k1:
            continue
        x = np.arange(i0, i1) + 0.5 - cx
        y = np.arange(j0, j1) + 0.5 - cy
        z = np.arange(k0, k1) + 0.5 - cz
        d2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
        m = d2 <= r * r
        eps_a[k0:k1, j0:j1, i0:i1][m] = np.float32(e)
        sig_a[k0:k1, j0:j1, i0:i1][m] = np.float32(s)
    return eps_a, sig_a


def probe_edges(nx: int, ny: int, nz: int, count: int = 16, seed: int = 1302, comp: int = 2):
    """`count` random interior Ez edges (comp, i, j, k), i,j in [1, n-1), k in [1, nz-1)."""
    g = SplitMix64(seed)
    out = []
    for _ in range(count):
        i = g.randint(1, max(2, nx - 1))
        j = g.randint(1, max(2, ny - 1))
        k = g.randint(1, max(2, nz - 1))
        out.append((comp, min(i, nx - 1), min(j, ny - 1), min(k, max(nz - 1, 0))))
    return out


def gaussian_sine_source(f0: float = 10e9, bw: float = 5e9, amp: float = 1.0):
    """Source parameters (amp, f0, bw, t0, kind=0); t0 = 5 envelope widths.

    The envelope width st = 1/(2 pi sf) with sf = bw / (2 sqrt(2 ln 2)), so that
    bw is the full width at half maximum of the spectrum's amplitude.
    """
    sf = bw / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    st = 1.0 / (2.0 * math.pi * sf)
    return amp, f0, bw, 5.0 * st, 0


def sphere_cavity(n: int = 256, seed_materials: int = 1301, seed_probes: int = 1302,
                  nprobes: int = 16):
    """The sphere-cavity workload: materials, the centre Ez source and probes."""
    eps_a, sig_a = sphere_materials(n, n, n, seed=seed_materials)
    amp, f0, bw, t0, kind = gaussian_sine_source()
    src = (2, n // 2, n // 2, n // 2, amp, f0, bw, t0, kind)
    probes = probe_edges(n, n, n, nprobes, seed_probes)
    return dict(nx=n, ny=n, nz=n, dx=DX_DEFAULT, dt=cfl_dt(DX_DEFAULT), eps=eps_a,
                sigma=sig_a, sources=[src], probes=probes)


def graded_widths(n: int, dx: float = DX_DEFAULT, fine: float = 0.5, spread: float = 0.125):
    """Cell widths of an axis refined around its centre: dx far from it, fine*dx
    at it, a Gaussian profile of width spread*n cells in between."""
    i = np.arange(n, dtype=np.float64) + 0.5
    return dx * (1.0 - (1.0 - fine) * np.exp(-(((i - n / 2.0) / (spread * n)) ** 2)))


def random_widths(n: int, seed: int, dx: float = DX_DEFAULT, lo: float = 0.6, hi: float = 1.6):
    """Cell widths drawn uniformly in [lo*dx, hi*dx) (independent per cell)."""
    return dx * np.random.default_rng(seed).uniform(lo, hi, n)


def mesh_dt(wx, wy, wz, frac: float = 0.99) -> float:
    """Time step at a fraction of the Courant limit of a mesh's smallest cells,
    1 / (c sqrt(1/min(wx)^2 + 1/min(wy)^2 + 1/min(wz)^2))."""
    inv2 = sum(1.0 / float(np.min(w)) ** 2 for w in (wx, wy, wz))
    return frac / (C0 * math.sqrt(inv2))


def sphere_cavity_graded(n: int = 256, fine: float = 0.5):
    """The sphere-cavity workload on a mesh refined around the source: every
    axis graded by graded_widths (dx = 1 mm far out, fine*dx at the centre),
    dt at 0.99 of the refined mesh's Courant limit."""
    w = sphere_cavity(n)
    widths = [graded_widths(n, w["dx"], fine) for _ in range(3)]
    w.update(widths=widths, dt=mesh_dt(*widths))
    return w


def random_fields(nx: int, ny: int, nz: int, seed: int, scale: float = 1.0):
    """Six random float32 fields of shape (nz+1, ny+1, nx+1) with zero PEC edges
    and zero entries outside each component's index range."""
    rng = np.random.default_rng(seed)
    shp = (nz + 1, ny + 1, nx + 1)
    f = [rng.standard_normal(shp).astype(np.float32) * np.float32(scale) for _ in range(6)]
    ex, ey, ez, hx, hy, hz = f
    # e_x: i in [0,nx), j in [1,ny), k in [1,nz)
    ex[:, :, nx] = 0; ex[:, 0, :] = 0; ex[:, ny, :] = 0; ex[0] = 0; ex[nz] = 0
    ey[:, ny, :] = 0; ey[:, :, 0] = 0; ey[:, :, nx] = 0; ey[0] = 0; ey[nz] = 0
    ez[nz] = 0; ez[:, :, 0] = 0; ez[:, :, nx] = 0; ez[:, 0, :] = 0; ez[:, ny, :] = 0
    hx[:, ny, :] = 0; hx[nz] = 0
    hy[:, :, nx] = 0; hy[nz] = 0
    hz[:, :, nx] = 0; hz[:, ny, :] = 0
    return f


def random_materials(nx: int, ny: int, nz: int, seed: int, nmat: int = 5,
                     eps=(1.0, 12.0), sigma=(0.0, 0.05)):
    """Per-cell materials drawn from a small palette (float32, shape (nz,ny,nx))."""
    rng = np.random.default_rng(seed)
    pal_e = rng.uniform(*eps, size=nmat).astype(np.float32)
    pal_s = rng.uniform(*sigma, size=nmat).astype(np.float32)
    idx = rng.integers(0, nmat, size=(nz, ny, nx))
    return pal_e[idx], pal_s[idx]


def gaussian_pulse_source(bw: float = 10e9, amp: float = 1.0):
    """Gaussian-pulse source parameters (amp, f0=0, bw, t0, kind=1); t0 = 5 widths."""
    amp, _, bw, t0, _ = gaussian_sine_source(0.0, bw, amp)
    return amp, 0.0, bw, t0, 1


def design_cavity(n: int = 128, design: tuple = (48, 80), eps_range=(1.0, 4.0),
                  seed_design: int = 1305, seed_cells: int = 1306, ncells: int = 16):
    """The differentiation workload: an n^3 vacuum PEC cavity with a cubic design
    region of cells [lo, hi)^3 whose eps_r is seeded uniform in eps_range, a
    Gaussian-pulse Ez source 8 cells inside the x = 0 wall, the objective's Ez
    probe 9 cells inside the x = n wall, and `ncells` seeded design cells at
    which gradients are compared."""
    lo, hi = design
    eps = np.ones((n, n, n), np.float32)
    rng = np.random.default_rng(seed_design)
    m = hi - lo
    eps[lo:hi, lo:hi, lo:hi] = rng.uniform(*eps_range, size=(m, m, m)).astype(np.float32)
    sig = np.zeros((n, n, n), np.float32)
    amp, f0, bw, t0, kind = gaussian_pulse_source()
    src = (2, 8, n // 2, n // 2, amp, f0, bw, t0, kind)
    probe = (2, n - 9, n // 2, n // 2)
    g = SplitMix64(seed_cells)
    cells = []
    while len(cells) < ncells:
        c = (g.randint(lo, hi), g.randint(lo, hi), g.randint(lo, hi))
        if c not in cells:
            cells.append(c)
    return dict(nx=n, ny=n, nz=n, dx=DX_DEFAULT, dt=cfl_dt(DX_DEFAULT), eps=eps, sigma=sig,
                sources=[src], probe=probe, design=(lo, lo, lo, m, m, m), cells=cells)


def batch_cavities(ncav: int = 4096, size_range=(16, 96), eps_range=(1.0, 12.0), block: int = 4,
                   seed: int = 1304):
    """The batching workload: `ncav` PEC cavities with per-axis sizes uniform in
    size_range (inclusive), eps_r uniform in eps_range per block^3-cell block
    (partial blocks at the high edges), sigma = 0, and one Gaussian-pulse Ez
    source at a random interior edge of each cavity. Returns the sizes
    (ncav x 3, nx ny nz), the cavities' eps_r one after the other (x fastest
    within each) and the source tuples (cav, comp, i, j, k, amp, f0, bw, t0,
    kind)."""
    rng = np.random.default_rng(seed)
    lo, hi = size_range
    dims = rng.integers(lo, hi + 1, size=(ncav, 3))
    eps_parts = []
    sources = []
    amp, f0, bw, t0, kind = gaussian_pulse_source()
    for c in range(ncav):
        nx, ny, nz = (int(v) for v in dims[c])
        nb = [(n + block - 1) // block for n in (nz, ny, nx)]
        blocks = rng.uniform(*eps_range, size=nb).astype(np.float32)
        e = np.repeat(np.repeat(np.repeat(blocks, block, 0), block, 1), block, 2)[:nz, :ny, :nx]
        eps_parts.append(np.ascontiguousarray(e).ravel())
        i = int(rng.integers(1, max(2, nx)))
        j = int(rng.integers(1, max(2, ny)))
        k = int(rng.integers(0, nz))
        sources.append((c, 2, min(i, nx - 1), min(j, ny - 1), k, amp, f0, bw, t0, kind))
    return dims.astype(np.int32), np.concatenate(eps_parts), sources
