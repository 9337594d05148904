"""Closed-form discrete eigenmodes of a PEC Yee cavity (test helpers).

Derived here from the scheme of Sec. 2.1 (not from any implementation): in
index units, with kx = m pi / nx, ky = n pi / ny, kz = p pi / nz and
sig_a = 2 sin(k_a / 2), the fields

  ex(i,j,k) = Ex cos(kx(i+1/2)) sin(ky j) sin(kz k)
  ey(i,j,k) = Ey sin(kx i) cos(ky(j+1/2)) sin(kz k)
  ez(i,j,k) = Ez sin(kx i) sin(ky j) cos(kz(k+1/2))

vanish on the walls and satisfy div e = 0 at the nodes iff E . sig = 0. One H
half step maps them to (S E x sig) times

  hx ~ sin(kx i) cos(ky(j+1/2)) cos(kz(k+1/2))
  hy ~ cos(kx(i+1/2)) sin(ky j) cos(kz(k+1/2))
  hz ~ cos(kx(i+1/2)) cos(ky(j+1/2)) sin(kz k)

and one E step maps h back with (H x sig). Hence, in a uniform medium eps_r
with no loss, e^n = E cos(w n dt) and h^{n-1/2} = H sin(w (n-1/2) dt) with
H = S (E x sig) / (2 sin(w dt/2)) and the discrete dispersion relation
sin^2(w dt / 2) = S^2 |sig|^2 / (4 eps_r), i.e. for eps_r = 1
sin^2(w dt/2)/(c dt)^2 = sum_a sin^2(k_a dx/2)/dx^2.

With loss, writing e^n = a_n E and h^{n+1/2} = b_n S (E x sig), the scheme
reduces to the scalar recurrence
  b_n = b_{n-1} + a_n,   (1+beta) a_{n+1} = (1-beta) a_n - (S^2 |sig|^2 / eps_r) b_n.
"""

from __future__ import annotations

import math

import numpy as np


def _grids(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)


class CavityMode:
    def __init__(self, nx, ny, nz, m, n, p, pol, S, eps_r=1.0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.kx, self.ky, self.kz = m * math.pi / nx, n * math.pi / ny, p * math.pi / nz
        self.sig = np.array([2 * math.sin(self.kx / 2), 2 * math.sin(self.ky / 2),
                             2 * math.sin(self.kz / 2)])
        E = np.asarray(pol, np.float64)
        assert abs(E @ self.sig) < 1e-12 * max(1.0, np.abs(E).max()), "E must be orthogonal to sig"
        self.E = E
        self.S = float(S)
        self.eps_r = float(eps_r)
        s2 = self.S ** 2 * (self.sig @ self.sig) / (4.0 * self.eps_r)
        assert 0 < s2 < 1
        self.half = math.sqrt(s2)                 # sin(w dt / 2)
        self.wdt = 2.0 * math.asin(self.half)     # w dt
        self.H = self.S * np.cross(E, self.sig) / (2.0 * self.half)

    @staticmethod
    def sig_of(nx, ny, nz, m, n, p):
        return np.array([2 * math.sin(m * math.pi / nx / 2), 2 * math.sin(n * math.pi / ny / 2),
                         2 * math.sin(p * math.pi / nz / 2)])

    @classmethod
    def transverse(cls, nx, ny, nz, m, n, p, u, S, eps_r=1.0):
        """Mode whose polarisation is sig x u (always divergence free)."""
        E = np.cross(cls.sig_of(nx, ny, nz, m, n, p), np.asarray(u, np.float64))
        return cls(nx, ny, nz, m, n, p, E, S, eps_r)

    # spatial shapes
    def e_shapes(self):
        i, j, k = _grids(self.nx, self.ny, self.nz)
        kx, ky, kz = self.kx, self.ky, self.kz
        ex = np.cos(kx * (i + 0.5)) * np.sin(ky * j) * np.sin(kz * k)
        ey = np.sin(kx * i) * np.cos(ky * (j + 0.5)) * np.sin(kz * k)
        ez = np.sin(kx * i) * np.sin(ky * j) * np.cos(kz * (k + 0.5))
        return self._mask_e(ex, ey, ez)

    def h_shapes(self):
        i, j, k = _grids(self.nx, self.ny, self.nz)
        kx, ky, kz = self.kx, self.ky, self.kz
        hx = np.sin(kx * i) * np.cos(ky * (j + 0.5)) * np.cos(kz * (k + 0.5))
        hy = np.cos(kx * (i + 0.5)) * np.sin(ky * j) * np.cos(kz * (k + 0.5))
        hz = np.cos(kx * (i + 0.5)) * np.cos(ky * (j + 0.5)) * np.sin(kz * k)
        return self._mask_h(hx, hy, hz)

    def _mask_e(self, ex, ey, ez):
        nx, ny, nz = self.nx, self.ny, self.nz
        ex[:, :, nx] = 0; ex[:, 0, :] = 0; ex[:, ny, :] = 0; ex[0] = 0; ex[nz] = 0
        ey[:, ny, :] = 0; ey[:, :, 0] = 0; ey[:, :, nx] = 0; ey[0] = 0; ey[nz] = 0
        ez[nz] = 0; ez[:, :, 0] = 0; ez[:, :, nx] = 0; ez[:, 0, :] = 0; ez[:, ny, :] = 0
        return ex, ey, ez

    def _mask_h(self, hx, hy, hz):
        nx, ny, nz = self.nx, self.ny, self.nz
        hx[:, ny, :] = 0; hx[nz] = 0
        hy[:, :, nx] = 0; hy[nz] = 0
        hz[:, :, nx] = 0; hz[:, ny, :] = 0
        return hx, hy, hz

    def state(self, n):
        """(ex, ey, ez, hx, hy, hz) holding e^n and h^{n-1/2}, float64."""
        ce = math.cos(self.wdt * n)
        sh = math.sin(self.wdt * (n - 0.5))
        es = self.e_shapes()
        hs = self.h_shapes()
        return ([self.E[a] * ce * es[a] for a in range(3)] +
                [self.H[a] * sh * hs[a] for a in range(3)])


def lossy_mode_amplitudes(S2sig2_over_eps, beta, nsteps, a0=1.0, bm1=None):
    """Scalar recurrence of a lossy mode; returns a_n for n = 0..nsteps."""
    q = S2sig2_over_eps
    a = a0
    b = 0.0 if bm1 is None else bm1
    out = [a]
    for _ in range(nsteps):
        b = b + a
        a = ((1.0 - beta) * a - q * b) / (1.0 + beta)
        out.append(a)
    return np.array(out)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = math.sqrt(float((b * b).sum()))
    return math.sqrt(float(((a - b) ** 2).sum())) / (den if den > 0 else 1.0)
