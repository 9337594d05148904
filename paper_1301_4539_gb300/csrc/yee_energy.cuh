// Per-index-point term of the discrete Yee energy (Sec. 2.1 antisymmetric
// form), shared by the single-grid and batched energy kernels:
//   sum over the point's three edges of eps_r(edge) (e^n)^2
//   + sum over its three faces of h^{n-1/2} h^{n+1/2},
// h^{n+1/2} formed with the float H update and never stored; double products.
#pragma once

#include "sophie_internal.h"
#include "yee_store.cuh"
#include "yee_update.cuh"

namespace sophie {

template <int F>
__device__ __forceinline__ float ld_s(const typename Store<F>::T* f, const Dims& d, const float* isc, int c, int x,
                                      int y, int z) {
  if (x < 0 || x >= d.nxp || y < 0 || y >= d.ny1 || z < 0 || z >= d.nz1) return 0.f;
  return ldc<F>(f + (long long)z * d.zstride + (long long)c * d.plane + (long long)y * d.nxp + x, isc[c], c, d.plane);
}

template <int F>
__device__ __forceinline__ double point_energy(const typename Store<F>::T* f, const Dims& d, const float* isc,
                                               float S, uint32_t m, const double* eps_tab, const double* eeps, int x,
                                               int y, int z) {
  const float ex = ld_s<F>(f, d, isc, 0, x, y, z), ey = ld_s<F>(f, d, isc, 1, x, y, z);
  const float ez = ld_s<F>(f, d, isc, 2, x, y, z);
  double e0, e1, e2;
  if (m & kExpFlag) {
    const double* p3 = eeps + 3ull * (m >> 3);
    e0 = p3[0];
    e1 = p3[1];
    e2 = p3[2];
  } else {
    e0 = eps_tab[cls_of(m, 0)];
    e1 = eps_tab[cls_of(m, 1)];
    e2 = eps_tab[cls_of(m, 2)];
  }
  double acc = e0 * ((double)ex * (double)ex);
  acc += e1 * ((double)ey * (double)ey);
  acc += e2 * ((double)ez * (double)ez);
  const float hx = ld_s<F>(f, d, isc, 3, x, y, z), hy = ld_s<F>(f, d, isc, 4, x, y, z);
  const float hz = ld_s<F>(f, d, isc, 5, x, y, z);
  const float hxn = h_upd(hx, S, ld_s<F>(f, d, isc, 1, x, y, z + 1), ey, ld_s<F>(f, d, isc, 2, x, y + 1, z), ez);
  const float hyn = h_upd(hy, S, ld_s<F>(f, d, isc, 2, x + 1, y, z), ez, ld_s<F>(f, d, isc, 0, x, y, z + 1), ex);
  const float hzn = h_upd(hz, S, ld_s<F>(f, d, isc, 0, x, y + 1, z), ex, ld_s<F>(f, d, isc, 1, x + 1, y, z), ey);
  acc += (double)hx * (double)hxn;
  acc += (double)hy * (double)hyn;
  acc += (double)hz * (double)hzn;
  return acc;
}

// The same term on a non-uniform mesh: each edge and face weighted by its
// volume in units of the reference cell -- 1 / (product of the ratios of the
// widths it spans: its own length and its dual face, or its area and its dual
// edge) -- formed in double from the float ratios, and h^{n+1/2} formed with
// the scaled H update. Components outside their index range contribute
// nothing (their stored values are zero, their weights undefined).
template <int F>
__device__ __forceinline__ double point_energy_nu(const typename Store<F>::T* f, const Dims& d, const float* isc,
                                                  float S, uint32_t m, const double* eps_tab, const double* eeps,
                                                  const float* const* rat, int x, int y, int z) {
  const float rx = ratio_at(rat[0], x, d.nx), ry = ratio_at(rat[1], y, d.ny), rz = ratio_at(rat[2], z, d.nz);
  const float rxd = ratio_at(rat[3], x, d.nx + 1), ryd = ratio_at(rat[4], y, d.ny + 1);
  const float rzd = ratio_at(rat[5], z, d.nz + 1);
  const bool xi = x < d.nx, yi = y < d.ny, zi = z < d.nz;  // primary index in range
  const bool xd = x >= 1 && x < d.nx, yd = y >= 1 && y < d.ny, zd = z >= 1 && z < d.nz;  // interior node
  const float ex = ld_s<F>(f, d, isc, 0, x, y, z), ey = ld_s<F>(f, d, isc, 1, x, y, z);
  const float ez = ld_s<F>(f, d, isc, 2, x, y, z);
  double e0, e1, e2;
  if (m & kExpFlag) {
    const double* p3 = eeps + 3ull * (m >> 3);
    e0 = p3[0];
    e1 = p3[1];
    e2 = p3[2];
  } else {
    e0 = eps_tab[cls_of(m, 0)];
    e1 = eps_tab[cls_of(m, 1)];
    e2 = eps_tab[cls_of(m, 2)];
  }
  auto w = [](float a, float b, float c) { return 1.0 / (((double)a * (double)b) * (double)c); };
  double acc = 0.0;
  if (xi && yd && zd) acc += w(rx, ryd, rzd) * (e0 * ((double)ex * (double)ex));
  if (xd && yi && zd) acc += w(rxd, ry, rzd) * (e1 * ((double)ey * (double)ey));
  if (xd && yd && zi) acc += w(rxd, ryd, rz) * (e2 * ((double)ez * (double)ez));
  if (x <= d.nx && yi && zi) {
    const float hx = ld_s<F>(f, d, isc, 3, x, y, z);
    const float hn = h_upd_r<true>(hx, S, rz, ld_s<F>(f, d, isc, 1, x, y, z + 1), ey, ry,
                                   ld_s<F>(f, d, isc, 2, x, y + 1, z), ez);
    acc += w(rxd, ry, rz) * ((double)hx * (double)hn);
  }
  if (xi && y <= d.ny && zi) {
    const float hy = ld_s<F>(f, d, isc, 4, x, y, z);
    const float hn = h_upd_r<true>(hy, S, rx, ld_s<F>(f, d, isc, 2, x + 1, y, z), ez, rz,
                                   ld_s<F>(f, d, isc, 0, x, y, z + 1), ex);
    acc += w(rx, ryd, rz) * ((double)hy * (double)hn);
  }
  if (xi && yi && z <= d.nz) {
    const float hz = ld_s<F>(f, d, isc, 5, x, y, z);
    const float hn = h_upd_r<true>(hz, S, ry, ld_s<F>(f, d, isc, 0, x, y + 1, z), ex, rx,
                                   ld_s<F>(f, d, isc, 1, x + 1, y, z), ey);
    acc += w(rx, ry, rzd) * ((double)hz * (double)hn);
  }
  return acc;
}

}  // namespace sophie
