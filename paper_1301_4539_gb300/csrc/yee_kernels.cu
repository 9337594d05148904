// Support kernels of libsophie and the reference-layout step kernel.
//
// yee_step_simple: one fused H+E leapfrog step (Sec. 2.1; Sec. 3.2's
// interleave: H and E of a plane are updated in one pass, so each field is
// read and written once per step). Each CTA owns a 32x8 (x,y) tile and walks
// a chunk of z planes; the H values one cell outside the tile's -x/-y edges
// are recomputed (identically) by halo threads so that no CTA waits on
// another. Reads go straight to global memory; the tuned kernels stage tiles
// with TMA instead and share the update expressions of yee_update.cuh, so all
// step kernels give bitwise identical fields.
#include "sophie_internal.h"
#include "yee_store.cuh"
#include "yee_energy.cuh"
#include "yee_update.cuh"

namespace sophie {

namespace {

constexpr int kSTX = 32;
constexpr int kSTY = 8;
constexpr int kSZ = 16;  // z planes per CTA

__device__ __forceinline__ float ld_f(const float* f, const Dims& d, int c, int x, int y, int z) {
  if (x < 0 || x >= d.nxp || y < 0 || y >= d.ny1 || z < 0 || z >= d.nz1) return 0.f;
  return f[(long long)z * d.zstride + (long long)c * d.plane + (long long)y * d.nxp + x];
}

// NU: non-uniform mesh, every difference scaled by its ratio (a.rat).
template <bool NU>
__global__ void __launch_bounds__((kSTX + 1) * (kSTY + 1))
yee_step_simple_kernel(StepArgs a) {
  __shared__ float sE[3][kSTY + 2][kSTX + 2];
  __shared__ float sH[3][kSTY + 1][kSTX + 1];
  const Dims d = a.d;
  const float* fin = static_cast<const float*>(a.fin);  // float storage only
  const int tx = threadIdx.x % (kSTX + 1);
  const int ty = threadIdx.x / (kSTX + 1);
  const int x0 = blockIdx.x * kSTX, y0 = blockIdx.y * kSTY;
  const int z0 = blockIdx.z * kSZ;
  const int z1 = min(z0 + kSZ, d.nz);
  const int x = x0 - 1 + tx, y = y0 - 1 + ty;
  const float S = a.S;
  const bool owner = tx >= 1 && ty >= 1 && x < d.nx && y < d.ny;
  float hxp = 0.f, hyp = 0.f;  // new hx, hy of the plane below (own column)
  // h^{n+1/2} at plane z0-1 is only needed for hx, hy of this column; it is
  // recomputed in the first loop pass below (no store).
  const int zs = z0 > 0 ? z0 - 1 : 0;
  // Ratios of this thread's column and row (1 and unused on a uniform mesh).
  float rx = 1.f, ry = 1.f, rxd = 1.f, ryd = 1.f;
  if constexpr (NU) {
    rx = ratio_at(a.rat[0], x, d.nx);
    ry = ratio_at(a.rat[1], y, d.ny);
    rxd = ratio_at(a.rat[3], x, d.nx + 1);
    ryd = ratio_at(a.rat[4], y, d.ny + 1);
  }
  for (int z = zs; z < z1; ++z) {
    float rz = 1.f, rzd = 1.f;
    if constexpr (NU) {
      rz = __ldg(a.rat[2] + z);
      rzd = __ldg(a.rat[5] + z);
    }
    for (int c = 0; c < 3; ++c) {
      sE[c][ty][tx] = ld_f(fin, d, c, x, y, z);
      if (tx == kSTX) sE[c][ty][tx + 1] = ld_f(fin, d, c, x + 1, y, z);
      if (ty == kSTY) sE[c][ty + 1][tx] = ld_f(fin, d, c, x, y + 1, z);
    }
    __syncthreads();
    const float ex0 = sE[0][ty][tx], ey0 = sE[1][ty][tx], ez0 = sE[2][ty][tx];
    float hx = ld_f(fin, d, 3, x, y, z);
    float hy = ld_f(fin, d, 4, x, y, z);
    float hz = ld_f(fin, d, 5, x, y, z);
    const float ey1 = ld_f(fin, d, 1, x, y, z + 1);
    const float ex1 = ld_f(fin, d, 0, x, y, z + 1);
    hx = h_upd_r<NU>(hx, S, rz, ey1, ey0, ry, sE[2][ty + 1][tx], ez0);
    hy = h_upd_r<NU>(hy, S, rx, sE[2][ty][tx + 1], ez0, rz, ex1, ex0);
    hz = h_upd_r<NU>(hz, S, ry, sE[0][ty + 1][tx], ex0, rx, sE[1][ty][tx + 1], ey0);
    sH[0][ty][tx] = hx;
    sH[1][ty][tx] = hy;
    sH[2][ty][tx] = hz;
    __syncthreads();
    if (z >= z0 && owner) {
      const long long pt = ((long long)z * d.ny1 + y) * d.nxp + x;
      const uint32_t m = a.mat[pt];
      const bool ex_pt = (m & kExpFlag) != 0;
      const float2* e3 = a.ecoef + 3ull * (m >> 3);
      const float2 cx = ex_pt ? e3[0] : a.coef[cls_of(m, 0)];
      const float2 cy = ex_pt ? e3[1] : a.coef[cls_of(m, 1)];
      const float2 cz = ex_pt ? e3[2] : a.coef[cls_of(m, 2)];
      float bx = bracket<NU>(ryd, hz, sH[2][ty - 1][tx], rzd, hy, hyp);
      float by = bracket<NU>(rzd, hx, hxp, rxd, hz, sH[2][ty][tx - 1]);
      float bz = bracket<NU>(rxd, hy, sH[1][ty][tx - 1], ryd, hx, sH[0][ty - 1][tx]);
      if (m & kSrcFlag) {
        for (int s = 0; s < a.src.n; ++s) {
          if (a.src.pos[s] != pt) continue;
          const float v = a.src.val[(long long)s * a.src.cap + a.n0];
          if (a.src.comp[s] == 0) bx = __fadd_rn(bx, v);
          else if (a.src.comp[s] == 1) by = __fadd_rn(by, v);
          else bz = __fadd_rn(bz, v);
        }
      }
      const float ex = e_upd(ex0, cx, bx);
      const float ey = e_upd(ey0, cy, by);
      const float ez = e_upd(ez0, cz, bz);
      float* o = static_cast<float*>(a.fout) + (long long)z * d.zstride + (long long)y * d.nxp + x;
      o[0] = ex;
      o[d.plane] = ey;
      o[2 * d.plane] = ez;
      o[3 * d.plane] = hx;
      o[4 * d.plane] = hy;
      o[5 * d.plane] = hz;
      if (m & kPrbFlag) {
        const float v6[6] = {ex, ey, ez, hx, hy, hz};
        for (int p = 0; p < a.prb.n; ++p)
          if (a.prb.pos[p] == pt) a.prb.buf[(long long)p * a.prb.cap + a.n0] = v6[a.prb.comp[p]];
      }
    }
    hxp = hx;
    hyp = hy;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Discrete energy, Sec. 2.1 antisymmetric form (see sophie_energy in sophie.h),
// volume-weighted on a non-uniform mesh. Grid-stride over index points;
// fixed-order block tree; deterministic.
constexpr int kEThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kEThreads / 32; ++i) t += sh[i];
  return t;
}


template <int F, bool NU>
__global__ void __launch_bounds__(kEThreads)
energy_partial_kernel(const __grid_constant__ StepArgs a, const double* eps_tab, double* partials) {
  __shared__ double sh[kEThreads / 32];
  const Dims d = a.d;
  const float S = a.S;
  const float* isc = a.isc;
  const auto* f = static_cast<const typename Store<F>::T*>(a.fin);
  const uint32_t* mat = a.mat;
  const long long npts = (long long)d.nz1 * d.ny1 * d.nxp;
  double acc = 0.0;
  for (long long pt = (long long)blockIdx.x * kEThreads + threadIdx.x; pt < npts;
       pt += (long long)gridDim.x * kEThreads) {
    const int x = (int)(pt % d.nxp);
    const long long r = pt / d.nxp;
    const int y = (int)(r % d.ny1);
    const int z = (int)(r / d.ny1);
    if constexpr (NU)
      acc += point_energy_nu<F>(f, d, isc, S, mat[pt], eps_tab, a.eeps, a.rat, x, y, z);
    else
      acc += point_energy<F>(f, d, isc, S, mat[pt], eps_tab, a.eeps, x, y, z);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kEThreads)
energy_final_kernel(const double* partials, int n, double scale, double* out) {
  __shared__ double sh[kEThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kEThreads) acc += partials[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = t * scale;
}

// Zero PEC edges and entries outside a component's valid range (see sophie.h).
// kF24 storage: the component's high half and its byte of the byte-pair plane.
__global__ void mask_component_kernel(unsigned char* f, int esz, Dims d, int comp, int fmt) {
  const long long npts = (long long)d.nz1 * d.ny1 * d.nxp;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < npts;
       pt += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(pt % d.nxp);
    const long long r = pt / d.nxp;
    const int y = (int)(r % d.ny1);
    const int z = (int)(r / d.ny1);
    bool keep;
    switch (comp) {
      case 0: keep = x < d.nx && y >= 1 && y < d.ny && z >= 1 && z < d.nz; break;
      case 1: keep = x >= 1 && x < d.nx && y < d.ny && z >= 1 && z < d.nz; break;
      case 2: keep = x >= 1 && x < d.nx && y >= 1 && y < d.ny && z < d.nz; break;
      case 3: keep = x <= d.nx && y < d.ny && z < d.nz; break;
      case 4: keep = x < d.nx && y <= d.ny && z < d.nz; break;
      default: keep = x < d.nx && y < d.ny && z <= d.nz; break;
    }
    if (!keep) {
      const long long e = (long long)z * d.zstride + (long long)y * d.nxp + x;
      unsigned char* p = f + (e + (long long)comp * d.plane) * esz;
      for (int b = 0; b < esz; ++b) p[b] = 0;
      if (fmt == kF24) f[(e + (long long)(6 + comp / 2) * d.plane) * esz + (comp & 1)] = 0;
    }
  }
}

__global__ void or_flag_kernel(uint32_t* mat, long long pos, uint32_t bit) { mat[pos] |= bit; }

}  // namespace

cudaError_t launch_step_simple(const StepArgs& a, cudaStream_t s) {
  dim3 grid((a.d.nx + kSTX - 1) / kSTX, (a.d.ny + kSTY - 1) / kSTY, (a.d.nz + kSZ - 1) / kSZ);
  if (a.rat[0])
    yee_step_simple_kernel<true><<<grid, (kSTX + 1) * (kSTY + 1), 0, s>>>(a);
  else
    yee_step_simple_kernel<false><<<grid, (kSTX + 1) * (kSTY + 1), 0, s>>>(a);
  return cudaGetLastError();
}

int energy_blocks(const Dims& d) {
  const long long npts = (long long)d.nz1 * d.ny1 * d.nxp;
  long long b = (npts + kEThreads * 8 - 1) / (kEThreads * 8);
  if (b < 1) b = 1;
  if (b > kEnergyMaxBlocks) b = kEnergyMaxBlocks;
  return (int)b;
}

template <int F>
cudaError_t launch_energy_f(const StepArgs& a, const double* eps_tab, double* partials, int nblocks, double scale,
                            double* out, cudaStream_t s) {
  if (a.rat[0])
    energy_partial_kernel<F, true><<<nblocks, kEThreads, 0, s>>>(a, eps_tab, partials);
  else
    energy_partial_kernel<F, false><<<nblocks, kEThreads, 0, s>>>(a, eps_tab, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  energy_final_kernel<<<1, kEThreads, 0, s>>>(partials, nblocks, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_scaled(const StepArgs& a, const double* eps_tab, double* partials, int nblocks,
                                 double scale, double* out, cudaStream_t s) {
  switch (a.fmt) {
    case kF32: return launch_energy_f<kF32>(a, eps_tab, partials, nblocks, scale, out, s);
    case kF16: return launch_energy_f<kF16>(a, eps_tab, partials, nblocks, scale, out, s);
    case kBF16: return launch_energy_f<kBF16>(a, eps_tab, partials, nblocks, scale, out, s);
    case kF16HL: return launch_energy_f<kF16HL>(a, eps_tab, partials, nblocks, scale, out, s);
    case kF24: return launch_energy_f<kF24>(a, eps_tab, partials, nblocks, scale, out, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_energy(const StepArgs& a, const double* eps_tab, double* partials, int nblocks, double* out,
                          cudaStream_t s) {
  return launch_energy_scaled(a, eps_tab, partials, nblocks, 1.0, out, s);
}

cudaError_t launch_mask_component(void* f, int esz, const Dims& d, int comp, cudaStream_t s, int fmt) {
  mask_component_kernel<<<152 * 4, 256, 0, s>>>(static_cast<unsigned char*>(f), esz, d, comp, fmt);
  return cudaGetLastError();
}

cudaError_t launch_or_flag(uint32_t* mat, long long pos, uint32_t bit, cudaStream_t s) {
  or_flag_kernel<<<1, 1, 0, s>>>(mat, pos, bit);
  return cudaGetLastError();
}

}  // namespace sophie
