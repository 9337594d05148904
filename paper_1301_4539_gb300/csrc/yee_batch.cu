// Batched cavities: many independent PEC cavities of different sizes, each
// with its own fields, material words and coefficient tables, advanced one
// leapfrog step (Sec. 2.1, fused H+E per plane as in Sec. 3.2-3.3) per
// launch by one persistent kernel.
//
// Work list: items (cavity, 32 x TY tile, z chunk). Persistent CTAs (as many
// as fit on the GPU) take items from a global counter in list order, so the
// uneven cavities balance themselves; the counter only grows and every CTA
// stops when it passes the end of the list (no waiting on other CTAs). Each
// item runs the plane-by-plane update with direct, coalesced loads: E of a
// plane (plus one halo row/column) goes through shared memory, H of the plane
// below stays in registers, and the H values one cell outside the tile's -x
// and -y edges are recomputed by halo threads so that items never depend on
// each other. The update expressions are those of yee_update.cuh, so every
// cavity's fields are bitwise those of a separate single-grid run.
#include "sophie_internal.h"
#include "yee_energy.cuh"
#include "yee_update.cuh"

namespace sophie {

namespace {

constexpr int kBTX = 32;
constexpr int kEThreadsB = 256;

__device__ __forceinline__ float ldb(const float* f, const Dims& d, int c, int x, int y, int z) {
  if (x < 0 || x >= d.nxp || y < 0 || y >= d.ny1 || z < 0 || z >= d.nz1) return 0.f;
  return f[(long long)z * d.zstride + (long long)c * d.plane + (long long)y * d.nxp + x];
}

template <int TY>
__global__ void __launch_bounds__((kBTX + 1) * (TY + 1))
yee_batch_kernel(const CavityDesc* __restrict__ descs, const BatchItem* __restrict__ items, int nitems, int* counter,
                 int cur, float S, long long nstep) {
  __shared__ float sE[3][TY + 2][kBTX + 2];
  __shared__ float sH[3][TY + 1][kBTX + 1];
  __shared__ int s_item;
  const int tx = threadIdx.x % (kBTX + 1);
  const int ty = threadIdx.x / (kBTX + 1);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) return;  // uniform: every thread read the same value
    const BatchItem w = items[it];
    const CavityDesc* cd = descs + w.cav;
    const Dims d = cd->d;
    const float* fin = static_cast<const float*>(cd->F[cur]);
    float* fout = static_cast<float*>(cd->F[1 - cur]);
    const uint32_t* mat = cd->mat;
    const int x = w.x0 - 1 + tx, y = w.y0 - 1 + ty;
    const bool owner = tx >= 1 && ty >= 1 && x < d.nx && y < d.ny;
    float hxp = 0.f, hyp = 0.f;
    const int zs = w.z0 > 0 ? w.z0 - 1 : 0;
    for (int z = zs; z < w.z1; ++z) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sE[c][ty][tx] = ldb(fin, d, c, x, y, z);
        if (tx == kBTX) sE[c][ty][tx + 1] = ldb(fin, d, c, x + 1, y, z);
        if (ty == TY) sE[c][ty + 1][tx] = ldb(fin, d, c, x, y + 1, z);
      }
      __syncthreads();
      const float ex0 = sE[0][ty][tx], ey0 = sE[1][ty][tx], ez0 = sE[2][ty][tx];
      const float ey1 = ldb(fin, d, 1, x, y, z + 1);
      const float ex1 = ldb(fin, d, 0, x, y, z + 1);
      const float hx = h_upd(ldb(fin, d, 3, x, y, z), S, ey1, ey0, sE[2][ty + 1][tx], ez0);
      const float hy = h_upd(ldb(fin, d, 4, x, y, z), S, sE[2][ty][tx + 1], ez0, ex1, ex0);
      const float hz = h_upd(ldb(fin, d, 5, x, y, z), S, sE[0][ty + 1][tx], ex0, sE[1][ty][tx + 1], ey0);
      sH[0][ty][tx] = hx;
      sH[1][ty][tx] = hy;
      sH[2][ty][tx] = hz;
      __syncthreads();
      if (z >= w.z0 && owner) {
        const long long pt = ((long long)z * d.ny1 + y) * d.nxp + x;
        const uint32_t m = mat[pt];
        float2 k0, k1, k2;
        if (m & kExpFlag) {
          const float2* e3 = cd->ecoef + 3ull * (m >> 3);
          k0 = e3[0];
          k1 = e3[1];
          k2 = e3[2];
        } else {
          k0 = cd->coef[cls_of(m, 0)];
          k1 = cd->coef[cls_of(m, 1)];
          k2 = cd->coef[cls_of(m, 2)];
        }
        float bx = curl_br(hz, sH[2][ty - 1][tx], hy, hyp);
        float by = curl_br(hx, hxp, hz, sH[2][ty][tx - 1]);
        float bz = curl_br(hy, sH[1][ty][tx - 1], hx, sH[0][ty - 1][tx]);
        if (m & kSrcFlag) {
          const SrcTable* st = &cd->src;
          for (int q = 0; q < st->n; ++q) {
            if (st->pos[q] != pt) continue;
            const float v = st->val[(long long)q * st->cap + nstep];
            if (st->comp[q] == 0) bx = __fadd_rn(bx, v);
            else if (st->comp[q] == 1) by = __fadd_rn(by, v);
            else bz = __fadd_rn(bz, v);
          }
        }
        float* o = fout + (long long)z * d.zstride + (long long)y * d.nxp + x;
        o[0] = e_upd(ex0, k0, bx);
        o[d.plane] = e_upd(ey0, k1, by);
        o[2 * d.plane] = e_upd(ez0, k2, bz);
        o[3 * d.plane] = hx;
        o[4 * d.plane] = hy;
        o[5 * d.plane] = hz;
      }
      hxp = hx;
      hyp = hy;
      __syncthreads();
    }
    __syncthreads();  // s_item is rewritten only after every thread has read it
  }
}

// Energy of every cavity: items (cavity, range of index points) give partial
// sums; each cavity's partials are then added in item order (deterministic).
__global__ void __launch_bounds__(kEThreadsB)
batch_energy_partial_kernel(const CavityDesc* __restrict__ descs, const EnergyItem* __restrict__ items, int cur,
                            float S, double* partials) {
  __shared__ double sh[kEThreadsB / 32];
  const EnergyItem w = items[blockIdx.x];
  const CavityDesc* cd = descs + w.cav;
  const Dims d = cd->d;
  const float* f = static_cast<const float*>(cd->F[cur]);
  const float isc[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
  double acc = 0.0;
  for (long long pt = w.p0 + threadIdx.x; pt < w.p1; pt += kEThreadsB) {
    const int x = (int)(pt % d.nxp);
    const long long r = pt / d.nxp;
    const int y = (int)(r % d.ny1);
    const int z = (int)(r / d.ny1);
    acc += point_energy<kF32>(f, d, isc, S, cd->mat[pt], cd->eps_tab, cd->eeps, x, y, z);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kEThreadsB / 32; ++i) t += sh[i];
    partials[blockIdx.x] = t;
  }
}

__global__ void batch_energy_final_kernel(const int* first, int ncav, const double* partials, double scale,
                                          double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncav) return;
  double t = 0.0;
  for (int i = first[c]; i < first[c + 1]; ++i) t += partials[i];
  out[c] = t * scale;
}

}  // namespace

bool batch_tile_supported(int ty) { return ty == 4 || ty == 8 || ty == 16; }

int batch_blocks_per_sm(int ty) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const int threads = (kBTX + 1) * (ty + 1);
  if (ty == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, yee_batch_kernel<4>, threads, 0);
  if (ty == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, yee_batch_kernel<8>, threads, 0);
  if (ty == 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, yee_batch_kernel<16>, threads, 0);
  return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t launch_batch_step(const CavityDesc* descs, const BatchItem* items, int nitems, int* counter, int cur,
                              float S, long long nstep, int ty, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int threads = (kBTX + 1) * (ty + 1);
  switch (ty) {
    case 4: yee_batch_kernel<4><<<grid, threads, 0, s>>>(descs, items, nitems, counter, cur, S, nstep); break;
    case 8: yee_batch_kernel<8><<<grid, threads, 0, s>>>(descs, items, nitems, counter, cur, S, nstep); break;
    case 16: yee_batch_kernel<16><<<grid, threads, 0, s>>>(descs, items, nitems, counter, cur, S, nstep); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_energy(const CavityDesc* descs, const EnergyItem* items, int nitems, const int* first,
                                int ncav, int cur, float S, double* partials, double scale, double* out,
                                cudaStream_t s) {
  if (nitems > 0) batch_energy_partial_kernel<<<nitems, kEThreadsB, 0, s>>>(descs, items, cur, S, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_energy_final_kernel<<<(ncav + 127) / 128, 128, 0, s>>>(first, ncav, partials, scale, out);
  return cudaGetLastError();
}

}  // namespace sophie
