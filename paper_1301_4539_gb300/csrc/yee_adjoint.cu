// Discrete adjoint of the float leapfrog step (reverse-time Yee sweep), for
// gradients of a probe objective with respect to eps_r (sophie_grad_eps).
//
// One forward step n (Sec. 2.1 scheme, sophie.h):
//   h' = h + S * A(e)                    A = H-update bracket ("-curl")
//   e' = Ca*e + Cb*(B(h') + s)           B = E-update bracket ("curl")
// The two brackets are mutual negative transposes (A^T = -B: the discrete
// antisymmetry Sec. 2.1 requires for stability). Given the adjoints (le', lh')
// of (e', h'), the adjoints of (e, h) are
//   lh = lh' - A(Cb * le')               (the "H half" of the reverse step)
//   le = Ca * le' - S * B(lh)            (the "E half")
// and the step's coefficients receive
//   dJ/dCb += le' * (B(h') + s),   dJ/dCa += le' * e.
// So the reverse step is a Yee sweep on (le, lh) with the E values replaced by
// Cb*le in the H half and coefficients (Ca, -S) in the E half; PEC edges
// (Ca = Cb = 0) keep le = 0.
#include "sophie_internal.h"
#include "tma_util.cuh"
#include "yee_update.cuh"

namespace sophie {

namespace {

constexpr int kTX = 32, kTY = 8, kTZ = 16;

__device__ __forceinline__ float ldf(const float* f, const Dims& d, int c, int x, int y, int z) {
  if (x < 0 || x >= d.nxp || y < 0 || y >= d.ny1 || z < 0 || z >= d.nz1) return 0.f;
  return f[(long long)z * d.zstride + (long long)c * d.plane + (long long)y * d.nxp + x];
}

__device__ __forceinline__ uint32_t ldm(const uint32_t* m, const Dims& d, int x, int y, int z) {
  if (x < 0 || x >= d.nxp || y < 0 || y >= d.ny1 || z < 0 || z >= d.nz1) return 0u;
  return m[((long long)z * d.ny1 + y) * d.nxp + x];
}

// (Ca, Cb) of edge component c of material word m.
__device__ __forceinline__ float2 coef_of(const StepArgs& a, uint32_t m, int c) {
  if (m & kExpFlag) return a.ecoef[3ull * (m >> 3) + c];
  return a.coef[cls_of(m, c)];
}

// Cb * le at one index point, component c (the E values the H half uses).
__device__ __forceinline__ float w_at(const StepArgs& a, const float* l, const Dims& d, int c, int x, int y, int z) {
  const uint32_t m = ldm(a.mat, d, x, y, z);
  return __fmul_rn(coef_of(a, m, c).y, ldf(l, d, c, x, y, z));
}

// One reverse step: a.fin holds (le', lh'), a.fout receives (le, lh).
__global__ void __launch_bounds__((kTX + 1) * (kTY + 1)) adj_step_kernel(const __grid_constant__ StepArgs a) {
  __shared__ float sW[3][kTY + 2][kTX + 2];
  __shared__ float sH[3][kTY + 1][kTX + 1];
  const Dims d = a.d;
  const float* lin = static_cast<const float*>(a.fin);
  float* lout = static_cast<float*>(a.fout);
  const int tx = threadIdx.x % (kTX + 1), ty = threadIdx.x / (kTX + 1);
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * kTZ;
  const int z1 = min(z0 + kTZ, d.nz);
  const int x = x0 - 1 + tx, y = y0 - 1 + ty;
  const bool owner = tx >= 1 && ty >= 1 && x < d.nx && y < d.ny;
  const float S = a.S;
  float hxp = 0.f, hyp = 0.f;
  const int zs = z0 > 0 ? z0 - 1 : 0;
  for (int z = zs; z < z1; ++z) {
    for (int c = 0; c < 3; ++c) {
      sW[c][ty][tx] = w_at(a, lin, d, c, x, y, z);
      if (tx == kTX) sW[c][ty][tx + 1] = w_at(a, lin, d, c, x + 1, y, z);
      if (ty == kTY) sW[c][ty + 1][tx] = w_at(a, lin, d, c, x, y + 1, z);
    }
    __syncthreads();
    const float w0 = sW[0][ty][tx], w1 = sW[1][ty][tx], w2 = sW[2][ty][tx];
    const float w1n = w_at(a, lin, d, 1, x, y, z + 1), w0n = w_at(a, lin, d, 0, x, y, z + 1);
    // lh = lh' - A(Cb*le'): the H-update bracket with coefficient -1
    const float hx = h_upd(ldf(lin, d, 3, x, y, z), -1.f, w1n, w1, sW[2][ty + 1][tx], w2);
    const float hy = h_upd(ldf(lin, d, 4, x, y, z), -1.f, sW[2][ty][tx + 1], w2, w0n, w0);
    const float hz = h_upd(ldf(lin, d, 5, x, y, z), -1.f, sW[0][ty + 1][tx], w0, sW[1][ty][tx + 1], w1);
    sH[0][ty][tx] = hx;
    sH[1][ty][tx] = hy;
    sH[2][ty][tx] = hz;
    __syncthreads();
    if (z >= z0 && owner) {
      const uint32_t m = ldm(a.mat, d, x, y, z);
      float2 k[3];
      for (int c = 0; c < 3; ++c) {
        const float2 cc = coef_of(a, m, c);
        k[c] = cc.y == 0.f ? make_float2(0.f, 0.f) : make_float2(cc.x, -S);
      }
      const float bx = curl_br(hz, sH[2][ty - 1][tx], hy, hyp);
      const float by = curl_br(hx, hxp, hz, sH[2][ty][tx - 1]);
      const float bz = curl_br(hy, sH[1][ty][tx - 1], hx, sH[0][ty - 1][tx]);
      float* o = lout + (long long)z * d.zstride + (long long)y * d.nxp + x;
      o[0] = e_upd(ldf(lin, d, 0, x, y, z), k[0], bx);
      o[d.plane] = e_upd(ldf(lin, d, 1, x, y, z), k[1], by);
      o[2 * d.plane] = e_upd(ldf(lin, d, 2, x, y, z), k[2], bz);
      o[3 * d.plane] = hx;
      o[4 * d.plane] = hy;
      o[5 * d.plane] = hz;
    }
    hxp = hx;
    hyp = hy;
    __syncthreads();
  }
}

// After forward step n (fin: state before, fout: after): for every design
// edge, e^n (before) and the step's E bracket B(h^{n+1/2}) + s (after).
__global__ void gather_kernel(const __grid_constant__ StepArgs a, const int* edge_comp, const long long* edge_pt,
                              int nedge, float* e_out, float* c_out) {
  pdl_wait();  // launched like the step kernels, between them
  pdl_launch_dependents();
  const Dims d = a.d;
  const float* fo = static_cast<const float*>(a.fin);
  const float* fn = static_cast<const float*>(a.fout);
  const long long sy = d.nxp, sz = (long long)d.ny1 * d.nxp;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nedge) return;
  const int c = edge_comp[t];
  const long long pt = edge_pt[t];
  const long long z = pt / sz, r = pt % sz;
  e_out[t] = fo[z * d.zstride + (long long)c * d.plane + r];
  // H component f at in-plane offset r + dr of plane z + dz (post-step buffer)
  auto H = [&](int f, long long dr, int dz) {
    return fn[(z + dz) * d.zstride + (long long)f * d.plane + r + dr];
  };
  float br;
  if (c == 0)
    br = curl_br(H(5, 0, 0), H(5, -sy, 0), H(4, 0, 0), H(4, 0, -1));
  else if (c == 1)
    br = curl_br(H(3, 0, 0), H(3, 0, -1), H(5, 0, 0), H(5, -1, 0));
  else
    br = curl_br(H(4, 0, 0), H(4, -1, 0), H(3, 0, 0), H(3, -sy, 0));
  for (int q = 0; q < a.src.n; ++q)
    if (a.src.pos[q] == pt && a.src.comp[q] == c) br = __fadd_rn(br, a.src.val[(long long)q * a.src.cap + a.n0]);
  c_out[t] = br;
}

// dJ/dCb += le' * c, dJ/dCa += le' * e on the design edges (double).
__global__ void grad_accum_kernel(const float* l, Dims d, const int* edge_comp, const long long* edge_pt, int nedge,
                                  const float* e_in, const float* c_in, double* gcb, double* gca) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nedge) return;
  const long long sz = (long long)d.ny1 * d.nxp;
  const long long pt = edge_pt[t];
  const double le = l[(pt / sz) * d.zstride + (long long)edge_comp[t] * d.plane + pt % sz];
  gcb[t] += le * (double)c_in[t];
  gca[t] += le * (double)e_in[t];
}

// The objective's direct term l[comp at pt] += 2 dt f (f = sample[0]) and
// then the accumulation of grad_accum_kernel, in one launch: the objective's
// entry is read and written by one thread only (the design edge on it, t_obj,
// or the extra thread nedge when it is not a design edge), so no thread reads
// it while it changes.
__global__ void objective_grad_accum_kernel(float* l, Dims d, int comp, long long opt, const float* sample,
                                            double two_dt, int t_obj, const int* edge_comp, const long long* edge_pt,
                                            int nedge, const float* e_in, const float* c_in, double* gcb, double* gca) {
  pdl_wait();  // launched like the step kernels, between them
  pdl_launch_dependents();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > nedge) return;
  const long long sz = (long long)d.ny1 * d.nxp;
  if (t == (t_obj >= 0 ? t_obj : nedge)) {
    float* p = l + (opt / sz) * d.zstride + (long long)comp * d.plane + opt % sz;
    *p = __fadd_rn(*p, (float)(two_dt * (double)sample[0]));
  }
  if (t == nedge) return;
  const long long pt = edge_pt[t];
  const double le = l[(pt / sz) * d.zstride + (long long)edge_comp[t] * d.plane + pt % sz];
  gcb[t] += le * (double)c_in[t];
  gca[t] += le * (double)e_in[t];
}

// The objective's direct term: l[comp at pt] += 2 dt f, f = sample[0].
__global__ void add_objective_kernel(float* l, Dims d, int comp, long long pt, const float* sample, double two_dt) {
  const long long sz = (long long)d.ny1 * d.nxp;
  float* p = l + (pt / sz) * d.zstride + (long long)comp * d.plane + pt % sz;
  *p = __fadd_rn(*p, (float)(two_dt * (double)sample[0]));
}

}  // namespace

cudaError_t launch_adj_step(const StepArgs& a, cudaStream_t s) {
  dim3 grid((a.d.nx + kTX - 1) / kTX, (a.d.ny + kTY - 1) / kTY, (a.d.nz + kTZ - 1) / kTZ);
  adj_step_kernel<<<grid, (kTX + 1) * (kTY + 1), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather(const StepArgs& a, const int* edge_comp, const long long* edge_pt, int nedge, float* e_out,
                          float* c_out, cudaStream_t s) {
  if (nedge <= 0) return cudaSuccess;
  return launch_step_kernel(gather_kernel, dim3((nedge + 255) / 256), dim3(256), 0, s, a, edge_comp, edge_pt, nedge,
                            e_out, c_out);
}

cudaError_t launch_grad_accum(const float* l, const Dims& d, const int* edge_comp, const long long* edge_pt, int nedge,
                              const float* e_in, const float* c_in, double* gcb, double* gca, cudaStream_t s) {
  if (nedge <= 0) return cudaSuccess;
  grad_accum_kernel<<<(nedge + 255) / 256, 256, 0, s>>>(l, d, edge_comp, edge_pt, nedge, e_in, c_in, gcb, gca);
  return cudaGetLastError();
}

cudaError_t launch_objective_grad_accum(float* l, const Dims& d, int comp, long long pt, const float* sample,
                                        double two_dt, int t_obj, const int* edge_comp, const long long* edge_pt,
                                        int nedge, const float* e_in, const float* c_in, double* gcb, double* gca,
                                        cudaStream_t s) {
  return launch_step_kernel(objective_grad_accum_kernel, dim3((nedge + 1 + 255) / 256), dim3(256), 0, s, l, d, comp,
                            pt, sample, two_dt, t_obj, edge_comp, edge_pt, nedge, e_in, c_in, gcb, gca);
}

cudaError_t launch_add_objective(float* l, const Dims& d, int comp, long long pt, const float* sample, double two_dt,
                                 cudaStream_t s) {
  add_objective_kernel<<<1, 1, 0, s>>>(l, d, comp, pt, sample, two_dt);
  return cudaGetLastError();
}

}  // namespace sophie
