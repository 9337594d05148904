// Host runtime of libsophie: the C ABI declared in include/sophie.h.
//
// Owns the grid handle, device memory (two ping-pong copies of the six fields,
// the per-point material words and class tables), source waveform tables,
// probe buffers, the energy reduction and error reporting. Every step of the
// method runs in the CUDA kernels; this file validates arguments, builds
// tables and enqueues launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/sophie.h"
#include "grid_state.h"
#include "sophie_internal.h"
#include "yee_store.cuh"

using namespace sophie;
using namespace sophie::grid;

namespace {
thread_local std::string g_err;
}  // namespace

namespace sophie {
namespace grid {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

}  // namespace grid

int report_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

namespace {
std::atomic<long long> g_fail_alloc_at{0};  // > 0: the n-th next allocation fails
std::mutex g_live_mu;
std::unordered_set<const void*> g_live;  // handles returned by the create calls
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  long long n = g_fail_alloc_at.load();
  while (n > 0 && !g_fail_alloc_at.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

void handle_register(const void* h) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  g_live.insert(h);
}

bool handle_release(const void* h) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  return g_live.erase(h) == 1;
}
}  // namespace sophie


namespace sophie {
namespace grid {

long long point_index(const Dims& d, int i, int j, int k) {
  return ((long long)k * d.ny1 + j) * d.nxp + i;
}

bool e_edge_interior(const Dims& d, int c, int i, int j, int k) {
  switch (c) {
    case 0: return i >= 0 && i < d.nx && j >= 1 && j < d.ny && k >= 1 && k < d.nz;
    case 1: return i >= 1 && i < d.nx && j >= 0 && j < d.ny && k >= 1 && k < d.nz;
    default: return i >= 1 && i < d.nx && j >= 1 && j < d.ny && k >= 0 && k < d.nz;
  }
}

bool comp_valid(const Dims& d, int c, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i > d.nx || j > d.ny || k > d.nz) return false;
  switch (c) {
    case 0: return i < d.nx;
    case 1: return j < d.ny;
    case 2: return k < d.nz;
    case 3: return j < d.ny && k < d.nz;
    case 4: return i < d.nx && k < d.nz;
    default: return i < d.nx && j < d.ny;
  }
}

}  // namespace grid
}  // namespace sophie

namespace {

// Fill g->mat_host and the host tables for per-cell eps/sigma (nullptr =
// vacuum); sources and probes flag their points.
int build_material_words(sophie_grid* g, const float* eps, const float* sig) {
  MaterialTables t;
  const int nth = std::max(1, std::min(32, (int)std::thread::hardware_concurrency()));
  if (build_material_tables(g->d, g->dt, g->S64, eps, sig, g->mat_host, &t, nth) != 0)
    return fail(SOPHIE_ETOOMANYMAT, "more than 2^29 explicit material points");
  uint32_t* w = g->mat_host;
  for (const Source& s : g->src) w[s.pos] |= kSrcFlag;
  for (const Probe& p : g->prb)
    if (!p.fixed) w[p.pos] |= kPrbFlag;
  g->coef_h = std::move(t.coef);
  g->eps_h = std::move(t.eps);
  g->sig_h = std::move(t.sig);
  g->ecoef_h = std::move(t.ecoef);
  g->eeps_h = std::move(t.eeps);
  g->esig_h = std::move(t.esig);
  return SOPHIE_OK;
}

}  // namespace

namespace sophie {
namespace grid {

int upload_materials(sophie_grid* g) {
  const Dims& d = g->d;
  const size_t npts = (size_t)d.nz1 * d.ny1 * d.nxp;
  CUDA_TRY(cudaMemcpyAsync(g->mat, g->mat_host, npts * 4, cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaMemcpyAsync(g->coef, g->coef_h.data(), g->coef_h.size() * sizeof(float2),
                           cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaMemcpyAsync(g->eps_tab, g->eps_h.data(), g->eps_h.size() * sizeof(double),
                           cudaMemcpyHostToDevice, g->stream));
  const size_t nexp = g->eeps_h.size() / 3;
  if (nexp > g->exp_cap) {
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->ecoef) cudaFree(g->ecoef);
    if (g->eeps) cudaFree(g->eeps);
    g->ecoef = nullptr;
    g->eeps = nullptr;
    g->exp_cap = 0;
    if (dev_malloc((void**)&g->ecoef, nexp * 3 * sizeof(float2)) != cudaSuccess ||
        dev_malloc((void**)&g->eeps, nexp * 3 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SOPHIE_ENOMEM, "explicit material table allocation failed");
    }
    g->exp_cap = nexp;
  }
  if (nexp) {
    CUDA_TRY(cudaMemcpyAsync(g->ecoef, g->ecoef_h.data(), nexp * 3 * sizeof(float2), cudaMemcpyHostToDevice,
                             g->stream));
    CUDA_TRY(cudaMemcpyAsync(g->eeps, g->eeps_h.data(), nexp * 3 * sizeof(double), cudaMemcpyHostToDevice,
                             g->stream));
  }
  CUDA_TRY(cudaEventRecord(g->mat_upload_done, g->stream));
  // The tables are pageable host memory: the copies above complete before return.
  return SOPHIE_OK;
}

}  // namespace grid
}  // namespace sophie

namespace {

double waveform(const Source& s, long long n, double dt) {
  return source_waveform(s.kind, s.amp, s.f0, s.bw, s.t0, dt, n);
}

// Make the source table cover steps [0, need) and the probe buffer [0, need).
}  // namespace

namespace sophie {
namespace grid {
int ensure_capacity(sophie_grid* g, long long need) {
  if (need > (1ll << 30)) return fail(SOPHIE_EINVAL, "step count too large");
  if (need > g->scap) {
    int cap = g->scap ? g->scap : 4096;
    while (cap < need) cap *= 2;
    std::vector<float> h((size_t)kMaxSources * cap, 0.f);
    for (size_t s = 0; s < g->src.size(); ++s)
      for (int m = 0; m < cap; ++m) h[s * cap + m] = (float)waveform(g->src[s], m, g->dt);
    float* dnew = nullptr;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (dev_malloc((void**)&dnew, h.size() * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(SOPHIE_ENOMEM, "source table allocation failed");
    }
    CUDA_TRY(cudaMemcpy(dnew, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
    if (g->sval) cudaFree(g->sval);
    g->sval = dnew;
    g->scap = cap;
  }
  if (need > g->pcap) {
    int cap = g->pcap ? g->pcap : 4096;
    while (cap < need) cap *= 2;
    float* dnew = nullptr;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (dev_malloc((void**)&dnew, (size_t)kMaxProbes * cap * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(SOPHIE_ENOMEM, "probe buffer allocation failed");
    }
    CUDA_TRY(cudaMemset(dnew, 0, (size_t)kMaxProbes * cap * 4));
    if (g->pbuf) {
      CUDA_TRY(cudaMemcpy2D(dnew, (size_t)cap * 4, g->pbuf, (size_t)g->pcap * 4, (size_t)g->pcap * 4,
                            kMaxProbes, cudaMemcpyDeviceToDevice));
      cudaFree(g->pbuf);
    }
    g->pbuf = dnew;
    g->pcap = cap;
  }
  return SOPHIE_OK;
}
}  // namespace grid
}  // namespace sophie

namespace {

// Rebuild one source's waveform column after it was added.
int refresh_source_table(sophie_grid* g, int s) {
  if (!g->sval) return SOPHIE_OK;
  std::vector<float> h(g->scap);
  for (int m = 0; m < g->scap; ++m) h[m] = (float)waveform(g->src[s], m, g->dt);
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  CUDA_TRY(cudaMemcpy(g->sval + (size_t)s * g->scap, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
  return SOPHIE_OK;
}

}  // namespace

namespace sophie {
namespace grid {
cudaEvent_t prof_event(sophie_grid* g) {
  if (!g->ev_pool.empty()) {
    cudaEvent_t e = g->ev_pool.back();
    g->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_drain(sophie_grid* g) {
  if (g->prof_live.empty()) return SOPHIE_OK;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  for (ProfEntry& p : g->prof_live) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g->prof_count[p.kernel] += 1;
      g->prof_ms[p.kernel] += ms;
    }
    g->ev_pool.push_back(p.a);
    g->ev_pool.push_back(p.b);
  }
  g->prof_live.clear();
  return SOPHIE_OK;
}

StepArgs make_step_args(sophie_grid* g) {
  StepArgs a{};
  a.fin = g->F[g->cur];
  a.fout = g->F[1 - g->cur];
  a.fmt = g->fmt;
  for (int c = 0; c < 6; ++c) {
    a.sc[c] = g->fmt == kF32 ? 1.f : g->sc[c];
    a.isc[c] = 1.f / a.sc[c];
  }
  a.mat = g->mat;
  a.coef = g->coef;
  a.ecoef = g->ecoef;
  a.eeps = g->eeps;
  a.d = g->d;
  a.S = g->S32;
  a.n0 = g->n;
  a.src.n = (int)g->src.size();
  for (size_t s = 0; s < g->src.size(); ++s) {
    a.src.comp[s] = g->src[s].comp;
    a.src.pos[s] = g->src[s].pos;
  }
  a.src.val = g->sval;
  a.src.cap = g->scap;
  if (g->big_n > 0) {
    a.src.n = 0;
    a.src.nbig = g->big_n;
    a.src.bpos = g->big_pos;
    a.src.bcomp = g->big_comp;
    a.src.brow = g->big_row;
    a.src.val = g->big_val;
    a.src.cap = g->big_cap;
  }
  a.prb.n = (int)g->prb.size();
  for (size_t p = 0; p < g->prb.size(); ++p) {
    a.prb.comp[p] = g->prb[p].comp;
    a.prb.pos[p] = g->prb[p].pos;
  }
  if (g->obj_rec) {
    // The objective's samples go to the first unused probe slot.
    a.prb.comp[a.prb.n] = g->tape.comp;
    a.prb.pos[a.prb.n] = g->tape.pt;
    a.prb.n += 1;
  }
  a.prb.buf = g->pbuf;
  // 2-byte and hi+lo storage with six equal scales: the step kernels compute
  // on the scaled values (no scale multiplications); currents are scaled and
  // probe samples unscaled instead (both exact: powers of two).
  if ((g->fmt == kF16 || g->fmt == kBF16 || g->fmt == kF16HL) && g->sc[0] == g->sc[1] && g->sc[0] == g->sc[2] &&
      g->sc[0] == g->sc[3] && g->sc[0] == g->sc[4] && g->sc[0] == g->sc[5]) {
    a.fold = 1;
    a.src.vmul_on = 1;
    a.src.vmul = a.sc[0];
    a.prb.pmul_on = 1;
    a.prb.pmul = a.isc[0];
  }
  if (g->rat) {
    const Dims& d = g->d;
    const long long off[6] = {0, d.nx, d.nx + d.ny, d.nx + d.ny + d.nz, 2ll * d.nx + d.ny + d.nz + 1,
                              2ll * (d.nx + d.ny) + d.nz + 2};
    for (int q = 0; q < 6; ++q) a.rat[q] = g->rat + off[q];
    for (int q = 0; q < 3; ++q) a.rpair[q] = reinterpret_cast<const float2*>(g->rat + g->rpair_off[q]);
  }
  a.prb.cap = g->pcap;
  a.err = g->err;
  a.box[0] = 0;
  a.box[1] = g->d.nxp;
  a.box[2] = 0;
  a.box[3] = g->d.ny1;
  a.box[4] = 0;
  a.box[5] = g->d.nz1;
  return a;
}

int check_err_word(sophie_grid* g) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (h != 0) {
    cudaMemsetAsync(g->err, 0, sizeof(int), g->stream);
    return fail(SOPHIE_ETIMEOUT, "a kernel ran out of its bounded wait (code %d)", h);
  }
  return SOPHIE_OK;
}
}  // namespace grid
}  // namespace sophie

namespace {

// Guard size around a field buffer: one z slab of six components (what an
// off-by-one-plane access would touch), at least 1 MiB.
size_t field_guard(const Dims& d, int esz) {
  const size_t slab = (size_t)d.zstride * esz;
  return (std::max(slab, (size_t)1 << 20) + 255) / 256 * 256;
}

// Allocate a field buffer of `bytes` between two guard regions filled with
// kGuardByte; *F gets the buffer, *base the allocation.
cudaError_t alloc_guarded(size_t bytes, size_t guard, void** F, void** base, cudaStream_t s) {
  *F = *base = nullptr;
  void* p = nullptr;
  cudaError_t e = dev_malloc(&p, bytes + 2 * guard);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  unsigned char* c = static_cast<unsigned char*>(p);
  if ((e = cudaMemsetAsync(c, kGuardByte, guard, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c + guard + bytes, kGuardByte, guard, s)) != cudaSuccess) {
    cudaFree(p);
    return e;
  }
  *base = p;
  *F = c + guard;
  return cudaSuccess;
}

}  // namespace

namespace sophie {
namespace grid {
void free_tape(Tape& t) {
  for (void* p : t.ck) cudaFree(p);
  t.ck.clear();
  void* bufs[] = {t.samples, t.R[0], t.R[1], t.L[0], t.L[1], t.ecomp, t.ept, t.etr, t.ctr, t.gcb, t.gca, t.etr_all, t.ctr_all};
  for (void* p : bufs)
    if (p) cudaFree(p);
  t = Tape{};
}
}  // namespace grid
}  // namespace sophie

namespace {

void free_grid(sophie_grid* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  free_tape(g->tape);
  for (int b = 0; b < 2; ++b)
    if (g->Fbase[b]) cudaFree(g->Fbase[b]);
  if (g->mat) cudaFree(g->mat);
  if (g->mat_host) cudaFreeHost(g->mat_host);
  if (g->coef) cudaFree(g->coef);
  if (g->ecoef) cudaFree(g->ecoef);
  if (g->eeps) cudaFree(g->eeps);
  if (g->eps_tab) cudaFree(g->eps_tab);
  if (g->sval) cudaFree(g->sval);
  if (g->pbuf) cudaFree(g->pbuf);
  if (g->e_partials) cudaFree(g->e_partials);
  if (g->e_out) cudaFree(g->e_out);
  if (g->err) cudaFree(g->err);
  if (g->rat) cudaFree(g->rat);
  if (g->mat_upload_done) cudaEventDestroy(g->mat_upload_done);
  for (ProfEntry& p : g->prof_live) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

// Copy plane `comp` of every z slab (elements of g->esz bytes; for the 24-bit
// format planes 0..5 are the high halves, 6..8 the byte pairs).
int copy_component(sophie_grid* g, int comp, void* host, bool to_device, int buf) {
  const Dims& d = g->d;
  cudaMemcpy3DParms p{};
  const size_t es = (size_t)g->esz;
  const size_t planes = (size_t)(d.zstride / d.plane);
  cudaPitchedPtr dev = make_cudaPitchedPtr(static_cast<unsigned char*>(g->F[buf]) + (size_t)comp * d.plane * es,
                                           (size_t)d.nxp * es, (size_t)d.nx + 1, planes * d.ny1);
  cudaPitchedPtr hst = make_cudaPitchedPtr(host, (size_t)(d.nx + 1) * es, (size_t)d.nx + 1, (size_t)d.ny1);
  p.extent = make_cudaExtent((size_t)(d.nx + 1) * es, (size_t)d.ny1, (size_t)d.nz1);
  if (to_device) {
    p.srcPtr = hst;
    p.dstPtr = dev;
    p.kind = cudaMemcpyHostToDevice;
  } else {
    p.srcPtr = dev;
    p.dstPtr = hst;
    p.kind = cudaMemcpyDeviceToHost;
  }
  CUDA_TRY(cudaMemcpy3DAsync(&p, g->stream));
  return SOPHIE_OK;
}

bool encode_all_maps(sophie_grid* g) {
  const Dims& d = g->d;
  const int bxp = plain_box_x(g->fmt), bxb = blocked_box_x(g->fmt);
  return encode_maps(d, g->fmt, g->F[0], g->mat, bxp, plain_box_y(), &g->tmF[0], &g->tmM) &&
         encode_maps(d, g->fmt, g->F[1], nullptr, bxp, plain_box_y(), &g->tmF[1], nullptr) &&
         encode_maps(d, g->fmt, g->F[0], g->mat, bxb, blocked_box_y(), &g->tmFB[0], &g->tmMB) &&
         encode_maps(d, g->fmt, g->F[1], nullptr, bxb, blocked_box_y(), &g->tmFB[1], nullptr);
}

// The 24-bit format's rounding (yee_store.cuh, Store<kF24>): Veltkamp's split
// into 16 significant bits, three float operations in round-to-nearest (host
// code is compiled without contraction), then the low byte dropped.
uint32_t f24_bits(float v) {
  const float c = v * 257.f;
  const float dlt = v - c;
  const float hi = c + dlt;
  uint32_t u;
  memcpy(&u, &hi, 4);
  return u & 0xFFFFFF00u;
}

float f24_value(uint32_t hi16, uint32_t lo8) {
  const uint32_t u = (hi16 << 16) | (lo8 << 8);
  float v;
  memcpy(&v, &u, 4);
  return v;
}

// float <-> stored value (host side), stored = field * scale, round to nearest even.
void to_store(int fmt, float scale, const float* in, void* out, size_t n) {
  if (fmt == kF16) {
    __half* o = static_cast<__half*>(out);
    for (size_t i = 0; i < n; ++i) o[i] = __float2half_rn(in[i] * scale);
  } else if (fmt == kBF16) {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
    for (size_t i = 0; i < n; ++i) o[i] = __float2bfloat16_rn(in[i] * scale);
  } else if (fmt == kF16HL) {
    __half* o = static_cast<__half*>(out);  // pairs (hi, lo)
    for (size_t i = 0; i < n; ++i) {
      const float v = in[i] * scale;
      const __half hi = __float2half_rn(v);
      o[2 * i] = hi;
      o[2 * i + 1] = __float2half_rn(v - __half2float(hi));
    }
  } else {
    memcpy(out, in, n * 4);
  }
}

void from_store(int fmt, float scale, const void* in, float* out, size_t n) {
  const float inv = 1.f / scale;
  if (fmt == kF16) {
    const __half* p = static_cast<const __half*>(in);
    for (size_t i = 0; i < n; ++i) out[i] = __half2float(p[i]) * inv;
  } else if (fmt == kBF16) {
    const __nv_bfloat16* p = static_cast<const __nv_bfloat16*>(in);
    for (size_t i = 0; i < n; ++i) out[i] = __bfloat162float(p[i]) * inv;
  } else if (fmt == kF16HL) {
    const __half* p = static_cast<const __half*>(in);
    for (size_t i = 0; i < n; ++i) out[i] = (__half2float(p[2 * i]) + __half2float(p[2 * i + 1])) * inv;
  } else {
    memcpy(out, in, n * 4);
  }
}

// 24-bit storage: the component's high halves (plane comp) and its byte of the
// byte-pair plane 6 + comp/2, read-modify-written so that the other
// component's bytes are kept.
int set_component_f24(sophie_grid* g, int comp, const float* host) {
  const Dims& d = g->d;
  const size_t n = (size_t)(d.nx + 1) * d.ny1 * d.nz1;
  std::vector<uint16_t> hi(n), lo(n);
  const int sh = (comp & 1) * 8;
  for (int b = 0; b < 2; ++b) {
    int rc = copy_component(g, 6 + comp / 2, lo.data(), false, b);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (size_t i = 0; i < n; ++i) {
      const uint32_t u = f24_bits(host[i]);
      hi[i] = (uint16_t)(u >> 16);
      lo[i] = (uint16_t)((lo[i] & ~(0xFFu << sh)) | (((u >> 8) & 0xFFu) << sh));
    }
    rc = copy_component(g, comp, hi.data(), true, b);
    if (rc) return rc;
    rc = copy_component(g, 6 + comp / 2, lo.data(), true, b);
    if (rc) return rc;
    cudaError_t e = launch_mask_component(g->F[b], g->esz, g->d, comp, g->stream, g->fmt);
    if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "mask launch failed: %s", cudaGetErrorString(e));
    g->launches++;
    CUDA_TRY(cudaStreamSynchronize(g->stream));  // the host arrays are reused
  }
  return SOPHIE_OK;
}

int get_component_f24(sophie_grid* g, int comp, float* host) {
  const Dims& d = g->d;
  const size_t n = (size_t)(d.nx + 1) * d.ny1 * d.nz1;
  std::vector<uint16_t> hi(n), lo(n);
  int rc = copy_component(g, comp, hi.data(), false, g->cur);
  if (rc) return rc;
  rc = copy_component(g, 6 + comp / 2, lo.data(), false, g->cur);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const int sh = (comp & 1) * 8;
  for (size_t i = 0; i < n; ++i) host[i] = f24_value(hi[i], (lo[i] >> sh) & 0xFFu);
  return SOPHIE_OK;
}

int set_component(sophie_grid* g, int comp, const float* host) {
  g->gen++;
  g->box_all = true;  // caller's fields: nothing is known to be zero
  if (g->fmt == kF24) return set_component_f24(g, comp, host);
  const Dims& d = g->d;
  const size_t n = (size_t)(d.nx + 1) * d.ny1 * d.nz1;
  std::vector<unsigned char> tmp;
  const void* src = host;
  if (g->fmt != kF32) {
    tmp.resize(n * g->esz);
    to_store(g->fmt, g->sc[comp], host, tmp.data(), n);
    src = tmp.data();
  }
  for (int b = 0; b < 2; ++b) {
    int rc = copy_component(g, comp, const_cast<void*>(src), true, b);
    if (rc) return rc;
    cudaError_t e = launch_mask_component(g->F[b], g->esz, g->d, comp, g->stream, g->fmt);
    if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "mask launch failed: %s", cudaGetErrorString(e));
    g->launches++;
  }
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return SOPHIE_OK;
}

int get_component(sophie_grid* g, int comp, float* host) {
  const Dims& d = g->d;
  const size_t n = (size_t)(d.nx + 1) * d.ny1 * d.nz1;
  if (g->fmt == kF32) return copy_component(g, comp, host, false, g->cur);
  if (g->fmt == kF24) return get_component_f24(g, comp, host);
  std::vector<unsigned char> tmp(n * g->esz);
  int rc = copy_component(g, comp, tmp.data(), false, g->cur);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  from_store(g->fmt, g->sc[comp], tmp.data(), host, n);
  return SOPHIE_OK;
}

// Re-store the current fields in format `fmt` with scales `sc` (host round trip).
int restore_fields(sophie_grid* g, int fmt, const float* sc) {
  const Dims& d = g->d;
  const size_t n = (size_t)(d.nx + 1) * d.ny1 * d.nz1;
  std::vector<float> all(6 * n);
  for (int c = 0; c < 6; ++c) {
    int rc = get_component(g, c, all.data() + c * n);
    if (rc) return rc;
  }
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const int esz = store_bytes(fmt);
  Dims nd = d;
  nd.zstride = (long long)store_planes(fmt) * d.plane;
  if (esz != g->esz || nd.zstride != d.zstride) {
    const size_t bytes = (size_t)nd.zstride * nd.nz1 * esz;
    const size_t guard = field_guard(nd, esz);
    void* nb[2] = {nullptr, nullptr};
    void* nbase[2] = {nullptr, nullptr};
    for (int b = 0; b < 2; ++b) {
      if (alloc_guarded(bytes, guard, &nb[b], &nbase[b], g->stream) != cudaSuccess) {
        if (nbase[0]) cudaFree(nbase[0]);
        return fail(SOPHIE_ENOMEM, "field buffer allocation failed");
      }
      CUDA_TRY(cudaMemsetAsync(nb[b], 0, bytes, g->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    cudaFree(g->Fbase[0]);
    cudaFree(g->Fbase[1]);
    for (int b = 0; b < 2; ++b) {
      g->F[b] = nb[b];
      g->Fbase[b] = nbase[b];
    }
    g->fguard = guard;
    g->esz = esz;
    g->d.zstride = nd.zstride;
  }
  g->fmt = fmt;
  for (int c = 0; c < 6; ++c) g->sc[c] = sc[c];
  if (!encode_all_maps(g)) return fail(SOPHIE_ECUDA, "cuTensorMapEncodeTiled failed");
  g->cur = 0;
  for (int c = 0; c < 6; ++c) {
    int rc = set_component(g, c, all.data() + c * n);
    if (rc) return rc;
  }
  return SOPHIE_OK;
}

// Time one candidate launch configuration: `launch` is enqueued `reps` times
// reading the current buffer and writing the other one (the state does not
// advance). Returns the mean milliseconds per launch, or < 0 on a launch error.
template <class Fn>
double time_candidate(sophie_grid* g, Fn&& launch, cudaEvent_t e0, cudaEvent_t e1) {
  if (launch() != cudaSuccess) return -1.0;  // warm-up
  cudaEventRecord(e0, g->stream);
  if (launch() != cudaSuccess) return -1.0;
  cudaEventRecord(e1, g->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const int reps = std::max(3, std::min(100, (int)(6.0 / std::max(ms, 1e-3f))));
  cudaEventRecord(e0, g->stream);
  for (int r = 0; r < reps; ++r)
    if (launch() != cudaSuccess) return -1.0;
  cudaEventRecord(e1, g->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
  cudaEventElapsedTime(&ms, e0, e1);
  g->launches += reps + 2;
  return (double)ms / reps;
}

// Autotuner: measure the plain kernel's z-chunk choices and the temporally
// blocked kernel at k = 2..4 with several work splits on this grid, keep the
// fastest per step. All candidates give bitwise identical float results, so
// the choice changes only speed. With 2-byte storage, where results depend
// on k, only the tilings are tuned and k stays 2. With a fixed temporal_k only
// the tilings of that k are tuned (and the plain kernel's, which also runs
// the remainder steps). The tuning knobs SOPHIE_ZCHUNK and
// SOPHIE_BLOCKED_ALIGNED, when set, replace the candidates they fix.
int run_autotune(sophie_grid* g, double* best_ms_per_step) {
  if (g->use_simple) {
    g->tuned = true;
    g->tuned_k = 1;
    if (best_ms_per_step) *best_ms_per_step = -1.0;
    return SOPHIE_OK;
  }
  int rc = ensure_capacity(g, g->n + 1);
  if (rc) return rc;
  StepArgs a = make_step_args(g);
  a.prb.n = 0;  // no probe samples from the trial launches
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const Dims& d = g->d;
  double best = 1e300;
  PlainTiling best_p = g->ptile;
  double best_plain = 1e300;
  BlockedTiling best_b{};
  int best_k = 1;
  const int kfix = g->temporal_k;  // 0: k is tuned too
  const char* zenv = getenv("SOPHIE_ZCHUNK");
  const char* aenv = getenv("SOPHIE_BLOCKED_ALIGNED");
  std::vector<int> zcs = {1, 2, 4, 8, 16, 32, 64};
  if (zenv) zcs = {atoi(zenv) > 0 ? atoi(zenv) : 0};
  for (int zc : zcs) {
    if (zc > 2 * d.nz && zc != zcs[0]) break;
    const PlainTiling pt = plain_tiling(d, g->num_sms, zc);
    const double ms = time_candidate(g, [&] { return launch_step_plain(a, g->tmF[g->cur], g->tmM, pt, g->stream); },
                                     e0, e1);
    if (ms < 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(SOPHIE_ECUDA, "autotune launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (ms < best_plain) {
      best_plain = ms;
      best_p = pt;
    }
  }
  if (kfix == 1 || (kfix == 0 && g->fmt == kF32)) {
    best = best_plain;
    best_k = 1;
  }
  const int k_lo = kfix ? kfix : 2, k_hi = kfix ? kfix : 4;
  for (int K = k_lo; K <= k_hi && K >= 2; ++K) {
    if (!kfix && g->fmt != kF32 && K != 2) continue;
    // the cost model's aligned split in both unit orders, its neighbours and
    // twice it, and the contiguous split
    std::vector<BlockedTiling> cands;
    const BlockedTiling model = blocked_tiling(d, K, g->num_sms, 1);
    const char* zsenv = getenv("SOPHIE_BLOCKED_ZSPLIT");
    if (zsenv && atoi(zsenv) > 0) {
      // a fixed number of z ranges in both unit orders (tuning knob)
      for (int order = 0; order < 2; ++order)
        cands.push_back(blocked_tiling_split(d, K, g->num_sms, atoi(zsenv), order));
    } else if (aenv) {
      const int mode = atoi(aenv);
      cands.push_back(blocked_tiling(d, K, g->num_sms, mode >= 0 && mode <= 3 ? mode : 1));
    } else {
      cands.push_back(model);
      cands.push_back(blocked_tiling_split(d, K, g->num_sms, model.zsplit, 1 - model.order));
      for (int zs : {model.zsplit + 1, model.zsplit - 1, 2 * model.zsplit})
        if (zs >= 1 && zs <= d.nz)
          for (int order = 0; order < 2; ++order) cands.push_back(blocked_tiling_split(d, K, g->num_sms, zs, order));
      cands.push_back(blocked_tiling(d, K, g->num_sms, 0));
    }
    // K = 2 also runs with 16 warps of 2 rows per thread (Lay<2> in the
    // blocked kernel): every split in both thread layouts
    const char* renv = getenv("SOPHIE_BLOCKED_ROWS");
    const int rows_fix = renv ? atoi(renv) : 0;
    if (K == 2) {
      const size_t nc = cands.size();
      for (size_t q = 0; q < nc; ++q) {
        cands[q].rows = 4;
        BlockedTiling b2 = cands[q];
        b2.rows = 2;
        cands.push_back(b2);
      }
    }
    if (rows_fix == 2 || rows_fix == 4) {
      std::vector<BlockedTiling> keep;
      for (const BlockedTiling& bt : cands)
        if ((bt.rows == 2 ? 2 : 4) == rows_fix) keep.push_back(bt);
      if (!keep.empty()) cands = keep;
    }
    for (const BlockedTiling& bt : cands) {
      const double ms = time_candidate(
          g, [&] { return launch_step_blocked(a, g->tmFB[g->cur], g->tmMB, bt, g->stream); }, e0, e1);
      if (ms < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(SOPHIE_ECUDA, "autotune launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      }
      if (ms / K < best) {
        best = ms / K;
        best_k = K;
        best_b = bt;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // The trial launches wrote the spare buffer everywhere. Zero-field skipping
  // relies on both buffers being zero outside the known-nonzero box (skipped
  // units are never written), so clear it: the next step writes every unit it
  // computes in full, and every other entry is zero in the state anyway.
  if (!g->box_all)
    CUDA_TRY(cudaMemsetAsync(g->F[1 - g->cur], 0, (size_t)d.zstride * d.nz1 * g->esz, g->stream));
  rc = check_err_word(g);
  if (rc) return rc;
  g->ptile = best_p;
  if (best_k >= 2) g->btile = best_b;
  g->tuned_k = best_k;
  g->tuned = true;
  if (best_ms_per_step) *best_ms_per_step = best;
  return SOPHIE_OK;
}

}  // namespace

namespace {

// Add index point (i, j, k) to the known-nonzero box.
void box_add_point(sophie_grid* g, int i, int j, int k) {
  int* b = g->zbox;
  if (b[0] >= b[1]) {
    b[0] = i; b[1] = i + 1; b[2] = j; b[3] = j + 1; b[4] = k; b[5] = k + 1;
    return;
  }
  b[0] = std::min(b[0], i); b[1] = std::max(b[1], i + 1);
  b[2] = std::min(b[2], j); b[3] = std::max(b[3], j + 1);
  b[4] = std::min(b[4], k); b[5] = std::max(b[5], k + 1);
}

// The box grown by r index points per side (one step moves nonzero values by
// at most one point per axis), clamped to the grid's points.
void box_grown(const sophie_grid* g, int r, int* out) {
  const int* b = g->zbox;
  if (b[0] >= b[1]) {
    for (int q = 0; q < 6; ++q) out[q] = 0;
    return;
  }
  const int hi[3] = {g->d.nx + 1, g->d.ny + 1, g->d.nz + 1};
  for (int a = 0; a < 3; ++a) {
    out[2 * a] = std::max(0, b[2 * a] - r);
    out[2 * a + 1] = std::min(hi[a], b[2 * a + 1] + r);
  }
}

// Reset the box to the source points (fields zero).
void box_from_sources(sophie_grid* g) {
  for (int q = 0; q < 6; ++q) g->zbox[q] = 0;
  g->box_all = false;
  for (const Source& s : g->src) box_add_point(g, s.i, s.j, s.k);
}

}  // namespace

extern "C" {

int sophie_version(void) { return 10000; }

const char* sophie_last_error(void) { return g_err.c_str(); }

int sophie_create_grid(int nx, int ny, int nz, double dx, double dt, sophie_grid** out) {
  g_err.clear();
  if (!out) return fail(SOPHIE_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(SOPHIE_EINVAL, "grid sizes must be >= 1");
  if (!(dx > 0) || !std::isfinite(dx)) return fail(SOPHIE_EINVAL, "dx must be finite and > 0");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(SOPHIE_EINVAL, "dt must be finite and > 0");
  if (kC0 * dt * std::sqrt(3.0) > dx * (1.0 + 1e-12))
    return fail(SOPHIE_EUNSTABLE, "dt above the 3-D Courant limit dx/(c sqrt 3)");
  if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
    return fail(SOPHIE_EINVAL, "grid size above 2^20 per axis");
  Dims d{};
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.nxp = ((nx + 1) + 7) / 8 * 8;
  d.ny1 = ny + 1;
  d.nz1 = nz + 1;
  d.plane = (long long)d.ny1 * d.nxp;
  d.zstride = 6 * d.plane;
  const double field_bytes = (double)d.zstride * d.nz1 * 4.0;
  const double pts = (double)d.plane * d.nz1;
  if (d.zstride > (1ll << 31) || field_bytes * 2 + pts * 4 > 2.5e11)
    return fail(SOPHIE_ENOMEM, "grid too large (%.3g bytes of fields)", field_bytes * 2);
  sophie_grid* g = new (std::nothrow) sophie_grid();
  if (!g) return fail(SOPHIE_ENOMEM, "host allocation failed");
  g->d = d;
  g->dx = dx;
  g->dt = dt;
  g->S64 = kC0 * dt / dx;
  g->S32 = (float)g->S64;
  int rc = SOPHIE_OK;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (dev_malloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(SOPHIE_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
      return false;
    }
    return true;
  };
  const size_t fbytes = (size_t)d.zstride * d.nz1 * 4;
  const size_t npts = (size_t)d.plane * d.nz1;
  do {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(SOPHIE_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    g->own_stream = true;
    g->fguard = field_guard(d, 4);
    if (alloc_guarded(fbytes, g->fguard, &g->F[0], &g->Fbase[0], g->stream) != cudaSuccess ||
        alloc_guarded(fbytes, g->fguard, &g->F[1], &g->Fbase[1], g->stream) != cudaSuccess) {
      rc = fail(SOPHIE_ENOMEM, "field buffer allocation (%zu bytes + guards) failed", fbytes);
      break;
    }
    if (!alloc((void**)&g->mat, npts * 4)) break;
    if (!alloc((void**)&g->coef, kMaxClasses * sizeof(float2))) break;
    if (!alloc((void**)&g->eps_tab, kMaxClasses * sizeof(double))) break;
    if (!alloc((void**)&g->err, sizeof(int))) break;
    g->e_blocks = energy_blocks(d);
    if (!alloc((void**)&g->e_partials, (size_t)g->e_blocks * 8)) break;
    if (!alloc((void**)&g->e_out, 8)) break;
    if (cudaMallocHost(&g->mat_host, npts * 4) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(SOPHIE_ENOMEM, "pinned host allocation failed");
      break;
    }
    if (cudaEventCreateWithFlags(&g->mat_upload_done, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(SOPHIE_ECUDA, "cudaEventCreate failed");
      break;
    }
    if (cudaMemsetAsync(g->F[0], 0, fbytes, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->F[1], 0, fbytes, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->err, 0, sizeof(int), g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->coef, 0, kMaxClasses * sizeof(float2), g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->eps_tab, 0, kMaxClasses * sizeof(double), g->stream) != cudaSuccess) {
      rc = fail(SOPHIE_ECUDA, "cudaMemsetAsync failed");
      break;
    }
    {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev);
      if (g->num_sms <= 0) g->num_sms = 1;
    }
    if (!encode_all_maps(g)) {
      rc = fail(SOPHIE_ECUDA, "cuTensorMapEncodeTiled failed");
      break;
    }
    {
      // SOPHIE_ZCHUNK: z planes per work unit of the TMA kernels (tuning knob;
      // any value gives identical results).
      const char* zc = getenv("SOPHIE_ZCHUNK");
      g->ptile = plain_tiling(d, g->num_sms, zc ? atoi(zc) : 0);
    }
    rc = build_material_words(g, nullptr, nullptr);
    if (rc) break;
    rc = upload_materials(g);
    if (rc) break;
    rc = ensure_capacity(g, 1);
    if (rc) break;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
      rc = fail(SOPHIE_ECUDA, "initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
  } while (0);
  if (rc != SOPHIE_OK) {
    free_grid(g);
    return rc;
  }
  handle_register(g);
  *out = g;
  return SOPHIE_OK;
}

int sophie_destroy_grid(sophie_grid* g) {
  if (!g) return SOPHIE_OK;
  if (!handle_release(g)) return fail(SOPHIE_EINVAL, "not a live grid (already destroyed?)");
  free_grid(g);
  return SOPHIE_OK;
}

int sophie_check_guards(sophie_grid* g, long long* bad_bytes) {
  if (!g || !bad_bytes) return fail(SOPHIE_EINVAL, "NULL argument");
  unsigned long long* d = nullptr;
  if (dev_malloc((void**)&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SOPHIE_ENOMEM, "guard check counter allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), g->stream);
  const size_t fbytes = (size_t)g->d.zstride * g->d.nz1 * g->esz;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    const unsigned char* base = static_cast<const unsigned char*>(g->Fbase[b]);
    e = launch_guard_check(base, g->fguard, kGuardByte, d, g->stream);
    if (e == cudaSuccess) e = launch_guard_check(base + g->fguard + fbytes, g->fguard, kGuardByte, d, g->stream);
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "guard check failed: %s", cudaGetErrorString(e));
  g->launches += 4;
  *bad_bytes = (long long)h;
  return SOPHIE_OK;
}

int sophie_selftest_wait_timeout(sophie_grid* g, double* waited_ms) {
  if (!g || !waited_ms) return fail(SOPHIE_EINVAL, "NULL argument");
  unsigned long long* d = nullptr;
  if (dev_malloc((void**)&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SOPHIE_ENOMEM, "self-test allocation failed");
  }
  cudaError_t e = launch_wait_timeout(g->err, d, g->stream);
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d, sizeof(ns), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "self-test launch failed: %s", cudaGetErrorString(e));
  g->launches++;
  *waited_ms = (double)ns * 1e-6;
  return SOPHIE_OK;
}

int sophie_debug_material_tables(int nx, int ny, int nz, double dx, double dt, const float* eps, const float* sig,
                                 int nthreads, unsigned int* words, float* class_coef, double* class_eps,
                                 float* exp_coef, double* exp_eps, long long exp_cap, long long* n_explicit) {
  if (!eps || !sig || !words || !class_coef || !class_eps || !n_explicit || exp_cap < 0 ||
      (exp_cap > 0 && (!exp_coef || !exp_eps)))
    return fail(SOPHIE_EINVAL, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
    return fail(SOPHIE_EINVAL, "grid sizes must be in [1, 4096]");
  if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt))
    return fail(SOPHIE_EINVAL, "dx and dt must be finite and > 0");
  if (nthreads < 1) return fail(SOPHIE_EINVAL, "nthreads must be >= 1");
  const long long ncell = (long long)nx * ny * nz;
  const long long c = first_bad_material(eps, sig, ncell, nthreads);
  if (c >= 0) return fail(SOPHIE_EINVAL, "bad material at cell %lld", c);
  Dims d{};
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.nxp = ((nx + 1) + 7) / 8 * 8;
  d.ny1 = ny + 1;
  d.nz1 = nz + 1;
  d.plane = (long long)d.ny1 * d.nxp;
  d.zstride = 6 * d.plane;
  MaterialTables t;
  if (build_material_tables(d, dt, kC0 * dt / dx, eps, sig, words, &t, nthreads) != 0)
    return fail(SOPHIE_ETOOMANYMAT, "more than 2^29 explicit material points");
  for (int q = 0; q < kMaxClasses; ++q) {
    const bool has = q < (int)t.coef.size();
    class_coef[2 * q] = has ? t.coef[q].x : 0.f;
    class_coef[2 * q + 1] = has ? t.coef[q].y : 0.f;
    class_eps[q] = has ? t.eps[q] : 0.0;
  }
  const long long ne = (long long)t.eeps.size() / 3;
  for (long long q = 0; q < std::min(ne, exp_cap) * 3; ++q) {
    exp_coef[2 * q] = t.ecoef[q].x;
    exp_coef[2 * q + 1] = t.ecoef[q].y;
    exp_eps[q] = t.eeps[q];
  }
  *n_explicit = ne;
  return SOPHIE_OK;
}

int sophie_debug_fail_alloc(int n) {
  if (n < 0) return fail(SOPHIE_EINVAL, "n must be >= 0");
  g_fail_alloc_at.store(n);
  return SOPHIE_OK;
}

int sophie_set_materials(sophie_grid* g, const float* eps, const float* sig) {
  if (!g || !eps || !sig) return fail(SOPHIE_EINVAL, "NULL argument");
  const long long ncell = (long long)g->d.nx * g->d.ny * g->d.nz;
  const long long c = first_bad_material(eps, sig, ncell, std::max(1, std::min(32, (int)std::thread::hardware_concurrency())));
  if (c >= 0) {
    if (!(eps[c] >= 1.0f))
      return fail(SOPHIE_EINVAL, "eps_r[%lld] = %g must be >= 1 (+inf: conductor)", c, (double)eps[c]);
    return fail(SOPHIE_EINVAL, "sigma[%lld] = %g must be finite and >= 0", c, (double)sig[c]);
  }
  // The staging buffer may still feed an earlier upload.
  CUDA_TRY(cudaEventSynchronize(g->mat_upload_done));
  std::vector<float2> old_coef = g->coef_h, old_ecoef = g->ecoef_h;
  std::vector<double> old_eps = g->eps_h, old_eeps = g->eeps_h, old_sig = g->sig_h, old_esig = g->esig_h;
  g->gen++;
  int rc = build_material_words(g, eps, sig);
  if (rc) {
    // Restore the words of the current materials.
    g->coef_h = old_coef;
    g->eps_h = old_eps;
    g->ecoef_h = old_ecoef;
    g->eeps_h = old_eeps;
    g->sig_h = old_sig;
    g->esig_h = old_esig;
    CUDA_TRY(cudaMemcpy(g->mat_host, g->mat, (size_t)g->d.plane * g->d.nz1 * 4, cudaMemcpyDeviceToHost));
    return rc;
  }
  return upload_materials(g);
}

int sophie_add_source(sophie_grid* g, int comp, int i, int j, int k, double amp, double f0,
                      double bw, double t0, int kind) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  if (comp < 0 || comp > 2) return fail(SOPHIE_EINVAL, "source component must be 0, 1 or 2 (E)");
  if (!e_edge_interior(g->d, comp, i, j, k))
    return fail(SOPHIE_EINVAL, "source edge (%d,%d,%d) of comp %d is not interior", i, j, k, comp);
  if (kind != SOPHIE_GAUSS_SINE && kind != SOPHIE_GAUSS) return fail(SOPHIE_EINVAL, "bad waveform kind");
  if (!std::isfinite(amp) || !std::isfinite(f0) || !std::isfinite(t0) || !(bw > 0) || !std::isfinite(bw))
    return fail(SOPHIE_EINVAL, "bad waveform parameters");
  if ((int)g->src.size() >= kMaxSources) return fail(SOPHIE_EINVAL, "at most %d sources", kMaxSources);
  Source s{comp, i, j, k, kind, amp, f0, bw, t0, point_index(g->d, i, j, k)};
  g->gen++;
  g->src.push_back(s);
  if (!g->box_all) box_add_point(g, i, j, k);
  int rc = refresh_source_table(g, (int)g->src.size() - 1);
  if (rc) {
    g->src.pop_back();
    return rc;
  }
  if (launch_or_flag(g->mat, s.pos, kSrcFlag, g->stream) != cudaSuccess)
    return fail(SOPHIE_ECUDA, "flag launch failed");
  g->launches++;
  return SOPHIE_OK;
}

int sophie_add_probe(sophie_grid* g, int comp, int i, int j, int k, int* probe_id) {
  if (!g || !probe_id) return fail(SOPHIE_EINVAL, "NULL argument");
  if (comp < 0 || comp > 5) return fail(SOPHIE_EINVAL, "probe component must be in 0..5");
  if (!comp_valid(g->d, comp, i, j, k))
    return fail(SOPHIE_EINVAL, "probe (%d,%d,%d) outside comp %d's range", i, j, k, comp);
  if ((int)g->prb.size() >= kMaxProbes) return fail(SOPHIE_EINVAL, "at most %d probes", kMaxProbes);
  Probe p{comp, i, j, k, point_index(g->d, i, j, k), i == g->d.nx || j == g->d.ny || k == g->d.nz, g->n};
  if (!p.fixed) {
    if (launch_or_flag(g->mat, p.pos, kPrbFlag, g->stream) != cudaSuccess)
      return fail(SOPHIE_ECUDA, "flag launch failed");
    g->launches++;
  }
  g->prb.push_back(p);
  *probe_id = (int)g->prb.size() - 1;
  return SOPHIE_OK;
}

int sophie_step(sophie_grid* g, int n) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  if (n < 0) return fail(SOPHIE_EINVAL, "n must be >= 0");
  if (n == 0) return SOPHIE_OK;
  int rc = ensure_capacity(g, g->n + n);
  if (rc) return rc;
  g->gen++;
  if (!g->tuned) {  // k and tilings, or (fixed temporal_k) the tilings only
    rc = run_autotune(g, nullptr);
    if (rc) return rc;
  }
  for (int m = 0; m < n;) {
    const int K = g->temporal_k == 0 ? g->tuned_k : g->temporal_k;
    const bool blocked = !g->use_simple && K >= 2 && n - m >= K && blocked_supported(K, g->fmt);
    StepArgs a = make_step_args(g);
    const int adv_steps = blocked ? K : 1;
    // Zero-field skipping: this launch covers only the tiles and planes of the
    // known-nonzero box grown by its steps (nothing at all if the box is empty).
    const bool sub = g->zskip && !g->box_all && !g->use_simple;
    PlainTiling pt_sub{};
    BlockedTiling bt_sub{};
    bool none = false;
    if (sub) {
      box_grown(g, adv_steps, a.box);
      if (blocked) {
        bt_sub = blocked_tiling_box(g->d, K, g->num_sms, a.box);
        bt_sub.rows = g->btile.K == K ? g->btile.rows : 0;  // the tuned thread layout
        none = bt_sub.grid == 0;
      } else {
        pt_sub = plain_tiling_box(g->d, g->num_sms, a.box);
        none = pt_sub.grid == 0;
      }
    }
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (g->prof && !none) {
      ea = prof_event(g);
      eb = prof_event(g);
      cudaEventRecord(ea, g->stream);
    }
    cudaError_t e = cudaSuccess;
    if (none) {
      // every field is zero in both buffers: nothing to compute
    } else if (blocked) {
      if (g->btile.K != K) {
        // SOPHIE_BLOCKED_ALIGNED=0 cuts the work into equal contiguous ranges
        // instead of equal z ranges per tile, 2 / 3 force the tile-major /
        // range-major unit order (tuning knob; same results).
        const char* al = getenv("SOPHIE_BLOCKED_ALIGNED");
        const int mode = al ? atoi(al) : 1;
        g->btile = blocked_tiling(g->d, K, g->num_sms, mode >= 0 && mode <= 3 ? mode : 1);
      }
      e = launch_step_blocked(a, g->tmFB[g->cur], g->tmMB, sub ? bt_sub : g->btile, g->stream);
    } else if (g->use_simple) {
      e = launch_step_simple(a, g->stream);
    } else {
      e = launch_step_plain(a, g->tmF[g->cur], g->tmM, sub ? pt_sub : g->ptile, g->stream);
    }
    if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "step launch failed: %s", cudaGetErrorString(e));
    if (g->prof && !none) {
      cudaEventRecord(eb, g->stream);
      g->prof_live.push_back({blocked ? SOPHIE_KERNEL_BLOCKED : SOPHIE_KERNEL_PLAIN, ea, eb});
      if (g->prof_live.size() > 20000) {
        rc = prof_drain(g);
        if (rc) return rc;
      }
    }
    if (!none) g->launches++;
    g->cur = 1 - g->cur;
    const int adv = adv_steps;
    if (!g->box_all) {
      int grown[6];
      box_grown(g, adv, grown);
      if (g->zbox[0] < g->zbox[1])
        for (int q = 0; q < 6; ++q) g->zbox[q] = grown[q];
    }
    g->n += adv;
    m += adv;
  }
  return SOPHIE_OK;
}

int sophie_get_step(sophie_grid* g, long long* n) {
  if (!g || !n) return fail(SOPHIE_EINVAL, "NULL argument");
  *n = g->n;
  return SOPHIE_OK;
}

int sophie_read_probe(sophie_grid* g, int probe_id, double* out, int cap, int* n_written) {
  if (!g || !out || !n_written) return fail(SOPHIE_EINVAL, "NULL argument");
  if (probe_id < 0 || probe_id >= (int)g->prb.size()) return fail(SOPHIE_EINVAL, "bad probe id");
  if (cap < 0) return fail(SOPHIE_EINVAL, "cap must be >= 0");
  const long long m = std::min<long long>(cap, g->n);
  const Probe& pr = g->prb[probe_id];
  std::vector<float> tmp((size_t)m);
  float fixed_v = 0.f;
  if (pr.fixed) {
    const Dims& d = g->d;
    const long long off = (long long)pr.k * d.zstride + (long long)pr.comp * d.plane + (long long)pr.j * d.nxp + pr.i;
    unsigned char raw[4] = {0, 0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(raw, static_cast<unsigned char*>(g->F[g->cur]) + off * g->esz, g->esz,
                             cudaMemcpyDeviceToHost, g->stream));
    if (g->fmt == kF24) {  // the component's byte of its byte-pair plane
      const long long lo = off + (long long)(6 + pr.comp / 2 - pr.comp) * d.plane;
      CUDA_TRY(cudaMemcpyAsync(raw + 2, static_cast<unsigned char*>(g->F[g->cur]) + lo * 2 + (pr.comp & 1), 1,
                               cudaMemcpyDeviceToHost, g->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->fmt == kF24) {
      uint16_t h;
      memcpy(&h, raw, 2);
      fixed_v = f24_value(h, raw[2]);
    } else {
      from_store(g->fmt, g->sc[pr.comp], raw, &fixed_v, 1);
    }
  } else if (m > 0) {
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), g->pbuf + (size_t)probe_id * g->pcap, (size_t)m * 4,
                             cudaMemcpyDeviceToHost, g->stream));
  }
  int rc = check_err_word(g);
  if (rc) return rc;
  if (pr.fixed)
    for (long long q = 0; q < m; ++q) tmp[q] = q >= pr.n_added ? fixed_v : 0.f;
  for (long long q = 0; q < m; ++q) out[q] = (double)tmp[q];
  *n_written = (int)m;
  return SOPHIE_OK;
}

int sophie_energy(sophie_grid* g, double* W) {
  if (!g || !W) return fail(SOPHIE_EINVAL, "NULL argument");
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (g->prof) {
    ea = prof_event(g);
    eb = prof_event(g);
    cudaEventRecord(ea, g->stream);
  }
  const StepArgs sa = make_step_args(g);
  cudaError_t e = launch_energy(sa, g->eps_tab, g->e_partials, g->e_blocks, g->e_out, g->stream);
  if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "energy launch failed: %s", cudaGetErrorString(e));
  if (g->prof) {
    cudaEventRecord(eb, g->stream);
    g->prof_live.push_back({SOPHIE_KERNEL_ENERGY, ea, eb});
  }
  g->launches += 2;
  double h = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&h, g->e_out, 8, cudaMemcpyDeviceToHost, g->stream));
  int rc = check_err_word(g);
  if (rc) return rc;
  const double dx = g->dx;
  *W = 0.5 * kEps0 * dx * dx * dx * h;
  if (!std::isfinite(*W)) return fail(SOPHIE_ENONFINITE, "energy is not finite");
  return SOPHIE_OK;
}

int sophie_energy_noalloc(sophie_grid* g, double* W_dev) {
  if (!g || !W_dev) return fail(SOPHIE_EINVAL, "NULL argument");
  const char* why = "";
  const double dx = g->dx;
  const StepArgs sa = make_step_args(g);
  const int rc = energy_noalloc(sa, g->eps_tab, 0.5 * kEps0 * dx * dx * dx, W_dev, g->stream, &why);
  if (rc == -1) return fail(SOPHIE_EINVAL, "%s", why);
  if (rc != 0) return fail(SOPHIE_ECUDA, "energy (no allocation) failed: %s", why);
  g->launches += 2;
  return SOPHIE_OK;
}

int sophie_set_fields(sophie_grid* g, int comp, const float* host) {
  if (!g || !host) return fail(SOPHIE_EINVAL, "NULL argument");
  if (comp < 0 || comp > 5) return fail(SOPHIE_EINVAL, "comp must be in 0..5");
  return set_component(g, comp, host);
}

int sophie_get_fields(sophie_grid* g, int comp, float* host) {
  if (!g || !host) return fail(SOPHIE_EINVAL, "NULL argument");
  if (comp < 0 || comp > 5) return fail(SOPHIE_EINVAL, "comp must be in 0..5");
  int rc = get_component(g, comp, host);
  if (rc) return rc;
  return check_err_word(g);
}

int sophie_set_storage_scale(sophie_grid* g, const float* scale) {
  if (!g || !scale) return fail(SOPHIE_EINVAL, "NULL argument");
  for (int c = 0; c < 6; ++c) {
    int ex = 0;
    const float m = std::frexp(scale[c], &ex);
    if (!(scale[c] > 0) || !std::isfinite(scale[c]) || m != 0.5f || ex < -60 || ex > 61)
      return fail(SOPHIE_EINVAL, "scale[%d] = %g must be a power of two in [2^-61, 2^60]", c, (double)scale[c]);
  }
  return restore_fields(g, g->fmt, scale);
}

int sophie_reset(sophie_grid* g) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  const size_t fbytes = (size_t)g->d.zstride * g->d.nz1 * g->esz;
  CUDA_TRY(cudaMemsetAsync(g->F[0], 0, fbytes, g->stream));
  CUDA_TRY(cudaMemsetAsync(g->F[1], 0, fbytes, g->stream));
  if (g->pbuf) CUDA_TRY(cudaMemsetAsync(g->pbuf, 0, (size_t)kMaxProbes * g->pcap * 4, g->stream));
  g->n = 0;
  g->cur = 0;
  g->gen++;
  box_from_sources(g);
  for (Probe& p : g->prb) p.n_added = 0;
  return SOPHIE_OK;
}

int sophie_set_stream(sophie_grid* g, void* cuda_stream) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  int rc = prof_drain(g);
  if (rc) return rc;
  if (g->own_stream) cudaStreamDestroy(g->stream);
  g->own_stream = false;
  g->stream = (cudaStream_t)cuda_stream;
  return SOPHIE_OK;
}

int sophie_sync(sophie_grid* g) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  return check_err_word(g);
}

int sophie_configure(sophie_grid* g, int temporal_k, int tile_x, int tile_y, int precision) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  if (temporal_k < 0 || temporal_k > 8) return fail(SOPHIE_EINVAL, "temporal_k must be in 0..8");
  if (temporal_k >= 2 && precision >= SOPHIE_FP32 && precision <= SOPHIE_FP24 &&
      !blocked_supported(temporal_k, precision))
    return fail(SOPHIE_ENOTSUP, "temporal_k = %d not built for precision %d (1..4; 6 and 8 with float storage)",
                temporal_k, precision);
  if (tile_x < 0 || tile_y < 0) return fail(SOPHIE_EINVAL, "tile sizes must be >= 0");
  if (tile_x != 0 && tile_x != 32 && tile_x != 64) return fail(SOPHIE_EINVAL, "tile_x must be 0, 32 or 64");
  if (precision < SOPHIE_FP32 || precision > SOPHIE_FP24)
    return fail(SOPHIE_ENOTSUP, "precision %d not supported", precision);
  if (tile_x == 32 && precision != SOPHIE_FP32)
    return fail(SOPHIE_ENOTSUP, "the 32x8 reference kernel stores float only");
  if (precision != g->fmt) {
    int rc = restore_fields(g, precision, g->sc);
    if (rc) return rc;
  }
  if (temporal_k != g->temporal_k || precision != g->precision || (tile_x == 32) != g->use_simple) {
    g->tuned = false;
    // the modelled tilings until the next step measures them
    const char* zc = getenv("SOPHIE_ZCHUNK");
    g->ptile = plain_tiling(g->d, g->num_sms, zc ? atoi(zc) : 0);
    g->btile = BlockedTiling{};
  }
  g->temporal_k = temporal_k;
  g->precision = precision;
  g->use_simple = tile_x == 32;
  return SOPHIE_OK;
}

int sophie_set_zero_skip(sophie_grid* g, int enable) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  g->zskip = enable != 0;
  return SOPHIE_OK;
}

int sophie_set_spacing(sophie_grid* g, const double* wx, const double* wy, const double* wz) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  const Dims& d = g->d;
  if (!wx && !wy && !wz) {
    if (g->rat) {
      CUDA_TRY(cudaStreamSynchronize(g->stream));
      cudaFree(g->rat);
      g->rat = nullptr;
      g->gen++;
      g->tuned = false;
    }
    return SOPHIE_OK;
  }
  const double* w[3] = {wx, wy, wz};
  const int n[3] = {d.nx, d.ny, d.nz};
  double inv2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double wmin = g->dx;
    if (w[a]) {
      wmin = HUGE_VAL;
      for (int i = 0; i < n[a]; ++i) {
        if (!(w[a][i] > 0) || !std::isfinite(w[a][i]))
          return fail(SOPHIE_EINVAL, "width %d along axis %d is %g (must be finite and > 0)", i, a, w[a][i]);
        wmin = std::min(wmin, w[a][i]);
      }
    }
    inv2 += 1.0 / (wmin * wmin);
  }
  if (kC0 * g->dt * std::sqrt(inv2) > 1.0 + 1e-12)
    return fail(SOPHIE_EUNSTABLE, "dt above the Courant limit of the smallest cells");
  // Ratios dx / width (primary) and dx / ((w[i-1] + w[i]) / 2) (dual; at a
  // wall node the end cell's own width, so the wall-normal faces weigh a whole
  // cell in the energy as on the uniform mesh), each computed in double and
  // rounded once.
  std::vector<float> h;
  h.reserve(2 * (size_t)(d.nx + d.ny + d.nz) + 3);
  auto width = [&](int a, int i) { return w[a] ? w[a][i] : g->dx; };
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n[a]; ++i) h.push_back((float)(g->dx / width(a, i)));
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i <= n[a]; ++i) {
      const double lo = width(a, i > 0 ? i - 1 : 0), hi = width(a, i < n[a] ? i : n[a] - 1);
      h.push_back((float)(g->dx / ((lo + hi) / 2.0)));
    }
  // Pair arrays: (r(i), rd(i)) at pair index i, zero outside [0, n) resp.
  // [0, n]; each starts on a 16-byte boundary with kRatioPad pairs before it.
  const size_t nplain = h.size();
  const long long doff[3] = {d.nx + d.ny + d.nz, 2ll * d.nx + d.ny + d.nz + 1, 2ll * (d.nx + d.ny) + d.nz + 2};
  long long rpo[3];
  size_t pos = (nplain + 3) / 4 * 4;
  for (int a = 0; a < 3; ++a) {
    const long long pairs = kRatioPad + n[a] + kRatioTail;
    rpo[a] = (long long)pos + 2 * kRatioPad;
    h.resize(pos + 2 * (size_t)pairs, 0.f);
    const long long poff = a == 0 ? 0 : a == 1 ? d.nx : d.nx + d.ny;
    for (int i = 0; i <= n[a]; ++i) {
      if (i < n[a]) h[(size_t)(rpo[a] + 2 * i)] = h[(size_t)(poff + i)];
      h[(size_t)(rpo[a] + 2 * i + 1)] = h[(size_t)(doff[a] + i)];
    }
    pos = (h.size() + 3) / 4 * 4;
  }
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (g->rat) {
    cudaFree(g->rat);
    g->rat = nullptr;
  }
  if (dev_malloc((void**)&g->rat, h.size() * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    g->rat = nullptr;
    return fail(SOPHIE_ENOMEM, "ratio array allocation failed");
  }
  for (int a = 0; a < 3; ++a) g->rpair_off[a] = rpo[a];
  CUDA_TRY(cudaMemcpy(g->rat, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  g->gen++;
  g->tuned = false;
  return SOPHIE_OK;
}

int sophie_autotune(sophie_grid* g, int* temporal_k, double* ms_per_step) {
  if (!g || !temporal_k || !ms_per_step) return fail(SOPHIE_EINVAL, "NULL argument");
  g->temporal_k = 0;
  int rc = run_autotune(g, ms_per_step);
  if (rc) return rc;
  *temporal_k = g->tuned_k;
  return SOPHIE_OK;
}

int sophie_launch_config(sophie_grid* g, int* out) {
  if (!g || !out) return fail(SOPHIE_EINVAL, "NULL argument");
  const int k = g->use_simple ? 1 : g->temporal_k ? g->temporal_k : g->tuned ? g->tuned_k : 1;
  out[0] = k;
  out[1] = g->ptile.zchunk;
  out[2] = g->ptile.grid;
  BlockedTiling bt{};
  if (k >= 2) bt = g->btile.K == k ? g->btile : blocked_tiling(g->d, k, g->num_sms, 1);
  out[3] = k >= 2 ? bt.grid : 0;
  out[4] = k >= 2 ? bt.zsplit : 0;
  out[5] = k >= 2 ? bt.order : 0;
  out[6] = k >= 2 ? (bt.rows == 2 ? 2 : 4) : 0;
  return SOPHIE_OK;
}

int sophie_launch_count(sophie_grid* g, long long* launches) {
  if (!g || !launches) return fail(SOPHIE_EINVAL, "NULL argument");
  *launches = g->launches;
  return SOPHIE_OK;
}

int sophie_profile(sophie_grid* g, int enable) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  int rc = prof_drain(g);
  if (rc) return rc;
  g->prof = enable != 0;
  if (enable)
    for (int i = 0; i < 4; ++i) {
      g->prof_count[i] = 0;
      g->prof_ms[i] = 0.0;
    }
  return SOPHIE_OK;
}

int sophie_profile_read(sophie_grid* g, int kernel, long long* launches, double* ms) {
  if (!g || !launches || !ms) return fail(SOPHIE_EINVAL, "NULL argument");
  if (kernel < 0 || kernel > 3) return fail(SOPHIE_EINVAL, "bad kernel id");
  int rc = prof_drain(g);
  if (rc) return rc;
  *launches = g->prof_count[kernel];
  *ms = g->prof_ms[kernel];
  return SOPHIE_OK;
}

}  // extern "C"
