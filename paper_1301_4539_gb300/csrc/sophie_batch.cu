// Host runtime of batched cavities (sophie_batch_* in include/sophie.h).
//
// A batch owns many independent PEC cavities that share dx and dt: one arena
// with each cavity's two field buffers, one material-word array, per-cavity
// class tables and explicit tables, per-cavity sources, a device table of
// cavity descriptors and the work lists of the step and energy kernels
// (yee_batch.cu). A run of n steps is n persistent launches; they are
// recorded once into a CUDA graph and replayed while the same run recurs.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sophie.h"
#include "sophie_internal.h"
#include "yee_store.cuh"

using namespace sophie;

namespace {

constexpr double kC0b = 299792458.0;
constexpr double kEps0b = 8.8541878128e-12;
constexpr long long kEnergyChunk = 16384;  // index points per energy item

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return report_error(code, buf);
}

#define BCUDA(call)                                                              \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return bfail(SOPHIE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct BSource {
  int comp, kind;
  double amp, f0, bw, t0;
  long long pos;
};

bool interior_edge(const Dims& d, int c, int i, int j, int k) {
  switch (c) {
    case 0: return i >= 0 && i < d.nx && j >= 1 && j < d.ny && k >= 1 && k < d.nz;
    case 1: return i >= 1 && i < d.nx && j >= 0 && j < d.ny && k >= 1 && k < d.nz;
    default: return i >= 1 && i < d.nx && j >= 1 && j < d.ny && k >= 0 && k < d.nz;
  }
}

}  // namespace

struct sophie_batch {
  int ncav = 0;
  double dx = 0, dt = 0, S64 = 0;
  float S32 = 0;
  std::vector<Dims> dims;
  std::vector<size_t> fofs, fbytes;  // cavity c: buffer b at arena + fofs[c] + b * fbytes[c]
  std::vector<size_t> wofs;          // first material word of cavity c
  long long cells = 0;
  unsigned char* arena = nullptr;   // guard | cavities' buffers | guard
  unsigned char* arena_base = nullptr;
  size_t aguard = 0, abytes = 0;
  uint32_t* words = nullptr;
  float2* coef = nullptr;     // ncav x kMaxClasses
  double* eps_tab = nullptr;  // ncav x kMaxClasses
  float2* ecoef = nullptr;    // explicit entries of all cavities
  double* eeps = nullptr;
  size_t ecap = 0;
  std::vector<size_t> eofs;  // first explicit entry of cavity c
  std::vector<std::vector<BSource>> src;
  float* sval = nullptr;  // [ncav][kBatchMaxSrc][scap]
  int scap = 0;
  std::vector<CavityDesc> h_desc;
  CavityDesc* d_desc = nullptr;
  BatchItem* d_items = nullptr;
  int nitems = 0;
  EnergyItem* d_eitems = nullptr;
  int neitems = 0;
  int* d_efirst = nullptr;
  double* e_part = nullptr;
  double* e_out = nullptr;
  int* counter = nullptr;
  int cur = 0;
  long long n = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int tile_x = 64, tile_y = 16, zchunk = 16, grid = 0, num_sms = 1;  // tile_x 64: TMA kernel, 32: direct
  int* err = nullptr;  // bounded waits of the TMA kernel that ran out
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  long long g_n0 = -1;
  int g_len = 0, g_cur = -1;
  long long launches = 0;
  // Packed layout (sophie_batch_create_packed): the cavities in one grid;
  // every call below goes to batch_packed.cu, only ncav, dims and cells above
  // are used.
  PackedBatch* pk = nullptr;
};

namespace {

void drop_graph(sophie_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_n0 = -1;
}

void free_batch(sophie_batch* b) {
  if (!b) return;
  if (b->pk) {
    packed_destroy(b->pk);
    delete b;
    return;
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  void* bufs[] = {b->arena_base, b->words, b->coef, b->eps_tab, b->ecoef, b->eeps, b->sval, b->d_desc,
                  b->d_items, b->d_eitems, b->d_efirst, b->e_part, b->e_out, b->counter, b->err};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

void fill_desc(sophie_batch* b, int c) {
  CavityDesc& cd = b->h_desc[c];
  cd.d = b->dims[c];
  cd.F[0] = b->arena + b->fofs[c];
  cd.F[1] = b->arena + b->fofs[c] + b->fbytes[c];
  cd.mat = b->words + b->wofs[c];
  cd.coef = b->coef + (size_t)c * kMaxClasses;
  cd.eps_tab = b->eps_tab + (size_t)c * kMaxClasses;
  cd.ecoef = b->ecoef ? b->ecoef + 3 * b->eofs[c] : nullptr;
  cd.eeps = b->eeps ? b->eeps + 3 * b->eofs[c] : nullptr;
  cd.src.n = (int)b->src[c].size();
  for (int q = 0; q < cd.src.n; ++q) {
    cd.src.comp[q] = b->src[c][q].comp;
    cd.src.pos[q] = b->src[c][q].pos;
  }
  cd.src.val = b->sval ? b->sval + (size_t)c * kBatchMaxSrc * b->scap : nullptr;
  cd.src.cap = b->scap;
}

// TMA maps of every cavity (its buffers and words do not move).
int encode_desc_maps(sophie_batch* b) {
  for (int c = 0; c < b->ncav; ++c) {
    CavityDesc& cd = b->h_desc[c];
    fill_desc(b, c);
    if (!encode_maps(cd.d, kF32, cd.F[0], const_cast<uint32_t*>(cd.mat), plain_box_x(kF32), plain_box_y(), &cd.tmF[0],
                     &cd.tmM) ||
        !encode_maps(cd.d, kF32, cd.F[1], nullptr, plain_box_x(kF32), plain_box_y(), &cd.tmF[1], nullptr))
      return bfail(SOPHIE_ECUDA, "cuTensorMapEncodeTiled failed for cavity %d", c);
  }
  return SOPHIE_OK;
}

int upload_desc(sophie_batch* b) {
  for (int c = 0; c < b->ncav; ++c) fill_desc(b, c);
  BCUDA(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), sizeof(CavityDesc) * b->ncav, cudaMemcpyHostToDevice,
                        b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  return SOPHIE_OK;
}

int upload_desc_one(sophie_batch* b, int c) {
  fill_desc(b, c);
  BCUDA(cudaMemcpyAsync(b->d_desc + c, &b->h_desc[c], sizeof(CavityDesc), cudaMemcpyHostToDevice, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  return SOPHIE_OK;
}

bool tiles_supported(int tx, int ty) {
  return (tx == 64 && ty == 16) || (tx == 32 && batch_tile_supported(ty));
}

// Step work list for tx x ty tiles and z chunk zc: cavity by cavity, then z
// chunk, y tile, x tile, so that the items taken together share planes in L2.
// tx = 64 (ty = 16) runs the TMA-staged plain kernel over the list, tx = 32
// the direct-load kernel.
int build_items(sophie_batch* b, int tx, int ty, int zc) {
  std::vector<BatchItem> it;
  for (int c = 0; c < b->ncav; ++c) {
    const Dims& d = b->dims[c];
    for (int z0 = 0; z0 < d.nz; z0 += zc)
      for (int y0 = 0; y0 < d.ny; y0 += ty)
        for (int x0 = 0; x0 < d.nx; x0 += tx) it.push_back({c, x0, y0, z0, std::min(z0 + zc, d.nz)});
  }
  if (it.size() > 0x7ffffff0u) return bfail(SOPHIE_EINVAL, "too many work items");
  drop_graph(b);
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  if (dev_malloc((void**)&b->d_items, it.size() * sizeof(BatchItem)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(SOPHIE_ENOMEM, "work list allocation failed");
  }
  BCUDA(cudaMemcpy(b->d_items, it.data(), it.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  b->nitems = (int)it.size();
  b->tile_x = tx;
  b->tile_y = ty;
  b->zchunk = zc;
  b->grid = tx == 64 ? 2 * b->num_sms : b->num_sms * batch_blocks_per_sm(ty);
  return SOPHIE_OK;
}

// Waveform tables covering steps [0, need).
int ensure_src_capacity(sophie_batch* b, long long need) {
  if (need > (1ll << 30)) return bfail(SOPHIE_EINVAL, "step count too large");
  if (need <= b->scap) return SOPHIE_OK;
  int cap = b->scap ? b->scap : 1024;
  while (cap < need) cap *= 2;
  std::vector<float> h((size_t)b->ncav * kBatchMaxSrc * cap, 0.f);
  for (int c = 0; c < b->ncav; ++c)
    for (size_t q = 0; q < b->src[c].size(); ++q) {
      const BSource& s = b->src[c][q];
      float* col = h.data() + ((size_t)c * kBatchMaxSrc + q) * cap;
      for (int m = 0; m < cap; ++m) col[m] = (float)source_waveform(s.kind, s.amp, s.f0, s.bw, s.t0, b->dt, m);
    }
  BCUDA(cudaStreamSynchronize(b->stream));
  float* nv = nullptr;
  if (dev_malloc((void**)&nv, h.size() * 4) != cudaSuccess) {
    cudaGetLastError();
    return bfail(SOPHIE_ENOMEM, "source table allocation failed");
  }
  BCUDA(cudaMemcpy(nv, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
  if (b->sval) cudaFree(b->sval);
  b->sval = nv;
  b->scap = cap;
  drop_graph(b);
  return upload_desc(b);
}

int copy_cavity_component(sophie_batch* b, int cav, int comp, void* host, bool to_device, int buf) {
  const Dims& d = b->dims[cav];
  cudaMemcpy3DParms p{};
  unsigned char* base = b->arena + b->fofs[cav] + (size_t)buf * b->fbytes[cav];
  cudaPitchedPtr dev = make_cudaPitchedPtr(base + (size_t)comp * d.plane * 4, (size_t)d.nxp * 4, (size_t)d.nx + 1,
                                           (size_t)6 * d.ny1);
  cudaPitchedPtr hst = make_cudaPitchedPtr(host, (size_t)(d.nx + 1) * 4, (size_t)d.nx + 1, (size_t)d.ny1);
  p.extent = make_cudaExtent((size_t)(d.nx + 1) * 4, (size_t)d.ny1, (size_t)d.nz1);
  if (to_device) {
    p.srcPtr = hst;
    p.dstPtr = dev;
    p.kind = cudaMemcpyHostToDevice;
  } else {
    p.srcPtr = dev;
    p.dstPtr = hst;
    p.kind = cudaMemcpyDeviceToHost;
  }
  BCUDA(cudaMemcpy3DAsync(&p, b->stream));
  return SOPHIE_OK;
}

int check_cav(sophie_batch* b, int cav) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (cav < 0 || cav >= b->ncav) return bfail(SOPHIE_EINVAL, "cavity %d outside [0, %d)", cav, b->ncav);
  return SOPHIE_OK;
}

// One step of every cavity reading buffer `cur` (step index nstep).
cudaError_t launch_one(sophie_batch* b, int cur, long long nstep) {
  if (b->tile_x == 64) {
    StepArgs a{};
    a.fmt = kF32;
    for (int c = 0; c < 6; ++c) a.sc[c] = a.isc[c] = 1.f;
    a.S = b->S32;
    a.n0 = nstep;
    a.err = b->err;
    const PlainBatch pb{b->d_desc, b->d_items, b->nitems, cur};
    return launch_step_plain_batch(a, pb, b->grid, b->stream);
  }
  return launch_batch_step(b->d_desc, b->d_items, b->nitems, b->counter, cur, b->S32, nstep, b->tile_y, b->grid,
                           b->stream);
}

// Enqueue the launches of steps [b->n, b->n + n) without a graph.
int enqueue_steps(sophie_batch* b, int n) {
  int cur = b->cur;
  for (int m = 0; m < n; ++m) {
    const cudaError_t e = launch_one(b, cur, b->n + m);
    if (e != cudaSuccess) return bfail(SOPHIE_ECUDA, "batch step launch failed: %s", cudaGetErrorString(e));
    cur = 1 - cur;
  }
  return SOPHIE_OK;
}

int check_err(sophie_batch* b) {
  int h = 0;
  BCUDA(cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  if (h != 0) {
    cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
    return bfail(SOPHIE_ETIMEOUT, "a batch kernel ran out of its bounded wait (code %d)", h);
  }
  return SOPHIE_OK;
}

}  // namespace

extern "C" {

int sophie_batch_create(int ncav, const int* dims, double dx, double dt, sophie_batch** out) {
  if (!out || !dims) return bfail(SOPHIE_EINVAL, "NULL argument");
  *out = nullptr;
  if (ncav < 1 || ncav > (1 << 22)) return bfail(SOPHIE_EINVAL, "cavity count must be in [1, 2^22]");
  if (!(dx > 0) || !std::isfinite(dx) || !(dt > 0) || !std::isfinite(dt))
    return bfail(SOPHIE_EINVAL, "dx and dt must be finite and > 0");
  if (kC0b * dt * std::sqrt(3.0) > dx * (1.0 + 1e-12))
    return bfail(SOPHIE_EUNSTABLE, "dt above the 3-D Courant limit dx/(c sqrt 3)");
  sophie_batch* b = new (std::nothrow) sophie_batch();
  if (!b) return bfail(SOPHIE_ENOMEM, "host allocation failed");
  b->ncav = ncav;
  b->dx = dx;
  b->dt = dt;
  b->S64 = kC0b * dt / dx;
  b->S32 = (float)b->S64;
  size_t fb = 0, wb = 0;
  for (int c = 0; c < ncav; ++c) {
    const int nx = dims[3 * c], ny = dims[3 * c + 1], nz = dims[3 * c + 2];
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) {
      free_batch(b);
      return bfail(SOPHIE_EINVAL, "cavity %d: sizes must be in [1, 4096]", c);
    }
    Dims d{};
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.nxp = ((nx + 1) + 7) / 8 * 8;
    d.ny1 = ny + 1;
    d.nz1 = nz + 1;
    d.plane = (long long)d.ny1 * d.nxp;
    d.zstride = 6 * d.plane;
    b->dims.push_back(d);
    const size_t bytes = ((size_t)d.zstride * d.nz1 * 4 + 255) / 256 * 256;
    b->fofs.push_back(fb);
    b->fbytes.push_back(bytes);
    fb += 2 * bytes;
    b->wofs.push_back(wb);
    wb += ((size_t)d.plane * d.nz1 + 63) / 64 * 64;
    b->cells += (long long)nx * ny * nz;
  }
  b->src.resize(ncav);
  b->eofs.assign(ncav, 0);
  b->h_desc.resize(ncav);
  int rc = SOPHIE_OK;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (dev_malloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = bfail(SOPHIE_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
      return false;
    }
    return true;
  };
  do {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "cudaStreamCreate failed");
      break;
    }
    b->own_stream = true;
    b->aguard = (size_t)1 << 20;
    b->abytes = fb;
    if (!alloc((void**)&b->arena_base, fb + 2 * b->aguard) || !alloc((void**)&b->words, wb * 4)) break;
    b->arena = b->arena_base + b->aguard;
    if (cudaMemsetAsync(b->arena_base, kGuardByte, b->aguard, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->arena + fb, kGuardByte, b->aguard, b->stream) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "cudaMemsetAsync failed");
      break;
    }
    if (!alloc((void**)&b->coef, (size_t)ncav * kMaxClasses * sizeof(float2))) break;
    if (!alloc((void**)&b->eps_tab, (size_t)ncav * kMaxClasses * sizeof(double))) break;
    if (!alloc((void**)&b->d_desc, (size_t)ncav * sizeof(CavityDesc))) break;
    if (!alloc((void**)&b->counter, sizeof(int)) || !alloc((void**)&b->err, sizeof(int))) break;
    if (cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "cudaMemsetAsync failed");
      break;
    }
    if (!alloc((void**)&b->e_out, (size_t)ncav * 8)) break;
    if (!alloc((void**)&b->d_efirst, (size_t)(ncav + 1) * 4)) break;
    if (cudaMemsetAsync(b->arena, 0, fb, b->stream) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "cudaMemsetAsync failed");
      break;
    }
    // Energy work list.
    std::vector<EnergyItem> ei;
    std::vector<int> first;
    for (int c = 0; c < ncav; ++c) {
      first.push_back((int)ei.size());
      const long long np = (long long)b->dims[c].plane * b->dims[c].nz1;
      for (long long p0 = 0; p0 < np; p0 += kEnergyChunk) ei.push_back({c, p0, std::min(p0 + kEnergyChunk, np)});
    }
    first.push_back((int)ei.size());
    b->neitems = (int)ei.size();
    if (!alloc((void**)&b->d_eitems, ei.size() * sizeof(EnergyItem)) ||
        !alloc((void**)&b->e_part, ei.size() * sizeof(double)))
      break;
    if (cudaMemcpy(b->d_eitems, ei.data(), ei.size() * sizeof(EnergyItem), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_efirst, first.data(), first.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "work list upload failed");
      break;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->num_sms <= 0) b->num_sms = 1;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    rc = encode_desc_maps(b);
    if (rc) break;
    rc = sophie_batch_set_materials(b, nullptr, nullptr);
    if (rc) break;
    rc = build_items(b, 64, 16, 16);
    if (rc) break;
    rc = ensure_src_capacity(b, 1);
    if (rc) break;
  } while (0);
  if (rc != SOPHIE_OK) {
    free_batch(b);
    return rc;
  }
  handle_register(b);
  *out = b;
  return SOPHIE_OK;
}

int sophie_batch_pack_plan(int ncav, const int* dims, int* origins, int* extent) {
  if (!dims || !origins || !extent) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (ncav < 1 || ncav > (1 << 22)) return bfail(SOPHIE_EINVAL, "cavity count must be in [1, 2^22]");
  for (int c = 0; c < 3 * ncav; ++c)
    if (dims[c] < 1 || dims[c] > 4096) return bfail(SOPHIE_EINVAL, "cavity %d: sizes must be in [1, 4096]", c / 3);
  return packed_plan(ncav, dims, origins, extent);
}

int sophie_batch_create_packed(int ncav, const int* dims, double dx, double dt, sophie_batch** out) {
  if (!out || !dims) return bfail(SOPHIE_EINVAL, "NULL argument");
  *out = nullptr;
  if (ncav < 1 || ncav > (1 << 22)) return bfail(SOPHIE_EINVAL, "cavity count must be in [1, 2^22]");
  if (!(dx > 0) || !std::isfinite(dx) || !(dt > 0) || !std::isfinite(dt))
    return bfail(SOPHIE_EINVAL, "dx and dt must be finite and > 0");
  if (kC0b * dt * std::sqrt(3.0) > dx * (1.0 + 1e-12))
    return bfail(SOPHIE_EUNSTABLE, "dt above the 3-D Courant limit dx/(c sqrt 3)");
  sophie_batch* b = new (std::nothrow) sophie_batch();
  if (!b) return bfail(SOPHIE_ENOMEM, "host allocation failed");
  b->ncav = ncav;
  b->dx = dx;
  b->dt = dt;
  for (int c = 0; c < ncav; ++c) {
    const int nx = dims[3 * c], ny = dims[3 * c + 1], nz = dims[3 * c + 2];
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) {
      delete b;
      return bfail(SOPHIE_EINVAL, "cavity %d: sizes must be in [1, 4096]", c);
    }
    Dims d{};
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.nxp = ((nx + 1) + 7) / 8 * 8;
    d.ny1 = ny + 1;
    d.nz1 = nz + 1;
    d.plane = (long long)d.ny1 * d.nxp;
    d.zstride = 6 * d.plane;
    b->dims.push_back(d);
    b->cells += (long long)nx * ny * nz;
  }
  b->src.resize(ncav);
  const int rc = packed_create(ncav, dims, dx, dt, &b->pk);
  if (rc) {
    delete b;
    return rc;
  }
  handle_register(b);
  *out = b;
  return SOPHIE_OK;
}

int sophie_batch_layout(sophie_batch* b, int* packed, int* extent, int* temporal_k) {
  if (!b || !packed || !extent || !temporal_k) return bfail(SOPHIE_EINVAL, "NULL argument");
  *packed = b->pk ? 1 : 0;
  extent[0] = extent[1] = extent[2] = 0;
  *temporal_k = 1;
  if (b->pk) {
    long long cells, gcells;
    int tx, ty;
    packed_info(b->pk, &cells, &gcells, &tx, &ty, temporal_k);
    packed_extent(b->pk, extent);
  }
  return SOPHIE_OK;
}

int sophie_batch_cavity_origin(sophie_batch* b, int cav, int* xyz) {
  const int rc = check_cav(b, cav);
  if (rc) return rc;
  if (!xyz) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (!b->pk) return bfail(SOPHIE_ENOTSUP, "not a packed batch");
  return packed_origin(b->pk, cav, xyz);
}

int sophie_batch_destroy(sophie_batch* b) {
  if (!b) return SOPHIE_OK;
  if (!handle_release(b)) return bfail(SOPHIE_EINVAL, "not a live batch (already destroyed?)");
  free_batch(b);
  return SOPHIE_OK;
}

int sophie_batch_check_guards(sophie_batch* b, long long* bad_bytes) {
  if (!b || !bad_bytes) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (b->pk) return packed_check_guards(b->pk, bad_bytes);
  unsigned long long* d = nullptr;
  if (dev_malloc((void**)&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(SOPHIE_ENOMEM, "guard check counter allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = launch_guard_check(b->arena_base, b->aguard, kGuardByte, d, b->stream);
  if (e == cudaSuccess) e = launch_guard_check(b->arena + b->abytes, b->aguard, kGuardByte, d, b->stream);
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(SOPHIE_ECUDA, "guard check failed: %s", cudaGetErrorString(e));
  b->launches += 2;
  *bad_bytes = (long long)h;
  return SOPHIE_OK;
}

int sophie_batch_set_materials(sophie_batch* b, const float* eps, const float* sig) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (!eps && sig) return bfail(SOPHIE_EINVAL, "sigma given without eps_r");
  const long long q = first_bad_material(eps, sig, b->cells, std::max(1, (int)std::thread::hardware_concurrency()));
  if (q >= 0) {
    if (eps && !(eps[q] >= 1.0f))
      return bfail(SOPHIE_EINVAL, "eps_r[%lld] = %g must be >= 1 (+inf: conductor)", q, (double)eps[q]);
    return bfail(SOPHIE_EINVAL, "sigma[%lld] = %g must be finite and >= 0", q, (double)sig[q]);
  }
  if (b->pk) return packed_set_materials(b->pk, eps, sig);
  BCUDA(cudaStreamSynchronize(b->stream));
  const int nc = b->ncav;
  std::vector<size_t> cofs(nc);
  {
    size_t o = 0;
    for (int c = 0; c < nc; ++c) {
      cofs[c] = o;
      o += (size_t)b->dims[c].nx * b->dims[c].ny * b->dims[c].nz;
    }
  }
  // Build every cavity's words and tables on worker threads; upload words as
  // each finishes.
  std::vector<MaterialTables> tabs(nc);
  std::atomic<int> next(0);
  std::atomic<int> err(0);
  const int nth = std::max(1, std::min<int>(nc, (int)std::thread::hardware_concurrency()));
  auto work = [&]() {
    std::vector<uint32_t> w;
    for (;;) {
      const int c = next.fetch_add(1);
      if (c >= nc || err.load()) return;
      const Dims& d = b->dims[c];
      w.assign((size_t)d.plane * d.nz1, 0u);
      if (build_material_tables(d, b->dt, b->S64, eps ? eps + cofs[c] : nullptr, sig ? sig + cofs[c] : nullptr,
                                w.data(), &tabs[c], 1) != 0) {
        err.store(1);
        return;
      }
      for (const BSource& s : b->src[c]) w[s.pos] |= kSrcFlag;
      if (cudaMemcpy(b->words + b->wofs[c], w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        err.store(2);
        return;
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(work);
  for (std::thread& t : th) t.join();
  if (err.load() == 1) return bfail(SOPHIE_ETOOMANYMAT, "more than 2^29 explicit material entries in a cavity");
  if (err.load() == 2) return bfail(SOPHIE_ECUDA, "material word upload failed");
  // Class tables (padded to kMaxClasses) and concatenated explicit tables.
  std::vector<float2> coef((size_t)nc * kMaxClasses, make_float2(0.f, 0.f));
  std::vector<double> epsv((size_t)nc * kMaxClasses, 0.0);
  size_t ne = 0;
  for (int c = 0; c < nc; ++c) {
    std::copy(tabs[c].coef.begin(), tabs[c].coef.end(), coef.begin() + (size_t)c * kMaxClasses);
    std::copy(tabs[c].eps.begin(), tabs[c].eps.end(), epsv.begin() + (size_t)c * kMaxClasses);
    b->eofs[c] = ne;
    ne += tabs[c].eeps.size() / 3;
  }
  BCUDA(cudaMemcpy(b->coef, coef.data(), coef.size() * sizeof(float2), cudaMemcpyHostToDevice));
  BCUDA(cudaMemcpy(b->eps_tab, epsv.data(), epsv.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (ne > b->ecap) {
    if (b->ecoef) cudaFree(b->ecoef);
    if (b->eeps) cudaFree(b->eeps);
    b->ecoef = nullptr;
    b->eeps = nullptr;
    b->ecap = 0;
    if (dev_malloc((void**)&b->ecoef, ne * 3 * sizeof(float2)) != cudaSuccess ||
        dev_malloc((void**)&b->eeps, ne * 3 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return bfail(SOPHIE_ENOMEM, "explicit material tables (%zu entries) allocation failed", ne);
    }
    b->ecap = ne;
  }
  for (int c = 0; c < nc; ++c) {
    const size_t k = tabs[c].eeps.size();
    if (!k) continue;
    BCUDA(cudaMemcpy(b->ecoef + 3 * b->eofs[c], tabs[c].ecoef.data(), k * sizeof(float2), cudaMemcpyHostToDevice));
    BCUDA(cudaMemcpy(b->eeps + 3 * b->eofs[c], tabs[c].eeps.data(), k * sizeof(double), cudaMemcpyHostToDevice));
  }
  drop_graph(b);
  return upload_desc(b);
}

int sophie_batch_add_source(sophie_batch* b, int cav, int comp, int i, int j, int k, double amp, double f0,
                            double bw, double t0, int kind) {
  int rc = check_cav(b, cav);
  if (rc) return rc;
  const Dims& d = b->dims[cav];
  if (comp < 0 || comp > 2) return bfail(SOPHIE_EINVAL, "source component must be 0, 1 or 2 (E)");
  if (!interior_edge(d, comp, i, j, k))
    return bfail(SOPHIE_EINVAL, "source edge (%d,%d,%d) of comp %d is not interior", i, j, k, comp);
  if (kind != SOPHIE_GAUSS_SINE && kind != SOPHIE_GAUSS) return bfail(SOPHIE_EINVAL, "bad waveform kind");
  if (!std::isfinite(amp) || !std::isfinite(f0) || !std::isfinite(t0) || !(bw > 0) || !std::isfinite(bw))
    return bfail(SOPHIE_EINVAL, "bad waveform parameters");
  if ((int)b->src[cav].size() >= kBatchMaxSrc)
    return bfail(SOPHIE_EINVAL, "at most %d sources per cavity", kBatchMaxSrc);
  if (b->pk) {
    rc = packed_add_source(b->pk, cav, comp, i, j, k, amp, f0, bw, t0, kind);
    if (rc) return rc;
    b->src[cav].push_back({comp, kind, amp, f0, bw, t0, ((long long)k * d.ny1 + j) * d.nxp + i});
    return SOPHIE_OK;
  }
  const long long pos = ((long long)k * d.ny1 + j) * d.nxp + i;
  b->src[cav].push_back({comp, kind, amp, f0, bw, t0, pos});
  BCUDA(cudaStreamSynchronize(b->stream));
  const size_t q = b->src[cav].size() - 1;
  std::vector<float> col(b->scap);
  for (int m = 0; m < b->scap; ++m) col[m] = (float)source_waveform(kind, amp, f0, bw, t0, b->dt, m);
  BCUDA(cudaMemcpy(b->sval + ((size_t)cav * kBatchMaxSrc + q) * b->scap, col.data(), col.size() * 4,
                   cudaMemcpyHostToDevice));
  if (launch_or_flag(b->words + b->wofs[cav], pos, kSrcFlag, b->stream) != cudaSuccess)
    return bfail(SOPHIE_ECUDA, "flag launch failed");
  b->launches++;
  drop_graph(b);
  return upload_desc_one(b, cav);
}

int sophie_batch_step(sophie_batch* b, int n) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (n < 0) return bfail(SOPHIE_EINVAL, "n must be >= 0");
  if (n == 0) return SOPHIE_OK;
  if (b->pk) return packed_step(b->pk, n);
  int rc = ensure_src_capacity(b, b->n + n);
  if (rc) return rc;
  if (!b->use_graph) {
    rc = enqueue_steps(b, n);
    if (rc) return rc;
  } else {
    if (!(b->gexec && b->g_n0 == b->n && b->g_len == n && b->g_cur == b->cur)) {
      drop_graph(b);
      cudaGraph_t graph = nullptr;
      BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_steps(b, n);
      const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return bfail(SOPHIE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        b->gexec = nullptr;
        return bfail(SOPHIE_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
      }
      b->g_n0 = b->n;
      b->g_len = n;
      b->g_cur = b->cur;
    }
    BCUDA(cudaGraphLaunch(b->gexec, b->stream));
  }
  b->launches += n;
  b->n += n;
  if (n & 1) b->cur = 1 - b->cur;
  return SOPHIE_OK;
}

int sophie_batch_get_step(sophie_batch* b, long long* n) {
  if (!b || !n) return bfail(SOPHIE_EINVAL, "NULL argument");
  *n = b->pk ? packed_step_count(b->pk) : b->n;
  return SOPHIE_OK;
}

int sophie_batch_info(sophie_batch* b, long long* cells, long long* work_items, int* tile_x, int* tile_y,
                      int* zchunk) {
  if (!b || !cells || !work_items || !tile_x || !tile_y || !zchunk) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (b->pk) {  // packed: the grid's cells, its step kernel's output tile, zchunk 0
    int K = 1;
    packed_info(b->pk, cells, work_items, tile_x, tile_y, &K);
    *zchunk = 0;
    return SOPHIE_OK;
  }
  *cells = b->cells;
  *work_items = b->nitems;
  *tile_x = b->tile_x;
  *tile_y = b->tile_y;
  *zchunk = b->zchunk;
  return SOPHIE_OK;
}

int sophie_batch_energy(sophie_batch* b, double* W) {
  if (!b || !W) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (b->pk) return packed_energy(b->pk, W);
  const double dx = b->dx;
  const cudaError_t e = launch_batch_energy(b->d_desc, b->d_eitems, b->neitems, b->d_efirst, b->ncav, b->cur, b->S32,
                                            b->e_part, 0.5 * kEps0b * dx * dx * dx, b->e_out, b->stream);
  if (e != cudaSuccess) return bfail(SOPHIE_ECUDA, "batch energy launch failed: %s", cudaGetErrorString(e));
  b->launches += 2;
  BCUDA(cudaMemcpyAsync(W, b->e_out, (size_t)b->ncav * 8, cudaMemcpyDeviceToHost, b->stream));
  int rc = check_err(b);
  if (rc) return rc;
  for (int c = 0; c < b->ncav; ++c)
    if (!std::isfinite(W[c])) return bfail(SOPHIE_ENONFINITE, "energy of cavity %d is not finite", c);
  return SOPHIE_OK;
}

int sophie_batch_set_fields(sophie_batch* b, int cav, int comp, const float* host) {
  int rc = check_cav(b, cav);
  if (rc) return rc;
  if (!host) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (comp < 0 || comp > 5) return bfail(SOPHIE_EINVAL, "comp must be in 0..5");
  if (b->pk) return packed_set_fields(b->pk, cav, comp, host);
  for (int buf = 0; buf < 2; ++buf) {
    rc = copy_cavity_component(b, cav, comp, const_cast<float*>(host), true, buf);
    if (rc) return rc;
    const cudaError_t e = launch_mask_component(b->arena + b->fofs[cav] + (size_t)buf * b->fbytes[cav], 4,
                                                b->dims[cav], comp, b->stream);
    if (e != cudaSuccess) return bfail(SOPHIE_ECUDA, "mask launch failed: %s", cudaGetErrorString(e));
    b->launches++;
  }
  BCUDA(cudaStreamSynchronize(b->stream));
  return SOPHIE_OK;
}

int sophie_batch_get_fields(sophie_batch* b, int cav, int comp, float* host) {
  int rc = check_cav(b, cav);
  if (rc) return rc;
  if (!host) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (comp < 0 || comp > 5) return bfail(SOPHIE_EINVAL, "comp must be in 0..5");
  if (b->pk) return packed_get_fields(b->pk, cav, comp, host);
  rc = copy_cavity_component(b, cav, comp, host, false, b->cur);
  if (rc) return rc;
  BCUDA(cudaStreamSynchronize(b->stream));
  return SOPHIE_OK;
}

int sophie_batch_reset(sophie_batch* b) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (b->pk) return packed_reset(b->pk);
  BCUDA(cudaMemsetAsync(b->arena, 0, b->abytes, b->stream));
  b->n = 0;
  b->cur = 0;
  return SOPHIE_OK;
}

int sophie_batch_set_stream(sophie_batch* b, void* cuda_stream) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (!cuda_stream) return bfail(SOPHIE_EINVAL, "the batch needs a created stream (graphs cannot record the legacy stream)");
  if (b->pk) return packed_set_stream(b->pk, cuda_stream);
  BCUDA(cudaStreamSynchronize(b->stream));
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = (cudaStream_t)cuda_stream;
  drop_graph(b);
  return SOPHIE_OK;
}

int sophie_batch_configure(sophie_batch* b, int tile_x, int tile_y, int zchunk, int use_graph) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (b->pk) {  // the packed grid's tilings come from its autotuner
    if (tile_x || tile_y || zchunk) return bfail(SOPHIE_ENOTSUP, "a packed batch takes no tile or z chunk settings");
    packed_set_graph(b->pk, use_graph != 0);
    return SOPHIE_OK;
  }
  const int tx = tile_x ? tile_x : b->tile_x;
  const int ty = tile_y ? tile_y : (tile_x == 64 ? 16 : b->tile_y);
  if (!tiles_supported(tx, ty)) return bfail(SOPHIE_ENOTSUP, "tiles %d x %d not built (64 x 16; 32 x 4, 8, 16)", tx, ty);
  if (zchunk < 0) return bfail(SOPHIE_EINVAL, "zchunk must be >= 0");
  b->use_graph = use_graph != 0;
  const int zc = zchunk ? zchunk : b->zchunk;
  if (tx != b->tile_x || ty != b->tile_y || zc != b->zchunk) return build_items(b, tx, ty, zc);
  return SOPHIE_OK;
}

int sophie_batch_autotune(sophie_batch* b, int* tile_x, int* tile_y, int* zchunk, double* ms_per_step) {
  if (!b || !tile_x || !tile_y || !zchunk || !ms_per_step) return bfail(SOPHIE_EINVAL, "NULL argument");
  if (b->pk) {  // k and the tilings of the packed grid; zchunk gets 0
    int K = 1;
    const int rc = packed_autotune(b->pk, &K, ms_per_step);
    if (rc) return rc;
    long long c0, c1;
    packed_info(b->pk, &c0, &c1, tile_x, tile_y, &K);
    *zchunk = 0;
    return SOPHIE_OK;
  }
  int rc = ensure_src_capacity(b, b->n + 1);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCUDA(cudaEventCreate(&e0));
  BCUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int btx = b->tile_x, bty = b->tile_y, bzc = b->zchunk;
  struct Cand {
    int tx, ty, zc;
  };
  const Cand cands[] = {{64, 16, 4}, {64, 16, 8},  {64, 16, 16}, {64, 16, 32}, {64, 16, 96},
                        {32, 8, 16}, {32, 16, 16}, {32, 16, 96}, {32, 4, 8}};
  for (const Cand& cd : cands) {
    rc = build_items(b, cd.tx, cd.ty, cd.zc);
    if (rc) break;
    // Trial launches read the current buffer and write the spare one; the
    // state does not advance.
    if (launch_one(b, b->cur, b->n) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "autotune launch failed");
      break;
    }
    cudaEventRecord(e0, b->stream);
    const int reps = 3;
    for (int r = 0; r < reps; ++r)
      if (launch_one(b, b->cur, b->n) != cudaSuccess) rc = bfail(SOPHIE_ECUDA, "autotune launch failed");
    cudaEventRecord(e1, b->stream);
    if (rc) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = bfail(SOPHIE_ECUDA, "autotune timing failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->launches += reps + 1;
    if (ms / reps < best) {
      best = ms / reps;
      btx = cd.tx;
      bty = cd.ty;
      bzc = cd.zc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = check_err(b);
  if (rc) return rc;
  rc = build_items(b, btx, bty, bzc);
  if (rc) return rc;
  *tile_x = btx;
  *tile_y = bty;
  *zchunk = bzc;
  *ms_per_step = best;
  return SOPHIE_OK;
}

int sophie_batch_launch_count(sophie_batch* b, long long* launches) {
  if (!b || !launches) return bfail(SOPHIE_EINVAL, "NULL argument");
  *launches = b->pk ? packed_launches(b->pk) : b->launches;
  return SOPHIE_OK;
}

int sophie_batch_sync(sophie_batch* b) {
  if (!b) return bfail(SOPHIE_EINVAL, "NULL batch");
  if (b->pk) return packed_sync(b->pk);
  return check_err(b);
}

}  // extern "C"
