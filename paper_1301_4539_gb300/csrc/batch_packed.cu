// Packed layout of a batch of cavities (sophie_batch_create_packed).
//
// The cavities are placed side by side in one large grid, each separated from
// its neighbours by one layer of perfectly conducting cells. A conducting cell
// makes every edge it touches a PEC edge (Ca = Cb = 0), exactly like an outer
// wall, so each cavity evolves exactly as it would alone: its wall edges are
// PEC, its wall-normal faces see only PEC zeros, and the faces inside the
// separator cells stay zero (the oracle pins this: a conducting layer splits a
// grid into cavities that equal separate runs bit for bit). The whole batch is
// then one grid for the tuned single-grid step kernels: one persistent
// temporally blocked launch per K steps (K and the tilings chosen by the
// grid's autotuner), recorded into a CUDA graph and replayed.
//
// Placement: cavities sorted by thickness bands and height are laid out in
// rows along x, rows stacked along y into layers, layers stacked along z
// (each layer as thick as its thickest row); several footprints and band
// widths are tried and the smallest packed volume is kept.
//
// Materials: each cavity's words and tables are built as for a single grid
// (materials.cu), then written into the packed word array: class points keep
// global classes when all cavities' class materials fit the 511-entry table,
// otherwise they become explicit entries; explicit indices are offset by the
// cavity's first entry. Cells outside the cavities are conductors (word 0).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "grid_state.h"
#include "yee_energy.cuh"

namespace sophie {

using grid::fail;

namespace {

constexpr long long kPackEnergyChunk = 16384;  // cavity points per energy item

struct PackSrc {
  int cav, comp, kind;
  double amp, f0, bw, t0;
  long long pos;  // packed index point
  int order;      // insertion rank (ties on one point keep it)
};

// Cavity c occupies cells [ox, ox + nx) x [oy, oy + ny) x [oz, oz + nz).
struct CavBox {
  int ox, oy, oz, nx, ny, nz;
};

// Rows of cavities along x, stacked along y into layers of width W and depth
// H, layers stacked along z; cavities sorted by (thickness band, height,
// width). Returns the packed extent in z; boxes get their origins.
int pack_layers(std::vector<CavBox>& box, int W, int H, int band) {
  const int n = (int)box.size();
  std::vector<int> order(n);
  for (int c = 0; c < n; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ba = box[a].nz / band, bb = box[b].nz / band;
    if (ba != bb) return ba > bb;
    if (box[a].ny != box[b].ny) return box[a].ny > box[b].ny;
    return box[a].nx > box[b].nx;
  });
  // rows: consecutive cavities of one band while they fit in W (one separator
  // cell after each cavity; the last may end on the grid wall)
  std::vector<std::vector<int>> rows;
  std::vector<int> cur;
  int x = 0;
  for (int c : order) {
    const bool fits = x + box[c].nx <= W;
    if (!cur.empty() && (!fits || box[c].nz / band != box[cur[0]].nz / band)) {
      rows.push_back(cur);
      cur.clear();
      x = 0;
    }
    cur.push_back(c);
    x += box[c].nx + 1;
  }
  if (!cur.empty()) rows.push_back(cur);
  int z = 0, y = 0, T = 0;
  std::vector<std::pair<const std::vector<int>*, int>> layer;
  auto flush = [&]() {
    for (auto& ry : layer) {
      int xx = 0;
      for (int c : *ry.first) {
        box[c].ox = xx;
        box[c].oy = ry.second;
        box[c].oz = z;
        xx += box[c].nx + 1;
      }
    }
    z += T + 1;
    y = 0;
    T = 0;
    layer.clear();
  };
  for (const auto& r : rows) {
    int h = 0, t = 0;
    for (int c : r) {
      h = std::max(h, box[c].ny);
      t = std::max(t, box[c].nz);
    }
    if (!layer.empty() && y + h > H) flush();
    layer.push_back({&r, y});
    y += h + 1;
    T = std::max(T, t);
  }
  if (!layer.empty()) flush();
  return z - 1;  // the last layer's separator is the grid wall
}

}  // namespace

struct PackedBatch {
  int ncav = 0;
  std::vector<CavBox> box;
  long long cells = 0;  // cells of all cavities
  int NX = 0, NY = 0, NZ = 0;
  double dx = 0, dt = 0;
  sophie_grid* g = nullptr;
  cudaStream_t stream = nullptr;
  // sources (device tables installed in the grid)
  std::vector<PackSrc> src;
  long long* d_pos = nullptr;
  int* d_comp = nullptr;
  int* d_row = nullptr;
  float* d_val = nullptr;
  int cap = 0;
  bool src_dirty = false;  // sources added since the device tables were built
  // per-cavity energy
  CavBox* d_box = nullptr;
  EnergyItem* d_items = nullptr;
  int nitems = 0;
  int* d_first = nullptr;
  double* d_part = nullptr;
  double* d_out = nullptr;
  // graph replay
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  long long g_n0 = -1;
  int g_len = 0, g_cur = -1;
  long long g_launch = 0;  // step launches in the recorded graph
  int g_flip = 0;          // whether they leave the state in the other buffer
  long long launches = 0;
};

namespace {

constexpr int kPackEThreads = 256;

// Energy of every cavity (the single grid's per-point term over the cavity's
// own index points, at their packed positions): item partial sums, then each
// cavity's partials added in item order (deterministic).
__global__ void __launch_bounds__(kPackEThreads)
packed_energy_partial_kernel(const __grid_constant__ StepArgs a, const CavBox* __restrict__ boxes,
                             const EnergyItem* __restrict__ items, const double* eps_tab, double* partials) {
  __shared__ double sh[kPackEThreads / 32];
  const EnergyItem w = items[blockIdx.x];
  const CavBox b = boxes[w.cav];
  const Dims d = a.d;
  const float* f = static_cast<const float*>(a.fin);
  const float isc[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
  const long long nx1 = b.nx + 1, ny1 = b.ny + 1;
  double acc = 0.0;
  for (long long p = w.p0 + threadIdx.x; p < w.p1; p += kPackEThreads) {
    const int i = (int)(p % nx1);
    const long long r = p / nx1;
    const int j = (int)(r % ny1);
    const int k = (int)(r / ny1);
    const int x = b.ox + i, y = b.oy + j, z = b.oz + k;
    const long long pt = ((long long)z * d.ny1 + y) * d.nxp + x;
    acc += point_energy<kF32>(f, d, isc, a.S, a.mat[pt], eps_tab, a.eeps, x, y, z);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kPackEThreads / 32; ++q) t += sh[q];
    partials[blockIdx.x] = t;
  }
}

__global__ void packed_energy_final_kernel(const int* first, int ncav, const double* partials, double scale,
                                           double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncav) return;
  double t = 0.0;
  for (int q = first[c]; q < first[c + 1]; ++q) t += partials[q];
  out[c] = t * scale;
}

void drop_graph(PackedBatch* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->g_n0 = -1;
}

void free_src(PackedBatch* p) {
  void* bufs[] = {p->d_pos, p->d_comp, p->d_row, p->d_val};
  for (void* q : bufs)
    if (q) cudaFree(q);
  p->d_pos = nullptr;
  p->d_comp = nullptr;
  p->d_row = nullptr;
  p->d_val = nullptr;
  p->cap = 0;
}

// Whether component c's index (i, j, k) is an edge or face the cavity keeps
// (PEC edges and out-of-range entries are zero; the rules of sophie_set_fields).
bool keep_entry(const CavBox& b, int c, int i, int j, int k) {
  switch (c) {
    case 0: return i < b.nx && j >= 1 && j < b.ny && k >= 1 && k < b.nz;
    case 1: return i >= 1 && i < b.nx && j < b.ny && k >= 1 && k < b.nz;
    case 2: return i >= 1 && i < b.nx && j >= 1 && j < b.ny && k < b.nz;
    case 3: return i <= b.nx && j < b.ny && k < b.nz;
    case 4: return i < b.nx && j <= b.ny && k < b.nz;
    default: return i < b.nx && j < b.ny && k <= b.nz;
  }
}

// Copy component comp of cavity c between the host array ((nz+1)(ny+1)(nx+1),
// x fastest) and field buffer `buf` of the packed grid.
int copy_box(PackedBatch* p, int c, int comp, void* host, bool to_device, int buf) {
  const sophie_grid* g = p->g;
  const Dims& d = g->d;
  const CavBox& b = p->box[c];
  cudaMemcpy3DParms q{};
  cudaPitchedPtr dev = make_cudaPitchedPtr(static_cast<unsigned char*>(g->F[buf]) + (size_t)comp * d.plane * 4,
                                           (size_t)d.nxp * 4, (size_t)d.nx + 1, (size_t)6 * d.ny1);
  cudaPitchedPtr hst = make_cudaPitchedPtr(host, (size_t)(b.nx + 1) * 4, (size_t)b.nx + 1, (size_t)b.ny + 1);
  q.extent = make_cudaExtent((size_t)(b.nx + 1) * 4, (size_t)b.ny + 1, (size_t)b.nz + 1);
  if (to_device) {
    q.srcPtr = hst;
    q.dstPtr = dev;
    q.dstPos = make_cudaPos((size_t)b.ox * 4, (size_t)b.oy, (size_t)b.oz);
    q.kind = cudaMemcpyHostToDevice;
  } else {
    q.srcPtr = dev;
    q.srcPos = make_cudaPos((size_t)b.ox * 4, (size_t)b.oy, (size_t)b.oz);
    q.dstPtr = hst;
    q.kind = cudaMemcpyDeviceToHost;
  }
  CUDA_TRY(cudaMemcpy3DAsync(&q, p->stream));
  return SOPHIE_OK;
}

}  // namespace

int packed_set_materials(PackedBatch* p, const float* eps, const float* sig);

void packed_destroy(PackedBatch* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  drop_graph(p);
  if (p->g) {
    p->g->big_n = 0;
    sophie_destroy_grid(p->g);
  }
  free_src(p);
  void* bufs[] = {p->d_box, p->d_items, p->d_first, p->d_part, p->d_out};
  for (void* q : bufs)
    if (q) cudaFree(q);
  delete p;
}

// Placement of ncav cavities of sizes dims (nx, ny, nz per cavity) in one
// grid with a conducting layer between neighbours: origins (cells) and the
// grid's extent.
void pack_plan(int ncav, const int* dims, std::vector<CavBox>& box, int& NX, int& NY, int& NZ) {
  box.resize(ncav);
  double vol = 0.0;
  int wmin = 1, hmin = 1;
  for (int c = 0; c < ncav; ++c) {
    CavBox& b = box[c];
    b.nx = dims[3 * c];
    b.ny = dims[3 * c + 1];
    b.nz = dims[3 * c + 2];
    b.ox = b.oy = b.oz = 0;
    vol += (double)(b.nx + 1) * (b.ny + 1) * (b.nz + 1);
    wmin = std::max(wmin, b.nx);
    hmin = std::max(hmin, b.ny);
  }
  // Footprints around the cube root of the volume (multiples of 60 in x and
  // 28 in y, the blocked kernel's two-step output tile), band widths 1..8:
  // keep the smallest packed volume (ties: the first tried).
  const double side = std::cbrt(vol / 0.8);
  double best = 1e300;
  std::vector<CavBox> tmp, keep;
  for (double fx : {0.5, 0.7, 1.0, 1.4, 2.0})
    for (double fy : {0.5, 0.7, 1.0, 1.4, 2.0})
      for (int band : {1, 2, 4, 8}) {
        const int W = std::max(wmin, (int)std::lround(side * fx / 60.0) * 60);
        const int H = std::max(hmin, (int)std::lround(side * fy / 28.0) * 28);
        tmp = box;
        const int Z = pack_layers(tmp, W, H, band);
        int X = 0, Y = 0;
        for (const CavBox& b : tmp) {
          X = std::max(X, b.ox + b.nx);
          Y = std::max(Y, b.oy + b.ny);
        }
        const double v = (double)X * Y * Z;
        if (v < best) {
          best = v;
          keep = tmp;
          NX = X;
          NY = Y;
          NZ = Z;
        }
      }
  box = keep;
}

int packed_create(int ncav, const int* dims, double dx, double dt, PackedBatch** out) {
  *out = nullptr;
  PackedBatch* p = new (std::nothrow) PackedBatch();
  if (!p) return fail(SOPHIE_ENOMEM, "host allocation failed");
  p->ncav = ncav;
  p->dx = dx;
  p->dt = dt;
  pack_plan(ncav, dims, p->box, p->NX, p->NY, p->NZ);
  for (const CavBox& b : p->box) p->cells += (long long)b.nx * b.ny * b.nz;
  int rc = sophie_create_grid(p->NX, p->NY, p->NZ, dx, dt, &p->g);
  if (rc) {
    delete p;
    return rc;
  }
  p->stream = p->g->stream;
  // energy work list: chunks of each cavity's index points
  std::vector<EnergyItem> items;
  std::vector<int> first;
  for (int c = 0; c < ncav; ++c) {
    first.push_back((int)items.size());
    const CavBox& b = p->box[c];
    const long long np = (long long)(b.nx + 1) * (b.ny + 1) * (b.nz + 1);
    for (long long p0 = 0; p0 < np; p0 += kPackEnergyChunk)
      items.push_back({c, p0, std::min(p0 + kPackEnergyChunk, np)});
  }
  first.push_back((int)items.size());
  p->nitems = (int)items.size();
  if (dev_malloc((void**)&p->d_box, sizeof(CavBox) * ncav) != cudaSuccess ||
      dev_malloc((void**)&p->d_items, sizeof(EnergyItem) * items.size()) != cudaSuccess ||
      dev_malloc((void**)&p->d_first, sizeof(int) * first.size()) != cudaSuccess ||
      dev_malloc((void**)&p->d_part, sizeof(double) * items.size()) != cudaSuccess ||
      dev_malloc((void**)&p->d_out, sizeof(double) * ncav) != cudaSuccess) {
    cudaGetLastError();
    packed_destroy(p);
    return fail(SOPHIE_ENOMEM, "packed batch tables: allocation failed");
  }
  if (cudaMemcpy(p->d_box, p->box.data(), sizeof(CavBox) * ncav, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_items, items.data(), sizeof(EnergyItem) * items.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(p->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    packed_destroy(p);
    return fail(SOPHIE_ECUDA, "packed batch tables: upload failed");
  }
  rc = packed_set_materials(p, nullptr, nullptr);  // vacuum cavities in conducting walls
  if (rc) {
    packed_destroy(p);
    return rc;
  }
  *out = p;
  return SOPHIE_OK;
}

// eps / sig: every cavity's cells one cavity after the other (x fastest within
// each), or nullptr (vacuum / lossless).
int packed_set_materials(PackedBatch* p, const float* eps, const float* sig) {
  sophie_grid* g = p->g;
  const int nc = p->ncav;
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  CUDA_TRY(cudaEventSynchronize(g->mat_upload_done));  // mat_host may feed an upload
  std::vector<size_t> cofs(nc + 1, 0);
  for (int c = 0; c < nc; ++c) cofs[c + 1] = cofs[c] + (size_t)p->box[c].nx * p->box[c].ny * p->box[c].nz;
  // 1. Each cavity's words and tables, as a single grid of its size.
  std::vector<std::vector<uint32_t>> words(nc);
  std::vector<MaterialTables> tabs(nc);
  std::vector<Dims> dc(nc);
  std::atomic<int> next(0), err(0);
  const int nth = std::max(1, std::min<int>(nc, (int)std::thread::hardware_concurrency()));
  auto run = [&](auto&& fn) {
    next.store(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&]() {
        for (int c = next.fetch_add(1); c < nc && !err.load(); c = next.fetch_add(1)) fn(c);
      });
    for (std::thread& t : th) t.join();
  };
  run([&](int c) {
    const CavBox& b = p->box[c];
    Dims& d = dc[c];
    d.nx = b.nx;
    d.ny = b.ny;
    d.nz = b.nz;
    d.nxp = ((b.nx + 1) + 7) / 8 * 8;
    d.ny1 = b.ny + 1;
    d.nz1 = b.nz + 1;
    d.plane = (long long)d.ny1 * d.nxp;
    d.zstride = 6 * d.plane;
    words[c].assign((size_t)d.plane * d.nz1, 0u);
    if (build_material_tables(d, p->dt, g->S64, eps ? eps + cofs[c] : nullptr, sig ? sig + cofs[c] : nullptr,
                              words[c].data(), &tabs[c], 1) != 0)
      err.store(1);
  });
  if (err.load()) return fail(SOPHIE_ETOOMANYMAT, "more than 2^29 explicit material entries in a cavity");
  // 2. Global classes: every cavity's class materials if they fit the table.
  std::map<std::pair<uint64_t, uint64_t>, int> gcls;
  for (int c = 0; c < nc; ++c)
    for (size_t k = 1; k < tabs[c].eps.size(); ++k) {
      uint64_t e, s;
      memcpy(&e, &tabs[c].eps[k], 8);
      memcpy(&s, &tabs[c].sig[k], 8);
      gcls.emplace(std::make_pair(e, s), 0);
    }
  const bool use_classes = (int)gcls.size() < kMaxClasses;
  std::vector<float2> coef(1, make_float2(0.f, 0.f));
  std::vector<double> ceps(1, 0.0), csig(1, 0.0);
  if (use_classes) {
    for (auto& kv : gcls) {
      double e, s;
      memcpy(&e, &kv.first.first, 8);
      memcpy(&s, &kv.first.second, 8);
      kv.second = (int)coef.size();
      coef.push_back(edge_coefficients(p->dt, g->S64, e, s));
      ceps.push_back(e);
      csig.push_back(s);
    }
  }
  // 3. Each cavity's points into the packed words (explicit indices local to
  // the cavity for now); class points outside the global classes get explicit
  // entries of their three class materials, shared by equal triples.
  std::vector<std::vector<int>> lmap(nc);                     // local class -> global class
  std::vector<std::vector<uint32_t>> synth(nc);               // synthesised triples (local classes)
  uint32_t* W = g->mat_host;
  const Dims& D = g->d;
  memset(W, 0, (size_t)D.plane * D.nz1 * 4);
  run([&](int c) {
    const CavBox& b = p->box[c];
    const Dims& d = dc[c];
    const MaterialTables& t = tabs[c];
    std::vector<int>& lm = lmap[c];
    lm.assign(t.eps.size(), -1);
    lm[0] = 0;
    if (use_classes)
      for (size_t k = 1; k < t.eps.size(); ++k) {
        uint64_t e, s;
        memcpy(&e, &t.eps[k], 8);
        memcpy(&s, &t.sig[k], 8);
        lm[k] = gcls.at(std::make_pair(e, s));
      }
    std::unordered_map<uint32_t, uint32_t> tri;  // class-bit pattern -> synthesised entry
    const uint32_t nexp = (uint32_t)(t.eeps.size() / 3);
    for (int k = 0; k <= b.nz; ++k)
      for (int j = 0; j <= b.ny; ++j) {
        const uint32_t* src = words[c].data() + ((size_t)k * d.ny1 + j) * d.nxp;
        uint32_t* dst = W + ((size_t)(b.oz + k) * D.ny1 + (b.oy + j)) * D.nxp + b.ox;
        for (int i = 0; i <= b.nx; ++i) {
          const uint32_t w = src[i];
          if (w & kExpFlag) {
            dst[i] = w;  // local explicit index, offset below
            continue;
          }
          const int gx = lm[cls_of(w, 0)], gy = lm[cls_of(w, 1)], gz = lm[cls_of(w, 2)];
          if (gx >= 0 && gy >= 0 && gz >= 0) {
            dst[i] = cls_word(gx, gy, gz);
            continue;
          }
          const uint32_t key = w & ~7u;
          auto it = tri.find(key);
          uint32_t q;
          if (it == tri.end()) {
            q = nexp + (uint32_t)synth[c].size();
            tri.emplace(key, q);
            synth[c].push_back(key);
          } else {
            q = it->second;
          }
          dst[i] = (q << 3) | kExpFlag;
        }
      }
    std::vector<uint32_t>().swap(words[c]);
  });
  // 4. Explicit tables, cavity after cavity; words shifted by the offsets.
  std::vector<size_t> off(nc + 1, 0);
  for (int c = 0; c < nc; ++c) off[c + 1] = off[c] + tabs[c].eeps.size() / 3 + synth[c].size();
  if (off[nc] >= (1u << 29)) return fail(SOPHIE_ETOOMANYMAT, "more than 2^29 explicit material entries");
  std::vector<float2> ecoef(off[nc] * 3);
  std::vector<double> eeps(off[nc] * 3);
  run([&](int c) {
    const CavBox& b = p->box[c];
    const MaterialTables& t = tabs[c];
    const size_t o = off[c];
    std::copy(t.ecoef.begin(), t.ecoef.end(), ecoef.begin() + 3 * o);
    std::copy(t.eeps.begin(), t.eeps.end(), eeps.begin() + 3 * o);
    const size_t ne = t.eeps.size() / 3;
    for (size_t q = 0; q < synth[c].size(); ++q)
      for (int e = 0; e < 3; ++e) {
        const uint32_t k = cls_of(synth[c][q], e);
        ecoef[3 * (o + ne + q) + e] = t.coef[k];
        eeps[3 * (o + ne + q) + e] = t.eps[k];
      }
    tabs[c] = MaterialTables();
    if (!o) return;
    const uint32_t add = (uint32_t)o << 3;
    for (int k = 0; k <= b.nz; ++k)
      for (int j = 0; j <= b.ny; ++j) {
        uint32_t* dst = W + ((size_t)(b.oz + k) * D.ny1 + (b.oy + j)) * D.nxp + b.ox;
        for (int i = 0; i <= b.nx; ++i)
          if (dst[i] & kExpFlag) dst[i] += add;
      }
  });
  for (const PackSrc& q : p->src) W[q.pos] |= kSrcFlag;
  g->coef_h = std::move(coef);
  g->eps_h = std::move(ceps);
  g->sig_h = std::move(csig);
  g->ecoef_h = std::move(ecoef);
  g->eeps_h = std::move(eeps);
  g->esig_h.clear();  // gradients are not offered on packed batches
  g->gen++;
  drop_graph(p);
  return grid::upload_materials(g);
}

// The waveform table covering steps [0, need) and the position-sorted source
// arrays, installed in the grid.
int packed_sources(PackedBatch* p, long long need) {
  if (need > (1ll << 30)) return fail(SOPHIE_EINVAL, "step count too large");
  const int ns = (int)p->src.size();
  sophie_grid* g = p->g;
  if (ns == 0) {
    g->big_n = 0;
    return SOPHIE_OK;
  }
  if (p->d_pos && need <= p->cap && !p->src_dirty) return SOPHIE_OK;
  int cap = std::max(p->cap, 1024);
  while (cap < need) cap *= 2;
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  free_src(p);
  std::vector<float> val((size_t)ns * cap);
  for (int q = 0; q < ns; ++q) {
    const PackSrc& s = p->src[q];
    for (int m = 0; m < cap; ++m)
      val[(size_t)q * cap + m] = (float)source_waveform(s.kind, s.amp, s.f0, s.bw, s.t0, p->dt, m);
  }
  std::vector<int> ord(ns);
  for (int q = 0; q < ns; ++q) ord[q] = q;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return p->src[a].pos < p->src[b].pos; });
  std::vector<long long> pos(ns);
  std::vector<int> comp(ns), row(ns);
  for (int q = 0; q < ns; ++q) {
    pos[q] = p->src[ord[q]].pos;
    comp[q] = p->src[ord[q]].comp;
    row[q] = ord[q];
  }
  if (dev_malloc((void**)&p->d_pos, ns * sizeof(long long)) != cudaSuccess ||
      dev_malloc((void**)&p->d_comp, ns * sizeof(int)) != cudaSuccess ||
      dev_malloc((void**)&p->d_row, ns * sizeof(int)) != cudaSuccess ||
      dev_malloc((void**)&p->d_val, val.size() * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    free_src(p);
    g->big_n = 0;
    return fail(SOPHIE_ENOMEM, "source table allocation failed");
  }
  CUDA_TRY(cudaMemcpy(p->d_pos, pos.data(), ns * sizeof(long long), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(p->d_comp, comp.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(p->d_row, row.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(p->d_val, val.data(), val.size() * sizeof(float), cudaMemcpyHostToDevice));
  p->cap = cap;
  g->big_n = ns;
  g->big_cap = cap;
  g->big_pos = p->d_pos;
  g->big_comp = p->d_comp;
  g->big_row = p->d_row;
  g->big_val = p->d_val;
  p->src_dirty = false;
  g->gen++;
  drop_graph(p);
  return SOPHIE_OK;
}

int packed_add_source(PackedBatch* p, int cav, int comp, int i, int j, int k, double amp, double f0, double bw,
                      double t0, int kind) {
  const CavBox& b = p->box[cav];
  const Dims& D = p->g->d;
  PackSrc s{cav, comp, kind, amp, f0, bw, t0,
            ((long long)(b.oz + k) * D.ny1 + (b.oy + j)) * D.nxp + (b.ox + i), (int)p->src.size()};
  // the device tables are rebuilt once before the next step (many sources
  // are typically added in a row)
  p->src.push_back(s);
  p->src_dirty = true;
  drop_graph(p);
  if (launch_or_flag(p->g->mat, s.pos, kSrcFlag, p->stream) != cudaSuccess)
    return fail(SOPHIE_ECUDA, "flag launch failed");
  p->launches++;
  return SOPHIE_OK;
}

int packed_step(PackedBatch* p, int n) {
  sophie_grid* g = p->g;
  int rc = packed_sources(p, g->n + n);
  if (rc) return rc;
  rc = grid::ensure_capacity(g, g->n + n);  // allocations stay outside any capture
  if (rc) return rc;
  if (!g->tuned) {
    int K = 0;
    double ms = 0;
    rc = sophie_autotune(g, &K, &ms);
    if (rc) return rc;
    drop_graph(p);
  }
  const long long l0 = g->launches;
  if (!p->use_graph) return sophie_step(g, n);
  if (!(p->gexec && p->g_n0 == g->n && p->g_len == n && p->g_cur == g->cur)) {
    drop_graph(p);
    const long long n0 = g->n;
    const int cur0 = g->cur;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    rc = sophie_step(g, n);
    const cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    // the capture only recorded the launches: the state is back at n0
    g->n = n0;
    g->cur = cur0;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&p->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      p->gexec = nullptr;
      return fail(SOPHIE_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    p->g_n0 = n0;
    p->g_len = n;
    p->g_cur = cur0;
    p->g_launch = g->launches - l0;
    // launches alternate the buffers: an odd number of them ends on the other one
    p->g_flip = (int)((g->launches - l0) & 1);
    g->launches = l0;
  }
  CUDA_TRY(cudaGraphLaunch(p->gexec, p->stream));
  g->n += n;
  if (p->g_flip) g->cur = 1 - g->cur;
  g->launches += p->g_launch;
  return SOPHIE_OK;
}

int packed_energy(PackedBatch* p, double* W) {
  sophie_grid* g = p->g;
  const StepArgs a = grid::make_step_args(g);
  const double dx = p->dx;
  if (p->nitems > 0)
    packed_energy_partial_kernel<<<p->nitems, kPackEThreads, 0, p->stream>>>(a, p->d_box, p->d_items, g->eps_tab,
                                                                             p->d_part);
  packed_energy_final_kernel<<<(p->ncav + 127) / 128, 128, 0, p->stream>>>(
      p->d_first, p->ncav, p->d_part, 0.5 * grid::kEps0 * dx * dx * dx, p->d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "packed energy launch failed: %s", cudaGetErrorString(e));
  p->launches += 2;
  CUDA_TRY(cudaMemcpyAsync(W, p->d_out, (size_t)p->ncav * 8, cudaMemcpyDeviceToHost, p->stream));
  const int rc = grid::check_err_word(g);
  if (rc) return rc;
  for (int c = 0; c < p->ncav; ++c)
    if (!std::isfinite(W[c])) return fail(SOPHIE_ENONFINITE, "energy of cavity %d is not finite", c);
  return SOPHIE_OK;
}

int packed_set_fields(PackedBatch* p, int cav, int comp, const float* host) {
  const CavBox& b = p->box[cav];
  std::vector<float> v(host, host + (size_t)(b.nx + 1) * (b.ny + 1) * (b.nz + 1));
  size_t q = 0;
  for (int k = 0; k <= b.nz; ++k)
    for (int j = 0; j <= b.ny; ++j)
      for (int i = 0; i <= b.nx; ++i, ++q)
        if (!keep_entry(b, comp, i, j, k)) v[q] = 0.f;
  for (int buf = 0; buf < 2; ++buf) {
    const int rc = copy_box(p, cav, comp, v.data(), true, buf);
    if (rc) return rc;
  }
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  p->g->gen++;
  p->g->box_all = true;
  return SOPHIE_OK;
}

int packed_get_fields(PackedBatch* p, int cav, int comp, float* host) {
  const int rc = copy_box(p, cav, comp, host, false, p->g->cur);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  return SOPHIE_OK;
}

int packed_reset(PackedBatch* p) { return sophie_reset(p->g); }

int packed_set_stream(PackedBatch* p, void* stream) {
  const int rc = sophie_set_stream(p->g, stream);
  if (rc) return rc;
  p->stream = p->g->stream;
  drop_graph(p);
  return SOPHIE_OK;
}

void packed_set_graph(PackedBatch* p, bool use_graph) {
  if (p->use_graph != use_graph) drop_graph(p);
  p->use_graph = use_graph;
}

// Tune the packed grid (k, tilings); *K gets k, *ms the milliseconds per step.
int packed_autotune(PackedBatch* p, int* K, double* ms) {
  int rc = packed_sources(p, p->g->n + 1);
  if (rc) return rc;
  rc = sophie_autotune(p->g, K, ms);
  drop_graph(p);
  return rc;
}

// Cells of the cavities and of the packed grid, the step kernel's output tile
// and the steps per launch.
void packed_info(PackedBatch* p, long long* cells, long long* grid_cells, int* tile_x, int* tile_y, int* K) {
  const sophie_grid* g = p->g;
  *cells = p->cells;
  *grid_cells = (long long)p->NX * p->NY * p->NZ;
  const int k = g->temporal_k ? g->temporal_k : g->tuned_k;
  *K = k;
  if (k >= 2) {
    *tile_x = 64 - 2 * k;
    *tile_y = 32 - 2 * k;
  } else {
    *tile_x = plain_tile_x();
    *tile_y = plain_tile_y();
  }
}

int packed_origin(PackedBatch* p, int cav, int* xyz) {
  xyz[0] = p->box[cav].ox;
  xyz[1] = p->box[cav].oy;
  xyz[2] = p->box[cav].oz;
  return SOPHIE_OK;
}

int packed_sync(PackedBatch* p) { return sophie_sync(p->g); }
void packed_extent(PackedBatch* p, int* ext) {
  ext[0] = p->NX;
  ext[1] = p->NY;
  ext[2] = p->NZ;
}
int packed_check_guards(PackedBatch* p, long long* bad) { return sophie_check_guards(p->g, bad); }
long long packed_step_count(PackedBatch* p) { return p->g->n; }
long long packed_launches(PackedBatch* p) { return p->launches + p->g->launches; }

int packed_plan(int ncav, const int* dims, int* origins, int* extent) {
  std::vector<CavBox> box;
  pack_plan(ncav, dims, box, extent[0], extent[1], extent[2]);
  for (int c = 0; c < ncav; ++c) {
    origins[3 * c] = box[c].ox;
    origins[3 * c + 1] = box[c].oy;
    origins[3 * c + 2] = box[c].oz;
  }
  return SOPHIE_OK;
}

}  // namespace sophie
