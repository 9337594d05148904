// Internal declarations shared by the host runtime (sophie_api.cu) and the
// CUDA kernels of libsophie. Not installed; the public ABI is include/sophie.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>

#include <utility>
#include <vector>

namespace sophie {

// Device field layout of one buffer: for z in [0,nz], comp f in [0,6),
// y in [0,ny], x in [0,nxp): addr = ((z*6 + f)*ny1 + y)*nxp + x.
// nxp = round_up(nx+1, 8) keeps every row 32-byte aligned (one DRAM sector)
// and satisfies the 16-byte stride rule of TMA tensor maps. The padding
// columns are zero and never written.
//
// Material word, one per index point (z*ny1 + y)*nxp + x:
//   bit  0      a source sits on one of this point's edges
//   bit  1      a probe sits on one of this point's components
//   bit  2      explicit point: bits 3..31 index the explicit tables
//               (3 x (Ca, Cb) and 3 x eps_r(edge) for ex, ey, ez); else:
//   bits  3..11 class of the ex edge at this index (0 = PEC / absent)
//   bits 12..20 class of the ey edge
//   bits 21..29 class of the ez edge
// Each class index sits 3 bits above a field boundary, so (word >> s) & 0xFF8
// is directly the byte offset of the class's 8-byte (Ca, Cb) entry.
// Class c has coefficients coef[c] = (Ca, Cb) (float) and eps_r(edge) in
// double (energy). Class 0 is (0, 0): the edge is never anything but 0.
constexpr int kMaxClasses = 512;
constexpr int kMaxSources = 16;
constexpr int kMaxProbes = 64;
constexpr uint32_t kSrcFlag = 1u;
constexpr uint32_t kPrbFlag = 2u;
constexpr uint32_t kExpFlag = 4u;
constexpr int kClsShift[3] = {3, 12, 21};
constexpr uint32_t kClsOffMask = 0xFF8u;  // 9-bit class index times 8

__host__ __device__ constexpr uint32_t cls_word(uint32_t cx, uint32_t cy, uint32_t cz) {
  return (cx << 3) | (cy << 12) | (cz << 21);
}
// Class index of edge component c (0..2) of a material word.
__host__ __device__ __forceinline__ uint32_t cls_of(uint32_t m, int c) {
  return (m >> (c == 0 ? 3 : c == 1 ? 12 : 21)) & 511u;
}
// Byte offset of that class's (Ca, Cb) pair in a float2 table.
__device__ __forceinline__ uint32_t cls_off_x(uint32_t m) { return m & kClsOffMask; }
__device__ __forceinline__ uint32_t cls_off_y(uint32_t m) { return (m >> 9) & kClsOffMask; }
__device__ __forceinline__ uint32_t cls_off_z(uint32_t m) { return (m >> 18) & kClsOffMask; }

struct Dims {
  int nx, ny, nz;   // cells
  int nxp, ny1, nz1;  // storage extents (nxp padded)
  long long plane;  // ny1*nxp: elements of one component plane
  long long zstride;  // elements of one z slab: 6*plane (9*plane for the 24-bit storage format)
};

// Source and probe tables passed by value to the step kernels.
struct SrcTable {
  int n;
  int comp[kMaxSources];
  long long pos[kMaxSources];  // index-point offset (z*ny1 + y)*nxp + x
  const float* val;            // [kMaxSources][cap]; val[s*cap + step]
  int cap;
  // Many sources (a packed batch of cavities): when nbig > 0 the arrays above
  // are unused and source q (0 <= q < nbig) is at point bpos[q], component
  // bcomp[q], waveform row brow[q] of val; bpos is sorted ascending, sources
  // on one point in the order they were added.
  int nbig;
  const long long* bpos;
  const int* bcomp;
  const int* brow;
  // Unit-scale storage forms (yee_store.cuh kF16U...): the kernels compute on
  // scaled fields, so the currents are multiplied by vmul when vmul_on.
  int vmul_on;
  float vmul;
};

struct PrbTable {
  int n;
  int comp[kMaxProbes];
  long long pos[kMaxProbes];
  float* buf;  // [kMaxProbes][cap]; buf[p*cap + step]
  int cap;
  // Unit-scale storage forms: samples of scaled fields, multiplied by pmul
  // (the inverse scale) when pmul_on.
  int pmul_on;
  float pmul;
};

struct StepArgs {
  const void* fin;  // field buffers in the storage format `fmt`
  void* fout;
  int fmt;          // StoreFmt (yee_store.cuh): 0 float, 1 half, 2 bfloat16
  int fold;         // 2-byte and hi+lo forms with six equal scales: the step
                    // kernels run the unit-scale form of fmt (kF16U, ...)
  float sc[6];      // stored value = field * sc[comp] (2-byte formats)
  float isc[6];     // 1 / sc
  const uint32_t* mat;
  const float2* coef;   // class table (Ca, Cb)
  const float2* ecoef;  // explicit points: 3 x (Ca, Cb) per entry
  const double* eeps;   // explicit points: 3 x eps_r per entry (energy)
  Dims d;
  float S;
  long long n0;  // absolute index of the first step this launch performs
  SrcTable src;
  PrbTable prb;
  int* err;      // device error word (bounded waits that ran out)
  // Output box of this launch, index points [box[0], box[1]) x [box[2], box[3])
  // x [box[4], box[5]): work units whose outputs lie outside it are skipped
  // (the fields there are known to be zero and stay zero; see sophie.h,
  // sophie_set_zero_skip). The full grid when skipping is off.
  int box[6];
  // Non-uniform mesh (sophie_set_spacing): device arrays of the float ratios
  // reference step / cell width, rat[0..2] = rx[nx], ry[ny], rz[nz] (primary
  // widths) and rat[3..5] = rxd[nx+1], ryd[ny+1], rzd[nz+1] (dual widths, the
  // mean of the two cells beside a node; the end cell's at a wall node). All
  // null on a uniform mesh.
  const float* rat[6];
  // The same ratios as (primary, dual) pairs per index, one array per axis,
  // zero-padded so that rpair[a][i] is readable for i in [-kRatioPad,
  // n_a + kRatioTail) and 16-byte aligned at even i (two pairs per 16-byte
  // load); entries outside an array's range are 0.
  const float2* rpair[3];
};

// Launch a step kernel with programmatic dependent launch allowed, so that its
// CTAs can start as the previous kernel's retire (the kernels wait with
// griddepcontrol.wait before touching global memory). Launches recorded into
// a CUDA graph (batches) keep plain edges, which replayed ~1 % faster there;
// SOPHIE_PDL=0 launches every step kernel plainly.
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("SOPHIE_PDL");
    return !(v && atoi(v) == 0);
  }();
  return on;
}
template <typename... P, typename... A>
cudaError_t launch_step_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaGetLastError();
  cfg.numAttrs = pdl_enabled() && cs == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

constexpr int kRatioPad = 8;    // pairs before index 0
constexpr int kRatioTail = 72;  // pairs from index n on (a 64-wide tile plus halo beyond the last cell)

// Ratio of a non-uniform mesh at index i, 0 outside [0, n) (such points only
// feed values that are discarded or multiplied by a zero coefficient).
__device__ __forceinline__ float ratio_at(const float* r, int i, int n) {
  return (unsigned)i < (unsigned)n ? r[i] : 0.f;
}

// Whether the output block [x0, x1) x [y0, y1) x [z0, z1) meets the launch box.
__host__ __device__ __forceinline__ bool box_meets(const int* b, int x0, int x1, int y0, int y1, int z0, int z1) {
  return x0 < b[1] && x1 > b[0] && y0 < b[3] && y1 > b[2] && z0 < b[5] && z1 > b[4];
}

// Work decomposition of the TMA step kernels: (x tile, y tile, z chunk) units
// walked by `grid` persistent CTAs.
struct PlainTiling {
  int tiles_x, tiles_y, zchunk, grid;
  long long units;
  int tx0, ty0, z0, z1;  // the tiles start at tile (tx0, ty0); output planes [z0, z1)
};

// Temporally blocked kernel: K steps per launch over (tiles_x x tiles_y)
// regions, walked by `grid` CTAs.
struct BlockedTiling {
  int K, tiles_x, tiles_y, grid;
  // > 0: every tile's planes are cut into the same zsplit z ranges and CTA b
  // takes units b, b + grid, ... in the order `order`: 0 tile-major (unit u is
  // range u % zsplit of tile u / zsplit: the CTAs working at the same time hold
  // all ranges of a run of neighbouring tiles), 1 range-major (range u / tiles
  // of tile u % tiles: they hold one range of many neighbouring tiles).
  // 0: the (tile, plane) items are cut into grid equal contiguous ranges.
  int zsplit;
  int order;
  int tx0, ty0, zlo, zhi;  // the tiles start at tile (tx0, ty0); output planes [zlo, zhi)
  // Rows of the 64 x 32 region per thread: 4 (8 warps; also 0) or 2 (16 warps).
  int rows;
};

// Coefficient tables behind the material words (host copies). Class c:
// coef[c] = (Ca, Cb), eps[c], sig[c] = the edge's mean material; class 0 is
// PEC / absent. Explicit entry q: three consecutive (Ca, Cb) / eps / sigma
// for the ex, ey, ez edges of the points that carry it.
struct MaterialTables {
  std::vector<float2> coef;
  std::vector<double> eps, sig;
  std::vector<float2> ecoef;
  std::vector<double> eeps, esig;
};

// (Ca, Cb) of an edge with mean material (e, s): beta = s dt / (2 eps0 e),
// Ca = (1-beta)/(1+beta), Cb = (S/e)/(1+beta), computed in double and
// rounded once to float (materials.cu).
float2 edge_coefficients(double dt, double S64, double e, double s);
// Words (row pitch d.nxp, (nz+1)(ny+1) rows) and tables for per-cell eps_r and
// sigma (x fastest; nullptr = vacuum; eps_r = +inf marks a perfectly
// conducting cell, whose edges are PEC). Edge material = mean of its four
// cells; the 511 most frequent edge materials become classes, points with an
// edge outside them share explicit entries by their three edge materials.
// No source or probe flags are set. The work is split into slabs of z planes
// fixed by the grid (at most 64, at least 16 planes each; explicit entries
// are shared within a slab) run on up to nthreads host threads; the result
// does not depend on nthreads. Returns 0, or -1 if
// more than 2^29 explicit entries would be needed.
int build_material_tables(const Dims& d, double dt, double S64, const float* eps, const float* sig, uint32_t* words,
                          MaterialTables* out, int nthreads);
// Index of the first of n cells with eps_r < 1 (or NaN) or sigma negative or
// not finite (a null array is not checked), or -1; checked on nthreads host
// threads.
long long first_bad_material(const float* eps, const float* sig, long long n, int nthreads);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_step_simple(const StepArgs& a, cudaStream_t s);
bool encode_maps(const Dims& d, int fmt, void* fields, uint32_t* mat, int box_x, int box_y, CUtensorMap* tmF,
                 CUtensorMap* tmM);
int plain_box_x(int fmt);
int plain_box_y();
PlainTiling plain_tiling(const Dims& d, int num_sms, int zchunk_override);
// Tilings of the sub-box of output points [box[0], box[1]) x ... x [box[4],
// box[5]) only (zero-field skipping): the tiles meeting it, and its planes.
// grid == 0 means there is nothing to compute.
PlainTiling plain_tiling_box(const Dims& d, int num_sms, const int* box);
BlockedTiling blocked_tiling_box(const Dims& d, int K, int num_sms, const int* box);
cudaError_t launch_step_plain(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                              const PlainTiling& t, cudaStream_t s);
// aligned: 0 contiguous split; 1 the modelled aligned split in its default
// unit order; 2 / 3 the same split tile-major / range-major.
BlockedTiling blocked_tiling(const Dims& d, int K, int num_sms, int aligned);
// The aligned split with exactly zsplit z ranges (clamped to [1, nz]) taken
// in unit order `order` (BlockedTiling::order).
BlockedTiling blocked_tiling_split(const Dims& d, int K, int num_sms, int zsplit, int order);
// K = 2..4 for every storage format; K = 6 and 8 (two-stage ring) for float
// storage only.
bool blocked_supported(int K, int fmt);
int blocked_box_x(int fmt);
int blocked_box_y();
cudaError_t launch_step_blocked(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                                const BlockedTiling& t, cudaStream_t s);
cudaError_t launch_energy(const StepArgs& a, const double* eps_tab, double* partials, int nblocks,
                          double* out, cudaStream_t s);
// Reduction blocks of the energy kernels: one per 8 x 256 index points, at
// most kEnergyMaxBlocks (a grid-stride loop covers larger grids), so every
// grid needs at most kEnergyMaxBlocks partial sums.
constexpr int kEnergyMaxBlocks = 152 * 16;
int energy_blocks(const Dims& d);
// Same reduction, final sum multiplied by `scale` and written to `out`.
cudaError_t launch_energy_scaled(const StepArgs& a, const double* eps_tab, double* partials, int nblocks,
                                 double scale, double* out, cudaStream_t s);
// Energy with partial sums in a fixed static device buffer (energy_noalloc.cu).
int energy_noalloc(const StepArgs& a, const double* eps_tab, double scale, double* W_dev, cudaStream_t s,
                   const char** why);
// fmt: the buffer's storage format (yee_store.cuh); kF24 also clears the
// component's byte of its byte-pair plane.
cudaError_t launch_mask_component(void* f, int esz, const Dims& d, int comp, cudaStream_t s, int fmt = 0);
cudaError_t launch_or_flag(uint32_t* mat, long long pos, uint32_t bit, cudaStream_t s);

// Batched cavities (yee_batch.cu, sophie_batch.cu). One descriptor per
// cavity in device memory; float field storage.
constexpr int kBatchMaxSrc = 4;
struct CavityDesc {
  CUtensorMap tmF[2];      // TMA maps of the two field buffers (plain kernel box)
  CUtensorMap tmM;         // TMA map of the material words
  Dims d;
  void* F[2];              // the cavity's two field buffers (ping-pong)
  const uint32_t* mat;     // material words (layout of a single grid)
  const float2* coef;      // class table (kMaxClasses entries)
  const double* eps_tab;   // class eps_r(edge) (energy)
  const float2* ecoef;     // explicit entries
  const double* eeps;
  SrcTable src;            // at most kBatchMaxSrc sources; val[q*cap + step]
};
// A step work item: x tile [x0, x0+32), y tile [y0, y0+TY), planes [z0, z1).
struct BatchItem {
  int cav, x0, y0, z0, z1;
};
// An energy work item: index points [p0, p1) of one cavity.
struct EnergyItem {
  int cav;
  long long p0, p1;
};
// The TMA-staged plain kernel over a batch work list (64 x 16 tiles; items
// with x0 % 64 == 0, y0 % 16 == 0). a supplies S, n0 and err; float storage.
struct PlainBatch {
  const CavityDesc* descs;
  const BatchItem* items;
  int nitems;
  int cur;
};
cudaError_t launch_step_plain_batch(const StepArgs& a, const PlainBatch& pb, int grid, cudaStream_t s);
int plain_tile_x();
int plain_tile_y();
bool batch_tile_supported(int ty);
int batch_blocks_per_sm(int ty);
// Memsets the work counter, then one persistent launch of `grid` CTAs.
cudaError_t launch_batch_step(const CavityDesc* descs, const BatchItem* items, int nitems, int* counter, int cur,
                              float S, long long nstep, int ty, int grid, cudaStream_t s);
// out[c] = scale * energy sum of cavity c; first[c]..first[c+1] are its items.
cudaError_t launch_batch_energy(const CavityDesc* descs, const EnergyItem* items, int nitems, const int* first,
                                int ncav, int cur, float S, double* partials, double scale, double* out,
                                cudaStream_t s);
// Packed layout of a batch (batch_packed.cu): the cavities in one grid with
// conducting layers between them, run by the single-grid step kernels.
struct PackedBatch;
int packed_plan(int ncav, const int* dims, int* origins, int* extent);
int packed_create(int ncav, const int* dims, double dx, double dt, PackedBatch** out);
void packed_destroy(PackedBatch* p);
int packed_set_materials(PackedBatch* p, const float* eps, const float* sig);
int packed_add_source(PackedBatch* p, int cav, int comp, int i, int j, int k, double amp, double f0, double bw,
                      double t0, int kind);
int packed_step(PackedBatch* p, int n);
int packed_energy(PackedBatch* p, double* W);
int packed_set_fields(PackedBatch* p, int cav, int comp, const float* host);
int packed_get_fields(PackedBatch* p, int cav, int comp, float* host);
int packed_reset(PackedBatch* p);
int packed_set_stream(PackedBatch* p, void* stream);
void packed_set_graph(PackedBatch* p, bool use_graph);
int packed_autotune(PackedBatch* p, int* K, double* ms);
void packed_info(PackedBatch* p, long long* cells, long long* grid_cells, int* tile_x, int* tile_y, int* K);
int packed_origin(PackedBatch* p, int cav, int* xyz);
long long packed_launches(PackedBatch* p);
int packed_sync(PackedBatch* p);
void packed_extent(PackedBatch* p, int* ext);
int packed_check_guards(PackedBatch* p, long long* bad);
long long packed_step_count(PackedBatch* p);
// Set the thread's last-error message (sophie_last_error) and return code.
int report_error(int code, const char* msg);

// cudaMalloc, except that a debug hook (sophie_debug_fail_alloc) can make the
// n-th following call fail as if the device were out of memory.
cudaError_t dev_malloc(void** p, size_t bytes);
// Registry of live handles (grids and batches), so that destroying a handle
// twice is reported instead of freeing freed memory.
void handle_register(const void* h);
bool handle_release(const void* h);
// Field buffers sit between two guard regions of kGuardByte (guard bytes
// each side); launch_guard_check counts the changed bytes of a region.
constexpr unsigned char kGuardByte = 0xA5;
cudaError_t launch_guard_check(const void* p, size_t n, unsigned char pattern, unsigned long long* bad,
                               cudaStream_t s);
// Bounded-wait self-test kernel (selftest.cu): sets code 32 in *err.
cudaError_t launch_wait_timeout(int* err, unsigned long long* waited_ns, cudaStream_t s);
// amp * w((n + 1/2) dt) of a soft source (kind 0: Gaussian-modulated sine,
// kind 1: Gaussian pulse; bw = FWHM of the envelope's amplitude spectrum).
double source_waveform(int kind, double amp, double f0, double bw, double t0, double dt, long long n);

// Reverse-mode sweep (yee_adjoint.cu). Adjoint fields use the float field
// layout; a.fin holds the adjoint of the state after a step, a.fout receives
// the adjoint of the state before it.
cudaError_t launch_adj_step(const StepArgs& a, cudaStream_t s);
// After the forward step a.fin -> a.fout (float storage, a.n0 = its index):
// e_out[t] = e^n and c_out[t] = B h^{n+1/2} + s on design edge t.
cudaError_t launch_gather(const StepArgs& a, const int* edge_comp, const long long* edge_pt, int nedge, float* e_out,
                          float* c_out, cudaStream_t s);
// gcb[t] += l_e(edge t) * c_in[t], gca[t] += l_e(edge t) * e_in[t] (double).
cudaError_t launch_grad_accum(const float* l, const Dims& d, const int* edge_comp, const long long* edge_pt, int nedge,
                              const float* e_in, const float* c_in, double* gcb, double* gca, cudaStream_t s);
// The two above in one launch: l(comp at pt) += two_dt * sample[0], then the
// accumulation; t_obj = the design edge on (comp, pt), or -1.
cudaError_t launch_objective_grad_accum(float* l, const Dims& d, int comp, long long pt, const float* sample,
                                        double two_dt, int t_obj, const int* edge_comp, const long long* edge_pt,
                                        int nedge, const float* e_in, const float* c_in, double* gcb, double* gca,
                                        cudaStream_t s);
// l(comp at point pt) += two_dt * sample[0].
cudaError_t launch_add_objective(float* l, const Dims& d, int comp, long long pt, const float* sample, double two_dt,
                                 cudaStream_t s);

}  // namespace sophie
