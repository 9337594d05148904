// Host-side state of a grid (struct sophie_grid behind include/sophie.h's
// opaque handle) and the host helpers shared by the files of the runtime
// (sophie_api.cu: grid, materials, stepping; sophie_objective.cu: objective
// record and gradient). Not installed.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sophie.h"
#include "sophie_internal.h"
#include "yee_store.cuh"

namespace sophie {
namespace grid {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;

// Set the thread's error message (printf format) and return `code`.
int fail(int code, const char* fmt, ...);

}  // namespace grid
}  // namespace sophie

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::sophie::grid::fail(SOPHIE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

namespace sophie {
namespace grid {

struct Source {
  int comp, i, j, k, kind;
  double amp, f0, bw, t0;
  long long pos;
};

struct Probe {
  int comp, i, j, k;
  long long pos;
  // Index on a plane no kernel updates (i == nx, j == ny or k == nz): a PEC
  // edge or a wall-normal face whose value never changes. Its samples are
  // filled from the field at read time instead of by the step kernels.
  bool fixed;
  long long n_added;
};

struct ProfEntry {
  int kernel;
  cudaEvent_t a, b;
};

// Recorded forward pass of a probe objective (sophie_objective_forward) and
// the workspace of its reverse sweep (sophie_objective_grad_eps).
struct Tape {
  bool valid = false;
  long long gen = -1;  // grid generation the record belongs to
  long long n0 = 0;    // first step of the recorded pass
  int N = 0, K = 50;   // steps, checkpoint interval
  int comp = 2;        // objective component and index point
  long long pt = 0;
  std::vector<void*> ck;     // states at n0 + s*K, s = 0 .. ceil(N/K)-1
  float* samples = nullptr;  // objective samples f^{n0+1} .. f^{n0+N}
  int samples_cap = 0;
  void* R[2] = {nullptr, nullptr};  // segment recompute (float fields)
  CUtensorMap tmR[2];
  CUtensorMap tmRM;
  void* L[2] = {nullptr, nullptr};  // adjoint fields
  CUtensorMap tmL[2];
  int* ecomp = nullptr;             // design edges: component, index point
  long long* ept = nullptr;
  float* etr = nullptr;  // [K][nedge] e^n on the design edges
  float* ctr = nullptr;  // [K][nedge] B h^{n+1/2} + s on the design edges
  double* gcb = nullptr;  // dJ/dCb, dJ/dCa per design edge
  double* gca = nullptr;
  int edge_cap = 0, tr_cap = 0;
  // Traced record (a design box registered before the forward pass): e^n and
  // the bracket on the box's design edges for every step, [N][nedge] each,
  // gathered during the forward pass, so the reverse sweep needs no recompute.
  bool traced = false;
  int tbox[6] = {0, 0, 0, 0, 0, 0};
  int tnedge = 0;
  float* etr_all = nullptr;
  float* ctr_all = nullptr;
};

}  // namespace grid
}  // namespace sophie

struct sophie_grid {
  sophie::Dims d{};
  CUtensorMap tmF[2];  // TMA maps of the two field buffers
  CUtensorMap tmM;     // TMA map of the material words
  sophie::PlainTiling ptile{};
  CUtensorMap tmFB[2];  // TMA maps with the temporally blocked kernel's box
  CUtensorMap tmMB;
  sophie::BlockedTiling btile{};
  int num_sms = 0;
  bool use_simple = false;  // tile_x == 32: untiled-load reference kernel
  double dx = 0, dt = 0, S64 = 0;
  float S32 = 0;
  void* F[2] = {nullptr, nullptr};  // field buffers in storage format `fmt`
  void* Fbase[2] = {nullptr, nullptr};  // their allocations: guard | buffer | guard
  size_t fguard = 0;                    // guard bytes on each side
  int fmt = sophie::kF32;            // StoreFmt
  int esz = 4;                      // bytes per stored value
  float sc[6] = {1, 1, 1, 1, 1, 1};  // stored = field * sc (2-byte formats)
  int cur = 0;
  uint32_t* mat = nullptr;     // device material words
  uint32_t* mat_host = nullptr;  // pinned staging for uploads
  float2* coef = nullptr;      // device class table (Ca, Cb)
  double* eps_tab = nullptr;   // device class table eps_r(edge)
  std::vector<float2> coef_h;
  std::vector<double> eps_h;
  std::vector<float2> ecoef_h;    // explicit points: (Ca, Cb) of ex, ey, ez
  std::vector<double> eeps_h;     // explicit points: eps_r of ex, ey, ez
  std::vector<double> sig_h;      // sigma(edge) of each class (host; gradients)
  std::vector<double> esig_h;     // explicit points: sigma of ex, ey, ez
  float2* ecoef = nullptr;        // device copies
  double* eeps = nullptr;
  size_t exp_cap = 0;
  cudaEvent_t mat_upload_done = nullptr;
  std::vector<sophie::grid::Source> src;
  std::vector<sophie::grid::Probe> prb;
  float* sval = nullptr;  // device [kMaxSources][scap]
  int scap = 0;
  // Many sources, installed by a packed batch of cavities (batch_packed.cu):
  // when big_n > 0 the step kernels take their sources from these device
  // arrays (SrcTable::nbig) instead of src / sval. Owned by the batch.
  int big_n = 0, big_cap = 0;
  const long long* big_pos = nullptr;
  const int* big_comp = nullptr;
  const int* big_row = nullptr;
  const float* big_val = nullptr;
  float* pbuf = nullptr;  // device [kMaxProbes][pcap]
  int pcap = 0;
  long long n = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int temporal_k = 0;  // 0: chosen by the autotuner at the first step
  bool tuned = false;  // autotuner result valid for the current format
  int tuned_k = 2;
  int precision = SOPHIE_FP32;
  double* e_partials = nullptr;
  double* e_out = nullptr;
  int e_blocks = 0;
  int* err = nullptr;
  long long launches = 0;
  bool prof = false;
  std::vector<sophie::grid::ProfEntry> prof_live;
  std::vector<cudaEvent_t> ev_pool;
  long long prof_count[4] = {0, 0, 0, 0};
  double prof_ms[4] = {0, 0, 0, 0};
  // Zero-field skipping (sophie_set_zero_skip): outside zbox (index points
  // [zbox[0], zbox[1]) x ... , empty if zbox[0] >= zbox[1]) every field is zero,
  // unless box_all (fields were written by the caller).
  bool zskip = false;
  bool box_all = false;
  int zbox[6] = {0, 0, 0, 0, 0, 0};
  // Non-uniform mesh (sophie_set_spacing): one device allocation holding the
  // six float ratio arrays rx, ry, rz, rxd, ryd, rzd back to back, then the
  // padded (primary, dual) pair arrays of x, y, z (StepArgs::rpair); null
  // when the mesh is uniform.
  float* rat = nullptr;
  long long rpair_off[3] = {0, 0, 0};  // float offset of each pair array's index 0
  long long gen = 0;       // bumped by every change of fields, materials, sources or mesh
  bool obj_rec = false;    // the step kernels also sample the objective point
  // Design box registered for the next objective record (sophie_objective_set_design).
  bool design_set = false;
  int design[6] = {0, 0, 0, 0, 0, 0};
  sophie::grid::Tape tape;
};

namespace sophie {
namespace grid {

long long point_index(const Dims& d, int i, int j, int k);
bool e_edge_interior(const Dims& d, int c, int i, int j, int k);
bool comp_valid(const Dims& d, int c, int i, int j, int k);
// Make the source table cover steps [0, need) and the probe buffer [0, need).
int ensure_capacity(sophie_grid* g, long long need);
cudaEvent_t prof_event(sophie_grid* g);
int prof_drain(sophie_grid* g);
// Arguments of a step launch on the current buffers at the current step.
StepArgs make_step_args(sophie_grid* g);
// Synchronise; ETIMEOUT (and clear the word) if a kernel gave up a wait.
int check_err_word(sophie_grid* g);
// Enqueue the upload of g->mat_host and the host coefficient tables (the
// explicit tables reallocated if they grew); records g->mat_upload_done.
int upload_materials(sophie_grid* g);
void free_tape(Tape& t);

}  // namespace grid
}  // namespace sophie
