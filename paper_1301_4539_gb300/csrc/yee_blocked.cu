// Host side of the temporally blocked step kernel (yee_blocked.cuh): work
// splits of the tiles and z ranges, and the launch dispatch by storage format
// to the per-format translation units.
#include <algorithm>

#include "sophie_internal.h"
#include "yee_store.cuh"

namespace sophie {

// Per-format launchers (yee_blocked_f*.cu).
cudaError_t launch_blocked_f32(const StepArgs&, const CUtensorMap&, const CUtensorMap&, const BlockedTiling&,
                               cudaStream_t);
cudaError_t launch_blocked_f16(const StepArgs&, const CUtensorMap&, const CUtensorMap&, const BlockedTiling&,
                               cudaStream_t);
cudaError_t launch_blocked_bf16(const StepArgs&, const CUtensorMap&, const CUtensorMap&, const BlockedTiling&,
                                cudaStream_t);
cudaError_t launch_blocked_f16hl(const StepArgs&, const CUtensorMap&, const CUtensorMap&, const BlockedTiling&,
                                 cudaStream_t);
cudaError_t launch_blocked_f24(const StepArgs&, const CUtensorMap&, const CUtensorMap&, const BlockedTiling&,
                               cudaStream_t);

namespace {
constexpr int kRX = 64;
constexpr int kRY = 32;
}  // namespace

// TMA box width: the 64-column region plus the 16-byte x granule.
int blocked_box_x(int fmt) { return kRX + (store_bytes(fmt) == 4 ? Store<kF32>::kAlign : Store<kF16>::kAlign); }
int blocked_box_y() { return kRY; }

// Work split of `tiles` tiles of nz planes over at most num_sms CTAs (one per
// SM). Aligned: the number of z ranges minimising the planes the busiest CTA
// streams, rounds x (range + the 4K-3 planes of level fill and drain).
static void choose_split(long long tiles, int nz, int K, int num_sms, int aligned, BlockedTiling& t) {
  if (!aligned) {
    const long long items = tiles * nz;
    t.zsplit = 0;
    t.grid = (int)(items < num_sms ? items : num_sms);
    return;
  }
  double best = 1e300;
  const int smax = std::max(1, std::min(nz / 8, 1024));
  for (int s = 1; s <= smax; ++s) {
    const long long units = tiles * s;
    const long long grid = units < num_sms ? units : num_sms;
    const long long rounds = (units + grid - 1) / grid;
    const double cost = (double)rounds * ((nz + s - 1) / s + (s > 1 ? 4 * K - 3 : K - 1));
    if (cost < best - 1e-9) {
      best = cost;
      t.zsplit = s;
      t.grid = (int)grid;
    }
  }
  // one round of units: tile-major (measured faster at 256^3); several:
  // range-major (measured faster at 512^3 to 768^3); aligned = 2 / 3 force
  // tile-major / range-major
  t.order = aligned >= 2 ? aligned - 2 : tiles * t.zsplit > t.grid ? 1 : 0;
}

BlockedTiling blocked_tiling(const Dims& d, int K, int num_sms, int aligned) {
  BlockedTiling t{};
  const int TX = kRX - 2 * K, TY = kRY - 2 * K, phi = K & 1;
  t.K = K;
  t.tiles_x = (d.nx + phi + TX - 1) / TX;
  t.tiles_y = (d.ny + TY - 1) / TY;
  t.tx0 = t.ty0 = t.zlo = 0;
  t.zhi = d.nz;
  choose_split((long long)t.tiles_x * t.tiles_y, d.nz, K, num_sms, aligned, t);
  return t;
}

BlockedTiling blocked_tiling_split(const Dims& d, int K, int num_sms, int zsplit, int order) {
  BlockedTiling t = blocked_tiling(d, K, num_sms, 1);
  const long long tiles = (long long)t.tiles_x * t.tiles_y;
  t.zsplit = std::max(1, std::min(zsplit, d.nz));
  t.order = order ? 1 : 0;
  const long long units = tiles * t.zsplit;
  t.grid = (int)(units < num_sms ? units : num_sms);
  return t;
}

BlockedTiling blocked_tiling_box(const Dims& d, int K, int num_sms, const int* box) {
  BlockedTiling t{};
  t.K = K;
  const int TX = kRX - 2 * K, TY = kRY - 2 * K, phi = K & 1;
  const int z0 = std::max(box[4], 0), z1 = std::min(box[5], d.nz);
  const int x1 = std::min(box[1], d.nx), y1 = std::min(box[3], d.ny);
  if (box[0] >= x1 || box[2] >= y1 || z0 >= z1) return t;  // nothing live: grid 0
  // tile tx covers output x [tx TX - phi, tx TX - phi + TX)
  const int tx0 = (box[0] + phi) / TX, tx1 = (x1 - 1 + phi) / TX + 1;
  const int ty0 = box[2] / TY, ty1 = (y1 - 1) / TY + 1;
  t.tiles_x = tx1 - tx0;
  t.tiles_y = ty1 - ty0;
  choose_split((long long)t.tiles_x * t.tiles_y, z1 - z0, K, num_sms, 1, t);
  t.tx0 = tx0;
  t.ty0 = ty0;
  t.zlo = z0;
  t.zhi = z1;
  return t;
}

bool blocked_supported(int K, int fmt) { return (K >= 2 && K <= 4) || ((K == 6 || K == 8) && fmt == kF32); }

cudaError_t launch_step_blocked(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                                const BlockedTiling& t, cudaStream_t s) {
  switch (a.fmt) {
    case kF32: return launch_blocked_f32(a, tmF, tmM, t, s);
    case kF16: return launch_blocked_f16(a, tmF, tmM, t, s);
    case kBF16: return launch_blocked_bf16(a, tmF, tmM, t, s);
    case kF16HL: return launch_blocked_f16hl(a, tmF, tmM, t, s);
    case kF24: return launch_blocked_f24(a, tmF, tmM, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sophie
