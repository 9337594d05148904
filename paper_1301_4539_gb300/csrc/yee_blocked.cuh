// yee_blocked<K>: K fused leapfrog steps per launch (temporal blocking).
//
// The kernel templates; yee_blocked_f*.cu instantiate them per storage
// format (compiled in parallel), yee_blocked.cu holds the host side.
//
// Method: Sec. 3.4 (two-step cache reuse, generalised to K steps in the
// conclusion): a tile of the grid is advanced several time steps while it is
// on chip, so each field byte fetched from HBM serves K steps. Sec. 3.1: the
// restructuring changes no output value; here every H and E value is the
// same float expression (yee_update.cuh) as in the one-step kernels, so the
// fields are bitwise identical to K plain steps.
//
// GPU design (one CTA of 8 warps per SM):
//  * A CTA owns a 64 x 32 (x, y) region. Each step needs the neighbour at +1
//    (H from E) and at -1 (E from H), so after K steps only the inner
//    (64-2K) x (32-2K) part is exact: that part is the output tile; the
//    regions of neighbouring tiles overlap by 2K columns / rows and compute
//    the overlap identically (no inter-CTA communication, no waits).
//  * Eight warps; thread 0 also issues the TMA loads: a stage is refilled right
//    after the first level barrier of the iteration that consumed it, which
//    proves every warp has copied it to registers (no empty barriers needed).
//  * z is streamed. Level t (step t of the K) lags level t-1 by one plane:
//    at iteration s, level t updates plane s-t using level t-1's state of that
//    plane (kept in registers since the previous iteration) and level t-1's
//    E of plane s-t+1 (just computed). Level 0 is the TMA-staged input
//    (3-stage ring of 68x32 boxes of the six fields and the material words).
//  * A lane owns two adjacent x, a thread four rows (R). x neighbours come
//    from warp shuffles; y neighbours from registers inside a thread's rows
//    and, at warp seams, from two small shared-memory row buffers per level
//    (E rows double-buffered by iteration parity, H rows per level), with one
//    named barrier per level.
//  * Work: the (tile, z plane) items are split into equal contiguous ranges,
//    one per CTA; a range that starts above z = 0 first replays 3K-2 planes
//    so that every level's state is exact from its first output plane.
#pragma once

#include <algorithm>

#include "sophie_internal.h"
#include "tma_util.cuh"
#include "yee_rare.cuh"
#include "yee_store.cuh"
#include "yee_update.cuh"

namespace sophie {

namespace {

constexpr int kRX = 64;
constexpr int kRY = 32;  // region rows: R rows per thread, 32 / R warps
// Stages of the TMA ring: 3; 2 for K >= 5, whose per-level seam rows leave no
// room for a third (the load of plane s+1 then overlaps the K-1 deeper levels
// of iteration s).
__host__ __device__ constexpr int ring_stages(int K) { return K >= 5 ? 2 : 3; }

// Thread layout of a CTA with R rows per thread: W warps of 32 lanes (thread 0
// also issues the TMA loads). R = 4: 8 warps; R = 2: 16 warps with half the
// carried state per thread (more warps to hide latency, more warp seams).
template <int R>
struct Lay {
  static constexpr int W = kRY / R;
  static constexpr int kThreads = W * 32;
  static_assert(W * R == kRY, "rows per thread must divide the region");
};

// TMA box of a storage format: the region rounded out to the 16-byte x granule,
// all planes of the format (six components; nine 2-byte planes for kF24).
template <int F>
struct BoxCfg {
  using T = typename Store<F>::T;
  static constexpr int GX = Store<F>::kAlign;
  static constexpr int BX = kRX + GX;
  static constexpr int P = store_planes(F);
  static constexpr uint32_t kFieldBytes = BX * kRY * P * sizeof(T);
  static constexpr uint32_t kMatOff = (kFieldBytes + 127) / 128 * 128;  // material box, 128-byte aligned
  static constexpr uint32_t kMatBytes = BX * kRY * 4;
  static constexpr uint32_t kLoadBytes = kFieldBytes + kMatBytes;
  static constexpr uint32_t kStageBytes = (kMatOff + kMatBytes + 127) / 128 * 128;
  static constexpr long long CS = (long long)kRY * BX;  // elements between component planes
};

template <int K, int F, int R = 4>
struct Cfg {
  static constexpr int kNS = ring_stages(K);
  static constexpr int W = Lay<R>::W;
  static constexpr uint32_t kStageBytes = BoxCfg<F>::kStageBytes;
  static constexpr int TX = kRX - 2 * K;
  static constexpr int TY = kRY - 2 * K;
  static constexpr int PHI = K & 1;  // x tiles shifted so that region starts are even
  // shared memory: stages | H seam rows [K][W][2][64] | E seam rows [K-1][2][W][2][64] |
  // class table | barriers | the loader's state (thread 0 only)
  static constexpr uint32_t kHpOff = kNS * kStageBytes;
  static constexpr uint32_t kHpBytes = K * W * 2 * kRX * 4;
  static constexpr uint32_t kEpOff = kHpOff + kHpBytes;
  static constexpr uint32_t kEpBytes = (K > 1 ? K - 1 : 1) * 2 * W * 2 * kRX * 4;
  static constexpr uint32_t kCoefOff = kEpOff + kEpBytes;
  static constexpr uint32_t kBarOff = kCoefOff + kMaxClasses * 8;
  static constexpr uint32_t kLdOff = kBarOff + kNS * 8;
  static constexpr uint32_t kPrbOff = kLdOff + 64;  // the probe table (PrbShared)
  static constexpr uint32_t kSmem = kPrbOff + sizeof(PrbShared);
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

template <int F>
__device__ __forceinline__ int FI(int f, int r, int c) { return (f * kRY + r) * BoxCfg<F>::BX + c; }

template <int R>
struct St {
  float ex[R][2], ey[R][2], ez[R][2], hx[R][2], hy[R][2], hz[R][2];
  uint32_t m[R][2];
};

__device__ __forceinline__ void set_err(int* err, int code) { atomicOr(err, code); }

// The (tile, plane) items of this CTA, walked as units. With zsplit > 0
// every tile's z column is cut into the same zsplit ranges and CTA b takes
// units b, b + grid, ... in tile-major or range-major order (BlockedTiling):
// either way the CTAs working at the same time include neighbouring tiles at
// the same range, whose regions stream the same planes together (their
// overlapping halos then come from L2). Otherwise the items are cut into
// equal contiguous ranges, tile after tile.
// Only the walking state is held (two counters); the tiling's constants are
// read from the kernel parameter where they are used, keeping them out of
// the registers of every thread.
struct UnitIter {
  long long i, hi;  // aligned split: next unit i; contiguous split: items [i, hi)
  __device__ void init(const BlockedTiling& t) {
    if (t.zsplit > 0) {
      i = blockIdx.x;
      hi = 0;
    } else {
      const long long n = (long long)t.tiles_x * t.tiles_y * (t.zhi - t.zlo);
      i = n * blockIdx.x / gridDim.x;
      hi = n * (blockIdx.x + 1) / gridDim.x;
    }
  }
  // Next unit: tile index and planes [z0, z1). False when done.
  __device__ bool next(const BlockedTiling& t, long long& tile, int& z0, int& z1) {
    const long long tiles = (long long)t.tiles_x * t.tiles_y;
    const int nz = t.zhi - t.zlo;
    if (t.zsplit > 0) {
      if (i >= tiles * t.zsplit) return false;
      const long long r = t.order ? i / tiles : i % t.zsplit;
      tile = t.order ? i % tiles : i / t.zsplit;
      z0 = t.zlo + (int)((long long)nz * r / t.zsplit);
      z1 = t.zlo + (int)((long long)nz * (r + 1) / t.zsplit);
      i += gridDim.x;
      return true;
    }
    if (i >= hi) return false;
    tile = i / nz;
    const int r0 = (int)(i % nz);
    const long long room = hi - i;
    const int r1 = (int)((long long)r0 + room < nz ? r0 + room : nz);
    i += r1 - r0;
    z0 = t.zlo + r0;
    z1 = t.zlo + r1;
    return true;
  }
};

// Tile coordinates of tile index `tile` of the tiling.
__device__ __forceinline__ void tile_xy(const BlockedTiling& t, long long tile, int& tx, int& ty) {
  tx = t.tx0 + (int)(tile % t.tiles_x);
  ty = t.ty0 + (int)(tile / t.tiles_x);
}

// Whether unit (tile, planes [z0, z1)) has outputs inside the launch box.
template <int K>
__device__ __forceinline__ bool unit_live(const StepArgs& a, const BlockedTiling& t, long long tile, int z0,
                                          int z1) {
  constexpr int TX = kRX - 2 * K, TY = kRY - 2 * K, PHI = K & 1;
  int tx, ty;
  tile_xy(t, tile, tx, ty);
  const int x0 = tx * TX - PHI, y0 = ty * TY;
  return box_meets(a.box, x0, x0 + TX, y0, y0 + TY, z0, z1);
}

// First iteration of a unit: level 1 updates plane s-1; planes below 0 are
// zero and exact, otherwise 3K-2 planes are replayed before z0.
template <int K>
__device__ __forceinline__ int first_iter(int z0) {
  const int s = z0 - 2 * K + 2;
  return s < 1 ? 1 : s;
}


// Issues the CTA's TMA loads in consumption order: for each unit, planes
// first_iter-1 .. z1-1+K of its tile. Only thread 0 issues. The per-plane
// counters stay in registers; the unit walk and the box origin, touched once
// per unit, live in shared memory so that they take no registers of the other
// threads.
struct LoaderState {
  UnitIter it;
  int bx, ry;
};

template <int K, int F>
struct Loader {
  LoaderState* st;
  int p, pend;
  long long issued;
  __device__ void init(const BlockedTiling& t) {
    st->it.init(t);
    st->bx = st->ry = 0;
    p = 0;
    pend = -1;
    issued = 0;
  }
  // Issue the next plane into its stage; false when the sequence is exhausted.
  __device__ bool issue(const StepArgs& a, const BlockedTiling& t, const CUtensorMap* tmF, const CUtensorMap* tmM,
                        unsigned char* base, uint32_t bar0) {
    if (p > pend) {
      long long tile;
      int z0, z1;
      do {
        if (!st->it.next(t, tile, z0, z1)) return false;
      } while (!unit_live<K>(a, t, tile, z0, z1));  // the consumers skip the same units
      int tx, ty;
      tile_xy(t, tile, tx, ty);
      const int rx = tx * Cfg<K, F>::TX - Cfg<K, F>::PHI - K;
      st->ry = ty * Cfg<K, F>::TY - K;
      st->bx = rx & ~(BoxCfg<F>::GX - 1);
      p = first_iter<K>(z0) - 1;
      pend = z1 - 1 + K;
    }
    constexpr int kNS = ring_stages(K);
    const int s = (int)(issued % kNS);
    const uint32_t bar = bar0 + 8u * s;
    using B = BoxCfg<F>;
    const int bx = st->bx, ry = st->ry;
    mbar_arrive_expect_tx(bar, B::kLoadBytes);
    tma_load_4d(smem_u32(base + s * B::kStageBytes), tmF, bx, ry, 0, p, bar);
    tma_load_3d(smem_u32(base + s * B::kStageBytes + B::kMatOff), tmM, bx, ry, p, bar);
    ++p;
    ++issued;
    return true;
  }
};

// NU: non-uniform mesh; every bracket in the scaled form (yee_update.cuh),
// the ratios of the lane's columns, its rows and the level's plane read per
// level from the padded pair arrays (L1) rather than held in registers.
template <int K, int FMT, bool NU, int R>
__global__ void __launch_bounds__(Lay<R>::kThreads, 1)
yee_blocked_kernel(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmM,
                   const __grid_constant__ StepArgs a, const __grid_constant__ BlockedTiling t) {
  constexpr int kW = Lay<R>::W;
  constexpr int kThreads = Lay<R>::kThreads;
  constexpr int kConsumers = kThreads;
  constexpr int kR = R;
  using St = sophie::St<R>;
  using C = Cfg<K, FMT, R>;
  constexpr int kNS = C::kNS;
  using B = BoxCfg<FMT>;
  using T = typename B::T;
  // Dynamic shared memory starts the CTA's shared window (no static shared
  // variables here), so it is 1024-byte aligned and its offsets are
  // compile-time constants.
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* const base = smem_raw;
  if (smem_u32(smem_raw) & 1023u) {  // never expected; refuse rather than misalign TMA
    if (threadIdx.x == 0) set_err(a.err, 16);
    return;
  }
  const uint32_t bar0 = smem_u32(base + C::kBarOff);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto sF = [&](int s) { return reinterpret_cast<const T*>(base + s * B::kStageBytes); };
  auto sM = [&](int s) { return reinterpret_cast<const uint32_t*>(base + s * B::kStageBytes + B::kMatOff); };
  // H seam rows: hp[level][warp][comp: 0 = hx, 1 = hz][64]
  float* hp = reinterpret_cast<float*>(base + C::kHpOff);
  // E seam rows: ep[level-1][parity][warp][comp: 0 = ex, 1 = ez][64]
  float* ep = reinterpret_cast<float*>(base + C::kEpOff);

  // (Ca, Cb) of every material class, read by all levels.
  float2* scoef = reinterpret_cast<float2*>(base + C::kCoefOff);
  const unsigned char* scoefb = base + C::kCoefOff;
  for (int c = threadIdx.x; c < kMaxClasses; c += kThreads) scoef[c] = a.coef[c];
  load_probes(reinterpret_cast<PrbShared*>(base + C::kPrbOff), a.prb, threadIdx.x, kThreads);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kNS; ++s) mbar_init(full(s), 1);
    fence_mbar_init();
  }
  __syncthreads();
  pdl_wait();  // (the class table above comes from a host copy, not a kernel)
  // Letting the next launch place its CTAs as this grid's retire changes which
  // SM each of its CTAs lands on. Measured at 768^3, K = 2: float storage
  // 183 -> 193 Gcell/s with the early trigger, the 24-bit form 231 -> 212, so
  // the 24-bit form keeps the implicit trigger at grid completion.
  if constexpr (FMT != kF24) pdl_launch_dependents();
  const Dims d = a.d;
  Loader<K, FMT> ld;
  ld.st = reinterpret_cast<LoaderState*>(base + C::kLdOff);
  if (threadIdx.x == 0) {
    ld.init(t);
    prefetch_tmap(&tmF);
    prefetch_tmap(&tmM);
    for (int s = 0; s < kNS; ++s)
      if (!ld.issue(a, t, &tmF, &tmM, base, bar0)) break;
  }

  const float S = a.S;
  const int wn = warp + 1 < kW ? warp + 1 : warp;  // seam partner below (clamped at the edge)
  const int wp = warp > 0 ? warp - 1 : warp;       // seam partner above
  UnitIter it;
  it.init(t);
  long long tile;
  int z0, z1;
  long long Cn = 0;  // consumed-plane counter (ring position)
  bool abort = false;
  while (!abort && it.next(t, tile, z0, z1)) {
    if (!unit_live<K>(a, t, tile, z0, z1)) continue;  // known zeros: no planes loaded for it
    int tx, ty;
    tile_xy(t, tile, tx, ty);
    const int rx = tx * C::TX - C::PHI - K, ry = ty * C::TY - K;
    const int ox = rx & (B::GX - 1);  // even: region start inside the TMA box
    const int col0 = ox + 2 * lane;
    const int x = rx + 2 * lane;  // global x of this lane's first position
    // output x range of this tile (the first tile of an odd K starts at -1)
    const int xo0 = max(tx * C::TX - C::PHI, 0), xo1 = tx * C::TX - C::PHI + C::TX;
    const int yo0 = ty * C::TY, yo1 = yo0 + C::TY;
    const int s0 = first_iter<K>(z0), s1 = z1 - 1 + K;
    // Output masks of this unit: rows of this thread inside the tile, and
    // which of its two x positions are inside it.
    const bool v0 = x >= xo0 && x < xo1 && x < d.nx;
    const bool v1 = x + 1 >= xo0 && x + 1 < xo1 && x + 1 < d.nx;
    uint32_t rowmask = 0;
    const long long rowbase = (long long)(ry + warp * kR) * d.nxp + x;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const int y = ry + warp * kR + r;
      if (y >= yo0 && y < yo1 && y < d.ny) rowmask |= 1u << r;
    }

    constexpr int NC = K > 1 ? K - 1 : 1;
    St carry[NC];
    // H of the plane below, per level: for levels 1..K-1 it is the level's own
    // output of the previous iteration, which sits in carry[lv-1] until this
    // iteration's output replaces it; only level K keeps a separate copy.
    float hxK[kR][2], hyK[kR][2];
#pragma unroll
    for (int l = 0; l < (K > 1 ? K - 1 : 1); ++l)
#pragma unroll
      for (int r = 0; r < kR; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          carry[l].ex[r][c] = carry[l].ey[r][c] = carry[l].ez[r][c] = 0.f;
          carry[l].hx[r][c] = carry[l].hy[r][c] = carry[l].hz[r][c] = 0.f;
          carry[l].m[r][c] = 0u;
        }
#pragma unroll
    for (int r = 0; r < kR; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) hxK[r][c] = hyK[r][c] = 0.f;
    // This warp's E seam rows start at zero, like the carries: in a unit's first
    // iteration level lv+1 reads the row "of the previous iteration", and for a
    // unit that starts at plane 0 that state is the (zero) state below the grid,
    // which reaches plane 0 through PEC coefficients -- a zero there, but a
    // NaN left in shared memory by an earlier launch would survive the multiply.
    // (Safe to write: every warp passed level lv+1's barrier of the previous
    // unit's last iteration only after all reads of these rows.)
#pragma unroll
    for (int l = 0; l < (K > 1 ? K - 1 : 0); ++l)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float* epz = ep + (l * 2 + q) * (kW * 2 * kRX);
        *reinterpret_cast<float2*>(&epz[(warp * 2 + 0) * kRX + 2 * lane]) = make_float2(0.f, 0.f);
        *reinterpret_cast<float2*>(&epz[(warp * 2 + 1) * kRX + 2 * lane]) = make_float2(0.f, 0.f);
      }

    for (int s = s0; s <= s1; ++s, ++Cn) {
      const int sc = (int)(Cn % kNS), sn = (int)((Cn + 1) % kNS);
      const bool ok = mbar_wait(full(sc), (uint32_t)((Cn / kNS) & 1)) &&
                      mbar_wait(full(sn), (uint32_t)(((Cn + 1) / kNS) & 1));
      if (!ok) set_err(a.err, 8);
      // (a failed wait is acted on at the first level barrier below; until then
      // the stage is only read, never written)
      const T* F = sF(sc);
      const T* Fn = sF(sn);
      const uint32_t* M = sM(sc);
      const int par = s & 1;

      // Level-0 state of plane s-1 and E of plane s (own positions).
      St in;
      float exn[kR][2], eyn[kR][2];
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int row = warp * kR + r;
        const float2 v0 = ld2c<FMT>(&F[FI<FMT>(0, row, col0)], a.isc[0], 0, B::CS);
        const float2 v1 = ld2c<FMT>(&F[FI<FMT>(1, row, col0)], a.isc[1], 1, B::CS);
        const float2 v2 = ld2c<FMT>(&F[FI<FMT>(2, row, col0)], a.isc[2], 2, B::CS);
        const float2 v3 = ld2c<FMT>(&F[FI<FMT>(3, row, col0)], a.isc[3], 3, B::CS);
        const float2 v4 = ld2c<FMT>(&F[FI<FMT>(4, row, col0)], a.isc[4], 4, B::CS);
        const float2 v5 = ld2c<FMT>(&F[FI<FMT>(5, row, col0)], a.isc[5], 5, B::CS);
        const uint2 mm = *reinterpret_cast<const uint2*>(&M[row * B::BX + col0]);
        const float2 n0 = ld2c<FMT>(&Fn[FI<FMT>(0, row, col0)], a.isc[0], 0, B::CS);
        const float2 n1 = ld2c<FMT>(&Fn[FI<FMT>(1, row, col0)], a.isc[1], 1, B::CS);
        in.ex[r][0] = v0.x; in.ex[r][1] = v0.y;
        in.ey[r][0] = v1.x; in.ey[r][1] = v1.y;
        in.ez[r][0] = v2.x; in.ez[r][1] = v2.y;
        in.hx[r][0] = v3.x; in.hx[r][1] = v3.y;
        in.hy[r][0] = v4.x; in.hy[r][1] = v4.y;
        in.hz[r][0] = v5.x; in.hz[r][1] = v5.y;
        in.m[r][0] = mm.x; in.m[r][1] = mm.y;
        exn[r][0] = n0.x; exn[r][1] = n0.y;
        eyn[r][0] = n1.x; eyn[r][1] = n1.y;
      }
      // E of the row below this warp's rows, level 0 (straight from the stage).
      float bex[2], bez[2];
      {
        const int brow = warp * kR + kR < kRY ? warp * kR + kR : kRY - 1;
        const float2 b0 = ld2c<FMT>(&F[FI<FMT>(0, brow, col0)], a.isc[0], 0, B::CS);
        const float2 b2 = ld2c<FMT>(&F[FI<FMT>(2, brow, col0)], a.isc[2], 2, B::CS);
        bex[0] = b0.x; bex[1] = b0.y;
        bez[0] = b2.x; bez[1] = b2.y;
      }
      // The level-0 planes are now in registers; stage sc is refilled by
      // thread 0 after the first level barrier below.

#pragma unroll
      for (int lv = 1; lv <= K; ++lv) {
        const int p = s - lv;  // plane updated by this level
        const long long nstep = a.n0 + lv - 1;
        // Non-uniform mesh: (primary, dual) ratios of the lane's two columns
        // (x is even: one aligned 16-byte load) and of the level's plane;
        // rows are read where they are used. Region and plane indices stay
        // within the arrays' zero padding (at least -K-1 and below n + 72).
        float4 rxp = make_float4(1.f, 1.f, 1.f, 1.f);
        float2 rzp = make_float2(1.f, 1.f);
        if constexpr (NU) {
          rxp = *reinterpret_cast<const float4*>(a.rpair[0] + x);
          rzp = a.rpair[2][p];
        }
        auto rrow = [&](int r) -> float2 {  // (ry, ryd) of row r of this thread
          if constexpr (NU)
            return a.rpair[1][ry + warp * kR + r];
          else
            return make_float2(1.f, 1.f);
        };
        // H of this level at plane p-1 (see hxK above)
        auto hxprev = [&](int lvl, int r, int c) -> float {
          return lvl < K ? carry[lvl - 1 < NC ? lvl - 1 : 0].hx[r][c] : hxK[r][c];
        };
        auto hyprev = [&](int lvl, int r, int c) -> float {
          return lvl < K ? carry[lvl - 1 < NC ? lvl - 1 : 0].hy[r][c] : hyK[r][c];
        };
        // ---- H of level lv at plane p ----
        float hx[kR][2], hy[kR][2], hz[kR][2];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const float ey_ip1 = __shfl_down_sync(0xffffffffu, in.ey[r][0], 1);
          const float ez_ip1 = __shfl_down_sync(0xffffffffu, in.ez[r][0], 1);
          float exj[2], ezj[2];
          if (r + 1 < kR) {
            exj[0] = in.ex[r + 1][0]; exj[1] = in.ex[r + 1][1];
            ezj[0] = in.ez[r + 1][0]; ezj[1] = in.ez[r + 1][1];
          } else {
            exj[0] = bex[0]; exj[1] = bex[1];
            ezj[0] = bez[0]; ezj[1] = bez[1];
          }
          // the lane's two x positions as packed pairs
          auto P = [](const float (&v)[2]) { return make_float2(v[0], v[1]); };
          float2 hx2, hy2, hz2;
          if constexpr (NU) {
            // scaled brackets with the b ratios negated (curl_br2_nu)
            const float2 S2 = make_float2(S, S);
            const float ryr = rrow(r).x;
            hx2 = __ffma2_rn(S2, curl_br2_nu(make_float2(rzp.x, rzp.x), P(eyn[r]), P(in.ey[r]),
                                             make_float2(-ryr, -ryr), P(ezj), P(in.ez[r])), P(in.hx[r]));
            hy2 = __ffma2_rn(S2, curl_br2_nu(make_float2(rxp.x, rxp.z), make_float2(in.ez[r][1], ez_ip1),
                                             P(in.ez[r]), make_float2(-rzp.x, -rzp.x), P(exn[r]), P(in.ex[r])),
                             P(in.hy[r]));
            hz2 = __ffma2_rn(S2, curl_br2_nu(make_float2(ryr, ryr), P(exj), P(in.ex[r]),
                                             make_float2(-rxp.x, -rxp.z), make_float2(in.ey[r][1], ey_ip1),
                                             P(in.ey[r])), P(in.hz[r]));
          } else {
            hx2 = h_upd2(P(in.hx[r]), S, P(eyn[r]), P(in.ey[r]), P(ezj), P(in.ez[r]));
            hy2 = h_upd2(P(in.hy[r]), S, make_float2(in.ez[r][1], ez_ip1), P(in.ez[r]), P(exn[r]), P(in.ex[r]));
            hz2 = h_upd2(P(in.hz[r]), S, P(exj), P(in.ex[r]), make_float2(in.ey[r][1], ey_ip1), P(in.ey[r]));
          }
          hx[r][0] = hx2.x; hx[r][1] = hx2.y;
          hy[r][0] = hy2.x; hy[r][1] = hy2.y;
          hz[r][0] = hz2.x; hz[r][1] = hz2.y;
        }
        float* hpl = hp + (lv - 1) * (kW * 2 * kRX);
        *reinterpret_cast<float2*>(&hpl[(warp * 2 + 0) * kRX + 2 * lane]) = make_float2(hx[kR - 1][0], hx[kR - 1][1]);
        *reinterpret_cast<float2*>(&hpl[(warp * 2 + 1) * kRX + 2 * lane]) = make_float2(hz[kR - 1][0], hz[kR - 1][1]);
        if (lv == 1) {
          if (named_bar_or(1, kConsumers, !ok)) {
            abort = true;
            break;
          }
        } else {
          named_bar(1, kConsumers);
        }
        if (lv == 1 && threadIdx.x == 0) {
          // Every warp has passed the copy of stage sc (and, in a unit's last
          // iteration, of stage sn, which holds no further plane of this unit).
          const long long released = Cn + 1 + (s == s1 ? 1 : 0);
          fence_proxy_async_smem();
          while (ld.issued < released + kNS)
            if (!ld.issue(a, t, &tmF, &tmM, base, bar0)) break;
        }
        float hxa[2], hza[2];  // H of the row above this warp's rows
        {
          const float2 u = *reinterpret_cast<const float2*>(&hpl[(wp * 2 + 0) * kRX + 2 * lane]);
          const float2 v = *reinterpret_cast<const float2*>(&hpl[(wp * 2 + 1) * kRX + 2 * lane]);
          hxa[0] = u.x; hxa[1] = u.y;
          hza[0] = v.x; hza[1] = v.y;
        }
        // ---- E of level lv at plane p ----
        // Source and probe points are rare: one warp-uniform test per level
        // picks the check-free loop or the one that handles them.
        uint32_t fl = 0;
#pragma unroll
        for (int r = 0; r < kR; ++r) fl |= in.m[r][0] | in.m[r][1];
        const bool rare = __any_sync(0xffffffffu, fl & (kSrcFlag | kPrbFlag | kExpFlag));
        St out;
        if (!rare) {
#pragma unroll
          for (int r = 0; r < kR; ++r) {
            const float hz_im1 = __shfl_up_sync(0xffffffffu, hz[r][1], 1);
            const float hy_im1 = __shfl_up_sync(0xffffffffu, hy[r][1], 1);
            const int rj = r > 0 ? r - 1 : 0;
            const float2 hzj = r > 0 ? make_float2(hz[rj][0], hz[rj][1]) : make_float2(hza[0], hza[1]);
            const float2 hxj = r > 0 ? make_float2(hx[rj][0], hx[rj][1]) : make_float2(hxa[0], hxa[1]);
            // brackets of the lane's two x positions as packed pairs
            float2 bx, by, bz;
            if constexpr (NU) {
              const float rydr = rrow(r).y;
              bx = curl_br2_nu(make_float2(rydr, rydr), make_float2(hz[r][0], hz[r][1]), hzj,
                               make_float2(-rzp.y, -rzp.y), make_float2(hy[r][0], hy[r][1]),
                               make_float2(hyprev(lv, r, 0), hyprev(lv, r, 1)));
              by = curl_br2_nu(make_float2(rzp.y, rzp.y), make_float2(hx[r][0], hx[r][1]),
                               make_float2(hxprev(lv, r, 0), hxprev(lv, r, 1)), make_float2(-rxp.y, -rxp.w),
                               make_float2(hz[r][0], hz[r][1]), make_float2(hz_im1, hz[r][0]));
              bz = curl_br2_nu(make_float2(rxp.y, rxp.w), make_float2(hy[r][0], hy[r][1]),
                               make_float2(hy_im1, hy[r][0]), make_float2(-rydr, -rydr), make_float2(hx[r][0], hx[r][1]),
                               hxj);
            } else {
              bx = curl_br2(make_float2(hz[r][0], hz[r][1]), hzj, make_float2(hy[r][0], hy[r][1]),
                            make_float2(hyprev(lv, r, 0), hyprev(lv, r, 1)));
              by = curl_br2(make_float2(hx[r][0], hx[r][1]), make_float2(hxprev(lv, r, 0), hxprev(lv, r, 1)),
                            make_float2(hz[r][0], hz[r][1]), make_float2(hz_im1, hz[r][0]));
              bz = curl_br2(make_float2(hy[r][0], hy[r][1]), make_float2(hy_im1, hy[r][0]),
                            make_float2(hx[r][0], hx[r][1]), hxj);
            }
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const uint32_t m = in.m[r][cc];
              out.ex[r][cc] = e_upd(in.ex[r][cc], *reinterpret_cast<const float2*>(scoefb + cls_off_x(m)), cc ? bx.y : bx.x);
              out.ey[r][cc] = e_upd(in.ey[r][cc], *reinterpret_cast<const float2*>(scoefb + cls_off_y(m)), cc ? by.y : by.x);
              out.ez[r][cc] = e_upd(in.ez[r][cc], *reinterpret_cast<const float2*>(scoefb + cls_off_z(m)), cc ? bz.y : bz.x);
              out.m[r][cc] = m;
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < kR; ++r) {
            const float hz_im1 = __shfl_up_sync(0xffffffffu, hz[r][1], 1);
            const float hy_im1 = __shfl_up_sync(0xffffffffu, hy[r][1], 1);
            const int y = ry + warp * kR + r;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const float hzj = r > 0 ? hz[r > 0 ? r - 1 : 0][cc] : hza[cc];
              const float hxj = r > 0 ? hx[r > 0 ? r - 1 : 0][cc] : hxa[cc];
              const float hzi = cc ? hz[r][0] : hz_im1;
              const float hyi = cc ? hy[r][0] : hy_im1;
              const float2 rr = rrow(r);  // ratios of the row, of the column (dual), scaled form if NU
              const float rxdc = cc ? rxp.w : rxp.y;
              float bx = bracket<NU>(rr.y, hz[r][cc], hzj, rzp.y, hy[r][cc], hyprev(lv, r, cc));
              float by = bracket<NU>(rzp.y, hx[r][cc], hxprev(lv, r, cc), rxdc, hz[r][cc], hzi);
              float bz = bracket<NU>(rxdc, hy[r][cc], hyi, rr.y, hx[r][cc], hxj);
              const uint32_t m = in.m[r][cc];
              if (m & kSrcFlag) {
                const float3 b3 = apply_sources(make_float3(bx, by, bz),
                                                ((long long)p * d.ny1 + y) * d.nxp + x + cc, nstep, &a.src);
                bx = b3.x;
                by = b3.y;
                bz = b3.z;
              }
              float2 k0, k1, k2;
              if (m & kExpFlag) {
                const float2* e3 = a.ecoef + 3ull * (m >> 3);
                k0 = __ldg(e3);
                k1 = __ldg(e3 + 1);
                k2 = __ldg(e3 + 2);
              } else {
                k0 = *reinterpret_cast<const float2*>(scoefb + cls_off_x(m));
                k1 = *reinterpret_cast<const float2*>(scoefb + cls_off_y(m));
                k2 = *reinterpret_cast<const float2*>(scoefb + cls_off_z(m));
              }
              out.ex[r][cc] = e_upd(in.ex[r][cc], k0, bx);
              out.ey[r][cc] = e_upd(in.ey[r][cc], k1, by);
              out.ez[r][cc] = e_upd(in.ez[r][cc], k2, bz);
              out.m[r][cc] = m;
              if ((m & kPrbFlag) && p >= z0 && p < z1 && y >= yo0 && y < yo1 && y < d.ny &&
                  x + cc >= xo0 && x + cc < xo1 && x + cc < d.nx)
                record_probes(((long long)p * d.ny1 + y) * d.nxp + x + cc, nstep, out.ex[r][cc], out.ey[r][cc],
                              out.ez[r][cc], hx[r][cc], hy[r][cc], hz[r][cc],
                              reinterpret_cast<const PrbShared*>(base + C::kPrbOff));
            }
          }
        }
#pragma unroll
        for (int r = 0; r < kR; ++r)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            out.hx[r][cc] = hx[r][cc];
            out.hy[r][cc] = hy[r][cc];
            out.hz[r][cc] = hz[r][cc];
            if (lv == K) {
              hxK[r][cc] = hx[r][cc];
              hyK[r][cc] = hy[r][cc];
            }
          }
        if (lv < K) {
          // Publish this warp's first E row for level lv+1 (next iteration), then
          // feed level lv+1: its input is this level's state of plane p-1 (carry),
          // its "E of the plane above" is what was just computed.
          float* epl = ep + ((lv - 1) * 2 + par) * (kW * 2 * kRX);
          *reinterpret_cast<float2*>(&epl[(warp * 2 + 0) * kRX + 2 * lane]) = make_float2(out.ex[0][0], out.ex[0][1]);
          *reinterpret_cast<float2*>(&epl[(warp * 2 + 1) * kRX + 2 * lane]) = make_float2(out.ez[0][0], out.ez[0][1]);
          const float* epo = ep + ((lv - 1) * 2 + (par ^ 1)) * (kW * 2 * kRX);
          const float2 u = *reinterpret_cast<const float2*>(&epo[(wn * 2 + 0) * kRX + 2 * lane]);
          const float2 v = *reinterpret_cast<const float2*>(&epo[(wn * 2 + 1) * kRX + 2 * lane]);
          bex[0] = u.x; bex[1] = u.y;
          bez[0] = v.x; bez[1] = v.y;
#pragma unroll
          for (int r = 0; r < kR; ++r)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              exn[r][cc] = out.ex[r][cc];
              eyn[r][cc] = out.ey[r][cc];
            }
          in = carry[lv - 1];
          carry[lv - 1] = out;
        } else if (p >= z0 && p < z1) {
          // ---- level K: store the output tile of plane p ----
#pragma unroll
          for (int r = 0; r < kR; ++r) {
            if (!((rowmask >> r) & 1)) continue;
            T* o = static_cast<T*>(a.fout) + (long long)p * d.zstride + rowbase + (long long)r * d.nxp;
            const float vals[6][2] = {{out.ex[r][0], out.ex[r][1]}, {out.ey[r][0], out.ey[r][1]},
                                      {out.ez[r][0], out.ez[r][1]}, {out.hx[r][0], out.hx[r][1]},
                                      {out.hy[r][0], out.hy[r][1]}, {out.hz[r][0], out.hz[r][1]}};
            if (v0 || v1) st6<FMT>(o, d.plane, vals, a.sc, (v0 ? 1 : 0) | (v1 ? 2 : 0));
          }
        }
      }
      if (abort) break;
    }
    if (abort) break;
    ++Cn;  // the unit's last staged plane was only read as "plane s"
  }
  if (abort && threadIdx.x == 0) {
    // Give the copies still in flight a bounded chance to land before exit.
    for (long long e = ld.issued - 1; e >= 0 && e >= ld.issued - kNS; --e)
      mbar_wait(full((int)(e % kNS)), (uint32_t)((e / kNS) & 1));
  }
}

template <int K, int F, bool NU, int R>
cudaError_t launch_knr(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const BlockedTiling& t,
                       cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(yee_blocked_kernel<K, F, NU, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<K, F, R>::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_step_kernel(yee_blocked_kernel<K, F, NU, R>, dim3(t.grid), dim3(Lay<R>::kThreads), Cfg<K, F, R>::kSmem,
                            s, tmF, tmM, a, t);
}

template <int K, int F, bool NU>
cudaError_t launch_kn(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const BlockedTiling& t,
                      cudaStream_t s) {
  // the 16-warp layout's seam rows fit in shared memory beside the ring for K = 2 only
  if constexpr (K == 2)
    if (t.rows == 2) return launch_knr<K, F, NU, 2>(a, tmF, tmM, t, s);
  return launch_knr<K, F, NU, 4>(a, tmF, tmM, t, s);
}

template <int K, int F>
cudaError_t launch_k(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const BlockedTiling& t,
                     cudaStream_t s) {
  return a.rat[0] ? launch_kn<K, F, true>(a, tmF, tmM, t, s) : launch_kn<K, F, false>(a, tmF, tmM, t, s);
}

template <int F>
cudaError_t launch_fmt(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const BlockedTiling& t,
                       cudaStream_t s) {
  switch (t.K) {
    case 2: return launch_k<2, F>(a, tmF, tmM, t, s);
    case 3: return launch_k<3, F>(a, tmF, tmM, t, s);
    case 4: return launch_k<4, F>(a, tmF, tmM, t, s);
    // the deep forms (a two-stage ring) are built for float storage only
    case 6: if constexpr (F == kF32) return launch_k<6, F>(a, tmF, tmM, t, s); else return cudaErrorInvalidValue;
    case 8: if constexpr (F == kF32) return launch_k<8, F>(a, tmF, tmM, t, s); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sophie
