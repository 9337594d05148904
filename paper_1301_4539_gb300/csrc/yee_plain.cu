// yee_plain: one fused H+E leapfrog step per launch, TMA-staged (sm_103a).
//
// Method: Sec. 2.1 leapfrog, with Sec. 3.2's interleave and Sec. 3.3's plane
// by plane order: within one (x,y) tile the H update of plane z is followed by
// the E update of plane z, so each field is read once and written once per
// step (48 B of fields per cell-update + a 4 B material word).
//
// GPU design:
//  * Persistent CTAs walk a list of work units (64x16 output tile, chunk of z
//    planes). One producer warp streams planes of all six fields plus the
//    material words into a 3-stage shared-memory ring with 4-D/3-D TMA tile
//    loads (72x18 box: the tile plus a 4-column / 1-row halo; out-of-range
//    parts of the box arrive as zeros, which is exactly the PEC / outside
//    value). Full/empty mbarriers pace the ring; every wait is bounded.
//  * Eight consumer warps own two rows each; a lane owns two adjacent x.
//    H of the plane is computed in place in the ring (plus the halo H at x0-1
//    and y0-1, recomputed identically to the neighbouring tile's), one named
//    barrier, then E from the updated H. H of the plane below stays in
//    registers (z streaming), so only x-y neighbours go through shared memory.
//  * Results go straight from registers to HBM (the other ping-pong buffer)
//    with coalesced 8-byte stores.
#include "sophie_internal.h"
#include "tma_util.cuh"
#include "yee_rare.cuh"
#include "yee_store.cuh"
#include "yee_update.cuh"

#include <cudaTypedefs.h>

#include <algorithm>

namespace sophie {

namespace {

constexpr int kPX = 64, kPY = 16;
constexpr int kBY = kPY + 2;
constexpr int kNS = 3;
constexpr int kCW = kPY / 2;  // consumer warps
constexpr int kConsumers = kCW * 32;
constexpr int kThreads = kConsumers + 32;

// Per storage format: the box starts OX columns left of the tile (OX = the
// TMA 16-byte granule in elements), so it is (64 + 2 OX) wide. With float
// storage the updated H is written back into the ring in place; with 2-byte
// storage it goes to a float buffer (two planes, by parity) instead.
template <int F>
struct PCfg {
  using T = typename Store<F>::T;
  static constexpr int OX = Store<F>::kAlign;
  static constexpr int BX = kPX + 2 * OX;
  static constexpr int P = store_planes(F);  // planes per slab (nine 2-byte planes for kF24)
  static constexpr bool kInPlace = sizeof(T) == 4;  // a float fits in the ring slot
  static constexpr uint32_t kFieldBytes = BX * kBY * P * sizeof(T);
  static constexpr uint32_t kMatOff = (kFieldBytes + 127) / 128 * 128;  // material box, 128-byte aligned
  static constexpr uint32_t kMatBytes = BX * kBY * 4;
  static constexpr uint32_t kLoadBytes = kFieldBytes + kMatBytes;
  static constexpr uint32_t kStageBytes = (kMatOff + kMatBytes + 127) / 128 * 128;
  static constexpr long long CS = (long long)kBY * BX;  // elements between component planes
  static constexpr uint32_t kHbOff = kNS * kStageBytes;
  static constexpr uint32_t kHbBytes = kInPlace ? 0 : 2 * 3 * kBY * BX * 4;
  static constexpr uint32_t kBarOff = kHbOff + kHbBytes;
  // class table (Ca, Cb) of a single grid, indexed by the material word's
  // pre-scaled byte offsets (batches read their cavities' tables from L1)
  static constexpr uint32_t kCoefOff = (kBarOff + 2 * kNS * 8 + 15) / 16 * 16;
  static constexpr uint32_t kPrbOff = kCoefOff + kMaxClasses * 8;  // the probe table (PrbShared)
  static constexpr uint32_t kSmemBytes = kPrbOff + sizeof(PrbShared) + 128;
};

struct Unit {
  int x0, y0, z0, z1;
};

__device__ __forceinline__ Unit unit_of(long long u, const PlainTiling& t) {
  Unit w;
  const int tx = t.tx0 + (int)(u % t.tiles_x);
  const long long q = u / t.tiles_x;
  const int ty = t.ty0 + (int)(q % t.tiles_y);
  const int zc = (int)(q / t.tiles_y);
  w.x0 = tx * kPX;
  w.y0 = ty * kPY;
  w.z0 = t.z0 + zc * t.zchunk;
  w.z1 = min(w.z0 + t.zchunk, t.z1);
  return w;
}

__device__ __forceinline__ void set_err(int* err, int code) { atomicOr(err, code); }

// BATCH: the work units are the items of a batch of cavities (one step of
// every cavity); each unit takes its tensor maps, sizes, output buffer,
// coefficient tables and sources from its cavity's descriptor. Otherwise the
// units tile the single grid of `a` as described by `t`.
// NU: non-uniform mesh; every difference is scaled by the ratio of the width
// it spans (a.rat): a lane keeps the ratios of its two columns and two rows,
// the plane's ratio is read per plane.
template <int FMT, bool BATCH, bool NU>
__global__ void __launch_bounds__(kThreads, 2)
yee_plain_kernel(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmM,
                 const __grid_constant__ StepArgs a, PlainTiling t, PlainBatch pb) {
  static_assert(!BATCH || FMT == kF32, "batches store float fields");
  static_assert(!(BATCH && NU), "batches are uniform meshes");
  using C = PCfg<FMT>;
  using T = typename C::T;
  constexpr int BX = C::BX;
  constexpr int OX = C::OX;
  auto FI = [](int f, int r, int c) { return (f * kBY + r) * BX + c; };
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const uint32_t bar0 = smem_u32(base + C::kBarOff);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kNS + s); };
  auto sF = [&](int s) { return reinterpret_cast<T*>(base + s * C::kStageBytes); };
  auto sM = [&](int s) { return reinterpret_cast<const uint32_t*>(base + s * C::kStageBytes + C::kMatOff); };
  float* const hbuf = reinterpret_cast<float*>(base + C::kHbOff);
  const unsigned char* const scoefb = base + C::kCoefOff;
  if constexpr (!BATCH)
    for (int c = threadIdx.x; c < kMaxClasses; c += kThreads)
      reinterpret_cast<float2*>(base + C::kCoefOff)[c] = a.coef[c];
  load_probes(reinterpret_cast<PrbShared*>(base + C::kPrbOff), a.prb, threadIdx.x, kThreads);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kNS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), kCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  pdl_wait();  // (the class table above comes from a host copy, not a kernel)
  pdl_launch_dependents();
  const long long nunits = BATCH ? (long long)pb.nitems : t.units;
  // Unit u: its tile and z range, and (batches) its cavity's descriptor.
  auto unit_at = [&](long long u, const CavityDesc*& cd) -> Unit {
    if constexpr (BATCH) {
      const BatchItem it = pb.items[u];
      cd = pb.descs + it.cav;
      return Unit{it.x0, it.y0, it.z0, it.z1};
    } else {
      cd = nullptr;
      return unit_of(u, t);
    }
  };

  if (warp == kCW) {
    // ---------------- producer warp ----------------
    if (lane != 0) return;
    if constexpr (!BATCH) {
      prefetch_tmap(&tmF);
      prefetch_tmap(&tmM);
    }
    long long L = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const CavityDesc* cd;
      const Unit w = unit_at(u, cd);
      if constexpr (!BATCH) {
        if (!box_meets(a.box, w.x0, w.x0 + kPX, w.y0, w.y0 + kPY, w.z0, w.z1)) continue;  // known zeros
      }
      const CUtensorMap* mF = BATCH ? &cd->tmF[pb.cur] : &tmF;
      const CUtensorMap* mM = BATCH ? &cd->tmM : &tmM;
      const int ps = w.z0 > 0 ? w.z0 - 1 : 0;
      for (int p = ps; p <= w.z1; ++p, ++L) {
        const int s = (int)(L % kNS);
        if (L >= kNS && !mbar_wait(empty(s), (uint32_t)(((L / kNS) - 1) & 1))) {
          set_err(a.err, 1);
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(full(s), C::kLoadBytes);
        tma_load_4d(smem_u32(sF(s)), mF, w.x0 - OX, w.y0 - 1, 0, p, full(s));
        tma_load_3d(smem_u32(sM(s)), mM, w.x0 - OX, w.y0 - 1, p, full(s));
      }
    }
    if (!ok) {
      // Give the copies already issued a bounded chance to land before exit.
      for (long long e = L - 1; e >= 0 && e >= L - kNS; --e)
        mbar_wait(full((int)(e % kNS)), (uint32_t)((e / kNS) & 1));
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int c0 = OX + 2 * lane;
  const int r0 = 1 + 2 * warp;
  int hr = -1, hc = -1;  // halo H position computed by this lane
  if (lane < 2) {
    hr = r0 + lane;
    hc = OX - 1;
  } else if (lane < 10) {
    hr = 0;
    hc = OX + 8 * warp + (lane - 2);
  }
  const float S = a.S;
  long long C_ = 0;
  bool abort = false;
  // Batches: the current unit's cavity context lives in shared memory (two
  // copies by unit parity: a warp can start unit u+1 while others finish the
  // stores of unit u, never later ones, because of the per-plane barrier),
  // keeping these values out of the consumers' registers.
  struct UnitCtx {
    T* fout;
    const float2* coef;
    const float2* ecoef;
    const SrcTable* srct;
    int nx, ny, nxp, ny1, plane, zstride;
  };
  __shared__ UnitCtx uctx[BATCH ? 2 : 1];
  int upar = 0;
  for (long long u = blockIdx.x; u < nunits && !abort; u += gridDim.x, upar ^= 1) {
    const CavityDesc* cd;
    const Unit w = unit_at(u, cd);
    if constexpr (!BATCH) {
      if (!box_meets(a.box, w.x0, w.x0 + kPX, w.y0, w.y0 + kPY, w.z0, w.z1)) continue;  // as the producer
    }
    if constexpr (BATCH) {
      if (threadIdx.x == 0) {
        UnitCtx& c = uctx[upar];
        c.fout = static_cast<T*>(cd->F[1 - pb.cur]);
        c.coef = cd->coef;
        c.ecoef = cd->ecoef;
        c.srct = &cd->src;
        c.nx = cd->d.nx;
        c.ny = cd->d.ny;
        c.nxp = cd->d.nxp;
        c.ny1 = cd->d.ny1;
        c.plane = (int)cd->d.plane;
        c.zstride = (int)cd->d.zstride;
      }
    }
    const UnitCtx* uc = &uctx[BATCH ? upar : 0];
    struct {
      const StepArgs& a;
      const UnitCtx* uc;
      __device__ int nx() const { return BATCH ? uc->nx : a.d.nx; }
      __device__ int ny() const { return BATCH ? uc->ny : a.d.ny; }
      __device__ long long nxp() const { return BATCH ? uc->nxp : a.d.nxp; }
      __device__ long long ny1() const { return BATCH ? uc->ny1 : a.d.ny1; }
      __device__ long long plane() const { return BATCH ? uc->plane : a.d.plane; }
      __device__ long long zstride() const { return BATCH ? uc->zstride : a.d.zstride; }
    } d{a, uc};
    auto fout = [&]() { return BATCH ? uc->fout : static_cast<T*>(a.fout); };
    auto coef = [&]() { return BATCH ? uc->coef : a.coef; };
    auto ecoef = [&]() { return BATCH ? uc->ecoef : a.ecoef; };
    auto srct = [&]() { return BATCH ? uc->srct : &a.src; };
    const int ps = w.z0 > 0 ? w.z0 - 1 : 0;
    float hxp[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, hyp[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int z = ps; z < w.z1; ++z, ++C_) {
      // Ratios of this lane's columns, rows, halo point and plane (1, unused,
      // on a uniform mesh): (primary, dual) pairs of the padded arrays, the
      // two columns (rows) in one 16-byte load, read per plane from L1 (once
      // for the H phase, again for the E phase) rather than held in
      // registers across the loop.
      float rxv[2] = {1.f, 1.f}, rxdv[2] = {1.f, 1.f}, ryv[2] = {1.f, 1.f}, rydv[2] = {1.f, 1.f};
      float rxh = 1.f, ryh = 1.f, rz = 1.f, rzd = 1.f;
      const int xl = w.x0 + 2 * lane, yl = w.y0 + 2 * warp;  // even: 16-byte aligned pairs
      if constexpr (NU) {
        const float4 px = *reinterpret_cast<const float4*>(a.rpair[0] + xl);
        const float4 py = *reinterpret_cast<const float4*>(a.rpair[1] + yl);
        rxv[0] = px.x;
        rxv[1] = px.z;
        ryv[0] = py.x;
        ryv[1] = py.z;
        if (hr >= 0) {
          rxh = a.rpair[0][w.x0 - OX + hc].x;
          ryh = a.rpair[1][w.y0 - 1 + hr].x;
        }
        rz = a.rpair[2][z].x;
      }
      const int sc = (int)(C_ % kNS), sn = (int)((C_ + 1) % kNS);
      const bool ok = mbar_wait(full(sc), (uint32_t)((C_ / kNS) & 1)) &&
                      mbar_wait(full(sn), (uint32_t)(((C_ + 1) / kNS) & 1));
      if (!ok) set_err(a.err, 2);
      T* F = sF(sc);
      const T* Fn = sF(sn);
      // Updated H of this plane: in the ring (float storage) or the float buffer.
      float* const Hb = hbuf + (z & 1) * (3 * kBY * BX);
      auto hp = [&](int comp, int r, int c) -> float* {
        if constexpr (C::kInPlace)
          return reinterpret_cast<float*>(&F[FI(3 + comp, r, c)]);
        else
          return &Hb[(comp * kBY + r) * BX + c];
      };
      float ex[2][2], ey[2][2], ez[2][2], hx[2][2], hy[2][2], hz[2][2];
      if (ok) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int row = r0 + r;
          const float2 vex = ld2c<FMT>(&F[FI(0, row, c0)], a.isc[0], 0, C::CS);
          const float2 vey = ld2c<FMT>(&F[FI(1, row, c0)], a.isc[1], 1, C::CS);
          const float2 vez = ld2c<FMT>(&F[FI(2, row, c0)], a.isc[2], 2, C::CS);
          ex[r][0] = vex.x; ex[r][1] = vex.y;
          ey[r][0] = vey.x; ey[r][1] = vey.y;
          ez[r][0] = vez.x; ez[r][1] = vez.y;
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int row = r0 + r;
          const float2 vhx = ld2c<FMT>(&F[FI(3, row, c0)], a.isc[3], 3, C::CS);
          const float2 vhy = ld2c<FMT>(&F[FI(4, row, c0)], a.isc[4], 4, C::CS);
          const float2 vhz = ld2c<FMT>(&F[FI(5, row, c0)], a.isc[5], 5, C::CS);
          const float2 nex = ld2c<FMT>(&Fn[FI(0, row, c0)], a.isc[0], 0, C::CS);
          const float2 ney = ld2c<FMT>(&Fn[FI(1, row, c0)], a.isc[1], 1, C::CS);
          float exj[2], ezj[2];
          if (r == 0) {
            exj[0] = ex[1][0]; exj[1] = ex[1][1];
            ezj[0] = ez[1][0]; ezj[1] = ez[1][1];
          } else {
            const float2 a2 = ld2c<FMT>(&F[FI(0, row + 1, c0)], a.isc[0], 0, C::CS);
            const float2 b2 = ld2c<FMT>(&F[FI(2, row + 1, c0)], a.isc[2], 2, C::CS);
            exj[0] = a2.x; exj[1] = a2.y;
            ezj[0] = b2.x; ezj[1] = b2.y;
          }
          const float ez_ip1 = ldc<FMT>(&F[FI(2, row, c0 + 2)], a.isc[2], 2, C::CS);
          const float ey_ip1 = ldc<FMT>(&F[FI(1, row, c0 + 2)], a.isc[1], 1, C::CS);
          // the lane's two x positions as packed pairs
          auto P = [](const float (&v)[2]) { return make_float2(v[0], v[1]); };
          if constexpr (NU) {
            // the b ratios negated (curl_br2_nu)
            const float2 S2 = make_float2(S, S);
            const float2 rz2 = make_float2(rz, rz), ry2 = make_float2(ryv[r], ryv[r]);
            const float2 rx2 = make_float2(rxv[0], rxv[1]);
            const float2 hx2 = __ffma2_rn(S2, curl_br2_nu(rz2, ney, P(ey[r]), make_float2(-ryv[r], -ryv[r]), P(ezj),
                                                          P(ez[r])), vhx);
            const float2 hy2 = __ffma2_rn(S2, curl_br2_nu(rx2, make_float2(ez[r][1], ez_ip1), P(ez[r]),
                                                          make_float2(-rz, -rz), nex, P(ex[r])), vhy);
            const float2 hz2 = __ffma2_rn(S2, curl_br2_nu(ry2, P(exj), P(ex[r]), make_float2(-rxv[0], -rxv[1]),
                                                          make_float2(ey[r][1], ey_ip1), P(ey[r])), vhz);
            hx[r][0] = hx2.x; hx[r][1] = hx2.y;
            hy[r][0] = hy2.x; hy[r][1] = hy2.y;
            hz[r][0] = hz2.x; hz[r][1] = hz2.y;
          } else {
            const float2 hx2 = h_upd2(vhx, S, ney, P(ey[r]), P(ezj), P(ez[r]));
            const float2 hy2 = h_upd2(vhy, S, make_float2(ez[r][1], ez_ip1), P(ez[r]), nex, P(ex[r]));
            const float2 hz2 = h_upd2(vhz, S, P(exj), P(ex[r]), make_float2(ey[r][1], ey_ip1), P(ey[r]));
            hx[r][0] = hx2.x; hx[r][1] = hx2.y;
            hy[r][0] = hy2.x; hy[r][1] = hy2.y;
            hz[r][0] = hz2.x; hz[r][1] = hz2.y;
          }
          *reinterpret_cast<float2*>(hp(0, row, c0)) = make_float2(hx[r][0], hx[r][1]);
          *reinterpret_cast<float2*>(hp(1, row, c0)) = make_float2(hy[r][0], hy[r][1]);
          *reinterpret_cast<float2*>(hp(2, row, c0)) = make_float2(hz[r][0], hz[r][1]);
        }
        if (hr >= 0) {
          const float e0 = ldc<FMT>(&F[FI(0, hr, hc)], a.isc[0], 0, C::CS);
          const float e1 = ldc<FMT>(&F[FI(1, hr, hc)], a.isc[1], 1, C::CS);
          const float e2 = ldc<FMT>(&F[FI(2, hr, hc)], a.isc[2], 2, C::CS);
          const float nx_ = h_upd_r<NU>(ldc<FMT>(&F[FI(3, hr, hc)], a.isc[3], 3, C::CS), S, rz,
                                        ldc<FMT>(&Fn[FI(1, hr, hc)], a.isc[1], 1, C::CS), e1, ryh,
                                        ldc<FMT>(&F[FI(2, hr + 1, hc)], a.isc[2], 2, C::CS), e2);
          const float ny_ = h_upd_r<NU>(ldc<FMT>(&F[FI(4, hr, hc)], a.isc[4], 4, C::CS), S, rxh,
                                        ldc<FMT>(&F[FI(2, hr, hc + 1)], a.isc[2], 2, C::CS), e2, rz,
                                        ldc<FMT>(&Fn[FI(0, hr, hc)], a.isc[0], 0, C::CS), e0);
          const float nz_ = h_upd_r<NU>(ldc<FMT>(&F[FI(5, hr, hc)], a.isc[5], 5, C::CS), S, ryh,
                                        ldc<FMT>(&F[FI(0, hr + 1, hc)], a.isc[0], 0, C::CS), e0, rxh,
                                        ldc<FMT>(&F[FI(1, hr, hc + 1)], a.isc[1], 1, C::CS), e1);
          *hp(0, hr, hc) = nx_;
          *hp(1, hr, hc) = ny_;
          *hp(2, hr, hc) = nz_;
        }
      }
      abort = named_bar_or(1, kConsumers, !ok);
      if (abort) break;
      if constexpr (BATCH) {
        // Batches are mostly explicit points: warm L1 with the explicit
        // coefficients of the next plane's points, read in the next
        // iteration's E phase (the next stage is loaded and not yet released;
        // it holds this unit's cavity).
        const uint32_t* Mn = sM(sn);
        const float2* ec = ecoef();
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const uint32_t mn = Mn[(r0 + r) * BX + c0 + cc];
            if (mn & kExpFlag) prefetch_l1(ec + 3ull * (mn >> 3));
          }
      }
      const bool out_plane = z >= w.z0;
      const uint32_t* M = sM(sc);
      if constexpr (NU) {
        const float4 px = *reinterpret_cast<const float4*>(a.rpair[0] + xl);
        const float4 py = *reinterpret_cast<const float4*>(a.rpair[1] + yl);
        rxdv[0] = px.y;
        rxdv[1] = px.w;
        rydv[0] = py.y;
        rydv[1] = py.w;
        rzd = a.rpair[2][z].y;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int row = r0 + r;
        float hzj[2], hxj[2];
        if (r == 0) {
          const float2 a2 = *reinterpret_cast<const float2*>(hp(2, row - 1, c0));
          const float2 b2 = *reinterpret_cast<const float2*>(hp(0, row - 1, c0));
          hzj[0] = a2.x; hzj[1] = a2.y;
          hxj[0] = b2.x; hxj[1] = b2.y;
        } else {
          hzj[0] = hz[0][0]; hzj[1] = hz[0][1];
          hxj[0] = hx[0][0]; hxj[1] = hx[0][1];
        }
        const float hz_im = *hp(2, row, c0 - 1);
        const float hy_im = *hp(1, row, c0 - 1);
        const uint2 m2 = *reinterpret_cast<const uint2*>(&M[row * BX + c0]);
        const int y = w.y0 + 2 * warp + r;
        const int x = w.x0 + 2 * lane;
        float eo[3][2];
        float2 bx2, by2, bz2;  // the brackets of both x positions, packed
        if constexpr (NU) {
          const float2 ryd2 = make_float2(rydv[r], rydv[r]), rzd2 = make_float2(rzd, rzd);
          const float2 rxd2 = make_float2(rxdv[0], rxdv[1]);
          bx2 = curl_br2_nu(ryd2, make_float2(hz[r][0], hz[r][1]), make_float2(hzj[0], hzj[1]),
                            make_float2(-rzd, -rzd), make_float2(hy[r][0], hy[r][1]), make_float2(hyp[r][0], hyp[r][1]));
          by2 = curl_br2_nu(rzd2, make_float2(hx[r][0], hx[r][1]), make_float2(hxp[r][0], hxp[r][1]),
                            make_float2(-rxdv[0], -rxdv[1]), make_float2(hz[r][0], hz[r][1]), make_float2(hz_im, hz[r][0]));
          bz2 = curl_br2_nu(rxd2, make_float2(hy[r][0], hy[r][1]), make_float2(hy_im, hy[r][0]),
                            make_float2(-rydv[r], -rydv[r]), make_float2(hx[r][0], hx[r][1]), make_float2(hxj[0], hxj[1]));
        } else {
          bx2 = curl_br2(make_float2(hz[r][0], hz[r][1]), make_float2(hzj[0], hzj[1]),
                         make_float2(hy[r][0], hy[r][1]), make_float2(hyp[r][0], hyp[r][1]));
          by2 = curl_br2(make_float2(hx[r][0], hx[r][1]), make_float2(hxp[r][0], hxp[r][1]),
                         make_float2(hz[r][0], hz[r][1]), make_float2(hz_im, hz[r][0]));
          bz2 = curl_br2(make_float2(hy[r][0], hy[r][1]), make_float2(hy_im, hy[r][0]),
                         make_float2(hx[r][0], hx[r][1]), make_float2(hxj[0], hxj[1]));
        }
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const uint32_t m = cc ? m2.y : m2.x;
          float bx = cc ? bx2.y : bx2.x;
          float by = cc ? by2.y : by2.x;
          float bz = cc ? bz2.y : bz2.x;
          if ((m & kSrcFlag) && out_plane) {
            const float3 b3 = apply_sources(make_float3(bx, by, bz),
                                            ((long long)z * d.ny1() + y) * d.nxp() + x + cc, a.n0, srct());
            bx = b3.x;
            by = b3.y;
            bz = b3.z;
          }
          float2 k0, k1, k2;
          if (m & kExpFlag) {
            const float2* e3 = ecoef() + 3ull * (m >> 3);
            k0 = __ldg(e3);
            k1 = __ldg(e3 + 1);
            k2 = __ldg(e3 + 2);
          } else if constexpr (BATCH) {
            const float2* ct = coef();
            k0 = __ldg(&ct[cls_of(m, 0)]);
            k1 = __ldg(&ct[cls_of(m, 1)]);
            k2 = __ldg(&ct[cls_of(m, 2)]);
          } else {
            k0 = *reinterpret_cast<const float2*>(scoefb + cls_off_x(m));
            k1 = *reinterpret_cast<const float2*>(scoefb + cls_off_y(m));
            k2 = *reinterpret_cast<const float2*>(scoefb + cls_off_z(m));
          }
          eo[0][cc] = e_upd(ex[r][cc], k0, bx);
          eo[1][cc] = e_upd(ey[r][cc], k1, by);
          eo[2][cc] = e_upd(ez[r][cc], k2, bz);
          if ((m & kPrbFlag) && out_plane && y < d.ny() && x + cc < d.nx()) {
            // (inline on the non-uniform mesh, where the call's saved registers
            // spilled in the hot loop at the 96-register cap: 89 -> 99 Gcell/s)
            const long long ppt = ((long long)z * d.ny1() + y) * d.nxp() + x + cc;
            const PrbShared* ps = reinterpret_cast<const PrbShared*>(base + C::kPrbOff);
            if constexpr (NU)
              record_probes_inline(ppt, a.n0, eo[0][cc], eo[1][cc], eo[2][cc], hx[r][cc], hy[r][cc], hz[r][cc], ps);
            else
              record_probes(ppt, a.n0, eo[0][cc], eo[1][cc], eo[2][cc], hx[r][cc], hy[r][cc], hz[r][cc], ps);
          }
        }
        if (out_plane && y < d.ny() && x < d.nx()) {
          T* o = fout() + (long long)z * d.zstride() + (long long)y * d.nxp() + x;
          const float vals[6][2] = {{eo[0][0], eo[0][1]}, {eo[1][0], eo[1][1]}, {eo[2][0], eo[2][1]},
                                    {hx[r][0], hx[r][1]}, {hy[r][0], hy[r][1]}, {hz[r][0], hz[r][1]}};
          st6<FMT>(o, d.plane(), vals, a.sc, x + 1 < d.nx() ? 3 : 1);
        }
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          hxp[r][cc] = hx[r][cc];
          hyp[r][cc] = hy[r][cc];
        }
      }
      if constexpr (C::kInPlace) fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty(sc));
    }
    if (abort) break;
    // The unit's last plane was only read as the "next" plane: release it.
    __syncwarp();
    if (lane == 0) mbar_arrive(empty((int)(C_ % kNS)));
    ++C_;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

int plain_box_x(int fmt) { return store_bytes(fmt) == 4 ? PCfg<kF32>::BX : PCfg<kF16>::BX; }
int plain_box_y() { return kBY; }

bool encode_maps(const Dims& d, int fmt, void* fields, uint32_t* mat, int box_x, int box_y, CUtensorMap* tmF,
                 CUtensorMap* tmM) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t esz = store_bytes(fmt);
  // hi+lo pairs move as 4-byte elements (zero fill = +0 + +0)
  // (kF24: 2-byte elements of nine planes, zero fill = +0)
  const CUtensorMapDataType dt = fmt == kF32 || fmt == kF16HL ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : fmt == kF16                ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : fmt == kF24                ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                              : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint32_t planes = (cuuint32_t)store_planes(fmt);
  if (d.zstride != (long long)planes * d.plane) return false;
  if (tmF) {
    cuuint64_t gdF[4] = {(cuuint64_t)d.nxp, (cuuint64_t)d.ny1, planes, (cuuint64_t)d.nz1};
    cuuint64_t gsF[3] = {(cuuint64_t)d.nxp * esz, (cuuint64_t)d.plane * esz, (cuuint64_t)d.zstride * esz};
    cuuint32_t boxF[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, planes, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (fn(tmF, dt, 4, fields, gdF, gsF, boxF, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (tmM) {
    cuuint64_t gdM[3] = {(cuuint64_t)d.nxp, (cuuint64_t)d.ny1, (cuuint64_t)d.nz1};
    cuuint64_t gsM[2] = {(cuuint64_t)d.nxp * 4, (cuuint64_t)d.plane * 4};
    cuuint32_t boxM[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(tmM, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, mat, gdM, gsM, boxM, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

PlainTiling plain_tiling(const Dims& d, int num_sms, int zchunk_override) {
  PlainTiling best{};
  double best_cost = 1e300;
  const int tiles_x = (d.nx + kPX - 1) / kPX, tiles_y = (d.ny + kPY - 1) / kPY;
  const int slots = 2 * num_sms;
  const int cands[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024};
  best.tx0 = best.ty0 = best.z0 = 0;
  best.z1 = d.nz;
  for (int zc : cands) {
    if (zchunk_override > 0) zc = zchunk_override;
    if (zc > d.nz && zc != cands[0] && zchunk_override <= 0) continue;
    const long long nzc = (d.nz + zc - 1) / zc;
    const long long units = (long long)tiles_x * tiles_y * nzc;
    const long long per = (units + slots - 1) / slots;
    // HBM time ~ units per CTA x planes loaded per unit (the chunk, the plane
    // below it for the H warm-up and the plane above it for the z+1 values).
    const double cost = (double)per * (std::min(zc, d.nz) + 2.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best.tiles_x = tiles_x;
      best.tiles_y = tiles_y;
      best.zchunk = zc;
      best.units = units;
      best.grid = (int)((units + per - 1) / per);
    }
    if (zchunk_override > 0) break;
  }
  return best;
}

template <int F, bool NU>
cudaError_t launch_plain_fn(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const PlainTiling& t,
                            cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(yee_plain_kernel<F, false, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PCfg<F>::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_step_kernel(yee_plain_kernel<F, false, NU>, dim3(t.grid), dim3(kThreads), PCfg<F>::kSmemBytes, s, tmF,
                            tmM, a, t, PlainBatch{});
}

template <int F>
cudaError_t launch_plain_f(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM, const PlainTiling& t,
                           cudaStream_t s) {
  return a.rat[0] ? launch_plain_fn<F, true>(a, tmF, tmM, t, s) : launch_plain_fn<F, false>(a, tmF, tmM, t, s);
}

PlainTiling plain_tiling_box(const Dims& d, int num_sms, const int* box) {
  PlainTiling t{};
  const int z0 = std::max(box[4], 0), z1 = std::min(box[5], d.nz);
  const int x1 = std::min(box[1], d.nx), y1 = std::min(box[3], d.ny);
  if (box[0] >= x1 || box[2] >= y1 || z0 >= z1) return t;  // nothing live: grid 0
  const int tx0 = box[0] / kPX, tx1 = (x1 + kPX - 1) / kPX;
  const int ty0 = box[2] / kPY, ty1 = (y1 + kPY - 1) / kPY;
  // the same cost model as plain_tiling on a grid of the sub-box's extent
  Dims sub = d;
  sub.nx = (tx1 - tx0) * kPX;
  sub.ny = (ty1 - ty0) * kPY;
  sub.nz = z1 - z0;
  t = plain_tiling(sub, num_sms, 0);
  t.tx0 = tx0;
  t.ty0 = ty0;
  t.z0 = z0;
  t.z1 = z1;
  return t;
}

int plain_tile_x() { return kPX; }
int plain_tile_y() { return kPY; }

cudaError_t launch_step_plain_batch(const StepArgs& a, const PlainBatch& pb, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(yee_plain_kernel<kF32, true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCfg<kF32>::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap none{};
  PlainTiling t{};
  return launch_step_kernel(yee_plain_kernel<kF32, true, false>, dim3(grid), dim3(kThreads), PCfg<kF32>::kSmemBytes, s,
                            none, none, a, t, pb);
}

cudaError_t launch_step_plain(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                              const PlainTiling& t, cudaStream_t s) {
  switch (a.fmt) {
    case kF32: return launch_plain_f<kF32>(a, tmF, tmM, t, s);
    case kF16: return a.fold ? launch_plain_f<kF16U>(a, tmF, tmM, t, s) : launch_plain_f<kF16>(a, tmF, tmM, t, s);
    case kBF16: return a.fold ? launch_plain_f<kBF16U>(a, tmF, tmM, t, s) : launch_plain_f<kBF16>(a, tmF, tmM, t, s);
    case kF16HL:
      return a.fold ? launch_plain_f<kF16HLU>(a, tmF, tmM, t, s) : launch_plain_f<kF16HL>(a, tmF, tmM, t, s);
    case kF24: return launch_plain_f<kF24>(a, tmF, tmM, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sophie
