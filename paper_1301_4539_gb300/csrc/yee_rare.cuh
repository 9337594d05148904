// Rare paths of the step kernels (source currents, probe samples), kept out
// of line so that the unrolled update loops stay small in the instruction
// cache. Both only run for index points whose material word carries the
// source or probe flag.
#pragma once

#include "sophie_internal.h"

namespace sophie {

// Sec. 3.3: a current added to Ampere's equation. Every source on index point
// pt adds amp*w(t^{n+1/2}) (tabulated per step) to its component's curl
// bracket, in the order the sources were added.
static __device__ __noinline__ float3 apply_sources(float3 b, long long pt, long long nstep,
                                                    const SrcTable* src) {
  if (src->nbig > 0) {
    // the first source at or after pt (binary search), then those on pt
    int lo = 0, hi = src->nbig;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (src->bpos[mid] < pt) lo = mid + 1;
      else hi = mid;
    }
    for (int q = lo; q < src->nbig && src->bpos[q] == pt; ++q) {
      float v = src->val[(long long)src->brow[q] * src->cap + nstep];
      if (src->vmul_on) v = __fmul_rn(v, src->vmul);
      const int c = src->bcomp[q];
      if (c == 0) b.x = __fadd_rn(b.x, v);
      else if (c == 1) b.y = __fadd_rn(b.y, v);
      else b.z = __fadd_rn(b.z, v);
    }
    return b;
  }
  for (int q = 0; q < src->n; ++q) {
    if (src->pos[q] != pt) continue;
    float v = src->val[(long long)q * src->cap + nstep];
    if (src->vmul_on) v = __fmul_rn(v, src->vmul);
    if (src->comp[q] == 0) b.x = __fadd_rn(b.x, v);
    else if (src->comp[q] == 1) b.y = __fadd_rn(b.y, v);
    else b.z = __fadd_rn(b.z, v);
  }
  return b;
}

// The probe table in shared memory: the kernels copy it there at start, so
// the search below reads shared memory rather than the kernel parameter
// through a generic pointer, whose indexed loads were slow enough for one
// probe search to delay its CTA, and with it the launch, by a few
// microseconds (16 probes: 2 % of a 256^3 step).
struct PrbShared {
  long long pos[kMaxProbes];
  int comp[kMaxProbes];
  float* buf;
  int n, cap, pmul_on;
  float pmul;
};

__device__ __forceinline__ void load_probes(PrbShared* s, const PrbTable& prb, int tid, int nthreads) {
  for (int q = tid; q < prb.n; q += nthreads) {
    s->pos[q] = prb.pos[q];
    s->comp[q] = prb.comp[q];
  }
  if (tid == 0) {
    s->buf = prb.buf;
    s->n = prb.n;
    s->cap = prb.cap;
    s->pmul_on = prb.pmul_on;
    s->pmul = prb.pmul;
  }
}

// Sec. 3.4 pin-point outputs: sample nstep of every probe on index point pt.
__device__ __forceinline__ void record_probes_inline(long long pt, long long nstep, float ex, float ey, float ez,
                                                     float hx, float hy, float hz, const PrbShared* s) {
  for (int q = 0; q < s->n; ++q) {
    if (s->pos[q] != pt) continue;
    const int c = s->comp[q];
    float v = c == 0 ? ex : c == 1 ? ey : c == 2 ? ez : c == 3 ? hx : c == 4 ? hy : hz;
    if (s->pmul_on) v = __fmul_rn(v, s->pmul);
    s->buf[(long long)q * s->cap + nstep] = v;
  }
}
// The same out of line (a call the kernels make only at flagged points),
// which keeps most kernels' register allocation of the hot loop unchanged.
static __device__ __noinline__ void record_probes(long long pt, long long nstep, float ex, float ey, float ez,
                                                  float hx, float hy, float hz, const PrbShared* s) {
  record_probes_inline(pt, nstep, ex, ey, ez, hx, hy, hz, s);
}

}  // namespace sophie
