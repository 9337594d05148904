// Host runtime of the differentiation form (sophie_objective_* in
// include/sophie.h): the recorded forward pass with checkpoints and the
// reverse sweep that accumulates dJ/d eps_r on a box of design cells. The
// kernels are the forward step kernels and those of yee_adjoint.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "grid_state.h"

using namespace sophie;
using namespace sophie::grid;

namespace {

// The design edges of a box of cells: the interior, non-conducting edges of
// its cells, with the float Cb the kernels use and the derivatives of the
// edge's (Cb, Ca) with respect to its mean eps (box index -> edge index map).
struct DesignEdges {
  int ext[3][3];
  std::vector<int> map[3];
  std::vector<int> comp;
  std::vector<long long> pt;
  std::vector<double> dcb, dca;
  std::vector<float> cbf;
};

void design_edges(const sophie_grid* g, int i0, int j0, int k0, int ni, int nj, int nk, DesignEdges& de) {
  const Dims& d = g->d;
  const int ext[3][3] = {{ni, nj + 1, nk + 1}, {ni + 1, nj, nk + 1}, {ni + 1, nj + 1, nk}};
  memcpy(de.ext, ext, sizeof ext);
  for (int c = 0; c < 3; ++c) {
    de.map[c].assign((size_t)ext[c][0] * ext[c][1] * ext[c][2], -1);
    for (int kk = 0; kk < ext[c][2]; ++kk)
      for (int jj = 0; jj < ext[c][1]; ++jj)
        for (int ii = 0; ii < ext[c][0]; ++ii) {
          const int i = i0 + ii, j = j0 + jj, k = k0 + kk;
          if (!e_edge_interior(d, c, i, j, k)) continue;
          const long long pt = point_index(d, i, j, k);
          const uint32_t w = g->mat_host[pt];
          const float cb_edge = (w & kExpFlag) ? g->ecoef_h[3 * (size_t)(w >> 3) + c].y : g->coef_h[cls_of(w, c)].y;
          if (cb_edge == 0.f) continue;  // edge of a conducting cell: no eps dependence
          double e, sg;
          if (w & kExpFlag) {
            const size_t q = w >> 3;
            e = g->eeps_h[3 * q + c];
            sg = g->esig_h[3 * q + c];
          } else {
            e = g->eps_h[cls_of(w, c)];
            sg = g->sig_h[cls_of(w, c)];
          }
          // Cb = (S/e)/(1+beta), Ca = (1-beta)/(1+beta), beta = sigma dt/(2 eps0 e)
          const double beta = (sg * g->dt) / (2.0 * kEps0 * e);
          const double cb = (g->S64 / e) / (1.0 + beta);
          de.map[c][((size_t)kk * ext[c][1] + jj) * ext[c][0] + ii] = (int)de.pt.size();
          de.cbf.push_back(cb_edge);
          de.comp.push_back(c);
          de.pt.push_back(pt);
          de.dcb.push_back(-cb / (e * (1.0 + beta)));
          de.dca.push_back(2.0 * beta / (e * (1.0 + beta) * (1.0 + beta)));
        }
  }
}

bool box_ok(const Dims& d, int i0, int j0, int k0, int ni, int nj, int nk) {
  return ni >= 1 && nj >= 1 && nk >= 1 && i0 >= 0 && j0 >= 0 && k0 >= 0 && i0 + ni <= d.nx && j0 + nj <= d.ny &&
         k0 + nk <= d.nz;
}

// Grow device array *p to hold `bytes` (contents not kept).
bool grow_dev(void** p, size_t bytes) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (dev_malloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

int sophie_objective_set_design(sophie_grid* g, int i0, int j0, int k0, int ni, int nj, int nk) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  if (ni == 0 && nj == 0 && nk == 0) {
    g->design_set = false;
    return SOPHIE_OK;
  }
  if (!box_ok(g->d, i0, j0, k0, ni, nj, nk)) return fail(SOPHIE_EINVAL, "design box outside the grid's cells");
  const int b[6] = {i0, j0, k0, ni, nj, nk};
  memcpy(g->design, b, sizeof b);
  g->design_set = true;
  return SOPHIE_OK;
}

int sophie_objective_release(sophie_grid* g) {
  if (!g) return fail(SOPHIE_EINVAL, "NULL grid");
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  free_tape(g->tape);
  return SOPHIE_OK;
}

int sophie_objective_forward(sophie_grid* g, int nsteps, int comp, int i, int j, int k, int checkpoint_every,
                             double* J) {
  if (!g || !J) return fail(SOPHIE_EINVAL, "NULL argument");
  if (nsteps < 1) return fail(SOPHIE_EINVAL, "nsteps must be >= 1");
  if (checkpoint_every < 0) return fail(SOPHIE_EINVAL, "checkpoint_every must be >= 0");
  if (comp < 0 || comp > 5 || !comp_valid(g->d, comp, i, j, k))
    return fail(SOPHIE_EINVAL, "objective point (%d,%d,%d) outside comp %d's range", i, j, k, comp);
  if (i == g->d.nx || j == g->d.ny || k == g->d.nz)
    return fail(SOPHIE_EINVAL, "objective point on a plane no step updates");
  if (g->fmt != kF32) return fail(SOPHIE_ENOTSUP, "gradients need float field storage");
  if (g->rat) return fail(SOPHIE_ENOTSUP, "gradients need a uniform mesh");
  if ((int)g->prb.size() >= kMaxProbes) return fail(SOPHIE_ENOTSUP, "all %d probe slots are in use", kMaxProbes);
  Tape& t = g->tape;
  t.valid = false;
  const int K = checkpoint_every == 0 ? 50 : checkpoint_every;
  const int nseg = (nsteps + K - 1) / K;
  const Dims& d = g->d;
  const size_t fbytes = (size_t)d.zstride * d.nz1 * 4;
  int rc = ensure_capacity(g, g->n + nsteps);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  // Traced record: with a registered design box whose traces fit (both
  // [nsteps][nedge] float arrays within a quarter of the free device memory
  // and 8 GB), the forward pass runs one step per launch and gathers e^n and
  // the bracket on the design edges after every step; the reverse sweep then
  // needs neither checkpoints nor recomputation.
  t.traced = false;
  bool trace = false;
  int nedge = 0;
  if (g->design_set) {
    DesignEdges de;
    design_edges(g, g->design[0], g->design[1], g->design[2], g->design[3], g->design[4], g->design[5], de);
    nedge = (int)de.pt.size();
    const size_t bytes = (size_t)nedge * nsteps * 4;
    size_t fr = 0, tot = 0;
    if (nedge > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && 2 * bytes <= std::min<size_t>(fr / 4, 8ull << 30)) {
      trace = grow_dev((void**)&t.etr_all, bytes) && grow_dev((void**)&t.ctr_all, bytes);
      if (trace && nedge > t.edge_cap) {
        trace = grow_dev((void**)&t.ecomp, (size_t)nedge * 4) && grow_dev((void**)&t.ept, (size_t)nedge * 8) &&
                grow_dev((void**)&t.gcb, (size_t)nedge * 8) && grow_dev((void**)&t.gca, (size_t)nedge * 8);
        t.edge_cap = trace ? nedge : 0;
        t.tr_cap = 0;
      }
      if (trace) {
        CUDA_TRY(cudaMemcpyAsync(t.ecomp, de.comp.data(), (size_t)nedge * 4, cudaMemcpyHostToDevice, g->stream));
        CUDA_TRY(cudaMemcpyAsync(t.ept, de.pt.data(), (size_t)nedge * 8, cudaMemcpyHostToDevice, g->stream));
      } else {
        if (t.etr_all) cudaFree(t.etr_all);
        if (t.ctr_all) cudaFree(t.ctr_all);
        t.etr_all = t.ctr_all = nullptr;
      }
    }
  }
  while (!trace && (int)t.ck.size() < nseg) {
    void* p = nullptr;
    if (dev_malloc((void**)&p, fbytes) != cudaSuccess) {
      cudaGetLastError();
      free_tape(t);
      return fail(SOPHIE_ENOMEM, "checkpoint allocation (%d x %zu bytes) failed", nseg, fbytes);
    }
    t.ck.push_back(p);
  }
  if (t.samples_cap < nsteps) {
    if (t.samples) cudaFree(t.samples);
    t.samples = nullptr;
    t.samples_cap = 0;
    if (dev_malloc((void**)&t.samples, (size_t)nsteps * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(SOPHIE_ENOMEM, "objective sample buffer allocation failed");
    }
    t.samples_cap = nsteps;
  }
  t.comp = comp;
  t.pt = point_index(d, i, j, k);
  t.n0 = g->n;
  t.N = nsteps;
  t.K = K;
  if (launch_or_flag(g->mat, t.pt, kPrbFlag, g->stream) != cudaSuccess)
    return fail(SOPHIE_ECUDA, "flag launch failed");
  g->launches++;
  const int slot = (int)g->prb.size();
  g->obj_rec = true;
  for (int n = 0; trace && n < nsteps; ++n) {
    rc = sophie_step(g, 1);
    if (rc) {
      g->obj_rec = false;
      return rc;
    }
    StepArgs a = make_step_args(g);
    a.fin = g->F[1 - g->cur];  // the state before the step
    a.fout = g->F[g->cur];     // after it
    a.n0 = g->n - 1;
    const cudaError_t e = launch_gather(a, t.ecomp, t.ept, nedge, t.etr_all + (size_t)n * nedge,
                                        t.ctr_all + (size_t)n * nedge, g->stream);
    if (e != cudaSuccess) {
      g->obj_rec = false;
      return fail(SOPHIE_ECUDA, "gather launch failed: %s", cudaGetErrorString(e));
    }
    g->launches++;
  }
  for (int sg = 0; !trace && sg < nseg; ++sg) {
    const cudaError_t e = cudaMemcpyAsync(t.ck[sg], g->F[g->cur], fbytes, cudaMemcpyDeviceToDevice, g->stream);
    if (e != cudaSuccess) {
      g->obj_rec = false;
      return fail(SOPHIE_ECUDA, "checkpoint copy failed: %s", cudaGetErrorString(e));
    }
    rc = sophie_step(g, std::min(K, nsteps - sg * K));
    if (rc) {
      g->obj_rec = false;
      return rc;
    }
  }
  g->obj_rec = false;
  float* slot_p = g->pbuf + (size_t)slot * g->pcap + t.n0;
  CUDA_TRY(cudaMemcpyAsync(t.samples, slot_p, (size_t)nsteps * 4, cudaMemcpyDeviceToDevice, g->stream));
  CUDA_TRY(cudaMemsetAsync(slot_p, 0, (size_t)nsteps * 4, g->stream));
  std::vector<float> f((size_t)nsteps);
  CUDA_TRY(cudaMemcpyAsync(f.data(), t.samples, (size_t)nsteps * 4, cudaMemcpyDeviceToHost, g->stream));
  rc = check_err_word(g);
  if (rc) return rc;
  double acc = 0.0;
  for (int n = 0; n < nsteps; ++n) acc += (double)f[n] * (double)f[n];
  *J = g->dt * acc;
  if (!std::isfinite(*J)) return fail(SOPHIE_ENONFINITE, "objective is not finite");
  t.valid = true;
  t.gen = g->gen;
  t.traced = trace;
  t.tnedge = nedge;
  if (trace) memcpy(t.tbox, g->design, sizeof t.tbox);
  return SOPHIE_OK;
}

int sophie_objective_grad_eps(sophie_grid* g, int i0, int j0, int k0, int ni, int nj, int nk, double* grad) {
  if (!g || !grad) return fail(SOPHIE_EINVAL, "NULL argument");
  Tape& t = g->tape;
  if (!t.valid || t.gen != g->gen)
    return fail(SOPHIE_EINVAL, "no objective recorded since the last change of the grid");
  const Dims& d = g->d;
  if (ni < 1 || nj < 1 || nk < 1 || i0 < 0 || j0 < 0 || k0 < 0 || i0 + ni > d.nx || j0 + nj > d.ny ||
      k0 + nk > d.nz)
    return fail(SOPHIE_EINVAL, "design box outside the grid's cells");
  // Design edges: interior edges of the box's cells; box index -> edge index.
  DesignEdges de;
  design_edges(g, i0, j0, k0, ni, nj, nk, de);
  const int(&ext)[3][3] = de.ext;
  const std::vector<int>* map = de.map;
  const std::vector<int>& hcomp = de.comp;
  const std::vector<long long>& hpt = de.pt;
  const std::vector<double>& dcb = de.dcb;
  const std::vector<double>& dca = de.dca;
  const std::vector<float>& cbf = de.cbf;  // the float Cb the step kernels use on each design edge
  const int nedge = (int)hpt.size();
  const size_t fbytes = (size_t)d.zstride * d.nz1 * 4;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  auto grow = [&](void** p, size_t bytes) -> bool {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (dev_malloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    return true;
  };
  if (!t.R[0]) {
    for (int b = 0; b < 2; ++b)
      if (!grow(&t.R[b], fbytes) || !grow(&t.L[b], fbytes))
        return fail(SOPHIE_ENOMEM, "adjoint workspace allocation failed");
    // Wall and padding entries are never written by the step kernels: they
    // must start (and stay) zero in both recompute buffers.
    CUDA_TRY(cudaMemsetAsync(t.R[0], 0, fbytes, g->stream));
    CUDA_TRY(cudaMemsetAsync(t.R[1], 0, fbytes, g->stream));
    for (int b = 0; b < 2; ++b)
      if (!encode_maps(d, kF32, t.R[b], g->mat, plain_box_x(kF32), plain_box_y(), &t.tmR[b], &t.tmRM) ||
          !encode_maps(d, kF32, t.L[b], nullptr, plain_box_x(kF32), plain_box_y(), &t.tmL[b], nullptr))
        return fail(SOPHIE_ECUDA, "cuTensorMapEncodeTiled failed");
  }
  if (nedge > t.edge_cap) {
    if (!grow((void**)&t.ecomp, (size_t)nedge * 4) || !grow((void**)&t.ept, (size_t)nedge * 8) ||
        !grow((void**)&t.gcb, (size_t)nedge * 8) || !grow((void**)&t.gca, (size_t)nedge * 8)) {
      t.edge_cap = 0;
      return fail(SOPHIE_ENOMEM, "design edge table allocation failed");
    }
    t.edge_cap = nedge;
    t.tr_cap = 0;
  }
  if ((long long)nedge * t.K > t.tr_cap) {
    if (!grow((void**)&t.etr, (size_t)nedge * t.K * 4) || !grow((void**)&t.ctr, (size_t)nedge * t.K * 4)) {
      t.tr_cap = 0;
      return fail(SOPHIE_ENOMEM, "design edge trace allocation failed");
    }
    t.tr_cap = nedge * t.K;
  }
  if (nedge) {
    CUDA_TRY(cudaMemcpyAsync(t.ecomp, hcomp.data(), (size_t)nedge * 4, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemcpyAsync(t.ept, hpt.data(), (size_t)nedge * 8, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemsetAsync(t.gcb, 0, (size_t)nedge * 8, g->stream));
    CUDA_TRY(cudaMemsetAsync(t.gca, 0, (size_t)nedge * 8, g->stream));
  }
  CUDA_TRY(cudaMemsetAsync(t.L[0], 0, fbytes, g->stream));
  CUDA_TRY(cudaMemsetAsync(t.L[1], 0, fbytes, g->stream));
  // Reverse sweep. Default form: in the variables u = Cb * l_e, mu = -S * l_h
  // the reverse step is the forward step itself with the same coefficients
  // (mu' = mu + S A u, u' = Ca u + Cb B mu'), so it runs on the forward step
  // kernel with sources and probes off; the objective's direct term enters as
  // u += Cb 2dt f (E component) or mu += -S 2dt f (H component), and the
  // accumulated sums of u * (bracket) and u * e are divided by Cb at the end.
  // SOPHIE_ADJOINT=direct runs the literal transposed step (yee_adjoint.cu)
  // on (l_e, l_h) instead (a cross-check; same gradient up to rounding).
  const char* am = getenv("SOPHIE_ADJOINT");
  const bool direct = am && strcmp(am, "direct") == 0;
  double obj_scale = 1.0;
  if (!direct) {
    if (t.comp < 3) {
      const uint32_t w = g->mat_host[t.pt];
      obj_scale = (w & kExpFlag) ? g->ecoef_h[3 * (size_t)(w >> 3) + t.comp].y : g->coef_h[cls_of(w, t.comp)].y;
      if (!e_edge_interior(d, t.comp, (int)(t.pt % d.nxp), (int)(t.pt / d.nxp % d.ny1), (int)(t.pt / d.plane)))
        obj_scale = 0.0;
    } else {
      obj_scale = -(double)g->S32;
    }
  }
  const double two_dt = 2.0 * g->dt * obj_scale;
  // the design edge on the objective's component and point, if any
  int t_obj = -1;
  for (int q = 0; q < nedge && t.comp < 3; ++q)
    if (hpt[q] == t.pt && hcomp[q] == t.comp) t_obj = q;
  int lc = 0;
  const int nseg = (t.N + t.K - 1) / t.K;
  // A traced record of this box: the traces of every step are on the device
  // already (gathered by the forward pass), so the reverse sweep runs as one
  // segment of all N steps with no recomputation.
  const int b6[6] = {i0, j0, k0, ni, nj, nk};
  const bool traced = t.traced && nedge == t.tnedge && memcmp(b6, t.tbox, sizeof b6) == 0;
  if (t.traced && !traced)  // a traced record keeps no checkpoints
    return fail(SOPHIE_EINVAL, "the objective record traced another design box; record again for this box");
  for (int sg = traced ? 0 : nseg - 1; sg >= 0; --sg) {
    const long long ns = traced ? t.n0 : t.n0 + (long long)sg * t.K;
    const int len = traced ? t.N : std::min(t.K, t.N - sg * t.K);
    float* const etr = traced ? t.etr_all : t.etr;
    float* const ctr = traced ? t.ctr_all : t.ctr;
    if (!traced) {
    // Recompute the segment from its checkpoint, keeping the design-edge values.
    CUDA_TRY(cudaMemcpyAsync(t.R[0], t.ck[sg], fbytes, cudaMemcpyDeviceToDevice, g->stream));
    for (int m = 0; m < len; ++m) {
      StepArgs a = make_step_args(g);
      a.fin = t.R[m & 1];
      a.fout = t.R[(m + 1) & 1];
      a.n0 = ns + m;
      a.prb.n = 0;
      cudaEvent_t ea = g->prof ? prof_event(g) : nullptr, eb = g->prof ? prof_event(g) : nullptr;
      if (ea) cudaEventRecord(ea, g->stream);
      cudaError_t e = launch_step_plain(a, t.tmR[m & 1], t.tmRM, g->ptile, g->stream);
      if (eb) {
        cudaEventRecord(eb, g->stream);
        g->prof_live.push_back({SOPHIE_KERNEL_PLAIN, ea, eb});
      }
      if (e == cudaSuccess)
        e = launch_gather(a, t.ecomp, t.ept, nedge, t.etr + (size_t)m * nedge, t.ctr + (size_t)m * nedge, g->stream);
      if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "recompute launch failed: %s", cudaGetErrorString(e));
      g->launches += nedge ? 2 : 1;
    }
    if (g->prof_live.size() > 20000) {
      int rc = prof_drain(g);
      if (rc) return rc;
    }
    }  // recompute
    // Reverse sweep over the segment.
    for (int m = len - 1; m >= 0; --m) {
      const long long n = ns + m;
      float* l = static_cast<float*>(t.L[lc]);
      cudaError_t e = launch_objective_grad_accum(l, d, t.comp, t.pt, t.samples + (n - t.n0), two_dt, t_obj, t.ecomp,
                                                  t.ept, nedge, etr + (size_t)m * nedge, ctr + (size_t)m * nedge,
                                                  t.gcb, t.gca, g->stream);
      if (e == cudaSuccess) {
        StepArgs a = make_step_args(g);
        a.fin = t.L[lc];
        a.fout = t.L[1 - lc];
        a.n0 = n;
        a.prb.n = 0;
        a.src.n = 0;
        a.src.nbig = 0;  // (the many-source table too: the reverse steps take no source)
        cudaEvent_t ea = g->prof ? prof_event(g) : nullptr, eb = g->prof ? prof_event(g) : nullptr;
        if (ea) cudaEventRecord(ea, g->stream);
        e = direct ? launch_adj_step(a, g->stream) : launch_step_plain(a, t.tmL[lc], t.tmRM, g->ptile, g->stream);
        if (eb) {
          cudaEventRecord(eb, g->stream);
          g->prof_live.push_back({SOPHIE_KERNEL_ADJOINT, ea, eb});
        }
      }
      if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "adjoint launch failed: %s", cudaGetErrorString(e));
      g->launches += 2;
      lc = 1 - lc;
    }
  }
  std::vector<double> gcb((size_t)nedge), gca((size_t)nedge);
  if (nedge) {
    CUDA_TRY(cudaMemcpyAsync(gcb.data(), t.gcb, (size_t)nedge * 8, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaMemcpyAsync(gca.data(), t.gca, (size_t)nedge * 8, cudaMemcpyDeviceToHost, g->stream));
  }
  int rc = check_err_word(g);
  if (rc) return rc;
  // Chain rule to cells: eps_r(edge) is the mean of its four cells.
  for (int kk = 0; kk < nk; ++kk)
    for (int jj = 0; jj < nj; ++jj)
      for (int ii = 0; ii < ni; ++ii) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c)
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
              const int ei = ii + (c == 0 ? 0 : a);
              const int ej = jj + (c == 0 ? a : c == 1 ? 0 : b);
              const int ek = kk + (c == 2 ? 0 : b);
              const int q = map[c][((size_t)ek * ext[c][1] + ej) * ext[c][0] + ei];
              if (q < 0) continue;
              // sums of u * (...) = Cb * sums of l_e * (...) in the default form
              const double un = direct ? 1.0 : (double)cbf[q];
              acc += 0.25 * (gcb[q] * dcb[q] + gca[q] * dca[q]) / un;
            }
        grad[((size_t)kk * nj + jj) * ni + ii] = acc;
      }
  return SOPHIE_OK;
}

}  // extern "C"
