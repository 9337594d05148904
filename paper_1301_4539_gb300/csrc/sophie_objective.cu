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

extern "C" {

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
  while ((int)t.ck.size() < nseg) {
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
  for (int sg = 0; sg < nseg; ++sg) {
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
  const int ext[3][3] = {{ni, nj + 1, nk + 1}, {ni + 1, nj, nk + 1}, {ni + 1, nj + 1, nk}};
  std::vector<int> map[3];
  std::vector<int> hcomp;
  std::vector<long long> hpt;
  std::vector<double> dcb, dca;
  std::vector<float> cbf;  // the float Cb the step kernels use on each design edge
  for (int c = 0; c < 3; ++c) {
    map[c].assign((size_t)ext[c][0] * ext[c][1] * ext[c][2], -1);
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
          map[c][((size_t)kk * ext[c][1] + jj) * ext[c][0] + ii] = (int)hpt.size();
          cbf.push_back(cb_edge);
          hcomp.push_back(c);
          hpt.push_back(pt);
          dcb.push_back(-cb / (e * (1.0 + beta)));
          dca.push_back(2.0 * beta / (e * (1.0 + beta) * (1.0 + beta)));
        }
  }
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
  int lc = 0;
  const int nseg = (t.N + t.K - 1) / t.K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const long long ns = t.n0 + (long long)sg * t.K;
    const int len = std::min(t.K, t.N - sg * t.K);
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
    // Reverse sweep over the segment.
    for (int m = len - 1; m >= 0; --m) {
      const long long n = ns + m;
      float* l = static_cast<float*>(t.L[lc]);
      cudaError_t e = launch_add_objective(l, d, t.comp, t.pt, t.samples + (n - t.n0), two_dt, g->stream);
      if (e == cudaSuccess)
        e = launch_grad_accum(l, d, t.ecomp, t.ept, nedge, t.etr + (size_t)m * nedge, t.ctr + (size_t)m * nedge,
                              t.gcb, t.gca, g->stream);
      if (e == cudaSuccess) {
        StepArgs a = make_step_args(g);
        a.fin = t.L[lc];
        a.fout = t.L[1 - lc];
        a.n0 = n;
        a.prb.n = 0;
        a.src.n = 0;
        cudaEvent_t ea = g->prof ? prof_event(g) : nullptr, eb = g->prof ? prof_event(g) : nullptr;
        if (ea) cudaEventRecord(ea, g->stream);
        e = direct ? launch_adj_step(a, g->stream) : launch_step_plain(a, t.tmL[lc], t.tmRM, g->ptile, g->stream);
        if (eb) {
          cudaEventRecord(eb, g->stream);
          g->prof_live.push_back({SOPHIE_KERNEL_ADJOINT, ea, eb});
        }
      }
      if (e != cudaSuccess) return fail(SOPHIE_ECUDA, "adjoint launch failed: %s", cudaGetErrorString(e));
      g->launches += nedge ? 3 : 2;
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
