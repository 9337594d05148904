/*
 * Plain CPU reference of the gradient of a probe objective with respect to
 * per-cell eps_r, by reverse-mode differentiation of the double-precision
 * leapfrog of yee_oracle.c (Sec. 2.1 scheme; the paper itself has no adjoint).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA
 * path.
 *
 * Objective over the nsteps steps n = 0 .. nsteps-1 taken from the given state:
 *   J = dt * sum_{n=1..nsteps} (f^n)^2,  f^n = component pcomp at (pi,pj,pk)
 *   after step n-1 (the value the probes of oracle_step record).
 * One step, from yee_oracle_body.h:
 *   h' = h + S * A e            A = H-update bracket over the faces it updates
 *   e' = Ca e + Cb (B h' + s)   on interior edges; wall edges are not written
 * Reverse sweep, n = nsteps-1 down to 0, with (le, lh) = dJ/d(e^{n+1}, h^{n+1/2}):
 *   le[probe] += 2 dt f^{n+1}
 *   dJ/dCb(edge) += le * (B h^{n+1/2} + s),   dJ/dCa(edge) += le * e^n
 *   reverse of the E half: for each interior edge, w = Cb*le is scattered into
 *     lh through the transpose of that edge's bracket row, then le = Ca*le;
 *   reverse of the H half: for each updated face, S*lh is scattered into le
 *     through the transpose of that face's bracket row.
 * The transposes are formed literally (scatter of each row), without using
 * the antisymmetry of the two brackets.
 * Chain to cells: the edge material is the 4-cell mean (Sec. 2.1 reading of
 * yee_oracle_body.h), so d eps_r(edge) / d eps_r(cell) = 1/4 for the four
 * cells around the edge; with beta = sigma dt / (2 eps0 eps_r):
 *   dCb/deps_r = -Cb / (eps_r (1 + beta)),  dCa/deps_r = 2 beta / (eps_r (1 + beta)^2).
 * Only interior edges carry eps-dependent coefficients.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define C0 299792458.0
#define EPS0 8.8541878128e-12

void oracle_coefs_f64(int nx, int ny, int nz, double dx, double dt,
                      const float *eps_cell, const float *sig_cell,
                      double *cax, double *cbx, double *cay, double *cby, double *caz, double *cbz,
                      double *epsx, double *epsy, double *epsz);
void oracle_step_f64(int nx, int ny, int nz, double S,
                     double *ex, double *ey, double *ez, double *hx, double *hy, double *hz,
                     const double *cax, const double *cbx, const double *cay,
                     const double *cby, const double *caz, const double *cbz,
                     int nsrc, const int *src, const double *sval, long sstride,
                     int nprb, const int *prb, double *pout, long pstride, int nsteps);

static int interior(int nx, int ny, int nz, int c, int i, int j, int k)
{
    if (c == 0) return i >= 0 && i < nx && j >= 1 && j < ny && k >= 1 && k < nz;
    if (c == 1) return i >= 1 && i < nx && j >= 0 && j < ny && k >= 1 && k < nz;
    return i >= 1 && i < nx && j >= 1 && j < ny && k >= 0 && k < nz;
}

/*
 * Gradient of J with respect to eps_r of each listed cell (cells: ncells x
 * {i,j,k}); grad[q] receives dJ/d eps_r(cell q). The six field arrays hold
 * the initial state and are advanced by nsteps steps in place. sval holds
 * nsrc x nsteps source values (row stride nsteps). Returns J; returns NaN if
 * memory runs out.
 */
double oracle_grad_f64(int nx, int ny, int nz, double dx, double dt,
                       const float *eps_cell, const float *sig_cell,
                       double *ex, double *ey, double *ez, double *hx, double *hy, double *hz,
                       int nsrc, const int *src, const double *sval,
                       int pcomp, int pi, int pj, int pk, int nsteps,
                       int ncells, const int *cells, double *grad)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    const long npt = sz * (nz + 1);
    const double S = C0 * dt / dx;
    const int nedge = 12 * ncells;
    double *co = malloc(6 * npt * sizeof(double));
    double *lam = calloc(6 * npt, sizeof(double));
    double *f = malloc((size_t)(nsteps + 1) * sizeof(double));
    double *tr_e = malloc((size_t)nsteps * nedge * sizeof(double) + 1);
    double *tr_c = malloc((size_t)nsteps * nedge * sizeof(double) + 1);
    double *gcb = calloc((size_t)nedge + 1, sizeof(double));
    double *gca = calloc((size_t)nedge + 1, sizeof(double));
    int *ec = malloc((size_t)nedge * 4 * sizeof(int) + 1);
    long *ep = malloc((size_t)nedge * sizeof(long) + 1);
    double J = 0.0;
    if (!co || !lam || !f || !tr_e || !tr_c || !gcb || !gca || !ec || !ep) {
        J = NAN;
        goto done;
    }
    oracle_coefs_f64(nx, ny, nz, dx, dt, eps_cell, sig_cell,
                     co, co + npt, co + 2 * npt, co + 3 * npt, co + 4 * npt, co + 5 * npt,
                     NULL, NULL, NULL);
    double *fld[6] = {ex, ey, ez, hx, hy, hz};
    const double *ca[3] = {co, co + 2 * npt, co + 4 * npt};
    const double *cb[3] = {co + npt, co + 3 * npt, co + 5 * npt};
    double *le[3] = {lam, lam + npt, lam + 2 * npt};
    double *lx = lam + 3 * npt, *ly = lam + 4 * npt, *lz = lam + 5 * npt;

    /* The twelve edges of each listed cell: offsets (d1, d2) in the two
     * directions transverse to the edge. */
    for (int q = 0; q < ncells; ++q) {
        const int i = cells[3 * q], j = cells[3 * q + 1], k = cells[3 * q + 2];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    int *e = ec + 4 * (12 * q + 4 * c + 2 * a + b);
                    e[0] = c;
                    e[1] = i + (c == 0 ? 0 : a);
                    e[2] = j + (c == 0 ? a : c == 1 ? 0 : b);
                    e[3] = k + (c == 2 ? 0 : b);
                    ep[12 * q + 4 * c + 2 * a + b] = e[3] * sz + e[2] * sy + e[1];
                }
    }

    /* Forward: one pinned oracle step at a time, keeping e^n and the step's
     * bracket B h^{n+1/2} + s on the listed edges, and the objective samples. */
    const int prb[4] = {pcomp, pi, pj, pk};
    f[0] = 0.0;
    for (int n = 0; n < nsteps; ++n) {
        for (int t = 0; t < nedge; ++t) tr_e[(size_t)n * nedge + t] = fld[ec[4 * t]][ep[t]];
        oracle_step_f64(nx, ny, nz, S, ex, ey, ez, hx, hy, hz, co, co + npt, co + 2 * npt,
                        co + 3 * npt, co + 4 * npt, co + 5 * npt, nsrc, src, sval + n, nsteps,
                        1, prb, f + n + 1, 1, 1);
        for (int t = 0; t < nedge; ++t) {
            const long p = ep[t];
            double br = 0.0;
            if (!interior(nx, ny, nz, ec[4 * t], ec[4 * t + 1], ec[4 * t + 2], ec[4 * t + 3]))
                br = 0.0; /* wall edge: no bracket, no coefficient */
            else if (ec[4 * t] == 0)
                br = (hz[p] - hz[p - sy]) - (hy[p] - hy[p - sz]);
            else if (ec[4 * t] == 1)
                br = (hx[p] - hx[p - sz]) - (hz[p] - hz[p - 1]);
            else
                br = (hy[p] - hy[p - 1]) - (hx[p] - hx[p - sy]);
            for (int s = 0; s < nsrc; ++s)
                if (src[4 * s] == ec[4 * t] && src[4 * s + 1] == ec[4 * t + 1] &&
                    src[4 * s + 2] == ec[4 * t + 2] && src[4 * s + 3] == ec[4 * t + 3])
                    br += sval[(long)s * nsteps + n];
            tr_c[(size_t)n * nedge + t] = br;
        }
    }
    for (int n = 1; n <= nsteps; ++n) J += f[n] * f[n];
    J *= dt;

    /* Reverse sweep. */
    const long pp = (long)pk * sz + (long)pj * sy + pi;
    for (int n = nsteps - 1; n >= 0; --n) {
        lam[(long)pcomp * npt + pp] += 2.0 * dt * f[n + 1];
        for (int t = 0; t < nedge; ++t) {
            const double l = le[ec[4 * t]][ep[t]];
            gcb[t] += l * tr_c[(size_t)n * nedge + t];
            gca[t] += l * tr_e[(size_t)n * nedge + t];
        }
        /* E half: rows of the interior edges. */
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    const long p = k * sz + j * sy + i;
                    if (interior(nx, ny, nz, 0, i, j, k)) {
                        const double w = cb[0][p] * le[0][p];
                        lz[p] += w;
                        lz[p - sy] -= w;
                        ly[p] -= w;
                        ly[p - sz] += w;
                        le[0][p] *= ca[0][p];
                    }
                    if (interior(nx, ny, nz, 1, i, j, k)) {
                        const double w = cb[1][p] * le[1][p];
                        lx[p] += w;
                        lx[p - sz] -= w;
                        lz[p] -= w;
                        lz[p - 1] += w;
                        le[1][p] *= ca[1][p];
                    }
                    if (interior(nx, ny, nz, 2, i, j, k)) {
                        const double w = cb[2][p] * le[2][p];
                        ly[p] += w;
                        ly[p - 1] -= w;
                        lx[p] -= w;
                        lx[p - sy] += w;
                        le[2][p] *= ca[2][p];
                    }
                }
        /* H half: rows of the updated faces. */
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    const long p = k * sz + j * sy + i;
                    if (k < nz && j < ny) {
                        const double v = S * lx[p];
                        le[1][p + sz] += v;
                        le[1][p] -= v;
                        le[2][p + sy] -= v;
                        le[2][p] += v;
                    }
                    if (k < nz && i < nx) {
                        const double v = S * ly[p];
                        le[2][p + 1] += v;
                        le[2][p] -= v;
                        le[0][p + sz] -= v;
                        le[0][p] += v;
                    }
                    if (j < ny && i < nx) {
                        const double v = S * lz[p];
                        le[0][p + sy] += v;
                        le[0][p] -= v;
                        le[1][p + 1] -= v;
                        le[1][p] += v;
                    }
                }
    }

    /* Chain rule to the cells. */
    for (int q = 0; q < ncells; ++q) {
        double g = 0.0;
        for (int u = 0; u < 12; ++u) {
            const int t = 12 * q + u;
            const int c = ec[4 * t], i = ec[4 * t + 1], j = ec[4 * t + 2], k = ec[4 * t + 3];
            if (!interior(nx, ny, nz, c, i, j, k)) continue;
            /* the four cells of the edge, in the mean's fixed order */
            int ci[4], cj[4], ck[4];
            for (int m = 0; m < 4; ++m) {
                const int a = m & 1, b = m >> 1;
                ci[m] = c == 0 ? i : i - 1 + a;
                cj[m] = c == 0 ? j - 1 + a : c == 1 ? j : j - 1 + b;
                ck[m] = c == 2 ? k : k - 1 + b;
            }
            double e4 = 0.0, s4 = 0.0;
            for (int m = 0; m < 4; ++m) {
                const long cell = ((long)ck[m] * ny + cj[m]) * nx + ci[m];
                e4 += (double)eps_cell[cell];
                s4 += (double)sig_cell[cell];
            }
            const double e = e4 * 0.25, s = s4 * 0.25;
            if (isinf(e)) continue; /* edge of a PEC cell: no eps dependence */
            const double beta = (s * dt) / (2.0 * EPS0 * e);
            const double cbv = (S / e) / (1.0 + beta);
            const double dcb = -cbv / (e * (1.0 + beta));
            const double dca = 2.0 * beta / (e * (1.0 + beta) * (1.0 + beta));
            g += 0.25 * (gcb[t] * dcb + gca[t] * dca);
        }
        grad[q] = g;
    }
done:
    free(co);
    free(lam);
    free(f);
    free(tr_e);
    free(tr_c);
    free(gcb);
    free(gca);
    free(ec);
    free(ep);
    return J;
}
