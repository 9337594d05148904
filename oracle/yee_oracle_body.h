/*
 * Body of the plain CPU oracle, instantiated twice by yee_oracle.c: once with
 * REAL = double (suffix _f64) and once with REAL = float (suffix _f32).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library links, includes or calls
 * this file; it shares no code with the CUDA path.
 *
 * Storage (one array per component, no padding, x fastest):
 *   value(i,j,k) = a[(k*(ny+1) + j)*(nx+1) + i],  0<=i<=nx, 0<=j<=ny, 0<=k<=nz.
 * Staggering (cell (i,j,k) occupies [i,i+1]x[j,j+1]x[k,k+1]):
 *   ex(i,j,k) at (i+1/2, j, k)      ey at (i, j+1/2, k)      ez at (i, j, k+1/2)
 *   hx(i,j,k) at (i, j+1/2, k+1/2)  hy at (i+1/2, j, k+1/2)  hz at (i+1/2, j+1/2, k)
 * Variables are the paper's antisymmetric pair scaled to V/m: e = E and
 * h = eta0*H, so that the leapfrog of Sec. 2.1 (Eqs. ma2, mf2) reads
 *   h += S * (discrete -curl e),   e = Ca*e + Cb*(discrete curl h),   S = c dt / dx.
 * Working-precision evaluation: with br the bracket (a1-a0)-(b1-b0),
 *   h = FMA(S, br, h)   and   e = FMA(Cb, br, Ca*e)
 * (one fused multiply-add each, every other operation rounded separately).
 */

#ifndef REAL
#error "define REAL before including yee_oracle_body.h"
#endif
#ifndef FMA
#error "define FMA (fma or fmaf) before including yee_oracle_body.h"
#endif

#define CAT_(a, b) a##_##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SUF)

/*
 * Per-edge update coefficients from per-cell material values.
 * eps_r(edge), sigma(edge) = arithmetic mean of the four cells sharing the
 * edge (summed in the fixed order (-,-), (+,-), (-,+), (+,+) of the two
 * transverse offsets, in double). Loss: semi-implicit average of sigma*E
 * (Taflove's standard lossy Yee update, cited by the paper in Sec. 2.1):
 *   beta = sigma*dt / (2*eps0*eps_r),  Ca = (1-beta)/(1+beta),
 *   Cb = (S/eps_r)/(1+beta),           S  = c*dt/dx  (double).
 * Only interior (non-PEC) edges get coefficients; wall edges keep Ca = Cb = 0.
 * A cell with eps_r = +inf is a perfect conductor: every edge it touches is a
 * PEC edge (Ca = Cb = 0, eps_r(edge) reported as 0), the same as a wall edge,
 * so a layer of such cells splits the grid into independent cavities.
 * epsx/epsy/epsz (double, may be NULL) receive eps_r(edge), 0 on walls.
 */
void FN(oracle_coefs)(int nx, int ny, int nz, double dx, double dt,
                      const float *eps_cell, const float *sig_cell,
                      REAL *cax, REAL *cbx, REAL *cay, REAL *cby, REAL *caz, REAL *cbz,
                      double *epsx, double *epsy, double *epsz)
{
    const long sx = 1, sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    const long ntot = sz * (nz + 1);
    const double S = C0 * dt / dx;
    for (long p = 0; p < ntot; ++p) {
        cax[p] = cbx[p] = cay[p] = cby[p] = caz[p] = cbz[p] = 0;
        if (epsx) epsx[p] = 0.0;
        if (epsy) epsy[p] = 0.0;
        if (epsz) epsz[p] = 0.0;
    }
    (void)sx;
#define CELL(arr, i, j, k) ((double)(arr)[((long)(k) * ny + (j)) * nx + (i)])
#define COEF(eps4, sig4, ca, cb)                                                  \
    do {                                                                          \
        const double e_ = (eps4) * 0.25, s_ = (sig4) * 0.25;                      \
        if (isinf(e_)) { /* an edge of a PEC cell: tangential E stays 0 */         \
            ca = 0;                                                               \
            cb = 0;                                                               \
            epsv = 0.0;                                                           \
            break;                                                                \
        }                                                                         \
        const double beta_ = (s_ * dt) / (2.0 * EPS0 * e_);                       \
        ca = (REAL)((1.0 - beta_) / (1.0 + beta_));                               \
        cb = (REAL)((S / e_) / (1.0 + beta_));                                    \
        epsv = e_;                                                                \
    } while (0)
    /* ex(i,j,k): cells (i, j-1..j, k-1..k) */
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double e4 = ((CELL(eps_cell, i, j - 1, k - 1) + CELL(eps_cell, i, j, k - 1)) +
                                   CELL(eps_cell, i, j - 1, k)) + CELL(eps_cell, i, j, k);
                const double s4 = ((CELL(sig_cell, i, j - 1, k - 1) + CELL(sig_cell, i, j, k - 1)) +
                                   CELL(sig_cell, i, j - 1, k)) + CELL(sig_cell, i, j, k);
                double epsv;
                COEF(e4, s4, cax[p], cbx[p]);
                if (epsx) epsx[p] = epsv;
            }
    /* ey(i,j,k): cells (i-1..i, j, k-1..k) */
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double e4 = ((CELL(eps_cell, i - 1, j, k - 1) + CELL(eps_cell, i, j, k - 1)) +
                                   CELL(eps_cell, i - 1, j, k)) + CELL(eps_cell, i, j, k);
                const double s4 = ((CELL(sig_cell, i - 1, j, k - 1) + CELL(sig_cell, i, j, k - 1)) +
                                   CELL(sig_cell, i - 1, j, k)) + CELL(sig_cell, i, j, k);
                double epsv;
                COEF(e4, s4, cay[p], cby[p]);
                if (epsy) epsy[p] = epsv;
            }
    /* ez(i,j,k): cells (i-1..i, j-1..j, k) */
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double e4 = ((CELL(eps_cell, i - 1, j - 1, k) + CELL(eps_cell, i, j - 1, k)) +
                                   CELL(eps_cell, i - 1, j, k)) + CELL(eps_cell, i, j, k);
                const double s4 = ((CELL(sig_cell, i - 1, j - 1, k) + CELL(sig_cell, i, j - 1, k)) +
                                   CELL(sig_cell, i - 1, j, k)) + CELL(sig_cell, i, j, k);
                double epsv;
                COEF(e4, s4, caz[p], cbz[p]);
                if (epsz) epsz[p] = epsv;
            }
#undef COEF
#undef CELL
}

/*
 * H update (Maxwell-Faraday, Sec. 2.1 displayed Hx formula and its analogues):
 *   hx += S*((ey(k+1)-ey(k)) - (ez(j+1)-ez(j)))     i in [0,nx], j in [0,ny), k in [0,nz)
 *   hy += S*((ez(i+1)-ez(i)) - (ex(k+1)-ex(k)))     i in [0,nx), j in [0,ny], k in [0,nz)
 *   hz += S*((ex(j+1)-ex(j)) - (ey(i+1)-ey(i)))     i in [0,nx), j in [0,ny), k in [0,nz]
 * Faces normal to a wall see only zero (PEC) tangential E and keep their value.
 */
static void FN(update_h)(int nx, int ny, int nz, REAL S,
                         const REAL *ex, const REAL *ey, const REAL *ez,
                         REAL *hx, REAL *hy, REAL *hz)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const long p = k * sz + j * sy + i;
                hx[p] = FMA(S, (ey[p + sz] - ey[p]) - (ez[p + sy] - ez[p]), hx[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                hy[p] = FMA(S, (ez[p + 1] - ez[p]) - (ex[p + sz] - ex[p]), hy[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                hz[p] = FMA(S, (ex[p + sy] - ex[p]) - (ey[p + 1] - ey[p]), hz[p]);
            }
}

/* Curl-h brackets of the E update (Maxwell-Ampere), at storage offset p. */
#define BR_X(p) ((hz[p] - hz[(p) - sy]) - (hy[p] - hy[(p) - sz]))
#define BR_Y(p) ((hx[p] - hx[(p) - sz]) - (hz[p] - hz[(p) - 1]))
#define BR_Z(p) ((hy[p] - hy[(p) - 1]) - (hx[p] - hx[(p) - sy]))

/*
 * E update on interior (non-PEC) edges, Sec. 2.1 leapfrog with loss:
 *   e = Ca*e + Cb*bracket.
 * Tangential E on the six walls is never written (PEC, Sec. 3.3).
 * A soft source is a current on the Ampere right-hand side (Sec. 3.3): at
 * its edge the bracket becomes (bracket + s), s = amp*w(t^{n+1/2}).
 * Source edges are evaluated after the sweep from their saved old value; the
 * sweep itself does not read E, so the result equals the in-loop form.
 */
static void FN(update_e)(int nx, int ny, int nz,
                         REAL *ex, REAL *ey, REAL *ez,
                         const REAL *hx, const REAL *hy, const REAL *hz,
                         const REAL *cax, const REAL *cbx, const REAL *cay,
                         const REAL *cby, const REAL *caz, const REAL *cbz,
                         int nsrc, const int *src, const REAL *sval, REAL *eold)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    for (int s = 0; s < nsrc; ++s) {
        const int c = src[4 * s];
        const long p = (long)src[4 * s + 3] * sz + (long)src[4 * s + 2] * sy + src[4 * s + 1];
        eold[s] = (c == 0 ? ex : c == 1 ? ey : ez)[p];
    }
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ex[p] = FMA(cbx[p], BR_X(p), cax[p] * ex[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ey[p] = FMA(cby[p], BR_Y(p), cay[p] * ey[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ez[p] = FMA(cbz[p], BR_Z(p), caz[p] * ez[p]);
            }
    /* Several sources on one edge add their currents in list order. */
    for (int s = 0; s < nsrc; ++s) {
        const int c = src[4 * s];
        const long p = (long)src[4 * s + 3] * sz + (long)src[4 * s + 2] * sy + src[4 * s + 1];
        int first = 1;
        for (int q = 0; q < s; ++q)
            if (src[4 * q] == c && src[4 * q + 1] == src[4 * s + 1] &&
                src[4 * q + 2] == src[4 * s + 2] && src[4 * q + 3] == src[4 * s + 3])
                first = 0;
        if (!first) continue;
        REAL br = (c == 0 ? BR_X(p) : c == 1 ? BR_Y(p) : BR_Z(p));
        for (int q = s; q < nsrc; ++q)
            if (src[4 * q] == c && src[4 * q + 1] == src[4 * s + 1] &&
                src[4 * q + 2] == src[4 * s + 2] && src[4 * q + 3] == src[4 * s + 3])
                br = br + sval[q];
        const REAL *ca = c == 0 ? cax : c == 1 ? cay : caz;
        const REAL *cb = c == 0 ? cbx : c == 1 ? cby : cbz;
        REAL *e = c == 0 ? ex : c == 1 ? ey : ez;
        e[p] = FMA(cb[p], br, ca[p] * eold[s]);
    }
}

/*
 * Advance nsteps leapfrog steps: for each step, all H (a1), then all E with
 * PEC and sources (a2-a4), then the probes (a5). Taflove-standard order, one
 * separate sweep per component.
 *   src:   nsrc x {comp(0..2), i, j, k}; edge must be interior.
 *   sval:  nsrc x sstride values; step m (0-based within this call) uses
 *          sval[s*sstride + m] = amp*w((n0+m+1/2)*dt) (computed by the caller).
 *   prb:   nprb x {comp(0..5), i, j, k}; after step m, E probes record e^{n+1},
 *          H probes record h^{n+1/2}, into pout[q*pstride + m].
 */
void FN(oracle_step)(int nx, int ny, int nz, REAL S,
                     REAL *ex, REAL *ey, REAL *ez, REAL *hx, REAL *hy, REAL *hz,
                     const REAL *cax, const REAL *cbx, const REAL *cay,
                     const REAL *cby, const REAL *caz, const REAL *cbz,
                     int nsrc, const int *src, const REAL *sval, long sstride,
                     int nprb, const int *prb, REAL *pout, long pstride, int nsteps)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    REAL eold[64];
    REAL sv[64];
    if (nsrc > 64) nsrc = 64;
    for (int m = 0; m < nsteps; ++m) {
        FN(update_h)(nx, ny, nz, S, ex, ey, ez, hx, hy, hz);
        for (int s = 0; s < nsrc; ++s) sv[s] = sval[s * sstride + m];
        FN(update_e)(nx, ny, nz, ex, ey, ez, hx, hy, hz, cax, cbx, cay, cby, caz, cbz,
                     nsrc, src, sv, eold);
        for (int q = 0; q < nprb; ++q) {
            const int c = prb[4 * q];
            const long p = (long)prb[4 * q + 3] * sz + (long)prb[4 * q + 2] * sy + prb[4 * q + 1];
            const REAL *f = c == 0 ? ex : c == 1 ? ey : c == 2 ? ez : c == 3 ? hx : c == 4 ? hy : hz;
            pout[q * pstride + m] = f[p];
        }
    }
}

/*
 * Discrete Yee energy at time level n (fields hold e^n and h^{n-1/2}):
 *   W^n = 1/2 eps0 dx^3 [ sum_edges eps_r(edge) (e^n)^2 + sum_faces h^{n-1/2} h^{n+1/2} ]
 * h^{n+1/2} is formed with the same H-update expression in REAL precision and
 * never stored; products and sums are in double, summed in storage order.
 */
double FN(oracle_energy)(int nx, int ny, int nz, REAL S, double dx,
                         const REAL *ex, const REAL *ey, const REAL *ez,
                         const REAL *hx, const REAL *hy, const REAL *hz,
                         const double *epsx, const double *epsy, const double *epsz)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    double we = 0.0, wh = 0.0;
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                we += epsx[p] * ((double)ex[p] * (double)ex[p]);
            }
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                we += epsy[p] * ((double)ey[p] * (double)ey[p]);
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                we += epsz[p] * ((double)ez[p] * (double)ez[p]);
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL hn = FMA(S, (ey[p + sz] - ey[p]) - (ez[p + sy] - ez[p]), hx[p]);
                wh += (double)hx[p] * (double)hn;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL hn = FMA(S, (ez[p + 1] - ez[p]) - (ex[p + sz] - ex[p]), hy[p]);
                wh += (double)hy[p] * (double)hn;
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL hn = FMA(S, (ex[p + sy] - ex[p]) - (ey[p + 1] - ey[p]), hz[p]);
                wh += (double)hz[p] * (double)hn;
            }
    return 0.5 * EPS0 * dx * dx * dx * (we + wh);
}

/*
 * Non-uniform mesh (1-D coefficient arrays per axis, the geometric
 * coefficients dx(i), dy(j), dz(k) of Sec. 2.2's loop). With a reference step
 * dx0 (the grid's dx, S = c dt / dx0) and cell widths wx(i), the ratio arrays
 *   rx(i)  = dx0 / wx(i)                          i in [0, nx)  (primary)
 *   rxd(i) = dx0 / ((wx(i-1) + wx(i)) / 2)        i in [0, nx]  (dual; wx(-1) = wx(0), wx(nx) = wx(nx-1))
 * (and likewise y, z) scale each difference of a curl bracket by the width it
 * spans: primary widths for the H update (differences of E across a face),
 * dual widths for the E update (differences of H across an edge's dual face):
 *   br = FMA(r_a, a1 - a0, -(r_b * (b1 - b0)))
 *   h  = FMA(S, br, h),   e = FMA(Cb, br [+ s], Ca*e)
 * With all ratios 1 this is exactly the uniform expression (1*x is exact and
 * FMA(1, x, -y) rounds x - y once). The wall-node duals rxd(0), rxd(nx) are
 * read by no update (the E edges there are PEC); they weigh the wall-normal
 * faces in the energy, a whole end cell as in the uniform energy.
 */
static void FN(update_h_nu)(int nx, int ny, int nz, REAL S,
                            const REAL *ex, const REAL *ey, const REAL *ez,
                            REAL *hx, REAL *hy, REAL *hz,
                            const REAL *rx, const REAL *ry, const REAL *rz)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(rz[k], ey[p + sz] - ey[p], -(ry[j] * (ez[p + sy] - ez[p])));
                hx[p] = FMA(S, br, hx[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(rx[i], ez[p + 1] - ez[p], -(rz[k] * (ex[p + sz] - ex[p])));
                hy[p] = FMA(S, br, hy[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(ry[j], ex[p + sy] - ex[p], -(rx[i] * (ey[p + 1] - ey[p])));
                hz[p] = FMA(S, br, hz[p]);
            }
}

#define BRN_X(p) FMA(ryd[j], hz[p] - hz[(p) - sy], -(rzd[k] * (hy[p] - hy[(p) - sz])))
#define BRN_Y(p) FMA(rzd[k], hx[p] - hx[(p) - sz], -(rxd[i] * (hz[p] - hz[(p) - 1])))
#define BRN_Z(p) FMA(rxd[i], hy[p] - hy[(p) - 1], -(ryd[j] * (hx[p] - hx[(p) - sy])))

/* Non-uniform E update; sources as in update_e (inside the bracket). */
static void FN(update_e_nu)(int nx, int ny, int nz,
                            REAL *ex, REAL *ey, REAL *ez,
                            const REAL *hx, const REAL *hy, const REAL *hz,
                            const REAL *cax, const REAL *cbx, const REAL *cay,
                            const REAL *cby, const REAL *caz, const REAL *cbz,
                            const REAL *rxd, const REAL *ryd, const REAL *rzd,
                            int nsrc, const int *src, const REAL *sval, REAL *eold)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    for (int s = 0; s < nsrc; ++s) {
        const int c = src[4 * s];
        const long p = (long)src[4 * s + 3] * sz + (long)src[4 * s + 2] * sy + src[4 * s + 1];
        eold[s] = (c == 0 ? ex : c == 1 ? ey : ez)[p];
    }
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ex[p] = FMA(cbx[p], BRN_X(p), cax[p] * ex[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ey[p] = FMA(cby[p], BRN_Y(p), cay[p] * ey[p]);
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                ez[p] = FMA(cbz[p], BRN_Z(p), caz[p] * ez[p]);
            }
    for (int s = 0; s < nsrc; ++s) {
        const int c = src[4 * s];
        const int i = src[4 * s + 1], j = src[4 * s + 2], k = src[4 * s + 3];
        const long p = (long)k * sz + (long)j * sy + i;
        int first = 1;
        for (int q = 0; q < s; ++q)
            if (src[4 * q] == c && src[4 * q + 1] == i && src[4 * q + 2] == j && src[4 * q + 3] == k)
                first = 0;
        if (!first) continue;
        REAL br = (c == 0 ? BRN_X(p) : c == 1 ? BRN_Y(p) : BRN_Z(p));
        for (int q = s; q < nsrc; ++q)
            if (src[4 * q] == c && src[4 * q + 1] == i && src[4 * q + 2] == j && src[4 * q + 3] == k)
                br = br + sval[q];
        const REAL *ca = c == 0 ? cax : c == 1 ? cay : caz;
        const REAL *cb = c == 0 ? cbx : c == 1 ? cby : cbz;
        REAL *e = c == 0 ? ex : c == 1 ? ey : ez;
        e[p] = FMA(cb[p], br, ca[p] * eold[s]);
    }
}

/* Steps on a non-uniform mesh; arguments as oracle_step plus the six ratio
 * arrays (rx[nx], ry[ny], rz[nz], rxd[nx+1], ryd[ny+1], rzd[nz+1]). */
void FN(oracle_step_nu)(int nx, int ny, int nz, REAL S,
                        REAL *ex, REAL *ey, REAL *ez, REAL *hx, REAL *hy, REAL *hz,
                        const REAL *cax, const REAL *cbx, const REAL *cay,
                        const REAL *cby, const REAL *caz, const REAL *cbz,
                        const REAL *rx, const REAL *ry, const REAL *rz,
                        const REAL *rxd, const REAL *ryd, const REAL *rzd,
                        int nsrc, const int *src, const REAL *sval, long sstride,
                        int nprb, const int *prb, REAL *pout, long pstride, int nsteps)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    REAL eold[64];
    REAL sv[64];
    if (nsrc > 64) nsrc = 64;
    for (int m = 0; m < nsteps; ++m) {
        FN(update_h_nu)(nx, ny, nz, S, ex, ey, ez, hx, hy, hz, rx, ry, rz);
        for (int s = 0; s < nsrc; ++s) sv[s] = sval[s * sstride + m];
        FN(update_e_nu)(nx, ny, nz, ex, ey, ez, hx, hy, hz, cax, cbx, cay, cby, caz, cbz,
                        rxd, ryd, rzd, nsrc, src, sv, eold);
        for (int q = 0; q < nprb; ++q) {
            const int c = prb[4 * q];
            const long p = (long)prb[4 * q + 3] * sz + (long)prb[4 * q + 2] * sy + prb[4 * q + 1];
            const REAL *f = c == 0 ? ex : c == 1 ? ey : c == 2 ? ez : c == 3 ? hx : c == 4 ? hy : hz;
            pout[q * pstride + m] = f[p];
        }
    }
}

/*
 * Discrete energy on a non-uniform mesh: every term is weighted by its
 * volume in units of dx0^3 -- an edge's length times its dual face, a face's
 * area times its dual edge -- formed in double from the ratio arrays:
 *   ex(i,j,k): 1 / (rx(i) ryd(j) rzd(k)),   hx(i,j,k): 1 / (rxd(i) ry(j) rz(k)), ...
 * h^{n+1/2} is formed with the non-uniform H update.
 */
double FN(oracle_energy_nu)(int nx, int ny, int nz, REAL S, double dx,
                            const REAL *ex, const REAL *ey, const REAL *ez,
                            const REAL *hx, const REAL *hy, const REAL *hz,
                            const double *epsx, const double *epsy, const double *epsz,
                            const REAL *rx, const REAL *ry, const REAL *rz,
                            const REAL *rxd, const REAL *ryd, const REAL *rzd)
{
    const long sy = nx + 1, sz = (long)(nx + 1) * (ny + 1);
    double we = 0.0, wh = 0.0;
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double v = 1.0 / (((double)rx[i] * (double)ryd[j]) * (double)rzd[k]);
                we += v * (epsx[p] * ((double)ex[p] * (double)ex[p]));
            }
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double v = 1.0 / (((double)rxd[i] * (double)ry[j]) * (double)rzd[k]);
                we += v * (epsy[p] * ((double)ey[p] * (double)ey[p]));
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const double v = 1.0 / (((double)rxd[i] * (double)ryd[j]) * (double)rz[k]);
                we += v * (epsz[p] * ((double)ez[p] * (double)ez[p]));
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(rz[k], ey[p + sz] - ey[p], -(ry[j] * (ez[p + sy] - ez[p])));
                const REAL hn = FMA(S, br, hx[p]);
                const double v = 1.0 / (((double)rxd[i] * (double)ry[j]) * (double)rz[k]);
                wh += v * ((double)hx[p] * (double)hn);
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(rx[i], ez[p + 1] - ez[p], -(rz[k] * (ex[p + sz] - ex[p])));
                const REAL hn = FMA(S, br, hy[p]);
                const double v = 1.0 / (((double)rx[i] * (double)ryd[j]) * (double)rz[k]);
                wh += v * ((double)hy[p] * (double)hn);
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long p = k * sz + j * sy + i;
                const REAL br = FMA(ry[j], ex[p + sy] - ex[p], -(rx[i] * (ey[p + 1] - ey[p])));
                const REAL hn = FMA(S, br, hz[p]);
                const double v = 1.0 / (((double)rx[i] * (double)ry[j]) * (double)rzd[k]);
                wh += v * ((double)hz[p] * (double)hn);
            }
    return 0.5 * EPS0 * dx * dx * dx * (we + wh);
}

#undef BRN_X
#undef BRN_Y
#undef BRN_Z
#undef BR_X
#undef BR_Y
#undef BR_Z
#undef FN
#undef CAT
#undef CAT_
