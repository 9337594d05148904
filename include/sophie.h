/*
 * libsophie - GB300 (sm_103a) 3-D Yee FDTD leapfrog sweep behind a C ABI.
 *
 * The method is the one of O. Cessenat, "Sophie, an FDTD code on the way to
 * multicore" (arXiv:1301.4539): Sec. 2.1 gives the scheme (Maxwell-Ampere and
 * Maxwell-Faraday in antisymmetric scaled form, Yee staggering, leapfrog in
 * time, displayed Hx update); Sec. 3.3 gives PEC walls (tangential E held at 0)
 * and sources (a current added to Ampere's equation); Sec. 3.4 gives pin-point
 * outputs and multi-step cache reuse; Sec. 3.1 states that any such
 * restructuring leaves every output value unchanged.
 *
 * Units and variables. e = E (V/m) and h = eta0*H (V/m), i.e. the paper's
 * (E~, H~) = eps0*(e, h). With S = c*dt/dx one step n -> n+1 is
 *   h^{n+1/2} = h^{n-1/2} + S * (discrete -curl e^n)              (Faraday)
 *   e^{n+1}   = Ca*e^n + Cb*(discrete curl h^{n+1/2} + s^{n+1/2}) (Ampere)
 * with, per edge, eps_r and sigma the mean of the four cells sharing the edge,
 *   beta = sigma*dt/(2*eps0*eps_r), Ca = (1-beta)/(1+beta),
 *   Cb = (S/eps_r)/(1+beta)   (computed in double, rounded once to float),
 * and s the source term (only on source edges). Fields are float32; with
 * br = (a1-a0) - (b1-b0) (plus s on a source edge), every update is one
 * fused multiply-add with every other operation rounded separately:
 *   h = fma(S, br, h)   and   e = fma(Cb, br, Ca*e),
 * so the results are fixed by the expression alone, whatever the kernel.
 * (On a non-uniform mesh br scales its two differences, sophie_set_spacing.)
 *
 * Storage indices (the "field layout" below). For a grid of nx*ny*nz cells,
 * every component is addressed on the (nx+1)*(ny+1)*(nz+1) index box, x
 * fastest; cell (i,j,k) occupies [i,i+1]x[j,j+1]x[k,k+1] (units of dx):
 *   comp 0 ex(i,j,k) at (i+1/2, j, k)      valid i<nx
 *   comp 1 ey(i,j,k) at (i, j+1/2, k)      valid j<ny
 *   comp 2 ez(i,j,k) at (i, j, k+1/2)      valid k<nz
 *   comp 3 hx(i,j,k) at (i, j+1/2, k+1/2)  valid j<ny, k<nz
 *   comp 4 hy(i,j,k) at (i+1/2, j, k+1/2)  valid i<nx, k<nz
 *   comp 5 hz(i,j,k) at (i+1/2, j+1/2, k)  valid i<nx, j<ny
 * Tangential E on the six walls (PEC) is always 0. Entries outside a
 * component's valid range are always 0.
 *
 * Threading: a grid handle is used by one host thread at a time. Errors are
 * reported by a negative return code and a thread-local message
 * (sophie_last_error). Device memory is owned by the library.
 */
#ifndef SOPHIE_H
#define SOPHIE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SOPHIE_OK           0
#define SOPHIE_EINVAL      -1  /* bad argument (NULL, range, state)            */
#define SOPHIE_EUNSTABLE   -2  /* dt above the 3-D Courant limit dx/(c*sqrt 3) */
#define SOPHIE_ENOMEM      -3  /* device or host allocation failed / too big   */
#define SOPHIE_ECUDA       -4  /* a CUDA runtime call failed                   */
#define SOPHIE_ENONFINITE  -5  /* a non-finite value was found (energy)        */
#define SOPHIE_ETIMEOUT    -6  /* a kernel's bounded wait ran out              */
#define SOPHIE_ETOOMANYMAT -7  /* more distinct edge materials than supported  */
#define SOPHIE_ENOTSUP     -8  /* option not supported by this build           */

/* Component ids (storage indices above). */
#define SOPHIE_EX 0
#define SOPHIE_EY 1
#define SOPHIE_EZ 2
#define SOPHIE_HX 3
#define SOPHIE_HY 4
#define SOPHIE_HZ 5

/* Source waveform kinds for sophie_add_source. */
#define SOPHIE_GAUSS_SINE 0
#define SOPHIE_GAUSS      1

/* Storage precision of the six field arrays (sophie_configure). Arithmetic is
 * float in every mode; the 2-byte modes store field * scale[comp] (see
 * sophie_set_storage_scale) rounded to nearest even once per launch. */
#define SOPHIE_FP32 0
#define SOPHIE_FP16 1
#define SOPHIE_BF16 2
#define SOPHIE_FP16HL 3  /* hi + lo pair of halves per value (4 B), see sophie_configure */
#define SOPHIE_FP24 4    /* upper 24 bits of the float (3 B), see sophie_configure */

/* Kernel ids for sophie_profile_read. */
#define SOPHIE_KERNEL_PLAIN   0  /* one fused H+E step per launch           */
#define SOPHIE_KERNEL_BLOCKED 1  /* k fused H+E steps per launch (k >= 2)   */
#define SOPHIE_KERNEL_ENERGY  2  /* discrete energy reduction               */
#define SOPHIE_KERNEL_ADJOINT 3  /* one reverse (adjoint) step per launch    */

typedef struct sophie_grid sophie_grid;

/* Library version, e.g. 10000 for 1.0.0. */
int sophie_version(void);

/*
 * Create a PEC cavity of nx*ny*nz cells of edge dx (m), time step dt (s).
 * Sec. 2.1: uniform Cartesian Yee grid. Requires nx,ny,nz >= 1, dx > 0,
 * 0 < dt <= dx/(c*sqrt(3)) (else SOPHIE_EUNSTABLE). All fields start at 0, the
 * medium is vacuum (eps_r = 1, sigma = 0), no sources, no probes, step 0.
 * Allocates two device copies of the six fields (ping-pong), one 32-bit
 * material word per index point and small tables. On success *out owns them.
 * Errors: EINVAL (bad argument, out == NULL), EUNSTABLE, ENOMEM, ECUDA.
 */
int sophie_create_grid(int nx, int ny, int nz, double dx, double dt, sophie_grid **out);

/* Free a grid and all its device memory; NULL is accepted. Waits for pending
 * work. A handle that is not live (e.g. destroyed already) gives EINVAL and
 * nothing is freed. */
int sophie_destroy_grid(sophie_grid *g);

/*
 * Per-cell relative permittivity and conductivity (S/m), host arrays of
 * nx*ny*nz floats each (x fastest, then y, then z), copied. eps_r >= 1, or
 * +inf for a perfectly conducting cell (every edge it touches is PEC, like
 * the outer walls); sigma >= 0 and finite (else EINVAL). Edge values are the
 * mean of the four cells sharing the edge (Sec. 2.1 coefficients, see top of
 * file). The 511 most frequent edge materials are held as classes in a
 * table; index points with an edge outside them carry explicit coefficients
 * (any number of distinct materials; points with the same three edge
 * materials share one 48-byte entry, read with the point). Enqueued on the
 * grid's stream; the host arrays may be reused on return.
 * Errors: EINVAL, ENOMEM, ECUDA, ETOOMANYMAT (more than 2^29 explicit entries).
 */
int sophie_set_materials(sophie_grid *g, const float *eps_r, const float *sigma);

/*
 * Add a soft current source on the E edge (comp in {0,1,2}, storage indices
 * i,j,k; the edge must be interior, i.e. not PEC). Sec. 3.3: a current added
 * to Ampere's equation. At step n -> n+1 the term s = amp*w((n+1/2)*dt),
 * computed in double and rounded once to float, is added inside the curl
 * bracket of that edge: e = Ca*e + Cb*(bracket + s). Waveforms:
 *   kind 0: w(t) = sin(2 pi f0 (t-t0)) * exp(-(t-t0)^2/(2 st^2))
 *   kind 1: w(t) = exp(-(t-t0)^2/(2 st^2))
 * with st = 1/(2 pi sf), sf = bw/(2 sqrt(2 ln 2)) (bw = FWHM of the amplitude
 * spectrum of the envelope). Up to 16 sources; several on one edge add in the
 * order they were added. Errors: EINVAL.
 */
int sophie_add_source(sophie_grid *g, int comp, int i, int j, int k,
                      double amp, double f0, double bw, double t0, int kind);

/*
 * Add a pin-point output (Sec. 3.4) on component comp (0..5) at storage
 * indices (i,j,k) within the component's valid range. Sample m (m >= 0) is the
 * value after step m -> m+1: e^{m+1} for E, h^{m+1/2} for H. Samples of steps
 * taken before the probe existed read 0. Up to 64 probes; *probe_id gets the
 * probe's index. Errors: EINVAL.
 */
int sophie_add_probe(sophie_grid *g, int comp, int i, int j, int k, int *probe_id);

/*
 * Advance n >= 0 leapfrog steps (H then E, PEC, sources, probes). Steps are
 * fused: one launch advances k steps when temporal blocking is configured
 * (Sec. 3.4 multi-step cache reuse); results are bitwise identical for every
 * k. Asynchronous: returns once the work is enqueued on the grid's stream.
 * Errors: EINVAL, ECUDA, ENOMEM.
 */
int sophie_step(sophie_grid *g, int n);

/* Steps taken since creation or the last sophie_reset. */
int sophie_get_step(sophie_grid *g, long long *n);

/*
 * Copy up to cap samples of probe probe_id, widened to double, into out
 * (host); *n_written gets min(cap, steps taken). Synchronises the stream.
 * Errors: EINVAL, ECUDA, ETIMEOUT.
 */
int sophie_read_probe(sophie_grid *g, int probe_id, double *out, int cap, int *n_written);

/*
 * Discrete Yee energy at the current step n (Sec. 2.1 antisymmetric form):
 *   W = 1/2 eps0 dx^3 [ sum_edges eps_r(edge) (e^n)^2 + sum_faces h^{n-1/2} h^{n+1/2} ]
 * with h^{n+1/2} formed from the same float update and never stored,
 * accumulated in double. Synchronises the stream.
 * Errors: EINVAL, ECUDA, ETIMEOUT, ENONFINITE (W not finite; *W still set).
 */
int sophie_energy(sophie_grid *g, double *W);

/*
 * The energy of sophie_energy, for callers that cannot allocate device memory
 * when they ask for it: an application that reserves its whole device-memory
 * budget up front (a caching allocator that owns the heap, or a host that
 * forbids allocation once it runs), where a cudaMalloc would fail or is not
 * allowed. The paper has no counterpart; it is an interface convenience.
 * W_dev is a caller-owned device pointer that receives W (double, J). No
 * memory is allocated: the reduction's partial sums live in a static device
 * array of 2432 doubles (19 KiB, held by every device that loads the library
 * until exit). That is the most any grid needs (the reduction's block count
 * is capped at 2432 and a grid-stride loop covers larger grids), so no grid
 * is rejected for its size. The first call on a device fetches the array's
 * address (make it before any stream capture). Enqueued on the grid's
 * stream; does not synchronise, does not check finiteness and does not read
 * the device error word of earlier launches (a later synchronising call such
 * as sophie_sync or sophie_energy reports a bounded wait that ran out); its
 * launches are not included in the sophie_profile timings. Calls whose
 * kernels overlap on the GPU (several grids or streams) race on the shared
 * array. Errors: EINVAL (NULL), ECUDA.
 */
int sophie_energy_noalloc(sophie_grid *g, double *W_dev);

/*
 * Copy one component from / to a host array of (nx+1)*(ny+1)*(nz+1) floats in
 * the storage layout above (x fastest). sophie_set_fields zeroes PEC edges
 * and out-of-range entries after the copy. Both synchronise.
 * Errors: EINVAL, ECUDA.
 */
int sophie_set_fields(sophie_grid *g, int comp, const float *host);
int sophie_get_fields(sophie_grid *g, int comp, float *host);

/* Zero all fields and probe samples and set the step counter to 0
 * (materials, sources and probes are kept). Enqueued on the stream. */
int sophie_reset(sophie_grid *g);

/*
 * Use cuda_stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream;
 * NULL = legacy default stream) for all later work of this grid. The caller
 * keeps the stream alive while the grid uses it. Synchronises the old stream.
 */
int sophie_set_stream(sophie_grid *g, void *cuda_stream);

/* Wait for all work of the grid; reports ETIMEOUT if a kernel gave up a wait. */
int sophie_sync(sophie_grid *g);

/*
 * temporal_k: steps fused per launch (1 = plain kernel, 2..4 = temporally
 * blocked; 6 and 8 = deeper blocking with float storage only, each 64x32
 * region then yielding (64-2k)x(32-2k) points; 5, 7 and 6 or 8 with another
 * precision: ENOTSUP), 0 = autotuned over 1..4 (the default: the first
 * sophie_step measures the candidates, see sophie_autotune). With a fixed k
 * the first sophie_step still measures that k's work splits (and the plain
 * kernel's z chunks) and keeps the fastest; results are the same. tile_x: 0 or 64 = TMA-staged 64x16 tiles
 * (default), 32 = 32x8 tiles with direct loads (a slower reference kernel;
 * identical results); tile_y: reserved, 0.
 * precision: SOPHIE_FP32, SOPHIE_FP16 or SOPHIE_BF16 storage of the fields,
 * or SOPHIE_FP16HL: each value v = field * scale kept as two halves
 * hi = half(v), lo = half(v - hi) (4 B, ~22 significant bits; the split
 * storage that wins back the accuracy half storage loses), or SOPHIE_FP24:
 * the upper 24 bits of each float (sign, the full 8-bit exponent, 15 mantissa
 * bits; 3 B per value, no scale), the value first rounded to 16 significant
 * bits by Veltkamp's splitting c = v * 257, hi = c + (v - c) in float
 * arithmetic (a rounding to nearest; for subnormal values the dropped low
 * byte is truncated). The device layout per z slab is then nine 2-byte
 * planes: the high halves of ex, ey, ez, hx, hy, hz and the byte pairs of
 * (ex, ey), (ez, hx), (hy, hz). A change converts
 * the current fields; synchronises. In the non-float modes one launch loads
 * the stored fields, computes its k steps in float and rounds once when
 * storing, so results depend on k (no longer bitwise equal across k).
 * Errors: EINVAL, ENOTSUP, ENOMEM.
 */
int sophie_configure(sophie_grid *g, int temporal_k, int tile_x, int tile_y, int precision);

/*
 * Per-component storage scales for the 2-byte modes (6 floats, powers of two
 * in [2^-61, 2^60], default 1): component c is stored as field * scale[c], so
 * a scale that brings the fields' working range near 1 keeps them clear of the
 * half format's subnormals and overflow. The current fields are converted.
 * No effect on float or 24-bit storage. With six equal scales the step kernels
 * run in unit-scale form (on the scaled values, with no scale multiplications;
 * the results are those of the scaled arithmetic, which a power-of-two scale
 * leaves exact outside the float subnormal range). Errors: EINVAL.
 */
int sophie_set_storage_scale(sophie_grid *g, const float *scale);

/*
 * Autotuner: times the step kernel candidates on this grid (plain kernel with
 * z chunks of 1..64 planes per work unit; temporally blocked kernel with
 * k = 2, 3, 4, each with the modelled split of every tile's planes into z
 * ranges, its neighbours and twice it, in two unit orders, and a split into
 * equal contiguous work ranges), each launch reading the current fields
 * and writing the spare buffer so the state does not advance, and keeps the
 * fastest per time step. The grid switches to temporal_k = 0 (autotuned) with
 * that choice. *temporal_k gets the chosen k, *ms_per_step the measured device
 * milliseconds per time step. All float-storage candidates give bitwise
 * identical fields; with 2-byte storage (results depend on k) k stays 2 and
 * only the tilings are tuned. Synchronises. Errors: EINVAL, ECUDA, ETIMEOUT.
 */
int sophie_autotune(sophie_grid *g, int *temporal_k, double *ms_per_step);

/*
 * The launch configuration the next sophie_step uses, in out[0..6]: steps per
 * launch (the fixed or tuned k; 1 = plain kernel, also for an autotuned grid
 * that has not measured yet), the plain kernel's z planes
 * per work unit and its CTAs, then the blocked kernel's CTAs, z ranges per tile
 * (0 = equal contiguous work ranges), unit order (0 tile-major, 1 range-major)
 * and rows of the region per thread (4: 8 warps, 2: 16 warps); the four
 * blocked entries are 0 when k = 1. Before the first step of a grid that is not
 * tuned yet these are the cost model's choices, which the first step's
 * measurements may replace. No synchronisation. Errors: EINVAL.
 */
int sophie_launch_config(sophie_grid *g, int *out);

/*
 * Zero-field skipping (early-time sparsity; the paper skips sub-domains whose
 * fields are all zero on their boundary, Sec. 4). With enable != 0 the step
 * kernels skip the work units whose outputs lie outside a box known to hold
 * every nonzero field value: after create or sophie_reset the box holds the
 * source points, and each step grows it by one index point per side (the
 * scheme moves a value by at most one point per axis and step); after the
 * caller writes fields (sophie_set_fields, a storage change) it is the whole
 * grid until the next reset. The skipped outputs are zero and stay zero, so
 * every field, probe and energy value is the same as without skipping.
 * Off by default. Errors: EINVAL.
 */
int sophie_set_zero_skip(sophie_grid *g, int enable);

/*
 * Non-uniform mesh (Sec. 2.2: the loop's geometric coefficients are 1-D
 * arrays dx(i), dy(j), dz(k)). wx (nx doubles), wy (ny), wz (nz): the cell
 * widths in metres along each axis, host arrays copied by the call; NULL
 * keeps that axis uniform with step dx, and all three NULL return the grid
 * to the uniform mesh. With the grid's dx as the reference step (S = c dt/dx
 * as before), every difference of a curl bracket is scaled by dx / (the
 * width it spans), rounded to float once per width:
 *   H update: primary widths, e.g. hx: rz(k) (ey(k+1) - ey(k)) - ry(j) (ez(j+1) - ez(j))
 *   E update: dual widths (the mean of the two cells beside the node; the
 *             end cell's width at a wall node, which only weighs the static
 *             wall-normal faces in the energy),
 *             e.g. ex: ryd(j) (hz(j) - hz(j-1)) - rzd(k) (hy(k) - hy(k-1))
 * evaluated as br = fma(ra, a1 - a0, -(rb * (b1 - b0))); with every width
 * equal to dx the fields and energies are bitwise those of the uniform mesh. Material
 * coefficients (Ca, Cb) are unchanged (the ratios carry the geometry), and
 * sophie_energy weights each term by its edge or face volume in units of
 * dx^3, so the lossless energy stays conserved.
 * Every step kernel (plain with either tile choice, temporally blocked k =
 * 2..4 with every storage format, 6 and 8 with float storage) and
 * zero-field skipping apply as on the
 * uniform mesh, with the same results across k for float storage.
 * Stability needs c dt sqrt(1/min(wx)^2 + 1/min(wy)^2 + 1/min(wz)^2) <= 1.
 * A probe objective record (sophie_objective_forward) is invalidated; probe
 * objectives need the uniform mesh.
 * Errors: EINVAL (NULL grid, a width not finite and > 0), EUNSTABLE (dt above
 * that limit), ENOMEM, ECUDA.
 */
int sophie_set_spacing(sophie_grid *g, const double *wx, const double *wy, const double *wz);

/* Number of kernels this grid has launched since creation. */
int sophie_launch_count(sophie_grid *g, long long *launches);

/*
 * Per-kernel timing with CUDA events recorded on the grid's stream around each
 * launch while enabled (enable != 0 also clears the totals). sophie_profile_read
 * synchronises and returns the launch count and the summed device milliseconds
 * of kernel id (SOPHIE_KERNEL_*).
 */
int sophie_profile(sophie_grid *g, int enable);
int sophie_profile_read(sophie_grid *g, int kernel, long long *launches, double *ms);

/*
 * Gradients of a probe objective with respect to eps_r (the differentiation
 * form; the paper has no adjoint, the steps it differentiates are Sec. 2.1's).
 *
 * sophie_objective_forward advances the grid by nsteps steps from its current
 * state, exactly as sophie_step(g, nsteps) would (user probes record as
 * usual), and returns in *J (host double)
 *   J = dt * sum_{n=1..nsteps} (f^n)^2,
 * f^n = component comp at index (i, j, k) after the n-th of these steps (an E
 * component is e^{n0+n}, an H component h^{n0+n-1/2}), summed in double. It
 * records the objective: the state every checkpoint_every steps (0 = 50), each
 * a device copy of the float fields (6 (nz+1)(ny+1) nxp floats, where nxp is
 * nx+1 rounded up to a multiple of 8), plus the nsteps samples. The record
 * stays valid until the grid's fields, materials or sources change (any step,
 * set_fields, reset, set_materials, add_source) and is freed by
 * sophie_objective_release or sophie_destroy_grid.
 * Errors: EINVAL (NULL, nsteps < 1, point outside comp's range or on a plane
 * i == nx, j == ny or k == nz), ENOTSUP (half or bfloat16 storage; all probe
 * slots in use, the objective needs one; a non-uniform mesh), ENOMEM
 * (checkpoints), ECUDA,
 * ETIMEOUT, ENONFINITE.
 *
 * sophie_objective_grad_eps returns dJ/d eps_r(cell) for the box of cells
 * [i0, i0+ni) x [j0, j0+nj) x [k0, k0+nk), in grad (host, ni*nj*nk doubles,
 * x fastest), sigma held fixed. It is the exact reverse mode of the recorded
 * float steps (with the float coefficients): segments between checkpoints are
 * recomputed, the adjoint fields are swept back in time by the transposed
 * step, and the coefficient sensitivities on the box's edges accumulate in
 * double; edge coefficients follow from the edge's mean material
 * (Cb = (S/eps)/(1+beta), Ca = (1-beta)/(1+beta), beta = sigma dt/(2 eps0 eps),
 * eps = mean of the 4 cells). The grid's state is not changed; the call may be
 * repeated for other boxes. Synchronises the stream.
 * Errors: EINVAL (NULL, box outside the cells, no valid record), ENOMEM,
 * ECUDA, ETIMEOUT.
 */
int sophie_objective_forward(sophie_grid *g, int nsteps, int comp, int i, int j, int k, int checkpoint_every,
                             double *J);
/*
 * sophie_objective_set_design registers the box of design cells (as for
 * sophie_objective_grad_eps) for the following objective records; ni = nj =
 * nk = 0 clears it. With a box registered, sophie_objective_forward runs one
 * step per launch and gathers, after every step, e^n and the E bracket on the
 * box's design edges ([nsteps][edges] floats twice, kept when they fit a
 * quarter of the free device memory and 8 GB; otherwise the record is the
 * checkpointed one); sophie_objective_grad_eps for that box then sweeps back
 * without recomputing any step. Gradients are the same either way (the same
 * float values are gathered). A traced record keeps no checkpoints: a
 * gradient for another box is refused (EINVAL) until the objective is
 * recorded again. Errors: EINVAL (NULL, box outside the cells).
 */
int sophie_objective_set_design(sophie_grid *g, int i0, int j0, int k0, int ni, int nj, int nk);
int sophie_objective_grad_eps(sophie_grid *g, int i0, int j0, int k0, int ni, int nj, int nk, double *grad);
int sophie_objective_release(sophie_grid *g);

/*
 * Batched cavities (the batching form): many independent PEC cavities of
 * uneven sizes sharing dx and dt, advanced together. Each cavity has its own
 * fields, materials (per-cell eps_r / sigma as for sophie_set_materials, its
 * own class and explicit tables) and up to 4 soft sources; its fields are
 * bitwise those of a single grid of the same size run alone. One time step of
 * the whole batch is one persistent launch over a work list of
 * (cavity, tile, z chunk) items: 64 x 16 tiles run the TMA-staged plain step
 * kernel (units walked in list order by the persistent CTAs, each unit taking
 * its cavity's tensor maps and tables from a device descriptor), 32 x tile_y
 * tiles a direct-load kernel whose CTAs take items from a global counter. A
 * run of n steps is recorded into a CUDA graph once and replayed while the
 * same (start step, n, buffer parity) recurs (e.g. reset + n steps). Field
 * storage is float. Indexing within a cavity is that of a single grid.
 *
 * sophie_batch_create: ncav cavities, dims = ncav x {nx, ny, nz} (each in
 *   [1, 4096]); fields zero, vacuum, step 0. Errors: EINVAL, EUNSTABLE,
 *   ENOMEM, ECUDA.
 * sophie_batch_set_materials: eps and sigma hold every cavity's nx*ny*nz
 *   cells (x fastest), cavities one after the other in index order; sigma
 *   NULL = lossless, both NULL = vacuum everywhere. Words and tables are built
 *   on host threads, one cavity per task. Errors: EINVAL, ENOMEM, ECUDA,
 *   ETOOMANYMAT.
 * sophie_batch_add_source: as sophie_add_source, for cavity cav (at most 4
 *   per cavity).
 * sophie_batch_step: advance all cavities by n steps (asynchronous).
 * sophie_batch_energy: W[c] = the energy of cavity c (as sophie_energy), host
 *   array of ncav doubles. Synchronises. Errors: EINVAL, ECUDA, ENONFINITE.
 * sophie_batch_set_fields / get_fields: one component of one cavity, host
 *   array laid out as for sophie_set_fields. Synchronise.
 * sophie_batch_reset: zero all fields, step 0.
 * sophie_batch_configure: tiles (tile_x, tile_y) = (64, 16) or (32, 4|8|16)
 *   (0 = keep), zchunk = z planes per work item (0 = keep), use_graph != 0
 *   records runs into CUDA graphs. Errors: EINVAL, ENOTSUP, ENOMEM.
 * sophie_batch_autotune: times one step for a set of (tiles, z chunk)
 *   candidates of both kernels (trial launches read the current fields and
 *   write the spare buffer, so the state does not advance) and keeps the
 *   fastest. Results do not depend on the choice. Synchronises.
 * sophie_batch_info: total cells, current work items, tiles and z chunk.
 * sophie_batch_sync: wait for the batch's work; ETIMEOUT if a kernel gave up
 *   a bounded wait.
 * sophie_batch_set_stream: a created (non-legacy) stream for later work.
 */
typedef struct sophie_batch sophie_batch;
int sophie_batch_create(int ncav, const int *dims, double dx, double dt, sophie_batch **out);
int sophie_batch_destroy(sophie_batch *b);
int sophie_batch_set_materials(sophie_batch *b, const float *eps_r, const float *sigma);
int sophie_batch_add_source(sophie_batch *b, int cav, int comp, int i, int j, int k, double amp, double f0,
                            double bw, double t0, int kind);
int sophie_batch_step(sophie_batch *b, int n);
int sophie_batch_get_step(sophie_batch *b, long long *n);
int sophie_batch_energy(sophie_batch *b, double *W);
int sophie_batch_set_fields(sophie_batch *b, int cav, int comp, const float *host);
int sophie_batch_get_fields(sophie_batch *b, int cav, int comp, float *host);
int sophie_batch_reset(sophie_batch *b);
int sophie_batch_set_stream(sophie_batch *b, void *cuda_stream);
int sophie_batch_configure(sophie_batch *b, int tile_x, int tile_y, int zchunk, int use_graph);
int sophie_batch_autotune(sophie_batch *b, int *tile_x, int *tile_y, int *zchunk, double *ms_per_step);
int sophie_batch_info(sophie_batch *b, long long *cells, long long *work_items, int *tile_x, int *tile_y,
                      int *zchunk);
int sophie_batch_launch_count(sophie_batch *b, long long *launches);
int sophie_batch_sync(sophie_batch *b);

/*
 * Packed layout of a batch (the batching form with temporal blocking; no
 * counterpart in the paper). sophie_batch_create_packed takes the arguments of
 * sophie_batch_create and places every cavity in ONE grid, each separated from
 * its neighbours (and the grid walls) by a layer of perfectly conducting
 * cells: a conducting cell makes every edge it touches a PEC edge, exactly
 * like a wall, so each cavity evolves bit for bit as it would alone (Sec. 3.3
 * PEC walls; the cells outside the cavities stay zero). A step of the batch
 * is then a step of that grid: the tuned single-grid kernels, temporally
 * blocked with k and the tilings chosen by the grid's autotuner at the first
 * step (or by sophie_batch_autotune), the launches of a run recorded into a
 * CUDA graph and replayed like the work-list layout's. Every sophie_batch_*
 * call applies to a packed batch, with these differences:
 *   - materials: each cavity's words and tables are built as for a single
 *     grid of its size; class materials are shared globally while all
 *     cavities' classes fit the 511-entry table, otherwise those points
 *     become explicit entries (same coefficients, same results);
 *   - sophie_batch_configure accepts only tile_x = tile_y = zchunk = 0 (else
 *     ENOTSUP) and the use_graph flag;
 *   - sophie_batch_info / sophie_batch_autotune: work_items gets the packed
 *     grid's cells, tile_x / tile_y the output tile of its step kernel
 *     ((64 - 2k) x (32 - 2k) blocked, 64 x 16 plain), zchunk 0;
 *   - energies are summed over each cavity's own index points (double), in a
 *     fixed order; they equal the work-list layout's within rounding of the
 *     sum (not bitwise).
 * Field storage is float. Errors: those of sophie_batch_create and of
 * sophie_create_grid for the packed grid (ENOMEM when it does not fit).
 *
 * sophie_batch_pack_plan: the placement alone, on the host (no GPU): origins
 *   gets ncav x {x, y, z}, the first cell of each cavity in the packed grid,
 *   extent the grid's {nx, ny, nz}. Cavities are sorted into rows along x by
 *   z-thickness bands and height, rows stacked along y into layers, layers
 *   along z; several footprints and band widths are tried, the smallest grid
 *   kept. Errors: EINVAL.
 * sophie_batch_layout: *packed = 1 for a packed batch (extent = its grid's
 *   size, *temporal_k = the steps per launch in use), else 0.
 * sophie_batch_cavity_origin: the first cell of cavity cav in the packed grid
 *   (ENOTSUP for the work-list layout).
 */
int sophie_batch_create_packed(int ncav, const int *dims, double dx, double dt, sophie_batch **out);
int sophie_batch_pack_plan(int ncav, const int *dims, int *origins, int *extent);
int sophie_batch_layout(sophie_batch *b, int *packed, int *extent, int *temporal_k);
int sophie_batch_cavity_origin(sophie_batch *b, int cav, int *xyz);

/*
 * Diagnostics (no counterpart in the paper).
 * sophie_check_guards: each field buffer sits between two guard regions
 *   (one z slab of the six components, at least 1 MiB) filled with 0xA5 at
 *   allocation; *bad_bytes gets the number of guard bytes that changed (0
 *   unless a kernel wrote outside its buffer). Synchronises.
 * sophie_batch_check_guards: the same for the guards around a batch's arena.
 * sophie_selftest_wait_timeout: runs a kernel in which one thread waits, with
 *   the bounded wait the step kernels use, for an mbarrier phase that never
 *   completes (nothing arrives); the wait gives up after its 1 s limit and the
 *   kernel sets the grid's error word and returns. *waited_ms gets how long
 *   the wait took. Afterwards sophie_sync reports SOPHIE_ETIMEOUT once (and
 *   clears the word); the grid stays usable.
 * sophie_debug_fail_alloc: the n-th device allocation made by the library
 *   after this call fails as if the device were out of memory (n = 0: off), to
 *   test the ENOMEM paths.
 */
int sophie_check_guards(sophie_grid *g, long long *bad_bytes);
int sophie_batch_check_guards(sophie_batch *b, long long *bad_bytes);
int sophie_selftest_wait_timeout(sophie_grid *g, double *waited_ms);
int sophie_debug_fail_alloc(int n);

/*
 * The host half of sophie_set_materials on its own, without a grid or a GPU
 * (for checking the material words on any machine). For an nx*ny*nz grid
 * with dx, dt and per-cell eps_r / sigma as for sophie_set_materials, built
 * on nthreads host threads (the result does not depend on it):
 *   words      (host, (nz+1)(ny+1)nxp uint32, nxp = nx+1 rounded up to a
 *              multiple of 8): the material word of every index point,
 *              x fastest (no source or probe flags): bit 2 set = explicit
 *              point with entry index = word >> 3, else bits 3..11 / 12..20 /
 *              21..29 = the class of the ex / ey / ez edge (0 = PEC / none);
 *   class_coef (host, 512 x (Ca, Cb) float), class_eps (512 double eps_r):
 *              the class table (class 0 = (0, 0), eps 0);
 *   exp_coef   (host, exp_cap x 3 x (Ca, Cb) float), exp_eps (exp_cap x 3):
 *              the explicit entries (edges ex, ey, ez of each), filled up to
 *              exp_cap; *n_explicit = the number of entries.
 * Errors: EINVAL (NULL, sizes, bad materials as for sophie_set_materials),
 * ETOOMANYMAT.
 */
int sophie_debug_material_tables(int nx, int ny, int nz, double dx, double dt, const float *eps_r, const float *sigma,
                                 int nthreads, unsigned int *words, float *class_coef, double *class_eps,
                                 float *exp_coef, double *exp_eps, long long exp_cap, long long *n_explicit);

/* Message of the last error on this thread ("" if none). */
const char *sophie_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SOPHIE_H */
