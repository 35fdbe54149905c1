/*
 * kl.h -- C ABI of libkl: tunable structured-grid stencil tendencies with
 * capture, tuning, wisdom files and run-time (NVRTC) kernel selection.
 *
 * The operations follow the workflow of Kernel Launcher (Heldens et al.,
 * arXiv 2303.12374): a kernel definition with a configuration space (Sec. 4.1),
 * capturing a launch so it can be replayed offline (Sec. 4.2), tuning it
 * (Sec. 4.3) into a wisdom file of per-device, per-problem-size records
 * (Sec. 4.4), and, at launch, selecting a record and compiling it at run time
 * with NVRTC, cached per problem size (Sec. 4.5).  The kernels are the CFD
 * stencils the paper tunes (Sec. 5.2: MicroHH advec_u and diff_uvw),
 * generalised to the u, v, w momentum tendencies.
 *
 * Conventions for every call:
 *  - Device pointers are CUDA global-memory pointers on the context's device;
 *    host pointers are ordinary process memory.  Each argument says which.
 *  - The caller owns every buffer and stream; the library owns contexts,
 *    compiled modules, internal device buffers and returned strings.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless their comment says they synchronise.
 *  - Errors are returned, never aborted on; kl_last_error() gives the text.
 *    Arguments are validated on the host before any launch; a rejected call
 *    launches nothing.
 *  - Not thread-safe per context: use one context per host thread, or
 *    serialise calls on a shared context.
 */
#ifndef KL_H
#define KL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int kl_status;
#define KL_OK                0
#define KL_ERR_INVALID_ARG  -1   /* bad pointer, size, stride, option or config */
#define KL_ERR_CUDA         -2   /* a CUDA runtime/driver call failed */
#define KL_ERR_NVRTC        -3   /* run-time compilation failed; log in kl_last_error */
#define KL_ERR_IO           -4   /* a file could not be read or written */
#define KL_ERR_WISDOM_PARSE -5   /* malformed wisdom or capture file */
#define KL_ERR_UNSUPPORTED  -6   /* valid request the library or device cannot run */
#define KL_ERR_BOUNDS       -7   /* strides/extent do not hold the stencil footprint */
#define KL_ERR_TIMEOUT      -8   /* a bounded device wait gave up */
#define KL_ERR_OOM          -9   /* a library-internal allocation failed */

typedef enum { KL_F64 = 0, KL_F32 = 1, KL_BF16 = 2, KL_F16 = 3 } kl_dtype;

/*
 * What to compute.  adv: 0 none, 2 centred 2nd-order, 5 upwind-biased
 * 5th-order interpolation in flux-form momentum advection (the 2nd-order
 * scheme with 5th-order face values of Sec. 5.2).  diff: 0 none,
 * 1 constant-nu Laplacian, 2 variable-nu stress divergence (the Smagorinsky
 * diffusion of Sec. 5.2 with a given nu field).  dtype: storage type of every
 * field; f64 computes in f64, the others in f32.  accumulate: 0 writes
 * t = tendency, 1 adds t += tendency.  out_f32: with 16-bit storage, 1 keeps
 * the tendencies in f32 buffers (no output rounding to 16 bits); 0 (and
 * always for f32 and f64) stores them in dtype.
 */
typedef struct {
    int32_t adv;
    int32_t diff;
    int32_t dtype;
    int32_t accumulate;
    int32_t out_f32;    /* 1: ut, vt, wt are f32 buffers (16-bit dtype only); 0: dtype */
} kl_op;

/*
 * Grid and memory layout, shared by every field of a call.
 * Interior points i in [0,nx), j in [0,ny), k in [0,nz); g ghost cells on each
 * side of every axis (g >= 3 for adv = 5, g >= 1 otherwise).  Element
 * (i,j,k) of a field lives at base[origin + i + j*sj + k*sk] (x stride 1);
 * negative i, j, k down to -g and up to n-1+g address the ghosts.  extent is
 * the number of elements of each buffer; every addressed element must lie in
 * [0, extent) and extent must be < 2^31.  Staggering is Arakawa C: u at
 * (i dx, (j+1/2) dy, z_k), v at ((i+1/2) dx, j dy, z_k), w at ((i+1/2) dx,
 * (j+1/2) dy, zh_k), nu at cell centres.  xybc = 0: x and y are periodic
 * and the library forms their ghosts; xybc = 1: the grid is one block of a
 * domain decomposed in x and y, whose x and y ghost cells the caller supplies
 * (kl_halo_pack / kl_halo_unpack below): the ghost fills then write only the
 * z ghost planes (over the padded x-y extent, from the same column) and every
 * kernel reads the x and y ghosts from memory.  zbc = 0 periodic z, zbc = 1
 * free-slip walls at zh_0 and zh_nz (w = 0 there; the w value stored at k = 0
 * must be 0).  zh (HOST, nz+1 face heights, increasing) gives a stretched
 * grid; zh = NULL means uniform spacing dz.  nu is the constant viscosity for
 * diff = 1.
 */
typedef struct {
    int32_t nx, ny, nz;
    int32_t g;
    int64_t sj, sk;
    int64_t origin;
    int64_t extent;
    int32_t zbc;
    int32_t xybc;       /* 0 periodic x, y; 1 x, y ghosts supplied by the caller */
    double dx, dy, dz;
    double nu;
    const double *zh;
} kl_grid;

/* Device pointers to the base (element 0) of each buffer.  nu is read only
 * for diff = 2 (may be NULL otherwise).  Outputs are written on interior
 * points only; their ghosts are untouched. */
typedef struct {
    const void *u, *v, *w, *nu;
    void *ut, *vt, *wt;
} kl_fields;

typedef struct kl_ctx kl_ctx;

/* Create a context on CUDA device `device`.  wisdom_dir (host string, may be
 * NULL) is where kl_launch looks for wisdom files; NULL uses $KL_WISDOM_DIR,
 * else no wisdom (default configurations).  *out receives the context. */
kl_status kl_create(kl_ctx **out, int device, const char *wisdom_dir);

/* Free the context: unloads compiled modules, frees internal device buffers.
 * Synchronises the device.  NULL is ignored. */
void kl_destroy(kl_ctx *ctx);

/* Text of the last error on this host thread (library-owned, never NULL). */
const char *kl_last_error(void);

/* Recommended layout for a field (host arithmetic only): the interior x start
 * and the row pitch are 128-byte aligned.  Writes sj, sk, origin, extent. */
kl_status kl_layout(int32_t nx, int32_t ny, int32_t nz, int32_t g, int32_t dtype,
                    int64_t *sj, int64_t *sk, int64_t *origin, int64_t *extent);

/*
 * Fill the ghost cells of u, v, w (and nu when non-NULL) in place (device
 * pointers, layout `grid`, storage `dtype`): periodic copies in x and y (and z
 * for zbc = 0); at walls u, v, nu are mirrored evenly, w oddly with w = 0 on
 * the top wall face.  Every ghost point is copied straight from an interior
 * point, so edges and corners are filled in the same single launch.  With
 * grid.xybc = 1 only the z ghost planes are written, each ghost from the same
 * (x, y) column (x and y ghost columns included: they hold the exchanged
 * halo), and the x and y ghosts of interior levels are left as they are.
 */
kl_status kl_fill_ghosts(kl_ctx *ctx, int32_t dtype, const kl_grid *grid,
                         void *u, void *v, void *w, void *nu, void *stream);

/*
 * Halo exchange of an (x, y) domain decomposition.  MicroHH, the code whose
 * kernels the paper tunes (Sec. 5.1-5.2), runs one grid split over many GPUs
 * in x and y; each block (grid.xybc = 1) receives its x and y ghost cells
 * from its neighbours.  The exchange runs in two phases so that corners need
 * no diagonal messages: x first (strips of the interior rows), then y (strips
 * that include the x ghosts just received).  These calls move one strip of
 * `nf` fields (1..4; device pointers fields[0..nf-1], layout `grid`, storage
 * dtype) between the padded arrays and a contiguous device buffer `buf`:
 *
 *   axis 0 (x): g columns x ny interior rows x nz interior levels.
 *     pack   side 0: x in [0, g)        side 1: x in [nx - g, nx)
 *     unpack side 0: x in [-g, 0)       side 1: x in [nx, nx + g)
 *   axis 1 (y): nx + 2g columns (x in [-g, nx + g)) x g rows x nz levels.
 *     pack   side 0: y in [0, g)        side 1: y in [ny - g, ny)
 *     unpack side 0: y in [-g, 0)       side 1: y in [ny, ny + g)
 *
 * The buffer holds [field][k][row][column], column fastest; kl_halo_bytes
 * gives its size.  A block sends its side-0 strip to the neighbour below it
 * on that axis (which unpacks it on side 1) and its side-1 strip to the one
 * above (unpacked on side 0); the transport between ranks is the caller's
 * (NCCL send / recv, for instance).  Only interior levels move: after both
 * phases, kl_fill_ghosts with xybc = 1 fills the z ghosts of every column,
 * the received ones included.  Raw bits are copied.  Asynchronous on
 * `stream`.  The buffer must not overlap the fields.
 */
kl_status kl_halo_bytes(const kl_grid *grid, int32_t dtype, int32_t axis, int32_t nf,
                        int64_t *bytes);
kl_status kl_halo_pack(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t axis,
                       int32_t side, int32_t nf, const void *const *fields, void *buf,
                       void *stream);
kl_status kl_halo_unpack(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t axis,
                         int32_t side, int32_t nf, void *const *fields, const void *buf,
                         void *stream);

/*
 * Interior data between a HOST array and a padded DEVICE field of layout
 * `grid` (storage dtype): kl_copy_in copies host[k][j][i] (nz x ny x nx,
 * contiguous, i fastest) to the interior points (i, j, k) of `dev` (the
 * padded buffer's base, as in kl_fields); kl_copy_out copies the interior of
 * `dev` to `host`.  Ghost cells are neither read nor written.  One strided
 * DMA copy per call (the layout's row and plane pitches), asynchronous on
 * `stream` when `host` is page-locked (cudaHostAlloc / cudaHostRegister),
 * otherwise as cudaMemcpy3DAsync behaves for pageable memory.  The copies
 * are the data movement around the paper's hot path (MicroHH keeps its
 * fields on the GPU; a caller whose data starts on the host uses these):
 * no stencil arithmetic.  KL_ERR_INVALID_ARG for NULL pointers, a bad dtype
 * or layout; KL_ERR_CUDA if the copy cannot be issued.
 */
kl_status kl_copy_in(int32_t dtype, const kl_grid *grid, const void *host, void *dev, void *stream);
kl_status kl_copy_out(int32_t dtype, const kl_grid *grid, const void *dev, void *host, void *stream);

/*
 * Tendencies ut, vt, wt of (u, v, w) on the interior (Sec. 5.2 stencils),
 * ghosts of the inputs already filled.  The configuration is selected from
 * the wisdom file of (op, dtype) by the heuristic of Sec. 4.5 and compiled
 * with NVRTC on the first call per problem size; later calls reuse it.
 */
kl_status kl_launch(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                    const kl_fields *fields, void *stream);

/*
 * The ghost fill that the configuration kl_launch selects for (op, grid)
 * reads: as kl_fill_ghosts, except that for a configuration of the zpack
 * family, which forms the periodic x halo of its tiles from interior columns
 * itself, the x ghosts of interior rows of interior levels are not written
 * (left as they were); y rows and z planes, their x ghosts included, are.
 * Same checks as kl_launch; nothing is launched when they fail.
 */
kl_status kl_fill_ghosts_op(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                            const kl_fields *fields, void *stream);

/*
 * One step of the hot path: kl_fill_ghosts_op then kl_launch, both on
 * `stream`, with one configuration selection.  The tendencies equal those of
 * kl_fill_ghosts + kl_launch.  The input fields must be writable (ghosts).
 */
kl_status kl_step(kl_ctx *ctx, const kl_op *op, const kl_grid *grid, const kl_fields *fields,
                  void *stream);

/*
 * As kl_launch with an explicit configuration string.  Configuration strings
 * name a family and its parameters (omitted keys take their defaults):
 *   "default"  the untuned default of Table 2 (direct, 256 x 1 x 1 threads)
 *   "direct:bx=,by=,bz=,tx=,ty=,tz=,ux=,uy=,uz=,cx=,cy=,cz=,perm=,minb="
 *              Table 2: block shape, points per thread, unroll and
 *              consecutive/strided per axis, unravel order (XYZ .. ZYX),
 *              minimum blocks per SM
 *   "zmarch:bx=,by=,px=,py=,kc=,ns=,minb="
 *              z-marching CTAs over a TMA plane ring: threads along x and y,
 *              points per thread along x and y, z levels per CTA, ring slots
 *   "zpack:w=,ly=,kc=,ns=,minb=,yx=,pk=,cs=,pe="
 *              z-marching over 64-column tiles with packed column pairs: warps,
 *              rows per warp, z levels per CTA, ring slots, minimum blocks,
 *              y faces exchanged between warps (yx), packed f32x2 arithmetic
 *              (pk), one warp group per tendency component (cs), persistent
 *              CTAs over (tile, level) ranges (pe: 1 equal ranges, 2 column-
 *              synchronous; kc is then unused)
 * A configuration outside the space or the op's constraints (threads, shared
 * memory, TMA box) is rejected with KL_ERR_INVALID_ARG.
 */
kl_status kl_launch_with_config(kl_ctx *ctx, const kl_op *op, const char *config,
                                const kl_grid *grid, const kl_fields *fields, void *stream);

/*
 * n independent grids (HOST arrays grids[n], fields[n]) of one op.  The
 * batch takes one configuration: the wisdom record tuned for the problem
 * whose point count is nearest to the batch's total (kl_wisdom_select_points,
 * per zbc), since the batch offers the parallelism of all its grids
 * together.  A grid that configuration does not fit (shared memory, TMA box)
 * takes the record of its own nearest tuned size (Sec. 4.5 fuzzy matching,
 * Sec. 6).  Records tuned with persistent CTAs (pe) run here as z chunks of
 * at most 32 levels.  Grids sharing a configuration run in one launch over a
 * device tile table, and the launches of all classes are issued on
 * `stream`; kl_stats reports the classes of the last batch planned.
 */
kl_status kl_launch_batched(kl_ctx *ctx, const kl_op *op, int32_t n, const kl_grid *grids,
                            const kl_fields *fields, void *stream);

/*
 * Shard a batch across `world` ranks with no communication (independent
 * grids, one rank per GPU): longest-processing-time bin packing by interior
 * point count.  Grids go in decreasing order of points[q] (host, n values;
 * ties by index) each to the rank with the least load so far (ties to the
 * lower rank), so every rank computes the same assignment.  The largest rank
 * load is at most (4/3 - 1/(3 world)) times the best possible (Graham's bound
 * for this rule) and at most the mean load plus the largest grid.  Writes
 * the indices owned by `rank`, ascending, to
 * out (host, room for n), their number to *count and their total points to
 * *load (may be NULL).  Host only.
 */
kl_status kl_batch_shard(int32_t n, const int64_t *points, int32_t world, int32_t rank,
                         int32_t *out, int32_t *count, int64_t *load);

/*
 * Capture (Sec. 4.2): synchronise `stream`, copy every input buffer of the
 * launch device->host and write the definition, problem, layout, scalars and
 * data to `path` (host string).  The launch can then be replayed by kl_tune.
 * If $KERNEL_LAUNCHER_CAPTURE lists "tendency" (comma-separated), kl_launch
 * captures into $KL_CAPTURE_DIR (default ".") before it launches.
 */
kl_status kl_capture(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                     const kl_fields *fields, const char *path, void *stream);

/*
 * Tune (Sec. 4.3): replay the capture at capture_path, search the
 * configuration space with the strategy in opts (host string of key=value
 * pairs: strategy=random|exhaustive|local|bayes, budget_s, max_evals, seed,
 * family=direct|zmarch|zpack|all, verify_tol, log=<path of a JSON-lines log>),
 * verify each candidate against the default configuration's output, and
 * append the best record with provenance to the wisdom file wisdom_path.
 * Synchronous; uses its own device buffers.
 */
kl_status kl_tune(kl_ctx *ctx, const char *capture_path, const char *opts,
                  const char *wisdom_path);

/*
 * FP64 diagnostics on the device of a tendency t (device, layout grid, type
 * dtype) against ref (device, same layout, f64; NULL = zero), over the
 * interior: out[6] (host) = {max|t-ref|, rms(t-ref), max|ref|, rms(ref),
 * sum t, sum t*dz}, dz = dz_k (level = 0) or dzh_k (level = 1, w points).
 * Synchronises `stream`.
 */
kl_status kl_diag(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t level,
                  const void *t, const double *ref, double out[6], void *stream);

/*
 * FP64 inner product over the interior of two fields a and b (device, layout
 * grid, both of type dtype): *out (host) = sum a(i,j,k) b(i,j,k) w_k with
 * w_k = dz_k (level = 0, u, v and centre points), dzh_k (level = 1, w
 * points) or 1 (level = -1).  The kinetic-energy tendency of a step (per unit
 * dx dy) is kl_dot(u, ut, 0) + kl_dot(v, vt, 0) + kl_dot(w, wt, 1).  Products
 * of f32 or 16-bit values are formed exactly and summed in float-float within
 * a level, then in FP64.  Synchronises `stream`.
 */
kl_status kl_dot(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, int32_t level, const void *a,
                 const void *b, double *out, void *stream);

/*
 * kl_diag_noalloc: the diagnostics of kl_diag, for callers that may not
 * allocate GPU memory while they run (an application that reserves its whole
 * device-memory budget at start-up and owns the allocator, or a time loop
 * that cannot take cudaMalloc's implicit synchronisation or failure between
 * steps).  The paper has no counterpart; this is a library convenience.
 * It needs no context and calls no allocating routine: its scratch is a
 * static device array of 8192 x 6 + 8 doubles (~384 KB) that every GPU which
 * loads libkl keeps until the process exits, so grids of at most 2^26
 * interior points are accepted (larger ones: KL_ERR_INVALID_ARG, use kl_diag).
 * t, ref, grid, out[6] as for kl_diag; wz (device, nz doubles, may be NULL
 * for weights 1) gives the per-level weight of out[5] = sum t*wz[k].
 * The first call on a device looks up the array's device address (a runtime
 * call), so make it before any stream capture.  Every call reuses the same
 * array: calls that overlap on the GPU race and must be serialised.
 * Synchronises `stream`.
 */
kl_status kl_diag_noalloc(int32_t dtype, const kl_grid *grid, const void *t, const double *ref,
                          const double *wz, double out[6], void *stream);

/*
 * Smagorinsky eddy viscosity, the nu that diff = 2 takes (the "Smagorinsky
 * diffusion" of Sec. 5.2): on `stream`, for every interior cell centre,
 *   nu = (cs * delta_k)^2 * sqrt(2 S_ij S_ij),  delta_k = (dx dy dz_k)^(1/3),
 * S_ij = (d_i u_j + d_j u_i)/2 on the staggered grid: the normal strains at
 * the centre, each shear strain squared on the four edges around the cell and
 * averaged.  u, v, w (device, layout grid, type dtype) are read with every
 * ghost cell filled as kl_fill_ghosts fills them (one ghost cell is enough).
 * The fill of kl_step and kl_fill_ghosts_op may leave the x ghosts of
 * interior rows unfilled (a zpack configuration wraps x itself), so a caller
 * coming from those calls kl_fill_ghosts first.  nu (device, same layout and type, not
 * aliasing them) gets the interior, and with fill_ghosts != 0 also its ghost
 * cells by the rules of kl_fill_ghosts (even mirror at walls).  Arithmetic
 * in f64 for f64 storage, else f32.  KL_ERR_INVALID_ARG for NULL or
 * misaligned fields, a bad dtype or a negative or non-finite cs.  The
 * context keeps one device table of delta_k^2 per vertical grid (dz profile,
 * dx, dy); cs is a kernel argument and creates none.  The first call for a
 * grid allocates its table (cudaMalloc) and uploads it synchronously, so make
 * it before any stream capture; later calls on that grid allocate nothing.
 * Tables are freed by kl_destroy.
 */
kl_status kl_smagorinsky(kl_ctx *ctx, int32_t dtype, const kl_grid *grid, double cs,
                         const void *u, const void *v, const void *w, void *nu,
                         int32_t fill_ghosts, void *stream);

/* Context statistics as JSON into buf (host, n bytes): cache hits/misses,
 * the four first-launch stage times of Sec. 5.6 (wisdom read, NVRTC,
 * module load, launch), launches, and the last selected record. */
kl_status kl_stats(kl_ctx *ctx, char *buf, size_t n);

/* ---- host-only helpers (no GPU needed) -------------------------------- */

/* Normalised text of a configuration ("default" expands to the default of
 * Table 2) into buf; KL_ERR_INVALID_ARG if it violates the space's
 * constraints for op.  family: 0 direct, 1 zmarch. */
kl_status kl_config_normalize(const kl_op *op, const char *config, char *buf, size_t n);

/* Number of configurations of the declared space for op and family, and the
 * idx-th (0-based, constraint-satisfying ones first counted) into buf. */
kl_status kl_space_size(const kl_op *op, int32_t family, int64_t *count);
kl_status kl_space_config(const kl_op *op, int32_t family, int64_t idx, char *buf, size_t n);

/*
 * Surrogate of the tuner's Bayesian optimisation (strategy=bayes; the paper
 * tunes with Bayesian optimisation and random search, Sec. 5.3), usable for
 * any search over encoded configurations.  Gaussian-process regression: the
 * n observations y (host, minimised) at the rows of X (host, n x d,
 * row-major) are standardised to zero mean and unit population variance;
 * prior variance 1 and noise variance `noise` (<= 0: 1e-4) in those units;
 * Matern-5/2 covariance k(r) = (1 + a + a^2/3) exp(-a), a = sqrt(5) r / l,
 * r the Euclidean distance of two rows.  length_scale <= 0 selects l from
 * {0.05, 0.1, 0.2, 0.3, 0.5, 0.75, 1, 1.5, 2, 3} by the log marginal
 * likelihood (first maximum).
 *
 * kl_bo_posterior: the posterior mean and latent variance (y's units) at the
 * m rows of Xq (host, m x d) into mean and var (host, m each); the length
 * scale used into *ls_used (may be NULL).
 *
 * kl_bo_suggest: the np pending rows P (host, np x d; chosen, not yet
 * measured) are added as observations equal to their posterior mean, with
 * the length scale of the fit to y; then the expected improvement over
 * min(y) with margin xi, EI = (b - m - xi) Phi(z) + s phi(z),
 * z = (b - m - xi)/s, of each of the m candidate rows C (host, m x d) goes to
 * ei (host, m; may be NULL) and the index of the largest (first on ties) to
 * *choice.
 *
 * Both: KL_ERR_INVALID_ARG for a non-positive n or d, a NULL array that is
 * needed, a non-finite value, or a covariance that is not positive definite
 * (duplicate rows with noise too small).  Host only, no GPU.
 */
kl_status kl_bo_posterior(int32_t n, int32_t d, const double *X, const double *y, int32_t m,
                          const double *Xq, double length_scale, double noise, double *mean,
                          double *var, double *ls_used);
kl_status kl_bo_suggest(int32_t n, int32_t d, const double *X, const double *y, int32_t np,
                        const double *P, int32_t m, const double *C, double xi,
                        double length_scale, double noise, int32_t *choice, double *ei);

/*
 * On-disk cubin cache.  The first launch of a configuration costs an NVRTC
 * compile (tens of ms; Sec. 5.6 measures the paper's first-launch stages).
 * With a cache directory, a context reads the cubin of every variant it
 * needs from <dir>/kl_<hash>.cubin when present and writes each one it
 * compiles.  A file records the identity of its variant (hash of the kernel
 * source, NVRTC version, target, compile defines) and a checksum; a file
 * that does not match is ignored and rewritten.  Files are written under a
 * temporary name and renamed, so processes may share a directory.  The
 * tuner's candidates are not cached.
 *
 * kl_set_cache_dir: use dir (host string, an existing directory) from now
 * on; NULL or "" turns the cache off.  A context starts with $KL_CACHE_DIR
 * (off if unset).  KL_ERR_IO if dir is not a directory.
 *
 * kl_cache_prepare (host only, no GPU): compile one configuration for op
 * (same configuration text as kl_compile_only, "batch+" prefix for the
 * batched variant) into dir unless it is already there; *hit (host) is 1 if
 * it was.  This is the variant a context with the default wait limit
 * launches, so a cache can be filled ahead of time from the wisdom records.
 * KL_ERR_INVALID_ARG for a bad op or configuration, KL_ERR_IO if dir is not
 * a writable directory, KL_ERR_NVRTC if compilation fails.
 */
kl_status kl_set_cache_dir(kl_ctx *ctx, const char *dir);
kl_status kl_cache_prepare(const char *dir, const kl_op *op, const char *config, int32_t zbc,
                           int32_t zuni, int32_t *hit);

/* ---- user-defined tunable kernels (Sec. 4.1 for any kernel) ------------ */

/*
 * A kernel definition: CUDA source text (host string, compiled by NVRTC for
 * sm_103a with -std=c++17), the name of its __global__ function (an
 * extern "C" name or a C++ name expression such as "scale<float>"), and a
 * name (a C identifier) that names its wisdom file <wisdom dir>/<name>.wisdom.
 * Tunable parameters, restrictions, geometry and extra compile options are
 * added with the calls below.  The definition owns copies of all strings;
 * it is host data, usable with any context.  Like a context, one definition
 * must not be used by two host threads at once (launches record their
 * selection in it).
 */
typedef struct kl_def kl_def;

/* One launch argument.  kind 0: a scalar, ptr points to its value (host),
 * bytes its size (1..64).  kind 1 input, 2 output, 3 input and output: a
 * device buffer at ptr of `bytes` bytes; dtype says how tuning compares its
 * contents (0 f64, 1 f32, 2 bf16, 3 f16: relative to the largest reference
 * magnitude; 4 i32, 5 raw bytes: exactly).  Arguments are passed to the
 * kernel in order, buffers as their device pointer. */
typedef struct {
    const void *ptr;
    int64_t bytes;
    int32_t kind;
    int32_t dtype;
} kl_arg;

kl_status kl_def_create(kl_def **out, const char *name, const char *source, const char *function);
void      kl_def_destroy(kl_def *def);

/* A tunable parameter: name (a C identifier; problem_x/y/z are reserved),
 * n distinct values (host) and the default, one of them.  Each compiled
 * variant gets -D<name>=<value> for every parameter.  The raw space is the
 * product of the value lists; its index runs over the first parameter
 * fastest. */
kl_status kl_def_param(kl_def *def, const char *name, int32_t n, const int64_t *values,
                       int64_t default_value);

/* A restriction: an integer expression over the declared parameters (C
 * syntax: + - * / % comparisons && || ! ?: and min, max, div_ceil, round_up)
 * that every configuration must make non-zero. */
kl_status kl_def_restrict(kl_def *def, const char *expr);

/* Launch geometry as integer expressions over the parameters and the
 * problem size problem_x, problem_y, problem_z: block[3], grid[3] (each may
 * be NULL or "") and the dynamic shared memory in bytes.  Defaults: block 1,
 * grid div_ceil(problem, block), no shared memory.  A configuration whose
 * block exceeds 1024 threads, whose grid is below 1 or above the device
 * limits, or whose shared memory exceeds 227 KB does not apply to that
 * problem. */
kl_status kl_def_geometry(kl_def *def, const char *const block[3], const char *const grid[3],
                          const char *shared_memory);

/* Extra NVRTC options (host string, space-separated; e.g. "-DT=float"). */
kl_status kl_def_options(kl_def *def, const char *options);

/* Host-only queries (no GPU): raw space size and the number of
 * configurations that satisfy the restrictions (-1 above 10^7 raw points);
 * the idx-th raw configuration as text "p=v,...", KL_ERR_INVALID_ARG if it
 * violates a restriction (text still written); the normalised text of a
 * configuration ("default" or p=v pairs; unnamed parameters keep their
 * defaults); the geometry {block x,y,z, grid x,y,z, shared bytes} of a
 * configuration for a problem; an NVRTC compile with the ptxas log. */
kl_status kl_def_space_size(const kl_def *def, int64_t *raw, int64_t *valid);
kl_status kl_def_config_at(const kl_def *def, int64_t idx, char *buf, size_t n);
kl_status kl_def_normalize(const kl_def *def, const char *config, char *buf, size_t n);
kl_status kl_def_launch_geometry(const kl_def *def, const char *config, const int64_t problem[3],
                                 int64_t out[7]);
kl_status kl_def_compile_only(const kl_def *def, const char *config, char *log, size_t n);

/*
 * Launch (Sec. 4.5): select the record of <wisdom dir>/<name>.wisdom for
 * this device and problem size (problem[3], host) by the rules of
 * kl_wisdom_select (zbc 0), falling back to the default when no record
 * applies to the problem; compile it with NVRTC once per context (or read it
 * from the context's cubin cache) and launch on `stream` with the nargs
 * arguments (host array).  The selection is made once per context, wisdom
 * directory and problem size.  kl_def_launch_config launches a given
 * configuration.  kl_def_selected: the configuration of the last launch and
 * the rule (1..5) of the last selection.
 */
kl_status kl_def_launch(kl_ctx *ctx, kl_def *def, const int64_t problem[3], int32_t nargs,
                        const kl_arg *args, void *stream);
kl_status kl_def_launch_config(kl_ctx *ctx, kl_def *def, const char *config,
                               const int64_t problem[3], int32_t nargs, const kl_arg *args,
                               void *stream);
kl_status kl_def_selected(const kl_def *def, char *buf, size_t n, int32_t *rule);

/*
 * Capture (Sec. 4.2): synchronise `stream`, then write the problem size,
 * the argument list and the contents of every scalar, input and in/out
 * buffer to `path` (outputs: size only).  kl_def_tune replays it: the
 * default configuration's outputs are the reference, every candidate runs
 * from the captured inputs (in/out buffers restored, outputs filled with
 * 0xff bytes) and must match it (verify_tol, else 1e-12 f64, 1e-5 f32, 1e-2
 * 16-bit, exact for i32/bytes); options as kl_tune (strategy=random|
 * exhaustive|bayes, budget_s, max_evals, seed, verify_tol, log, reps, warm,
 * threads).  The fastest of the three best candidates and the default,
 * re-timed, is appended to wisdom_path.  Synchronous; its own device buffers.
 */
kl_status kl_def_capture(kl_ctx *ctx, const kl_def *def, const int64_t problem[3], int32_t nargs,
                         const kl_arg *args, const char *path, void *stream);
kl_status kl_def_tune(kl_ctx *ctx, kl_def *def, const char *capture_path, const char *opts,
                      const char *wisdom_path);

/* Compile a configuration with NVRTC for sm_103a without loading it; the
 * compiler log (with ptxas register/spill lines) goes to log (host, n). */
kl_status kl_compile_only(const kl_op *op, const char *config, int32_t zbc, int32_t zuni,
                          char *log, size_t n);

/*
 * Wisdom selection (Sec. 4.5) over the file at path: the record matching
 * device name and size (several such records, one per tuning session: the
 * fastest, ties to the newest); else the same device, nearest size (Euclidean);
 * else the same architecture (compute capability), nearest size; else any
 * record, nearest size; else (empty, missing or unreadable file) the
 * default.  Records of another zbc are never chosen.  Writes the chosen
 * configuration to cfg (host, n) and the rule that fired (1..5) to *rule.
 */
kl_status kl_wisdom_select(const char *path, const char *device, int32_t cc_major,
                           int32_t cc_minor, int32_t zbc, int32_t nx, int32_t ny, int32_t nz,
                           char *cfg, size_t n, int32_t *rule);

/*
 * The selection kl_launch_batched makes for a batch of `points` interior
 * points in all: rules 2..5 of kl_wisdom_select with the distance between a
 * record and the batch taken as |ln(record nx*ny*nz) - ln(points)| (no rule
 * 1).  Same arguments, output and error behaviour as kl_wisdom_select.
 */
kl_status kl_wisdom_select_points(const char *path, const char *device, int32_t cc_major,
                                  int32_t cc_minor, int32_t zbc, int64_t points, char *cfg,
                                  size_t n, int32_t *rule);

/* Append one record (host strings) to the wisdom file at path, creating it. */
kl_status kl_wisdom_append(const char *path, const char *device, int32_t cc_major,
                           int32_t cc_minor, int32_t zbc, int32_t nx, int32_t ny, int32_t nz,
                           const char *config, double time_us, const char *extra);

/*
 * Failure detection.  Every device wait of the kernels (for a TMA copy into
 * shared memory) is bounded; a wait that gives up makes its CTA record
 * KL_ERR_TIMEOUT in the context's device status word, wait (bounded) for its
 * copies still in flight and return, so the GPU and the context stay usable.
 * kl_check synchronises `stream`, reads and clears that word: KL_OK, or
 * KL_ERR_TIMEOUT when a launch since the last check gave up somewhere (its
 * outputs are then incomplete).  kl_set_wait_limit sets the limit of one wait
 * in SM clock cycles for later launches (0 restores the default, 2^31, about
 * a second); the waits for in-flight copies keep the default.  A context with
 * a non-default limit compiles separate kernels whose waits poll against it.
 */
kl_status kl_check(kl_ctx *ctx, void *stream);
kl_status kl_set_wait_limit(kl_ctx *ctx, int64_t cycles);

/* Library version string (static). */
const char *kl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KL_H */
