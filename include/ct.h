/*
 * ct.h -- C ABI of the GB300 (sm_103a) cone-beam CT operator and Krylov solvers.
 *
 * The operator is the sparse CBCT system matrix A of Materials and Methods
 * (Eq. 1, b = A x), never stored: A_ij is the length in mm of ray i inside
 * voxel j (the Siddon ray-caster named in the Software section).  The
 * solvers are CGLS with delayed residual computation (Algorithm 1) and LSQR
 * (Paige & Saunders 1982, cited in Materials and Methods), with the diagonal
 * preconditioners of the Software and Discussion sections.
 *
 * Conventions (the paper fixes none of them; every call uses these):
 *   lengths in mm, angles in radians;
 *   circular orbit about +z: source s = SID (cos th, sin th, 0);
 *   flat detector centred at -(SDD - SID) (cos th, sin th, 0) with axes
 *   e_u = (-sin th, cos th, 0) and e_v = (0, 0, 1);
 *   pixel (u, v) centre = centre + ((u - (nu-1)/2) du + det_off_u) e_u
 *                                + ((v - (nv-1)/2) dv + det_off_v) e_v;
 *   one ray per pixel, from the source to the pixel centre;
 *   volume box = [-n h / 2 + off, +n h / 2 + off] per axis (off-centre
 *   reconstruction, Software section);
 *   volume  float32 [nz][ny][nx], x fastest;
 *   sinogram float32 [nviews][nv][nu], u fastest.
 *
 * Memory: every vector argument named d_* is a DEVICE pointer on the device
 * that was current when the geometry was created; the caller owns it.  The
 * library owns the geometry and any workspace it allocates (stream-ordered,
 * cudaMallocAsync / cudaFreeAsync on the call's stream).
 *
 * Streams: ``stream`` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  ct_project / ct_backproject / ct_project_norm2 only
 * enqueue work and return; ct_count_nnz, ct_precond_weights, ct_cgls and
 * ct_lsqr return after the stream has completed their work.
 *
 * Errors: every call validates its arguments and returns a ct_status; it
 * never aborts.  ct_last_error() gives a message for the calling thread's
 * last failure.  A CT_ERR_CUDA status leaves the CUDA error in the message.
 */
#ifndef CT_H
#define CT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_ERR_INVALID_ARG = 1, /* NULL pointer, bad size, unsupported option   */
    CT_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed  */
    CT_ERR_OOM = 3,         /* device workspace allocation failed           */
    CT_ERR_TIMEOUT = 4,     /* reserved: a bounded device wait gave up      */
    CT_ERR_INTERNAL = 5     /* a device-side consistency check failed       */
} ct_status;

/* Storage element type of a volume or sinogram.  Arithmetic is FP32 along
 * each ray (and FP64 for the Krylov scalars) whatever the storage; BF16/FP16
 * only change what is read and what is rounded on store (the Discussion notes
 * that much of the double precision could give way to lower precision). */
typedef enum { CT_F32 = 0, CT_BF16 = 1, CT_F16 = 2 } ct_dtype;

/* Opaque geometry: per-view ray constants on the device, library-owned. */
typedef struct ct_geometry ct_geometry;

/* Caller-owned description of the scan (Results section: a C-arm-like
 * circular cone-beam orbit).  angles_rad may be NULL: views are then
 * 2 pi k / nviews, k = 0 .. nviews-1 (uniform over 360 degrees, endpoint
 * excluded).  Otherwise it points to nviews host doubles, copied at create. */
typedef struct {
    int32_t nx, ny, nz;          /* volume size in voxels                    */
    double vx, vy, vz;           /* voxel pitch, mm                          */
    double off_x, off_y, off_z;  /* volume centre, mm (off-centre recon)     */
    int32_t nu, nv;              /* detector size in pixels                  */
    double du, dv;               /* pixel pitch, mm                          */
    double det_off_u, det_off_v; /* detector shift along e_u / e_v, mm       */
    double sid, sdd;             /* source-isocentre, source-detector, mm    */
    int32_t nviews;              /* number of views                          */
    const double *angles_rad;    /* NULL or nviews view angles               */
} ct_geometry_desc;

/* Create a geometry on the current CUDA device.  Requires nx, ny, nz >= 1,
 * nu, nv, nviews >= 0, positive pitches, 0 < sid < sdd, fewer than 2^31
 * voxels, nx * ny < 2^31, nx, ny, nz <= 65535 (the walks' integer lines stay
 * inside int64), nviews <= 65535 and nv <= 524280 (CUDA grid limits);
 * anything else is CT_ERR_INVALID_ARG.  *out receives the handle. */
ct_status ct_geometry_create(const ct_geometry_desc *desc, ct_geometry **out);

/* Free the geometry (NULL is a no-op).  No call using it may be in flight. */
void ct_geometry_destroy(ct_geometry *g);

/* Deterministic accumulation (default off).  When on, every scatter with
 * this geometry sums its contributions as 64-bit fixed-point integers: each
 * value is scaled by a power of two chosen from max |input| and a bound on
 * the sum, rounded to an integer and added with integer atomics.  Integer
 * addition does not depend on order, so results are bitwise reproducible
 * from run to run and independent of other work sharing the GPU; each
 * contribution is rounded to a multiple of at most 2^-61 times the bound.
 * Siddon: the backprojections (ct_backproject, the solvers, the
 * preconditioner weights) scatter; the bound is the rays through one voxel
 * times the longest chord; 16 bytes per voxel of workspace.  Footprint
 * projectors: the forward projection scatters; the bound is the voxel count
 * times the longest footprint amplitude; 8 bytes per ray of workspace (which
 * ct_project_norm2_noalloc cannot take).  The other direction of each
 * projector, the vector updates and the FP64 reductions are deterministic in
 * both modes.  Change the mode only while no call on this geometry is in
 * flight. */
ct_status ct_geometry_set_deterministic(ct_geometry *g, int32_t on);

/* Projector of a geometry (Materials and Methods names Siddon, the TT
 * footprint projector of Long et al. 2010 and cutting voxels).
 *   CT_PROJ_SIDDON: A_ij = length in mm of the pixel-centre ray i in voxel j
 *                   (the default).
 *   CT_PROJ_SF_TR / CT_PROJ_SF_TT: separable footprints averaged over the
 *                   detector cell: A_ij = l_j Fbar_u Fbar_v, with the
 *                   transaxial footprint the trapezoid of the voxel's four
 *                   projected vertical edges, the axial one a rectangle (TR)
 *                   or the trapezoid of the z faces projected at the nearest
 *                   and farthest corner depths (TT), and l_j the chord of the
 *                   ray through the voxel centre across its x and y faces.
 * The same matrix serves ct_project, ct_backproject (exactly adjoint), the
 * solvers and the preconditioner weights.  The footprint projectors need
 * FP32 storage (CT_ERR_INVALID_ARG for BF16/FP16 in ct_project_ex,
 * ct_backproject_ex and the solvers' storage), scatter their forward
 * projection (float atomics, or int64 fixed point in deterministic mode)
 * and gather their backprojection (reproducible in both modes), and
 * need ny <= 524280 and the volume's xy extent inside the source circle
 * (every voxel in front of the source).  Change the projector only while no
 * call on this geometry is in flight. */
typedef enum { CT_PROJ_SIDDON = 0, CT_PROJ_SF_TR = 1, CT_PROJ_SF_TT = 2 } ct_projector;
ct_status ct_geometry_set_projector(ct_geometry *g, int32_t kind);

/* Sizes of the geometry: voxels (n = nx ny nz) and rays (m = nviews nv nu). */
ct_status ct_geometry_sizes(const ct_geometry *g, int64_t *n_vox, int64_t *n_rays);

/* Forward projection (Eq. 1; Algorithm 1 steps p_b = A x and p_b = A d_x):
 *   d_sino = alpha * (A d_vol) + beta * d_sino.
 * With beta == 0, d_sino is not read (it may hold anything).  d_vol and
 * d_sino must not overlap. */
ct_status ct_project(const ct_geometry *g, const float *d_vol, float *d_sino, float alpha,
                     float beta, void *stream);

/* Backprojection, the exact transpose of ct_project (Algorithm 1 step
 * r_x = A^T e_b):   d_vol = alpha * (A^T d_sino) + beta * d_vol.
 * With beta == 0, d_vol is not read.  With the Siddon projector the sums are
 * accumulated with float atomics, so the last bits may differ between runs
 * (see ct_geometry_set_deterministic); the footprint projectors gather, and
 * their backprojection is reproducible. */
ct_status ct_backproject(const ct_geometry *g, const float *d_sino, float *d_vol, float alpha,
                         float beta, void *stream);

/* ct_project applied to each item of a batch of volumes of one geometry
 * (Eq. 1, item by item): for i < nbatch,
 *   d_sinos[i m ..] = alpha * (A d_vols[i n ..]) + beta * d_sinos[i m ..],
 * with n = nx ny nz and m = nviews nv nu; both arrays hold nbatch contiguous
 * items (device pointers, caller-owned).  For a column-major Siddon
 * geometry the projector is one launch over all items, each item's result
 * bitwise that of ct_project; otherwise the items run one after another.
 * Uses a stream-ordered workspace of nbatch * n floats.  nbatch == 0 does
 * nothing; nbatch < 0 or a NULL vector gives CT_ERR_INVALID_ARG. */
ct_status ct_project_batch(const ct_geometry *g, const float *d_vols, float *d_sinos,
                           int32_t nbatch, float alpha, float beta, void *stream);

/* ct_backproject applied to each item of a batch of sinograms (Algorithm 1
 * step r_x = A^T e_b, item by item), in the same layout:
 *   d_vols[i n ..] = alpha * (A^T d_sinos[i m ..]) + beta * d_vols[i n ..].
 * One projector launch over all items for a column-major Siddon geometry
 * with float accumulation (results as ct_backproject's, up to the order of
 * the float atomics); item by item otherwise.  Workspace nbatch * n floats. */
ct_status ct_backproject_batch(const ct_geometry *g, const float *d_sinos, float *d_vols,
                               int32_t nbatch, float alpha, float beta, void *stream);

/* ct_project / ct_backproject with typed storage: d_vol holds vol_dtype and
 * d_sino sino_dtype elements (ct_dtype).  Values are read and converted to
 * FP32, every ray or voxel sum is accumulated in FP32, and the result is
 * rounded to the output type on store (round to nearest even).  Same layouts,
 * alpha/beta semantics and errors as the FP32 calls. */
ct_status ct_project_ex(const ct_geometry *g, const void *d_vol, int32_t vol_dtype, void *d_sino,
                        int32_t sino_dtype, float alpha, float beta, void *stream);
ct_status ct_backproject_ex(const ct_geometry *g, const void *d_sino, int32_t sino_dtype,
                            void *d_vol, int32_t vol_dtype, float alpha, float beta,
                            void *stream);

/* ct_project plus the squared norm of the result (Algorithm 1 step
 * NP2 = ||p_b||_2^2), accumulated in FP64 in a fixed order (deterministic):
 *   d_sino = alpha * (A d_vol) + beta * d_sino;  *d_norm2 = ||d_sino||^2.
 * d_norm2 is a DEVICE pointer to one double.  Uses a stream-ordered
 * device workspace of 8 bytes per 256 rays. */
ct_status ct_project_norm2(const ct_geometry *g, const float *d_vol, float *d_sino, float alpha,
                           float beta, double *d_norm2, void *stream);

/* ct_project_norm2 without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot let a library allocate device
 * memory once they run (a service that reserves HBM up front for its own
 * pool, or a real-time pipeline whose latency budget has no room for an
 * allocator call).  Same arguments and results as ct_project_norm2; the
 * volume is read in place, and the FP64 partial sums live in a fixed 2 MiB
 * device array that every GPU loading the library holds until exit.
 * Limit (Siddon): the launch's CTA count, ceil(nu/32) * ceil(nv/8) * V,
 * must not exceed 262144, where V = nviews rounded up to a multiple of the
 * view group G = ceil(nviews / floor(65535 / ceil(nv/8))) (G = 1, V = nviews,
 * unless nviews * ceil(nv/8) > 65535); else CT_ERR_INVALID_ARG with a message
 * giving the count.  The footprint projectors need at most 1216 partials;
 * a deterministic footprint geometry (which sums in int64 workspace) is
 * rejected with CT_ERR_INVALID_ARG.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  The address stays cached for the life of the process:
 * do not call this entry point on a device after a device reset
 * (cudaDeviceReset), which moves the array and also invalidates every
 * geometry created on that device before it.  All calls share the array: calls that overlap on the
 * GPU (other streams, other threads) race on it and must be serialised by the
 * caller.  Each call overwrites what it reads, so the contents a previous
 * call left behind never matter.  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
ct_status ct_project_norm2_noalloc(const ct_geometry *g, const float *d_vol, float *d_sino,
                                   float alpha, float beta, double *d_norm2, void *stream);

/* Bounds checking (no counterpart in the paper).  The library built with
 * -DCT_DEBUG_BOUNDS (libct_gb300_debug.so) checks every voxel and
 * detector-pixel index its projector kernels are about to touch; an index
 * out of range is not accessed, and the first one records its source line.
 * ct_debug_status waits for the current device, then returns
 * CT_ERR_INTERNAL (message: file and line) if a violation was recorded
 * since the last call, and clears it; CT_OK otherwise (always, in the normal
 * build).  ct_debug_bounds_build returns 1 in the checking build, else 0. */
ct_status ct_debug_status(void);
int32_t ct_debug_bounds_build(void);

/* Number of (ray, voxel) pairs with positive intersection length, i.e. the
 * nonzeros of A (the unit of the ray-voxel update rate).  *out is a HOST
 * int64.  Blocks until done. */
ct_status ct_count_nnz(const ct_geometry *g, int64_t *out, void *stream);
/* (With a footprint projector: the (ray, voxel) pairs with a positive
 * footprint weight.) */

typedef enum {
    CT_PRECOND_NONE = 0,
    /* Jacobi (Software and Discussion sections): the normal-equation
     * matrix A^T A approximated by its diagonal; x = D^-1/2 y. */
    CT_PRECOND_JACOBI = 1,
    /* Diagonal row/column sums: min || R^-1/2 (A C^-1/2 y - b) ||, x = C^-1/2 y,
     * R = A 1 (row sums), C = A^T 1 (column sums).  Left scaling changes the
     * least-squares solution when b is inconsistent (it weights the rays). */
    CT_PRECOND_ROWCOL = 2
} ct_precond;

/* Preconditioner weights.  JACOBI: d_vol_w = diag(A^T A)^-1/2 (d_sino_w
 * unused, may be NULL).  ROWCOL: d_sino_w = (A 1)^-1/2, d_vol_w = (A^T 1)^-1/2.
 * Entries whose sum is <= 1e-6 times the largest are set to 0: those voxels
 * or rays carry no data (the tiny cone-boundary values of the Discussion).
 * Blocks until done. */
ct_status ct_precond_weights(const ct_geometry *g, int32_t kind, float *d_vol_w, float *d_sino_w,
                             void *stream);

/* Solver options (Algorithm 1 input: x0, ERR, K; Software section:
 * preconditioning; Discussion: periodic recomputation of the discrepancy). */
typedef struct {
    int32_t max_iter;        /* K >= 1: number of x updates at most            */
    double err_tol;          /* ERR >= 0: stop once NB / NB0 <= ERR            */
    int32_t precond;         /* a ct_precond value                            */
    double tikhonov_lambda;  /* lam >= 0 (Software section: Tikhonov
                                regularisation).  CGLS minimises
                                ||L (A x - b)||^2 + lam ||x||^2 (L: ROWCOL
                                row weights, else 1); NB and the stopping
                                test stay on the data term ||L (b - A x)||.
                                LSQR: must be 0. */
    int32_t recompute_every; /* k > 0: e_b = b - A x every k updates (CGLS)    */
    int32_t timing;          /* nonzero: time every A and A^T with CUDA events
                                and launch every kernel directly.  Otherwise
                                (and with recompute_every == 0) one update is
                                captured as a CUDA graph on a private stream
                                and replayed on `stream`, one graph launch per
                                update; results are the same. */
    int32_t storage;         /* ct_dtype of the Krylov vectors d_x, e_b, p_b
                                (CGLS; LSQR needs CT_F32).  x and the
                                backprojection sums stay FP32. */
} ct_solver_opts;

/* Solver report, filled on return.  history_nb (HOST, caller-owned, may be
 * NULL) receives NB / NB0 after each x update, up to history_cap entries.
 * For LSQR, NB is the recurrence estimate phi_bar of the discrepancy.  With
 * preconditioning the discrepancy is the weighted one, || R^-1/2 (b - A x) ||
 * for ROWCOL.  history_nr (HOST, caller-owned, may be NULL; history_cap
 * entries) receives for each x update the norm of the least-squares
 * gradient at the iterate before it (x0 for the first): ||A^T e_b||, the
 * NR of Algorithm 1 for CGLS (computed), the Paige-Saunders estimate
 * phi_bar alpha |c| for LSQR; with preconditioning ||W A^T L e||, with
 * Tikhonov the regularised gradient.  SIRT leaves it untouched. */
typedef struct {
    int32_t iterations;   /* i of Algorithm 1: x updates done               */
    double nb0, nb;       /* NB0 = ||b|| and the final NB                   */
    double *history_nb;   /* in: host array or NULL                         */
    int32_t history_cap;  /* in: its length (also of history_nr)            */
    int32_t n_forward;    /* operator calls made: A                         */
    int32_t n_back;       /* operator calls made: A^T                       */
    double ms_forward;    /* with opts.timing: total device time in A, ms   */
    double ms_back;       /* with opts.timing: total device time in A^T, ms */
    double *history_nr;   /* in: host array or NULL (see above)             */
} ct_solver_report;

/* CGLS with delayed residual computation (Algorithm 1, with the direction
 * update read as d_x = r_x + beta d_x).  d_b: sinogram (device, read only);
 * d_x: in = x0, out = x (device).  A zero x0 skips the A x0 call, so K updates
 * cost 2K operator calls (2K + 1 with a nonzero x0).  Device workspace:
 * 3 volumes + 2 sinograms (+ weights).  Blocks until done. */
ct_status ct_cgls(const ct_geometry *g, const float *d_b, float *d_x, const ct_solver_opts *opts,
                  ct_solver_report *report, void *stream);
/* (The solvers return CT_ERR_INVALID_ARG when ||b|| or the final discrepancy
 * is not finite: NaN or Inf in b or x0 propagates into every later value.
 * With err_tol > 0 the iterations stop at the first such value.) */

/* Checkpoint / resume of CGLS (no counterpart in the paper; Algorithm 1 needs
 * only x, d_x, e_b and the scalars NB0, NR2 between two updates).  A state is
 * library-owned device memory for those vectors (2 volumes + 1 sinogram,
 * FP32) plus the scalars and the history, for one geometry size and device.
 * ct_cgls_resume runs CGLS like ct_cgls, FP32 storage only, continuing from
 * the state when it holds updates (d_x's input is then ignored; else d_x is
 * x0), until the TOTAL update count reaches max_iter or the stopping rule
 * fires, saves the state and returns x in d_x; the report covers all updates
 * so far.  With a deterministic geometry a run resumed from a state is
 * bitwise equal to the uninterrupted run.  export writes the state to host
 * bytes (host NULL: only *bytes), import reads such bytes back (same
 * sizes, same library version, else CT_ERR_INVALID_ARG). */
typedef struct ct_cgls_state ct_cgls_state;
ct_status ct_cgls_state_create(const ct_geometry *g, ct_cgls_state **out);
void ct_cgls_state_destroy(ct_cgls_state *state);
ct_status ct_cgls_state_iterations(const ct_cgls_state *state, int32_t *iterations);
ct_status ct_cgls_state_export(const ct_cgls_state *state, void *host, int64_t capacity,
                               int64_t *bytes);
ct_status ct_cgls_state_import(ct_cgls_state *state, const void *host, int64_t bytes);
ct_status ct_cgls_resume(const ct_geometry *g, const float *d_b, float *d_x,
                         const ct_solver_opts *opts, ct_solver_report *report,
                         ct_cgls_state *state, void *stream);

/* LSQR (Paige & Saunders 1982) on the same operator; K iterations cost
 * 2K + 1 operator calls (+1 with a nonzero x0).  Same arguments as ct_cgls;
 * recompute_every is ignored.  Blocks until done. */
ct_status ct_lsqr(const ct_geometry *g, const float *d_b, float *d_x, const ct_solver_opts *opts,
                  ct_solver_report *report, void *stream);

/* SIRT options (ct_sirt). */
typedef struct {
    int32_t max_iter;   /* K >= 1: number of x updates at most                 */
    double err_tol;     /* ERR >= 0: stop once ||b - A x|| / ||b|| <= ERR      */
    double relax;       /* step lam in (0, 2): 1 = SIRT, 1.5 = PSIRT           */
    int32_t timing;     /* nonzero: time every A and A^T with CUDA events      */
} ct_sirt_opts;

/* SIRT and its over-relaxed PSIRT reading, the classical comparison methods
 * of the Software and Results sections (the paper gives no formula):
 *   x = x + relax * C^-1 A^T R^-1 (b - A x),  R = A 1, C = A^T 1,
 * with row or column sums <= 1e-6 of their maximum given weight 0 (no data
 * there).  PSIRT is read as relax = 2 / (1 + eps) with eps = 1/3, i.e. 1.5.
 * d_b: sinogram (device, read only); d_x: in = x0, out = x (device).  Each
 * update costs one A^T and one A (the discrepancy b - A x is recomputed, so
 * NB in the report is ||b - A x|| of the returned x, NB0 = ||b||).  The
 * report's history holds NB / NB0 after each update.  Device workspace:
 * 2 volumes + 2 sinograms + the weights.  Blocks until done. */
ct_status ct_sirt(const ct_geometry *g, const float *d_b, float *d_x, const ct_sirt_opts *opts,
                  ct_solver_report *report, void *stream);

/* ---- batched CGLS (continuous batching of several solves) ----------------
 *
 * A ct_batch advances several independent CGLS solves (Algorithm 1, each
 * with its own geometry, data and options) in lock step: every
 * ct_batch_step performs one x update of every active job.  The A^T of all
 * jobs whose geometry uses the column-major Siddon kernels runs as ONE
 * persistent kernel launch over all their rays (jobs with fixed-point
 * backprojection in a second one), and likewise their A; the other jobs
 * (ray-major geometries, footprint projectors) launch their own projectors
 * inside the same step.  The step of a fixed set of jobs is captured as a
 * CUDA graph and replayed until a job joins or leaves.  Each job's arithmetic
 * is exactly that of ct_cgls with the same arguments, tile for tile: with a
 * deterministic geometry (ct_geometry_set_deterministic) x and the report are
 * bitwise those of a ct_cgls call; with float-atomic backprojection they
 * agree to the run-to-run rounding of the atomics.
 *
 * Jobs join between steps (ct_batch_add_cgls) and leave when their stopping
 * rule fires (i = K or NB / NB0 <= ERR, tested after every step) or when
 * removed.  A batch belongs to the device current at ct_batch_create and to
 * one host thread at a time; all its work is enqueued on `stream`.  The
 * caller keeps every geometry, d_b and d_x alive until the job is removed or
 * the batch destroyed.  Device workspace per job: that of ct_cgls. */
typedef struct ct_batch ct_batch;

/* New empty batch whose work runs on `stream` (a cudaStream_t, NULL = the
 * legacy default stream).  Free with ct_batch_destroy. */
ct_status ct_batch_create(void *stream, ct_batch **out);
/* Waits for the batch's stream, then frees the batch and its jobs' workspace
 * (the x of an unfinished job keeps its last completed update).  NULL: no-op. */
ct_status ct_batch_destroy(ct_batch *b);
/* Adds a CGLS job: d_b (device, read only) and d_x (device, in = x0, out = x)
 * as for ct_cgls, opts with storage CT_F32, timing 0 and recompute_every 0
 * (else CT_ERR_INVALID_ARG).  Runs the initialisation and the first update
 * on the batch's stream before returning (blocking), and returns the job's
 * id in *job.  A job whose stopping rule already holds is done at once. */
ct_status ct_batch_add_cgls(ct_batch *b, const ct_geometry *g, const float *d_b, float *d_x,
                            const ct_solver_opts *opts, int32_t *job);
/* One x update of every active job, then the stopping rules (one host wait
 * for the jobs with err_tol > 0).  *n_active: jobs still active afterwards.
 * A job that stops here gets its final x and report (blocking). */
ct_status ct_batch_step(ct_batch *b, int32_t *n_active);
/* *done = 1 once job has stopped; then, if report is not NULL, fills it as
 * ct_cgls would (history_nb / history_cap are the caller's, as there).  An
 * unknown id is CT_ERR_INVALID_ARG. */
ct_status ct_batch_poll(ct_batch *b, int32_t job, int32_t *done, ct_solver_report *report);
/* Removes a job (finishing its x first if it is still active) and frees its
 * workspace; returns after the batch's stream has drained. */
ct_status ct_batch_remove(ct_batch *b, int32_t job);

/* Message of the calling thread's last failed call ("" if none). */
const char *ct_last_error(void);

/* Library version string. */
const char *ct_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices).  A profiling counter; memsets and copies are
 * not kernels and are not counted. */
int64_t ct_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* CT_H */
