// Internal declarations of the GB300 CBCT library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ct.h"

namespace ct {

// Per-view ray constants in VOXEL units, relative to the volume box's low
// corner: a point q (mm) maps to (q - box_lo) / h per axis.  A ray of pixel
// (u, v) runs from s to p00 + uc * eu + vc * ev, where p00 is the centre of
// the pixel grid, uc = u - (nu-1)/2 and vc = v - (nv-1)/2.  FP64: the
// ray-major kernels set up the rays that advance mostly along z from them.
struct ViewConst {
    double s[3];
    double p00[3];
    double eu[3];
    double ev[3];
};

// Per detector column (view, u) ray parameters, computed in FP64 on the host.
// For a flat detector whose v axis is the rotation axis,
// the in-plane direction of ray (u, v) depends on u only, so the slab axis s
// (x or y, whichever the ray advances along faster), the walk direction and
// the lateral slope A are per column; the z terms are affine in v.
//
// Coordinates are in voxel units, centred on integer planes: walk coordinate
// w = (sigma or Ns - sigma) - Ns/2 (sigma = coordinate along s, increasing
// along the ray), lateral xi = coordinate along the other in-plane axis
// minus Na/2, zeta = z coordinate minus Nz/2 (integer halves).  On the ray:
//   xi(w)   = XI0 + A w,            zeta(w) = (Z0 + vc Z1) + (C0 + vc C1) w,
// with vc = v - (nv-1)/2, and w runs from wsrc (source) to wpix (pixel).
//
// The lines are stored in Q.44 fixed point (value * 2^44, rounded to the
// nearest int64), which the walks turn into exact integer lines
// (projector.cu).  A row v has vc2 = 2 v - (nv - 1) and
//   C = (c0 + vc2 c1h) 2^-44,   Z0 + vc Z1 = (z0 + vc2 z1h) 2^-44,
// so the per-row slope and offset are exact integer sums.  XI0 and Z0 are
// clamped to +-2^16 voxels (such a ray misses every volume the column-major
// kernels accept).
struct __align__(16) ColFixed {
    long long a, xi;     // A, XI0
    long long c0, c1h;   // C0, C1 / 2
    long long z0, z1h;   // Z0, Z1 / 2
    float wsrc, wpix;    // FP32
    int flags;           // bit 0: slab axis is x (else y); bit 1: walk reversed;
                         // bit 2: the z lines do not fit Q.44 (c0 = c1h = 0):
                         // every ray of the column is set up as advancing along z
    int pad;
};

// Everything a projector kernel needs, passed by value.
struct ProjGeom {
    const ViewConst *views;  // device array [nviews] (rays advancing along z)
    const ColFixed *col_q;   // device array [nviews * nu]: the column lines (all walks)
    int nx, ny, nz;
    int nu, nv, nviews;
    float hx, hy, hz;        // voxel pitch, mm
    int cm;                  // 1: column-major kernels and the [y][x][z] volume copy
                             // (no ray advances mostly along z), 0: ray-major, [z][x][y]
    int proj;                // ct_projector
    const float4 *sf_view;   // footprint projectors: 2 float4 per view (sf_view_constants)
    float sf_ku, sf_kv, sf_cu, sf_cv, sf_oz;
    int sf_det;              // footprint A sums in int64 fixed point (deterministic geometry)
    double sf_row_bound;     // bound on one detector cell's sum of A_ij (fixed-point scale)
    void *sf_ws;             // scratch of sf_det_ws_bytes(pg) bytes, or NULL (sf_forward then
                             // allocates its own on the stream)
    int vgroup;              // launch order of A: views per group (set_launch_order)
    int vgroup_bt;           // launch order of A^T
    int nvb;                 // row blocks of the projector grid
    int bt_pairs;            // column-major A^T: pairs of row blocks, a warp every other row
};

// Choose the order in which the projector kernels visit (view, row block)
// tiles; call once the sizes of pg are set.
void set_launch_order(ProjGeom &pg);
// Then choose the lane-to-row mapping of the column-major A^T from the
// height of a detector row at the isocentre in voxels (dv SID / (SDD vz)).
void set_row_pairing(ProjGeom &pg, double row_vox);

}  // namespace ct

struct ct_geometry {
    ct_geometry_desc desc;       // copy; desc.angles_rad points into angles
    std::vector<double> angles;  // nviews
    int device;
    int64_t nvox, nrays;
    ct::ViewConst *d_views;      // device
    void *d_cols;                // device: the column table (ColFixed)
    ct::ProjGeom pg;
    int deterministic;           // backprojections accumulate in int64 fixed point
    float4 *d_sf;                // device: footprint-projector view constants (or NULL)
    double det_bound;            // bound on (rays through one voxel) * lsig_max
};

namespace ct {

// ---- error reporting (thread-local message) --------------------------------
ct_status set_error(ct_status st, const std::string &msg);
ct_status cuda_error(cudaError_t e, const char *where);
void clear_error();

#define CT_CUDA_TRY(expr)                                          \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::ct::cuda_error(_e, #expr); \
    } while (0)

#define CT_TRY(expr)                      \
    do {                                  \
        ct_status _s = (expr);            \
        if (_s != CT_OK) return _s;       \
    } while (0)

// Counts one kernel launch of this library (ct_kernel_launches) and checks
// that it was accepted.
void note_launch();
// Kernels this thread has launched (or captured into a graph) so far.
long long thread_launches();
// Adds n to the process-wide count (graph replays; negative: undo a capture).
void note_launches(long long n);
#define CT_CHECK_LAUNCH()                               \
    do {                                                \
        ::ct::note_launch();                            \
        CT_CUDA_TRY(cudaGetLastError());                \
    } while (0)

// ---- tracing ------------------------------------------------------------------
// An NVTX range named after a C-ABI call, open for the call's host-side
// duration (the enqueue, and the wait of the blocking calls).  Nsight tools
// attached to the process show it (ncu can filter kernels by it with
// --nvtx --nvtx-include); without a tool it costs a pointer check.
class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define CT_TRACE(name) ::ct::TraceRange ct_trace_range_(name)

// ---- stream-ordered device workspace ---------------------------------------
// Allocations are freed on the same stream when the Workspace goes out of
// scope, so kernels enqueued before the free still see valid memory.
class Workspace {
public:
    explicit Workspace(cudaStream_t s) : stream_(s) {}
    ~Workspace();
    Workspace(const Workspace &) = delete;
    Workspace &operator=(const Workspace &) = delete;
    // Returns CT_OK and sets *p, or CT_ERR_OOM / CT_ERR_CUDA.
    ct_status alloc(void **p, size_t bytes);
    template <class T>
    ct_status alloc(T **p, size_t count) {
        return alloc(reinterpret_cast<void **>(p), count * sizeof(T));
    }

private:
    cudaStream_t stream_;
    std::vector<void *> ptrs_;
};

// ---- projector launches (projector.cu) -------------------------------------
// Coefficients of an epilogue out = alpha * op(in) + beta * out.  When dev is
// non-NULL the pair is read on the device from dev[0], dev[1] (FP64).
struct Coef {
    float alpha = 1.f, beta = 0.f;
    const double *dev = nullptr;
};

// Number of FP64 norm partials a forward launch writes (one per CTA).
int64_t forward_partials(const ProjGeom &pg);
// The same for launch_forward_direct (one ray per thread, ray-major grid).
int64_t forward_direct_partials(const ProjGeom &pg);

// p = alpha * rho o (A vol) + beta * p.  vol_t is the same volume in the
// transposed layout [nz][nx][ny] (used by rays that advance mostly along x).
// rho may be NULL (all ones).  partials may be NULL; else one FP64 partial
// sum of p^2 per CTA.
ct_status launch_forward(const ProjGeom &pg, const float *vol, const float *vol_t, float *p,
                         const float *rho, Coef c, double *partials, cudaStream_t st);

// acc += alpha * A^T (rho o e), scattered with float atomics into acc
// ([nz][ny][nx]) for rays that advance mostly along y or z and into acc_t
// ([nz][nx][ny]) for rays that advance mostly along x.  power = 2 scatters
// squared lengths (diag(A^T A) with e = 1).
ct_status launch_backward(const ProjGeom &pg, const float *e, const float *rho, Coef c,
                          float *acc, float *acc_t, int power, cudaStream_t st);

// One job of a batched projector launch (launch_batch): a column-major
// Siddon geometry (batchable) with its vectors.  A: in = the [y][x][z] copy
// of the volume, out = p (FP32), partials = FP64 sums of p^2 per tile (or
// NULL).  A^T: in = e (FP32), out = the [y][x][z] accumulator (float, or
// int64 fixed point with det_scale).  rho may be NULL.
struct BatchJob {
    ProjGeom g;              // with the launch order of the operator (batch_job_grid)
    const void *in;
    void *out;
    const float *rho;
    Coef c;
    double *partials;
    const float *det_scale;
    unsigned tile0;          // first tile of the job in the batch's tile sequence
    unsigned gx, gy;         // the job's grid (x, y); z = tiles / (gx gy)
    unsigned tiles;
};
// Can A and A^T of this geometry join a batched launch?
bool batchable(const ProjGeom &pg);
// Fills g, gx, gy, tiles of *b for A (backward = false) or A^T.
ct_status batch_job_grid(const ProjGeom &pg, bool backward, BatchJob *b);
// Finds the resident CTAs of the batched kernels on the current device; call
// once per device before launch_batch, outside stream capture.
ct_status batch_prepare();
// One persistent launch over the ntiles tiles of njobs jobs (device table
// d_jobs, tile0 ascending, the same operator for all).  flag: A -> FP64 norm
// partials, A^T -> fixed-point sums.  d_next: a device counter (reset here).
ct_status launch_batch(const BatchJob *d_jobs, int njobs, unsigned ntiles, bool backward,
                       bool flag, unsigned *d_next, cudaStream_t st);

// Count the (ray, voxel) pairs with positive length into *d_count (int64).
ct_status launch_count(const ProjGeom &pg, unsigned long long *d_count, cudaStream_t st);

// Typed storage (ct_dtype): p (sdt) = alpha rho o (A vol (vdt)) + beta p.
ct_status launch_forward_typed(const ProjGeom &pg, const void *vol, const void *vol_t, int vdt,
                               void *p, int sdt, const float *rho, Coef c, double *partials,
                               cudaStream_t st);
// Typed input e (sdt); accumulators float (det = false) or int64 (det = true).
ct_status launch_backward_typed(const ProjGeom &pg, const void *e, int sdt, const float *rho,
                                Coef c, void *acc, void *acc_t, int power, bool det,
                                const float *det_scale, cudaStream_t st);
// Bytes of one element of a ct_dtype (0 if unknown).
inline size_t dtype_size(int dt) { return dt == CT_F32 ? 4 : (dt == CT_BF16 || dt == CT_F16) ? 2 : 0; }

// The same scatter accumulating rint(value * scale) in int64 (scale =
// det_scale[0], a power of two): order-independent, hence deterministic.
ct_status launch_backward_det(const ProjGeom &pg, const float *e, const float *rho, Coef c,
                              long long *acc, long long *acc_t, int power,
                              const float *det_scale, cudaStream_t st);
// scale[0] = 2^k (float) and inv[0] = 2^-k (double) with k the largest integer
// such that |alpha| max|e rho| bound 2^k <= 2^62.  part: vec_grid(m) floats.
ct_status launch_det_scale(const void *e, int edt, const float *rho, int64_t m, double bound,
                           Coef c, float *part, float *scale, double *inv, cudaStream_t st);
// The same scale for a forward projection: max|x| over the n voxels (x NULL:
// 1) times max|rho| over the m rays (rho NULL: 1).  part: vec_grid(n) +
// vec_grid(m) floats.
ct_status launch_det_scale_fwd(const float *x, int64_t n, const float *rho, int64_t m,
                               double bound, Coef c, float *part, float *scale, double *inv,
                               cudaStream_t st);
// out = beta out + (acc + transpose(acc_t)) inv; optional partials of (w out)^2.
ct_status launch_combine_det(const ProjGeom &pg, float *out, float beta, const long long *acc,
                             const long long *acc_t, const double *inv, const float *w,
                             double *partials, cudaStream_t st);

// p = alpha * A vol + beta * p reading vol in place (no transposed copy),
// with forward_direct_partials(pg) FP64 partial sums of p^2.
ct_status launch_forward_direct(const ProjGeom &pg, const float *vol, float *p, float alpha,
                                float beta, double *partials, cudaStream_t st);

// CT_DEBUG_BOUNDS build (ct_debug.cuh): read and clear the bounds-violation
// word of projector.cu / footprint.cu on the current device (0: none;
// (line << 1) | 1 otherwise).  The normal build reports 0.
ct_status debug_take_projector(unsigned long long *word);
ct_status debug_take_footprint(unsigned long long *word);

// ---- separable-footprint projectors (footprint.cu) -----------------------------
// Per-view constants (2 float4 per view) and the global scalars
// scal[5] = {SDD/du, SDD/dv, cu, cv, off_z}, FP64 on the host.
void sf_view_constants(const ct_geometry_desc &d, const std::vector<double> &ang,
                       std::vector<float4> &out, float *scal);
// p = alpha rho o (A x) + beta p (vol NULL: all ones) with the FP64 partials
// of ||p||^2 (sf_forward_partials of them) when partials is set.
ct_status sf_forward(const ProjGeom &pg, const float *vol, float *p, const float *rho, Coef c,
                     double *partials, cudaStream_t st);
int64_t sf_forward_partials(const ProjGeom &pg);
// Scratch of a fixed-point footprint forward projection (pg.sf_det): int64
// sums of every ray, the scale and the maxima partials.
size_t sf_det_ws_bytes(const ProjGeom &pg);
// Bound on one detector cell's sum over voxels of A_ij for the footprint
// projectors of geometry d (every voxel in front of the source).
double sf_row_bound(const ct_geometry_desc &d);
// acc += alpha (A o ...)^T (rho o e), power 1 or 2 (e NULL: e = 1), caller's layout.
ct_status sf_backward(const ProjGeom &pg, const float *e, const float *rho, Coef c, float *acc,
                      int power, cudaStream_t st);
ct_status sf_count(const ProjGeom &pg, unsigned long long *d_count, cudaStream_t st);
// out = beta out + acc
ct_status sf_axpby(float *out, const float *acc, int64_t n, float beta, cudaStream_t st);

// ---- volume / sinogram kernels (vector_ops.cu) ------------------------------
int vec_grid(int64_t n);  // CTAs of a streaming kernel (also its partial count)
constexpr int kVecThreads = 256;

// t = transpose of v: [nz][ny][nx] -> [nz][nx][ny]; optional scale w (t = w v)
// and optional plain copy out (out = w v in the original layout).
ct_status launch_transpose(const ProjGeom &pg, const float *v, const float *w, float *t,
                           float *out_plain, cudaStream_t st);
// g = acc + transpose(acc_t)  ([nz][nx][ny] -> [nz][ny][nx]); with partials,
// one FP64 partial per CTA of sum (w o g)^2 (w may be NULL).  Column-major
// geometries keep all of A^T in acc_t ([y][x][z]): there g = beta g +
// acc_t transposed (beta 0: g is not read); the others add (beta ignored).
int transpose_grid_count(const ProjGeom &pg);
ct_status launch_combine(const ProjGeom &pg, float *g, const float *acc_t, const float *w,
                         double *partials, cudaStream_t st, float beta = 1.f);
// Typed transpose: t (dt) = transpose of v (dt), [nz][ny][nx] -> [nz][nx][ny].
ct_status launch_transpose_typed(const ProjGeom &pg, const void *v, void *t, int dt,
                                 cudaStream_t st);
// out (dt) = beta out + acc + transpose(acc_t) with FP32 accumulators, or
// (when q != NULL) with int64 accumulators q, q + nvox scaled by inv[0].
ct_status launch_combine_typed(const ProjGeom &pg, void *out, int dt, float beta, const float *acc,
                               const float *acc_t, const long long *q, const double *inv,
                               cudaStream_t st);
// out = beta * out (beta == 0 writes zeros without reading)
ct_status launch_scale(float *out, int64_t n, float beta, cudaStream_t st);
// out = v o w (elementwise).
ct_status launch_mul(float *out, const float *v, const float *w, int64_t n, cudaStream_t st);
ct_status launch_scale_dev(float *out, int64_t n, const double *beta, cudaStream_t st);
// Sum of partials[0..n) in a fixed order into *out (FP64, deterministic).
ct_status launch_sum(const double *partials, int64_t n, double *out, cudaStream_t st);
// partial sums of (w o v)^2 (w may be NULL), vec_grid(n) partials
ct_status launch_norm2(const float *v, const float *w, int64_t n, double *partials,
                       cudaStream_t st);

}  // namespace ct

namespace ct {
// v = 1/sqrt(v) where v > rel * max(v), else 0.  part: vec_grid(n) floats.
ct_status launch_inv_sqrt_guarded(float *v, int64_t n, float rel, float *part, cudaStream_t st);

// Device scratch of backprojections: a float accumulator in the transposed
// layout, or, for a deterministic geometry, two int64 accumulators and the
// fixed-point scale.  Allocate once per solve and reuse.
struct BackScratch {
    float *acc_t = nullptr;      // nvox floats
    long long *q = nullptr;      // 2 nvox int64: main layout, then transposed
    float *part = nullptr;       // vec_grid(nrays) floats
    float *scale = nullptr;      // 1 float
    double *inv = nullptr;       // 1 double
};
// Backprojections of g sum in int64 fixed point: a deterministic geometry
// with the Siddon projector (the footprint A^T gathers, in a fixed order).
inline bool fixed_back(const ct_geometry *g) {
    return g->deterministic && g->pg.proj == CT_PROJ_SIDDON;
}
// acc_t may be a caller buffer of nvox floats (reused between calls).
ct_status back_scratch_alloc(const ct_geometry *g, Workspace &ws, float *acc_t, BackScratch *s);
// Bound on one voxel's backprojected sum per unit |alpha e rho| (power 1:
// lengths, power 2: squared lengths), for the fixed-point scale.
double det_value_bound(const ct_geometry *g, int power);

// out = beta * out + alpha * A^T (rho o e) (POWER 2: squared lengths), in the
// geometry's accumulation mode (float atomics, or int64 fixed point when the
// geometry is deterministic); partials (may be NULL) receive per-CTA sums of
// (w o out)^2, transpose_grid_count(pg) of them.
ct_status backproject_impl(const ct_geometry *g, const BackScratch &s, const float *e,
                           const float *rho, Coef c, float *out, float beta, int power,
                           const float *w, double *partials, cudaStream_t st);

// Preconditioner weights into caller buffers (see ct_precond_weights).
ct_status precond_weights_impl(const ct_geometry *g, int kind, float *vol_w, float *sino_w,
                               Workspace &ws, cudaStream_t st);

// Makes g's device current for the lifetime of the guard.
class DeviceGuard {
public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    ct_status status() const { return st_; }

private:
    int prev_ = -1;
    bool changed_ = false;
    ct_status st_ = CT_OK;
};
}  // namespace ct
