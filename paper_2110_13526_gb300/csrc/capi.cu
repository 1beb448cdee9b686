// C ABI: geometry, projector entry points, nnz count, preconditioner
// weights, error strings.  The solvers live in solvers.cu.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "ct_internal.h"

namespace ct {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};
}

namespace {
thread_local long long t_launches = 0;
}

void note_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}

long long thread_launches() { return t_launches; }

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ct_status set_error(ct_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

ct_status cuda_error(cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    return set_error(e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA, m);
}

void clear_error() { g_last_error.clear(); }

Workspace::~Workspace() {
    for (void *p : ptrs_) cudaFreeAsync(p, stream_);
}

ct_status Workspace::alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, stream_);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "cudaMallocAsync (workspace)");
    }
    ptrs_.push_back(*p);
    return CT_OK;
}

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
        st_ = set_error(CT_ERR_CUDA, "cudaGetDevice failed");
        return;
    }
    if (prev_ != dev) {
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) {
            st_ = cuda_error(e, "cudaSetDevice");
            return;
        }
        changed_ = true;
    }
}

DeviceGuard::~DeviceGuard() {
    if (changed_) cudaSetDevice(prev_);
}

ct_status back_scratch_alloc(const ct_geometry *g, Workspace &ws, float *acc_t, BackScratch *s) {
    *s = BackScratch{};
    if (!fixed_back(g)) {
        if (acc_t) {
            s->acc_t = acc_t;
            return CT_OK;
        }
        return ws.alloc(&s->acc_t, (size_t)g->nvox);
    }
    CT_TRY(ws.alloc(&s->q, 2 * (size_t)g->nvox));
    CT_TRY(ws.alloc(&s->part, (size_t)vec_grid(std::max<int64_t>(g->nrays, 1))));
    CT_TRY(ws.alloc(&s->scale, 1));
    CT_TRY(ws.alloc(&s->inv, 1));
    return CT_OK;
}

double det_value_bound(const ct_geometry *g, int power) {
    // a segment contributes at most |alpha e rho| * hdiag^power (hdiag: voxel
    // diagonal, the longest chord), and at most det_bound / 2 rays cross a voxel
    const double hdiag = std::sqrt(g->desc.vx * g->desc.vx + g->desc.vy * g->desc.vy +
                                   g->desc.vz * g->desc.vz);
    return g->det_bound * (power == 2 ? hdiag * hdiag : hdiag);
}

ct_status backproject_impl(const ct_geometry *g, const BackScratch &s, const float *e,
                           const float *rho, Coef c, float *out, float beta, int power,
                           const float *w, double *partials, cudaStream_t st) {
    const ProjGeom &pg = g->pg;
    const int64_t n = g->nvox;
    if (!fixed_back(g)) {
        // column-major Siddon kernels accumulate in acc_t only, and the
        // combine applies beta; the others accumulate into out itself
        const bool zfast_only = pg.proj == CT_PROJ_SIDDON && pg.cm;
        if (!zfast_only) CT_TRY(launch_scale(out, n, beta, st));
        CT_CUDA_TRY(cudaMemsetAsync(s.acc_t, 0, (size_t)n * sizeof(float), st));
        CT_TRY(launch_backward(pg, e, rho, c, out, s.acc_t, power, st));
        return launch_combine(pg, out, s.acc_t, w, partials, st, zfast_only ? beta : 1.f);
    }
    CT_CUDA_TRY(cudaMemsetAsync(s.q, 0, 2 * (size_t)n * sizeof(long long), st));
    CT_TRY(launch_det_scale(e, CT_F32, rho, g->nrays, det_value_bound(g, power), c, s.part,
                            s.scale, s.inv, st));
    CT_TRY(launch_backward_det(pg, e, rho, c, s.q, s.q + n, power, s.scale, st));
    return launch_combine_det(pg, out, beta, s.q, s.q + n, s.inv, w, partials, st);
}

ct_status precond_weights_impl(const ct_geometry *g, int kind, float *vol_w, float *sino_w,
                               Workspace &ws, cudaStream_t st) {
    const ProjGeom &pg = g->pg;
    float *part = nullptr;
    const int64_t np = std::max<int64_t>(vec_grid(g->nvox), vec_grid(g->nrays));
    CT_TRY(ws.alloc(&part, (size_t)np));
    BackScratch bs;
    CT_TRY(back_scratch_alloc(g, ws, nullptr, &bs));
    Coef one;
    if (kind == CT_PRECOND_JACOBI) {
        // D = diag(A^T A) = (A o A)^T 1: squared lengths scattered from unit rays
        CT_TRY(backproject_impl(g, bs, nullptr, nullptr, one, vol_w, 0.f, 2, nullptr, nullptr, st));
        CT_TRY(launch_inv_sqrt_guarded(vol_w, g->nvox, 1e-6f, part, st));
        return CT_OK;
    }
    if (kind == CT_PRECOND_ROWCOL) {
        // R = A 1 (row sums) and C = A^T 1 (column sums)
        CT_TRY(launch_forward(pg, nullptr, nullptr, sino_w, nullptr, one, nullptr, st));
        CT_TRY(launch_inv_sqrt_guarded(sino_w, g->nrays, 1e-6f, part, st));
        CT_TRY(backproject_impl(g, bs, nullptr, nullptr, one, vol_w, 0.f, 1, nullptr, nullptr, st));
        CT_TRY(launch_inv_sqrt_guarded(vol_w, g->nvox, 1e-6f, part, st));
        return CT_OK;
    }
    return set_error(CT_ERR_INVALID_ARG, "unknown preconditioner kind");
}

}  // namespace ct

using namespace ct;

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

ct_status check_geom(const ct_geometry *g) {
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    return CT_OK;
}

// Per-view ray constants, FP64, in voxel units.
void view_constants(const ct_geometry_desc &d, const std::vector<double> &ang,
                    std::vector<ViewConst> &out) {
    const double h[3] = {d.vx, d.vy, d.vz};
    const double lo[3] = {-0.5 * d.nx * d.vx + d.off_x, -0.5 * d.ny * d.vy + d.off_y,
                          -0.5 * d.nz * d.vz + d.off_z};
    out.resize(ang.size());
    for (size_t k = 0; k < ang.size(); ++k) {
        const double c = std::cos(ang[k]), s = std::sin(ang[k]);
        const double src[3] = {d.sid * c, d.sid * s, 0.0};
        const double cd = -(d.sdd - d.sid);
        const double eu[3] = {-s, c, 0.0}, ev[3] = {0.0, 0.0, 1.0};
        // centre of the pixel grid (u = (nu-1)/2, v = (nv-1)/2) incl. offsets
        double pc[3];
        for (int a = 0; a < 3; ++a) {
            const double dc = (a == 0 ? cd * c : (a == 1 ? cd * s : 0.0));
            pc[a] = dc + d.det_off_u * eu[a] + d.det_off_v * ev[a];
        }
        ViewConst &vc = out[k];
        for (int a = 0; a < 3; ++a) {
            vc.s[a] = (src[a] - lo[a]) / h[a];
            vc.p00[a] = (pc[a] - lo[a]) / h[a];
            vc.eu[a] = d.du * eu[a] / h[a];
            vc.ev[a] = d.dv * ev[a] / h[a];
        }
    }
}

// x * 2^44 rounded to the nearest integer (ColFixed).
long long q44(double x) { return std::llround(std::ldexp(x, 44)); }

// Per-column ray lines (ColFixed), computed in FP64 and stored in fixed point.
void column_params(const ct_geometry_desc &d, const std::vector<double> &ang,
                   std::vector<ColFixed> &cq_out) {
    const double h[3] = {d.vx, d.vy, d.vz};
    const int N[3] = {d.nx, d.ny, d.nz};
    const double lo[3] = {-0.5 * d.nx * d.vx + d.off_x, -0.5 * d.ny * d.vy + d.off_y,
                          -0.5 * d.nz * d.vz + d.off_z};
    const size_t ncol = ang.size() * (size_t)d.nu;
    cq_out.resize(ncol);
    for (size_t k = 0; k < ang.size(); ++k) {
        const double c = std::cos(ang[k]), s = std::sin(ang[k]);
        const double src[3] = {d.sid * c, d.sid * s, 0.0};
        const double cd = -(d.sdd - d.sid);
        const double eu[3] = {-s, c, 0.0};
        const double pc[3] = {cd * c + d.det_off_u * eu[0], cd * s + d.det_off_u * eu[1],
                              d.det_off_v};
        double S[3], Pc[3], EU[3];
        for (int a = 0; a < 3; ++a) {
            S[a] = (src[a] - lo[a]) / h[a];
            Pc[a] = (pc[a] - lo[a]) / h[a];
            EU[a] = d.du * eu[a] / h[a];
        }
        const double EVz = d.dv / h[2];
        for (int u = 0; u < d.nu; ++u) {
            const double uc = u - 0.5 * (d.nu - 1);
            double P[3], D[3];
            for (int a = 0; a < 3; ++a) {
                P[a] = Pc[a] + uc * EU[a];
                D[a] = P[a] - S[a];
            }
            const int ax = std::fabs(D[0]) >= std::fabs(D[1]) ? 0 : 1;
            const int la = 1 - ax;
            const bool rev = D[ax] < 0.0;
            const int Ns = N[ax], Na = N[la], Nb = N[2];
            const int cs = Ns / 2, cl = Na / 2, cz = Nb / 2;
            const double Ds = D[ax];
            const double sig0 = rev ? (double)(Ns - cs) : (double)cs;
            const double adx = std::fabs(Ds);
            const size_t i = k * (size_t)d.nu + (size_t)u;
            if (adx == 0.0) {  // degenerate: never hits (pixel at the source)
                cq_out[i] = ColFixed{0, q44(65536.0), 0, 0, q44(65536.0), 0, 0.f, -1.f, 0, 0};
                continue;
            }
            const double A = D[la] / adx;
            const double XI0 = S[la] - cl + (sig0 - S[ax]) * D[la] / Ds;
            const double C0 = D[2] / adx;
            const double C1 = EVz / adx;
            const double Z0 = S[2] - cz + (sig0 - S[ax]) * D[2] / Ds;
            const double Z1 = (sig0 - S[ax]) * EVz / Ds;
            const double wsrc = (rev ? Ns - S[ax] : S[ax]) - cs;
            const double wpix = (rev ? Ns - P[ax] : P[ax]) - cs;
            const int fl = (ax == 0 ? 1 : 0) | (rev ? 2 : 0);
            const double lim = 65536.0;   // a ray this far out misses the volume
            // z lines held in Q.44 only while c0 + vc2 c1h stays far inside int64
            const bool zfit = std::fabs(C0) < 1e5 && std::fabs(C1) * (double)(d.nv + 1) < 1e5;
            cq_out[i] = ColFixed{q44(A), q44(std::fmin(std::fmax(XI0, -lim), lim)),
                                 zfit ? q44(C0) : 0, zfit ? q44(0.5 * C1) : 0,
                                 zfit ? q44(std::fmin(std::fmax(Z0, -lim), lim)) : 0,
                                 zfit ? q44(0.5 * Z1) : 0, (float)wsrc, (float)wpix,
                                 fl | (zfit ? 0 : 4), 0};
        }
    }
}

}  // namespace

// Column-major kernels unless some ray advances mostly along z or the
// fixed-point lines could leave their int64 range.  A row's z slope is
// c0 + vc2 c1h (Q.44) with vc2 = 2 v - (nv - 1), linear in v, so the first
// and last rows bound |C|; the test uses the kernels' integer arithmetic.
// Limits: every dimension at most 2^15 voxels (slab products below 2^59) and
// the detector's z extent at the centre plane within 2^16 voxels.
static bool cm_eligible(const ct_geometry_desc &d, const std::vector<ColFixed> &colq) {
    if (d.nx > 32768 || d.ny > 32768 || d.nz > 32768) return false;
    const long long one = 1LL << 44, m = (long long)std::max(d.nv - 1, 0);
    for (const ColFixed &q : colq) {
        if (q.flags & 4) return false;
        const double cf = std::fabs((double)q.c0) + (double)m * std::fabs((double)q.c1h);
        const double zf = (double)m * std::fabs((double)q.z1h);
        if (cf > 2.0 * (double)one || zf > std::ldexp(1.0, 60)) return false;
        const long long c_lo = q.c0 - m * q.c1h, c_hi = q.c0 + m * q.c1h;
        if (std::llabs(c_lo) > one || std::llabs(c_hi) > one) return false;
    }
    return true;
}

extern "C" {

ct_status ct_geometry_create(const ct_geometry_desc *desc, ct_geometry **out) {
    clear_error();
    if (!desc || !out) return set_error(CT_ERR_INVALID_ARG, "desc and out must be non-NULL");
    *out = nullptr;
    const ct_geometry_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1)
        return set_error(CT_ERR_INVALID_ARG, "nx, ny, nz must be >= 1");
    if (d.nu < 0 || d.nv < 0 || d.nviews < 0)
        return set_error(CT_ERR_INVALID_ARG, "nu, nv, nviews must be >= 0");
    if (!finite_pos(d.vx) || !finite_pos(d.vy) || !finite_pos(d.vz) || !finite_pos(d.du) ||
        !finite_pos(d.dv))
        return set_error(CT_ERR_INVALID_ARG, "voxel and pixel pitches must be finite and > 0");
    if (!finite_pos(d.sid) || !std::isfinite(d.sdd) || !(d.sdd > d.sid))
        return set_error(CT_ERR_INVALID_ARG, "need 0 < sid < sdd");
    if (!std::isfinite(d.off_x) || !std::isfinite(d.off_y) || !std::isfinite(d.off_z) ||
        !std::isfinite(d.det_off_u) || !std::isfinite(d.det_off_v))
        return set_error(CT_ERR_INVALID_ARG, "offsets must be finite");
    const int64_t nvox = (int64_t)d.nx * d.ny * d.nz;
    if (nvox >= (int64_t(1) << 31))
        return set_error(CT_ERR_INVALID_ARG, "volume must hold fewer than 2^31 voxels");
    if (d.nx > 65535 || d.ny > 65535 || d.nz > 65535 || d.nviews > 65535)
        return set_error(CT_ERR_INVALID_ARG, "nx, ny, nz and nviews must be <= 65535");
    if (d.nv > 65535 * 8)
        return set_error(CT_ERR_INVALID_ARG, "nv must be <= 524280");
    if ((int64_t)d.nx * d.ny >= (int64_t(1) << 31))
        return set_error(CT_ERR_INVALID_ARG, "nx * ny too large");
    if (d.nviews > 0 && d.angles_rad) {
        for (int k = 0; k < d.nviews; ++k)
            if (!std::isfinite(d.angles_rad[k]))
                return set_error(CT_ERR_INVALID_ARG, "angles must be finite");
    }
    ct_geometry *g = new (std::nothrow) ct_geometry();
    if (!g) return set_error(CT_ERR_OOM, "host allocation failed");
    g->desc = d;
    g->angles.resize((size_t)d.nviews);
    for (int k = 0; k < d.nviews; ++k)
        g->angles[(size_t)k] = d.angles_rad ? d.angles_rad[k] : 2.0 * M_PI * k / d.nviews;
    g->desc.angles_rad = g->angles.data();
    g->nvox = nvox;
    g->nrays = (int64_t)d.nviews * d.nv * d.nu;
    g->d_views = nullptr;
    g->deterministic = 0;
    {
        // rays through one voxel in all views: the voxel's detector footprint
        // at the largest magnification (volume corner nearest the source),
        // plus a margin of two pixels per axis; never more than all rays
        double rmax = 0.0;
        for (int cx = 0; cx < 2; ++cx)
            for (int cy = 0; cy < 2; ++cy) {
                const double x = (cx ? 0.5 : -0.5) * d.nx * d.vx + d.off_x;
                const double y = (cy ? 0.5 : -0.5) * d.ny * d.vy + d.off_y;
                rmax = std::max(rmax, std::sqrt(x * x + y * y));
            }
        const double hd = std::sqrt(d.vx * d.vx + d.vy * d.vy + d.vz * d.vz);
        double rays = (double)g->nrays;
        if (d.sid > rmax) {
            const double mag = d.sdd / (d.sid - rmax);
            const double per_view =
                (std::ceil(hd * mag / d.du) + 2.0) * (std::ceil(hd * mag / d.dv) + 2.0);
            rays = std::min(rays, (double)d.nviews * per_view);
        }
        g->det_bound = 2.0 * std::max(rays, 1.0);
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_error(e, "cudaGetDevice");
    }
    std::vector<ViewConst> vcs;
    view_constants(d, g->angles, vcs);
    std::vector<ColFixed> colq;
    column_params(d, g->angles, colq);
    g->d_cols = nullptr;
    const size_t ncol = colq.size();
    if (d.nviews > 0) {
        e = cudaMalloc(&g->d_views, sizeof(ViewConst) * vcs.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_views, vcs.data(), sizeof(ViewConst) * vcs.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess && ncol > 0) {
            e = cudaMalloc(&g->d_cols, ncol * sizeof(ColFixed));
            if (e == cudaSuccess)
                e = cudaMemcpy(g->d_cols, colq.data(), ncol * sizeof(ColFixed),
                               cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            if (g->d_views) cudaFree(g->d_views);
            if (g->d_cols) cudaFree(g->d_cols);
            delete g;
            return cuda_error(e, "geometry upload");
        }
    }
    g->pg.views = g->d_views;
    g->pg.col_q = (const ColFixed *)g->d_cols;
    g->pg.nx = d.nx; g->pg.ny = d.ny; g->pg.nz = d.nz;
    g->pg.nu = d.nu; g->pg.nv = d.nv; g->pg.nviews = d.nviews;
    g->pg.hx = (float)d.vx; g->pg.hy = (float)d.vy; g->pg.hz = (float)d.vz;
    g->pg.proj = CT_PROJ_SIDDON;
    g->pg.sf_view = nullptr;
    g->pg.sf_ku = g->pg.sf_kv = g->pg.sf_cu = g->pg.sf_cv = g->pg.sf_oz = 0.f;
    g->pg.sf_det = 0;
    g->pg.sf_row_bound = 0.0;
    g->pg.sf_ws = nullptr;
    g->d_sf = nullptr;
    g->pg.cm = cm_eligible(d, colq) ? 1 : 0;
    set_launch_order(g->pg);
    set_row_pairing(g->pg, d.dv * d.sid / (d.sdd * d.vz));
    *out = g;
    return CT_OK;
}

void ct_geometry_destroy(ct_geometry *g) {
    if (!g) return;
    if (g->d_views || g->d_cols || g->d_sf) {
        DeviceGuard dg(g->device);
        if (g->d_views) cudaFree(g->d_views);
        if (g->d_cols) cudaFree(g->d_cols);
        if (g->d_sf) cudaFree(g->d_sf);
    }
    delete g;
}

ct_status ct_geometry_sizes(const ct_geometry *g, int64_t *n_vox, int64_t *n_rays) {
    clear_error();
    CT_TRY(check_geom(g));
    if (n_vox) *n_vox = g->nvox;
    if (n_rays) *n_rays = g->nrays;
    return CT_OK;
}

ct_status ct_project(const ct_geometry *g, const float *d_vol, float *d_sino, float alpha,
                     float beta, void *stream) {
    CT_TRACE("ct_project");
    clear_error();
    CT_TRY(check_geom(g));
    if (g->nrays == 0) return CT_OK;
    if (!d_vol || !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws(st);
    float *vol_t = nullptr;
    CT_TRY(ws.alloc(&vol_t, (size_t)g->nvox));
    CT_TRY(launch_transpose(g->pg, d_vol, nullptr, vol_t, nullptr, st));
    Coef c;
    c.alpha = alpha;
    c.beta = beta;
    return launch_forward(g->pg, d_vol, vol_t, d_sino, nullptr, c, nullptr, st);
}

ct_status ct_project_norm2(const ct_geometry *g, const float *d_vol, float *d_sino, float alpha,
                           float beta, double *d_norm2, void *stream) {
    CT_TRACE("ct_project_norm2");
    clear_error();
    CT_TRY(check_geom(g));
    if (!d_norm2) return set_error(CT_ERR_INVALID_ARG, "d_norm2 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (g->nrays == 0) {
        DeviceGuard dg(g->device);
        CT_TRY(dg.status());
        CT_CUDA_TRY(cudaMemsetAsync(d_norm2, 0, sizeof(double), st));
        return CT_OK;
    }
    if (!d_vol || !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    Workspace ws(st);
    float *vol_t = nullptr;
    double *part = nullptr;
    const int64_t np = forward_partials(g->pg);
    CT_TRY(ws.alloc(&vol_t, (size_t)g->nvox));
    CT_TRY(ws.alloc(&part, (size_t)np));
    CT_TRY(launch_transpose(g->pg, d_vol, nullptr, vol_t, nullptr, st));
    Coef c;
    c.alpha = alpha;
    c.beta = beta;
    CT_TRY(launch_forward(g->pg, d_vol, vol_t, d_sino, nullptr, c, part, st));
    return launch_sum(part, np, d_norm2, st);
}

ct_status ct_backproject(const ct_geometry *g, const float *d_sino, float *d_vol, float alpha,
                         float beta, void *stream) {
    CT_TRACE("ct_backproject");
    clear_error();
    CT_TRY(check_geom(g));
    if (!d_vol) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (g->nrays > 0 && !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    if (g->nrays == 0 || alpha == 0.f) return launch_scale(d_vol, g->nvox, beta, st);
    Workspace ws(st);
    BackScratch bs;
    CT_TRY(back_scratch_alloc(g, ws, nullptr, &bs));
    Coef c;
    c.alpha = alpha;
    return backproject_impl(g, bs, d_sino, nullptr, c, d_vol, beta, 1, nullptr, nullptr, st);
}

ct_status ct_project_ex(const ct_geometry *g, const void *d_vol, int32_t vol_dtype, void *d_sino,
                        int32_t sino_dtype, float alpha, float beta, void *stream) {
    CT_TRACE("ct_project_ex");
    clear_error();
    CT_TRY(check_geom(g));
    if (dtype_size(vol_dtype) == 0 || dtype_size(sino_dtype) == 0)
        return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
    if (g->nrays == 0) return CT_OK;
    if (!d_vol || !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws(st);
    void *vol_t = nullptr;
    CT_TRY(ws.alloc(&vol_t, (size_t)g->nvox * dtype_size(vol_dtype)));
    CT_TRY(launch_transpose_typed(g->pg, d_vol, vol_t, vol_dtype, st));
    Coef c;
    c.alpha = alpha;
    c.beta = beta;
    return launch_forward_typed(g->pg, d_vol, vol_t, vol_dtype, d_sino, sino_dtype, nullptr, c,
                                nullptr, st);
}

ct_status ct_backproject_ex(const ct_geometry *g, const void *d_sino, int32_t sino_dtype,
                            void *d_vol, int32_t vol_dtype, float alpha, float beta,
                            void *stream) {
    CT_TRACE("ct_backproject_ex");
    clear_error();
    CT_TRY(check_geom(g));
    if (dtype_size(vol_dtype) == 0 || dtype_size(sino_dtype) == 0)
        return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
    if (!d_vol) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (g->nrays > 0 && !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->nvox;
    Workspace ws(st);
    Coef c;
    c.alpha = alpha;
    if (fixed_back(g) && g->nrays > 0 && alpha != 0.f) {
        BackScratch bs;
        CT_TRY(back_scratch_alloc(g, ws, nullptr, &bs));
        CT_CUDA_TRY(cudaMemsetAsync(bs.q, 0, 2 * (size_t)n * sizeof(long long), st));
        CT_TRY(launch_det_scale(d_sino, sino_dtype, nullptr, g->nrays, det_value_bound(g, 1), c,
                                bs.part, bs.scale, bs.inv, st));
        CT_TRY(launch_backward_typed(g->pg, d_sino, sino_dtype, nullptr, c, bs.q, bs.q + n, 1,
                                     true, bs.scale, st));
        return launch_combine_typed(g->pg, d_vol, vol_dtype, beta, nullptr, nullptr, bs.q, bs.inv,
                                    st);
    }
    float *acc = nullptr;
    CT_TRY(ws.alloc(&acc, 2 * (size_t)n));
    CT_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * (size_t)n * sizeof(float), st));
    if (g->nrays > 0 && alpha != 0.f)
        CT_TRY(launch_backward_typed(g->pg, d_sino, sino_dtype, nullptr, c, acc, acc + n, 1, false,
                                     nullptr, st));
    return launch_combine_typed(g->pg, d_vol, vol_dtype, beta, acc, acc + n, nullptr, nullptr, st);
}

ct_status ct_geometry_set_deterministic(ct_geometry *g, int32_t on) {
    clear_error();
    CT_TRY(check_geom(g));
    g->deterministic = on ? 1 : 0;
    g->pg.sf_det = (on && g->pg.proj != CT_PROJ_SIDDON) ? 1 : 0;
    return CT_OK;
}

ct_status ct_geometry_set_projector(ct_geometry *g, int32_t kind) {
    clear_error();
    CT_TRY(check_geom(g));
    if (kind != CT_PROJ_SIDDON && kind != CT_PROJ_SF_TR && kind != CT_PROJ_SF_TT)
        return set_error(CT_ERR_INVALID_ARG, "unknown projector");
    if (kind != CT_PROJ_SIDDON) {
        if (g->desc.ny > 65535 * 8)
            return set_error(CT_ERR_INVALID_ARG, "footprint projectors need ny <= 524280");
        // every voxel corner in front of the source in every view: the
        // footprint divides by the depth along the central ray
        const ct_geometry_desc &d = g->desc;
        double rmax = 0.0;
        for (int cx = 0; cx < 2; ++cx)
            for (int cy = 0; cy < 2; ++cy) {
                const double x = (cx ? 0.5 : -0.5) * d.nx * d.vx + d.off_x;
                const double y = (cy ? 0.5 : -0.5) * d.ny * d.vy + d.off_y;
                rmax = std::max(rmax, std::sqrt(x * x + y * y));
            }
        if (!(rmax < d.sid))
            return set_error(CT_ERR_INVALID_ARG,
                             "footprint projectors need the volume inside the source circle");
        if (!g->d_sf && g->desc.nviews > 0) {
            DeviceGuard dg(g->device);
            CT_TRY(dg.status());
            std::vector<float4> sv;
            float scal[5];
            sf_view_constants(g->desc, g->angles, sv, scal);
            float4 *d = nullptr;
            CT_CUDA_TRY(cudaMalloc(&d, sv.size() * sizeof(float4)));
            const cudaError_t e =
                cudaMemcpy(d, sv.data(), sv.size() * sizeof(float4), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(d);
                return cuda_error(e, "footprint constants upload");
            }
            g->d_sf = d;
            g->pg.sf_ku = scal[0];
            g->pg.sf_kv = scal[1];
            g->pg.sf_cu = scal[2];
            g->pg.sf_cv = scal[3];
            g->pg.sf_oz = scal[4];
        }
        g->pg.sf_view = g->d_sf;
        g->pg.sf_row_bound = sf_row_bound(g->desc);
    }
    g->pg.proj = kind;
    g->pg.sf_det = (g->deterministic && kind != CT_PROJ_SIDDON) ? 1 : 0;
    return CT_OK;
}

ct_status ct_debug_status(void) {
    clear_error();
    CT_CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long wp = 0, wf = 0;
    CT_TRY(debug_take_projector(&wp));
    CT_TRY(debug_take_footprint(&wf));
    if (wp)
        return set_error(CT_ERR_INTERNAL, "index out of range in projector.cu line " +
                                              std::to_string(wp >> 1));
    if (wf)
        return set_error(CT_ERR_INTERNAL, "index out of range in footprint.cu line " +
                                              std::to_string(wf >> 1));
    return CT_OK;
}

int32_t ct_debug_bounds_build(void) {
#ifdef CT_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

ct_status ct_count_nnz(const ct_geometry *g, int64_t *out, void *stream) {
    CT_TRACE("ct_count_nnz");
    clear_error();
    CT_TRY(check_geom(g));
    if (!out) return set_error(CT_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws(st);
    unsigned long long *d = nullptr;
    CT_TRY(ws.alloc(&d, 1));
    CT_TRY(launch_count(g->pg, d, st));
    unsigned long long h = 0;
    CT_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    CT_CUDA_TRY(cudaStreamSynchronize(st));
    *out = (int64_t)h;
    return CT_OK;
}

ct_status ct_precond_weights(const ct_geometry *g, int32_t kind, float *d_vol_w, float *d_sino_w,
                             void *stream) {
    CT_TRACE("ct_precond_weights");
    clear_error();
    CT_TRY(check_geom(g));
    if (kind != CT_PRECOND_JACOBI && kind != CT_PRECOND_ROWCOL)
        return set_error(CT_ERR_INVALID_ARG, "kind must be CT_PRECOND_JACOBI or CT_PRECOND_ROWCOL");
    if (!d_vol_w || (kind == CT_PRECOND_ROWCOL && g->nrays > 0 && !d_sino_w))
        return set_error(CT_ERR_INVALID_ARG, "NULL weight vector");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    {
        Workspace ws(st);
        CT_TRY(precond_weights_impl(g, kind, d_vol_w, d_sino_w, ws, st));
    }
    CT_CUDA_TRY(cudaStreamSynchronize(st));
    return CT_OK;
}

const char *ct_last_error(void) { return g_last_error.c_str(); }

const char *ct_version(void) { return "ct-gb300 0.1.0 (sm_103a)"; }

int64_t ct_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
