// Separable-footprint projector pair (SF-TR / SF-TT) for sm_103a.
//
// Materials and Methods computes the paper's results with the "TT" footprint
// projector of Long, Fessler and Balter (2010), which the paper names without
// writing it out.  Read here as follows (conventions of include/ct.h):
//   * a point P projects to detector pixel-index coordinates
//       u = (SDD / du) s_u(P) / t(P) + cu,   v = (SDD / dv) z(P) / t(P) + cv,
//     with t the depth along the central ray and s_u the coordinate along e_u;
//   * transaxial footprint: the unit trapezoid whose breakpoints are the
//     sorted u of the voxel's four vertical edges (u does not depend on z);
//   * axial footprint: TR -- the unit rectangle between the v of the two z
//     faces at the depth of the voxel centre; TT -- the unit trapezoid of the
//     v of the two z faces at the smallest and largest depth of the corners;
//   * amplitude: the chord of the ray through the voxel centre across the x
//     and y faces, l = |d| min(hx / |d_x|, hy / |d_y|), d = centre - source;
//   * a detector cell averages the footprint:
//       A_ij = l * Fbar_u(k) * Fbar_v(l),  Fbar(k) = integral over [k-1/2, k+1/2].
// A^T uses the same entries, so the pair is exactly adjoint.
//
// Kernels.  A is voxel-driven: one thread per voxel column (i, j) and view
// computes the transaxial footprint once and walks the column in z, adding
// its contributions to the detector cells with float reductions (the 32
// lanes of a warp are 32 neighbouring columns, whose footprints are
// neighbouring cells); in deterministic mode the contributions are added as
// int64 fixed point instead.  A^T gathers: one thread per column segment of
// kSfZB voxels loops over all views and sums the cells under each voxel's
// footprint into shared memory, so every voxel is written once, without
// reductions; the transaxial footprint of a column and the u-weighted sums
// of the detector rows under the segment are computed once per view and
// segment.  Neighbouring voxels of a segment share their common z face: a
// voxel's axial trapezoid is the difference of its two faces' ramps, so the
// cells under each face are integrated once, not once per voxel.  Ramp
// reciprocals are taken once per trapezoid or face, not per cell.
// Coordinates are relative to the volume centre (per-view constants computed
// in FP64 on the host), which keeps the FP32 breakpoints accurate.
#include "ct_debug.cuh"
#include <algorithm>
#include <cmath>
#include <vector>

#include "ct_internal.h"

namespace ct {
namespace {

// Transaxial cells kept in registers per pass (footprints wider than that
// take several passes), in A and A^T (measured at 256^3, 1 mm voxels and
// pixels, magnification 1.6: footprints of 2-4 cells).
constexpr int kSfKUF = 4;
constexpr int kSfZB = 16;    // voxels per A^T thread (a column segment; sums in shared memory)
constexpr int kSfRows = 32;  // detector rows under one A^T segment kept in shared memory

struct SfColumn {
    float tau[4];          // sorted transaxial breakpoints (pixel index units)
    float qa, qb;          // SDD / (dv t) at the two axial depths (TR: both the centre's)
    float r01, r23;        // 1 / (2 ramp width) of the transaxial trapezoid
    float m;               // min(hx / |d_x|, hy / |d_y|)
    float dxy2;            // d_x^2 + d_y^2
    int ku0, ku1;          // cells overlapping the footprint, clipped to the detector
};

__device__ __forceinline__ void sort4(float &a, float &b, float &c, float &d) {
    float t;
#define CT_CSWAP(x, y) \
    if (y < x) {       \
        t = x;         \
        x = y;         \
        y = t;         \
    }
    CT_CSWAP(a, b);
    CT_CSWAP(c, d);
    CT_CSWAP(a, c);
    CT_CSWAP(b, d);
    CT_CSWAP(b, c);
#undef CT_CSWAP
}

// 1 / (2 w): the factor of a ramp of width w in trap_cell, taken once per
// trapezoid (a zero width gives infinity, which trap_cell never reaches: an
// empty ramp has no overlap with any cell).
__device__ __forceinline__ float half_rcp(float w) { return 0.5f / w; }

// Integral of the unit trapezoid t0 <= t1 <= t2 <= t3 over [a, b], summed
// piece by piece (no difference of large antiderivatives); r01 and r23 are
// half_rcp of the two ramp widths.
__device__ __forceinline__ float trap_cell(float t0, float t1, float t2, float t3, float r01,
                                           float r23, float a, float b) {
    float r = 0.f;
    float x1 = fmaxf(a, t0), x2 = fminf(b, t1);
    if (x2 > x1) r += (x2 - x1) * (x2 + x1 - 2.f * t0) * r01;
    x1 = fmaxf(a, t1);
    x2 = fminf(b, t2);
    if (x2 > x1) r += x2 - x1;
    x1 = fmaxf(a, t2);
    x2 = fminf(b, t3);
    if (x2 > x1) r += (x2 - x1) * (2.f * t3 - x1 - x2) * r23;
    return r;
}

// Integral over [a, b] of the ramp that rises from 0 at lo to 1 at hi and
// stays 1 above (r = half_rcp(hi - lo)); RAMP false: a step at lo == hi.
template <bool RAMP>
__device__ __forceinline__ float ramp_cell(float lo, float hi, float r, float a, float b) {
    float s = 0.f;
    if (RAMP) {
        const float x1 = fmaxf(a, lo), x2 = fminf(b, hi);
        if (x2 > x1) s = (x2 - x1) * (x2 + x1 - 2.f * lo) * r;
    }
    const float x1 = fmaxf(a, hi);
    if (b > x1) s += b - x1;
    return s;
}

// Column (i, j) of view `view`: transaxial footprint, axial depths, amplitude.
template <bool TT>
__device__ __forceinline__ bool sf_column(const ProjGeom &g, int view, int i, int j, SfColumn &c) {
    const float4 a = __ldg(g.sf_view + 2 * view);      // s0, t0, eux, euy
    const float4 b = __ldg(g.sf_view + 2 * view + 1);  // ecx, ecy, dx0, dy0
    const float rx = ((float)i - 0.5f * (float)(g.nx - 1)) * g.hx;
    const float ry = ((float)j - 0.5f * (float)(g.ny - 1)) * g.hy;
    const float hx = 0.5f * g.hx, hy = 0.5f * g.hy;
    float u[4], t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float px = rx + ((q & 1) ? hx : -hx);
        const float py = ry + ((q & 2) ? hy : -hy);
        const float su = fmaf(px, a.z, fmaf(py, a.w, a.x));
        t[q] = fmaf(px, b.x, fmaf(py, b.y, a.y));
        u[q] = fmaf(g.sf_ku, su / t[q], g.sf_cu);
    }
    c.tau[0] = u[0];
    c.tau[1] = u[1];
    c.tau[2] = u[2];
    c.tau[3] = u[3];
    sort4(c.tau[0], c.tau[1], c.tau[2], c.tau[3]);
    c.r01 = half_rcp(c.tau[1] - c.tau[0]);
    c.r23 = half_rcp(c.tau[3] - c.tau[2]);
    if (TT) {
        const float tmin = fminf(fminf(t[0], t[1]), fminf(t[2], t[3]));
        const float tmax = fmaxf(fmaxf(t[0], t[1]), fmaxf(t[2], t[3]));
        c.qa = g.sf_kv / tmin;
        c.qb = g.sf_kv / tmax;
    } else {
        const float tc = fmaf(rx, b.x, fmaf(ry, b.y, a.y));
        c.qa = c.qb = g.sf_kv / tc;
    }
    const float dx = b.z + rx, dy = b.w + ry;
    const float mx = dx != 0.f ? g.hx / fabsf(dx) : INFINITY;
    const float my = dy != 0.f ? g.hy / fabsf(dy) : INFINITY;
    c.m = fminf(mx, my);
    c.dxy2 = fmaf(dx, dx, dy * dy);
    c.ku0 = max(0, (int)floorf(c.tau[0] + 0.5f));
    c.ku1 = min(g.nu - 1, (int)floorf(c.tau[3] + 0.5f));
    return c.ku0 <= c.ku1;
}

// Axial footprint (breakpoints vb, half_rcp of its ramps) and amplitude of
// voxel k of the column.
template <bool TT>
__device__ __forceinline__ void sf_axial(const ProjGeom &g, const SfColumn &c, int k, float *vb,
                                         float &amp, float &r01, float &r23) {
    const float rz = ((float)k - 0.5f * (float)(g.nz - 1)) * g.hz;
    const float z = g.sf_oz + rz;
    const float zlo = z - 0.5f * g.hz, zhi = z + 0.5f * g.hz;
    if (TT) {
        vb[0] = fmaf(zlo, c.qa, g.sf_cv);
        vb[1] = fmaf(zlo, c.qb, g.sf_cv);
        vb[2] = fmaf(zhi, c.qa, g.sf_cv);
        vb[3] = fmaf(zhi, c.qb, g.sf_cv);
        sort4(vb[0], vb[1], vb[2], vb[3]);
        r01 = half_rcp(vb[1] - vb[0]);
        r23 = half_rcp(vb[3] - vb[2]);
    } else {
        const float p = fmaf(zlo, c.qa, g.sf_cv), q = fmaf(zhi, c.qa, g.sf_cv);
        vb[0] = vb[1] = fminf(p, q);
        vb[2] = vb[3] = fmaxf(p, q);
        r01 = r23 = 0.f;
    }
    amp = c.m * sqrtf(fmaf(z, z, c.dxy2));
}

__device__ __forceinline__ void coef_sf(const Coef &c, float &alpha) {
    alpha = c.dev ? (float)c.dev[0] : c.alpha;
}

// out[view][v][u] += alpha * rho * A x over the columns (i, j) of one view.
// DET: each contribution is scaled by det_scale[0] (a power of two), rounded
// to an integer and added to the int64 sums qacc instead, which makes the
// result independent of the order of the additions.
template <bool HAS_RHO, bool UNIT_VOL, bool TT, bool DET>
__global__ void __launch_bounds__(256) k_sf_forward(ProjGeom g, const float *__restrict__ vol,
                                                    float *__restrict__ out,
                                                    const float *__restrict__ rho, Coef cf,
                                                    long long *__restrict__ qacc,
                                                    const float *__restrict__ det_scale) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int view = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    SfColumn c;
    if (!sf_column<TT>(g, view, i, j, c)) return;
    float alpha;
    coef_sf(cf, alpha);
    const float scale = DET ? __ldg(det_scale) : 1.f;
    const size_t vbase = (size_t)view * g.nv * g.nu;
    const size_t plane = (size_t)g.nx * g.ny;
    for (int k0 = c.ku0; k0 <= c.ku1; k0 += kSfKUF) {
        float fu[kSfKUF];
        const int nk = min(kSfKUF, c.ku1 - k0 + 1);
#pragma unroll
        for (int q = 0; q < kSfKUF; ++q)
            fu[q] = q < nk ? trap_cell(c.tau[0], c.tau[1], c.tau[2], c.tau[3], c.r01, c.r23,
                                       (float)(k0 + q) - 0.5f, (float)(k0 + q) + 0.5f)
                           : 0.f;
        const size_t col = (size_t)j * g.nx + i;
        auto load = [&](int k) -> float {
            const size_t vi = (size_t)k * plane + col;
            return UNIT_VOL || !CT_IN_BOUNDS(vi, plane * g.nz) ? 1.f : vol[vi];
        };
        float xn = load(0);  // each voxel's value is loaded one voxel ahead
        for (int k = 0; k < g.nz; ++k) {
            const float xv = xn;
            if (k + 1 < g.nz) xn = load(k + 1);
            if (xv == 0.f) continue;
            float vb[4], amp, vr01, vr23;
            sf_axial<TT>(g, c, k, vb, amp, vr01, vr23);
            const int kv0 = max(0, (int)floorf(vb[0] + 0.5f));
            const int kv1 = min(g.nv - 1, (int)floorf(vb[3] + 0.5f));
            for (int l = kv0; l <= kv1; ++l) {
                const float fv = trap_cell(vb[0], vb[1], vb[2], vb[3], vr01, vr23,
                                           (float)l - 0.5f, (float)l + 0.5f);
                if (fv == 0.f) continue;
                const float base = alpha * amp * fv * xv;
                const size_t row = vbase + (size_t)l * g.nu;
#pragma unroll
                for (int q = 0; q < kSfKUF; ++q) {
                    if (q < nk && fu[q] != 0.f &&
                        CT_IN_BOUNDS(k0 + q, g.nu) && CT_IN_BOUNDS(l, g.nv)) {
                        float val = base * fu[q];
                        if (HAS_RHO) val *= rho[row + k0 + q];
                        if (DET)
                            atomicAdd(reinterpret_cast<unsigned long long *>(qacc) + row + k0 + q,
                                      (unsigned long long)__float2ll_rn(val * scale));
                        else
                            atomicAdd(out + row + k0 + q, val);
                    }
                }
            }
        }
    }
}

// acc[z][y][x] += alpha * sum over views and cells of A_ij^POWER rho_i e_i
// (e == NULL: e = 1).  A CTA covers 32 x 8 voxel columns and kSfZB voxels of
// each column, one thread per column, with its kSfZB sums in shared memory:
// the transaxial footprint of a column and view is computed once for the
// whole segment, in passes of kSfKUF cells kept in registers, and so is the
// u-weighted sum of each detector row under the segment (up to kSfRows rows
// in shared memory; a segment spanning more rows sums them per voxel), and
// the cell integrals under each z face of the segment (power 1).
template <bool HAS_RHO, int POWER, bool TT>
__global__ void __launch_bounds__(256) k_sf_backward(ProjGeom g, const float *__restrict__ e,
                                                     const float *__restrict__ rho, Coef cf,
                                                     float *__restrict__ acc) {
    __shared__ float sacc[kSfZB][256];
    __shared__ float srow[kSfRows][256];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int kz0 = blockIdx.z * kSfZB;
    const int nzs = min(kSfZB, g.nz - kz0);
    for (int dz = 0; dz < kSfZB; ++dz) sacc[dz][tid] = 0.f;
    // no CTA-wide synchronisation: every thread touches its own column only
    if (i < g.nx && j < g.ny) {
        for (int view = 0; view < g.nviews; ++view) {
            SfColumn c;
            if (!sf_column<TT>(g, view, i, j, c)) continue;
            const size_t vbase = (size_t)view * g.nv * g.nu;
            for (int k0 = c.ku0; k0 <= c.ku1; k0 += kSfKUF) {
                float fu[kSfKUF];
                const int nk = min(kSfKUF, c.ku1 - k0 + 1);
#pragma unroll
                for (int q = 0; q < kSfKUF; ++q)
                    fu[q] = q < nk ? trap_cell(c.tau[0], c.tau[1], c.tau[2], c.tau[3], c.r01,
                                               c.r23, (float)(k0 + q) - 0.5f,
                                               (float)(k0 + q) + 0.5f)
                                   : 0.f;
                auto row_sum = [&](int l) -> float {
                    const size_t row = vbase + (size_t)l * g.nu + k0;
                    float su = 0.f;
#pragma unroll
                    for (int q = 0; q < kSfKUF; ++q) {
                        if (q < nk && fu[q] != 0.f &&
                            CT_IN_BOUNDS(k0 + q, g.nu) && CT_IN_BOUNDS(l, g.nv)) {
                            float w = e ? e[row + q] : 1.f;
                            if (HAS_RHO) w *= rho[row + q];
                            su = POWER == 1 ? fmaf(fu[q], w, su) : fmaf(fu[q] * fu[q], w, su);
                        }
                    }
                    return su;
                };
                // The faces of the segment: face f is the bottom of voxel
                // kz0 + f, seen as the ramp from lo (its lower projection)
                // to hi (its upper one; TR: lo == hi, a step).  Both grow
                // with z (every depth is positive), so voxel k's axial
                // footprint is ramp_k - ramp_{k+1} wherever the two ramps
                // do not overlap (hi_k <= lo_{k+1}), and its sum over the
                // rows is W_k - W_{k+1} plus the rows wholly above ramp k
                // and not above ramp k+1 (W_f: the ramp's cells weighted
                // by the rows' sums).  Voxels whose ramps overlap sum their
                // own trapezoid.  POWER 2 squares every cell and sums
                // trapezoids throughout.
                const bool faces = POWER == 1 && c.qb > 0.f;
                auto face = [&](int f, float &lo, float &hi, int &a, int &b) {
                    const float z = fmaf((float)(kz0 + f) - 0.5f * (float)g.nz, g.hz, g.sf_oz);
                    const float p = fmaf(z, c.qa, g.sf_cv);
                    const float q = TT ? fmaf(z, c.qb, g.sf_cv) : p;
                    lo = fminf(p, q);
                    hi = fmaxf(p, q);
                    a = max(0, (int)floorf(lo + 0.5f));
                    b = min(max((int)floorf(hi + 0.5f), -1), g.nv - 1);
                };
                // rows under the segment (v grows with z): their u-weighted
                // sums once each, shared by the voxels above them
                float vb[4], amp, vr01, vr23;
                int lf, ll;
                if (faces) {
                    float lo, hi;
                    int a, b;
                    face(0, lo, hi, lf, b);
                    face(nzs, lo, hi, a, ll);
                } else {
                    sf_axial<TT>(g, c, kz0, vb, amp, vr01, vr23);
                    lf = max(0, (int)floorf(vb[0] + 0.5f));
                    sf_axial<TT>(g, c, kz0 + nzs - 1, vb, amp, vr01, vr23);
                    ll = min(g.nv - 1, (int)floorf(vb[3] + 0.5f));
                }
                const unsigned ncached = ll - lf < kSfRows ? (unsigned)max(ll - lf + 1, 0) : 0u;
                for (int l = lf; l < lf + (int)ncached; ++l) srow[l - lf][tid] = row_sum(l);
                auto su_of = [&](int l) -> float {
                    const unsigned r = (unsigned)(l - lf);
                    return r < ncached ? srow[r][tid] : row_sum(l);
                };
                // voxel kz0 + dz from its own trapezoid
                auto voxel_trap = [&](int dz) -> float {
                    sf_axial<TT>(g, c, kz0 + dz, vb, amp, vr01, vr23);
                    const int kv0 = max(0, (int)floorf(vb[0] + 0.5f));
                    const int kv1 = min(g.nv - 1, (int)floorf(vb[3] + 0.5f));
                    float s = 0.f;
                    for (int l = kv0; l <= kv1; ++l) {
                        const float fv = trap_cell(vb[0], vb[1], vb[2], vb[3], vr01, vr23,
                                                   (float)l - 0.5f, (float)l + 0.5f);
                        if (fv == 0.f) continue;
                        s = POWER == 1 ? fmaf(fv, su_of(l), s) : fmaf(fv * fv, su_of(l), s);
                    }
                    return s;
                };
                if (faces) {
                    auto ramp_sum = [&](float lo, float hi, int a, int b) -> float {
                        const float r = TT ? half_rcp(hi - lo) : 0.f;
                        float w = 0.f;
                        for (int l = a; l <= b; ++l)
                            w = fmaf(ramp_cell<TT>(lo, hi, r, (float)l - 0.5f, (float)l + 0.5f),
                                     su_of(l), w);
                        return w;
                    };
                    float lo0, hi0, w0;
                    int a0, b0;
                    face(0, lo0, hi0, a0, b0);
                    w0 = ramp_sum(lo0, hi0, a0, b0);
                    for (int dz = 0; dz < nzs; ++dz) {
                        float lo1, hi1;
                        int a1, b1;
                        face(dz + 1, lo1, hi1, a1, b1);
                        const float w1 = ramp_sum(lo1, hi1, a1, b1);
                        float s;
                        if (hi0 <= lo1) {
                            s = w0 - w1;
                            for (int l = max(b0 + 1, 0); l <= b1; ++l) s += su_of(l);
                        } else {
                            s = voxel_trap(dz);
                        }
                        if (s != 0.f) {
                            const float z = g.sf_oz + ((float)(kz0 + dz) - 0.5f * (float)(g.nz - 1)) * g.hz;
                            amp = c.m * sqrtf(fmaf(z, z, c.dxy2));
                            sacc[dz][tid] = fmaf(amp, s, sacc[dz][tid]);
                        }
                        lo0 = lo1;
                        hi0 = hi1;
                        w0 = w1;
                        b0 = b1;
                    }
                } else {
                    for (int dz = 0; dz < nzs; ++dz) {
                        const float s = voxel_trap(dz);
                        if (s != 0.f)
                            sacc[dz][tid] = POWER == 1 ? fmaf(amp, s, sacc[dz][tid])
                                                       : fmaf(amp * amp, s, sacc[dz][tid]);
                    }
                }
            }
        }
        float alpha;
        coef_sf(cf, alpha);
        const size_t plane = (size_t)g.nx * g.ny;
        for (int dz = 0; dz < nzs; ++dz) {
            const size_t idx = (size_t)(kz0 + dz) * plane + (size_t)j * g.nx + i;
            if (CT_IN_BOUNDS(idx, plane * g.nz)) acc[idx] = fmaf(alpha, sacc[dz][tid], acc[idx]);
        }
    }
}

// Number of (ray, voxel) pairs with A_ij > 0.
template <bool TT>
__global__ void __launch_bounds__(256) k_sf_count(ProjGeom g, unsigned long long *__restrict__ n) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int view = blockIdx.z;
    unsigned long long cnt = 0;
    if (i < g.nx && j < g.ny) {
        SfColumn c;
        if (sf_column<TT>(g, view, i, j, c)) {
            int nu_nz = 0;
            for (int k = c.ku0; k <= c.ku1; ++k)
                nu_nz += trap_cell(c.tau[0], c.tau[1], c.tau[2], c.tau[3], c.r01, c.r23,
                                   (float)k - 0.5f, (float)k + 0.5f) > 0.f;
            for (int k = 0; k < g.nz; ++k) {
                float vb[4], amp, vr01, vr23;
                sf_axial<TT>(g, c, k, vb, amp, vr01, vr23);
                const int kv0 = max(0, (int)floorf(vb[0] + 0.5f));
                const int kv1 = min(g.nv - 1, (int)floorf(vb[3] + 0.5f));
                int nv_nz = 0;
                for (int l = kv0; l <= kv1; ++l)
                    nv_nz += trap_cell(vb[0], vb[1], vb[2], vb[3], vr01, vr23, (float)l - 0.5f,
                                       (float)l + 0.5f) > 0.f;
                cnt += (unsigned long long)(nu_nz * nv_nz);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n, cnt);
}

// p = beta p + q inv (beta from c; beta 0: p is not read), int64 sums q of
// a fixed-point forward projection.
__global__ void k_sf_combine_det(float *__restrict__ p, const long long *__restrict__ q,
                                 const double *__restrict__ inv, int64_t m, Coef c) {
    const double s = __ldg(inv);
    const float beta = c.dev ? (float)c.dev[1] : c.beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        float val = (float)((double)q[i] * s);
        if (beta != 0.f) val = fmaf(beta, p[i], val);
        p[i] = val;
    }
}

// out = beta * out + acc (volumes in the caller's layout).
__global__ void k_sf_axpby(float *__restrict__ out, const float *__restrict__ acc, int64_t n,
                           float beta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = beta != 0.f ? fmaf(beta, out[i], acc[i]) : acc[i];
}

dim3 sf_cols_grid(const ProjGeom &pg, int z) {
    return dim3((unsigned)((pg.nx + 31) / 32), (unsigned)((pg.ny + 7) / 8), (unsigned)z);
}

}  // namespace

void sf_view_constants(const ct_geometry_desc &d, const std::vector<double> &ang,
                       std::vector<float4> &out, float *scal) {
    // scal: ku = SDD / du, kv = SDD / dv, cu, cv, oz
    out.resize(2 * ang.size());
    const double O[3] = {d.off_x, d.off_y, d.off_z};
    for (size_t k = 0; k < ang.size(); ++k) {
        const double c = std::cos(ang[k]), s = std::sin(ang[k]);
        const double src[3] = {d.sid * c, d.sid * s, 0.0};
        const double eu[2] = {-s, c}, ec[2] = {-c, -s};
        const double r0[2] = {O[0] - src[0], O[1] - src[1]};
        const double s0 = r0[0] * eu[0] + r0[1] * eu[1];
        const double t0 = r0[0] * ec[0] + r0[1] * ec[1];
        out[2 * k] = make_float4((float)s0, (float)t0, (float)eu[0], (float)eu[1]);
        out[2 * k + 1] = make_float4((float)ec[0], (float)ec[1], (float)r0[0], (float)r0[1]);
    }
    scal[0] = (float)(d.sdd / d.du);
    scal[1] = (float)(d.sdd / d.dv);
    scal[2] = (float)(0.5 * (d.nu - 1) - d.det_off_u / d.du);
    scal[3] = (float)(0.5 * (d.nv - 1) - d.det_off_v / d.dv);
    scal[4] = (float)d.off_z;
}

int64_t sf_forward_partials(const ProjGeom &pg) {
    return (int64_t)vec_grid((int64_t)pg.nviews * pg.nv * pg.nu);
}

namespace {
// Byte offsets in the fixed-point forward scratch: int64 sums of the m rays,
// the inverse scale (double), the scale (float), the maxima partials.
struct SfDetLayout {
    size_t q, inv, scale, part, bytes;
    explicit SfDetLayout(const ProjGeom &pg) {
        const int64_t m = (int64_t)pg.nviews * pg.nv * pg.nu;
        const int64_t n = (int64_t)pg.nx * pg.ny * pg.nz;
        q = 0;
        inv = (size_t)m * sizeof(long long);
        scale = inv + 16;
        part = scale + 16;
        bytes = part + (size_t)(vec_grid(n) + vec_grid(m)) * sizeof(float);
    }
};

template <bool DET>
ct_status sf_forward_launch(const ProjGeom &pg, const float *vol, float *p, const float *rho,
                            Coef c, long long *qacc, const float *det_scale, cudaStream_t st) {
    const dim3 gr = sf_cols_grid(pg, pg.nviews), bl(32, 8);
    const bool tt = pg.proj == CT_PROJ_SF_TT, hr = rho != nullptr, unit = vol == nullptr;
#define CT_SFF(HR, UV, TT_) \
    k_sf_forward<HR, UV, TT_, DET><<<gr, bl, 0, st>>>(pg, vol, p, rho, c, qacc, det_scale)
    if (tt) {
        if (hr) { if (unit) CT_SFF(true, true, true); else CT_SFF(true, false, true); }
        else    { if (unit) CT_SFF(false, true, true); else CT_SFF(false, false, true); }
    } else {
        if (hr) { if (unit) CT_SFF(true, true, false); else CT_SFF(true, false, false); }
        else    { if (unit) CT_SFF(false, true, false); else CT_SFF(false, false, false); }
    }
#undef CT_SFF
    CT_CHECK_LAUNCH();
    return CT_OK;
}
}  // namespace

size_t sf_det_ws_bytes(const ProjGeom &pg) { return SfDetLayout(pg).bytes; }

double sf_row_bound(const ct_geometry_desc &d) {
    // A_ij = l_j Fbar_u Fbar_v with both cell averages of unit-height
    // footprints at most 1, so a cell's sum is at most (voxels) * max l_j.
    // l = |d| min(vx / |d_x|, vy / |d_y|) <= sqrt(2) max(vx, vy) |d| / |d_xy|
    // for d = centre - source, and |d| / |d_xy| <= sqrt(1 + z^2 / r^2) with
    // z the largest |z| of a voxel centre and r = SID - (largest xy radius of
    // the volume's corners) the smallest distance in the xy plane.
    double rmax = 0.0;
    for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy) {
            const double x = (cx ? 0.5 : -0.5) * d.nx * d.vx + d.off_x;
            const double y = (cy ? 0.5 : -0.5) * d.ny * d.vy + d.off_y;
            rmax = std::max(rmax, std::sqrt(x * x + y * y));
        }
    const double r = d.sid - rmax;
    const double z = std::fabs(d.off_z) + 0.5 * std::max(d.nz - 1, 0) * d.vz;
    const double lmax = std::sqrt(2.0) * std::max(d.vx, d.vy) * std::sqrt(1.0 + (z * z) / (r * r));
    // 2x slack covers the FP32 rounding of the footprint factors
    return 2.0 * lmax * (double)d.nx * (double)d.ny * (double)std::max(d.nz, 1);
}

ct_status sf_forward(const ProjGeom &pg, const float *vol, float *p, const float *rho, Coef c,
                     double *partials, cudaStream_t st) {
    const int64_t m = (int64_t)pg.nviews * pg.nv * pg.nu;
    if (!pg.sf_det) {
        if (c.dev) CT_TRY(launch_scale_dev(p, m, c.dev + 1, st));
        else CT_TRY(launch_scale(p, m, c.beta, st));
        CT_TRY(sf_forward_launch<false>(pg, vol, p, rho, c, nullptr, nullptr, st));
    } else {
        // int64 fixed point: sums, then p = beta p + sums * 2^-k
        const SfDetLayout lay(pg);
        Workspace ws(st);
        char *base = static_cast<char *>(pg.sf_ws);
        if (!base) CT_TRY(ws.alloc(reinterpret_cast<void **>(&base), lay.bytes));
        long long *q = reinterpret_cast<long long *>(base + lay.q);
        double *inv = reinterpret_cast<double *>(base + lay.inv);
        float *scale = reinterpret_cast<float *>(base + lay.scale);
        float *part = reinterpret_cast<float *>(base + lay.part);
        const int64_t n = (int64_t)pg.nx * pg.ny * pg.nz;
        CT_CUDA_TRY(cudaMemsetAsync(q, 0, (size_t)m * sizeof(long long), st));
        CT_TRY(launch_det_scale_fwd(vol, n, rho, m, pg.sf_row_bound, c, part, scale, inv, st));
        CT_TRY(sf_forward_launch<true>(pg, vol, p, rho, c, q, scale, st));
        k_sf_combine_det<<<vec_grid(m), kVecThreads, 0, st>>>(p, q, inv, m, c);
        CT_CHECK_LAUNCH();
    }
    if (partials) CT_TRY(launch_norm2(p, nullptr, m, partials, st));
    return CT_OK;
}

ct_status sf_backward(const ProjGeom &pg, const float *e, const float *rho, Coef c, float *acc,
                      int power, cudaStream_t st) {
    const dim3 gr = sf_cols_grid(pg, (pg.nz + kSfZB - 1) / kSfZB), bl(32, 8);
    const bool tt = pg.proj == CT_PROJ_SF_TT, hr = rho != nullptr;
#define CT_SFB(HR, P, TT_) k_sf_backward<HR, P, TT_><<<gr, bl, 0, st>>>(pg, e, rho, c, acc)
    if (tt) {
        if (power == 2) { if (hr) CT_SFB(true, 2, true); else CT_SFB(false, 2, true); }
        else            { if (hr) CT_SFB(true, 1, true); else CT_SFB(false, 1, true); }
    } else {
        if (power == 2) { if (hr) CT_SFB(true, 2, false); else CT_SFB(false, 2, false); }
        else            { if (hr) CT_SFB(true, 1, false); else CT_SFB(false, 1, false); }
    }
#undef CT_SFB
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status sf_count(const ProjGeom &pg, unsigned long long *d_count, cudaStream_t st) {
    const dim3 gr = sf_cols_grid(pg, pg.nviews), bl(32, 8);
    if (pg.proj == CT_PROJ_SF_TT) k_sf_count<true><<<gr, bl, 0, st>>>(pg, d_count);
    else k_sf_count<false><<<gr, bl, 0, st>>>(pg, d_count);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status sf_axpby(float *out, const float *acc, int64_t n, float beta, cudaStream_t st) {
    if (n <= 0) return CT_OK;
    k_sf_axpby<<<vec_grid(n), kVecThreads, 0, st>>>(out, acc, n, beta);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace ct

CT_DEBUG_ACCESSOR(debug_take_footprint)
