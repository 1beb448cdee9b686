/*
 * FP64 CPU oracle for the cone-beam CT operator A and its transpose.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code with the CUDA library and is deliberately slow and plain.
 *
 * What it computes (Materials and Methods, Eq. 1: b = A x, with A the sparse
 * CBCT system matrix, never stored; Software section: the Siddon ray-caster):
 *   A_ij = length in mm of ray i inside voxel j (Siddon 1985, the exact
 *   radiological path of a straight ray through a grid of box voxels).
 *
 * The plain definition is written out directly:
 *   1. clip the segment source->pixel centre, r(t) = s + t (p - s), t in [0,1],
 *      against the volume box (slab method) -> [t_min, t_max];
 *   2. collect every t where the ray crosses an x-, y- or z-grid plane inside
 *      (t_min, t_max), each computed directly as (plane - s_a) / d_a;
 *   3. sort all of them together with t_min and t_max;
 *   4. every consecutive pair (t_a, t_b) with t_b > t_a is one segment: the
 *      voxel is floor((r((t_a + t_b)/2) - box_lo) / h) per axis (midpoint
 *      rule) and its length is (t_b - t_a) * |p - s|.
 * A^T is the same loop scattering length * e_i into the voxel, so it is the
 * transpose of A by construction.
 *
 * Geometry (the paper fixes none of it; the reading used throughout):
 *   circular orbit about +z, view angle theta;
 *   source  s = SID (cos th, sin th, 0);
 *   detector centre c = -(SDD - SID) (cos th, sin th, 0), flat;
 *   e_u = (-sin th, cos th, 0), e_v = (0, 0, 1);
 *   pixel (u, v) centre = c + ((u - (Nu-1)/2) du + off_u) e_u
 *                           + ((v - (Nv-1)/2) dv + off_v) e_v;
 *   volume box lo = -N h / 2 + o per axis (o = off-centre offset),
 *   voxel (i, j, k) stored at k*Ny*Nx + j*Nx + i;
 *   sinogram (view, v, u) stored at (view*Nv + v)*Nu + u.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny, nz;
    double vx, vy, vz;
    double ox, oy, oz;
    int32_t nu, nv;
    double du, dv;
    double det_off_u, det_off_v;
    double sid, sdd;
    int32_t nviews;
    const double *angles; /* nviews view angles in radians */
} oref_geom;

static void box_lo(const oref_geom *g, double lo[3], double h[3], int n[3]) {
    n[0] = g->nx; n[1] = g->ny; n[2] = g->nz;
    h[0] = g->vx; h[1] = g->vy; h[2] = g->vz;
    lo[0] = -0.5 * g->nx * g->vx + g->ox;
    lo[1] = -0.5 * g->ny * g->vy + g->oy;
    lo[2] = -0.5 * g->nz * g->vz + g->oz;
}

/* Source and pixel-centre positions of ray (view, u, v). */
static void ray_endpoints(const oref_geom *g, int view, int u, int v,
                          double s[3], double p[3]) {
    double th = g->angles[view];
    double ct = cos(th), st = sin(th);
    s[0] = g->sid * ct; s[1] = g->sid * st; s[2] = 0.0;
    double cdist = -(g->sdd - g->sid);
    double uu = (u - 0.5 * (g->nu - 1)) * g->du + g->det_off_u;
    double vv = (v - 0.5 * (g->nv - 1)) * g->dv + g->det_off_v;
    p[0] = cdist * ct + uu * (-st);
    p[1] = cdist * st + uu * ct;
    p[2] = vv;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Segments of the ray s->p through the voxel grid: linear voxel index and
 * length in mm.  tbuf must hold nx+ny+nz+5 doubles.  Returns the count. */
static int ray_segments(const oref_geom *g, const double s[3], const double p[3],
                        int64_t *idx, double *len, double *tbuf) {
    double lo[3], h[3];
    int n[3];
    box_lo(g, lo, h, n);
    double d[3] = {p[0] - s[0], p[1] - s[1], p[2] - s[2]};
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double tmin = 0.0, tmax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double hi = lo[a] + n[a] * h[a];
        if (d[a] != 0.0) {
            double t0 = (lo[a] - s[a]) / d[a];
            double t1 = (hi - s[a]) / d[a];
            double ta = t0 < t1 ? t0 : t1, tb = t0 < t1 ? t1 : t0;
            if (ta > tmin) tmin = ta;
            if (tb < tmax) tmax = tb;
        } else if (s[a] < lo[a] || s[a] >= hi) {
            return 0;
        }
    }
    if (!(tmin < tmax)) return 0;
    int nt = 0;
    tbuf[nt++] = tmin;
    tbuf[nt++] = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        for (int q = 0; q <= n[a]; ++q) {
            double t = (lo[a] + q * h[a] - s[a]) / d[a];
            if (t > tmin && t < tmax) tbuf[nt++] = t;
        }
    }
    qsort(tbuf, (size_t)nt, sizeof(double), cmp_double);
    int ns = 0;
    for (int q = 0; q + 1 < nt; ++q) {
        double ta = tbuf[q], tb = tbuf[q + 1];
        if (!(tb > ta)) continue;
        double tm = 0.5 * (ta + tb);
        int64_t ijk[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            double c = (s[a] + tm * d[a] - lo[a]) / h[a];
            int64_t i = (int64_t)floor(c);
            if (i < 0 || i >= n[a]) inside = 0;
            ijk[a] = i;
        }
        if (!inside) continue;
        idx[ns] = (ijk[2] * g->ny + ijk[1]) * (int64_t)g->nx + ijk[0];
        len[ns] = (tb - ta) * L;
        ++ns;
    }
    return ns;
}

static int cap_of(const oref_geom *g) { return g->nx + g->ny + g->nz + 5; }

static int valid(const oref_geom *g) {
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nu < 0 || g->nv < 0 ||
        g->nviews < 0)
        return 0;
    if (!(g->vx > 0 && g->vy > 0 && g->vz > 0 && g->du > 0 && g->dv > 0)) return 0;
    if (g->nviews > 0 && !g->angles) return 0;
    return 1;
}

/* Segments of one ray, for tests.  Returns the count, or -1 if cap is short. */
int oref_ray(const oref_geom *g, int view, int u, int v, int64_t *idx, double *len,
             int cap) {
    if (!valid(g) || cap < cap_of(g)) return -1;
    double s[3], p[3];
    double *tbuf = (double *)malloc(sizeof(double) * (size_t)cap_of(g));
    if (!tbuf) return -1;
    ray_endpoints(g, view, u, v, s, p);
    int ns = ray_segments(g, s, p, idx, len, tbuf);
    free(tbuf);
    return ns;
}

/* Segments of an arbitrary segment s->p, for hand-built tests. */
int oref_segment(const oref_geom *g, const double *s, const double *p, int64_t *idx,
                 double *len, int cap) {
    if (!valid(g) || cap < cap_of(g)) return -1;
    double *tbuf = (double *)malloc(sizeof(double) * (size_t)cap_of(g));
    if (!tbuf) return -1;
    int ns = ray_segments(g, s, p, idx, len, tbuf);
    free(tbuf);
    return ns;
}

/* sino = A vol.  vol: [nz][ny][nx]; sino: [nviews][nv][nu].  0 on success. */
int oref_project(const oref_geom *g, const double *vol, double *sino, int nthreads) {
    if (!valid(g)) return 1;
    int64_t nrays = (int64_t)g->nviews * g->nv * g->nu;
    int cap = cap_of(g);
    int failed = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
        double *tbuf = (double *)malloc(sizeof(double) * (size_t)cap);
        if (!idx || !len || !tbuf) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < nrays; ++r) {
                int u = (int)(r % g->nu);
                int v = (int)((r / g->nu) % g->nv);
                int view = (int)(r / ((int64_t)g->nu * g->nv));
                double s[3], p[3];
                ray_endpoints(g, view, u, v, s, p);
                int ns = ray_segments(g, s, p, idx, len, tbuf);
                double acc = 0.0;
                for (int q = 0; q < ns; ++q) acc += len[q] * vol[idx[q]];
                sino[r] = acc;
            }
        }
        free(idx); free(len); free(tbuf);
    }
    return failed ? 2 : 0;
}

/* vol = A^T sino (power = 1) or vol = (A o A)^T sino (power = 2, squared
 * lengths; with sino = 1 this is diag(A^T A)).  Per-thread buffers are summed
 * in thread order, so the result does not depend on scheduling. */
int oref_backproject(const oref_geom *g, const double *sino, double *vol, int nthreads,
                     int power) {
    if (!valid(g) || (power != 1 && power != 2)) return 1;
    int64_t nvox = (int64_t)g->nx * g->ny * g->nz;
    int64_t nrays = (int64_t)g->nviews * g->nv * g->nu;
    int nt = nthreads > 0 ? nthreads : 1;
    /* keep the private buffers under ~8 GB */
    int64_t maxnt = (int64_t)(8.0e9 / (8.0 * (double)nvox));
    if (maxnt < 1) maxnt = 1;
    if (nt > maxnt) nt = (int)maxnt;
    double *buf = (double *)calloc((size_t)nt * (size_t)nvox, sizeof(double));
    if (!buf) return 2;
    int cap = cap_of(g);
    int failed = 0;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = buf + (size_t)tid * (size_t)nvox;
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
        double *tbuf = (double *)malloc(sizeof(double) * (size_t)cap);
        if (!idx || !len || !tbuf) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t r = 0; r < nrays; ++r) {
                double e = sino[r];
                if (e == 0.0) continue;
                int u = (int)(r % g->nu);
                int v = (int)((r / g->nu) % g->nv);
                int view = (int)(r / ((int64_t)g->nu * g->nv));
                double s[3], p[3];
                ray_endpoints(g, view, u, v, s, p);
                int ns = ray_segments(g, s, p, idx, len, tbuf);
                for (int q = 0; q < ns; ++q) {
                    double w = power == 2 ? len[q] * len[q] : len[q];
                    mine[idx[q]] += w * e;
                }
            }
        }
        free(idx); free(len); free(tbuf);
    }
    if (!failed) {
        for (int64_t j = 0; j < nvox; ++j) {
            double acc = 0.0;
            for (int t = 0; t < nt; ++t) acc += buf[(size_t)t * (size_t)nvox + (size_t)j];
            vol[j] = acc;
        }
    }
    free(buf);
    return failed ? 2 : 0;
}

/* Number of ray-voxel pairs with positive length (nnz of A). */
int oref_count_nnz(const oref_geom *g, int64_t *out, int nthreads) {
    if (!valid(g) || !out) return 1;
    int64_t nrays = (int64_t)g->nviews * g->nv * g->nu;
    int cap = cap_of(g);
    int64_t total = 0;
    int failed = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : total)
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
        double *tbuf = (double *)malloc(sizeof(double) * (size_t)cap);
        if (!idx || !len || !tbuf) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < nrays; ++r) {
                int u = (int)(r % g->nu);
                int v = (int)((r / g->nu) % g->nv);
                int view = (int)(r / ((int64_t)g->nu * g->nv));
                double s[3], p[3];
                ray_endpoints(g, view, u, v, s, p);
                total += ray_segments(g, s, p, idx, len, tbuf);
            }
        }
        free(idx); free(len); free(tbuf);
    }
    *out = total;
    return failed ? 2 : 0;
}
