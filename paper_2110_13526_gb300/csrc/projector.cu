// Ray-driven Siddon projector pair for sm_103a: A (gather) and its exact
// transpose A^T (atomic scatter), plus an nnz counter.
//
// The operator (Materials and Methods, Eq. 1; Software section: Siddon
// ray-caster): A_ij = length in mm of ray i inside voxel j.
//
// Traversal ("slab walk").  Every ray picks its dominant axis s (largest
// |direction| in voxel units) and is walked one voxel slab of that axis at a
// time.  In voxel units the lateral coordinates along the ray are affine in
// the slab coordinate sigma, xi(sigma) = xi0 + A sigma and zeta(sigma) =
// ze0 + C sigma with |A|, |C| <= 1, so inside one slab the ray crosses at
// most one plane of each lateral axis: at most three voxels per slab.  The
// crossing order inside a slab decides the middle voxel.  Summing (segment
// length in slabs) * value and multiplying by the ray's mm-per-slab factor
// gives the Siddon line integral.
//
// Precision.  Both lateral lines of a ray are exact integer lines in Q.32
// fixed point, X(k) = X0 +- k dX, rounded once from FP64 (a per-column table
// computed on the host, since a ray's in-plane direction depends on its
// detector column only, and an exact integer sum per row; an FP64 setup for
// the rays that advance mostly along z).  A slab crosses a plane iff the
// distance to it, phi mod 2^32, is below dX, at the fraction phi / dX of the
// slab; integer steps do not drift, so a crossing is off by at most 2^-33
// voxel per slab walked plus 2^-23 of a slab, wherever it lies in the volume.
//
// Coherence.  The slab loop is warp-synchronous (the loop index is the same
// physical slab for all lanes), and a warp's 32 rays are neighbours on the
// detector, so at every step its lanes touch neighbouring voxels along one
// axis, laid out contiguously.  Two mappings:
//  * column-major (the default): the lanes are 32 consecutive rows of one
//    detector column; they share the in-plane walk and differ in z, and read
//    a copy of the volume laid out [y][x][z] (z fastest).  See the column-
//    major section below.
//  * ray-major (geometries with rays that advance mostly along z, the nnz
//    counter and the allocation-free projection): the lanes are 32 adjacent
//    columns of one row and differ along the lateral axis that varies with
//    u: x for rays advancing along y or z (the caller's layout [z][y][x])
//    and y for rays advancing along x, which read a copy laid out [z][x][y]
//    (the allocation-free projection reads [z][y][x] in place, strided).
// Otherwise the warp's gathers (and the reductions) fall on 1-2 lines.
#include <algorithm>
#include <atomic>
#include <climits>
#include <type_traits>

#include "ct_debug.cuh"
#include "ct_internal.h"
#include "ct_types.cuh"

namespace ct {
namespace {

constexpr int kTU = 32;  // ray-major tile: detector columns per CTA (one warp row)
constexpr int kTV = 8;   // detector rows per CTA
constexpr int kCU = 8;   // column-major tile: detector columns per CTA (one per warp)
constexpr int kCV = 32;  // detector rows per CTA (one per lane)
// Resident CTAs per SM the column-major forward kernels are compiled for
// (32 registers a thread).  The gather waits on L1/L2 hits, so warps in
// flight pay more than the registers they give up: measured on the 256^3
// workload, 5 CTAs/SM (48 registers) 11.1 ms, 6 (40) 10.2 ms, 7 (32) 10.0 ms.
// The backprojection is bound by instruction issue and keeps 5 (48).
constexpr int kFwdCtas = 7;
// Launch order (set_launch_order): views visited together by A and by A^T
// (ray-major A^T: kWideGroupBack) when the volume and its transposed copy take
// more than kL2GroupBytes.
constexpr int64_t kL2GroupBytes = int64_t(160) << 20;
constexpr int kWideGroupFwd = 65535;
// set_row_pairing: detector rows per voxel in z below which A^T pairs rows.
constexpr double kPairRowVox = 0.75;
constexpr int kWideGroupBack = 16;

// Slab coordinate at which the Q.32 line X(k) = X0 + k s reaches the integer
// plane P (s: signed slope per slab, in units of 2^-32).
__device__ __forceinline__ float plane_k(int P, long long X0, float s) {
    return __ll2float_rn(((long long)P << 32) - X0) / s;
}

// 1 + q 2^-32 truncated to a float in [1, 2): the exponent bits of 1.0f
// (0x7f << 23) funnel-shifted in above the top 23 bits of q.
__device__ __forceinline__ float one_plus_frac(unsigned q) {
    return __uint_as_float(__funnelshift_r(q, 0x7fu, 9));
}

// ---- ray-major kernels: one ray per lane, exact integer lines ---------------
// Each lane walks its own ray slab by slab along the axis it advances along
// fastest, with two lateral lines in Q.32 fixed point, X(k) = X0 +- k dX
// (the same exact integer lines as the column-major walk below): for a ray
// advancing along x or y, the in-plane lateral axis (the column's line from
// the host table) and z (the row's line, an exact integer sum); for a ray
// advancing along z, x and y, rounded to Q.44 from an FP64 setup of the ray.
// A slab holds at most three segments.  Offsets index the kernel's copy of
// the volume: [z][y][x] for rays advancing along y or z, [z][x][y] (except
// in ray_setup<true>: [z][y][x]) for rays advancing along x, so adjacent
// lanes touch adjacent words along their in-plane lateral axis.
struct Ray {
    long long X0 = 0, Y0 = 0;        // lines a and b at the start of slab 0 (Q.32)
    unsigned dX = 0u, dY = 0u;       // |slope| per slab (Q.32)
    bool x_up = false, y_up = false; // lines increasing along the walk
    float kx = 0.f, ky = 0.f;        // slabs per unit of each line (1 / slope)
    int Na = 0, Nb = 0, ca = 0, cb = 0;  // lateral sizes and centres
    int Ns = 0, sstride = 0, astride = 0, bstride = 0;  // slab count, memory strides
    bool rev = false;                // walk runs towards decreasing slab index
    float ksrc = 0.f, kpix = 0.f;    // slab coordinate of the source and of the pixel
    int k_lo = INT_MAX, k_hi = -1;   // slabs that may hold a part of the ray
    int k_in0 = INT_MIN, k_in1 = INT_MAX;  // slabs wholly inside the volume
    float lsig = 0.f;                // mm of ray per slab
    bool transposed = false;         // offsets index the [z][x][y] copy
};

// Q.44 (value * 2^44) -> the Q.32 line at the start of slab 0, its step and
// direction; cs is the centre slab.
__device__ __forceinline__ void ray_line(long long a, long long xi, int cs, long long &X0,
                                         unsigned &dX, bool &up) {
    X0 = (xi - a * cs) >> 12;
    dX = (unsigned)min(((unsigned long long)llabs(a) + 2048ull) >> 12, 0xffffffffull);
    up = a > 0 && dX != 0u;
}

// Ray (u, v) of one view; returns false if it misses the volume box.  With
// DIRECT every ray's offsets index the caller's layout [z][y][x] (a ray
// advancing along x then steps by 1 per slab and by nx along its lateral
// line), for the kernel that reads the volume in place.
template <bool DIRECT = false>
__device__ __forceinline__ bool ray_setup(const ProjGeom &g, int view, int u, int v, Ray &r) {
    const longlong2 *q = reinterpret_cast<const longlong2 *>(g.col_q + ((size_t)view * g.nu + u));
    const longlong2 qa = __ldg(q), qc = __ldg(q + 1), qz = __ldg(q + 2);
    const float4 qw = __ldg(reinterpret_cast<const float4 *>(q + 3));
    const int fl = __float_as_int(qw.z);
    const long long vc2 = 2LL * v - (g.nv - 1);
    const long long c = qc.x + vc2 * qc.y;
    float hs, ha, hb, wsrc, wpix;
    int cs;
    if (!(fl & 4) && llabs(c) <= (1LL << 44)) {
        // advancing along x or y: line a = the column's lateral line, b = z
        if (fl & 1) {   // slabs along x, lateral y: [z][x][y] (DIRECT: [z][y][x])
            r.Ns = g.nx; r.Na = g.ny; hs = g.hx; ha = g.hy;
            r.sstride = DIRECT ? 1 : g.ny;
            r.astride = DIRECT ? g.nx : 1;
            r.transposed = !DIRECT;
        } else {        // slabs along y, lateral x: [z][y][x]
            r.Ns = g.ny; r.Na = g.nx; r.sstride = g.nx; hs = g.hy; ha = g.hx;
            r.astride = 1;
            r.transposed = false;
        }
        r.Nb = g.nz;
        r.bstride = g.nx * g.ny;
        hb = g.hz;
        r.rev = (fl & 2) != 0;
        cs = r.Ns / 2;
        ray_line(qa.x, qa.y, cs, r.X0, r.dX, r.x_up);
        ray_line(c, qz.x + vc2 * qz.y, cs, r.Y0, r.dY, r.y_up);
        wsrc = qw.x;
        wpix = qw.y;
    } else {
        // advancing along z: slabs along z, lines x (a) and y (b), [z][y][x]
        const ViewConst &vw = g.views[view];
        const double uc = (double)u - 0.5 * (double)(g.nu - 1);
        const double vc = (double)v - 0.5 * (double)(g.nv - 1);
        double S[3], D[3];
        for (int a = 0; a < 3; ++a) {
            S[a] = vw.s[a];
            D[a] = fma(vc, vw.ev[a], fma(uc, vw.eu[a], vw.p00[a])) - S[a];
        }
        if (!(D[2] != 0.0)) return false;
        r.Ns = g.nz; r.Na = g.nx; r.Nb = g.ny;
        r.sstride = g.nx * g.ny; r.astride = 1; r.bstride = g.nx;
        hs = g.hz; ha = g.hx; hb = g.hy;
        r.transposed = false;
        r.rev = D[2] < 0.0;
        cs = r.Ns / 2;
        const double sig0 = r.rev ? (double)(r.Ns - cs) : (double)cs;
        const double adz = fabs(D[2]), t = (sig0 - S[2]) / D[2];
        const double lim = 65536.0;   // a ray this far out misses the volume
        const double xi = fmin(fmax(S[0] - (double)(g.nx / 2) + t * D[0], -lim), lim);
        const double yi = fmin(fmax(S[1] - (double)(g.ny / 2) + t * D[1], -lim), lim);
        ray_line(__double2ll_rn(ldexp(D[0] / adz, 44)), __double2ll_rn(ldexp(xi, 44)), cs, r.X0,
                 r.dX, r.x_up);
        ray_line(__double2ll_rn(ldexp(D[1] / adz, 44)), __double2ll_rn(ldexp(yi, 44)), cs, r.Y0,
                 r.dY, r.y_up);
        wsrc = (float)((r.rev ? (double)r.Ns - S[2] : S[2]) - (double)cs);
        wpix = (float)((r.rev ? (double)r.Ns - (S[2] + D[2]) : S[2] + D[2]) - (double)cs);
    }
    r.ca = r.Na / 2;
    r.cb = r.Nb / 2;
    const float af = (float)r.dX * 0x1p-32f, bf = (float)r.dY * 0x1p-32f;
    r.kx = 1.f / af;
    r.ky = 1.f / bf;
    r.ksrc = wsrc + (float)cs;
    r.kpix = wpix + (float)cs;
    // slab ranges from the integer lines, as in cm_setup below
    float e = fmaxf(0.f, r.ksrc), x = fminf((float)r.Ns, r.kpix);
    bool ok = true;
    if (r.dX != 0u) {
        const float s = r.x_up ? (float)r.dX : -(float)r.dX;
        const float t0 = plane_k(-r.ca, r.X0, s), t1 = plane_k(r.Na - r.ca, r.X0, s);
        e = fmaxf(e, fminf(t0, t1));
        x = fminf(x, fmaxf(t0, t1));
    } else {
        ok = r.X0 >= ((long long)(-r.ca) << 32) && r.X0 < ((long long)(r.Na - r.ca) << 32);
    }
    if (r.dY != 0u) {
        const float s = r.y_up ? (float)r.dY : -(float)r.dY;
        const float t0 = plane_k(-r.cb, r.Y0, s), t1 = plane_k(r.Nb - r.cb, r.Y0, s);
        e = fmaxf(e, fminf(t0, t1));
        x = fminf(x, fmaxf(t0, t1));
    } else {
        ok = ok && r.Y0 >= ((long long)(-r.cb) << 32) && r.Y0 < ((long long)(r.Nb - r.cb) << 32);
    }
    ok = ok && e < x;
    e = fminf(fmaxf(e, -2.f), (float)r.Ns + 2.f);
    x = fminf(fmaxf(x, -2.f), (float)r.Ns + 2.f);
    const float de = fmaf(fabsf(e), 0x1p-16f, 0x1p-16f), dx = fmaf(fabsf(x), 0x1p-16f, 0x1p-16f);
    r.k_lo = max(0, (int)floorf(e - de));
    r.k_hi = min(r.Ns - 1, (int)floorf(x + dx));
    r.k_in0 = (int)ceilf(e + de);
    r.k_in1 = (int)floorf(x - dx) - 1;
    ok = ok && r.k_lo <= r.k_hi;
    const float la = af * (ha / hs), lb = bf * (hb / hs);
    r.lsig = hs * sqrtf(fmaf(la, la, fmaf(lb, lb, 1.f)));
    return ok;
}

// Warp-synchronous slab walk; fn(offset, length in slabs, p) is called for
// the segments of each slab and may touch memory only where p is set (the
// offset is then inside the volume).  Must be called by all 32 lanes of the
// warp.  Every lane walks its own lines; the loop runs over the slabs any
// lane's ray may touch.  In the interior (slabs wholly inside the volume and
// the source..pixel part for every ray of the warp) a slab holds the lane's
// current voxel, the next one along whichever line crosses first and, where
// both cross, the diagonal one, all in range; the other slabs check each
// segment's indices and clip to the source..pixel part.  A lane without a
// ray (ok false) keeps offset 0 with zero steps and sets no p.
template <class Fn>
__device__ __forceinline__ void walk(const Ray &r, bool ok, Fn &&fn) {
    const unsigned full = 0xffffffffu;
    const int kb = __reduce_min_sync(full, ok ? r.k_lo : INT_MAX);
    const int ke = __reduce_max_sync(full, ok ? r.k_hi : -1);
    if (kb > ke) return;
    const int k_mid0 = max(kb, __reduce_max_sync(full, ok ? r.k_in0 : INT_MIN));
    const int k_mid1 = min(ke, __reduce_min_sync(full, ok ? r.k_in1 : INT_MAX));
    const long long X = r.X0 + (r.x_up ? (long long)kb * r.dX : -(long long)kb * r.dX);
    const long long Y = r.Y0 + (r.y_up ? (long long)kb * r.dY : -(long long)kb * r.dY);
    int ai = (int)((r.x_up ? X - 1 : X) >> 32) + r.ca;   // lateral indices (may lie outside)
    int bi = (int)((r.y_up ? Y - 1 : Y) >> 32) + r.cb;
    unsigned phi = r.x_up ? (unsigned)(-X) : (unsigned)X;
    unsigned psi = r.y_up ? (unsigned)(-Y) : (unsigned)Y;
    const unsigned dX = ok ? r.dX : 0u, dY = ok ? r.dY : 0u;
    const float kx = r.kx, ky = r.ky;
    const int Na = r.Na, Nb = r.Nb;
    const unsigned sstep = !ok ? 0u : r.rev ? 0u - (unsigned)r.sstride : (unsigned)r.sstride;
    const unsigned astep = !ok ? 0u : r.x_up ? (unsigned)r.astride : 0u - (unsigned)r.astride;
    const unsigned bstep = !ok ? 0u : r.y_up ? (unsigned)r.bstride : 0u - (unsigned)r.bstride;
    const int da = r.x_up ? 1 : -1, db = r.y_up ? 1 : -1;
    unsigned o = !ok ? 0u
                     : (r.rev ? (unsigned)(r.Ns - 1) * (unsigned)r.sstride : 0u) +
                           (unsigned)kb * sstep + (unsigned)ai * (unsigned)r.astride +
                           (unsigned)bi * (unsigned)r.bstride;
    const float ksrc = ok ? r.ksrc : 0.f, kpix = ok ? r.kpix : 0.f;
    // the lanes of a warp may walk different axes: the loop runs over the
    // union of their slabs, and a lane's own slab index must be checked too
    const unsigned Nsl = ok ? (unsigned)r.Ns : 0u;
    auto clamped = [&](int k) {
        const bool cx = phi < dX, cy = psi < dY;
        const float sx = cx ? fmaf(one_plus_frac(phi), kx, -kx) : 1.f;
        const float sy = cy ? fmaf(one_plus_frac(psi), ky, -ky) : 1.f;
        const float s1 = fminf(sx, sy), s2 = fmaxf(sx, sy);
        const float kf = (float)k;
        const float c_lo = fminf(fmaxf(ksrc - kf, 0.f), 1.f);
        const float c_hi = fminf(fmaxf(kpix - kf, 0.f), 1.f);
        const float b1 = fminf(fmaxf(s1, c_lo), c_hi), b2 = fminf(fmaxf(s2, c_lo), c_hi);
        const float l1 = b1 - c_lo, l2 = b2 - b1, l3 = c_hi - b2;
        const bool sk = (unsigned)k < Nsl;
        const bool a0 = sk && (unsigned)ai < (unsigned)Na;
        const bool a1 = sk && (unsigned)(ai + da) < (unsigned)Na;
        const bool z0 = (unsigned)bi < (unsigned)Nb, z1 = (unsigned)(bi + db) < (unsigned)Nb;
        const bool mx = sx <= sy;   // the middle segment is past the crossing of line a
        fn((int)o, l1, a0 && z0 && l1 > 0.f);
        fn((int)(o + (mx ? astep : bstep)), l2, (mx ? (a1 && z0) : (a0 && z1)) && l2 > 0.f);
        fn((int)(o + (cx ? astep : 0u) + (cy ? bstep : 0u)), l3,
           (cx ? a1 : a0) && (cy ? z1 : z0) && l3 > 0.f);
        phi -= dX;
        psi -= dY;
        if (cx) {
            ai += da;
            o += astep;
        }
        if (cy) {
            bi += db;
            o += bstep;
        }
        o += sstep;
    };
    // In the interior every offset handed to fn with p set is in range.
    auto interior = [&]() {
        const bool cx = phi < dX, cy = psi < dY;
        const float sx = cx ? fmaf(one_plus_frac(phi), kx, -kx) : 1.f;
        const float sy = cy ? fmaf(one_plus_frac(psi), ky, -ky) : 1.f;
        const float s1 = fminf(sx, sy), s2 = fmaxf(sx, sy);
        const unsigned ax = cx ? astep : 0u, by = cy ? bstep : 0u;
        fn((int)o, s1, ok);
        fn((int)(o + (sx <= sy ? astep : bstep)), s2 - s1, cx || cy);
        fn((int)(o + ax + by), 1.f - s2, cx && cy);
        phi -= dX;
        psi -= dY;
        o += sstep + ax + by;
    };
    int k = kb;
    const int k_entry_end = min(k_mid0, ke + 1);
    for (; k < k_entry_end; ++k) clamped(k);
    if (k <= k_mid1) {
#pragma unroll 2
        for (; k <= k_mid1; ++k) interior();
        // the lateral indices, tracked only by the clamped slabs, from the offset
        if (k <= ke && ok) {
            const unsigned rem = o - (r.rev ? (unsigned)(r.Ns - 1) * (unsigned)r.sstride : 0u) -
                                 (unsigned)k * sstep;
            bi = (int)(rem / (unsigned)r.bstride);
            ai = (int)((rem - (unsigned)bi * (unsigned)r.bstride) / (unsigned)r.astride);
        }
    }
    for (; k <= ke; ++k) clamped(k);
}

// Predicated float reduction into global memory (no branch around it): the
// lanes of a warp reach it together whether or not they have a segment.
__device__ __forceinline__ void red_add_if(float *addr, float val, bool pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t@p red.global.add.f32 [%0], %1;\n\t}"
        :
        : "l"(addr), "f"(val), "r"((int)pred));
}

// Predicated 64-bit integer reduction into global memory.
__device__ __forceinline__ void red_add_u64_if(unsigned long long *addr, long long val, bool pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t@p red.global.add.u64 [%0], %1;\n\t}"
        :
        : "l"(addr), "l"(val), "r"((int)pred));
}

__device__ __forceinline__ double block_sum_d(double x, double *sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread (0, 0)
}

// The rays of this thread.  CTA (bx, by, bz) covers columns 32 bx .. 32 bx + 31
// and rows 8 vb .. 8 vb + 7 of view grp * vgroup + by, where bz = grp * nvb + vb
// (proj_grid).  The last group may run past the last view (view >= nviews).
__device__ __forceinline__ void tile_of(const ProjGeom &g, int &u, int &v, int &view) {
    const int grp = (int)blockIdx.z / g.nvb;
    const int vb = (int)blockIdx.z - grp * g.nvb;
    u = blockIdx.x * kTU + threadIdx.x;
    v = vb * kTV + threadIdx.y;
    view = grp * g.vgroup + (int)blockIdx.y;
}

__device__ __forceinline__ void coef_of(const Coef &c, float &alpha, float &beta) {
    if (c.dev) {
        alpha = (float)c.dev[0];
        beta = (float)c.dev[1];
    } else {
        alpha = c.alpha;
        beta = c.beta;
    }
}

// p = alpha * rho o (A vol) + beta * p.  vol == NULL means the all-ones volume.
template <bool HAS_RHO, bool NORM, bool UNIT_VOL, class TV = float, class TS = float>
__global__ void __launch_bounds__(kTU *kTV, 6) k_forward(ProjGeom g, const TV *__restrict__ vol,
                                                      const TV *__restrict__ vol_t,
                                                      TS *__restrict__ out,
                                                      const float *__restrict__ rho, Coef c,
                                                      double *__restrict__ partials) {
    __shared__ double sh[32];
    int u, v, view;
    tile_of(g, u, v, view);
    const bool inb = (u < g.nu) && (v < g.nv) && (view < g.nviews);
    Ray r;
    const bool valid = inb && ray_setup(g, view, u, v, r);
    const TV *base = r.transposed ? vol_t : vol;
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
    float acc = 0.f;
    walk(r, valid, [&](int o, float l, bool p) {
        float val = 0.f;
        if (p && CT_IN_BOUNDS(o, nvox)) val = UNIT_VOL ? 1.f : ld_f(base + o);
        acc = fmaf(l, val, acc);
    });
    float alpha, beta;
    coef_of(c, alpha, beta);
    double sq = 0.0;
    const size_t idx = ((size_t)view * g.nv + v) * g.nu + u;
    if (inb && CT_IN_BOUNDS(idx, (int64_t)g.nviews * g.nv * g.nu)) {
        float val = valid ? acc * r.lsig : 0.f;
        if (HAS_RHO) val *= rho[idx];
        float o = alpha * val;
        if (beta != 0.f) o = fmaf(beta, to_f(out[idx]), o);
        const TS st = from_f<TS>(o);
        out[idx] = st;
        if (NORM) {
            const double q = (double)to_f(st);  // the norm of what is stored
            sq = q * q;
        }
    }
    if (NORM) {
        double t = block_sum_d(sq, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
    }
}

// acc += alpha * (A o A ... )^T: POWER 1 scatters length * w, POWER 2 scatters
// length^2 * w, w = alpha * rho_i * e_i (e == NULL means e = 1).  DET
// accumulates q = rint(value * scale) in 64-bit integers (scale = a power of
// two read from det_scale[0]): integer addition is associative, so the sums
// do not depend on the order in which rays arrive.
template <bool HAS_RHO, int POWER, bool DET, class TS = float>
__global__ void __launch_bounds__(kTU *kTV, 6) k_backward(ProjGeom g, const TS *__restrict__ e,
                                                       const float *__restrict__ rho, Coef c,
                                                       void *__restrict__ acc,
                                                       void *__restrict__ acc_t,
                                                       const float *__restrict__ det_scale) {
    int u, v, view;
    tile_of(g, u, v, view);
    const bool inb = (u < g.nu) && (v < g.nv) && (view < g.nviews);
    Ray r;
    bool valid = inb && ray_setup(g, view, u, v, r);
    float alpha, beta;
    coef_of(c, alpha, beta);
    float w = 0.f;
    const size_t idx = ((size_t)view * g.nv + v) * g.nu + u;
    if (valid && CT_IN_BOUNDS(idx, (int64_t)g.nviews * g.nv * g.nu)) {
        w = alpha * (e ? to_f(e[idx]) : 1.f);
        if (HAS_RHO) w *= rho[idx];
        if (POWER == 1) w *= r.lsig;
    }
    valid = valid && (w != 0.f);
    const float ls = r.lsig;
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
    if constexpr (DET) {
        const float scale = __ldg(det_scale);
        unsigned long long *base =
            static_cast<unsigned long long *>(r.transposed ? acc_t : acc);
        walk(r, valid, [&](int o, float l, bool p) {
            const float lm = l * ls;
            const float val = POWER == 1 ? w * l : w * lm * lm;
            red_add_u64_if(base + o, __float2ll_rn(val * scale), p && CT_IN_BOUNDS(o, nvox));
        });
    } else {
        float *base = static_cast<float *>(r.transposed ? acc_t : acc);
        walk(r, valid, [&](int o, float l, bool p) {
            const float lm = l * ls;
            red_add_if(base + o, POWER == 1 ? w * l : w * lm * lm, p && CT_IN_BOUNDS(o, nvox));
        });
    }
}

__global__ void __launch_bounds__(kTU *kTV) k_count(ProjGeom g,
                                                    unsigned long long *__restrict__ count) {
    __shared__ double sh[32];
    int u, v, view;
    tile_of(g, u, v, view);
    const bool inb = (u < g.nu) && (v < g.nv) && (view < g.nviews);
    Ray r;
    const bool valid = inb && ray_setup(g, view, u, v, r);
    int n = 0;
    walk(r, valid, [&](int, float l, bool p) { n += (p && l > 0.f) ? 1 : 0; });
    double t = block_sum_d((double)n, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(count, (unsigned long long)(t + 0.5));
}

// Variant of k_forward with the FP64 norm partials that reads only the
// caller's volume in its own layout [nz][ny][nx]: every ray walks offsets of
// that layout.  The lanes of a warp holding rays that advance along x
// gather with a stride of nx (adjacent lanes are adjacent in y), so this is
// slower, but it needs no transposed copy.
__global__ void __launch_bounds__(kTU *kTV) k_forward_direct(ProjGeom g,
                                                             const float *__restrict__ vol,
                                                             float *__restrict__ out, float alpha,
                                                             float beta,
                                                             double *__restrict__ partials) {
    __shared__ double sh[32];
    int u, v, view;
    tile_of(g, u, v, view);
    const bool inb = (u < g.nu) && (v < g.nv) && (view < g.nviews);
    Ray r;
    const bool valid = inb && ray_setup<true>(g, view, u, v, r);
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
    float acc = 0.f;
    walk(r, valid, [&](int o, float l, bool p) {
        if (p && l > 0.f && CT_IN_BOUNDS(o, nvox)) acc = fmaf(l, __ldg(vol + o), acc);
    });
    double sq = 0.0;
    const size_t idx = ((size_t)view * g.nv + v) * g.nu + u;
    if (inb && CT_IN_BOUNDS(idx, (int64_t)g.nviews * g.nv * g.nu)) {
        const float val = valid ? acc * r.lsig : 0.f;
        float o = alpha * val;
        if (beta != 0.f) o = fmaf(beta, out[idx], o);
        out[idx] = o;
        sq = (double)o * (double)o;
    }
    const double t = block_sum_d(sq, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partials[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
}

// ---- column-major kernels ---------------------------------------------------
// The rays of one detector column share their projection onto the xy plane:
// slab axis, direction, lateral slope A and lateral plane crossings depend on
// the column only; the detector row changes only the z part (C, ze0).  In the
// column-major kernels the 32 lanes of a warp are 32 consecutive rows v of
// one column u, so the in-plane walk (slab bounds, lateral crossings) is the
// same in every lane and its branch is warp-uniform; only the z crossing is
// per lane.  The volume is read from (and A^T accumulates into) a copy laid
// out [y][x][z], z fastest, in which the lanes of a warp, about one z row
// apart, touch consecutive words whichever axis the column advances along.
// A slab costs two gathers per lane (the second only where the lane crosses
// a z plane) plus one where the column crosses a lateral plane, with no vote
// and no per-lane lateral state.  Rays advancing mostly along z (|C| > 1) do
// not fit this scheme; geometries that have any use the ray-major kernels
// above instead (ProjGeom::cm).
//
// Fixed-point walk.  A column's lateral line and a row's z line (ColFixed,
// Q.44 values of the host's FP64 parameters) become integer lines in Q.32,
// anchored at the start of the volume's first slab along the walk:
//   X(k) = X(0) +- k dX,   dX = round(|A| 2^32)   (k: slab index of the walk)
// and likewise Z(k) with dZ = round(|C| 2^32).  The integer part of X is the
// lateral voxel index (centred), the fraction the position inside it.  The
// walk keeps phi = the distance from X(k) to the next plane in the direction
// of travel, mod 2^32, and subtracts dX once per slab: the slab crosses that
// plane iff phi < dX (the borrow is the crossing), at the fraction phi / dX
// of the slab, and the wrap-around leaves phi at the distance to the plane
// after.  Integer steps are exact, so no rounding accumulates along the ray:
// a crossing is off by at most 2^-33 voxel per slab walked (the rounding of
// dX) plus the 2^-23 of the fraction's conversion to float, both in units of
// a voxel relative to the slab.  (Crossings computed in FP32 relative to the
// volume centre carry 2^-24 |w| instead: 1.5e-5 voxel at 256 voxels from the
// centre, which a backprojected voxel, a sum of segments of unrelated rays,
// does not average away.)  Segment lengths are therefore fractions of one
// slab in [0, 1], multiplied by the mm-per-slab factor lsig of the ray.
// A line exactly in a grid plane with zero slope (dX = 0) is credited to the
// voxel above it, as the midpoint rule does.

// Tile (bx, by, bz) of the projector grid (blockIdx in a plain launch; a
// batched launch maps its work items onto each job's grid).
__device__ __forceinline__ void tile_of_cm(const ProjGeom &g, uint3 bid, int &u, int &v,
                                           int &view) {
    const int grp = (int)bid.z / g.nvb;
    const int vb = (int)bid.z - grp * g.nvb;
    u = bid.x * kCU + threadIdx.y;
    v = vb * kCV + threadIdx.x;
    view = grp * g.vgroup + (int)bid.y;
}

// One warp's column (the same in all lanes) and one lane's row of it.
struct CmRay {
    long long X0 = 0, Z0 = 0;        // lateral and z lines at slab 0, Q.32, centred
    unsigned dX = 0, dZ = 0;         // |slope| per slab, Q0.32
    bool x_up = false, z_up = false; // the line runs towards higher indices
    float kx = 0.f, kz = 0.f;        // 1 / |A|, 1 / |C| (slabs per unit of the axis)
    int Ns = 0, Na = 0, Nb = 0, ca = 0, cb = 0;
    int sstride = 0, astride = 0;    // [y][x][z] strides of the slab and lateral axes
    bool rev = false;                // walk runs towards decreasing slab index
    float ksrc = 0.f, kpix = 0.f;    // slab coordinate of the source and of the pixel
    int k_lo = INT_MAX, k_hi = -1;   // slabs that may hold a part of the ray
    int k_in0 = INT_MIN, k_in1 = INT_MAX;  // slabs wholly inside the volume
    float lsig = 0.f;                // mm of ray per slab
};

// A load the compiler may not merge with an earlier load of the same address
// (so that values re-derived from it need no register in between).
__device__ __forceinline__ float4 ld_volatile_f4(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Set up ray (u, v) of a column-major warp; returns whether it crosses the
// volume.  col_live (u and view in range) must be warp-uniform.
//
// The slab range comes from the same integer lines the walk steps along: the
// face crossings are computed in FP32 from exact integer distances (relative
// error below 2^-22), and widened by a margin of 2^-16 (|k| + 1) slab, so
// that [k_lo, k_hi] holds every slab with a part of the ray inside and
// [k_in0, k_in1] only slabs whose every segment lies inside (their voxel
// indices need no check).
__device__ __forceinline__ bool cm_setup(const ProjGeom &g, int view, int u, int v, bool col_live,
                                         CmRay &r) {
    if (!col_live) return false;
    const longlong2 *q = reinterpret_cast<const longlong2 *>(g.col_q + ((size_t)view * g.nu + u));
    const longlong2 qa = __ldg(q), qc = __ldg(q + 1), qz = __ldg(q + 2);
    const float4 qw = __ldg(reinterpret_cast<const float4 *>(q + 3));
    const int fl = __float_as_int(qw.z);
    float hs, ha;
    if (fl & 1) {      // slabs along x, lateral y
        r.Ns = g.nx; r.Na = g.ny; r.sstride = g.nz; r.astride = g.nx * g.nz; hs = g.hx; ha = g.hy;
    } else {           // slabs along y, lateral x
        r.Ns = g.ny; r.Na = g.nx; r.sstride = g.nx * g.nz; r.astride = g.nz; hs = g.hy; ha = g.hx;
    }
    r.Nb = g.nz;
    r.rev = (fl & 2) != 0;
    const int cs = r.Ns / 2;
    r.ca = r.Na / 2;
    r.cb = r.Nb / 2;
    const long long vc2 = 2LL * v - (g.nv - 1);
    const long long a = qa.x, xi = qa.y;
    const long long c = qc.x + vc2 * qc.y, z = qz.x + vc2 * qz.y;
    r.dX = (unsigned)min(((unsigned long long)llabs(a) + 2048ull) >> 12, 0xffffffffull);
    r.dZ = (unsigned)min(((unsigned long long)llabs(c) + 2048ull) >> 12, 0xffffffffull);
    r.x_up = a > 0 && r.dX != 0u;
    r.z_up = c > 0 && r.dZ != 0u;
    r.X0 = (xi - a * cs) >> 12;   // Q.44 -> Q.32 (floor)
    r.Z0 = (z - c * cs) >> 12;
    const float af = (float)r.dX * 0x1p-32f, cf = (float)r.dZ * 0x1p-32f;
    r.kx = 1.f / af;
    r.kz = 1.f / cf;
    r.ksrc = qw.x + (float)cs;
    r.kpix = qw.y + (float)cs;
    float e = fmaxf(0.f, r.ksrc), x = fminf((float)r.Ns, r.kpix);
    bool ok = v < g.nv;
    if (r.dX != 0u) {
        const float s = r.x_up ? (float)r.dX : -(float)r.dX;
        const float t0 = plane_k(-r.ca, r.X0, s), t1 = plane_k(r.Na - r.ca, r.X0, s);
        e = fmaxf(e, fminf(t0, t1));
        x = fminf(x, fmaxf(t0, t1));
    } else {
        ok = ok && r.X0 >= ((long long)(-r.ca) << 32) && r.X0 < ((long long)(r.Na - r.ca) << 32);
    }
    if (r.dZ != 0u) {
        const float s = r.z_up ? (float)r.dZ : -(float)r.dZ;
        const float t0 = plane_k(-r.cb, r.Z0, s), t1 = plane_k(r.Nb - r.cb, r.Z0, s);
        e = fmaxf(e, fminf(t0, t1));
        x = fminf(x, fmaxf(t0, t1));
    } else {
        ok = ok && r.Z0 >= ((long long)(-r.cb) << 32) && r.Z0 < ((long long)(r.Nb - r.cb) << 32);
    }
    ok = ok && e < x;
    e = fminf(fmaxf(e, -2.f), (float)r.Ns + 2.f);
    x = fminf(fmaxf(x, -2.f), (float)r.Ns + 2.f);
    const float de = fmaf(fabsf(e), 0x1p-16f, 0x1p-16f), dx = fmaf(fabsf(x), 0x1p-16f, 0x1p-16f);
    r.k_lo = max(0, (int)floorf(e - de));
    r.k_hi = min(r.Ns - 1, (int)floorf(x + dx));
    r.k_in0 = (int)ceilf(e + de);
    r.k_in1 = (int)floorf(x - dx) - 1;
    ok = ok && r.k_lo <= r.k_hi;
    const float la = af * (ha / hs), lb = cf * (g.hz / hs);
    r.lsig = hs * sqrtf(fmaf(la, la, fmaf(lb, lb, 1.f)));
    return ok;
}

// Column-major slab walk; fn(offset, length in slabs, p) is called for the
// segments of each slab (with WS the lengths times ws, a per-lane weight),
// and may touch memory only where p is set (the offset is then inside the
// volume).  Must be called by all 32 lanes of the
// warp, which hold rows of one column; ci = view * nu + u is the column.
//
// The warp walks the slabs any of its rays may touch.  Slabs that lie wholly
// inside the volume for every ray of the warp (the interior, nearly all of a
// ray) need no index checks: a slab holds the lane's current voxel, the next
// one along z where the lane crosses a z plane, and, where the column crosses
// a lateral plane, one more.  In the other slabs each segment is checked
// against the volume's index ranges and clipped to the source..pixel part of
// the ray.  A lane without a ray (ok false) keeps offset 0 with zero steps,
// so it may touch voxel 0 but nothing else; its segments must be discarded
// by fn (a zero weight, or a sum that is dropped).  Offsets are unsigned:
// outside the volume they may wrap, and they are exact again whenever the
// indices are in range.
//
// Everything the exit slabs need beyond the loop state is re-derived after
// the interior from the column's parameters, so that it holds no registers
// during the loop (the forward kernel runs at 32 registers a thread).
template <int DZ, bool WS, class Fn>
__device__ __forceinline__ void walk_cm_dir(const ProjGeom &g, int ci, const CmRay &r, bool ok,
                                            int kb, int ke, int k_mid0, int k_mid1, Fn &&fn,
                                            float ws) {
    // state of both lines at the start of slab kb
    const long long X = r.X0 + (r.x_up ? (long long)kb * r.dX : -(long long)kb * r.dX);
    const long long Z = r.Z0 + (r.z_up ? (long long)kb * r.dZ : -(long long)kb * r.dZ);
    int ai = (int)((r.x_up ? X - 1 : X) >> 32) + r.ca;   // voxel indices (may lie outside)
    int zi = (int)((r.z_up ? Z - 1 : Z) >> 32) + r.cb;
    unsigned phi = r.x_up ? (unsigned)(-X) : (unsigned)X;
    unsigned psi = r.z_up ? (unsigned)(-Z) : (unsigned)Z;
    // a lane without a ray never crosses a z plane (dZ = 0), so with a
    // compile-time direction DZ its z neighbour is never touched either
    const unsigned dX = r.dX, dZ = ok ? r.dZ : 0u;
    const float kx = r.kx, kz = r.kz;
    const unsigned sstep = !ok ? 0u : r.rev ? 0u - (unsigned)r.sstride : (unsigned)r.sstride;
    const unsigned astep = !ok ? 0u : r.x_up ? (unsigned)r.astride : 0u - (unsigned)r.astride;
    const unsigned dzu = DZ != 0 ? (unsigned)DZ : !ok ? 0u : r.z_up ? 1u : 0xffffffffu;
    unsigned o = !ok ? 0u
                     : (r.rev ? (unsigned)(r.Ns - 1) * (unsigned)r.sstride : 0u) +
                           (unsigned)kb * sstep + (unsigned)ai * (unsigned)r.astride +
                           (unsigned)zi;
    // column constants of the entry and exit slabs (re-derived for the exit)
    int Na = r.Na, astride = r.astride;
    unsigned obase = r.rev ? (unsigned)(r.Ns - 1) * (unsigned)r.sstride : 0u;
    float ksrc = r.ksrc, kpix = r.kpix;
    auto clamped = [&](int k) {
        const int da = (int)astep > 0 ? 1 : -1, dz = (int)dzu;
        const bool cx = phi < dX, cz = psi < dZ;
        const float sx = cx ? fmaf(one_plus_frac(phi), kx, -kx) : 1.f;
        const float sz = cz ? fmaf(one_plus_frac(psi), kz, -kz) : 1.f;
        const float s1 = fminf(sx, sz), s2 = fmaxf(sx, sz);
        const float kf = (float)k;
        const float c_lo = fminf(fmaxf(ksrc - kf, 0.f), 1.f);
        const float c_hi = fminf(fmaxf(kpix - kf, 0.f), 1.f);
        const float b1 = fminf(fmaxf(s1, c_lo), c_hi), b2 = fminf(fmaxf(s2, c_lo), c_hi);
        const float l1 = b1 - c_lo, l2 = b2 - b1, l3 = c_hi - b2;
        const bool a0 = (unsigned)ai < (unsigned)Na, a1 = (unsigned)(ai + da) < (unsigned)Na;
        const bool z0 = (unsigned)zi < (unsigned)g.nz, z1 = (unsigned)(zi + dz) < (unsigned)g.nz;
        const bool mx = sx <= sz;   // the middle segment is past the lateral crossing
        fn((int)o, WS ? ws * l1 : l1, a0 && z0 && l1 > 0.f);
        fn((int)(o + (mx ? astep : dzu)), WS ? ws * l2 : l2,
           (mx ? (a1 && z0) : (a0 && z1)) && l2 > 0.f);
        fn((int)(o + (cx ? astep : 0u) + (cz ? dzu : 0u)), WS ? ws * l3 : l3,
           (cx ? a1 : a0) && (cz ? z1 : z0) && l3 > 0.f);
        phi -= dX;
        psi -= dZ;
        if (cx) {
            ai += da;
            o += astep;
        }
        if (cz) {
            zi += dz;
            o += dzu;
        }
        o += sstep;
    };
    // In the interior every offset handed to fn is in range or unused, so
    // they are formed as int sums: the z neighbour (o + dz) is then a
    // constant displacement of o's address when DZ is fixed.
    const int dzi = DZ != 0 ? DZ : (int)dzu, ast = (int)astep;
    // With WS a two-segment slab hands fn ws sz and ws (1 - sz) straight
    // from the z step scaled by ws.
    const float kzw = WS ? ws * kz : kz;
    auto interior = [&]() {
        const bool cz = psi < dZ;
        if constexpr (WS) {
            const float fz = one_plus_frac(psi);
            psi -= dZ;
            const int oi = (int)o;
            if (phi >= dX) {   // no lateral crossing (warp-uniform)
                const float szw = cz ? fmaf(fz, kzw, -kzw) : ws;
                fn(oi, szw, true);
                fn(oi + dzi, ws - szw, cz);
            } else {
                const float sz = cz ? fmaf(fz, kz, -kz) : 1.f;
                const float sx = fmaf(one_plus_frac(phi), kx, -kx);
                const float s1 = fminf(sx, sz), s2 = fmaxf(sx, sz);
                fn(oi, ws * s1, true);
                fn(sx <= sz ? oi + ast : oi + dzi, ws * (s2 - s1), true);
                fn(oi + ast + (cz ? dzi : 0), ws * (1.f - s2), cz);
                o += astep;
            }
        } else {
            const float sz = cz ? fmaf(one_plus_frac(psi), kz, -kz) : 1.f;
            psi -= dZ;
            const int oi = (int)o;
            if (phi >= dX) {   // no lateral crossing (warp-uniform)
                fn(oi, sz, true);
                fn(oi + dzi, 1.f - sz, cz);
            } else {
                const float sx = fmaf(one_plus_frac(phi), kx, -kx);
                const float s1 = fminf(sx, sz), s2 = fmaxf(sx, sz);
                fn(oi, s1, true);
                fn(sx <= sz ? oi + ast : oi + dzi, s2 - s1, true);
                fn(oi + ast + (cz ? dzi : 0), 1.f - s2, cz);
                o += astep;
            }
        }
        phi -= dX;
        o += sstep + (cz ? dzu : 0u);
    };
    int k = kb;
    const int k_entry_end = min(k_mid0, ke + 1);
    for (; k < k_entry_end; ++k) clamped(k);
    if (k <= k_mid1) {
#pragma unroll 4
        for (; k <= k_mid1; ++k) interior();
        if (k > ke) return;
        // Re-derive the column constants from its parameters (a fresh load,
        // so they need not stay in registers through the loop), then the
        // indices from the offset: the interior tracks them only there, and
        // ends with them in range (meaningless in a lane without a ray).
        const float4 qw = ld_volatile_f4(reinterpret_cast<const float4 *>(g.col_q + ci) + 3);
        const int fl = __float_as_int(qw.z);
        const int Ns = (fl & 1) ? g.nx : g.ny, cs = Ns / 2;
        const int sstride = (fl & 1) ? g.nz : g.nx * g.nz;
        Na = (fl & 1) ? g.ny : g.nx;
        astride = (fl & 1) ? g.nx * g.nz : g.nz;
        obase = (fl & 2) ? (unsigned)(Ns - 1) * (unsigned)sstride : 0u;
        ksrc = qw.x + (float)cs;
        kpix = qw.y + (float)cs;
        const unsigned rem = o - obase - (unsigned)k * sstep;
        ai = (int)(rem / (unsigned)astride);
        zi = (int)(rem - (unsigned)ai * (unsigned)astride);
    }
    for (; k <= ke; ++k) clamped(k);
}

// The walk with the z direction fixed at compile time where all lanes of
// the warp that hold a ray move the same way along z (every warp but the one
// holding the column's horizontal row): the z neighbour of a voxel is then a
// constant offset from its address.
template <bool WS = false, class Fn>
__device__ __forceinline__ void walk_cm(const ProjGeom &g, int ci, const CmRay &r, bool ok,
                                        Fn &&fn, float ws = 1.f) {
    const unsigned full = 0xffffffffu;
    const int kb = __reduce_min_sync(full, ok ? r.k_lo : INT_MAX);
    const int ke = __reduce_max_sync(full, ok ? r.k_hi : -1);
    if (kb > ke) return;
    const int k_mid0 = max(kb, __reduce_max_sync(full, ok ? r.k_in0 : INT_MIN));
    const int k_mid1 = min(ke, __reduce_min_sync(full, ok ? r.k_in1 : INT_MAX));
    if (__all_sync(full, !ok || r.z_up))
        walk_cm_dir<1, WS>(g, ci, r, ok, kb, ke, k_mid0, k_mid1, fn, ws);
    else if (__all_sync(full, !ok || !r.z_up))
        walk_cm_dir<-1, WS>(g, ci, r, ok, kb, ke, k_mid0, k_mid1, fn, ws);
    else
        walk_cm_dir<0, WS>(g, ci, r, ok, kb, ke, k_mid0, k_mid1, fn, ws);
}

// One tile of p = alpha * rho o (A vol) + beta * p from the [y][x][z] copy
// vol_z (NULL: the all-ones volume); with NORM the tile's FP64 sum of p^2
// goes to partials[tile index in grid gdim].  All threads of the CTA call it.
template <bool HAS_RHO, bool NORM, bool UNIT_VOL, class TV, class TS>
__device__ __forceinline__ void forward_cm_tile(const ProjGeom &g, uint3 bid, uint3 gdim,
                                                const TV *__restrict__ vol_z,
                                                TS *__restrict__ out,
                                                const float *__restrict__ rho, const Coef &c,
                                                double *__restrict__ partials, double *sh) {
    int u, v, view;
    tile_of_cm(g, bid, u, v, view);
    const bool col_live = (u < g.nu) && (view < g.nviews);
    CmRay r;
    const bool ok = cm_setup(g, view, u, v, col_live, r);
    float acc = 0.f;
    if (col_live) {
        const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
        walk_cm(g, view * g.nu + u, r, ok, [&](int o, float l, bool p) {
            float val = 0.f;
            if (p && CT_IN_BOUNDS(o, nvox)) val = UNIT_VOL ? 1.f : ld_f(vol_z + o);
            acc = fmaf(l, val, acc);
        });
    }
    float alpha, beta;
    coef_of(c, alpha, beta);
    double sq = 0.0;
    const size_t idx = ((size_t)view * g.nv + v) * g.nu + u;
    if (col_live && v < g.nv && CT_IN_BOUNDS(idx, (int64_t)g.nviews * g.nv * g.nu)) {
        float val = ok ? acc * r.lsig : 0.f;
        if (HAS_RHO) val *= rho[idx];
        float o = alpha * val;
        if (beta != 0.f) o = fmaf(beta, to_f(out[idx]), o);
        const TS st = from_f<TS>(o);
        out[idx] = st;
        if (NORM) {
            const double q = (double)to_f(st);  // the norm of what is stored
            sq = q * q;
        }
    }
    if (NORM) {
        double t = block_sum_d(sq, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[bid.x + gdim.x * (bid.y + (size_t)gdim.y * bid.z)] = t;
    }
}

template <bool HAS_RHO, bool NORM, bool UNIT_VOL, class TV = float, class TS = float>
__global__ void __launch_bounds__(kCU *kCV, kFwdCtas) k_forward_cm(ProjGeom g,
                                                         const TV *__restrict__ vol_z,
                                                         TS *__restrict__ out,
                                                         const float *__restrict__ rho, Coef c,
                                                         double *__restrict__ partials) {
    __shared__ double sh[32];
    forward_cm_tile<HAS_RHO, NORM, UNIT_VOL, TV, TS>(g, blockIdx, gridDim, vol_z, out, rho, c,
                                                     partials, sh);
}

// One tile of acc_z ([y][x][z]) += the k_backward contributions of the
// column-major rays.  No CTA-wide synchronisation.
template <bool HAS_RHO, int POWER, bool DET, class TS>
__device__ __forceinline__ void backward_cm_tile(const ProjGeom &g, uint3 bid,
                                                 const TS *__restrict__ e,
                                                 const float *__restrict__ rho, const Coef &c,
                                                 void *__restrict__ acc_z,
                                                 const float *__restrict__ det_scale) {
    int u, v, view;
    tile_of_cm(g, bid, u, v, view);
    if (g.bt_pairs) {
        // Row blocks 2P and 2P + 1 (but a last unpaired one) swap to 4
        // columns x 64 rows each, a warp taking every other row: adjacent
        // lanes then sit ~2 rows apart in z, so no two lanes of a reduction
        // hit the same voxel when a detector row is less than a voxel high.
        const int vb = (int)bid.z % g.nvb;
        const int pair = vb >> 1, h = vb & 1;
        if (2 * pair + 1 < g.nvb) {
            const int w = threadIdx.y;
            u = bid.x * kCU + (kCU / 2) * h + (w >> 1);
            v = pair * 2 * kCV + 2 * threadIdx.x + (w & 1);
        }
    }
    const bool col_live = (u < g.nu) && (view < g.nviews);
    if (!col_live) return;   // warp-uniform
    CmRay r;
    const bool ok = cm_setup(g, view, u, v, col_live, r);
    float alpha, beta;
    coef_of(c, alpha, beta);
    float w = 0.f;
    const size_t idx = ((size_t)view * g.nv + v) * g.nu + u;
    if (ok && CT_IN_BOUNDS(idx, (int64_t)g.nviews * g.nv * g.nu)) {
        w = alpha * (e ? to_f(e[idx]) : 1.f);
        if (HAS_RHO) w *= rho[idx];
        if (POWER == 1) w *= r.lsig;
    }
    const bool nz = (w != 0.f);
    const float ls = r.lsig;
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
    if constexpr (DET) {
        const float scale = __ldg(det_scale);
        unsigned long long *base = static_cast<unsigned long long *>(acc_z);
        walk_cm(g, view * g.nu + u, r, ok, [&](int o, float l, bool p) {
            const float lm = l * ls;
            const float val = POWER == 1 ? w * l : w * lm * lm;
            red_add_u64_if(base + o, __float2ll_rn(val * scale),
                           p && nz && CT_IN_BOUNDS(o, nvox));
        });
    } else if constexpr (POWER == 1) {
        // the walk hands over the contributions w l themselves
        float *base = static_cast<float *>(acc_z);
        walk_cm<true>(g, view * g.nu + u, r, ok, [&](int o, float wl, bool p) {
            red_add_if(base + o, wl, p && nz && CT_IN_BOUNDS(o, nvox));
        }, w);
    } else {
        float *base = static_cast<float *>(acc_z);
        walk_cm(g, view * g.nu + u, r, ok, [&](int o, float l, bool p) {
            const float lm = l * ls;
            red_add_if(base + o, w * lm * lm, p && nz && CT_IN_BOUNDS(o, nvox));
        });
    }
}

template <bool HAS_RHO, int POWER, bool DET, class TS = float>
__global__ void __launch_bounds__(kCU *kCV, 5) k_backward_cm(ProjGeom g,
                                                          const TS *__restrict__ e,
                                                          const float *__restrict__ rho, Coef c,
                                                          void *__restrict__ acc_z,
                                                          const float *__restrict__ det_scale) {
    backward_cm_tile<HAS_RHO, POWER, DET, TS>(g, blockIdx, e, rho, c, acc_z, det_scale);
}

// ---- batched launches over several jobs -------------------------------------
// A persistent grid (resident CTAs only) takes tiles from a work counter in
// order: the tiles of job 0 in its own grid order, then those of job 1, and
// so on.  A tile runs exactly the code of a plain launch on that job (the
// same rays per CTA, the same partial sums in the same slots), so each job's
// result is the one of its own launch: bitwise for A and for fixed-point
// A^T.  Several small jobs thus share one launch and fill the GPU together.

// Next tile of the CTA (the same in all its threads), or UINT_MAX when none.
__device__ __forceinline__ unsigned next_tile(unsigned *next, unsigned ntiles, unsigned *slot) {
    if (threadIdx.x == 0 && threadIdx.y == 0) *slot = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned t = *slot;
    __syncthreads();   // read by all before thread 0 overwrites it
    return t < ntiles ? t : UINT_MAX;
}

// The job owning tile t (jobs sorted by tile0) and the tile within its grid.
__device__ __forceinline__ const BatchJob &job_of(const BatchJob *__restrict__ jobs, int njobs,
                                                  unsigned t, uint3 &bid, uint3 &gdim) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {   // the last job with tile0 <= t
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const BatchJob &b = jobs[lo];
    const unsigned lt = t - b.tile0;
    gdim = make_uint3(b.gx, b.gy, 0u);
    bid = make_uint3(lt % b.gx, (lt / b.gx) % b.gy, lt / (b.gx * b.gy));
    return b;
}

template <bool NORM>
__global__ void __launch_bounds__(kCU *kCV, kFwdCtas) k_forward_cm_batch(
    const BatchJob *__restrict__ jobs, int njobs, unsigned ntiles, unsigned *__restrict__ next) {
    __shared__ double sh[32];
    __shared__ unsigned slot;
    for (unsigned t = next_tile(next, ntiles, &slot); t != UINT_MAX;
         t = next_tile(next, ntiles, &slot)) {
        uint3 bid, gdim;
        const BatchJob &b = job_of(jobs, njobs, t, bid, gdim);
        const float *vz = static_cast<const float *>(b.in);
        float *out = static_cast<float *>(b.out);
        if (b.rho)
            forward_cm_tile<true, NORM, false, float, float>(b.g, bid, gdim, vz, out, b.rho, b.c,
                                                            b.partials, sh);
        else
            forward_cm_tile<false, NORM, false, float, float>(b.g, bid, gdim, vz, out, nullptr,
                                                             b.c, b.partials, sh);
    }
}

template <bool DET>
__global__ void __launch_bounds__(kCU *kCV, 5) k_backward_cm_batch(
    const BatchJob *__restrict__ jobs, int njobs, unsigned ntiles, unsigned *__restrict__ next) {
    __shared__ unsigned slot;
    for (unsigned t = next_tile(next, ntiles, &slot); t != UINT_MAX;
         t = next_tile(next, ntiles, &slot)) {
        uint3 bid, gdim;
        const BatchJob &b = job_of(jobs, njobs, t, bid, gdim);
        const float *e = static_cast<const float *>(b.in);
        if (b.rho)
            backward_cm_tile<true, 1, DET, float>(b.g, bid, e, b.rho, b.c, b.out, b.det_scale);
        else
            backward_cm_tile<false, 1, DET, float>(b.g, bid, e, nullptr, b.c, b.out, b.det_scale);
    }
}

// Grid of the projector kernels (column-major tiles when pg.cm, else
// ray-major ones); see set_launch_order for the order.
dim3 proj_grid(const ProjGeom &pg) {
    const int ngroups = (pg.nviews + pg.vgroup - 1) / pg.vgroup;
    const int tu = pg.cm ? kCU : kTU;
    return dim3((unsigned)((pg.nu + tu - 1) / tu), (unsigned)pg.vgroup,
                (unsigned)(pg.nvb * ngroups));
}

// CTA shape of the projector kernels: kCV lanes x kCU warps (column-major)
// or kTU x kTV (ray-major).
dim3 proj_block(const ProjGeom &pg) { return pg.cm ? dim3(kCV, kCU) : dim3(kTU, kTV); }

// View groups that keep grid z = nvb * ceil(nviews / vgroup) <= 65535.
int min_view_group(int nviews, int nvb) {
    const int max_groups = std::max(1, 65535 / nvb);
    return (nviews + max_groups - 1) / max_groups;
}

// The ray-major order used by the nnz counter and the direct forward
// projection, whatever pg.cm says: one view at a time.
ProjGeom rays_order(const ProjGeom &pg) {
    ProjGeom pr = pg;
    pr.cm = 0;
    pr.nvb = std::max(1, (pg.nv + kTV - 1) / kTV);
    pr.vgroup = std::max(1, std::min(min_view_group(pg.nviews, pr.nvb), std::max(pg.nviews, 1)));
    pr.vgroup_bt = pr.vgroup;
    return pr;
}

// The same geometry with the launch order of A^T.
ProjGeom back_order(const ProjGeom &pg) {
    ProjGeom pb = pg;
    pb.vgroup = pg.vgroup_bt;
    return pb;
}

bool empty(const ProjGeom &pg) { return pg.nu <= 0 || pg.nv <= 0 || pg.nviews <= 0; }

}  // namespace

// CTAs are issued roughly in linear order, x fastest, so the tiles in flight
// at a time are all columns of vgroup views for a few row blocks, then the
// next row blocks of the same views.  vgroup = 1 visits a view at a time: its
// rays are nearly disjoint (few reductions into the same voxel at once) but
// every view sweeps the whole volume.  A large vgroup keeps the CTAs in flight
// on a band of z slices (the rows of a few row blocks) of the volume for all
// views of the group: for a volume that does not fit in L2 (512^3 FP32 plus
// its transposed copy: 1 GB) that band stays resident, which takes fewer DRAM
// reads and, in A^T, fewer L2 misses of the reductions.  Measured on 512^3
// with 720 views (ray-major kernels): A 229 ms with one view at a time,
// 139 ms with all views in one group; A^T 264 ms with one view, 165 ms with
// groups of 16 and 169 ms with all views (more views at once put more
// reductions on the same voxels at the same time).  The column-major A^T
// takes 145 ms with groups of 16 and 142.5 ms with all views.  On 256^3
// (2 x 64 MB) one view at a time is best for both.
void set_launch_order(ProjGeom &pg) {
    const int tv = pg.cm ? kCV : kTV;
    pg.nvb = std::max(1, (pg.nv + tv - 1) / tv);
    const int64_t vol_bytes = 2 * (int64_t)pg.nx * pg.ny * pg.nz * (int64_t)sizeof(float);
    const bool wide = vol_bytes > kL2GroupBytes;
    const int need = min_view_group(pg.nviews, pg.nvb);
    auto clampg = [&](int g) { return std::max(1, std::min(std::max(g, need), std::max(pg.nviews, 1))); };
    pg.vgroup = clampg(wide ? kWideGroupFwd : 1);
    pg.vgroup_bt = clampg(wide ? (pg.cm ? kWideGroupFwd : kWideGroupBack) : 1);
    pg.bt_pairs = 0;
}

// Row pairing of the column-major A^T (ProjGeom::bt_pairs).  A warp's lanes
// are rows of one column; where a detector row spans less than a voxel in z
// (at the isocentre: row_vox = dv * SID / (SDD * vz)), neighbouring lanes
// often reduce into the same voxel, and the reduction replays.  Taking every
// other row halves that.  Measured on 256^3 (row_vox 0.625, one view at a
// time): A^T 11.94 -> 11.11 ms.  On 512^3 (row_vox 0.94, all views in one
// group) it spread each warp over more sectors and broke the band order
// (140.8 -> 178.5 ms), hence the conditions.
void set_row_pairing(ProjGeom &pg, double row_vox) {
    pg.bt_pairs = (pg.cm && pg.vgroup_bt == 1 && row_vox < kPairRowVox) ? 1 : 0;
}

int64_t forward_partials(const ProjGeom &pg) {
    if (empty(pg)) return 0;
    if (pg.proj != CT_PROJ_SIDDON) return sf_forward_partials(pg);
    dim3 gr = proj_grid(pg);
    return (int64_t)gr.x * gr.y * gr.z;
}

int64_t forward_direct_partials(const ProjGeom &pg) {
    if (empty(pg)) return 0;
    if (pg.proj != CT_PROJ_SIDDON) return sf_forward_partials(pg);
    dim3 gr = proj_grid(rays_order(pg));
    return (int64_t)gr.x * gr.y * gr.z;
}

ct_status launch_forward(const ProjGeom &pg, const float *vol, const float *vol_t, float *p,
                         const float *rho, Coef c, double *partials, cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) return sf_forward(pg, vol, p, rho, c, partials, st);
    dim3 gr = proj_grid(pg), bl = proj_block(pg);
    const bool unit = (vol == nullptr);
    const bool hr = (rho != nullptr), nm = (partials != nullptr);
#define CT_FWD(HR, NM, UV)                                                             \
    do {                                                                               \
        if (pg.cm)                                                                     \
            k_forward_cm<HR, NM, UV><<<gr, bl, 0, st>>>(pg, vol_t, p, rho, c, partials);  \
        else                                                                           \
            k_forward<HR, NM, UV><<<gr, bl, 0, st>>>(pg, vol, vol_t, p, rho, c, partials); \
    } while (0)
    if (unit) {
        if (hr) { if (nm) CT_FWD(true, true, true); else CT_FWD(true, false, true); }
        else    { if (nm) CT_FWD(false, true, true); else CT_FWD(false, false, true); }
    } else {
        if (hr) { if (nm) CT_FWD(true, true, false); else CT_FWD(true, false, false); }
        else    { if (nm) CT_FWD(false, true, false); else CT_FWD(false, false, false); }
    }
#undef CT_FWD
    CT_CHECK_LAUNCH();
    return CT_OK;
}

namespace {

template <class TV, class TS>
ct_status fwd_typed(const ProjGeom &pg, const void *vol, const void *vol_t, void *p,
                    const float *rho, Coef c, double *partials, cudaStream_t st) {
    dim3 gr = proj_grid(pg), bl = proj_block(pg);
    const TV *v = static_cast<const TV *>(vol);
    const TV *vt = static_cast<const TV *>(vol_t);
    TS *o = static_cast<TS *>(p);
#define CT_FWDT(HR, NM)                                                                         \
    do {                                                                                        \
        if (pg.cm)                                                                              \
            k_forward_cm<HR, NM, false, TV, TS><<<gr, bl, 0, st>>>(pg, vt, o, rho, c, partials);  \
        else                                                                                    \
            k_forward<HR, NM, false, TV, TS><<<gr, bl, 0, st>>>(pg, v, vt, o, rho, c, partials); \
    } while (0)
    if (rho) {
        if (partials) CT_FWDT(true, true);
        else          CT_FWDT(true, false);
    } else {
        if (partials) CT_FWDT(false, true);
        else          CT_FWDT(false, false);
    }
#undef CT_FWDT
    CT_CHECK_LAUNCH();
    return CT_OK;
}

template <class TV>
ct_status fwd_typed_s(const ProjGeom &pg, const void *vol, const void *vol_t, void *p, int sdt,
                      const float *rho, Coef c, double *partials, cudaStream_t st) {
    switch (sdt) {
        case CT_F32: return fwd_typed<TV, float>(pg, vol, vol_t, p, rho, c, partials, st);
        case CT_BF16: return fwd_typed<TV, __nv_bfloat16>(pg, vol, vol_t, p, rho, c, partials, st);
        case CT_F16: return fwd_typed<TV, __half>(pg, vol, vol_t, p, rho, c, partials, st);
    }
    return set_error(CT_ERR_INVALID_ARG, "unknown sinogram dtype");
}

template <class TS>
ct_status back_typed(const ProjGeom &pg, const void *e, const float *rho, Coef c, void *acc,
                     void *acc_t, int power, bool det, const float *det_scale, cudaStream_t st) {
    const ProjGeom pb = back_order(pg);
    dim3 gr = proj_grid(pb), bl = proj_block(pb);
    const TS *et = static_cast<const TS *>(e);
    const bool hr = rho != nullptr;
#define CT_BWD(HR, P, D)                                                                      \
    do {                                                                                      \
        if (pg.cm)                                                                            \
            k_backward_cm<HR, P, D, TS><<<gr, bl, 0, st>>>(pb, et, rho, c, acc_t, det_scale);  \
        else                                                                                  \
            k_backward<HR, P, D, TS><<<gr, bl, 0, st>>>(pb, et, rho, c, acc, acc_t, det_scale); \
    } while (0)
    if (det) {
        if (power == 2) { if (hr) CT_BWD(true, 2, true); else CT_BWD(false, 2, true); }
        else            { if (hr) CT_BWD(true, 1, true); else CT_BWD(false, 1, true); }
    } else {
        if (power == 2) { if (hr) CT_BWD(true, 2, false); else CT_BWD(false, 2, false); }
        else            { if (hr) CT_BWD(true, 1, false); else CT_BWD(false, 1, false); }
    }
#undef CT_BWD
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace

ct_status launch_forward_typed(const ProjGeom &pg, const void *vol, const void *vol_t, int vdt,
                               void *p, int sdt, const float *rho, Coef c, double *partials,
                               cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) {
        if (vdt != CT_F32 || sdt != CT_F32)
            return set_error(CT_ERR_INVALID_ARG, "footprint projectors need FP32 storage");
        return sf_forward(pg, static_cast<const float *>(vol), static_cast<float *>(p), rho, c,
                          partials, st);
    }
    switch (vdt) {
        case CT_F32: return fwd_typed_s<float>(pg, vol, vol_t, p, sdt, rho, c, partials, st);
        case CT_BF16:
            return fwd_typed_s<__nv_bfloat16>(pg, vol, vol_t, p, sdt, rho, c, partials, st);
        case CT_F16: return fwd_typed_s<__half>(pg, vol, vol_t, p, sdt, rho, c, partials, st);
    }
    return set_error(CT_ERR_INVALID_ARG, "unknown volume dtype");
}

ct_status launch_backward_typed(const ProjGeom &pg, const void *e, int sdt, const float *rho,
                                Coef c, void *acc, void *acc_t, int power, bool det,
                                const float *det_scale, cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) {
        if (sdt != CT_F32 || det)
            return set_error(CT_ERR_INVALID_ARG,
                             "footprint projectors need FP32 storage and float accumulation");
        return sf_backward(pg, static_cast<const float *>(e), rho, c, static_cast<float *>(acc),
                           power, st);
    }
    switch (sdt) {
        case CT_F32:
            return back_typed<float>(pg, e, rho, c, acc, acc_t, power, det, det_scale, st);
        case CT_BF16:
            return back_typed<__nv_bfloat16>(pg, e, rho, c, acc, acc_t, power, det, det_scale, st);
        case CT_F16:
            return back_typed<__half>(pg, e, rho, c, acc, acc_t, power, det, det_scale, st);
    }
    return set_error(CT_ERR_INVALID_ARG, "unknown sinogram dtype");
}

ct_status launch_backward(const ProjGeom &pg, const float *e, const float *rho, Coef c,
                          float *acc, float *acc_t, int power, cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) return sf_backward(pg, e, rho, c, acc, power, st);
    return back_typed<float>(pg, e, rho, c, acc, acc_t, power, false, nullptr, st);
}

ct_status launch_backward_det(const ProjGeom &pg, const float *e, const float *rho, Coef c,
                              long long *acc, long long *acc_t, int power,
                              const float *det_scale, cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON)
        return set_error(CT_ERR_INVALID_ARG, "footprint projectors: no fixed-point mode");
    return back_typed<float>(pg, e, rho, c, acc, acc_t, power, true, det_scale, st);
}

bool batchable(const ProjGeom &pg) { return pg.proj == CT_PROJ_SIDDON && pg.cm && !empty(pg); }

ct_status batch_job_grid(const ProjGeom &pg, bool backward, BatchJob *b) {
    if (!batchable(pg)) return set_error(CT_ERR_INVALID_ARG, "geometry cannot be batched");
    b->g = backward ? back_order(pg) : pg;
    const dim3 gr = proj_grid(b->g);
    b->gx = gr.x;
    b->gy = gr.y;
    b->tiles = gr.x * gr.y * gr.z;
    return CT_OK;
}

namespace {
constexpr int kMaxDevices = 64;
// Resident CTAs of the four batched kernels per device (0: not yet known),
// found by batch_prepare outside any stream capture.
std::atomic<int> g_batch_grid[kMaxDevices][4];

template <class K>
ct_status resident_ctas(K kernel, int dev, int *grid) {
    int sms = 0, per_sm = 0;
    CT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kCU * kCV, 0));
    *grid = std::max(1, sms * std::max(per_sm, 1));
    return CT_OK;
}
}  // namespace

ct_status batch_prepare() {
    int dev = 0;
    CT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(CT_ERR_INVALID_ARG, "device index");
    int gr[4];
    CT_TRY(resident_ctas(k_backward_cm_batch<false>, dev, &gr[0]));
    CT_TRY(resident_ctas(k_backward_cm_batch<true>, dev, &gr[1]));
    CT_TRY(resident_ctas(k_forward_cm_batch<false>, dev, &gr[2]));
    CT_TRY(resident_ctas(k_forward_cm_batch<true>, dev, &gr[3]));
    for (int k = 0; k < 4; ++k) g_batch_grid[dev][k].store(gr[k]);
    return CT_OK;
}

ct_status launch_batch(const BatchJob *d_jobs, int njobs, unsigned ntiles, bool backward,
                       bool flag, unsigned *d_next, cudaStream_t st) {
    if (njobs <= 0 || ntiles == 0) return CT_OK;
    int dev = 0;
    CT_CUDA_TRY(cudaGetDevice(&dev));
    const int which = (backward ? 0 : 2) + (flag ? 1 : 0);
    const int resident = (dev >= 0 && dev < kMaxDevices) ? g_batch_grid[dev][which].load() : 0;
    if (resident <= 0) return set_error(CT_ERR_INVALID_ARG, "launch_batch before batch_prepare");
    const unsigned grid = std::min<unsigned>((unsigned)resident, ntiles);
    CT_CUDA_TRY(cudaMemsetAsync(d_next, 0, sizeof(unsigned), st));
    const dim3 bl(kCV, kCU);
    if (backward) {
        if (flag) k_backward_cm_batch<true><<<grid, bl, 0, st>>>(d_jobs, njobs, ntiles, d_next);
        else      k_backward_cm_batch<false><<<grid, bl, 0, st>>>(d_jobs, njobs, ntiles, d_next);
    } else {
        if (flag) k_forward_cm_batch<true><<<grid, bl, 0, st>>>(d_jobs, njobs, ntiles, d_next);
        else      k_forward_cm_batch<false><<<grid, bl, 0, st>>>(d_jobs, njobs, ntiles, d_next);
    }
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_count(const ProjGeom &pg, unsigned long long *d_count, cudaStream_t st) {
    CT_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) return sf_count(pg, d_count, st);
    const ProjGeom pr = rays_order(pg);
    k_count<<<proj_grid(pr), dim3(kTU, kTV), 0, st>>>(pr, d_count);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_forward_direct(const ProjGeom &pg, const float *vol, float *p, float alpha,
                                float beta, double *partials, cudaStream_t st) {
    if (empty(pg)) return CT_OK;
    if (pg.proj != CT_PROJ_SIDDON) {
        Coef c;
        c.alpha = alpha;
        c.beta = beta;
        return sf_forward(pg, vol, p, nullptr, c, partials, st);
    }
    const ProjGeom pr = rays_order(pg);
    k_forward_direct<<<proj_grid(pr), dim3(kTU, kTV), 0, st>>>(pr, vol, p, alpha, beta,
                                                               partials);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace ct

CT_DEBUG_ACCESSOR(debug_take_projector)
