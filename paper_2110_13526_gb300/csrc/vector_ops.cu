// Streaming volume / sinogram kernels and deterministic FP64 reductions.
//
// Norms feeding the Krylov scalars (Algorithm 1: NR2 = ||r_x||^2,
// NP2 = ||p_b||^2, NB = ||e_b||) are accumulated in FP64 (the Discussion
// notes the package relies on double precision): each CTA writes one partial,
// and one CTA sums the partials in a fixed order, so a result never depends
// on scheduling.
#include <algorithm>

#include "ct_internal.h"
#include "ct_types.cuh"

namespace ct {
namespace {

constexpr int kTile = 32;

__device__ __forceinline__ double block_sum_1d(double x, double *sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// in [nz][ny][nx] -> t [nz][nx][ny]; optionally scaled by w, optionally also
// writing the scaled volume in the original layout.
__global__ void __launch_bounds__(256) k_transpose(int nx, int ny, const float *__restrict__ in,
                                                   const float *__restrict__ w,
                                                   float *__restrict__ t,
                                                   float *__restrict__ plain) {
    __shared__ float tile[kTile][kTile + 1];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t zoff = (size_t)blockIdx.z * nx * ny;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + j;
        if (x < nx && y < ny) {
            const size_t i = zoff + (size_t)y * nx + x;
            float val = in[i];
            if (w) val *= w[i];
            if (plain) plain[i] = val;
            tile[j][threadIdx.x] = val;
        }
    }
    __syncthreads();
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + j;
        if (x < nx && y < ny) t[zoff + (size_t)x * ny + y] = tile[threadIdx.x][j];
    }
}

// g[z][y][x] += acc_t[z][x][y]; optional partial of sum (w g)^2 per CTA.
__global__ void __launch_bounds__(256) k_combine(int nx, int ny, float *__restrict__ g,
                                                 const float *__restrict__ acc_t,
                                                 const float *__restrict__ w,
                                                 double *__restrict__ partials) {
    __shared__ float tile[kTile][kTile + 1];
    __shared__ double sh[32];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t zoff = (size_t)blockIdx.z * nx * ny;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (x < nx && y < ny) tile[j][threadIdx.x] = acc_t[zoff + (size_t)x * ny + y];
    }
    __syncthreads();
    SqSum sq;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (x < nx && y < ny) {
            const size_t i = zoff + (size_t)y * nx + x;
            const float val = g[i] + tile[threadIdx.x][j];
            g[i] = val;
            sq.add(w ? w[i] * val : val);
        }
    }
    if (partials) {
        const double t = block_sum_1d(sq.value(), sh);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
    }
}

__global__ void k_mul(float *__restrict__ out, const float *__restrict__ v,
                      const float *__restrict__ w, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = v[i] * w[i];
}

__global__ void k_scale(float *__restrict__ out, int64_t n, float beta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (beta == 0.f) ? 0.f : beta * out[i];
}

__global__ void k_scale_dev(float *__restrict__ out, int64_t n, const double *__restrict__ beta) {
    const float b = (float)beta[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (b == 0.f) ? 0.f : b * out[i];
}

__global__ void k_norm2(const float *__restrict__ v, const float *__restrict__ w, int64_t n,
                        double *__restrict__ partials) {
    __shared__ double sh[32];
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        sq.add(w ? w[i] * v[i] : v[i]);
    const double t = block_sum_1d(sq.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// One CTA of 1024 threads: thread t sums partials t, t + 1024, ... in order,
// then a fixed tree.
__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ partials, int64_t n,
                                              double *__restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    const double t = block_sum_1d(s, sh);
    if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

// ---- [y][x][z] copies of the column-major kernels ----------------------------
// Each CTA transposes one 32 x 32 tile of the (z, x) plane of y = blockIdx.z,
// blockIdx.z + gridDim.z, ... (gridDim.z <= 65535 whatever ny is), reading
// and writing along the fastest axis of each layout.
namespace {

// Tiles of (x, z) for every CTA, about two waves of 8 CTAs on each of 152
// SMs, each CTA walking y planes (at least two, handled in pairs by
// k_from_zfast so that twice the loads are in flight per sync).
dim3 zfast_grid(const ProjGeom &pg) {
    const int64_t gx = (pg.nx + kTile - 1) / kTile, gy = (pg.nz + kTile - 1) / kTile;
    int64_t gz = (int64_t(152) * 8 * 2 + gx * gy - 1) / (gx * gy);
    gz = std::min<int64_t>(gz, (pg.ny + 1) / 2);
    gz = std::max<int64_t>(1, std::min<int64_t>(gz, 65535));
    return dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
}

// in [nz][ny][nx] -> t [ny][nx][nz]; optionally scaled by w (FP32 only) and
// optionally writing the scaled volume in the original layout too.
template <class T>
__global__ void __launch_bounds__(256) k_to_zfast(int nx, int ny, int nz, const T *__restrict__ in,
                                                  const float *__restrict__ w, T *__restrict__ t,
                                                  T *__restrict__ plain) {
    __shared__ T tile[kTile][kTile + 1];
    const int x0 = blockIdx.x * kTile, z0 = blockIdx.y * kTile;
    for (int y = blockIdx.z; y < ny; y += gridDim.z) {
        for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
            const int x = x0 + threadIdx.x, z = z0 + j;
            if (x < nx && z < nz) {
                const size_t i = ((size_t)z * ny + y) * nx + x;
                T val = in[i];
                if (w) val = from_f<T>(to_f(val) * w[i]);
                if (plain) plain[i] = val;
                tile[j][threadIdx.x] = val;
            }
        }
        __syncthreads();
        for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
            const int z = z0 + threadIdx.x, x = x0 + j;
            if (x < nx && z < nz) t[((size_t)y * nx + x) * nz + z] = tile[threadIdx.x][j];
        }
        __syncthreads();
    }
}

// A [y][x][z] accumulator: FP32 sums f, or int64 sums q worth q * inv[0]
// (inv: device pointer to the exact inverse of the fixed-point scale).
struct ZAcc {
    const float *f;
    const long long *q;
    const double *inv;
};

// out[z][y][x] = beta out + acc[y][x][z] (stored as T); int64 sums are scaled
// in FP64 and rounded once to FP32.  Optional FP64 partial per CTA of
// sum (w out)^2 over the stored values.
template <class T>
__global__ void __launch_bounds__(256) k_from_zfast(int nx, int ny, int nz, T *__restrict__ out,
                                                    float beta, ZAcc acc,
                                                    const float *__restrict__ w,
                                                    double *__restrict__ partials) {
    __shared__ float tile[2][kTile][kTile + 1];
    __shared__ double sh[32];
    const int x0 = blockIdx.x * kTile, z0 = blockIdx.y * kTile;
    const double s = acc.q ? acc.inv[0] : 1.0;
    SqSum sq;
    // planes y and y + gridDim.z together (the second may not exist)
    for (int y = blockIdx.z; y < ny; y += 2 * (int)gridDim.z) {
        const int yy[2] = {y, y + (int)gridDim.z};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (yy[h] >= ny) continue;   // uniform in the CTA
            for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
                const int x = x0 + j, z = z0 + threadIdx.x;
                if (x < nx && z < nz) {
                    const size_t it = ((size_t)yy[h] * nx + x) * nz + z;
                    tile[h][j][threadIdx.x] = acc.q ? (float)((double)acc.q[it] * s) : acc.f[it];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (yy[h] >= ny) continue;
            for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
                const int z = z0 + j, x = x0 + threadIdx.x;
                if (x < nx && z < nz) {
                    const size_t i = ((size_t)z * ny + yy[h]) * nx + x;
                    float val = tile[h][threadIdx.x][j];
                    if (beta != 0.f) val = fmaf(beta, to_f(out[i]), val);  // beta 1: a plain add
                    const T st = from_f<T>(val);
                    out[i] = st;
                    if (partials) {
                        const float vs = to_f(st);
                        sq.add(w ? w[i] * vs : vs);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (partials) {
        const double t = block_sum_1d(sq.value(), sh);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
    }
}

template <class T>
ct_status from_zfast(const ProjGeom &pg, T *out, float beta, ZAcc acc, const float *w,
                     double *partials, cudaStream_t st) {
    k_from_zfast<T><<<zfast_grid(pg), dim3(kTile, 8), 0, st>>>(pg.nx, pg.ny, pg.nz, out, beta,
                                                               acc, w, partials);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace

int vec_grid(int64_t n) {
    int64_t b = (n + kVecThreads * 4 - 1) / (kVecThreads * 4);
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

int transpose_grid_count(const ProjGeom &pg) {
    // the footprint projectors accumulate A^T in place; their combine only
    // takes the norm partials
    if (pg.proj != CT_PROJ_SIDDON) return vec_grid((int64_t)pg.nx * pg.ny * pg.nz);
    if (pg.cm) {
        const dim3 g = zfast_grid(pg);
        return (int)(g.x * g.y * g.z);
    }
    return ((pg.nx + kTile - 1) / kTile) * ((pg.ny + kTile - 1) / kTile) * pg.nz;
}

ct_status launch_transpose(const ProjGeom &pg, const float *v, const float *w, float *t,
                           float *out_plain, cudaStream_t st) {
    if (pg.proj != CT_PROJ_SIDDON) {
        // the footprint projectors read the caller's layout: only the scaled copy
        if (!out_plain) return CT_OK;
        const int64_t n = (int64_t)pg.nx * pg.ny * pg.nz;
        if (w) return launch_mul(out_plain, v, w, n, st);
        CT_CUDA_TRY(cudaMemcpyAsync(out_plain, v, (size_t)n * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
        return CT_OK;
    }
    if (pg.cm) {
        k_to_zfast<float><<<zfast_grid(pg), dim3(kTile, 8), 0, st>>>(pg.nx, pg.ny, pg.nz, v, w, t,
                                                                     out_plain);
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    dim3 gr((pg.nx + kTile - 1) / kTile, (pg.ny + kTile - 1) / kTile, pg.nz), bl(kTile, 8);
    k_transpose<<<gr, bl, 0, st>>>(pg.nx, pg.ny, v, w, t, out_plain);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_combine(const ProjGeom &pg, float *g, const float *acc_t, const float *w,
                         double *partials, cudaStream_t st, float beta) {
    if (pg.proj != CT_PROJ_SIDDON) {
        if (!partials) return CT_OK;
        return launch_norm2(g, w, (int64_t)pg.nx * pg.ny * pg.nz, partials, st);
    }
    if (pg.cm)
        return from_zfast<float>(pg, g, beta, ZAcc{acc_t, nullptr, nullptr}, w, partials, st);
    dim3 gr((pg.nx + kTile - 1) / kTile, (pg.ny + kTile - 1) / kTile, pg.nz), bl(kTile, 8);
    k_combine<<<gr, bl, 0, st>>>(pg.nx, pg.ny, g, acc_t, w, partials);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_mul(float *out, const float *v, const float *w, int64_t n, cudaStream_t st) {
    if (n <= 0) return CT_OK;
    k_mul<<<vec_grid(n), kVecThreads, 0, st>>>(out, v, w, n);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_scale(float *out, int64_t n, float beta, cudaStream_t st) {
    if (n <= 0) return CT_OK;
    if (beta == 0.f) {
        CT_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)n * sizeof(float), st));
        return CT_OK;
    }
    if (beta == 1.f) return CT_OK;
    k_scale<<<vec_grid(n), kVecThreads, 0, st>>>(out, n, beta);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_scale_dev(float *out, int64_t n, const double *beta, cudaStream_t st) {
    if (n <= 0) return CT_OK;
    k_scale_dev<<<vec_grid(n), kVecThreads, 0, st>>>(out, n, beta);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_sum(const double *partials, int64_t n, double *out, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(partials, n, out);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_norm2(const float *v, const float *w, int64_t n, double *partials,
                       cudaStream_t st) {
    k_norm2<<<vec_grid(n), kVecThreads, 0, st>>>(v, w, n, partials);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace ct

// ---- guarded inverse square roots (preconditioner weights) ------------------
namespace ct {
namespace {

__global__ void k_max_partials(const float *__restrict__ v, int64_t n, float *__restrict__ part) {
    __shared__ float sh[32];
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_down_sync(0xffffffffu, t, o));
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// v = 1 / sqrt(v) where v > rel * max(v), else 0.  part[0..np) hold block maxima.
__global__ void k_inv_sqrt_guard(float *__restrict__ v, int64_t n, const float *__restrict__ part,
                                 int np, float rel) {
    float m = 0.f;
    for (int i = 0; i < np; ++i) m = fmaxf(m, part[i]);
    const float thr = rel * m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[i];
        v[i] = (x > thr && x > 0.f) ? 1.f / sqrtf(x) : 0.f;
    }
}

}  // namespace

ct_status launch_inv_sqrt_guarded(float *v, int64_t n, float rel, float *part, cudaStream_t st) {
    if (n <= 0) return CT_OK;
    const int gb = vec_grid(n);
    k_max_partials<<<gb, kVecThreads, 0, st>>>(v, n, part);
    CT_CHECK_LAUNCH();
    k_inv_sqrt_guard<<<gb, kVecThreads, 0, st>>>(v, n, part, gb, rel);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

// ---- deterministic (fixed-point) backprojection support ---------------------
namespace {

// Block maxima of |e_i rho_i| (e or rho NULL: 1).
template <class TE>
__global__ void k_absmax_partials(const TE *__restrict__ e, const float *__restrict__ rho,
                                  int64_t n, float *__restrict__ part) {
    __shared__ float sh[32];
    float m = 0.f;
    if (!e && !rho) {
        m = n > 0 ? 1.f : 0.f;
    } else {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf((e ? to_f(e[i]) : 1.f) * (rho ? rho[i] : 1.f)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_down_sync(0xffffffffu, t, o));
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// scale = 2^k with k the largest integer such that |alpha| max|e rho| * bound
// * 2^k <= 2^62 (clamped to [-126, 126]); out[0] = scale (float), and the
// exact inverse 2^-k goes to inv[0] (double).
__device__ void det_scale_of(double top, float *__restrict__ out, double *__restrict__ inv) {
    int k = 126;
    if (top > 0.0 && top < 1e300) {
        int ex = 0;
        (void)frexp(top, &ex);   // top = f 2^ex, f in [0.5, 1)
        k = 62 - ex;
        k = k > 126 ? 126 : (k < -126 ? -126 : k);
    }
    out[0] = __int_as_float((k + 127) << 23);
    inv[0] = __longlong_as_double((long long)(1023 - k) << 52);
}

__global__ void k_det_scale(const float *__restrict__ part, int np, double bound, Coef c,
                            float *__restrict__ out, double *__restrict__ inv) {
    float m = 0.f;
    for (int i = 0; i < np; ++i) m = fmaxf(m, part[i]);
    const double alpha = c.dev ? fabs(c.dev[0]) : fabs((double)c.alpha);
    det_scale_of((double)m * alpha * bound, out, inv);
}

// Forward projection: the maxima of |x| (part[0, npx)) and |rho|
// (part[npx, npx + npr); npr 0: rho = 1) multiply.
__global__ void k_det_scale_fwd(const float *__restrict__ part, int npx, int npr, double bound,
                                Coef c, float *__restrict__ out, double *__restrict__ inv) {
    float mx = 0.f, mr = npr > 0 ? 0.f : 1.f;
    for (int i = 0; i < npx; ++i) mx = fmaxf(mx, part[i]);
    for (int i = 0; i < npr; ++i) mr = fmaxf(mr, part[npx + i]);
    const double alpha = c.dev ? fabs(c.dev[0]) : fabs((double)c.alpha);
    det_scale_of((double)mx * (double)mr * alpha * bound, out, inv);
}

// out = beta * out + (acc + transpose(acc_t)) * inv; optional partials of
// (w out)^2 per CTA.  acc: [nz][ny][nx], acc_t: [nz][nx][ny] (int64).
__global__ void __launch_bounds__(256) k_combine_det(int nx, int ny, float *__restrict__ out,
                                                     float beta, const long long *__restrict__ acc,
                                                     const long long *__restrict__ acc_t,
                                                     const double *__restrict__ inv,
                                                     const float *__restrict__ w,
                                                     double *__restrict__ partials) {
    __shared__ long long tile[kTile][kTile + 1];
    __shared__ double sh[32];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t zoff = (size_t)blockIdx.z * nx * ny;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (x < nx && y < ny) tile[j][threadIdx.x] = acc_t[zoff + (size_t)x * ny + y];
    }
    __syncthreads();
    const double s = inv[0];
    SqSum sq;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (x < nx && y < ny) {
            const size_t i = zoff + (size_t)y * nx + x;
            const long long q = acc[i] + tile[threadIdx.x][j];
            float val = (float)((double)q * s);
            if (beta != 0.f) val = fmaf(beta, out[i], val);
            out[i] = val;
            sq.add(w ? w[i] * val : val);
        }
    }
    if (partials) {
        const double t = block_sum_1d(sq.value(), sh);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
    }
}

}  // namespace

ct_status launch_det_scale(const void *e, int edt, const float *rho, int64_t m, double bound,
                           Coef c, float *part, float *scale, double *inv, cudaStream_t st) {
    const int gb = vec_grid(m);
    switch (edt) {
        case CT_BF16:
            k_absmax_partials<<<gb, kVecThreads, 0, st>>>((const __nv_bfloat16 *)e, rho, m, part);
            break;
        case CT_F16:
            k_absmax_partials<<<gb, kVecThreads, 0, st>>>((const __half *)e, rho, m, part);
            break;
        default:
            k_absmax_partials<<<gb, kVecThreads, 0, st>>>((const float *)e, rho, m, part);
    }
    CT_CHECK_LAUNCH();
    k_det_scale<<<1, 1, 0, st>>>(part, gb, bound, c, scale, inv);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_det_scale_fwd(const float *x, int64_t n, const float *rho, int64_t m,
                               double bound, Coef c, float *part, float *scale, double *inv,
                               cudaStream_t st) {
    const int gx = vec_grid(n), gr = rho ? vec_grid(m) : 0;
    k_absmax_partials<<<gx, kVecThreads, 0, st>>>(x, nullptr, n, part);
    CT_CHECK_LAUNCH();
    if (rho) {
        k_absmax_partials<<<gr, kVecThreads, 0, st>>>(rho, nullptr, m, part + gx);
        CT_CHECK_LAUNCH();
    }
    k_det_scale_fwd<<<1, 1, 0, st>>>(part, gx, gr, bound, c, scale, inv);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_combine_det(const ProjGeom &pg, float *out, float beta, const long long *acc,
                             const long long *acc_t, const double *inv, const float *w,
                             double *partials, cudaStream_t st) {
    if (pg.proj != CT_PROJ_SIDDON)
        return set_error(CT_ERR_INVALID_ARG, "footprint projectors: no fixed-point mode");
    if (pg.cm) return from_zfast<float>(pg, out, beta, ZAcc{nullptr, acc_t, inv}, w, partials, st);
    dim3 gr((pg.nx + kTile - 1) / kTile, (pg.ny + kTile - 1) / kTile, pg.nz), bl(kTile, 8);
    k_combine_det<<<gr, bl, 0, st>>>(pg.nx, pg.ny, out, beta, acc, acc_t, inv, w, partials);
    CT_CHECK_LAUNCH();
    return CT_OK;
}

// ---- typed storage -------------------------------------------------------------
namespace {

template <class T>
__global__ void __launch_bounds__(256) k_transpose_t(int nx, int ny, const T *__restrict__ in,
                                                     T *__restrict__ t) {
    __shared__ T tile[kTile][kTile + 1];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t zoff = (size_t)blockIdx.z * nx * ny;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + j;
        if (x < nx && y < ny) tile[j][threadIdx.x] = in[zoff + (size_t)y * nx + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + j;
        if (x < nx && y < ny) t[zoff + (size_t)x * ny + y] = tile[threadIdx.x][j];
    }
}

// out (T) = beta out + acc + transpose(acc_t) (FP32 sums), or the int64 sums
// q, q + nvox times inv[0] when q is set.
template <class T>
__global__ void __launch_bounds__(256) k_combine_t(int nx, int ny, int64_t nvox, T *__restrict__ out,
                                                   float beta, const float *__restrict__ acc,
                                                   const float *__restrict__ acc_t,
                                                   const long long *__restrict__ q,
                                                   const double *__restrict__ inv) {
    __shared__ double tile[kTile][kTile + 1];
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const size_t zoff = (size_t)blockIdx.z * nx * ny;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (x < nx && y < ny) {
            const size_t it = zoff + (size_t)x * ny + y;
            tile[j][threadIdx.x] = q ? (double)q[nvox + it] : (double)acc_t[it];
        }
    }
    __syncthreads();
    const double s = q ? inv[0] : 1.0;
    for (int j = threadIdx.y; j < kTile; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (x < nx && y < ny) {
            const size_t i = zoff + (size_t)y * nx + x;
            float val;
            if (q) val = (float)(((double)q[i] + tile[threadIdx.x][j]) * s);
            else   val = acc[i] + (float)tile[threadIdx.x][j];
            if (beta != 0.f) val = fmaf(beta, to_f(out[i]), val);
            out[i] = from_f<T>(val);
        }
    }
}

}  // namespace

ct_status launch_transpose_typed(const ProjGeom &pg, const void *v, void *t, int dt,
                                 cudaStream_t st) {
    if (pg.proj != CT_PROJ_SIDDON) return CT_OK;   // read in place
    if (pg.cm) {
        const dim3 gz = zfast_grid(pg), bz(kTile, 8);
        switch (dt) {
            case CT_F32:
                k_to_zfast<float><<<gz, bz, 0, st>>>(pg.nx, pg.ny, pg.nz, (const float *)v,
                                                     nullptr, (float *)t, nullptr);
                break;
            case CT_BF16:
                k_to_zfast<__nv_bfloat16><<<gz, bz, 0, st>>>(pg.nx, pg.ny, pg.nz,
                                                             (const __nv_bfloat16 *)v, nullptr,
                                                             (__nv_bfloat16 *)t, nullptr);
                break;
            case CT_F16:
                k_to_zfast<__half><<<gz, bz, 0, st>>>(pg.nx, pg.ny, pg.nz, (const __half *)v,
                                                      nullptr, (__half *)t, nullptr);
                break;
            default:
                return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
        }
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    dim3 gr((pg.nx + kTile - 1) / kTile, (pg.ny + kTile - 1) / kTile, pg.nz), bl(kTile, 8);
    switch (dt) {
        case CT_F32:
            k_transpose_t<float><<<gr, bl, 0, st>>>(pg.nx, pg.ny, (const float *)v, (float *)t);
            break;
        case CT_BF16:
            k_transpose_t<__nv_bfloat16><<<gr, bl, 0, st>>>(
                pg.nx, pg.ny, (const __nv_bfloat16 *)v, (__nv_bfloat16 *)t);
            break;
        case CT_F16:
            k_transpose_t<__half><<<gr, bl, 0, st>>>(pg.nx, pg.ny, (const __half *)v, (__half *)t);
            break;
        default:
            return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
    }
    CT_CHECK_LAUNCH();
    return CT_OK;
}

ct_status launch_combine_typed(const ProjGeom &pg, void *out, int dt, float beta, const float *acc,
                               const float *acc_t, const long long *q, const double *inv,
                               cudaStream_t st) {
    const int64_t n = (int64_t)pg.nx * pg.ny * pg.nz;
    if (pg.proj != CT_PROJ_SIDDON) {
        if (dt != CT_F32 || q)
            return set_error(CT_ERR_INVALID_ARG,
                             "footprint projectors need FP32 storage and float accumulation");
        return sf_axpby(static_cast<float *>(out), acc, n, beta, st);
    }
    if (pg.cm) {
        // the column-major backprojection accumulates into the second half
        const ZAcc za{acc_t, q ? q + n : nullptr, inv};
        switch (dt) {
            case CT_F32: return from_zfast<float>(pg, (float *)out, beta, za, nullptr, nullptr, st);
            case CT_BF16:
                return from_zfast<__nv_bfloat16>(pg, (__nv_bfloat16 *)out, beta, za, nullptr,
                                                 nullptr, st);
            case CT_F16: return from_zfast<__half>(pg, (__half *)out, beta, za, nullptr, nullptr, st);
            default: return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
        }
    }
    dim3 gr((pg.nx + kTile - 1) / kTile, (pg.ny + kTile - 1) / kTile, pg.nz), bl(kTile, 8);
    switch (dt) {
        case CT_F32:
            k_combine_t<float><<<gr, bl, 0, st>>>(pg.nx, pg.ny, n, (float *)out, beta, acc, acc_t, q, inv);
            break;
        case CT_BF16:
            k_combine_t<__nv_bfloat16><<<gr, bl, 0, st>>>(pg.nx, pg.ny, n, (__nv_bfloat16 *)out,
                                                          beta, acc, acc_t, q, inv);
            break;
        case CT_F16:
            k_combine_t<__half><<<gr, bl, 0, st>>>(pg.nx, pg.ny, n, (__half *)out, beta, acc,
                                                   acc_t, q, inv);
            break;
        default:
            return set_error(CT_ERR_INVALID_ARG, "unknown dtype");
    }
    CT_CHECK_LAUNCH();
    return CT_OK;
}

}  // namespace ct
