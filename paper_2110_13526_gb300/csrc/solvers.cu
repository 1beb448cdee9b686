// CGLS (Algorithm 1, CGLS with delayed residual computation) and LSQR
// (Paige & Saunders 1982) drivers.
//
// Vectors are FP32 in device memory; the Krylov scalars (NB0, NR2, NP2,
// alpha, beta, NB and LSQR's rotation scalars) live in device memory in FP64
// and are updated by one-CTA kernels that also finish the FP64 reductions, so
// the host never needs them inside the loop.  The host reads NB back only
// when a discrepancy tolerance ERR > 0 has to be tested.
//
// Preconditioning runs the unchanged recurrences on L A W (left ray weights
// L, right voxel weights W) with x = x0 + W y: the direction is kept in
// x-space, z = W d_y, so A is applied to z directly, and the weights are
// folded into the streaming kernels (L into the projector's epilogue and the
// backprojector's ray weight).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <memory>
#include <vector>

#include "ct_internal.h"
#include "ct_types.cuh"

namespace ct {
namespace {

__device__ __forceinline__ double block_sum(double x, double *sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// Fixed-order sum of partials by one CTA (1024 threads); result in thread 0.
// Four running sums per thread keep four loads in flight (A's 155520 CTA
// partials at 256^3 took 50 us one load at a time).
__device__ __forceinline__ double sum_partials(const double *__restrict__ p, int64_t n,
                                               double *sh) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const int64_t st = blockDim.x;
    int64_t i = threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {
        s0 += p[i];
        s1 += p[i + st];
        s2 += p[i + 2 * st];
        s3 += p[i + 3 * st];
    }
    for (; i < n; i += st) s0 += p[i];
    return block_sum((s0 + s1) + (s2 + s3), sh);
}

__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// First stage of a long partial sum: CTA b adds p[b chunk, (b + 1) chunk) in
// a fixed order into out[b].  One SM adds FP64 at about 4e9 per second on
// GB300, so A's 155520 CTA partials at 256^3 took 50 us in one CTA.
__global__ void __launch_bounds__(256) k_partials_stage(const double *__restrict__ p, int64_t n,
                                                        int64_t chunk, double *__restrict__ out) {
    __shared__ double sh[32];
    const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += p[i];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// Partial counts above this are first summed in chunks by k_partials_stage.
constexpr int64_t kStageMin = 8192;
constexpr int kStageMax = 256;   // CTAs (and second-stage partials) at most

// ---- CGLS ------------------------------------------------------------------
// zs: the direction is stored as z~ = zs z (zs a power of two, 1 in FP32
// storage) so that it fits BF16/FP16; the step alpha then applies to z~ and
// p~ = A z~ directly: alpha~ = NR2 zs / ||p~||^2.
struct CglsS {
    double nb0, nr2_old, nr2_now, np2, alpha, beta, nb, a_pend, tmp, zs;
    int it;   // next history slot (k_cgls_nb with i < 0)
};

// A CGLS state between two updates (checkpoint / resume, FP32 storage): x
// before its pending step alpha d_x, d_x, e_b and the FP64 scalars on the
// device, the history on the host.  Device buffers are owned here.
struct CglsCkpt {
    int device = 0;
    int64_t n = 0, m = 0;
    float *x = nullptr, *z = nullptr, *e = nullptr;
    CglsS *s = nullptr;
    std::vector<double> hist;      // NB / NB0 after each update
    std::vector<double> hist_nr;   // ||r_x|| before each update
    int i = 0;   // updates done
};

// NB0 and NB of a finished solve must be finite: NaN or Inf in b (or x0)
// propagates into every later value, and is reported instead of returned as
// a result.
ct_status finite_or_error(double nb0, double nb) {
    if (!std::isfinite(nb0))
        return set_error(CT_ERR_INVALID_ARG, "b holds non-finite values (NaN or Inf): ||b|| = " +
                                                 std::to_string(nb0));
    if (!std::isfinite(nb))
        return set_error(CT_ERR_INVALID_ARG,
                         "the discrepancy became non-finite: x0 or b hold NaN or Inf, or the "
                         "data overflow FP32");
    return CT_OK;
}

// e = L o b, stored as S; partial sums of the stored e^2 (one per CTA).
template <class S>
__global__ void k_sino_weighted_copy(S *__restrict__ e, const float *__restrict__ b,
                                     const float *__restrict__ L, int64_t n,
                                     double *__restrict__ part) {
    __shared__ double sh[32];
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const S v = from_f<S>(L ? L[i] * b[i] : b[i]);
        e[i] = v;
        sq.add(to_f(v));
    }
    const double t = block_sum(sq.value(), sh);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = t;
}

// e_b = e_b - alpha p_b; partial sums of e_b^2 (Algorithm 1: NB = ||e_b||).
template <class S>
__global__ void k_sino_axpy(S *__restrict__ e, const S *__restrict__ p, int64_t n,
                            const double *__restrict__ alpha, double *__restrict__ part) {
    __shared__ double sh[32];
    const float a = (float)alpha[0];
    SqSum sq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // four elements per pass: their loads are in flight together
    for (; i + 3 * stride < n; i += 4 * stride) {
        float ev[4], pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ev[k] = to_f(e[i + k * stride]);
            pv[k] = to_f(p[i + k * stride]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const S v = from_f<S>(fmaf(-a, pv[k], ev[k]));
            e[i + k * stride] = v;
            sq.add(to_f(v));
        }
    }
    for (; i < n; i += stride) {
        const S v = from_f<S>(fmaf(-a, to_f(p[i]), to_f(e[i])));
        e[i] = v;
        sq.add(to_f(v));
    }
    const double t = block_sum(sq.value(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// partial sums of v^2 (one per CTA)
template <class S>
__global__ void k_norm2_t(const S *__restrict__ v, int64_t n, double *__restrict__ part) {
    __shared__ double sh[32];
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        sq.add(to_f(v[i]));
    const double t = block_sum(sq.value(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// x = x + a_pend z (the x update delayed from the previous iteration), then
// z = W^2 g + beta z (d_x = r_x + beta d_x in y-space, stored as z = W d).
// first: z = W^2 g, neither x nor the old z is read.  x stays FP32; z is
// stored as S.
// zpart (may be NULL): partial sums of the stored z^2, one per CTA (the
// lam ||z||^2 term of NP2 with Tikhonov regularisation).
template <class S, bool ZNORM>
__global__ void k_vol_update(float *__restrict__ x, S *__restrict__ z,
                             const float *__restrict__ g, const float *__restrict__ W, int64_t n,
                             const double *__restrict__ a_pend, const double *__restrict__ beta,
                             const double *__restrict__ zs, int first,
                             double *__restrict__ zpart) {
    __shared__ double sh[32];
    const float a = first ? 0.f : (float)a_pend[0];
    const float b = first ? 0.f : (float)beta[0];
    const float gs = (float)zs[0];
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float r = g[i] * gs;
        if (W) {
            const float w = W[i];
            r *= w * w;
        }
        S zn;
        if (first) {
            zn = from_f<S>(r);
        } else {
            const float zo = to_f(z[i]);
            if (a != 0.f) x[i] = fmaf(a, zo, x[i]);
            zn = from_f<S>(fmaf(b, zo, r));
        }
        z[i] = zn;
        if (ZNORM) sq.add(to_f(zn));
    }
    if (ZNORM) {
        const double t = block_sum(sq.value(), sh);
        if (threadIdx.x == 0) zpart[blockIdx.x] = t;
    }
}

// Tikhonov term of the gradient: g = g - lam x_cur, x_cur = x + a_pend z (the
// x update still pending from the previous iteration, exactly as
// k_vol_update will apply it; first: x_cur = x and z is not read), with
// partial sums of (W g)^2 (NR2).
template <class S>
__global__ void k_tikhonov_grad(float *__restrict__ g, const float *__restrict__ x,
                                const S *__restrict__ z, const float *__restrict__ W, int64_t n,
                                const double *__restrict__ a_pend, double lam, int first,
                                double *__restrict__ part) {
    __shared__ double sh[32];
    const float a = first ? 0.f : (float)a_pend[0];
    const float l = (float)lam;
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float xc = x[i];
        if (!first && a != 0.f) xc = fmaf(a, to_f(z[i]), xc);
        const float gi = fmaf(-l, xc, g[i]);
        g[i] = gi;
        sq.add(W ? W[i] * gi : gi);
    }
    const double t = block_sum(sq.value(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <class S>
__global__ void k_vol_axpy(float *__restrict__ x, const S *__restrict__ z, int64_t n,
                           const double *__restrict__ a) {
    const float s = (float)a[0];
    if (s == 0.f) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fmaf(s, to_f(z[i]), x[i]);
}

__global__ void __launch_bounds__(1024) k_cgls_nb0(const double *__restrict__ p, int64_t n,
                                                   CglsS *S) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        S->nb0 = sqrt(t);
        S->a_pend = 0.0;
        S->beta = 0.0;
        S->alpha = 0.0;
        S->zs = 1.0;
    }
}

__global__ void __launch_bounds__(1024) k_store_sum(const double *__restrict__ p, int64_t n,
                                                    double *out) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) out[0] = t;
}

// NR2_now = ||r_x||^2; beta = NR2_now / NR2_old; NR2_old = NR2_now.  With
// maxpart (the block maxima of |W^2 g|), the new direction scale zs puts
// max |zs W^2 g| in [1/2, 1) and beta absorbs the ratio to the old scale.
__global__ void __launch_bounds__(1024) k_cgls_nr2(const double *__restrict__ p, int64_t n,
                                                   CglsS *S, int first,
                                                   const float *__restrict__ maxpart, int nmax) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        double zs = 1.0;
        if (maxpart) {
            float mx = 0.f;
            for (int i = 0; i < nmax; ++i) mx = fmaxf(mx, maxpart[i]);
            if (mx > 0.f && mx < 3.0e38f) {
                int ex = 0;
                (void)frexp((double)mx, &ex);
                zs = ldexp(1.0, -ex);
            }
        }
        const double zs_old = first ? zs : S->zs;
        S->nr2_now = t;
        S->beta = first ? 0.0 : safe_div(t, S->nr2_old) * (zs / zs_old);
        S->nr2_old = t;
        S->zs = zs;
    }
}

// Block maxima of |W^2 g| (W NULL: |g|).
__global__ void k_absmax_w2g(const float *__restrict__ g, const float *__restrict__ W, int64_t n,
                             float *__restrict__ part) {
    __shared__ float sh[32];
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float r = g[i];
        if (W) r *= W[i] * W[i];
        m = fmaxf(m, fabsf(r));
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

// NP2 = ||p_b||^2 (+ lam ||z||^2 from zp, the partials of z^2, with
// Tikhonov regularisation); alpha = NR2_old / NP2 (also the pending x step).
__global__ void __launch_bounds__(1024) k_cgls_np2(const double *__restrict__ p, int64_t n,
                                                   CglsS *S, const double *__restrict__ zp,
                                                   int64_t nz, double lam) {
    __shared__ double sh[32];
    double t = sum_partials(p, n, sh);
    if (zp) {
        __syncthreads();   // sh is reused
        const double tz = sum_partials(zp, nz, sh);
        t += lam * tz;
    }
    if (threadIdx.x == 0) {
        S->np2 = t;
        S->alpha = safe_div(S->nr2_old * S->zs, t);
        S->a_pend = S->alpha;
    }
}

// NB = ||e_b||; history[i] = NB / NB0 and (hist_nr not NULL) hist_nr[i] =
// NR = ||r_x|| of the update, the gradient norm at the iterate before it.
__global__ void __launch_bounds__(1024) k_cgls_nb(const double *__restrict__ p, int64_t n,
                                                  CglsS *S, double *hist, int i,
                                                  double *hist_nr) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        S->nb = sqrt(t);
        const int k = i >= 0 ? i : S->it++;   // i < 0: the slot counter on the device
        hist[k] = safe_div(S->nb, S->nb0);
        if (hist_nr) hist_nr[k] = sqrt(S->nr2_old);
    }
}

__global__ void k_set_zero(double *p) { p[0] = 0.0; }

// ---- SIRT / PSIRT --------------------------------------------------------------
// v = v * v (guarded R^-1/2 -> R^-1; zeros stay zero).
__global__ void k_square(float *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = v[i] * v[i];
}

// x = x + relax * Cinv o g.
__global__ void k_sirt_update(float *__restrict__ x, const float *__restrict__ g,
                              const float *__restrict__ cinv, int64_t n, float relax) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fmaf(relax * cinv[i], g[i], x[i]);
}

// ---- LSQR ------------------------------------------------------------------
struct LsqrS {
    double nb0, alpha, beta, inv_beta, inv_alpha, rhobar, phibar, x_step, w_step, tmp;
    double nrb;           // ||A^T r|| estimate at the current iterate (phibar alpha |c|)
    double coef_fwd[2];   // projector epilogue: u = 1 * L A t - alpha / beta_old * u
    double coef_back[2];  // backprojector scale: 1 / beta
    int it;               // next history slot (k_lsqr_rot with i < 0)
};

__global__ void __launch_bounds__(1024) k_lsqr_nb0(const double *__restrict__ p, int64_t n,
                                                   LsqrS *S) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) S->nb0 = sqrt(t);
}

// beta u = A v - alpha u: beta = ||u_s||, u = u_s / beta (kept as a scale).
__global__ void __launch_bounds__(1024) k_lsqr_beta(const double *__restrict__ p, int64_t n,
                                                    LsqrS *S) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        S->beta = sqrt(t);
        S->inv_beta = safe_div(1.0, S->beta);
        S->coef_back[0] = S->inv_beta;
        S->coef_back[1] = 0.0;
    }
}

// alpha_1 = ||W A^T u_1||; rhobar = alpha_1; phibar = beta_1.
__global__ void __launch_bounds__(1024) k_lsqr_alpha0(const double *__restrict__ p, int64_t n,
                                                      LsqrS *S) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        S->alpha = sqrt(t);
        S->inv_alpha = safe_div(1.0, S->alpha);
        S->rhobar = S->alpha;
        S->phibar = S->beta;
        S->nrb = S->alpha * S->beta;   // ||A^T r_0|| = alpha_1 beta_1
    }
}

__global__ void k_lsqr_coef_fwd(LsqrS *S) {
    S->coef_fwd[0] = 1.0;
    S->coef_fwd[1] = -S->alpha * S->inv_beta;
}

// v = W g / alpha; w = v.
__global__ void k_lsqr_vinit(float *__restrict__ v, float *__restrict__ wv,
                             const float *__restrict__ g, const float *__restrict__ W, int64_t n,
                             const LsqrS *__restrict__ S) {
    const float ia = (float)S->inv_alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float t = g[i] * ia;
        if (W) t *= W[i];
        v[i] = t;
        wv[i] = t;
    }
}

// alpha v = A^T u - beta v: v_s = W g - beta v (v normalised); partial ||v_s||^2.
__global__ void k_lsqr_v(float *__restrict__ v, const float *__restrict__ g,
                         const float *__restrict__ W, int64_t n, const LsqrS *__restrict__ S,
                         double *__restrict__ part) {
    __shared__ double sh[32];
    const float b = (float)S->beta;
    SqSum sq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float t = g[i];
        if (W) t *= W[i];
        t = fmaf(-b, v[i], t);
        v[i] = t;
        sq.add(t);
    }
    const double t = block_sum(sq.value(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Plane rotation of the bidiagonal (Paige & Saunders): rho, c, s, theta,
// rhobar, phi, phibar; history[i] = phibar / NB0, hist_nr[i] = the estimate
// of ||A^T r|| before this update, and the estimate after it,
// phibar_{k+1} alpha_{k+1} |c_k|, is kept for the next one.
__global__ void __launch_bounds__(1024) k_lsqr_rot(const double *__restrict__ p, int64_t n,
                                                   LsqrS *S, double *hist, int i,
                                                   double *hist_nr) {
    __shared__ double sh[32];
    const double t = sum_partials(p, n, sh);
    if (threadIdx.x == 0) {
        const double alpha = sqrt(t);
        const double beta = S->beta;
        const double rho = sqrt(S->rhobar * S->rhobar + beta * beta);
        const double c = rho != 0.0 ? S->rhobar / rho : 1.0;
        const double s = rho != 0.0 ? beta / rho : 0.0;
        const double theta = s * alpha;
        S->rhobar = -c * alpha;
        const double phi = c * S->phibar;
        S->phibar = s * S->phibar;
        S->x_step = safe_div(phi, rho);
        S->w_step = safe_div(theta, rho);
        S->alpha = alpha;
        S->inv_alpha = safe_div(1.0, alpha);
        const int k = i >= 0 ? i : S->it++;   // i < 0: the slot counter on the device
        hist[k] = safe_div(S->phibar, S->nb0);
        if (hist_nr) hist_nr[k] = S->nrb;
        S->nrb = S->phibar * alpha * fabs(c);
    }
}

// v = v_s / alpha; x += (phi / rho) W w; w = v - (theta / rho) w.
__global__ void k_lsqr_update(float *__restrict__ x, float *__restrict__ v, float *__restrict__ wv,
                              const float *__restrict__ W, int64_t n,
                              const LsqrS *__restrict__ S) {
    const float ia = (float)S->inv_alpha, xs = (float)S->x_step, ws = (float)S->w_step;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float vn = v[i] * ia;
        const float wo = wv[i];
        const float step = W ? xs * W[i] : xs;
        x[i] = fmaf(step, wo, x[i]);
        v[i] = vn;
        wv[i] = fmaf(-ws, wo, vn);
    }
}

// ---- helpers -----------------------------------------------------------------
struct OpTimer {
    bool on;
    cudaStream_t st;
    std::vector<cudaEvent_t> fwd, back;
    OpTimer(bool enabled, cudaStream_t s) : on(enabled), st(s) {}
    ~OpTimer() {
        for (auto e : fwd) cudaEventDestroy(e);
        for (auto e : back) cudaEventDestroy(e);
    }
    ct_status mark(std::vector<cudaEvent_t> &v) {
        if (!on) return CT_OK;
        cudaEvent_t e;
        CT_CUDA_TRY(cudaEventCreate(&e));
        v.push_back(e);
        CT_CUDA_TRY(cudaEventRecord(e, st));
        return CT_OK;
    }
    double total(const std::vector<cudaEvent_t> &v) const {
        double ms = 0.0;
        for (size_t k = 0; k + 1 < v.size(); k += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, v[k], v[k + 1]) == cudaSuccess) ms += t;
        }
        return ms;
    }
};

ct_status check_opts(const ct_geometry *g, const float *b, float *x, const ct_solver_opts *o) {
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    if (!o) return set_error(CT_ERR_INVALID_ARG, "opts is NULL");
    if (!x || (g->nrays > 0 && !b)) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (o->max_iter < 1) return set_error(CT_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!std::isfinite(o->err_tol) || o->err_tol < 0.0)
        return set_error(CT_ERR_INVALID_ARG, "err_tol must be finite and >= 0");
    if (o->precond != CT_PRECOND_NONE && o->precond != CT_PRECOND_JACOBI &&
        o->precond != CT_PRECOND_ROWCOL)
        return set_error(CT_ERR_INVALID_ARG, "unknown precond");
    if (!std::isfinite(o->tikhonov_lambda) || o->tikhonov_lambda < 0.0)
        return set_error(CT_ERR_INVALID_ARG, "tikhonov_lambda must be finite and >= 0");
    if (o->recompute_every < 0) return set_error(CT_ERR_INVALID_ARG, "recompute_every < 0");
    if (dtype_size(o->storage) == 0) return set_error(CT_ERR_INVALID_ARG, "unknown storage dtype");
    if (g->pg.proj != CT_PROJ_SIDDON && o->storage != CT_F32)
        return set_error(CT_ERR_INVALID_ARG, "footprint projectors need FP32 storage");
    return CT_OK;
}

// Common state of one solve: workspace vectors, weights, timing, op counts.
struct Solve {
    const ct_geometry *g;
    ProjGeom pg;                  // g's, with the scratch of this solve's projections
    cudaStream_t st;
    Workspace ws;
    OpTimer tm;
    int n_fwd = 0, n_back = 0;
    float *T = nullptr;           // transposed scratch volume (input copy / accumulator)
    BackScratch bs;               // backprojection scratch (T, or int64 accumulators)
    double *part = nullptr;       // FP64 partial sums
    double *part2 = nullptr;      // their first-stage sums (reduce)
    float *W = nullptr, *L = nullptr;
    int64_t n, m;
    Solve(const ct_geometry *g_, cudaStream_t s, bool timing)
        : g(g_), pg(g_->pg), st(s), ws(s), tm(timing, s), n(g_->nvox), m(g_->nrays) {}

    ct_status init(int precond) {
        CT_TRY(ws.alloc(&T, (size_t)n));
        CT_TRY(back_scratch_alloc(g, ws, T, &bs));
        if (pg.sf_det) CT_TRY(ws.alloc(&pg.sf_ws, sf_det_ws_bytes(pg)));
        int64_t np = std::max<int64_t>(forward_partials(pg), transpose_grid_count(pg));
        np = std::max<int64_t>(np, std::max(vec_grid(n), vec_grid(m)));
        CT_TRY(ws.alloc(&part, (size_t)np));
        CT_TRY(ws.alloc(&part2, (size_t)kStageMax));
        if (precond != CT_PRECOND_NONE) {
            CT_TRY(ws.alloc(&W, (size_t)n));
            if (precond == CT_PRECOND_ROWCOL) CT_TRY(ws.alloc(&L, (size_t)std::max<int64_t>(m, 1)));
            CT_TRY(precond_weights_impl(g, precond, W, L, ws, st));
        }
        return CT_OK;
    }
    // out = c.alpha * L o (A vol) + c.beta * out (vol_main may already be
    // accompanied by its transposed copy in T when have_t).
    ct_status forward(const float *vol, bool have_t, float *out, Coef c, double *partials) {
        if (!have_t) CT_TRY(launch_transpose(pg, vol, nullptr, T, nullptr, st));
        CT_TRY(tm.mark(tm.fwd));
        CT_TRY(launch_forward(pg, vol, T, out, L, c, partials, st));
        CT_TRY(tm.mark(tm.fwd));
        ++n_fwd;
        return CT_OK;
    }
    // out (sdt) = c.alpha * L o (A vol (vdt)) + c.beta * out; tbuf receives the
    // transposed copy of vol (same dtype) first.  In two parts, so that a
    // batched step can launch the projectors of several solves together:
    // fwd_pre writes the copy, fwd_proj projects.
    ct_status fwd_pre(const void *vol, int vdt, void *tbuf) {
        return launch_transpose_typed(pg, vol, tbuf, vdt, st);
    }
    ct_status fwd_proj(const void *vol, int vdt, const void *tbuf, void *out, int sdt, Coef c,
                       double *partials) {
        CT_TRY(tm.mark(tm.fwd));
        CT_TRY(launch_forward_typed(pg, vol, tbuf, vdt, out, sdt, L, c, partials, st));
        CT_TRY(tm.mark(tm.fwd));
        ++n_fwd;
        return CT_OK;
    }
    ct_status forward_t(const void *vol, int vdt, void *tbuf, void *out, int sdt, Coef c,
                        double *partials) {
        CT_TRY(fwd_pre(vol, vdt, tbuf));
        return fwd_proj(vol, vdt, tbuf, out, sdt, c, partials);
    }
    // fwd_proj of FP32 vectors as a job of a batched launch (batchable(pg)).
    ct_status fwd_job(const float *tbuf, float *out, Coef c, double *partials, BatchJob *b) const {
        CT_TRY(batch_job_grid(pg, false, b));
        b->in = tbuf;
        b->out = out;
        b->rho = L;
        b->c = c;
        b->partials = partials;
        b->det_scale = nullptr;
        return CT_OK;
    }
    // gout = c * A^T (L o e) (e of dtype edt), then partials of (Wg)^2 if
    // requested; the geometry decides float-atomic or fixed-point
    // (deterministic) sums.  In three parts: back_pre clears the accumulators
    // (and finds the fixed-point scale), back_proj scatters, back_post
    // combines them into gout.
    // Column-major Siddon kernels accumulate A^T in T only; their combine
    // then overwrites gout (beta 0) instead of adding to a cleared one.
    bool zfast_only() const { return pg.proj == CT_PROJ_SIDDON && pg.cm; }
    ct_status back_pre(const void *e, int edt, float *gout, Coef c) {
        if (!fixed_back(g)) {
            if (!zfast_only())
                CT_CUDA_TRY(cudaMemsetAsync(gout, 0, (size_t)n * sizeof(float), st));
            CT_CUDA_TRY(cudaMemsetAsync(T, 0, (size_t)n * sizeof(float), st));
            return CT_OK;
        }
        CT_CUDA_TRY(cudaMemsetAsync(bs.q, 0, 2 * (size_t)n * sizeof(long long), st));
        return launch_det_scale(e, edt, L, m, det_value_bound(g, 1), c, bs.part, bs.scale,
                                bs.inv, st);
    }
    ct_status back_proj(const void *e, int edt, float *gout, Coef c) {
        CT_TRY(tm.mark(tm.back));
        if (!fixed_back(g))
            CT_TRY(launch_backward_typed(pg, e, edt, L, c, gout, T, 1, false, nullptr, st));
        else
            CT_TRY(launch_backward_typed(pg, e, edt, L, c, bs.q, bs.q + n, 1, true, bs.scale, st));
        CT_TRY(tm.mark(tm.back));
        ++n_back;
        return CT_OK;
    }
    ct_status back_post(float *gout, const float *wnorm, double *partials) {
        if (!fixed_back(g))
            return launch_combine(pg, gout, T, wnorm, partials, st, zfast_only() ? 0.f : 1.f);
        return launch_combine_det(pg, gout, 0.f, bs.q, bs.q + n, bs.inv, wnorm, partials, st);
    }
    ct_status back_t(const void *e, int edt, float *gout, Coef c, const float *wnorm,
                     double *partials) {
        CT_TRY(back_pre(e, edt, gout, c));
        CT_TRY(back_proj(e, edt, gout, c));
        return back_post(gout, wnorm, partials);
    }
    // back_proj of an FP32 e as a job of a batched launch (batchable(pg)); the
    // column-major kernels accumulate into the [y][x][z] buffer only.
    ct_status back_job(const float *e, Coef c, BatchJob *b) const {
        CT_TRY(batch_job_grid(pg, true, b));
        b->in = e;
        b->out = fixed_back(g) ? static_cast<void *>(bs.q + n) : static_cast<void *>(T);
        b->rho = L;
        b->c = c;
        b->partials = nullptr;
        b->det_scale = fixed_back(g) ? bs.scale : nullptr;
        return CT_OK;
    }
    ct_status back(const float *e, float *gout, Coef c, const float *wnorm, double *partials) {
        return back_t(e, CT_F32, gout, c, wnorm, partials);
    }
    // The partials p[0, n) a one-CTA scalar kernel will sum: long lists are
    // first summed in fixed chunks (k_partials_stage); *pp, *np: what to sum.
    ct_status reduce(const double *p, int64_t n, const double **pp, int64_t *np) {
        *pp = p;
        *np = n;
        if (n <= kStageMin) return CT_OK;
        const int64_t blocks = std::min<int64_t>(kStageMax, (n + 1023) / 1024);
        const int64_t chunk = (n + blocks - 1) / blocks;
        const int64_t used = (n + chunk - 1) / chunk;
        k_partials_stage<<<(unsigned)used, 256, 0, st>>>(p, n, chunk, part2);
        CT_CHECK_LAUNCH();
        *pp = part2;
        *np = used;
        return CT_OK;
    }
    // Is x0 nonzero?  (One reduction and one host read.)
    ct_status nonzero(const float *x, bool *out) {
        CT_TRY(launch_norm2(x, nullptr, n, part, st));
        double *d = nullptr;
        CT_TRY(ws.alloc(&d, 1));
        k_store_sum<<<1, 1024, 0, st>>>(part, vec_grid(n), d);
        CT_CHECK_LAUNCH();
        double h = 0.0;
        CT_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, st));
        CT_CUDA_TRY(cudaStreamSynchronize(st));
        *out = (h != 0.0);
        return CT_OK;
    }
    void report(ct_solver_report *r, int iters, double nb0, double nb, const std::vector<double> &h,
                const std::vector<double> *h_nr = nullptr) {
        if (!r) return;
        r->iterations = iters;
        r->nb0 = nb0;
        r->nb = nb;
        r->n_forward = n_fwd;
        r->n_back = n_back;
        r->ms_forward = tm.on ? tm.total(tm.fwd) : 0.0;
        r->ms_back = tm.on ? tm.total(tm.back) : 0.0;
        if (r->history_nb && r->history_cap > 0) {
            const int k = std::min<int>(iters, r->history_cap);
            for (int j = 0; j < k; ++j) r->history_nb[j] = h[(size_t)j];
        }
        if (r->history_nr && h_nr && r->history_cap > 0) {
            const int k = std::min<int>(std::min<int>(iters, r->history_cap), (int)h_nr->size());
            for (int j = 0; j < k; ++j) r->history_nr[j] = (*h_nr)[(size_t)j];
        }
    }
};

template <class S>
ct_status read_scalars(const S *d, S *h, cudaStream_t st) {
    CT_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(S), cudaMemcpyDeviceToHost, st));
    CT_CUDA_TRY(cudaStreamSynchronize(st));
    return CT_OK;
}


// One solver update as a CUDA graph: captured once on a private stream
// (the caller's stream may be the legacy default stream, which cannot
// capture), then replayed on the solve's stream, one graph launch per update.
struct UpdateGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;  // stream of the last replay (may be the legacy stream)
    bool launched = false;
    long long nk = 0;             // kernels per replay (ct_kernel_launches)
    UpdateGraph() = default;
    UpdateGraph(const UpdateGraph &) = delete;
    UpdateGraph &operator=(const UpdateGraph &) = delete;
    ~UpdateGraph() {
        if (launched) cudaStreamSynchronize(last);   // replays finish before the graph goes
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
    }
    // body() enqueues one update on the stream(s) that set_stream(s) points
    // at (the capture stream meanwhile, the original one afterwards).
    // Nothing runs during capture, so the kernels it counted are taken back
    // from ct_kernel_launches and added again per replay.
    template <class F>
    ct_status capture(F &&body, cudaStream_t *sref) {
        const cudaStream_t saved = *sref;
        return capture(body, [&](cudaStream_t s) { *sref = s ? s : saved; });
    }
    template <class F, class G>
    ct_status capture(F &&body, G &&set_stream) {
        CT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const long long k0 = thread_launches();
        CT_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        set_stream(cs);
        const ct_status sb = body();
        set_stream(nullptr);
        cudaGraph_t gr = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &gr);
        nk = thread_launches() - k0;
        note_launches(-nk);
        if (sb != CT_OK) {
            if (gr) cudaGraphDestroy(gr);
            return sb;
        }
        if (ec != cudaSuccess) return cuda_error(ec, "cudaStreamEndCapture");
        g = gr;
        CT_CUDA_TRY(cudaGraphInstantiate(&exec, g, 0));
        return CT_OK;
    }
    ct_status launch(cudaStream_t st) {
        CT_CUDA_TRY(cudaGraphLaunch(exec, st));
        last = st;
        launched = true;
        note_launches(nk);
        return CT_OK;
    }
};

// The state of one CGLS solve (Algorithm 1) and its steps.  ct_cgls runs
// one of these to the end; a ct_batch advances several together, launching
// their projectors as one batched kernel (the phases of update() below).
template <class ST>
struct CglsJob {
    const float *b;
    float *x;
    ct_solver_opts o;
    Solve sv;
    int sd, K;
    double ERR, lam;
    int64_t n, m;
    int gn = 0, gm = 0;
    int64_t nfp = 0, ncp = 0, nrp = 0;
    ST *z = nullptr, *e = nullptr, *p = nullptr;
    float *gv = nullptr;
    void *Ts = nullptr;          // transposed copy of z (the float scratch T when ST is float)
    float *mxp = nullptr;        // block maxima of |W^2 g| (direction scaling, reduced storage)
    CglsS *S = nullptr;
    double *hist = nullptr;
    double *zpart = nullptr;     // partials of ||z||^2 for NP2 (Tikhonov)
    Coef one, sub;               // (1, 0) and (-1, 1): e = e - L A x
    int i = 0;                   // updates done
    CglsS hs{};

    CglsJob(const ct_geometry *g, const float *b_, float *x_, const ct_solver_opts *o_,
            cudaStream_t st)
        : b(b_), x(x_), o(*o_), sv(g, st, o_->timing != 0), sd(o_->storage), K(o_->max_iter),
          ERR(o_->err_tol), lam(o_->tikhonov_lambda), n(g->nvox), m(g->nrays) {
        sub.alpha = -1.f;
        sub.beta = 1.f;
    }

    // x = x + alpha d_x (delayed); d_x = r_x + beta d_x (+ ||d_x||^2 partials)
    ct_status vol_update(int first) {
        const cudaStream_t s = sv.st;
        if (zpart)
            k_vol_update<ST, true><<<gn, kVecThreads, 0, s>>>(x, z, gv, sv.W, n, &S->a_pend,
                                                              &S->beta, &S->zs, first, zpart);
        else
            k_vol_update<ST, false><<<gn, kVecThreads, 0, s>>>(x, z, gv, sv.W, n, &S->a_pend,
                                                               &S->beta, &S->zs, first, nullptr);
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    // r_x = A^T e_b (- lam x) into gv and the NR2 partials into sv.part, in
    // the three parts of Solve::back_t; nrp = the partials' count.
    ct_status grad_pre() { return sv.back_pre(e, sd, gv, Coef()); }
    ct_status grad_proj() { return sv.back_proj(e, sd, gv, Coef()); }
    ct_status grad_post(int first) {
        if (lam == 0.0) {
            CT_TRY(sv.back_post(gv, sv.W, sv.part));
            nrp = ncp;
            return CT_OK;
        }
        CT_TRY(sv.back_post(gv, sv.W, nullptr));
        k_tikhonov_grad<<<gn, kVecThreads, 0, sv.st>>>(gv, x, z, sv.W, n, &S->a_pend, lam, first,
                                                       sv.part);
        CT_CHECK_LAUNCH();
        nrp = gn;
        return CT_OK;
    }
    // NR2 and beta, then x += alpha_prev d_x; d_x = r_x + beta d_x, then the
    // transposed copy of d_x for A.
    ct_status middle(int first) {
        const cudaStream_t s = sv.st;
        if (mxp) {
            k_absmax_w2g<<<gn, kVecThreads, 0, s>>>(gv, sv.W, n, mxp);
            CT_CHECK_LAUNCH();
        }
        k_cgls_nr2<<<1, 1024, 0, s>>>(sv.part, nrp, S, first, mxp, gn);
        CT_CHECK_LAUNCH();
        CT_TRY(vol_update(first));
        return sv.fwd_pre(z, sd, Ts);
    }
    // p_b = A d_x with the NP2 partials
    ct_status fwd_proj() { return sv.fwd_proj(z, sd, Ts, p, sd, one, sv.part); }
    // NP2 (+ lam ||d_x||^2), alpha; e_b = e_b - alpha p_b with the NB partials
    ct_status tail() {
        const cudaStream_t s = sv.st;
        const double *pp = nullptr;
        int64_t np = 0;
        CT_TRY(sv.reduce(sv.part, nfp, &pp, &np));
        k_cgls_np2<<<1, 1024, 0, s>>>(pp, np, S, zpart, gn, lam);
        CT_CHECK_LAUNCH();
        k_sino_axpy<<<gm, kVecThreads, 0, s>>>(e, p, m, &S->alpha, sv.part);
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    // NB = ||e_b|| into S and the history
    ct_status finish() {
        k_cgls_nb<<<1, 1024, 0, sv.st>>>(sv.part, gm, S, hist, -1, hist + K);
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    // One x update after the first; ends with the NB partials in sv.part.
    ct_status update() {
        CT_TRY(grad_pre());
        CT_TRY(grad_proj());
        CT_TRY(grad_post(0));
        CT_TRY(middle(0));
        CT_TRY(fwd_proj());
        return tail();
    }
    // The batched launch descriptors of grad_proj and fwd_proj (FP32 storage).
    ct_status back_job(BatchJob *bj) const {
        return sv.back_job(reinterpret_cast<const float *>(e), Coef(), bj);
    }
    ct_status fwd_job(BatchJob *bj) const {
        return sv.fwd_job(static_cast<const float *>(Ts), reinterpret_cast<float *>(p), one,
                          sv.part, bj);
    }

    // Allocations, NB0, and the first update (i = 1).
    ct_status start() {
        CT_TRY(alloc());
        return first();
    }
    // The solve's weights and vectors.
    ct_status alloc() {
        CT_TRY(sv.init(o.precond));
        const cudaStream_t st = sv.st;
        gn = vec_grid(n);
        gm = vec_grid(m);
        nfp = forward_partials(sv.pg);
        ncp = transpose_grid_count(sv.pg);
        CT_TRY(sv.ws.alloc(&z, (size_t)n));
        CT_TRY(sv.ws.alloc(&gv, (size_t)n));
        if (sd == CT_F32) {
            Ts = sv.T;
        } else {
            CT_TRY(sv.ws.alloc(&mxp, (size_t)gn));
            ST *t = nullptr;
            CT_TRY(sv.ws.alloc(&t, (size_t)n));
            Ts = t;
        }
        CT_TRY(sv.ws.alloc(&e, (size_t)std::max<int64_t>(m, 1)));
        CT_TRY(sv.ws.alloc(&p, (size_t)std::max<int64_t>(m, 1)));
        CT_TRY(sv.ws.alloc(&S, 1));
        CT_TRY(sv.ws.alloc(&hist, 2 * (size_t)K));   // NB / NB0, then NR, per update
        CT_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(CglsS), st));
        // Tikhonov regularisation (Software section): minimise
        // ||L (A x - b)||^2 + lam ||x||^2, Algorithm 1 on [L A W; sqrt(lam) W]
        if (lam > 0.0) CT_TRY(sv.ws.alloc(&zpart, (size_t)gn));
        return CT_OK;
    }
    ct_status first() {
        const cudaStream_t st = sv.st;
        // NB0 = ||b||; e_b = b - A x0 (the A x0 call is skipped for x0 = 0)
        bool x0nz = false;
        CT_TRY(sv.nonzero(x, &x0nz));
        k_sino_weighted_copy<<<gm, kVecThreads, 0, st>>>(e, b, sv.L, m, sv.part);
        CT_CHECK_LAUNCH();
        k_cgls_nb0<<<1, 1024, 0, st>>>(sv.part, gm, S);
        CT_CHECK_LAUNCH();
        if (x0nz) CT_TRY(sv.forward_t(x, CT_F32, sv.T, e, sd, sub, nullptr));
        // r_x = A^T e_b (- lam x); d_x = r_x; NR2_old = ||r_x||^2
        CT_TRY(grad_pre());
        CT_TRY(grad_proj());
        CT_TRY(grad_post(1));
        CT_TRY(middle(1));
        // p_b = A d_x; NP2 (+ lam ||d_x||^2); alpha
        // (x = x + alpha d_x is delayed into the next volume update)
        // e_b = e_b - alpha p_b; NB = ||e_b||
        CT_TRY(fwd_proj());
        CT_TRY(tail());
        CT_TRY(finish());
        i = 1;
        return CT_OK;
    }
    // Continue a solve from a saved state (x before its pending step, d_x, e_b,
    // the scalars and the history; FP32 storage): the next update is i + 1.
    ct_status resume(const CglsCkpt &c) {
        CT_TRY(alloc());
        const cudaStream_t st = sv.st;
        const size_t nb = (size_t)n * sizeof(float), mb = (size_t)m * sizeof(float);
        CT_CUDA_TRY(cudaMemcpyAsync(x, c.x, nb, cudaMemcpyDeviceToDevice, st));
        CT_CUDA_TRY(cudaMemcpyAsync(z, c.z, nb, cudaMemcpyDeviceToDevice, st));
        if (m > 0) CT_CUDA_TRY(cudaMemcpyAsync(e, c.e, mb, cudaMemcpyDeviceToDevice, st));
        CT_CUDA_TRY(cudaMemcpyAsync(S, c.s, sizeof(CglsS), cudaMemcpyDeviceToDevice, st));
        const int keep = std::min(c.i, K);
        if (keep > 0) {
            CT_CUDA_TRY(cudaMemcpyAsync(hist, c.hist.data(), sizeof(double) * (size_t)keep,
                                        cudaMemcpyHostToDevice, st));
            CT_CUDA_TRY(cudaMemcpyAsync(hist + K, c.hist_nr.data(), sizeof(double) * (size_t)keep,
                                        cudaMemcpyHostToDevice, st));
        }
        i = c.i;
        return CT_OK;
    }
    // Save the state after update i into c (before end() applies the pending
    // step to x); waits for the stream.
    ct_status save(CglsCkpt &c) {
        const cudaStream_t st = sv.st;
        const size_t nb = (size_t)n * sizeof(float), mb = (size_t)m * sizeof(float);
        CT_CUDA_TRY(cudaMemcpyAsync(c.x, x, nb, cudaMemcpyDeviceToDevice, st));
        CT_CUDA_TRY(cudaMemcpyAsync(c.z, z, nb, cudaMemcpyDeviceToDevice, st));
        if (m > 0) CT_CUDA_TRY(cudaMemcpyAsync(c.e, e, mb, cudaMemcpyDeviceToDevice, st));
        CT_CUDA_TRY(cudaMemcpyAsync(c.s, S, sizeof(CglsS), cudaMemcpyDeviceToDevice, st));
        c.hist.assign((size_t)i, 0.0);
        c.hist_nr.assign((size_t)i, 0.0);
        if (i > 0) {
            CT_CUDA_TRY(cudaMemcpyAsync(c.hist.data(), hist, sizeof(double) * (size_t)i,
                                        cudaMemcpyDeviceToHost, st));
            CT_CUDA_TRY(cudaMemcpyAsync(c.hist_nr.data(), hist + K, sizeof(double) * (size_t)i,
                                        cudaMemcpyDeviceToHost, st));
        }
        CT_CUDA_TRY(cudaStreamSynchronize(st));
        c.i = i;
        return CT_OK;
    }
    // The stopping rule of Algorithm 1 given the scalars h read back after
    // update i (only read when ERR > 0).
    bool go_on(const CglsS &h) const {
        if (i >= K) return false;
        if (ERR > 0.0 && !(std::isfinite(h.nb0) && std::isfinite(h.nb))) return false;
        return ERR <= 0.0 || ((h.nb0 > 0.0) && (h.nb / h.nb0 > ERR));
    }
    ct_status keep_going(bool *go) {
        if (i < K && ERR > 0.0) CT_TRY(read_scalars(S, &hs, sv.st));
        *go = go_on(hs);
        return CT_OK;
    }
    // Periodic recomputation of the discrepancy from the solution (Discussion).
    ct_status recompute() {
        const cudaStream_t st = sv.st;
        k_vol_axpy<<<gn, kVecThreads, 0, st>>>(x, z, n, &S->a_pend);
        CT_CHECK_LAUNCH();
        k_set_zero<<<1, 1, 0, st>>>(&S->a_pend);
        CT_CHECK_LAUNCH();
        k_sino_weighted_copy<<<gm, kVecThreads, 0, st>>>(e, b, sv.L, m, nullptr);
        CT_CHECK_LAUNCH();
        CT_TRY(sv.forward_t(x, CT_F32, sv.T, e, sd, sub, nullptr));
        k_norm2_t<<<gm, kVecThreads, 0, st>>>(e, m, sv.part);
        CT_CHECK_LAUNCH();
        return CT_OK;
    }
    // The last pending x = x + alpha d_x, then the report (waits for the stream).
    ct_status end(ct_solver_report *rep) {
        const cudaStream_t st = sv.st;
        k_vol_axpy<<<gn, kVecThreads, 0, st>>>(x, z, n, &S->a_pend);
        CT_CHECK_LAUNCH();
        std::vector<double> h((size_t)K, 0.0), h_nr((size_t)K, 0.0);
        CT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * (size_t)i,
                                    cudaMemcpyDeviceToHost, st));
        CT_CUDA_TRY(cudaMemcpyAsync(h_nr.data(), hist + K, sizeof(double) * (size_t)i,
                                    cudaMemcpyDeviceToHost, st));
        CT_TRY(read_scalars(S, &hs, st));
        sv.report(rep, i, hs.nb0, hs.nb, h, &h_nr);
        return finite_or_error(hs.nb0, hs.nb);
    }
};

template <class ST>
ct_status cgls_impl(const ct_geometry *g, const float *b, float *x, const ct_solver_opts *o,
                    ct_solver_report *rep, cudaStream_t st, CglsCkpt *ck = nullptr) {
    CglsJob<ST> job(g, b, x, o, st);
    if (ck && ck->i > 0)
        CT_TRY(job.resume(*ck));
    else
        CT_TRY(job.start());
    // Without per-operator timing or recomputation every update enqueues the
    // same launches with the same arguments (the scalars live on the device),
    // so the first one is captured as a CUDA graph and replayed: one launch
    // per update instead of a dozen.
    UpdateGraph graph;
    const bool use_graph = !o->timing && o->recompute_every == 0 && job.K > 2;
    bool go = false;
    CT_TRY(job.keep_going(&go));
    Solve &sv = job.sv;
    int dfwd = 0, dback = 0;               // operator calls per replayed update
    if (go && use_graph) {
        const int f0 = sv.n_fwd, b0 = sv.n_back;
        CT_TRY(graph.capture([&]() -> ct_status {
            CT_TRY(job.update());
            return job.finish();
        }, &sv.st));
        dfwd = sv.n_fwd - f0;
        dback = sv.n_back - b0;
        sv.n_fwd = f0;
        sv.n_back = b0;
    }
    while (go) {
        CT_TRACE("cgls update");
        if (graph.exec) {
            CT_TRY(graph.launch(st));
            sv.n_fwd += dfwd;
            sv.n_back += dback;
        } else {
            CT_TRY(job.update());
            if (o->recompute_every > 0 && (job.i + 1) % o->recompute_every == 0)
                CT_TRY(job.recompute());
            CT_TRY(job.finish());
        }
        ++job.i;
        CT_TRY(job.keep_going(&go));
    }
    if (ck) CT_TRY(job.save(*ck));
    return job.end(rep);
}

ct_status lsqr_impl(const ct_geometry *g, const float *b, float *x, const ct_solver_opts *o,
                    ct_solver_report *rep, cudaStream_t st) {
    const int K = o->max_iter;
    const double ERR = o->err_tol;
    Solve sv(g, st, o->timing != 0);
    CT_TRY(sv.init(o->precond));
    const int64_t n = sv.n, m = sv.m;
    const int gn = vec_grid(n), gm = vec_grid(m);
    const int64_t nfp = forward_partials(sv.pg), ncp = transpose_grid_count(sv.pg);
    float *u = nullptr, *v = nullptr, *wv = nullptr, *gv = nullptr, *t = nullptr;
    LsqrS *S = nullptr;
    double *hist = nullptr;
    CT_TRY(sv.ws.alloc(&u, (size_t)std::max<int64_t>(m, 1)));
    CT_TRY(sv.ws.alloc(&v, (size_t)n));
    CT_TRY(sv.ws.alloc(&wv, (size_t)n));
    CT_TRY(sv.ws.alloc(&gv, (size_t)n));
    if (sv.W) CT_TRY(sv.ws.alloc(&t, (size_t)n));
    CT_TRY(sv.ws.alloc(&S, 1));
    CT_TRY(sv.ws.alloc(&hist, 2 * (size_t)std::max(K, 1)));   // phibar / NB0, then NR
    CT_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(LsqrS), st));
    Coef sub;
    sub.alpha = -1.f;
    sub.beta = 1.f;
    Coef cf, cb;
    cf.dev = S->coef_fwd;
    cb.dev = S->coef_back;

    // NB0 = ||L b||; beta_1 u_1 = L (b - A x0)
    bool x0nz = false;
    CT_TRY(sv.nonzero(x, &x0nz));
    k_sino_weighted_copy<<<gm, kVecThreads, 0, st>>>(u, b, sv.L, m, sv.part);
    CT_CHECK_LAUNCH();
    k_lsqr_nb0<<<1, 1024, 0, st>>>(sv.part, gm, S);
    CT_CHECK_LAUNCH();
    if (x0nz) {
        CT_TRY(sv.forward(x, false, u, sub, nullptr));
        CT_TRY(launch_norm2(u, nullptr, m, sv.part, st));
    }
    k_lsqr_beta<<<1, 1024, 0, st>>>(sv.part, gm, S);
    CT_CHECK_LAUNCH();
    // alpha_1 v_1 = W A^T L u_1; w_1 = v_1; phibar = beta_1; rhobar = alpha_1
    CT_TRY(sv.back(u, gv, cb, sv.W, sv.part));
    k_lsqr_alpha0<<<1, 1024, 0, st>>>(sv.part, ncp, S);
    CT_CHECK_LAUNCH();
    k_lsqr_vinit<<<gn, kVecThreads, 0, st>>>(v, wv, gv, sv.W, n, S);
    CT_CHECK_LAUNCH();
    int i = 0;
    LsqrS hs{};
    bool go = K > 0;
    if (go && ERR > 0.0) {
        CT_TRY(read_scalars(S, &hs, st));
        go = hs.nb0 > 0.0 && hs.phibar / hs.nb0 > ERR;
    }
    // One LSQR iteration, enqueued on sv.st (captured and replayed as a CUDA
    // graph like the CGLS update, see UpdateGraph).
    auto update = [&]() -> ct_status {
        const cudaStream_t s = sv.st;
        // beta u = L A W v - alpha u
        const float *tin = v;
        if (sv.W) {
            CT_TRY(launch_transpose(sv.pg, v, sv.W, sv.T, t, s));
            tin = t;
        }
        k_lsqr_coef_fwd<<<1, 1, 0, s>>>(S);
        CT_CHECK_LAUNCH();
        CT_TRY(sv.forward(tin, sv.W != nullptr, u, cf, sv.part));
        const double *pp = nullptr;
        int64_t np = 0;
        CT_TRY(sv.reduce(sv.part, nfp, &pp, &np));
        k_lsqr_beta<<<1, 1024, 0, s>>>(pp, np, S);
        CT_CHECK_LAUNCH();
        // alpha v = W A^T L u - beta v
        CT_TRY(sv.back(u, gv, cb, nullptr, nullptr));
        k_lsqr_v<<<gn, kVecThreads, 0, s>>>(v, gv, sv.W, n, S, sv.part);
        CT_CHECK_LAUNCH();
        k_lsqr_rot<<<1, 1024, 0, s>>>(sv.part, gn, S, hist, -1, hist + K);
        CT_CHECK_LAUNCH();
        k_lsqr_update<<<gn, kVecThreads, 0, s>>>(x, v, wv, sv.W, n, S);
        CT_CHECK_LAUNCH();
        return CT_OK;
    };
    UpdateGraph graph;
    int dfwd = 0, dback = 0;
    if (go && !o->timing && K > 2) {
        const int f0 = sv.n_fwd, b0 = sv.n_back;
        CT_TRY(graph.capture(update, &sv.st));
        dfwd = sv.n_fwd - f0;
        dback = sv.n_back - b0;
        sv.n_fwd = f0;
        sv.n_back = b0;
    }
    while (go) {
        if (graph.exec) {
            CT_TRY(graph.launch(st));
            sv.n_fwd += dfwd;
            sv.n_back += dback;
        } else {
            CT_TRY(update());
        }
        ++i;
        go = i < K;
        if (go && ERR > 0.0) {
            CT_TRY(read_scalars(S, &hs, st));
            go = hs.nb0 > 0.0 && hs.phibar / hs.nb0 > ERR;
        }
    }
    std::vector<double> h((size_t)K, 0.0), h_nr((size_t)K, 0.0);
    if (i > 0) {
        CT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * (size_t)i,
                                    cudaMemcpyDeviceToHost, st));
        CT_CUDA_TRY(cudaMemcpyAsync(h_nr.data(), hist + K, sizeof(double) * (size_t)i,
                                    cudaMemcpyDeviceToHost, st));
    }
    CT_TRY(read_scalars(S, &hs, st));
    sv.report(rep, i, hs.nb0, hs.phibar, h, &h_nr);
    return finite_or_error(hs.nb0, hs.phibar);
}


// SIRT / PSIRT (Software and Results sections; no formula in the paper):
// x += relax C^-1 A^T R^-1 (b - A x), R = A 1, C = A^T 1 with the guarded
// inverses of the row/column-sum preconditioner (sums <= 1e-6 max: weight 0).
// Per update one A^T (rays weighted by R^-1) and one A recomputing
// e = b - A x, whose FP64 norm gives NB and the history.
ct_status sirt_impl(const ct_geometry *g, const float *b, float *x, const ct_sirt_opts *o,
                    ct_solver_report *rep, cudaStream_t st) {
    const int K = o->max_iter;
    const double ERR = o->err_tol;
    Solve sv(g, st, o->timing != 0);
    CT_TRY(sv.init(CT_PRECOND_ROWCOL));     // L = R^-1/2, W = C^-1/2
    const int64_t n = sv.n, m = sv.m;
    const int gn = vec_grid(n), gm = vec_grid(m);
    const int64_t nfp = forward_partials(sv.pg);
    k_square<<<gm, kVecThreads, 0, st>>>(sv.L, m);            // R^-1
    CT_CHECK_LAUNCH();
    k_square<<<gn, kVecThreads, 0, st>>>(sv.W, n);            // C^-1
    CT_CHECK_LAUNCH();
    float *e = nullptr, *gv = nullptr;
    CglsS *S = nullptr;
    double *hist = nullptr;
    CT_TRY(sv.ws.alloc(&e, (size_t)std::max<int64_t>(m, 1)));
    CT_TRY(sv.ws.alloc(&gv, (size_t)n));
    CT_TRY(sv.ws.alloc(&S, 1));
    CT_TRY(sv.ws.alloc(&hist, (size_t)K));
    CT_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(CglsS), st));
    Coef sub;                               // e = b - A x
    sub.alpha = -1.f;
    sub.beta = 1.f;
    // e = b (with partials of ||b||^2 when requested); the forward calls below
    // then subtract A x without row weights
    auto copy_b = [&](double *partials) -> ct_status {
        k_sino_weighted_copy<<<gm, kVecThreads, 0, st>>>(e, b, nullptr, m, partials);
        CT_CHECK_LAUNCH();
        return CT_OK;
    };
    bool x0nz = false;
    CT_TRY(sv.nonzero(x, &x0nz));
    CT_TRY(copy_b(sv.part));                // NB0 = ||b||
    k_cgls_nb0<<<1, 1024, 0, st>>>(sv.part, gm, S);
    CT_CHECK_LAUNCH();
    auto project_residual = [&](double *partials) -> ct_status {
        CT_TRY(launch_transpose(sv.pg, x, nullptr, sv.T, nullptr, st));
        CT_TRY(sv.tm.mark(sv.tm.fwd));
        CT_TRY(launch_forward(sv.pg, x, sv.T, e, nullptr, sub, partials, st));
        CT_TRY(sv.tm.mark(sv.tm.fwd));
        ++sv.n_fwd;
        return CT_OK;
    };
    if (x0nz) CT_TRY(project_residual(nullptr));
    Coef one;
    int i = 0;
    CglsS hs{};
    bool go = K > 0;
    while (go) {
        // x = x + relax C^-1 A^T R^-1 e
        CT_TRY(sv.back(e, gv, one, nullptr, nullptr));
        k_sirt_update<<<gn, kVecThreads, 0, st>>>(x, gv, sv.W, n, (float)o->relax);
        CT_CHECK_LAUNCH();
        // e = b - A x; NB = ||e||
        CT_TRY(copy_b(nullptr));
        CT_TRY(project_residual(sv.part));
        k_cgls_nb<<<1, 1024, 0, st>>>(sv.part, nfp, S, hist, i, nullptr);
        CT_CHECK_LAUNCH();
        ++i;
        go = i < K;
        if (go && ERR > 0.0) {
            CT_TRY(read_scalars(S, &hs, st));
            go = hs.nb0 > 0.0 && hs.nb / hs.nb0 > ERR;
        }
    }
    std::vector<double> h((size_t)K, 0.0);
    CT_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * (size_t)i,
                                cudaMemcpyDeviceToHost, st));
    CT_TRY(read_scalars(S, &hs, st));
    sv.report(rep, i, hs.nb0, hs.nb, h);
    return finite_or_error(hs.nb0, hs.nb);
}
}  // namespace
}  // namespace ct

using namespace ct;

// Opaque to callers (include/ct.h): a CGLS state between two updates.
struct ct_cgls_state {
    CglsCkpt ck;
};

// Several CGLS solves advanced in lock step (continuous batching): each
// ct_batch_step runs one update of every active job, with the A^T of all
// batchable jobs in one persistent launch and their A in another (the
// vector kernels stay per job).  Jobs join (ct_batch_add_cgls) and leave
// (their stopping rule, ct_batch_remove) between steps.  The step of a fixed
// set of jobs is captured as a CUDA graph and replayed until the set changes.
// Side streams over which a batched step spreads the jobs' vector kernels.
constexpr int kBatchSideStreams = 8;

// Steps with an unchanged set of jobs after which ct_batch captures its step
// as a CUDA graph (before that, and after every join or leave, it launches
// the step's kernels directly).
constexpr int kStableSteps = 3;

struct ct_batch {
    struct Entry {
        int32_t id = 0;
        std::unique_ptr<CglsJob<float>> job;
        bool done = false;
        bool batched = false;           // its projectors run in the batched launches
        ct_solver_report rep{};
        std::vector<double> hist, hist_nr;
    };
    int device = 0;
    cudaStream_t st = nullptr;
    std::vector<Entry> jobs;
    int32_t next_id = 1;
    bool dirty = true;                  // the set of active jobs changed since the tables
    BatchJob *h_tab = nullptr;          // pinned host staging of the launch tables
    BatchJob *d_tab = nullptr;          // [A^T float | A^T fixed point | A] tables
    size_t tab_cap = 0;
    unsigned *d_next = nullptr;         // work counter of the batched launches
    CglsS *h_s = nullptr;               // pinned copies of the jobs' scalars
    size_t s_cap = 0;
    int nbf = 0, nbd = 0, nfw = 0;      // jobs in each table
    unsigned tbf = 0, tbd = 0, tfw = 0; // tiles in each table
    std::unique_ptr<UpdateGraph> graph;
    int stable = 0;                     // steps since the set of active jobs last changed
    std::vector<cudaStream_t> side;     // streams of the per-job phases
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;

    ct_status init_streams(int n) {
        CT_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        for (int k = 0; k < n; ++k) {
            cudaStream_t s = nullptr;
            CT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            side.push_back(s);
            cudaEvent_t e = nullptr;
            CT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            ev_join.push_back(e);
        }
        return CT_OK;
    }

    ~ct_batch() {
        graph.reset();
        jobs.clear();                   // frees their workspaces on st
        if (st) cudaStreamSynchronize(st);
        for (auto s : side) cudaStreamDestroy(s);
        for (auto e : ev_join) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (d_tab) cudaFree(d_tab);
        if (d_next) cudaFree(d_next);
        if (h_tab) cudaFreeHost(h_tab);
        if (h_s) cudaFreeHost(h_s);
    }

    Entry *find(int32_t id) {
        for (auto &e : jobs)
            if (e.id == id) return &e;
        return nullptr;
    }

    // Rebuild and upload the launch tables of the active jobs.
    ct_status build_tables() {
        CT_CUDA_TRY(cudaStreamSynchronize(st));   // the old tables are no longer read
        std::vector<BatchJob> bf, bd, fw;
        unsigned t;
        for (auto &en : jobs) {
            if (en.done) continue;
            CglsJob<float> &j = *en.job;
            en.batched = batchable(j.sv.pg) && !j.sv.tm.on;
            if (!en.batched) continue;
            BatchJob bb{}, fb{};
            CT_TRY(j.back_job(&bb));
            CT_TRY(j.fwd_job(&fb));
            (fixed_back(j.sv.g) ? bd : bf).push_back(bb);
            fw.push_back(fb);
        }
        auto offsets = [&](std::vector<BatchJob> &v, unsigned *total) -> ct_status {
            t = 0;
            for (auto &x : v) {
                x.tile0 = t;
                if ((uint64_t)t + x.tiles > 0xffffff00ull)
                    return set_error(CT_ERR_INVALID_ARG, "batch: too many tiles in one launch");
                t += x.tiles;
            }
            *total = t;
            return CT_OK;
        };
        CT_TRY(offsets(bf, &tbf));
        CT_TRY(offsets(bd, &tbd));
        CT_TRY(offsets(fw, &tfw));
        nbf = (int)bf.size();
        nbd = (int)bd.size();
        nfw = (int)fw.size();
        const size_t need = bf.size() + bd.size() + fw.size();
        if (need > tab_cap) {
            if (d_tab) CT_CUDA_TRY(cudaFree(d_tab));
            if (h_tab) CT_CUDA_TRY(cudaFreeHost(h_tab));
            d_tab = nullptr;
            h_tab = nullptr;
            tab_cap = 0;
            CT_CUDA_TRY(cudaMalloc(&d_tab, need * sizeof(BatchJob)));
            CT_CUDA_TRY(cudaMallocHost(&h_tab, need * sizeof(BatchJob)));
            tab_cap = need;
        }
        std::copy(bf.begin(), bf.end(), h_tab);
        std::copy(bd.begin(), bd.end(), h_tab + nbf);
        std::copy(fw.begin(), fw.end(), h_tab + nbf + nbd);
        if (need)
            CT_CUDA_TRY(cudaMemcpyAsync(d_tab, h_tab, need * sizeof(BatchJob),
                                        cudaMemcpyHostToDevice, st));
        graph.reset();
        dirty = false;
        return CT_OK;
    }

    // Runs fn(entry) for every active job, the jobs spread over the side
    // streams (forked from and joined back into the jobs' stream), so that
    // the small vector kernels of different jobs overlap.
    template <class F>
    ct_status phase(F &&fn) {
        const cudaStream_t m = jobs_stream();
        int act = 0;
        for (auto &en : jobs) act += !en.done;
        const int used = std::min<int>(act, (int)side.size());
        CT_CUDA_TRY(cudaEventRecord(ev_fork, m));
        for (int k = 0; k < used; ++k) CT_CUDA_TRY(cudaStreamWaitEvent(side[k], ev_fork, 0));
        int k = 0;
        for (auto &en : jobs) {
            if (en.done) continue;
            en.job->sv.st = side[(size_t)(k++ % used)];
            CT_TRY(fn(en));
            en.job->sv.st = m;
        }
        for (int j = 0; j < used; ++j) {
            CT_CUDA_TRY(cudaEventRecord(ev_join[j], side[j]));
            CT_CUDA_TRY(cudaStreamWaitEvent(m, ev_join[j], 0));
        }
        return CT_OK;
    }

    // One update of every active job (the phases of CglsJob::update), with
    // the batchable jobs' A^T and A as batched launches between the phases.
    ct_status step_body() {
        CT_TRY(phase([](Entry &en) -> ct_status {
            CT_TRY(en.job->grad_pre());
            return en.batched ? CT_OK : en.job->grad_proj();
        }));
        const cudaStream_t s = jobs_stream();
        CT_TRY(launch_batch(d_tab, nbf, tbf, true, false, d_next, s));
        CT_TRY(launch_batch(d_tab + nbf, nbd, tbd, true, true, d_next, s));
        CT_TRY(phase([](Entry &en) -> ct_status {
            CT_TRY(en.job->grad_post(0));
            CT_TRY(en.job->middle(0));
            return en.batched ? CT_OK : en.job->fwd_proj();
        }));
        CT_TRY(launch_batch(d_tab + nbf + nbd, nfw, tfw, false, true, d_next, s));
        return phase([](Entry &en) -> ct_status {
            CT_TRY(en.job->tail());
            return en.job->finish();
        });
    }
    // The stream the jobs currently launch on (the capture stream meanwhile).
    cudaStream_t cur = nullptr;
    cudaStream_t jobs_stream() const { return cur ? cur : st; }
    void set_stream(cudaStream_t s) {
        cur = s;
        for (auto &en : jobs)
            if (!en.done) en.job->sv.st = s ? s : st;
    }

    ct_status step(int32_t *n_active) {
        int active = 0;
        for (auto &en : jobs) active += !en.done;
        if (active > 0) {
            if (dirty) {
                CT_TRY(build_tables());
                stable = 0;
            }
            // A graph pays only if the same step is replayed: while jobs join
            // or leave step after step (a busy server), launch the step
            // directly, and capture it once the set has held for kStableSteps.
            if (!graph && stable < kStableSteps) {
                std::vector<int> f0, b0;   // counted below, one A and one A^T per update
                for (auto &en : jobs) {
                    f0.push_back(en.job->sv.n_fwd);
                    b0.push_back(en.job->sv.n_back);
                }
                const ct_status ds = step_body();
                for (size_t k = 0; k < jobs.size(); ++k) {
                    jobs[k].job->sv.n_fwd = f0[k];
                    jobs[k].job->sv.n_back = b0[k];
                }
                CT_TRY(ds);
            } else if (!graph) {
                // the same launches with the same arguments until the set changes
                graph.reset(new UpdateGraph());
                std::vector<int> f0, b0;
                for (auto &en : jobs) {
                    f0.push_back(en.job->sv.n_fwd);
                    b0.push_back(en.job->sv.n_back);
                }
                const ct_status cs = graph->capture([&]() { return step_body(); },
                                                    [&](cudaStream_t c) { set_stream(c); });
                for (size_t k = 0; k < jobs.size(); ++k) {   // counted again per replay
                    jobs[k].job->sv.n_fwd = f0[k];
                    jobs[k].job->sv.n_back = b0[k];
                }
                if (cs != CT_OK) {   // nothing ran; the next step captures again
                    graph.reset();
                    return cs;
                }
            }
            if (graph) CT_TRY(graph->launch(st));
            ++stable;
            // scalars of the jobs that test a tolerance, one wait for all
            if (jobs.size() > s_cap) {
                if (h_s) CT_CUDA_TRY(cudaFreeHost(h_s));
                h_s = nullptr;
                s_cap = 0;
                CT_CUDA_TRY(cudaMallocHost(&h_s, jobs.size() * sizeof(CglsS)));
                s_cap = jobs.size();
            }
            bool any_read = false;
            for (size_t k = 0; k < jobs.size(); ++k) {
                Entry &en = jobs[k];
                if (en.done) continue;
                CglsJob<float> &j = *en.job;
                ++j.i;
                ++j.sv.n_back;   // one A^T and one A per update
                ++j.sv.n_fwd;
                if (j.i < j.K && j.ERR > 0.0) {
                    CT_CUDA_TRY(cudaMemcpyAsync(h_s + k, j.S, sizeof(CglsS),
                                                cudaMemcpyDeviceToHost, st));
                    any_read = true;
                }
            }
            if (any_read) CT_CUDA_TRY(cudaStreamSynchronize(st));
            for (size_t k = 0; k < jobs.size(); ++k) {
                Entry &en = jobs[k];
                if (en.done) continue;
                CglsJob<float> &j = *en.job;
                if (j.i < j.K && j.ERR > 0.0) j.hs = h_s[k];
                if (!j.go_on(j.hs)) CT_TRY(retire(en));
            }
        }
        int left = 0;
        for (auto &en : jobs) left += !en.done;
        *n_active = left;
        return CT_OK;
    }

    // The job's stopping rule fired: finish x and keep the report.
    ct_status retire(Entry &en) {
        en.hist.assign((size_t)en.job->K, 0.0);
        en.hist_nr.assign((size_t)en.job->K, 0.0);
        en.rep = ct_solver_report{};
        en.rep.history_nb = en.hist.data();
        en.rep.history_nr = en.hist_nr.data();
        en.rep.history_cap = en.job->K;
        CT_TRY(en.job->end(&en.rep));
        en.done = true;
        dirty = true;
        return CT_OK;
    }
};

extern "C" {

ct_status ct_batch_create(void *stream, ct_batch **out) {
    clear_error();
    if (!out) return set_error(CT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::unique_ptr<ct_batch> b(new ct_batch());
    b->st = (cudaStream_t)stream;
    CT_CUDA_TRY(cudaGetDevice(&b->device));
    CT_TRY(batch_prepare());
    CT_TRY(b->init_streams(kBatchSideStreams));
    CT_CUDA_TRY(cudaMalloc(&b->d_next, sizeof(unsigned)));
    *out = b.release();
    return CT_OK;
}

ct_status ct_batch_destroy(ct_batch *b) {
    clear_error();
    if (!b) return CT_OK;
    DeviceGuard dg(b->device);
    CT_TRY(dg.status());
    delete b;
    return CT_OK;
}

ct_status ct_batch_add_cgls(ct_batch *b, const ct_geometry *g, const float *d_b, float *d_x,
                            const ct_solver_opts *opts, int32_t *job) {
    CT_TRACE("ct_batch_add_cgls");
    clear_error();
    if (!b || !job) return set_error(CT_ERR_INVALID_ARG, "NULL batch or job");
    CT_TRY(check_opts(g, d_b, d_x, opts));
    if (g->device != b->device)
        return set_error(CT_ERR_INVALID_ARG, "batch: geometry on another device");
    if (opts->storage != CT_F32 || opts->timing != 0 || opts->recompute_every != 0)
        return set_error(CT_ERR_INVALID_ARG,
                         "batch: FP32 storage, no timing and no recomputation only");
    DeviceGuard dg(b->device);
    CT_TRY(dg.status());
    ct_batch::Entry en;
    en.id = b->next_id++;
    en.job.reset(new CglsJob<float>(g, d_b, d_x, opts, b->st));
    ct_status s = en.job->start();
    bool go = false;
    if (s == CT_OK) s = en.job->keep_going(&go);
    if (s != CT_OK) {
        cudaStreamSynchronize(b->st);
        return s;
    }
    b->jobs.push_back(std::move(en));
    ct_batch::Entry &added = b->jobs.back();
    if (!go) CT_TRY(b->retire(added));
    b->dirty = true;
    *job = added.id;
    return CT_OK;
}

ct_status ct_batch_step(ct_batch *b, int32_t *n_active) {
    CT_TRACE("ct_batch_step");
    clear_error();
    if (!b || !n_active) return set_error(CT_ERR_INVALID_ARG, "NULL batch or n_active");
    DeviceGuard dg(b->device);
    CT_TRY(dg.status());
    return b->step(n_active);
}

ct_status ct_batch_poll(ct_batch *b, int32_t job, int32_t *done, ct_solver_report *report) {
    clear_error();
    if (!b || !done) return set_error(CT_ERR_INVALID_ARG, "NULL batch or done");
    ct_batch::Entry *en = b->find(job);
    if (!en) return set_error(CT_ERR_INVALID_ARG, "batch: unknown job");
    *done = en->done ? 1 : 0;
    if (en->done && report) {
        double *hn = report->history_nb, *hr = report->history_nr;
        const int32_t cap = report->history_cap;
        *report = en->rep;
        report->history_nb = hn;
        report->history_nr = hr;
        report->history_cap = cap;
        const int k = std::min<int>(cap, std::min<int>(en->rep.iterations, (int)en->hist.size()));
        for (int j = 0; hn && j < k; ++j) hn[j] = en->hist[(size_t)j];
        for (int j = 0; hr && j < k; ++j) hr[j] = en->hist_nr[(size_t)j];
    }
    return CT_OK;
}

ct_status ct_batch_remove(ct_batch *b, int32_t job) {
    clear_error();
    if (!b) return set_error(CT_ERR_INVALID_ARG, "NULL batch");
    DeviceGuard dg(b->device);
    CT_TRY(dg.status());
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        if (b->jobs[k].id != job) continue;
        if (!b->jobs[k].done) CT_TRY(b->retire(b->jobs[k]));   // x gets its pending update
        b->jobs.erase(b->jobs.begin() + (long)k);
        b->dirty = true;
        CT_CUDA_TRY(cudaStreamSynchronize(b->st));
        return CT_OK;
    }
    return set_error(CT_ERR_INVALID_ARG, "batch: unknown job");
}

ct_status ct_cgls(const ct_geometry *g, const float *d_b, float *d_x, const ct_solver_opts *opts,
                  ct_solver_report *report, void *stream) {
    CT_TRACE("ct_cgls");
    clear_error();
    CT_TRY(check_opts(g, d_b, d_x, opts));
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    ct_status s;
    switch (opts->storage) {
        case CT_BF16: s = cgls_impl<__nv_bfloat16>(g, d_b, d_x, opts, report, st); break;
        case CT_F16: s = cgls_impl<__half>(g, d_b, d_x, opts, report, st); break;
        default: s = cgls_impl<float>(g, d_b, d_x, opts, report, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == CT_OK && e != cudaSuccess) return cuda_error(e, "ct_cgls");
    return s;
}

ct_status ct_lsqr(const ct_geometry *g, const float *d_b, float *d_x, const ct_solver_opts *opts,
                  ct_solver_report *report, void *stream) {
    CT_TRACE("ct_lsqr");
    clear_error();
    CT_TRY(check_opts(g, d_b, d_x, opts));
    if (opts->tikhonov_lambda != 0.0)
        return set_error(CT_ERR_INVALID_ARG, "LSQR: tikhonov_lambda must be 0 (use ct_cgls)");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    if (opts->storage != CT_F32)
        return set_error(CT_ERR_INVALID_ARG, "LSQR supports FP32 storage only");
    ct_status s = lsqr_impl(g, d_b, d_x, opts, report, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == CT_OK && e != cudaSuccess) return cuda_error(e, "ct_lsqr");
    return s;
}

ct_status ct_sirt(const ct_geometry *g, const float *d_b, float *d_x, const ct_sirt_opts *opts,
                  ct_solver_report *report, void *stream) {
    CT_TRACE("ct_sirt");
    clear_error();
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    if (!opts) return set_error(CT_ERR_INVALID_ARG, "opts is NULL");
    if (!d_x || (g->nrays > 0 && !d_b)) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (opts->max_iter < 1) return set_error(CT_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!std::isfinite(opts->err_tol) || opts->err_tol < 0.0)
        return set_error(CT_ERR_INVALID_ARG, "err_tol must be finite and >= 0");
    if (!std::isfinite(opts->relax) || !(opts->relax > 0.0) || !(opts->relax < 2.0))
        return set_error(CT_ERR_INVALID_ARG, "relax must lie in (0, 2)");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    const ct_status s = sirt_impl(g, d_b, d_x, opts, report, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == CT_OK && e != cudaSuccess) return cuda_error(e, "ct_sirt");
    return s;
}

// ---- CGLS checkpoint / resume -----------------------------------------------

ct_status ct_cgls_state_create(const ct_geometry *g, ct_cgls_state **out) {
    clear_error();
    if (!g || !out) return set_error(CT_ERR_INVALID_ARG, "geometry and out must be non-NULL");
    *out = nullptr;
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    ct_cgls_state *st = new (std::nothrow) ct_cgls_state();
    if (!st) return set_error(CT_ERR_OOM, "host allocation failed");
    CglsCkpt &c = st->ck;
    c.device = g->device;
    c.n = g->nvox;
    c.m = g->nrays;
    cudaError_t e = cudaMalloc(&c.x, (size_t)c.n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c.z, (size_t)c.n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c.e, (size_t)std::max<int64_t>(c.m, 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c.s, sizeof(CglsS));
    if (e != cudaSuccess) {
        ct_cgls_state_destroy(st);
        return e == cudaErrorMemoryAllocation ? set_error(CT_ERR_OOM, "cgls state: out of memory")
                                              : cuda_error(e, "cgls state allocation");
    }
    *out = st;
    return CT_OK;
}

void ct_cgls_state_destroy(ct_cgls_state *st) {
    if (!st) return;
    {
        DeviceGuard dg(st->ck.device);
        if (st->ck.x) cudaFree(st->ck.x);
        if (st->ck.z) cudaFree(st->ck.z);
        if (st->ck.e) cudaFree(st->ck.e);
        if (st->ck.s) cudaFree(st->ck.s);
    }
    delete st;
}

ct_status ct_cgls_state_iterations(const ct_cgls_state *st, int32_t *iterations) {
    clear_error();
    if (!st || !iterations) return set_error(CT_ERR_INVALID_ARG, "NULL state or iterations");
    *iterations = st->ck.i;
    return CT_OK;
}

namespace {
// Serialised form of a state: this header, then x, d_x (n floats each), e_b
// (m floats), the scalar block, the NB / NB0 history and the NR history (i
// doubles each), native byte order.
struct CkptHeader {
    uint32_t magic, version;
    int64_t n, m;
    int32_t i, pad;
    uint64_t scalar_bytes;
};
constexpr uint32_t kCkptMagic = 0x47435443u;   // "CTCG"
constexpr uint32_t kCkptVersion = 2;

int64_t ckpt_bytes(const CglsCkpt &c) {
    return (int64_t)sizeof(CkptHeader) + (2 * c.n + c.m) * (int64_t)sizeof(float) +
           (int64_t)sizeof(CglsS) + 2 * c.i * (int64_t)sizeof(double);
}
}  // namespace

ct_status ct_cgls_state_export(const ct_cgls_state *st, void *host, int64_t capacity,
                               int64_t *bytes) {
    clear_error();
    if (!st || !bytes) return set_error(CT_ERR_INVALID_ARG, "NULL state or bytes");
    const CglsCkpt &c = st->ck;
    *bytes = ckpt_bytes(c);
    if (!host) return CT_OK;
    if (capacity < *bytes) return set_error(CT_ERR_INVALID_ARG, "export buffer too small");
    DeviceGuard dg(c.device);
    CT_TRY(dg.status());
    char *p = static_cast<char *>(host);
    CkptHeader h{kCkptMagic, kCkptVersion, c.n, c.m, c.i, 0, sizeof(CglsS)};
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    CT_CUDA_TRY(cudaMemcpy(p, c.x, (size_t)c.n * sizeof(float), cudaMemcpyDeviceToHost));
    p += c.n * sizeof(float);
    CT_CUDA_TRY(cudaMemcpy(p, c.z, (size_t)c.n * sizeof(float), cudaMemcpyDeviceToHost));
    p += c.n * sizeof(float);
    if (c.m > 0) CT_CUDA_TRY(cudaMemcpy(p, c.e, (size_t)c.m * sizeof(float), cudaMemcpyDeviceToHost));
    p += c.m * sizeof(float);
    CT_CUDA_TRY(cudaMemcpy(p, c.s, sizeof(CglsS), cudaMemcpyDeviceToHost));
    p += sizeof(CglsS);
    if (c.i > 0) {
        std::memcpy(p, c.hist.data(), sizeof(double) * (size_t)c.i);
        p += c.i * sizeof(double);
        std::memcpy(p, c.hist_nr.data(), sizeof(double) * (size_t)c.i);
    }
    return CT_OK;
}

ct_status ct_cgls_state_import(ct_cgls_state *st, const void *host, int64_t bytes) {
    clear_error();
    if (!st || !host) return set_error(CT_ERR_INVALID_ARG, "NULL state or buffer");
    CglsCkpt &c = st->ck;
    CkptHeader h;
    if (bytes < (int64_t)sizeof(h)) return set_error(CT_ERR_INVALID_ARG, "state buffer too short");
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != kCkptMagic || h.version != kCkptVersion || h.scalar_bytes != sizeof(CglsS))
        return set_error(CT_ERR_INVALID_ARG, "not a CGLS state of this library version");
    if (h.n != c.n || h.m != c.m)
        return set_error(CT_ERR_INVALID_ARG, "state sizes do not match this geometry");
    if (h.i < 0) return set_error(CT_ERR_INVALID_ARG, "state: negative update count");
    CglsCkpt probe;
    probe.n = h.n;
    probe.m = h.m;
    probe.i = h.i;
    if (bytes != ckpt_bytes(probe)) return set_error(CT_ERR_INVALID_ARG, "state buffer size");
    DeviceGuard dg(c.device);
    CT_TRY(dg.status());
    const char *p = static_cast<const char *>(host) + sizeof(h);
    CT_CUDA_TRY(cudaMemcpy(c.x, p, (size_t)c.n * sizeof(float), cudaMemcpyHostToDevice));
    p += c.n * sizeof(float);
    CT_CUDA_TRY(cudaMemcpy(c.z, p, (size_t)c.n * sizeof(float), cudaMemcpyHostToDevice));
    p += c.n * sizeof(float);
    if (c.m > 0) CT_CUDA_TRY(cudaMemcpy(c.e, p, (size_t)c.m * sizeof(float), cudaMemcpyHostToDevice));
    p += c.m * sizeof(float);
    CT_CUDA_TRY(cudaMemcpy(c.s, p, sizeof(CglsS), cudaMemcpyHostToDevice));
    p += sizeof(CglsS);
    c.hist.assign((size_t)h.i, 0.0);
    c.hist_nr.assign((size_t)h.i, 0.0);
    if (h.i > 0) {
        std::memcpy(c.hist.data(), p, sizeof(double) * (size_t)h.i);
        p += h.i * sizeof(double);
        std::memcpy(c.hist_nr.data(), p, sizeof(double) * (size_t)h.i);
    }
    c.i = h.i;
    return CT_OK;
}

ct_status ct_cgls_resume(const ct_geometry *g, const float *d_b, float *d_x,
                         const ct_solver_opts *opts, ct_solver_report *report, ct_cgls_state *state,
                         void *stream) {
    CT_TRACE("ct_cgls_resume");
    clear_error();
    CT_TRY(check_opts(g, d_b, d_x, opts));
    if (!state) return set_error(CT_ERR_INVALID_ARG, "state is NULL");
    CglsCkpt &c = state->ck;
    if (c.n != g->nvox || c.m != g->nrays || c.device != g->device)
        return set_error(CT_ERR_INVALID_ARG, "state belongs to another geometry size or device");
    if (opts->storage != CT_F32)
        return set_error(CT_ERR_INVALID_ARG, "resumable CGLS supports FP32 storage only");
    if (opts->max_iter < c.i)
        return set_error(CT_ERR_INVALID_ARG, "max_iter is below the updates the state holds");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    ct_status s = cgls_impl<float>(g, d_b, d_x, opts, report, st, &c);
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == CT_OK && e != cudaSuccess) return cuda_error(e, "ct_cgls_resume");
    return s;
}

}  // extern "C"
