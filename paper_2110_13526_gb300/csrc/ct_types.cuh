// Storage element types of volumes and sinograms (FP32, BF16, FP16).
// Arithmetic is always FP32 (ray sums, updates) or FP64 (Krylov scalars);
// these helpers only load, convert and round on store.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ct {

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// Read-only cached load converted to FP32.
__device__ __forceinline__ float ld_f(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_f(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_f(const __half *p) { return __half2float(__ldg(p)); }

template <class T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) {
    return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half from_f<__half>(float v) {
    return __float2half_rn(v);
}

// Per-thread sum of squares of FP32 values for the FP64 norm partials.  Each
// q^2 is split exactly into p + pe (p = fl(q q), pe = fma(q, q, -p)); p goes
// into a float-float pair (hi, lo) by Knuth's two-sum, whose rounding error
// and pe collect in lo.  After k terms the pair is off by about k 2^-48 of
// the sum (the rounding of lo), against k 2^-53 for an FP64 accumulator, but
// it runs on the FP32 pipes: at GB300's FP64 rate (about 1/64 of FP32) one
// conversion and one DFMA per element bounded the streaming kernels, not
// HBM.  Terms outside [2^-50, 2^50] (or NaN) go to an FP64 accumulator, so
// that no square under- or overflows FP32 and a thread's up to 2^20 terms
// keep hi below 2^120.  value() hands the partial to the FP64 block sums.
struct SqSum {
    float hi = 0.f, lo = 0.f;
    double far = 0.0;
    __device__ __forceinline__ void add(float q) {
        const float aq = fabsf(q);
        if (!(aq <= 0x1p50f && (aq >= 0x1p-50f || aq == 0.f))) {
            far = fma((double)q, (double)q, far);
            return;
        }
        const float p = __fmul_rn(q, q);
        const float pe = __fmaf_rn(q, q, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, pe));
    }
    __device__ __forceinline__ double value() const { return ((double)hi + (double)lo) + far; }
};

}  // namespace ct
