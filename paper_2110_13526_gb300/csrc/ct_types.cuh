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

}  // namespace ct
