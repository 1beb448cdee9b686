// Bounds checks of the CT_DEBUG_BOUNDS build.
//
// Compiled with -DCT_DEBUG_BOUNDS, every voxel and detector-pixel index the
// projector kernels are about to touch is checked against its array's size:
// an index out of range is not accessed, and the first one seen records its
// source line in a device error word of the translation unit, which
// ct_debug_status() reads back (and clears) as CT_ERR_INTERNAL.  In the
// normal build CT_IN_BOUNDS is the constant true and costs nothing.
#pragma once

#include "ct_internal.h"

#ifdef CT_DEBUG_BOUNDS
namespace ct {
namespace {
// (source line << 1) | 1 of the first violation in this translation unit.
__device__ unsigned long long g_debug_word = 0ull;

__device__ __forceinline__ bool in_bounds(long long i, long long n, int line) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_debug_word, 0ull, ((unsigned long long)line << 1) | 1ull);
    return false;
}
}  // namespace
}  // namespace ct
#define CT_IN_BOUNDS(i, n) ::ct::in_bounds((long long)(i), (long long)(n), __LINE__)
// Host side: reads and clears this translation unit's word (0: no violation).
#define CT_DEBUG_ACCESSOR(fn)                                                          \
    namespace ct {                                                                     \
    ct_status fn(unsigned long long *word) {                                           \
        CT_CUDA_TRY(cudaMemcpyFromSymbol(word, g_debug_word, sizeof(*word)));          \
        const unsigned long long zero = 0ull;                                          \
        CT_CUDA_TRY(cudaMemcpyToSymbol(g_debug_word, &zero, sizeof(zero)));            \
        return CT_OK;                                                                  \
    }                                                                                  \
    }
#else
#define CT_IN_BOUNDS(i, n) true
#define CT_DEBUG_ACCESSOR(fn)                      \
    namespace ct {                                 \
    ct_status fn(unsigned long long *word) {       \
        *word = 0ull;                              \
        return CT_OK;                              \
    }                                              \
    }
#endif
