// ct_project_norm2_noalloc: forward projection plus its squared norm without
// any device allocation.
//
// ct_project_norm2 allocates, on every call, a transposed copy of the volume
// and one FP64 partial sum per CTA.  Some callers cannot let a library
// allocate device memory once they are running: a reconstruction service
// that reserves HBM up front for its own pool, or a real-time pipeline whose
// latency budget has no room for an allocator call.  This entry point reads
// the volume in place and keeps its partial sums in a file-scope device
// array of fixed size instead.
#include <mutex>

#include "ct_internal.h"

namespace ct {
namespace {

// At most this many CTAs (32 x 8 rays each), one FP64 partial each: 2 MiB,
// resident on every device that loads the library until the process exits.
constexpr int64_t kNoAllocMaxPartials = int64_t(1) << 18;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// Device address of g_noalloc_partials per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, called once per device with that device current.  The
// cache lives as long as the process: a device reset (cudaDeviceReset, or
// anything else that destroys the primary context) reloads the module, may
// move the array and invalidates the cached address, together with every
// geometry created on that device before the reset.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

ct_status scratch_address(int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(CT_ERR_INVALID_ARG, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return CT_OK;
}

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_project_norm2_noalloc(const ct_geometry *g, const float *d_vol,
                                              float *d_sino, float alpha, float beta,
                                              double *d_norm2, void *stream) {
    CT_TRACE("ct_project_norm2_noalloc");
    clear_error();
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    if (!d_norm2) return set_error(CT_ERR_INVALID_ARG, "d_norm2 is NULL");
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    if (g->nrays == 0) {
        CT_CUDA_TRY(cudaMemsetAsync(d_norm2, 0, sizeof(double), st));
        return CT_OK;
    }
    if (!d_vol || !d_sino) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (g->pg.sf_det)
        return set_error(CT_ERR_INVALID_ARG,
                         "ct_project_norm2_noalloc: a deterministic footprint geometry sums "
                         "in int64 scratch of 8 bytes per ray; use ct_project_norm2");
    const int64_t np = forward_direct_partials(g->pg);
    if (np > kNoAllocMaxPartials)
        return set_error(CT_ERR_INVALID_ARG,
                         "ct_project_norm2_noalloc: geometry needs " + std::to_string(np) +
                             " CTAs of 32x8 rays, the static scratch holds " +
                             std::to_string(kNoAllocMaxPartials) +
                             " (CTAs = ceil(nu/32) * ceil(nv/8) * nviews rounded up to a "
                             "multiple of the view group G = ceil(nviews / floor(65535 / "
                             "ceil(nv/8))), G = 1 unless nviews * ceil(nv/8) > 65535)");
    double *part = nullptr;
    CT_TRY(scratch_address(g->device, &part));
    // every CTA overwrites its own partial, and the sum reads exactly those,
    // so nothing left in the array by an earlier call needs clearing
    CT_TRY(launch_forward_direct(g->pg, d_vol, d_sino, alpha, beta, part, st));
    return launch_sum(part, np, d_norm2, st);
}
