// ct_project_batch / ct_backproject_batch: the projector pair applied to a
// batch of volumes (or sinograms) of one geometry, e.g. the items of a
// differentiable training batch.
//
// For a column-major Siddon geometry the projector runs ONE persistent
// launch over the tiles of all items (the batched kernels of projector.cu,
// one job per item: every tile runs the code of a plain launch, so each
// item's A is bitwise that of ct_project); only the layout transposes
// around it run per item.  Other geometries (ray-major or footprint
// projectors, fixed-point backprojection) run the single-item path for each
// item in turn, with the same results.
#include <vector>

#include "ct_internal.h"

using namespace ct;

namespace {

ct_status check_batch(const ct_geometry *g, int32_t nbatch, const void *in, const void *out) {
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    if (nbatch < 0) return set_error(CT_ERR_INVALID_ARG, "nbatch must be >= 0");
    if (nbatch > 0 && (!in || !out)) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    return CT_OK;
}

// Uploads the job table (host copy) and runs one batched projector launch.
ct_status run_jobs(std::vector<BatchJob> &jobs, bool backward, Workspace &ws, cudaStream_t st) {
    unsigned total = 0;
    for (auto &j : jobs) {
        j.tile0 = total;
        if ((uint64_t)total + j.tiles > 0xffffff00ull)
            return set_error(CT_ERR_INVALID_ARG, "batch: too many tiles in one launch");
        total += j.tiles;
    }
    BatchJob *d_tab = nullptr;
    unsigned *d_next = nullptr;
    CT_TRY(ws.alloc(&d_tab, jobs.size()));
    CT_TRY(ws.alloc(&d_next, 1));
    // pageable source: the copy has taken the bytes when the call returns
    CT_CUDA_TRY(cudaMemcpyAsync(d_tab, jobs.data(), jobs.size() * sizeof(BatchJob),
                                cudaMemcpyHostToDevice, st));
    CT_TRY(batch_prepare());
    return launch_batch(d_tab, (int)jobs.size(), total, backward, false, d_next, st);
}

}  // namespace

extern "C" ct_status ct_project_batch(const ct_geometry *g, const float *d_vols, float *d_sinos,
                                      int32_t nbatch, float alpha, float beta, void *stream) {
    CT_TRACE("ct_project_batch");
    clear_error();
    CT_TRY(check_batch(g, nbatch, d_vols, d_sinos));
    if (nbatch == 0 || g->nrays == 0) return CT_OK;
    const size_t nv = (size_t)g->nvox, nr = (size_t)g->nrays;
    if (!batchable(g->pg)) {
        for (int32_t i = 0; i < nbatch; ++i)
            CT_TRY(ct_project(g, d_vols + i * nv, d_sinos + i * nr, alpha, beta, stream));
        return CT_OK;
    }
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws(st);
    float *vol_t = nullptr;
    CT_TRY(ws.alloc(&vol_t, (size_t)nbatch * nv));
    std::vector<BatchJob> jobs((size_t)nbatch);
    for (int32_t i = 0; i < nbatch; ++i) {
        CT_TRY(launch_transpose(g->pg, d_vols + i * nv, nullptr, vol_t + i * nv, nullptr, st));
        BatchJob &b = jobs[(size_t)i];
        b = BatchJob{};
        CT_TRY(batch_job_grid(g->pg, false, &b));
        b.in = vol_t + i * nv;
        b.out = d_sinos + i * nr;
        b.rho = nullptr;
        b.c.alpha = alpha;
        b.c.beta = beta;
        b.partials = nullptr;
        b.det_scale = nullptr;
    }
    return run_jobs(jobs, false, ws, st);
}

extern "C" ct_status ct_backproject_batch(const ct_geometry *g, const float *d_sinos,
                                          float *d_vols, int32_t nbatch, float alpha, float beta,
                                          void *stream) {
    CT_TRACE("ct_backproject_batch");
    clear_error();
    if (!g) return set_error(CT_ERR_INVALID_ARG, "geometry is NULL");
    if (nbatch < 0) return set_error(CT_ERR_INVALID_ARG, "nbatch must be >= 0");
    if (nbatch > 0 && !d_vols) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (nbatch > 0 && g->nrays > 0 && !d_sinos) return set_error(CT_ERR_INVALID_ARG, "NULL vector");
    if (nbatch == 0) return CT_OK;
    const size_t nv = (size_t)g->nvox, nr = (size_t)g->nrays;
    if (g->nrays == 0 || !batchable(g->pg) || g->deterministic) {
        for (int32_t i = 0; i < nbatch; ++i)
            CT_TRY(ct_backproject(g, g->nrays ? d_sinos + i * nr : nullptr, d_vols + i * nv, alpha,
                                  beta, stream));
        return CT_OK;
    }
    DeviceGuard dg(g->device);
    CT_TRY(dg.status());
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws(st);
    float *acc_t = nullptr;
    CT_TRY(ws.alloc(&acc_t, (size_t)nbatch * nv));
    CT_CUDA_TRY(cudaMemsetAsync(acc_t, 0, (size_t)nbatch * nv * sizeof(float), st));
    std::vector<BatchJob> jobs((size_t)nbatch);
    for (int32_t i = 0; i < nbatch; ++i) {
        BatchJob &b = jobs[(size_t)i];
        b = BatchJob{};
        CT_TRY(batch_job_grid(g->pg, true, &b));
        b.in = d_sinos + i * nr;
        b.out = acc_t + i * nv;
        b.rho = nullptr;
        b.c.alpha = alpha;
        b.c.beta = 0.f;
        b.partials = nullptr;
        b.det_scale = nullptr;
    }
    CT_TRY(run_jobs(jobs, true, ws, st));
    // the column-major accumulators hold all of A^T; the combine writes
    // out = beta out + acc (beta 0: out is not read)
    for (int32_t i = 0; i < nbatch; ++i)
        CT_TRY(launch_combine(g->pg, d_vols + i * nv, acc_t + i * nv, nullptr, nullptr, st, beta));
    return CT_OK;
}
