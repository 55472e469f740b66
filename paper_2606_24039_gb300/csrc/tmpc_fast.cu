// Host side of the shared-memory small-model path (tmpc_fast_api.h): arena
// sizes, occupancy queries and launches, dispatched per model through the
// kernel tables of tmpc_fast_di.cu, tmpc_fast_bicycle.cu and tmpc_fast_quad.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/tmpc.h"
#include "tmpc_direct.cuh"
#include "tmpc_fast.cuh"
#include "tmpc_fast_api.h"

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace tmpc {
namespace fast {

long long arena_floats_host(int model, int T, int policy, int cluster) {
    const int cl = cluster ? 1 : 0;
    switch (model) {
        case MODEL_DI: return arena_floats<MODEL_DI>(T, policy, cl);
        case MODEL_BICYCLE: return arena_floats<MODEL_BICYCLE>(T, policy, cl);
        case MODEL_QUAD: return arena_floats<MODEL_QUAD>(T, policy, cl);
    }
    return -1;
}

long long direct_ws_doubles(int model, int T) {
    switch (model) {
        case MODEL_DI: return (long long)T * DRec<MODEL_DI>::Stage;
        case MODEL_BICYCLE: return (long long)T * DRec<MODEL_BICYCLE>::Stage;
        case MODEL_QUAD: return (long long)T * DRec<MODEL_QUAD>::Stage;
    }
    return 0;
}

bool supported(int model) { return model == MODEL_DI || model == MODEL_BICYCLE || model == MODEL_QUAD; }

static const KernelTable* table_of(int model) {
    switch (model) {
        case MODEL_DI: return &kernel_table<MODEL_DI>();
        case MODEL_BICYCLE: return &kernel_table<MODEL_BICYCLE>();
        case MODEL_QUAD: return &kernel_table<MODEL_QUAD>();
    }
    return nullptr;
}

static const void* kernel_of(int model, int policy) {
    const KernelTable* t = table_of(model);
    return t ? t->solve[policy == kLDL ? 1 : 0] : nullptr;
}

cudaError_t prepare(int model, int policy, size_t smem_bytes, int threads, int* blocks_per_sm) {
    const void* k = kernel_of(model, policy);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem_bytes);
}

static const void* cluster_kernel_of(int model, int policy) {
    const KernelTable* t = table_of(model);
    return t ? t->cluster[policy == kLDL ? 1 : 0] : nullptr;
}

cudaError_t prepare_cluster(int model, int policy, int cl, int threads, int* max_clusters) {
    const void* k = cluster_kernel_of(model, policy);
    if (!k) return cudaErrorInvalidValue;
    if (cl > 8) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, k, &cfg);
}

cudaError_t launch_cluster(int model, int policy, int cl, int nclusters, int threads, cudaStream_t s,
                           const KLayout& L, const KOpts& o, const KParams& p, const KSol& out, float* gws,
                           long long gstride, const int* order, int count, const float* x0, int warm,
                           int* gflags) {
    const void* k = cluster_kernel_of(model, policy);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl * nclusters);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&L, (void*)&o, (void*)&p, (void*)&out, (void*)&gws, (void*)&gstride, (void*)&order,
                    (void*)&count, (void*)&x0, (void*)&warm, (void*)&gflags};
    return cudaLaunchKernelExC(&cfg, k, args);
}

static const void* bwd_kernel_of(int model, bool cluster) {
    const KernelTable* t = table_of(model);
    return t ? (cluster ? t->backward_cluster : t->backward) : nullptr;
}

cudaError_t prepare_backward(int model, int cl, size_t smem_bytes, int threads, int* per) {
    const void* k = bwd_kernel_of(model, cl > 0);
    if (!k) return cudaErrorInvalidValue;
    if (cl > 0) {
        if (cl > 8) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        *per = 1;
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k, threads, smem_bytes);
}

cudaError_t launch_backward(int model, int cl, int grid, int threads, size_t smem_bytes, cudaStream_t s,
                            const KLayout& L, const KOpts& o, const KParams& p, const KSol& sol, float* gws,
                            long long gstride, const int* order, int count, int* queue, const float* x0,
                            int* gflags, const float* dLdz, const float* dLdxi, const KGrads& g, double* dws,
                            long long dstride, int* dq_flag, int* dq_ctr, int nsm) {
    const void* k = bwd_kernel_of(model, cl > 0);
    if (!k) return cudaErrorInvalidValue;
    if (cl > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cl * grid);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {(void*)&L, (void*)&o, (void*)&p, (void*)&sol, (void*)&gws, (void*)&gstride, (void*)&order,
                        (void*)&count, (void*)&x0, (void*)&gflags, (void*)&dLdz, (void*)&dLdxi, (void*)&g,
                        (void*)&dws, (void*)&dstride};
        return cudaLaunchKernelExC(&cfg, k, args);
    }
    // CTA teams: instances that need the direct solve are flagged by the first pass,
    // swept by the warp kernel and finished by a second pass of the backward kernel
    // (dq_flag: one per instance, global index; dq_ctr: [1] sweep cursor, [2] queue
    // of the finishing pass; all zeroed by the caller)
    const bool direct = dws && dq_flag && dq_ctr && !((o.bwd_solver == 1 || o.bwd_solver == 3) && !o.exact_hessian);
    DirectQueue dq{direct ? dq_flag : nullptr};
    int finish = 0;
    const long long sf = (long long)(smem_bytes / sizeof(float));
    double* dw = direct ? dws : nullptr;
    void* args[] = {(void*)&L, (void*)&o, (void*)&p, (void*)&sol, (void*)&gws, (void*)&gstride, (void*)&order,
                    (void*)&count, (void*)&queue, (void*)&x0, (void*)&sf, (void*)&dLdz, (void*)&dLdxi, (void*)&g,
                    (void*)&dw, (void*)&dstride, (void*)&dq, (void*)&finish};
    cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem_bytes, s);
    if (e != cudaSuccess || !direct) return e;
    const KernelTable* t = table_of(model);
    const int* Np = p.N;
    const int* flg = dq_flag;
    int* cursor = dq_ctr + 1;
    int exact = o.exact_hessian ? 1 : 0;
    // one CTA of kDirectWarps warps on every SM (the occupancy limit): the sweeps are
    // bound by each SM's FP64 pipe, so the instances are spread over all SMs (the
    // warps take them from the cursor as they start), not packed eight to a CTA
    const int blocks = std::max(1, std::min(nsm, count));
    void* dargs[] = {(void*)&Np, (void*)&order, (void*)&count, (void*)&flg, (void*)&cursor, (void*)&dws,
                     (void*)&dstride, (void*)&exact};
    e = cudaLaunchKernel(t->direct, dim3(blocks), dim3(kDirectWarps * 32), dargs, 0, s);
    if (e != cudaSuccess) return e;
    finish = 1;
    int* q2 = dq_ctr + 2;
    void* fargs[] = {(void*)&L, (void*)&o, (void*)&p, (void*)&sol, (void*)&gws, (void*)&gstride, (void*)&order,
                     (void*)&count, (void*)&q2, (void*)&x0, (void*)&sf, (void*)&dLdz, (void*)&dLdxi, (void*)&g,
                     (void*)&dw, (void*)&dstride, (void*)&dq, (void*)&finish};
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), fargs, smem_bytes, s);
}

int backward_launches(int cl, const KOpts& o, bool have_dws) {
    if (cl > 0 || !have_dws || ((o.bwd_solver == 1 || o.bwd_solver == 3) && !o.exact_hessian)) return 1;
    return 3;
}

cudaError_t launch_plain(int model, int threads, cudaStream_t s, const KLayout& L, const KOpts& o, const KParams& p,
                         const KSol& out, float* gws, long long gstride, const int* order, int count,
                         const float* x0, int warm, PlainState* ps) {
    const KernelTable* t = table_of(model);
    if (!t) return cudaErrorInvalidValue;
    return t->plain(threads, s, L, o, p, out, gws, gstride, order, count, x0, warm, ps);
}

int plain_launches(int max_sqp, int max_admm) { return 2 + max_sqp * (2 + max_admm); }

cudaError_t launch(int model, int policy, int grid, int threads, size_t smem_bytes, cudaStream_t s,
                   const KLayout& L, const KOpts& o, const KParams& p, const KSol& out, float* gws,
                   long long gstride, const int* order, int count, int* queue, const float* x0, int warm) {
    const long long sf = (long long)(smem_bytes / sizeof(float));
    const void* k = kernel_of(model, policy);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&L, (void*)&o, (void*)&p, (void*)&out, (void*)&gws, (void*)&gstride, (void*)&order,
                    (void*)&count, (void*)&queue, (void*)&x0, (void*)&warm, (void*)&sf};
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem_bytes, s);
}

}  // namespace fast
}  // namespace tmpc
