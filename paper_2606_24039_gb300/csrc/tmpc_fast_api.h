// Host interface of the shared-memory small-model kernels (tmpc_fast.cu).
#pragma once
#include <cuda_runtime.h>

#include "tmpc_backward.cuh"
#include "tmpc_solver.cuh"

namespace tmpc {
namespace fast {

// per-instance state of the plain per-phase form (between launches)
struct PlainState {
    float rho, rp, rd, alpha_last;
    int admm_total, nfact, sqp_done;
    int ls_hist[2];
    int flags[4];
};

// factorisation policies of the shared-memory kernels
constexpr int kPolicyCR = 0, kPolicyLDL = 1;
// floats of per-instance storage needed by the shared-memory path for T stages
// (cluster != 0: the arena of a cluster team, with its exchange area)
long long arena_floats_host(int model, int T, int policy, int cluster = 0);
// models handled by the shared-memory path
bool supported(int model);
// set the dynamic shared-memory limit of the model's kernel and query its occupancy
cudaError_t prepare(int model, int policy, size_t smem_bytes, int threads, int* blocks_per_sm);
// launch the persistent kernel over `count` instances listed in `order`
cudaError_t launch(int model, int policy, int grid, int threads, size_t smem_bytes, cudaStream_t s, const KLayout& L,
                   const KOpts& o, const KParams& p, const KSol& out, float* gws, long long gstride,
                   const int* order, int count, int* queue, const float* x0, int warm);

// thread-block-cluster variant (one cluster of `cl` CTAs per instance, global arenas)
cudaError_t prepare_cluster(int model, int policy, int cl, int threads, int* max_clusters);
cudaError_t launch_cluster(int model, int policy, int cl, int nclusters, int threads, cudaStream_t s,
                           const KLayout& L, const KOpts& o, const KParams& p, const KSol& out, float* gws,
                           long long gstride, const int* order, int count, const float* x0, int warm,
                           int* gflags);

// backward kernels (Algorithm 2) of the shared-memory path, cyclic-reduction policy;
// cl > 0: one cluster of cl CTAs per instance (grid = clusters)
cudaError_t prepare_backward(int model, int cl, size_t smem_bytes, int threads, int* per);
cudaError_t launch_backward(int model, int cl, int grid, int threads, size_t smem_bytes, cudaStream_t s,
                            const KLayout& L, const KOpts& o, const KParams& p, const KSol& sol, float* gws,
                            long long gstride, const int* order, int count, int* queue, const float* x0,
                            int* gflags, const float* dLdz, const float* dLdxi, const KGrads& g, double* dws,
                            long long dstride, int* dq_flag, int* dq_ctr, int nsm);
// kernels launch_backward enqueues (1, or 3 when the direct solve may run: the backward
// pass, the sweep kernel and the finishing pass)
int backward_launches(int cl, const KOpts& o, bool have_dws);
// doubles of the direct backward's FP64 workspace per instance of T stages
long long direct_ws_doubles(int model, int T);

// plain per-phase form: one launch per phase, fixed counts, one CTA per instance,
// global arenas; kernels launched on s in host order (plain_launches of them)
cudaError_t launch_plain(int model, int threads, cudaStream_t s, const KLayout& L, const KOpts& o, const KParams& p,
                         const KSol& out, float* gws, long long gstride, const int* order, int count,
                         const float* x0, int warm, PlainState* ps);
int plain_launches(int max_sqp, int max_admm);

// Kernels of one model (each model's kernels live in a translation unit of their
// own; the host code above dispatches through these tables).
struct KernelTable {
    const void* solve[2];     // persistent kernel, policy kCR / kLDL
    const void* cluster[2];   // one thread-block cluster per instance, kCR / kLDL
    const void* backward;     // persistent backward kernel (cyclic reduction)
    const void* backward_cluster;
    const void* direct;       // sweeps of the direct backward, one warp per instance
    cudaError_t (*plain)(int threads, cudaStream_t s, const KLayout& L, const KOpts& o, const KParams& p,
                         const KSol& out, float* gws, long long gstride, const int* order, int count,
                         const float* x0, int warm, PlainState* ps);
};
template <int M>
const KernelTable& kernel_table();
template <> const KernelTable& kernel_table<MODEL_DI>();
template <> const KernelTable& kernel_table<MODEL_BICYCLE>();
template <> const KernelTable& kernel_table<MODEL_QUAD>();

}  // namespace fast
}  // namespace tmpc
