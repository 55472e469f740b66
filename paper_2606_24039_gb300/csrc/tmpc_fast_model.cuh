// Instantiates the shared-memory kernels of one model (TMPC_FAST_MODEL) and
// publishes them in its kernel table; included once per model translation unit.
#pragma once
#include "tmpc_fast_kernels.cuh"

#ifndef TMPC_FAST_MODEL
#error "define TMPC_FAST_MODEL before including tmpc_fast_model.cuh"
#endif

namespace tmpc {
namespace fast {

namespace {
constexpr int kM = TMPC_FAST_MODEL;

// plain per-phase form: the host loop over the phases of Algorithm 1
cudaError_t launch_plain_model(int threads, cudaStream_t s, const KLayout& L, const KOpts& o, const KParams& p,
                               const KSol& out, float* gws, long long gstride, const int* order, int count,
                               const float* x0, int warm, PlainState* ps) {
    const dim3 g(count), b(threads);
    plain_init<kM><<<g, b, 0, s>>>(L, o, p, out, gws, gstride, order, count, x0, warm, ps);
    for (int it = 0; it < o.max_sqp; ++it) {
        plain_sqp_begin<kM><<<g, b, 0, s>>>(L, o, p, gws, gstride, order, count, x0, ps);
        for (int k = 1; k <= o.max_admm; ++k)
            plain_admm<kM><<<g, b, 0, s>>>(L, o, p, gws, gstride, order, count, x0, ps, k);
        plain_sqp_end<kM><<<g, b, 0, s>>>(L, o, p, gws, gstride, order, count, x0, ps, it);
    }
    plain_final<kM><<<g, b, 0, s>>>(L, o, p, out, gws, gstride, order, count, x0, ps);
    return cudaGetLastError();
}
}  // namespace

template <>
const KernelTable& kernel_table<TMPC_FAST_MODEL>() {
    static const KernelTable t = {
        {(const void*)solve_kernel<kM, kCR>, (const void*)solve_kernel<kM, kLDL>},
        {(const void*)solve_kernel_cluster<kM, kCR>, (const void*)solve_kernel_cluster<kM, kLDL>},
        (const void*)backward_kernel<kM>,
        (const void*)backward_kernel_cluster<kM>,
        (const void*)direct_kernel<kM>,
        &launch_plain_model};
    return t;
}

}  // namespace fast
}  // namespace tmpc
