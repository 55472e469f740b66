// Generic forward kernel: Algorithm 1 around Algorithm 3, one CTA per instance,
// instances popped from a device work queue in longest-first order.
#include "tmpc_generic.cuh"

namespace tmpc {

__global__ void __launch_bounds__(256, 2) solve_kernel(KLayout L, KOpts o, KParams p, KSol out, float* ws, WsOff off,
                             const int* order, int count, int* queue, const float* x0, int warm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const Smem sm = carve_smem(smem_raw, L);
    block_stream_init(sm.mbar, sm.flags + 12, o.wait_polls, o.force_timeout);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_item;
        __syncthreads();
        if (q >= count) break;
        const int i = order[q];
        const Ctx c = make_ctx(L, p, ws, off, i, x0, sm.vs);
        solve_instance(c, o, sm, L, out, i, warm);
    }
}

}  // namespace tmpc
