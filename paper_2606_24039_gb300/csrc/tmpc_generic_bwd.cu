// Generic backward kernel: Algorithm 2 for one instance per CTA, instances
// popped from a device work queue.
#include "tmpc_generic.cuh"

namespace tmpc {

__global__ void __launch_bounds__(256, 2) backward_kernel(KLayout L, KOpts o, KParams p, KSol sol, float* ws, WsOff off,
                                const int* order, int count, int* queue, const float* x0, const float* dLdz,
                                const float* dLdxi, KGrads g, double* dws, long long dstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double dsh[kGenDirectScratch];
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
        backward_instance(c, o, sm, L, sol, i, dLdz, dLdxi, g, dws ? dws + (long long)i * dstride : nullptr, dsh);
    }
}

}  // namespace tmpc
