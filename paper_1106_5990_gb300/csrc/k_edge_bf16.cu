// k_edge_bf16.cu -- instantiations of the edge pass (k_edge.cuh) for BF16 storage, plain FP32
// sums; the FP64 row fixup
#include "k_edge.cuh"

namespace amgd {

cudaError_t launch_edge_bf16_comp(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s);

cudaError_t launch_edge_bf16(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.defer_count, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    e = a.compensated ? launch_edge_bf16_comp(sh, unit_w, a, s)
                      : edge_impl::dispatch_g<__nv_bfloat16, false>(sh, unit_w, a, s);
    if (e != cudaSuccess || a.n == 0) return e;
    if (sh.stage >= 2) edge_impl::k_edge_fixup<__nv_bfloat16, true><<<152, 256, 0, s>>>(a);
    else edge_impl::k_edge_fixup<__nv_bfloat16, false><<<152, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace amgd
