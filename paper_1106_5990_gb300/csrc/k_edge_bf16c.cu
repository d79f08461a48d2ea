// k_edge_bf16c.cu -- instantiations of the edge pass (k_edge.cuh) for BF16 storage, compensated
// FP32 sums
#include "k_edge.cuh"

namespace amgd {

cudaError_t launch_edge_bf16_comp(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return edge_impl::dispatch_g<__nv_bfloat16, true>(sh, unit_w, a, s);
}

}  // namespace amgd
