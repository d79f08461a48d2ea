// k_edge_f32c.cu -- instantiations of the edge pass (k_edge.cuh) for FP32 storage, compensated
// FP32 sums
#include "k_edge.cuh"

namespace amgd {

cudaError_t launch_edge_f32_comp(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return edge_impl::dispatch_g<float, true>(sh, unit_w, a, s);
}

}  // namespace amgd
