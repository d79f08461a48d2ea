// k_edge_f32.cu -- instantiations of the edge pass (k_edge.cuh) for FP32 storage
#include "k_edge.cuh"

namespace amgd {

cudaError_t launch_edge_f32(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return edge_impl::dispatch_g<float>(sh, unit_w, a, s);
}

}  // namespace amgd
