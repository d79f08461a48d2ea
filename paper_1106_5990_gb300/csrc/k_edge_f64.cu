// k_edge_f64.cu -- instantiations of the edge pass (k_edge.cuh) for FP64 storage, FP64 sums
#include "k_edge.cuh"

namespace amgd {

cudaError_t launch_edge_f64(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return edge_impl::dispatch_g<double, false>(sh, unit_w, a, s);
}

}  // namespace amgd
