// k_edge.cu -- storage dispatch of the edge pass (kernels in k_edge.cuh,
// one translation unit per storage type)
#include "amgd_internal.cuh"

namespace amgd {

cudaError_t launch_edge_f64(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s);
cudaError_t launch_edge_f32(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s);
cudaError_t launch_edge_bf16(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s);

cudaError_t launch_edge(int storage, Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    switch (storage) {
    case ST_FP64: return launch_edge_f64(sh, unit_w, a, s);
    case ST_FP32: return launch_edge_f32(sh, unit_w, a, s);
    case ST_BF16: return launch_edge_bf16(sh, unit_w, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace amgd
