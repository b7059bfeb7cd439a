// stream_f32_k1.cu -- streaming kernel variants for FP32 factors, residual weights (sparse CP fit, adjoint).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_f32_k1(StreamParams &p, cudaStream_t s) {
    return launch_typed<float, 1>(p, s);
}

}  // namespace fcx
