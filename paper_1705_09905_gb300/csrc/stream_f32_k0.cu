// stream_f32_k0.cu -- streaming kernel variants for FP32 factors, value weights (SpMTTKRP / SpTTM).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_f32_k0(StreamParams &p, cudaStream_t s) {
    return launch_typed<float, 0>(p, s);
}

}  // namespace fcx
