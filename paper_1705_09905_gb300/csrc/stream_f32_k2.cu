// stream_f32_k2.cu -- streaming kernel variants for FP32 factors with Kronecker output columns (SpTTMc).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_f32_k2(StreamParams &p, cudaStream_t s) {
    return launch_kron<float>(p, s);
}

}  // namespace fcx
