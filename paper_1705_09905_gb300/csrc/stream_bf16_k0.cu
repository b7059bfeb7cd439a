// stream_bf16_k0.cu -- streaming kernel variants for BF16 factors, value weights (SpMTTKRP / SpTTM).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_bf16_k0(StreamParams &p, cudaStream_t s) {
    return launch_typed<__nv_bfloat16, 0>(p, s);
}

}  // namespace fcx
