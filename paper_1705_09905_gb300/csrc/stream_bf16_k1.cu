// stream_bf16_k1.cu -- streaming kernel variants for BF16 factors, residual weights (sparse CP fit, adjoint).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_bf16_k1(StreamParams &p, cudaStream_t s) {
    return launch_typed<__nv_bfloat16, 1>(p, s);
}

}  // namespace fcx
