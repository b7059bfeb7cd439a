// stream_bf16_k2.cu -- streaming kernel variants for BF16 factors with Kronecker output columns (SpTTMc).
#include "stream_kernel.cuh"

namespace fcx {

int launch_stream_bf16_k2(StreamParams &p, cudaStream_t s) {
    return launch_kron<__nv_bfloat16>(p, s);
}

}  // namespace fcx
