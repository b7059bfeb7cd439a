// fibre.cu -- the fibre tensor of an SpTTM handle (see fibre.cuh).
#include <stdio.h>

#include <algorithm>

#include "fibre.cuh"

namespace fcx {
namespace {

// coordinates (k0, k1, f) and value 1 of each fibre f
__global__ void k_fibre_coords(const uint32_t *keys, int64_t nfib, uint32_t *i0, uint32_t *i1, uint32_t *iff,
                               float *ones) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nfib; f += (int64_t)gridDim.x * blockDim.x) {
        i0[f] = keys[2 * f];
        i1[f] = keys[2 * f + 1];
        iff[f] = (uint32_t)f;
        ones[f] = 1.f;
    }
}

}  // namespace

int fibre_tensor_build(const fcoo_t *Xttm, int mode, int threadlen, cudaStream_t s, fcoo_t **out) {
    *out = nullptr;
    if (!Xttm || Xttm->op != FCOO_OP_TTM || Xttm->nmodes != 3 || mode < 0 || mode > 1)
        return fail(FCOO_ERR_INVALID_ARG, "fibre tensor: needs a 3-way SpTTM handle and mode 0 or 1");
    const int64_t nf = Xttm->nseg;
    void *tmp = nullptr;
    cudaError_t e = dev_alloc(&tmp, (size_t)(nf > 0 ? nf : 1) * 16);
    if (e != cudaSuccess) return cuda_fail(e, "fibre tensor: scratch");
    uint32_t *i0 = static_cast<uint32_t *>(tmp), *i1 = i0 + nf, *iff = i1 + nf;
    float *ones = reinterpret_cast<float *>(iff + nf);
    int st = FCOO_OK;
    if (nf > 0) {
        const int grid = (int)std::min<int64_t>(ceil_div(nf, 256), (int64_t)num_sms() * 8);
        k_fibre_coords<<<grid, 256, 0, s>>>(Xttm->segkeys, nf, i0, i1, iff, ones);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "k_fibre_coords");
    }
    if (st == FCOO_OK) {
        const uint32_t dims[3] = {Xttm->dims[Xttm->idx_modes[0]], Xttm->dims[Xttm->idx_modes[1]],
                                  (uint32_t)(nf > 0 ? nf : 1)};
        const uint32_t *idx[3] = {i0, i1, iff};
        st = fcoo_build(3, dims, nf, idx, ones, mode, FCOO_OP_MTTKRP, threadlen, (fcoo_stream_t)s, out);
        if (st != FCOO_OK) {
            char msg[400];
            snprintf(msg, sizeof(msg), "%s", fcoo_last_error());
            st = fail(st, "fibre tensor: %s", msg);
        }
    }
    dev_free(tmp);
    return st;
}

}  // namespace fcx
