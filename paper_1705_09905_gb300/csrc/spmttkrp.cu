// spmttkrp.cu -- SpMTTKRP (Eq. 6), SpTTM (Eq. 3) and SpTTMc (Eq. 4) entry points and the
// dispatch of the streaming kernel (stream_kernel.cuh) by factor type and
// weight kind; the variants themselves are compiled in stream_*.cu.
#include <string.h>

#include "internal.cuh"

namespace fcx {

int launch_stream_kernel(StreamParams &p, int dtype, cudaStream_t s, int kind) {
    if (kind == 2) return dtype == FCOO_BF16 ? launch_stream_bf16_k2(p, s) : launch_stream_f32_k2(p, s);
    if (dtype == FCOO_BF16) return kind == 0 ? launch_stream_bf16_k0(p, s) : launch_stream_bf16_k1(p, s);
    return kind == 0 ? launch_stream_f32_k0(p, s) : launch_stream_f32_k1(p, s);
}

}  // namespace fcx

using namespace fcx;

static int check_common(const fcoo_t *X, int want_op, int dtype, int R, const void *out, const char *who) {
    if (!X) return fail(FCOO_ERR_INVALID_ARG, "%s: NULL handle", who);
    if (X->op != want_op) return fail(FCOO_ERR_INVALID_ARG, "%s: handle was built for the other operation", who);
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "%s: dtype=%d unknown", who, dtype);
    if (R < 1 || R > FCOO_MAX_RANK) return fail(FCOO_ERR_INVALID_ARG, "%s: R=%d outside 1..%d", who, R, FCOO_MAX_RANK);
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "%s: out is NULL", who);
    if (((uintptr_t)out & 3u) != 0) return fail(FCOO_ERR_INVALID_ARG, "%s: out is not 4-byte aligned", who);
    return FCOO_OK;
}

extern "C" int spmttkrp(const fcoo_t *X, const void *const *factors, int dtype, int R, float *out,
                        fcoo_stream_t stream) {
    clear_error();
    int st = check_common(X, FCOO_OP_MTTKRP, dtype, R, out, "spmttkrp");
    if (st) return st;
    if (!factors) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp: factors is NULL");
    for (int m = 0; m < X->nprod; ++m)
        if (!factors[X->prod_modes[m]])
            return fail(FCOO_ERR_INVALID_ARG, "spmttkrp: factors[%d] is NULL", X->prod_modes[m]);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rows = X->dims[X->mode];
    if (X->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(out, 0, (size_t)rows * R * 4, s));
        return FCOO_OK;
    }
    StreamParams p;
    stream_params_from(X, p);
    for (int m = 0; m < X->nprod; ++m) p.F[m] = factors[X->prod_modes[m]];
    p.out = out;
    p.R = R;
    p.out_rows = rows;
    return launch_stream_kernel(p, dtype, s);
}

extern "C" int spttm(const fcoo_t *X, const void *U, int dtype, int R, float *out, fcoo_stream_t stream) {
    clear_error();
    int st = check_common(X, FCOO_OP_TTM, dtype, R, out, "spttm");
    if (st) return st;
    if (!U) return fail(FCOO_ERR_INVALID_ARG, "spttm: U is NULL");
    if (X->nnz == 0) return FCOO_OK;
    StreamParams p;
    stream_params_from(X, p);
    p.F[0] = U;
    p.out = out;
    p.R = R;
    p.out_rows = X->nseg;
    return launch_stream_kernel(p, dtype, (cudaStream_t)stream);
}

extern "C" int spttmc(const fcoo_t *X, const void *const *factors, int dtype, int R, float *out,
                      fcoo_stream_t stream) {
    clear_error();
    if (!X) return fail(FCOO_ERR_INVALID_ARG, "spttmc: NULL handle");
    if (X->op != FCOO_OP_MTTKRP)
        return fail(FCOO_ERR_INVALID_ARG, "spttmc: the handle must be built with op = FCOO_OP_MTTKRP");
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "spttmc: dtype=%d unknown", dtype);
    if (R < 1) return fail(FCOO_ERR_INVALID_ARG, "spttmc: R=%d below 1", R);
    int64_t width = 1;
    for (int m = 0; m < X->nprod; ++m) {
        width *= R;
        if (width > FCOO_MAX_RANK)
            return fail(FCOO_ERR_UNSUPPORTED, "spttmc: output width R^%d above %d", X->nprod, FCOO_MAX_RANK);
    }
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "spttmc: out is NULL");
    if (((uintptr_t)out & 3u) != 0) return fail(FCOO_ERR_INVALID_ARG, "spttmc: out is not 4-byte aligned");
    if (!factors) return fail(FCOO_ERR_INVALID_ARG, "spttmc: factors is NULL");
    for (int m = 0; m < X->nprod; ++m)
        if (!factors[X->prod_modes[m]])
            return fail(FCOO_ERR_INVALID_ARG, "spttmc: factors[%d] is NULL", X->prod_modes[m]);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rows = X->dims[X->mode];
    if (X->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(out, 0, (size_t)rows * width * 4, s));
        return FCOO_OK;
    }
    StreamParams p;
    stream_params_from(X, p);
    for (int m = 0; m < X->nprod; ++m) p.F[m] = factors[X->prod_modes[m]];
    p.out = out;
    p.R = (int)width;
    p.Rin = R;
    p.out_rows = rows;
    return launch_stream_kernel(p, dtype, s, 2);
}
