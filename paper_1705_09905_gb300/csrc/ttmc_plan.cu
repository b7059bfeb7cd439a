// ttmc_plan.cu -- SpTTMc of a 3-way tensor by fibres: Eq. 4 regrouped.
//
// For index mode n, product modes a < b, Eq. 4 reads
//   Y(i, r_a * R + r_b) = sum_{(i,j,k)} X(i,j,k) U_a(j, r_a) U_b(k, r_b).
// Summing first over k along each mode-b fibre (i, j) gives the SpTTM of
// Eq. 3 along mode b,
//   T(f, :) = sum_k X(i,j,k) U_b(k, :)      for fibre f = (i, j),
// and then
//   Y(i, r_a * R + r_b) = sum_{fibres f of slice i} U_a(j_f, r_a) T(f, r_b),
// which is Eq. 4 again, on the 3-way "fibre tensor" X'(i, j_f, f) = 1 with
// factors U_a and T (fibre.cu).  A nonzero then costs R FMAs (plus R^2 per fibre)
// instead of R^2: fewer operations wherever fibres hold more than one
// nonzero.  Both passes are the streaming kernel: SpTTM (kind 0, one
// product mode) into T, then the Kronecker-column kind over X'.
#include <stdio.h>

#include <algorithm>
#include <new>

#include "fibre.cuh"

struct fcoo_ttmc_plan {
    const fcoo_t *Xttm;  // SpTTM handle along mode b (not owned)
    fcoo_t *Xf;          // the fibre tensor X'(k0, k1, f), an SpMTTKRP handle on mode `pos`
    int mode, a, b, R;
    int pos;             // position of `mode` among the SpTTM handle's index modes
    int64_t nfib;
    float *T;  // nfib x R fibre sums
};

using namespace fcx;

extern "C" int spttmc_plan_create(const fcoo_t *Xttm, int mode, int R, int threadlen, fcoo_ttmc_plan_t **plan,
                                  fcoo_stream_t stream) {
    clear_error();
    if (!plan) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_create: plan is NULL");
    *plan = nullptr;
    if (!Xttm) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_create: NULL handle");
    if (Xttm->op != FCOO_OP_TTM || Xttm->nmodes != 3)
        return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_create: needs a 3-way handle built with op = FCOO_OP_TTM");
    if (mode < 0 || mode > 2) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_create: mode=%d outside 0..2", mode);
    const int b = mode == 2 ? 1 : 2;  // the last product mode
    const int a = 3 - mode - b;       // the first
    if (Xttm->mode != b)
        return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_create: SpTTMc on mode %d needs the SpTTM handle along mode %d",
                    mode, b);
    if (R < 1 || (int64_t)R * R > FCOO_MAX_RANK)
        return fail(FCOO_ERR_UNSUPPORTED, "spttmc_plan_create: R=%d outside 1..16", R);
    cudaStream_t s = (cudaStream_t)stream;
    fcoo_ttmc_plan_t *P = new (std::nothrow) fcoo_ttmc_plan_t();
    if (!P) return fail(FCOO_ERR_NOMEM, "spttmc_plan_create: host allocation failed");
    P->Xttm = Xttm;
    P->mode = mode;
    P->a = a;
    P->b = b;
    P->R = R;
    P->nfib = Xttm->nseg;
    const int64_t nf = P->nfib;
    // the fibre tuples hold (index modes ascending) = mode and a: the fibre
    // tensor's rows are the coordinate of `mode`
    P->pos = Xttm->idx_modes[0] == mode ? 0 : 1;
    int st = fibre_tensor_build(Xttm, P->pos, threadlen, s, &P->Xf);
    cudaError_t e;
    if (st == FCOO_OK && nf > 0) {
        e = dev_alloc(reinterpret_cast<void **>(&P->T), (size_t)nf * R * 4);
        if (e != cudaSuccess) st = cuda_fail(e, "spttmc_plan_create: fibre sums");
    }
    if (st != FCOO_OK) {
        if (P->Xf) fcoo_destroy(P->Xf);
        dev_free(P->T);
        delete P;
        return st;
    }
    *plan = P;
    return FCOO_OK;
}

extern "C" int spttmc_plan_run(const fcoo_ttmc_plan_t *P, const void *const *factors, int dtype, float *out,
                               fcoo_stream_t stream) {
    clear_error();
    if (!P) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_run: NULL plan");
    if (!factors || !factors[P->a] || !factors[P->b])
        return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_run: factors[%d] and factors[%d] are required", P->a, P->b);
    if (dtype != FCOO_F32) return fail(FCOO_ERR_UNSUPPORTED, "spttmc_plan_run: FP32 factors only");
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_run: out is NULL");
    const int R = P->R;
    if (P->nfib == 0) {
        FCOO_CUDA(cudaMemsetAsync(out, 0, (size_t)P->Xttm->dims[P->mode] * R * R * 4, (cudaStream_t)stream));
        return FCOO_OK;
    }
    // pass 1: fibre sums along mode b (Eq. 3)
    int st = spttm(P->Xttm, factors[P->b], FCOO_F32, R, P->T, stream);
    if (st != FCOO_OK) return st;
    // pass 2: Eq. 4 over the fibre tensor, factors U_a and the fibre sums
    const void *f2[3] = {nullptr, nullptr, P->T};
    f2[1 - P->pos] = factors[P->a];
    return spttmc(P->Xf, f2, FCOO_F32, R, out, stream);
}

extern "C" int spttmc_plan_destroy(fcoo_ttmc_plan_t *P) {
    clear_error();
    if (!P) return FCOO_OK;
    if (P->Xf) fcoo_destroy(P->Xf);
    dev_free(P->T);
    delete P;
    return FCOO_OK;
}

extern "C" int spttmc_plan_info(const fcoo_ttmc_plan_t *P, int64_t *nfib, int64_t *device_bytes) {
    clear_error();
    if (!P) return fail(FCOO_ERR_INVALID_ARG, "spttmc_plan_info: NULL plan");
    if (nfib) *nfib = P->nfib;
    if (device_bytes) {
        fcoo_info_t inf;
        int64_t b = P->nfib * P->R * 4;
        if (P->Xf && fcoo_info(P->Xf, &inf) == FCOO_OK)
            b += inf.bytes_table2 + inf.bytes_segmap + inf.bytes_aux + inf.bytes_scratch;
        *device_bytes = b;
    }
    return FCOO_OK;
}
