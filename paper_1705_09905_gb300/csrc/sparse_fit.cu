// sparse_fit.cu -- differentiation built on the one-shot product of Eq. 6.
//
// kind 0, sparse CP fit over the observed entries:
//   e(p) = sum_r prod_k F_k(idx_k(p), r) - x(p),  loss = 1/2 sum e(p)^2
//   dF_n(i,:) = sum_{p: idx_n(p) = i} e(p) prod_{k != n} F_k(idx_k(p), :)
// The first requested dF_n is one pass of the streaming kernel over the
// mode-n F-COO copy with residual weights: the segment's own row F_n(i,:) is
// loaded once per segment, e(p) is a group-wide dot product per nonzero, and
// e(p) times the Hadamard product of the gathered rows is reduced per segment
// exactly like SpMTTKRP.  The same pass writes the loss partials and e itself,
// in its own F-COO order (sequential stores).  Every other dF_m is then a
// plain SpMTTKRP of the mode-m copy whose value stream is e gathered into
// mode-m order through a position map built once per pair of handles (e is
// the same for every mode): one 4-byte gather per nonzero instead of
// recomputing the dot product.
// kind 1, adjoint of M = SpMTTKRP_mode(X, F) for a cotangent G = dL/dM:
//   dF_k = SpMTTKRP_k(X, F with F_mode := G)        (plain value-weighted pass)
//   dval(p) = <G(idx_mode(p), :), prod_{k != mode} F_k(idx_k(p), :)>
//                                                   (residual pass, no output rows)
#include <string.h>

#include <algorithm>

#include "internal.cuh"

namespace fcx {
namespace {

__global__ void k_half_sum(const double *part, int n, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += 256) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * red[0];
}

// w[p] = e[map[p]] for p < nnz, four independent loads in flight per thread
__global__ void k_gather_vals(const float *e, const uint32_t *map, int64_t nnz, float *w) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; p + 3 * stride < nnz; p += 4 * stride) {
        uint32_t m[4];
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) m[u] = __ldg(map + p + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldg(e + m[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) w[p + u * stride] = v[u];
    }
    for (; p < nnz; p += stride) w[p] = __ldg(e + __ldg(map + p));
}

// inv[perm[p]] = p for p < nnz (the caller's COO position -> F-COO position)
__global__ void k_invert_perm(const uint32_t *perm, int64_t nnz, uint32_t *inv) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        inv[perm[p]] = (uint32_t)p;
}

// out[perm[p]] = sign * in[p] for p < nnz
__global__ void k_scatter_scaled(const float *in, const uint32_t *perm, int64_t nnz, float sign, float *out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        out[perm[p]] = sign * in[p];
}

unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * 1024));
}

int check_handles(const fcoo_t *const *Xn, int &nmodes, const char *who) {
    if (!Xn || !Xn[0]) return fail(FCOO_ERR_INVALID_ARG, "%s: Xn or Xn[0] is NULL", who);
    nmodes = Xn[0]->nmodes;
    for (int n = 0; n < nmodes; ++n) {
        const fcoo_t *X = Xn[n];
        if (!X) return fail(FCOO_ERR_INVALID_ARG, "%s: Xn[%d] is NULL", who, n);
        if (X->op != FCOO_OP_MTTKRP || X->mode != n || X->nmodes != nmodes)
            return fail(FCOO_ERR_INVALID_ARG, "%s: Xn[%d] is not an SpMTTKRP handle for mode %d", who, n, n);
        if (X->nnz != Xn[0]->nnz) return fail(FCOO_ERR_INVALID_ARG, "%s: handles hold different tensors", who);
        for (int k = 0; k < nmodes; ++k)
            if (X->dims[k] != Xn[0]->dims[k]) return fail(FCOO_ERR_INVALID_ARG, "%s: handles differ in dims", who);
    }
    return FCOO_OK;
}

// Residual-weighted pass over handle X: target rows T, product rows from
// `factors` (indexed by mode), optional output rows, loss partials, dvals.
int residual_pass(const fcoo_t *X, const void *const *factors, const void *T, int dtype, int R, float *out,
                  bool with_loss, float *dvals, float dsign, int sub_val, cudaStream_t s, int *grid,
                  int dvals_fcoo = 0) {
    StreamParams p;
    stream_params_from(X, p);
    for (int m = 0; m < X->nprod; ++m) p.F[m] = factors[X->prod_modes[m]];
    p.out = out;
    p.R = R;
    p.out_rows = X->dims[X->mode];
    p.T = T;
    p.dvals = dvals;
    p.dvals_fcoo = dvals_fcoo;
    p.dsign = dsign;
    p.sub_val = sub_val;
    p.loss_part = with_loss ? X->red_part : nullptr;
    int rc = launch_stream_kernel(p, dtype, s, 1);
    *grid = p.grid;
    return rc;
}

}  // namespace
}  // namespace fcx

using namespace fcx;

extern "C" int spmttkrp_backward(const fcoo_t *const *Xn, const void *const *factors, int dtype, int R,
                                 const float *gradM, int kind, int mode, float *const *dfactors, float *dvals,
                                 double *loss, fcoo_stream_t stream) {
    clear_error();
    int nmodes = 0;
    int rc = check_handles(Xn, nmodes, "spmttkrp_backward");
    if (rc) return rc;
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: bad dtype");
    if (R < 1 || R > FCOO_MAX_RANK) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: R=%d outside 1..%d", R, FCOO_MAX_RANK);
    if (!factors) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: factors is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nnz = Xn[0]->nnz;
    if (kind == 0) {
        for (int k = 0; k < nmodes; ++k)
            if (!factors[k]) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: factors[%d] is NULL", k);
        if (nnz == 0) {
            for (int n = 0; n < nmodes; ++n)
                if (dfactors && dfactors[n])
                    FCOO_CUDA(cudaMemsetAsync(dfactors[n], 0, (size_t)Xn[0]->dims[n] * R * 4, s));
            if (loss) FCOO_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
            return FCOO_OK;
        }
        bool first = true;
        int loss_grid = 0;
        const fcoo_t *loss_X = nullptr;
        int nwant = 0;
        for (int n = 0; n < nmodes; ++n) nwant += (dfactors && dfactors[n]) ? 1 : 0;
        float *ebuf = nullptr, *wbuf = nullptr;
        for (int n = 0; n < nmodes; ++n) {
            float *out = dfactors ? dfactors[n] : nullptr;
            if (!out) continue;
            if (first) {
                int grid = 0;
                if (nwant > 1) {
                    // e in this handle's F-COO order, kept for the other modes
                    fcoo_t *Xs = const_cast<fcoo_t *>(Xn[n]);
                    if (!Xs->grad_scratch) {
                        void *q = nullptr;
                        FCOO_CUDA(dev_alloc(&q, (size_t)Xs->npad * 12));
                        Xs->grad_scratch = (float *)q;
                        FCOO_CUDA(cudaMemsetAsync(q, 0, (size_t)Xs->npad * 12, s));
                    }
                    ebuf = Xs->grad_scratch;
                    wbuf = ebuf + Xs->npad;
                    rc = residual_pass(Xs, factors, factors[n], dtype, R, out, loss != nullptr, ebuf, 1.0f, 1, s,
                                       &grid, 1);
                } else {
                    rc = residual_pass(Xn[n], factors, factors[n], dtype, R, out, loss != nullptr, dvals, -1.0f, 1,
                                       s, &grid);
                }
                if (rc) return rc;
                loss_grid = grid;
                loss_X = Xn[n];
                first = false;
                continue;
            }
            // dF_n = SpMTTKRP_n with the values e gathered into mode-n order
            fcoo_t *Xm = const_cast<fcoo_t *>(Xn[n]);
            if (!Xm->gmap || Xm->gmap_src != loss_X->uid) {
                if (!Xm->gmap) {
                    void *q = nullptr;
                    FCOO_CUDA(dev_alloc(&q, (size_t)Xm->npad * 4));
                    Xm->gmap = (uint32_t *)q;
                }
                uint32_t *inv = reinterpret_cast<uint32_t *>(ebuf + 2 * loss_X->npad);
                k_invert_perm<<<grid_for(nnz), 256, 0, s>>>(loss_X->perm, nnz, inv);
                FCOO_CUDA(cudaGetLastError());
                k_gather_vals<<<grid_for(nnz), 256, 0, s>>>(reinterpret_cast<const float *>(inv), Xm->perm, nnz,
                                                            reinterpret_cast<float *>(Xm->gmap));
                FCOO_CUDA(cudaGetLastError());
                Xm->gmap_src = loss_X->uid;
            }
            k_gather_vals<<<grid_for(nnz), 256, 0, s>>>(ebuf, Xm->gmap, nnz, wbuf);
            FCOO_CUDA(cudaGetLastError());
            StreamParams p;
            stream_params_from(Xm, p);
            for (int m = 0; m < Xm->nprod; ++m) p.F[m] = factors[Xm->prod_modes[m]];
            p.val = wbuf;
            p.out = out;
            p.R = R;
            p.out_rows = Xm->dims[n];
            rc = launch_stream_kernel(p, dtype, s, 0);
            if (rc) return rc;
        }
        if (ebuf && dvals) {
            k_scatter_scaled<<<grid_for(nnz), 256, 0, s>>>(ebuf, loss_X->perm, nnz, -1.0f, dvals);
            FCOO_CUDA(cudaGetLastError());
        }
        if (first && (loss || dvals)) {  // no gradient asked for: one loss / dvals pass
            rc = residual_pass(Xn[0], factors, factors[0], dtype, R, nullptr, loss != nullptr, dvals, -1.0f, 1, s,
                               &loss_grid);
            if (rc) return rc;
            loss_X = Xn[0];
        }
        if (loss) {
            k_half_sum<<<1, 256, 0, s>>>(loss_X->red_part, loss_grid, loss);
            FCOO_CUDA(cudaGetLastError());
        }
        return FCOO_OK;
    }
    if (kind != 1) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: kind=%d unknown", kind);
    if (mode < 0 || mode >= nmodes) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: mode=%d out of range", mode);
    if (!gradM) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: gradM is NULL");
    if (dtype != FCOO_F32)
        return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_backward: the adjoint (kind 1) takes float32 factors");
    for (int k = 0; k < nmodes; ++k)
        if (k != mode && !factors[k]) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_backward: factors[%d] is NULL", k);
    // factor list with F_mode replaced by the cotangent
    const void *fl[FCOO_MAX_MODES];
    for (int k = 0; k < nmodes; ++k) fl[k] = k == mode ? (const void *)gradM : factors[k];
    for (int k = 0; k < nmodes; ++k) {
        if (k == mode || !dfactors || !dfactors[k]) continue;
        if (nnz == 0) {
            FCOO_CUDA(cudaMemsetAsync(dfactors[k], 0, (size_t)Xn[0]->dims[k] * R * 4, s));
            continue;
        }
        StreamParams p;
        stream_params_from(Xn[k], p);
        for (int m = 0; m < Xn[k]->nprod; ++m) p.F[m] = fl[Xn[k]->prod_modes[m]];
        p.out = dfactors[k];
        p.R = R;
        p.out_rows = Xn[k]->dims[k];
        rc = launch_stream_kernel(p, dtype, s, 0);
        if (rc) return rc;
    }
    if (dvals && nnz > 0) {
        int grid = 0;
        rc = residual_pass(Xn[mode], factors, gradM, dtype, R, nullptr, false, dvals, 1.0f, 0, s, &grid);
        if (rc) return rc;
    }
    return FCOO_OK;
}

extern "C" int sparse_cp_loss(const fcoo_t *X, const void *const *factors, int dtype, int R, double *loss,
                              fcoo_stream_t stream) {
    clear_error();
    if (!X || !factors || !loss) return fail(FCOO_ERR_INVALID_ARG, "sparse_cp_loss: NULL argument");
    if (X->op != FCOO_OP_MTTKRP) return fail(FCOO_ERR_INVALID_ARG, "sparse_cp_loss: needs an SpMTTKRP handle");
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "sparse_cp_loss: bad dtype");
    if (R < 1 || R > FCOO_MAX_RANK) return fail(FCOO_ERR_INVALID_ARG, "sparse_cp_loss: R=%d outside 1..%d", R, FCOO_MAX_RANK);
    for (int k = 0; k < X->nmodes; ++k)
        if (!factors[k]) return fail(FCOO_ERR_INVALID_ARG, "sparse_cp_loss: factors[%d] is NULL", k);
    cudaStream_t s = (cudaStream_t)stream;
    if (X->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
        return FCOO_OK;
    }
    int grid = 0;
    int rc = residual_pass(X, factors, factors[X->mode], dtype, R, nullptr, true, nullptr, -1.0f, 1, s, &grid);
    if (rc) return rc;
    k_half_sum<<<1, 256, 0, s>>>(X->red_part, grid, loss);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}
