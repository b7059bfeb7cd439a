// capi.cu -- status plumbing, allocation hook and the handle queries of the
// libfcoo C ABI (fcoo_last_error, fcoo_info, fcoo_copy_layout, ...).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace fcx {

static thread_local char g_msg[512] = "";

void clear_error() { g_msg[0] = 0; }

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    int st = (e == cudaErrorMemoryAllocation) ? FCOO_ERR_NOMEM : FCOO_ERR_CUDA;
    cudaGetLastError();  // clear the sticky-free error state for the next call
    return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// FCOO_FAULT_ALLOC=k: the k-th device allocation of the process fails.
static std::atomic<long> g_alloc_count{0};
static long fault_at() {
    static long v = -2;
    if (v == -2) {
        const char *s = getenv("FCOO_FAULT_ALLOC");
        v = (s && *s) ? atol(s) : -1;
    }
    return v;
}

static bool inject_alloc_fault() {
    long k = fault_at();
    long n = ++g_alloc_count;
    return k > 0 && n == k;
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    if (bytes == 0) bytes = 256;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    if (bytes == 0) bytes = 256;
    return cudaMallocAsync(p, bytes, s);
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

void dev_free_async(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Two 32-bit indices (each < 65,536) -> one word of two 16-bit indices, the
// lower position in the low half.
__global__ void k_narrow_u16(const uint32_t *in, int64_t n2, uint32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 v = reinterpret_cast<const uint2 *>(in)[i];
        out[i] = (v.x & 0xffffu) | (v.y << 16);
    }
}

int device_sms(int dev) {
    static std::atomic<int> cache[kMaxDevices];
    if (dev < 0 || dev >= kMaxDevices) return num_sms();
    int n = cache[dev].load(std::memory_order_acquire);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cache[dev].store(n, std::memory_order_release);
    }
    return n;
}

void stream_params_from(const fcoo_t *X, StreamParams &p) {
    memset(&p, 0, sizeof(p));
    for (int m = 0; m < X->nprod; ++m) {
        p.pidx[m] = X->pidx[m];
        p.pidx16[m] = X->pidx16[m];
    }
    p.val = X->val;
    p.bf = X->bf;
    p.sf = X->sf;
    p.hcount = X->hcount;
    p.segrow = X->op == FCOO_OP_MTTKRP ? X->segkeys : nullptr;
    p.carry_val = X->carry_val;
    p.carry_seg = X->carry_seg;
    p.counter = X->counter;
    p.perm = X->perm;
    p.nnz = X->nnz;
    p.nseg = X->nseg;
    p.nprod = X->nprod;
    p.threadlen = X->threadlen;
    p.grid = X->max_grid;
}

}  // namespace fcx

using namespace fcx;

extern "C" {

const char *fcoo_last_error(void) { return g_msg; }

const char *fcoo_status_string(int status) {
    switch (status) {
        case FCOO_OK: return "FCOO_OK";
        case FCOO_ERR_INVALID_ARG: return "FCOO_ERR_INVALID_ARG";
        case FCOO_ERR_INDEX_RANGE: return "FCOO_ERR_INDEX_RANGE";
        case FCOO_ERR_DUPLICATE: return "FCOO_ERR_DUPLICATE";
        case FCOO_ERR_NOMEM: return "FCOO_ERR_NOMEM";
        case FCOO_ERR_CUDA: return "FCOO_ERR_CUDA";
        case FCOO_ERR_NOT_PD: return "FCOO_ERR_NOT_PD";
        case FCOO_ERR_NONFINITE: return "FCOO_ERR_NONFINITE";
        case FCOO_ERR_TIMEOUT: return "FCOO_ERR_TIMEOUT";
        case FCOO_ERR_UNSUPPORTED: return "FCOO_ERR_UNSUPPORTED";
        default: return "FCOO_ERR_UNKNOWN";
    }
}

int fcoo_version(void) { return 10000; }

int64_t fcoo_table2_bytes_ex(int nprod, int64_t nnz, int threadlen, int index_bytes) {
    if (nprod < 1 || nprod >= FCOO_MAX_MODES || nnz < 0 || threadlen < 1 || threadlen > 64 ||
        (threadlen & (threadlen - 1)) != 0 || (index_bytes != 4 && index_bytes != 2))
        return -1;
    int64_t npart = ceil_div(nnz, threadlen);
    return 4 * nnz + (int64_t)index_bytes * nprod * nnz + 4 * ceil_div(nnz, 32) + 4 * ceil_div(npart, 32);
}

int64_t fcoo_table2_bytes(int nprod, int64_t nnz, int threadlen) {
    return fcoo_table2_bytes_ex(nprod, nnz, threadlen, 4);
}

int fcoo_destroy(fcoo_t *X) {
    clear_error();
    if (!X) return FCOO_OK;
    cudaDeviceSynchronize();
    dev_free(X->segkeys);
    dev_free(X->grad_scratch);
    dev_free(X->gmap);
    dev_free(X->base);
    dev_free(X->base16);
    free(X);
    return FCOO_OK;
}

int fcoo_info(const fcoo_t *X, fcoo_info_t *info) {
    clear_error();
    if (!X || !info) return fail(FCOO_ERR_INVALID_ARG, "fcoo_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->nmodes = X->nmodes;
    info->mode = X->mode;
    info->op = X->op;
    info->threadlen = X->threadlen;
    info->nnz = X->nnz;
    info->nseg = X->nseg;
    info->nfib = X->nfib;
    for (int k = 0; k < X->nmodes; ++k) info->dims[k] = X->dims[k];
    info->nprod = X->nprod;
    info->nidx = X->nidx;
    for (int k = 0; k < X->nprod; ++k) info->prod_modes[k] = X->prod_modes[k];
    for (int k = 0; k < X->nidx; ++k) info->idx_modes[k] = X->idx_modes[k];
    info->bytes_val = X->bytes_val;
    info->bytes_pidx = X->bytes_pidx;
    info->bytes_bf = X->bytes_bf;
    info->bytes_sf = X->bytes_sf;
    info->bytes_table2 = X->bytes_val + X->bytes_pidx + X->bytes_bf + X->bytes_sf;
    info->bytes_segmap = X->bytes_segmap;
    info->bytes_aux = X->bytes_aux;
    info->bytes_scratch = X->bytes_scratch;
    info->bytes_pidx16 = X->base16 ? 2 * (int64_t)X->nprod * X->nnz : 0;
    return FCOO_OK;
}

int fcoo_copy_layout(const fcoo_t *X, uint32_t *perm, uint32_t *bf, uint32_t *sf, uint32_t *segkeys,
                     uint32_t *pidx, float *val, fcoo_stream_t stream) {
    clear_error();
    if (!X) return fail(FCOO_ERR_INVALID_ARG, "fcoo_copy_layout: NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    size_t n = (size_t)X->nnz;
    if (perm && n) FCOO_CUDA(cudaMemcpyAsync(perm, X->perm, n * 4, cudaMemcpyDefault, s));
    if (bf && n) FCOO_CUDA(cudaMemcpyAsync(bf, X->bf, ceil_div(n, 32) * 4, cudaMemcpyDefault, s));
    if (sf && n)
        FCOO_CUDA(cudaMemcpyAsync(sf, X->sf, ceil_div(ceil_div(n, X->threadlen), 32) * 4, cudaMemcpyDefault, s));
    if (segkeys && X->nseg)
        FCOO_CUDA(cudaMemcpyAsync(segkeys, X->segkeys, (size_t)X->nseg * X->nidx * 4, cudaMemcpyDefault, s));
    if (pidx && n)
        for (int m = 0; m < X->nprod; ++m)
            FCOO_CUDA(cudaMemcpyAsync(pidx + m * n, X->pidx[m], n * 4, cudaMemcpyDefault, s));
    if (val && n) FCOO_CUDA(cudaMemcpyAsync(val, X->val, n * 4, cudaMemcpyDefault, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    return FCOO_OK;
}

int fcoo_compress_indices(fcoo_t *X, fcoo_stream_t stream) {
    clear_error();
    if (!X) return fail(FCOO_ERR_INVALID_ARG, "fcoo_compress_indices: NULL handle");
    if (X->base16) return FCOO_OK;
    for (int m = 0; m < X->nprod; ++m)
        if (X->dims[X->prod_modes[m]] > 65536u)
            return fail(FCOO_ERR_UNSUPPORTED, "fcoo_compress_indices: product mode %d has dimension %u > 65536",
                        X->prod_modes[m], X->dims[X->prod_modes[m]]);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npad = X->npad;
    void *b = nullptr;
    FCOO_CUDA(dev_alloc(&b, (size_t)npad * 2 * X->nprod));
    uint16_t *out[FCOO_MAX_MODES] = {};
    for (int m = 0; m < X->nprod; ++m) out[m] = static_cast<uint16_t *>(b) + (size_t)m * npad;
    for (int m = 0; m < X->nprod; ++m) {
        const int64_t n2 = npad / 2;  // two indices per thread, npad is even
        k_narrow_u16<<<(unsigned)std::min<int64_t>(ceil_div(n2, 256), (int64_t)num_sms() * 16), 256, 0, s>>>(
            X->pidx[m], n2, reinterpret_cast<uint32_t *>(out[m]));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            dev_free(b);
            return cuda_fail(e, "fcoo_compress_indices");
        }
    }
    for (int m = 0; m < X->nprod; ++m) X->pidx16[m] = out[m];
    X->base16 = b;
    return FCOO_OK;
}

int fcoo_fibre_indices(const fcoo_t *X, uint32_t *keys, fcoo_stream_t stream) {
    clear_error();
    if (!X || (!keys && X->nseg)) return fail(FCOO_ERR_INVALID_ARG, "fcoo_fibre_indices: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (X->nseg)
        FCOO_CUDA(cudaMemcpyAsync(keys, X->segkeys, (size_t)X->nseg * X->nidx * 4, cudaMemcpyDefault, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    return FCOO_OK;
}

}  // extern "C"
