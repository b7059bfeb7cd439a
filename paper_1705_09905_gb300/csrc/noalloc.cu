// noalloc.cu -- SpMTTKRP for callers that cannot allocate device memory.
//
// Same streaming kernel as spmttkrp; the only difference is where its
// scratch lives.  spmttkrp's per-CTA carry slots belong to the handle that
// fcoo_build allocated; here the layout arrives as caller-owned buffers and
// the carry slots are a fixed file-scope __device__ array, so no call
// allocates anything.
#include <atomic>
#include <string.h>

#include "internal.cuh"

namespace fcx {
namespace {

constexpr int kScratchCtas = FCOO_NOALLOC_MAX_CTAS;
constexpr int kScratchRank = FCOO_NOALLOC_MAX_RANK;
constexpr size_t kCarryValBytes = (size_t)2 * kScratchCtas * kScratchRank * sizeof(double);
constexpr size_t kCarrySegBytes = (size_t)2 * kScratchCtas * sizeof(int64_t);

// The scratch: carry values, then carry segment ids.  Its name in host code
// is only a stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCarryValBytes + kCarrySegBytes];

constexpr int kMaxDevices = 64;
std::atomic<void *> g_scratch_addr[kMaxDevices];

// Device address of the scratch on the current device, looked up once per
// device (the lookup may load the module, so it belongs before any capture).
int scratch_address(void **out) {
    int dev = 0;
    FCOO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_noalloc: device %d", dev);
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "spmttkrp_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return FCOO_OK;
}

bool pow2_threadlen(int t) { return t >= 1 && t <= 64 && (t & (t - 1)) == 0; }
bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace fcx

using namespace fcx;

extern "C" int spmttkrp_noalloc(const fcoo_view_t *v, const void *const *factors, int dtype, int R, float *out,
                                fcoo_stream_t stream) {
    clear_error();
    if (!v || !factors || !out) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: NULL argument");
    if (((uintptr_t)out & 3u) != 0) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: out is not 4-byte aligned");
    if (v->nmodes < 2 || v->nmodes > FCOO_MAX_MODES || v->mode < 0 || v->mode >= v->nmodes)
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: bad nmodes/mode");
    if (!pow2_threadlen(v->threadlen)) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: bad threadlen");
    if (v->nnz < 0 || v->nnz > FCOO_MAX_NNZ || v->nseg < 0 || (v->nnz > 0 && v->nseg < 1))
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: bad nnz/nseg");
    if (v->nseg > (int64_t)v->dims[v->mode])
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: nseg=%lld above dims[mode]=%u", (long long)v->nseg,
                    v->dims[v->mode]);
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: bad dtype");
    if (R < 1) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: R=%d", R);
    if (R > kScratchRank)
        return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_noalloc: R=%d above the fixed scratch limit %d", R, kScratchRank);
    const int nprod = v->nmodes - 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rows = v->dims[v->mode];
    if (v->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(out, 0, (size_t)rows * R * 4, s));
        return FCOO_OK;
    }
    if (!v->val || !v->bf || !v->sf || !v->segrow || !v->hcount || !al16(v->val))
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: missing or misaligned layout array");
    StreamParams p;
    memset(&p, 0, sizeof(p));
    for (int m = 0, k = 0; k < v->nmodes; ++k) {
        if (k == v->mode) continue;
        if (!v->pidx[m] || !al16(v->pidx[m]))
            return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: pidx[%d] missing or misaligned", m);
        if (!factors[k]) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_noalloc: factors[%d] is NULL", k);
        p.pidx[m] = v->pidx[m];
        p.F[m] = factors[k];
        ++m;
    }
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    p.val = v->val;
    p.bf = v->bf;
    p.sf = v->sf;
    p.hcount = v->hcount;
    p.segrow = v->segrow;
    p.carry_val = static_cast<double *>(scratch);
    p.carry_seg = reinterpret_cast<int64_t *>(static_cast<unsigned char *>(scratch) + kCarryValBytes);
    p.nnz = v->nnz;
    p.nseg = v->nseg;
    p.nprod = nprod;
    p.threadlen = v->threadlen;
    p.grid = kScratchCtas;  // the launch never uses more CTAs than the scratch holds
    p.out = out;
    p.R = R;
    p.out_rows = rows;
    return launch_stream_kernel(p, dtype, s);
}
