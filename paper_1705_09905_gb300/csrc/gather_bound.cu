// gather_bound.cu -- the gather-only bound of SpMTTKRP on a 3-way tensor
// (Eq. 6; Sec. IV-D on reading the factor rows through the read-only cache).
//
// SpMTTKRP of mode n reads, per nonzero, the row C(k,:) of the last product
// mode and, where a fibre (or an output row) starts, the row B(j,:) of the
// first.  On GB300 those row reads, not the HBM stream, set the rate of the
// streaming kernel.  spmttkrp_gather_bound issues exactly those row reads, in
// the same lane layout (groups of R/8 lanes, eight columns per lane) and the
// same order along each run, and nothing else: no products, no reduction, no
// output.  Its time is the bound the gathers alone set on SpMTTKRP for this
// tensor and these factors; the ratio of the two times is the fraction of that
// bound the full kernel reaches.
//
// Layout: the F-COO streams of the handle (product-mode index streams, padded
// to a multiple of kPad entries, and the segment-head bit words).  Each group
// takes a contiguous range of 32-nonzero chunks and copies each chunk's B and
// C indices and head word into its own shared-memory buffer with cp.async,
// one chunk ahead (two buffers).  Row loads go into register rings (NF C rows
// and NF B rows per lane); each ring slot is read before it is reused, so
// that the loads stay in flight concurrently and complete within the kernel.
#include <algorithm>

#include "internal.cuh"

namespace fcx {
namespace {

constexpr unsigned kAll = 0xffffffffu;

struct GatherParams {
    const uint32_t *jidx, *kidx;  // first / last product-mode index streams
    const uint32_t *bf;           // segment-head bit words
    const void *B, *C;            // factor rows (dtype), R columns each
    int64_t nnz;
    int64_t cpg;                  // chunks of 32 nonzeros per group
    int R;
    unsigned long long *count;    // rows loaded
};

// eight consecutive factor elements as raw 32-bit words, loaded only where f
// holds (unspecified elsewhere); fold() reads every word, so that all of a
// load's registers stay its own until the slot is reused
template <typename TF>
struct Piece;
template <>
struct Piece<float> {
    uint32_t w[8];
    __device__ __forceinline__ uint32_t fold() const {
        return (w[0] ^ w[1] ^ w[2]) ^ (w[3] ^ w[4] ^ w[5]) ^ (w[6] ^ w[7]);
    }
    __device__ __forceinline__ void load_if(const void *p, bool f) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %9, 0;\n\t"
            "@q ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t}"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
            : "l"(p), "r"((unsigned)f));
    }
};
template <>
struct Piece<__nv_bfloat16> {
    uint32_t w[4];
    __device__ __forceinline__ uint32_t fold() const { return (w[0] ^ w[1]) ^ (w[2] ^ w[3]); }
    __device__ __forceinline__ void load_if(const void *p, bool f) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
            "@q ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];\n\t}"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
            : "l"(p), "r"((unsigned)f));
    }
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// shared memory of one group: two chunk buffers of 32 C indices, 32 B
// indices and the head word (padded to 16 bytes)
constexpr int kBufWords = 32 + 32 + 4;
constexpr int kGroupBytes = 2 * kBufWords * 4;

template <typename TF, int LPR, int NF>
__global__ void __launch_bounds__(kThreads, 2) k_gather_bound(const GatherParams q) {
    extern __shared__ __align__(16) uint32_t s_idx[];
    const int lane = threadIdx.x & 31;
    const int lig = lane & (LPR - 1);
    const int g = threadIdx.x / LPR;
    const int64_t group = (int64_t)blockIdx.x * (kThreads / LPR) + g;
    const int64_t nchunk = (q.nnz + 31) / 32;
    const int64_t cbeg = group * q.cpg, cend = min(cbeg + q.cpg, nchunk);
    const int64_t rowb = (int64_t)q.R * sizeof(TF);  // bytes per factor row
    const char *Bl = reinterpret_cast<const char *>(q.B) + lig * 8 * sizeof(TF);
    const char *Cl = reinterpret_cast<const char *>(q.C) + lig * 8 * sizeof(TF);
    uint32_t *gs = s_idx + (size_t)g * (2 * kBufWords);
    const uint32_t gs_addr = (uint32_t)__cvta_generic_to_shared(gs);

    // copy chunk ch into buffer b: 16 pieces of 16 bytes (C then B indices)
    // spread over the group's lanes, and the head word
    auto issue = [&](int b, int64_t ch) {
        if (ch < cend) {
            const uint32_t d = gs_addr + (uint32_t)(b * kBufWords) * 4u;
            for (int pc = lig; pc < 16; pc += LPR) {
                const uint32_t *src = (pc < 8 ? q.kidx : q.jidx) + ch * 32 + (pc & 7) * 4;
                cp_async16(d + (uint32_t)pc * 16u, src);
            }
            if (lig == 0) cp_async4(d + 64u * 4u, q.bf + ch);
        }
        cp_async_commit();
    };
    Piece<TF> vc[NF], vb[NF];
    constexpr int NW = (int)(sizeof(Piece<TF>) / 4);
#pragma unroll
    for (int s = 0; s < NF; ++s)
#pragma unroll
        for (int i = 0; i < NW; ++i) vc[s].w[i] = vb[s].w[i] = 0u;
    uint32_t sink = 0u, rows = 0u;
    uint32_t jprev = kAll;

    issue(0, cbeg);
    cp_async_wait_all();
    __syncwarp();
    // every lane of the warp runs the same trip counts; chunks past the
    // group's range have no valid nonzeros
    for (int64_t i = 0; i < q.cpg; ++i) {
        const int64_t ch = cbeg + i;
        const int b = (int)(i & 1);
        issue(b ^ 1, ch + 1);
        const uint32_t *kb = gs + b * kBufWords, *jb = kb + 32;
        const int nvalid = ch < cend ? (int)min((int64_t)32, q.nnz - ch * 32) : 0;
        const uint32_t hw = ch < cend ? kb[64] : 0u;
#pragma unroll 1
        for (int t = 0; t < 32; t += NF) {
#pragma unroll
            for (int u = 0; u < NF; ++u) {
                const int j = t + u;
                const uint32_t kk = kb[j], jj = jb[j];
                const bool valid = j < nvalid;
                const bool f = valid && (((hw >> j) & 1u) != 0u || jj != jprev);
                jprev = valid ? jj : jprev;
                // each ring slot is read before it is reused, so its previous
                // load completes first and NF loads of each kind stay in flight
                sink ^= vc[u].fold() ^ vb[u].fold();
                vc[u].load_if(Cl + (uint64_t)kk * rowb, valid);
                vb[u].load_if(Bl + (uint64_t)jj * rowb, f);
                rows += (uint32_t)valid + (uint32_t)f;
            }
        }
        cp_async_wait_all();
        __syncwarp();  // buffer b is no longer read; buffer b^1 has landed
    }
#pragma unroll
    for (int s = 0; s < NF; ++s) sink ^= vc[s].fold() ^ vb[s].fold();
    // every lane of a group counted the same rows
    const unsigned warp_rows = __reduce_add_sync(kAll, rows) / LPR;
    if (lane == 0) atomicAdd(q.count, (unsigned long long)warp_rows);
    // keeps the loaded words observable; the added value is 0
    if (sink == 0x7fc00001u) atomicAdd(q.count, 0ull);
}

template <typename TF, int LPR>
int launch(GatherParams &q, int dev, cudaStream_t s) {
    constexpr int NF = 4;
    auto kern = k_gather_bound<TF, LPR, NF>;
    const size_t smem = (size_t)(kThreads / LPR) * kGroupBytes;
    FCOO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    FCOO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    occ = std::max(1, std::min(occ, kMaxCtasPerSm));
    const int64_t nchunk = (q.nnz + 31) / 32;
    const int64_t groups_per_cta = kThreads / LPR;
    const int64_t max_ctas = (int64_t)device_sms(dev) * occ;
    const int64_t ctas = std::max<int64_t>(1, std::min(max_ctas, ceil_div(nchunk, groups_per_cta)));
    q.cpg = ceil_div(nchunk, ctas * groups_per_cta);
    kern<<<(unsigned)ctas, kThreads, smem, s>>>(q);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}

template <typename TF>
int launch_lpr(GatherParams &q, int dev, cudaStream_t s) {
    switch (q.R) {
        case 8: return launch<TF, 1>(q, dev, s);
        case 16: return launch<TF, 2>(q, dev, s);
        case 32: return launch<TF, 4>(q, dev, s);
        case 64: return launch<TF, 8>(q, dev, s);
        case 128: return launch<TF, 16>(q, dev, s);
        default: return launch<TF, 32>(q, dev, s);
    }
}

}  // namespace
}  // namespace fcx

using namespace fcx;

extern "C" int spmttkrp_gather_bound(const fcoo_t *X, const void *const *factors, int dtype, int R,
                                     unsigned long long *rows_loaded, fcoo_stream_t stream) {
    clear_error();
    if (!X) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: NULL handle");
    if (X->op != FCOO_OP_MTTKRP)
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: handle was built for the other operation");
    if (dtype != FCOO_F32 && dtype != FCOO_BF16)
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: dtype=%d unknown", dtype);
    if (!factors) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: factors is NULL");
    if (!rows_loaded || ((uintptr_t)rows_loaded & 7u) != 0)
        return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: rows_loaded is NULL or not 8-byte aligned");
    if (X->nprod != 2)
        return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_gather_bound: %d-way tensor (3-way only)", X->nmodes);
    if (R < 8 || R > 256 || (R & (R - 1)) != 0)
        return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_gather_bound: R=%d (8, 16, 32, 64, 128 or 256 only)", R);
    const size_t align = dtype == FCOO_F32 ? 32 : 16;  // one lane's eight elements
    for (int m = 0; m < 2; ++m) {
        const void *f = factors[X->prod_modes[m]];
        if (!f) return fail(FCOO_ERR_INVALID_ARG, "spmttkrp_gather_bound: factors[%d] is NULL", X->prod_modes[m]);
        if (((uintptr_t)f & (align - 1)) != 0)
            return fail(FCOO_ERR_UNSUPPORTED, "spmttkrp_gather_bound: factors[%d] is not %zu-byte aligned",
                        X->prod_modes[m], align);
    }
    cudaStream_t s = (cudaStream_t)stream;
    FCOO_CUDA(cudaMemsetAsync(rows_loaded, 0, sizeof(unsigned long long), s));
    if (X->nnz == 0) return FCOO_OK;
    GatherParams q;
    q.jidx = X->pidx[0];
    q.kidx = X->pidx[1];
    q.bf = X->bf;
    q.B = factors[X->prod_modes[0]];
    q.C = factors[X->prod_modes[1]];
    q.nnz = X->nnz;
    q.cpg = 0;
    q.R = R;
    q.count = rows_loaded;
    return dtype == FCOO_F32 ? launch_lpr<float>(q, X->device, s) : launch_lpr<__nv_bfloat16>(q, X->device, s);
}
