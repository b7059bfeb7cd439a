// fcoo_build.cu -- builds the F-COO layout (Sec. IV-B, Table I, Table II,
// Fig. 2) of an N-way COO tensor on the GPU.
//
// Pipeline (every step is a kernel in this file):
//   1. range check of every index                         (k_validate)
//   2. mixed-radix sort keys, lowest key mode first        (k_make_key)
//   3. stable LSD radix sort of (key, position) pairs      (k_rs_hist, scan, k_rs_scatter)
//   4. gather product-mode streams and values              (k_gather)
//   5. head flags / duplicate check / fibre count          (k_flags, one ballot per 32 nonzeros)
//   6. segment numbering by a scan of per-word popcounts   (scan, k_hcount, k_segkeys)
//   7. start flags, one bit per threadlen partition        (k_sf)
// The paper does this preprocessing on the host once per mode (Sec. IV-D);
// here it runs on the device because the sort of ~10^8 keys is the dominant
// cost and the result has to end up in HBM anyway.
#include <stdio.h>
#include <string.h>

#include <vector>

#include <atomic>

#include "internal.cuh"

namespace fcx {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct IdxPtrs {
    const uint32_t *p[FCOO_MAX_MODES];
};
struct OutPtrs {
    uint32_t *p[FCOO_MAX_MODES];
};
struct DimArr {
    uint32_t d[FCOO_MAX_MODES];
};

// ---------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t before = w ? warp_tot[w - 1] : 0;
    if (total) *total = warp_tot[kScanThreads / 32 - 1];
    return before + x - v;
}

__global__ void k_scan_reduce(const uint32_t *in, int64_t n, uint32_t *partial) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t p = base + i;
        if (p < n) s += in[p];
    }
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan_tile(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *block_off) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], t = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        t += v[i];
    }
    uint32_t run = block_exclusive_scan(t, nullptr) + (block_off ? block_off[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// Exclusive prefix sum of n uint32 values (in may equal out).
int exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return FCOO_OK;
    int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        FCOO_CUDA(cudaGetLastError());
        return FCOO_OK;
    }
    uint32_t *part = nullptr;
    FCOO_CUDA(dev_alloc_async((void **)&part, nb * 4, s));
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part);
    int st = exclusive_scan(part, part, nb, s);
    if (st == FCOO_OK) {
        k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "k_scan_tile");
    }
    dev_free_async(part, s);
    return st;
}

// ---------------------------------------------------------------- radix sort

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t *keys, int64_t n, int shift, uint32_t *hist,
                                                        int nblk) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsItems; ++i) {
        int64_t p = base + (int64_t)i * kRsThreads + threadIdx.x;
        if (p < n) atomicAdd(&cnt[(unsigned)(keys[p] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: each warp ranks its 512 items in order (slot-major, lane
// order within a slot) with match.any; warps are ordered inside the block,
// blocks by the digit-major offsets of the scanned histogram.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                                           uint32_t *vout, int64_t n, int shift,
                                                           const uint32_t *offs, int nblk) {
    __shared__ uint32_t wcnt[kRsWarps][257];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 257; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t wbase = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (kRsItems * 32);
    uint64_t k[kRsItems];
    uint32_t v[kRsItems], rank[kRsItems];
#pragma unroll
    for (int s = 0; s < kRsItems; ++s) {
        int64_t p = wbase + s * 32 + lane;
        bool valid = p < n;
        k[s] = valid ? kin[p] : 0ull;
        v[s] = valid ? vin[p] : 0u;
        unsigned d = valid ? ((unsigned)(k[s] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        uint32_t before = wcnt[w][d];
        rank[s] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
        for (int ww = 0; ww < kRsWarps; ++ww) {
            uint32_t t = wcnt[ww][threadIdx.x];
            wcnt[ww][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kRsItems; ++s) {
        int64_t p = wbase + s * 32 + lane;
        if (p < n) {
            unsigned d = (unsigned)(k[s] >> shift) & 255u;
            uint32_t pos = offs[(int64_t)d * nblk + blockIdx.x] + wcnt[w][d] + rank[s];
            kout[pos] = k[s];
            vout[pos] = v[s];
        }
    }
}

// Sort (keys, vals) by the low `nbits` bits of keys, stable.  Result ends in
// (*k0, *v0) -- the buffers are swapped as needed.
int radix_sort_pairs(uint64_t **k0, uint32_t **v0, uint64_t **k1, uint32_t **v1, int64_t n, int nbits,
                     cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return FCOO_OK;
    int nblk = (int)ceil_div(n, kRsTile);
    uint32_t *hist = nullptr;
    FCOO_CUDA(dev_alloc_async((void **)&hist, (size_t)256 * nblk * 4, s));
    int st = FCOO_OK;
    for (int shift = 0; shift < nbits && st == FCOO_OK; shift += 8) {
        k_rs_hist<<<nblk, kRsThreads, 0, s>>>(*k0, n, shift, hist, nblk);
        st = exclusive_scan(hist, hist, (int64_t)256 * nblk, s);
        if (st) break;
        k_rs_scatter<<<nblk, kRsThreads, 0, s>>>(*k0, *v0, *k1, *v1, n, shift, hist, nblk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "k_rs_scatter");
        uint64_t *tk = *k0;
        *k0 = *k1;
        *k1 = tk;
        uint32_t *tv = *v0;
        *v0 = *v1;
        *v1 = tv;
    }
    dev_free_async(hist, s);
    return st;
}

// ---------------------------------------------------------------- build kernels

__global__ void k_validate(IdxPtrs idx, DimArr dims, int nmodes, int64_t n, unsigned long long *bad) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < nmodes; ++k)
            if (idx.p[k][p] >= dims.d[k]) atomicMin(bad, (unsigned long long)p * FCOO_MAX_MODES + k);
    }
}

struct KeySpec {
    int nm;
    int mode[FCOO_MAX_MODES];
    int shift[FCOO_MAX_MODES];
    int nbits;
};

__global__ void k_make_key(KeySpec ks, IdxPtrs idx, const uint32_t *perm, int64_t n, uint64_t *key,
                           uint32_t *pout) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q = perm ? perm[p] : (uint32_t)p;
        uint64_t k = 0;
        for (int t = 0; t < ks.nm; ++t) k |= (uint64_t)idx.p[ks.mode[t]][q] << ks.shift[t];
        key[p] = k;
        pout[p] = q;
    }
}

struct GatherSpec {
    int nprod, nidx;
    int prod_modes[FCOO_MAX_MODES];
    int idx_modes[FCOO_MAX_MODES];
};

__global__ void k_gather(GatherSpec g, IdxPtrs idx, const float *val_in, const uint32_t *perm, int64_t n,
                         int64_t npad, OutPtrs pidx_out, float *val_out, uint32_t *perm_out, OutPtrs sidx_out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad; p += (int64_t)gridDim.x * blockDim.x) {
        if (p < n) {
            uint32_t q = perm[p];
            for (int m = 0; m < g.nprod; ++m) pidx_out.p[m][p] = idx.p[g.prod_modes[m]][q];
            for (int t = 0; t < g.nidx; ++t) sidx_out.p[t][p] = idx.p[g.idx_modes[t]][q];
            val_out[p] = val_in[q];
            perm_out[p] = q;
        } else {
            for (int m = 0; m < g.nprod; ++m) pidx_out.p[m][p] = 0u;
            val_out[p] = 0.0f;
            perm_out[p] = 0u;
        }
    }
}

// One warp per 32 consecutive nonzeros (grid covers npad exactly).
__global__ void k_flags(int nprod, int nidx, IdxPtrs pidx, IdxPtrs sidx, int64_t n, uint32_t *bf, uint32_t *cnt,
                        unsigned long long *nfib, unsigned long long *dup) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool valid = p < n;
    bool head = false, fib = false, same = false;
    if (valid) {
        if (p == 0) {
            head = fib = true;
        } else {
            for (int t = 0; t < nidx; ++t) head |= sidx.p[t][p] != sidx.p[t][p - 1];
            fib = head;
            for (int m = 0; m < nprod - 1; ++m) fib |= pidx.p[m][p] != pidx.p[m][p - 1];
            same = !fib && pidx.p[nprod - 1][p] == pidx.p[nprod - 1][p - 1];
        }
    }
    unsigned hb = __ballot_sync(kFull, head);
    unsigned fb = __ballot_sync(kFull, fib);
    if (same) atomicMin(dup, (unsigned long long)p);
    if (lane == 0) {
        bf[p >> 5] = hb;
        cnt[p >> 5] = __popc(hb);
        if (fb) atomicAdd(nfib, (unsigned long long)__popc(fb));
    }
}

__global__ void k_hcount(const uint32_t *word_base, int64_t nchunk, uint32_t *hcount) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= nchunk; c += (int64_t)gridDim.x * blockDim.x)
        hcount[c] = word_base[c * (kChunk / 32)];
}

__global__ void k_segkeys(int nidx, IdxPtrs sidx, const uint32_t *bf, const uint32_t *word_base, int64_t n,
                          uint32_t *segkeys) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w = bf[p >> 5];
        unsigned b = (unsigned)(p & 31);
        if ((w >> b) & 1u) {
            int64_t sg = (int64_t)word_base[p >> 5] + __popc(w & ((1u << b) - 1u));
            for (int t = 0; t < nidx; ++t) segkeys[sg * nidx + t] = sidx.p[t][p];
        }
    }
}

// One thread per partition; grid covers the padded partition count exactly.
__global__ void k_sf(const uint32_t *bf, int64_t n, int threadlen, uint32_t *sf) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t p = t * threadlen;
    bool bit = p < n && ((bf[p >> 5] >> (p & 31)) & 1u);
    unsigned b = __ballot_sync(kFull, bit);
    if ((threadIdx.x & 31) == 0) sf[t >> 5] = b;
}

unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = ceil_div(n, threads);
    int64_t cap = (int64_t)num_sms() * 32;
    if (b > cap) b = cap;
    return (unsigned)(b > 0 ? b : 1);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int bits_for(uint32_t d) {
    if (d <= 1) return 0;
    return 32 - __builtin_clz(d - 1);
}

// Temporaries freed (stream-ordered) on every exit path.
struct Temps {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Temps(cudaStream_t st) : s(st) {}
    ~Temps() {
        for (void *p : ptrs) dev_free_async(p, s);
    }
    cudaError_t alloc(void **p, size_t bytes) {
        cudaError_t e = dev_alloc_async(p, bytes, s);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

}  // namespace
}  // namespace fcx

using namespace fcx;

extern "C" int fcoo_build(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                          const float *val, int mode, int op, int threadlen, fcoo_stream_t stream, fcoo_t **out) {
    clear_error();
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: out is NULL");
    *out = nullptr;
    if (nmodes < 2 || nmodes > FCOO_MAX_MODES)
        return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: nmodes=%d outside 2..%d", nmodes, FCOO_MAX_MODES);
    if (!dims) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: dims is NULL");
    for (int k = 0; k < nmodes; ++k)
        if (dims[k] == 0) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: dims[%d] is 0", k);
    if (nnz < 0 || nnz > FCOO_MAX_NNZ)
        return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: nnz=%lld outside 0..%lld", (long long)nnz,
                    (long long)FCOO_MAX_NNZ);
    if (nnz > 0) {
        if (!idx) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: idx is NULL");
        for (int k = 0; k < nmodes; ++k)
            if (!idx[k]) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: idx[%d] is NULL", k);
        if (!val) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: val is NULL");
    }
    if (mode < 0 || mode >= nmodes) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: mode=%d outside 0..%d", mode, nmodes - 1);
    if (op != FCOO_OP_MTTKRP && op != FCOO_OP_TTM) return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: op=%d unknown", op);
    if (threadlen < 1 || threadlen > 64 || (threadlen & (threadlen - 1)) != 0)
        return fail(FCOO_ERR_INVALID_ARG, "fcoo_build: threadlen=%d is not a power of two in 1..64", threadlen);

    cudaStream_t s = (cudaStream_t)stream;
    fcoo_t *X = (fcoo_t *)calloc(1, sizeof(fcoo_t));
    if (!X) return fail(FCOO_ERR_NOMEM, "fcoo_build: host allocation failed");
    X->nmodes = nmodes;
    X->mode = mode;
    X->op = op;
    X->threadlen = threadlen;
    X->nnz = nnz;
    X->npad = round_up(nnz > 0 ? nnz : 1, kPad);
    for (int k = 0; k < nmodes; ++k) X->dims[k] = dims[k];
    // Table I: product and index modes
    if (op == FCOO_OP_MTTKRP) {
        X->nidx = 1;
        X->idx_modes[0] = mode;
        for (int k = 0; k < nmodes; ++k)
            if (k != mode) X->prod_modes[X->nprod++] = k;
    } else {
        for (int k = 0; k < nmodes; ++k)
            if (k != mode) X->idx_modes[X->nidx++] = k;
        X->nprod = 1;
        X->prod_modes[0] = mode;
    }
    cudaGetDevice(&X->device);
    X->max_grid = num_sms() * kMaxCtasPerSm;
    {
        static std::atomic<uint64_t> next_uid{1};
        X->uid = next_uid.fetch_add(1);
    }

    const int64_t n = nnz, npad = X->npad;
    const int64_t nwords = npad / 32;
    const int64_t nchunk = npad / kChunk;
    const int64_t nsfw = ceil_div(ceil_div(npad, threadlen), 32);
    X->bytes_val = 4 * n;
    X->bytes_pidx = 4 * (int64_t)X->nprod * n;
    X->bytes_bf = 4 * ceil_div(n, 32);
    X->bytes_sf = 4 * ceil_div(ceil_div(n, threadlen), 32);
    X->bytes_aux = 4 * (nchunk + 1) + 4 * n;
    X->bytes_scratch = (int64_t)2 * X->max_grid * FCOO_MAX_RANK * 8 + (int64_t)3 * X->max_grid * 8 + 256;

    // carve the persistent allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += round_up((int64_t)bytes, 256);
        return o;
    };
    size_t o_pidx[FCOO_MAX_MODES];
    for (int m = 0; m < X->nprod; ++m) o_pidx[m] = take(npad * 4);
    size_t o_val = take(npad * 4), o_bf = take(nwords * 4), o_sf = take(nsfw * 4), o_hc = take((nchunk + 1) * 4);
    size_t o_perm = take(npad * 4);
    size_t o_cv = take((size_t)2 * X->max_grid * FCOO_MAX_RANK * 8), o_cs = take((size_t)2 * X->max_grid * 8);
    size_t o_cnt = take(256);
    size_t o_red = take((size_t)X->max_grid * 8);
    X->base_bytes = off;
    cudaError_t e = dev_alloc(&X->base, off);
    if (e != cudaSuccess) {
        free(X);
        return cuda_fail(e, "fcoo_build: cudaMalloc(layout)");
    }
    char *b = (char *)X->base;
    for (int m = 0; m < X->nprod; ++m) X->pidx[m] = (uint32_t *)(b + o_pidx[m]);
    X->val = (float *)(b + o_val);
    X->bf = (uint32_t *)(b + o_bf);
    X->sf = (uint32_t *)(b + o_sf);
    X->hcount = (uint32_t *)(b + o_hc);
    X->perm = (uint32_t *)(b + o_perm);
    X->carry_val = (double *)(b + o_cv);
    X->carry_seg = (int64_t *)(b + o_cs);
    X->counter = (unsigned int *)(b + o_cnt);
    X->red_part = (double *)(b + o_red);

    int st = FCOO_OK;
    {
        Temps tmp(s);
#define TRY_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            st = cuda_fail(e_, #call);                   \
            goto done;                                   \
        }                                                \
    } while (0)
        IdxPtrs din;
        memset(&din, 0, sizeof(din));
        const float *dval = val;
        uint64_t *k0 = nullptr, *k1 = nullptr;
        uint32_t *v0 = nullptr, *v1 = nullptr, *cnt = nullptr;
        unsigned long long *flags = nullptr;  // [0] bad index, [1] dup position, [2] nfib
        unsigned long long hflags[3];
        uint32_t nseg32 = 0;
        OutPtrs sidx_w, pidx_out;
        IdxPtrs sidx, pidx_in;
        memset(&sidx_w, 0, sizeof(sidx_w));
        memset(&sidx, 0, sizeof(sidx));
        memset(&pidx_out, 0, sizeof(pidx_out));
        memset(&pidx_in, 0, sizeof(pidx_in));
        TRY_CUDA(cudaMemsetAsync(X->base, 0, X->base_bytes, s));
        TRY_CUDA(tmp.alloc((void **)&flags, 3 * sizeof(unsigned long long)));
        {
            unsigned long long init[3] = {~0ull, ~0ull, 0ull};
            TRY_CUDA(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s));
            TRY_CUDA(cudaStreamSynchronize(s));  // `init` lives on this stack frame
        }
        if (n > 0) {
            // 0. stage inputs on the device
            for (int k = 0; k < nmodes; ++k) {
                if (is_device_ptr(idx[k])) {
                    din.p[k] = idx[k];
                } else {
                    void *d = nullptr;
                    TRY_CUDA(tmp.alloc(&d, n * 4));
                    TRY_CUDA(cudaMemcpyAsync(d, idx[k], n * 4, cudaMemcpyHostToDevice, s));
                    din.p[k] = (const uint32_t *)d;
                }
            }
            if (!is_device_ptr(val)) {
                void *d = nullptr;
                TRY_CUDA(tmp.alloc(&d, n * 4));
                TRY_CUDA(cudaMemcpyAsync(d, val, n * 4, cudaMemcpyHostToDevice, s));
                dval = (const float *)d;
            }
            // 1. range check
            {
                DimArr da;
                for (int k = 0; k < FCOO_MAX_MODES; ++k) da.d[k] = k < nmodes ? dims[k] : 1u;
                k_validate<<<grid_for(n), 256, 0, s>>>(din, da, nmodes, n, flags);
            }
            TRY_CUDA(cudaGetLastError());
            TRY_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            if (hflags[0] != ~0ull) {
                unsigned long long p = hflags[0] / FCOO_MAX_MODES;
                int k = (int)(hflags[0] % FCOO_MAX_MODES);
                st = fail(FCOO_ERR_INDEX_RANGE, "fcoo_build: idx[%d][%llu] >= dims[%d]=%u", k, p, k, dims[k]);
                goto done;
            }
            // 2-3. sort keys: modes in sort order (index modes, then product
            // modes), packed from the least significant mode upwards into
            // 64-bit words; words sorted LSD-first, each by a stable radix sort.
            int order[FCOO_MAX_MODES], no = 0;
            for (int t = 0; t < X->nidx; ++t) order[no++] = X->idx_modes[t];
            for (int m = 0; m < X->nprod; ++m) order[no++] = X->prod_modes[m];
            std::vector<KeySpec> words;
            {
                KeySpec cur;
                memset(&cur, 0, sizeof(cur));
                for (int q = nmodes - 1; q >= 0; --q) {
                    int bits = bits_for(dims[order[q]]);
                    if (bits == 0) continue;
                    if (cur.nbits + bits > 64) {
                        words.push_back(cur);
                        memset(&cur, 0, sizeof(cur));
                    }
                    cur.mode[cur.nm] = order[q];
                    cur.shift[cur.nm] = cur.nbits;
                    cur.nm++;
                    cur.nbits += bits;
                }
                if (cur.nm) words.push_back(cur);
            }
            TRY_CUDA(tmp.alloc((void **)&k0, n * 8));
            TRY_CUDA(tmp.alloc((void **)&k1, n * 8));
            TRY_CUDA(tmp.alloc((void **)&v0, n * 4));
            TRY_CUDA(tmp.alloc((void **)&v1, n * 4));
            bool have_perm = false;
            for (size_t wdx = 0; wdx < words.size(); ++wdx) {
                // keys of this word for the current order; positions carried along
                k_make_key<<<grid_for(n), 256, 0, s>>>(words[wdx], din, have_perm ? v0 : nullptr, n, k1, v1);
                TRY_CUDA(cudaGetLastError());
                { uint64_t *t = k0; k0 = k1; k1 = t; uint32_t *tv = v0; v0 = v1; v1 = tv; }
                st = radix_sort_pairs(&k0, &v0, &k1, &v1, n, words[wdx].nbits, s);
                if (st) goto done;
                have_perm = true;
            }
            if (!have_perm) {  // every dimension is 1: a single cell
                k_make_key<<<grid_for(n), 256, 0, s>>>(KeySpec{}, din, nullptr, n, k1, v0);
                TRY_CUDA(cudaGetLastError());
            }
            // 4. gather streams
            GatherSpec g;
            memset(&g, 0, sizeof(g));
            g.nprod = X->nprod;
            g.nidx = X->nidx;
            for (int m = 0; m < X->nprod; ++m) g.prod_modes[m] = X->prod_modes[m];
            for (int t = 0; t < X->nidx; ++t) g.idx_modes[t] = X->idx_modes[t];
            for (int t = 0; t < X->nidx; ++t) {
                void *d = nullptr;
                TRY_CUDA(tmp.alloc(&d, npad * 4));
                sidx_w.p[t] = (uint32_t *)d;
                sidx.p[t] = (const uint32_t *)d;
            }
            for (int m = 0; m < X->nprod; ++m) {
                pidx_out.p[m] = X->pidx[m];
                pidx_in.p[m] = X->pidx[m];
            }
            k_gather<<<grid_for(npad), 256, 0, s>>>(g, din, dval, v0, n, npad, pidx_out, X->val, X->perm, sidx_w);
            TRY_CUDA(cudaGetLastError());
            // 5. flags
            TRY_CUDA(tmp.alloc((void **)&cnt, (nwords + 1) * 4));
            TRY_CUDA(cudaMemsetAsync(cnt + nwords, 0, 4, s));
            k_flags<<<(unsigned)(npad / 256), 256, 0, s>>>(X->nprod, X->nidx, pidx_in, sidx, n, X->bf, cnt,
                                                           flags + 2, flags + 1);
            TRY_CUDA(cudaGetLastError());
            // 6. segment numbering
            st = exclusive_scan(cnt, cnt, nwords + 1, s);
            if (st) goto done;
            TRY_CUDA(cudaMemcpyAsync(&nseg32, cnt + nwords, 4, cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            if (hflags[1] != ~0ull) {
                st = fail(FCOO_ERR_DUPLICATE, "fcoo_build: duplicate coordinate at sorted position %llu",
                          hflags[1]);
                goto done;
            }
            X->nseg = nseg32;
            X->nfib = (int64_t)hflags[2];
            k_hcount<<<grid_for(nchunk + 1), 256, 0, s>>>(cnt, nchunk, X->hcount);
            TRY_CUDA(cudaGetLastError());
            X->bytes_segmap = (int64_t)X->nseg * X->nidx * 4;
            {
                void *sk = nullptr;
                TRY_CUDA(dev_alloc(&sk, X->bytes_segmap));
                X->segkeys = (uint32_t *)sk;
            }
            k_segkeys<<<grid_for(n), 256, 0, s>>>(X->nidx, sidx, X->bf, cnt, n, X->segkeys);
            TRY_CUDA(cudaGetLastError());
            // 7. start flags
            {
                int64_t nthreads = nsfw * 32;
                k_sf<<<(unsigned)ceil_div(nthreads, 256), 256, 0, s>>>(X->bf, n, threadlen, X->sf);
                TRY_CUDA(cudaGetLastError());
            }
        }
        TRY_CUDA(cudaStreamSynchronize(s));
    done:;
#undef TRY_CUDA
    }
    if (st == FCOO_OK) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess) st = cuda_fail(e2, "fcoo_build: stream synchronize");
    }
    if (st != FCOO_OK) {
        cudaStreamSynchronize(s);
        dev_free(X->segkeys);
        dev_free(X->base);
        free(X);
        return st;
    }
    *out = X;
    return FCOO_OK;
}
