// stream_kernel.cuh -- the F-COO streaming kernel (templates), shared by the
// translation units that instantiate it for one factor type and one weight
// kind each, so that nvcc compiles the variants in parallel.
// It is the kernel behind SpMTTKRP (Eq. 6) and SpTTM (Eq. 3): the one-shot
// product (Sec. IV-C) fused with the segmented reduction over the bit-flags
// (Sec. IV-D).  The same kernel, with residual weights, computes the sparse
// CP-fit loss and its adjoint, and, with Kronecker output columns, SpTTMc
// (Eq. 4, Table I row 3).
//
// Work split (GB300 design; the paper's Maxwell layout of one thread per
// column r and per threadlen partition is replaced):
//   * a CTA owns a contiguous range of nonzeros (equal count per CTA: the
//     paper's nnz-balanced partitioning), split into G equal "runs", one per
//     lane group; a run is a whole number of threadlen partitions, so the
//     partition's start-flag tells whether the run opens a new segment;
//   * a lane group of LPR lanes spans the R columns of one output row: each
//     lane holds E contiguous columns of every gathered factor row (eight:
//     one 32-byte FP32 or 16-byte BF16 load; four for FP32 R <= 16; one on
//     the scalar fallback), so one row gather is a fully coalesced access;
//   * the group walks its run in stages of 32 nonzeros.  The index / value
//     streams and the bit-flag word of a stage are copied by cp.async into a
//     two-slot ring in shared memory, one stage ahead of use; groups' rings
//     are offset by 16 bytes modulo 128 so that the 128-bit reads of one warp
//     hit distinct banks;
//   * gathers are software-pipelined in "quarters" of Q nonzeros (2, or 4
//     for four-column lanes), double-buffered in registers and walked by a
//     rolled loop over quarter pairs: the last-product-mode rows of quarter
//     h+1 (and, for 3-way SpMTTKRP, the rows of the other product mode where
//     a new fibre starts) are requested before quarter h is consumed, across
//     stage boundaries too; a row address is one 32x32->64-bit multiply-add;
//   * the rows of the non-last product modes change only where a new fibre
//     starts (fixed index mode and non-last product modes): their product brow
//     is kept in registers and replaced by a predicated select, and each
//     nonzero adds (val * brow) * row with the paired FP32 instructions
//     (FMUL2 / FFMA2, two elements per instruction); only quarters that
//     contain a segment start take a branch (SpTTM, whose fibres are mostly
//     one or two nonzeros long, takes predicated stores instead);
//   * at the end of every stage of 32 nonzeros that holds no segment start,
//     the register sum is folded into the segment sum with Kahan compensation
//     in shared memory, so the error of a long (Zipf-hot) segment grows with
//     its number of stages, not nonzeros, and no register sum spans more than
//     two stages; a segment that starts and ends between two folds never
//     leaves registers (short segments, such as SpTTM's fibres of one or two
//     nonzeros, are stored straight from registers);
//   * a segment that starts and ends inside a run is stored directly (one
//     FP32 row per segment); segments cut by run boundaries are combined per
//     CTA in shared memory (FP64, run order); segments cut by CTA boundaries
//     leave one FP64 carry per CTA side, and k_carry_fixup adds the carries
//     of each such segment in CTA order and stores the row.  No atomics on
//     the output, no pre-zeroing, and the result is bitwise reproducible for
//     a given handle, R and GPU.
// The paper replaces atomics with a segmented scan whose inter-block carry is
// passed by adjacent synchronisation (CTAs spinning on their predecessor); the
// carry-slot + fixup pass gives the same atomic-free result without any CTA
// waiting on another.
#pragma once

#include <limits.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace fcx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int T = 32;   // nonzeros per stage
constexpr int NS = 2;   // stages in the ring (one in flight while one is consumed)

// ------------------------------------------------------------ row loads

template <typename TF, int E>
struct RowIO;

template <>
struct RowIO<float, 4> {
    using raw = float4;
    static __device__ __forceinline__ raw load(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    // as RowIO<float, 8>::load_if: unspecified where f is false
    static __device__ __forceinline__ raw load_if(const float *p, bool f) {
        raw r;
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
            "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n\t}"
            : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
            : "l"(p), "r"((unsigned)f));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw &r, float (&v)[4]) {
        v[0] = r.x;
        v[1] = r.y;
        v[2] = r.z;
        v[3] = r.w;
    }
};

// 32-byte lanes: one 256-bit load per lane and row (eight FP32 columns)
struct F8 {
    float v[8];
};
template <>
struct RowIO<float, 8> {
    using raw = F8;
    static __device__ __forceinline__ raw load(const float *p) {
        raw r;
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
              "=f"(r.v[7])
            : "l"(p));
        return r;
    }
    // the load only where f holds, as one predicated instruction; where f is
    // false the result is unspecified (callers select it away)
    static __device__ __forceinline__ raw load_if(const float *p, bool f) {
        raw r;
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %9, 0;\n\t"
            "@q ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t}"
            : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
              "=f"(r.v[7])
            : "l"(p), "r"((unsigned)f));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw &r, float (&v)[8]) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = r.v[i];
    }
};

template <>
struct RowIO<__nv_bfloat16, 8> {
    using raw = uint4;
    static __device__ __forceinline__ raw load(const __nv_bfloat16 *p) {
        return __ldg(reinterpret_cast<const uint4 *>(p));
    }
    // as RowIO<float, 8>::load_if: unspecified where f is false
    static __device__ __forceinline__ raw load_if(const __nv_bfloat16 *p, bool f) {
        raw r;
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
            "@q ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
            : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
            : "l"(p), "r"((unsigned)f));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw &r, float (&v)[8]) {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // bf16 -> fp32 is exact: the bits move up 16 places
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

template <>
struct RowIO<float, 1> {
    using raw = float;
    static __device__ __forceinline__ raw load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ raw zero() { return 0.f; }
    static __device__ __forceinline__ raw load_if(const float *p, bool f) { return f ? load(p) : zero(); }
    static __device__ __forceinline__ void cvt(const raw &r, float (&v)[1]) { v[0] = r; }
};

template <>
struct RowIO<__nv_bfloat16, 1> {
    using raw = unsigned short;
    static __device__ __forceinline__ raw load(const __nv_bfloat16 *p) {
        return __ldg(reinterpret_cast<const unsigned short *>(p));
    }
    static __device__ __forceinline__ raw zero() { return 0; }
    static __device__ __forceinline__ raw load_if(const __nv_bfloat16 *p, bool f) { return f ? load(p) : zero(); }
    static __device__ __forceinline__ void cvt(const raw &r, float (&v)[1]) { v[0] = __uint_as_float((uint32_t)r << 16); }
};

// one factor element as FP32
template <typename TF>
__device__ __forceinline__ float ld_elem(const TF *p) {
    float v[1];
    RowIO<TF, 1>::cvt(RowIO<TF, 1>::load(p), v);
    return v[0];
}

// the products of the two BF16 pairs packed in a and b, each exact in FP32
// (8-bit significands: the 16-bit product fits in 24 bits), by the mixed
// BF16 x BF16 + FP32 fused multiply-add with a zero addend
__device__ __forceinline__ float2 bf16_prod2(uint32_t a, uint32_t b) {
    float2 r;
    asm("{\n\t.reg .b16 al, ah, bl, bh;\n\tmov.b32 {al, ah}, %2;\n\tmov.b32 {bl, bh}, %3;\n\t"
        "fma.rn.f32.bf16 %0, al, bl, 0f00000000;\n\tfma.rn.f32.bf16 %1, ah, bh, 0f00000000;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(a), "r"(b));
    return r;
}

template <int E>
__device__ __forceinline__ void store_row(float *dst, const float (&v)[E]) {
    if constexpr (E == 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (E == 8) {
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) dst[e] = v[e];
    }
}

// ------------------------------------------------------------ async copies

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Number of heads (segment starts) strictly before nonzero position pos
// (pos a multiple of 32): chunk checkpoint plus popcounts of the words since.
__device__ __forceinline__ int64_t heads_before(const StreamParams &p, int64_t pos, int lig, int lpr,
                                                unsigned gmask) {
    int64_t c = pos / kChunk;
    int64_t w0 = c * (kChunk / 32), w1 = pos >> 5;
    uint32_t cnt = 0;
    for (int64_t w = w0 + lig; w < w1; w += lpr) cnt += __popc(__ldg(p.bf + w));
    for (int o = 1; o < lpr; o <<= 1) cnt += __shfl_xor_sync(gmask, cnt, o);
    return (int64_t)__ldg(p.hcount + c) + cnt;
}

__device__ __forceinline__ bool head_at(const StreamParams &p, int64_t pos) {
    return (__ldg(p.bf + (pos >> 5)) >> (pos & 31)) & 1u;
}

// Bytes of one stage in the ring (streams + bit-flag word, 16-byte padded)
// and the per-group region stride (16 mod 128 so groups hit different banks).
// After its run a group reuses its region for the FP64 partial of its last
// segment (rt columns), so the region holds whichever is larger.
// nstream arrays, of which the first nidx are index streams of ix bytes per
// nonzero (4, or 2 after index compression) and the others 4-byte streams.
__host__ __device__ constexpr int slot_bytes(int nstream, int nidx = 0, int ix = 4) {
    return nidx * T * ix + (nstream - nidx) * T * 4 + 16;
}
__host__ __device__ constexpr int group_stride(int nstream, int rt, int nidx = 0, int ix = 4) {
    return (((NS * slot_bytes(nstream, nidx, ix) > rt * 8 ? NS * slot_bytes(nstream, nidx, ix) : rt * 8) + 127) /
            128) * 128 + 16;
}
// Bytes of dynamic shared memory of one CTA of the streaming kernel.
__host__ __device__ constexpr size_t stream_smem_bytes(int nstream, int G, int RT, int nidx = 0, int ix = 4) {
    return (size_t)G * group_stride(nstream, RT, nidx, ix)  // stream rings / last-segment partials
           + (size_t)G * RT * 8                   // first-segment partials (FP64)
           + (size_t)2 * G * 8 + (size_t)2 * G * 4 + (size_t)G * 4  // segment ids, flags, loss
           + (size_t)G * 2 * RT * 4;              // Kahan sums and compensations
}

// ------------------------------------------------------------ segment output

// Float offset of element e of column chunk c of lane lig in a group's Kahan
// sum / compensation arrays: the 16-byte pieces of the lanes of a warp are
// contiguous, so 128-bit accesses are conflict-free.
template <int E, int LPR>
__device__ __forceinline__ int acc_slot(int c, int e, int lig) {
    if constexpr (E % 4 == 0)
        return ((c * (E / 4) + e / 4) * LPR + lig) * 4 + e % 4;
    else
        return (c * LPR + lig) * E + e;
}

template <int E, int NCH>
struct SegAcc {
    float v[NCH][E];
};

// A finished segment that reached a fold or was cut by the run: its value is
// the stage sum a plus, when in_smem, the Kahan sum minus its compensation.
// Written to the output row orow (part == NULL, FP32) or to the FP64 partial
// part[] of the CTA combine.  It runs once per run or per long segment; the
// out-of-line copies below keep the loop of the short-segment variants small.
template <int E, int NCH, int LPR>
__device__ __forceinline__ void emit_segment_body(const SegAcc<E, NCH> &a, bool in_smem, const float *s_acc,
                                                  const float *s_cmp, int lig, const int (&colv)[NCH], int R,
                                                  float *orow, double *part) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int col = colv[c];
        if (part) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = acc_slot<E, LPR>(c, e, lig);
                part[col + e] = in_smem ? (double)s_acc[i] + ((double)a.v[c][e] - (double)s_cmp[i]) : (double)a.v[c][e];
            }
        } else if (col < R) {
            float v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = acc_slot<E, LPR>(c, e, lig);
                v[e] = in_smem ? s_acc[i] + (a.v[c][e] - s_cmp[i]) : a.v[c][e];
            }
            store_row<E>(orow + col, v);
        }
    }
}

template <int E, int NCH, int LPR>
__device__ __noinline__ void emit_segment_outlined(SegAcc<E, NCH> a, bool in_smem, const float *s_acc,
                                                   const float *s_cmp, int lig, const int (&colv)[NCH], int R,
                                                   float *orow, double *part) {
    emit_segment_body<E, NCH, LPR>(a, in_smem, s_acc, s_cmp, lig, colv, R, orow, part);
}

// Rows from+1 .. to-1 of out hold no nonzeros: zero this lane's columns.
template <int E, int NCH>
__device__ __forceinline__ void zero_rows(float *out, int R, const int (&colv)[NCH], int64_t from, int64_t to) {
    float z[E];
#pragma unroll
    for (int e = 0; e < E; ++e) z[e] = 0.f;
    for (int64_t rr = from + 1; rr < to; ++rr) {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            if (colv[c] < R) store_row<E>(out + rr * R + colv[c], z);
    }
}

// ------------------------------------------------------------ the kernel

// TF: factor element type; E: elements per lane per chunk (16 bytes for the
// vector variants); LPR: lanes per group; NCH: column chunks per lane
// (columns of lane l, chunk c: (c * LPR + l) * E ... + E - 1); NP: number of
// product modes (0: runtime value p.nprod); KIND: 0 = value weights
// (SpMTTKRP / SpTTM), 1 = residual weights, 2 = value weights with Kronecker
// output columns (SpTTMc: the R = Rin^nprod columns of a row are the base-Rin
// digit tuples of the product modes, the first product mode most significant;
// a lane's E columns share every digit but the last).
// Resident CTAs per SM the register budget is set for: 3 (80 registers) for
// the one-product value pass with at most four columns per lane (SpTTM at
// R <= 16: short segments, two-nonzero quarters; measured 9 % faster with 24
// warps per SM than with 16), 2 (128 registers) for the others, whose row
// buffers need them.
template <int E, int NCH, int NP, int KIND>
constexpr bool stream_three_ctas() {
    return NP == 1 && KIND == 0 && E * NCH <= 4;
}
template <int E, int NCH, int NP, int KIND>
constexpr int stream_min_blocks() {
    return stream_three_ctas<E, NCH, NP, KIND>() ? 3 : 2;
}

// IX: bytes per product-mode index in the stage (4, or 2 for the 16-bit
// streams of a compressed handle: value kind with one or two product modes).
template <typename TF, int E, int LPR, int NCH, int NP, int KIND, int IX = 4>
__global__ void __launch_bounds__(kThreads, stream_min_blocks<E, NCH, NP, KIND>()) k_stream(const StreamParams p) {
    static_assert(IX == 4 || (KIND == 0 && (NP == 1 || NP == 2)), "16-bit indices: value kind, 1 or 2 product modes");
    using IO = RowIO<TF, E>;
    using raw = typename IO::raw;
    constexpr int G = kThreads / LPR;  // groups per CTA
    constexpr int RT = NCH * LPR * E;  // columns covered by a group
    const int nprod = NP > 0 ? NP : p.nprod;
    // stage layout: the product-mode index streams (IX bytes per nonzero),
    // the values and, for the residual kind, the permutation to the caller's
    // COO order (for dvals), then the bit-flag word
    const int nstream = nprod + 1 + (KIND == 1 ? 1 : 0);
    const int val_off = nprod * T * IX;  // byte offset of the values in a slot
    const int flag_off = val_off + (nstream - nprod) * T * 4;
    // index u of product-mode stream a, and value u, of a slot
    auto idx_at = [&](const unsigned char *slot, int a, int u) -> uint32_t {
        if constexpr (IX == 4)
            return reinterpret_cast<const uint32_t *>(slot + a * T * 4)[u];
        else
            return reinterpret_cast<const uint16_t *>(slot + a * T * 2)[u];
    };
    const int R = p.R;
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = tid / LPR, lig = tid % LPR;
    const unsigned gmask = LPR == 32 ? kFull : (((1u << LPR) - 1u) << (lane / LPR * LPR));
    const bool has_out = p.out != nullptr;

    extern __shared__ __align__(128) unsigned char smem[];
    const int sbytes = slot_bytes(nstream, nprod, IX);
    const int gstride = group_stride(nstream, RT, nprod, IX);
    unsigned char *ring = smem + (size_t)g * gstride;
    double *s_first = reinterpret_cast<double *>(smem + (size_t)G * gstride);  // [G][RT]
    int64_t *s_pseg = reinterpret_cast<int64_t *>(s_first + (size_t)G * RT);
    int *s_pflag = reinterpret_cast<int *>(s_pseg + 2 * G);
    float *s_loss = reinterpret_cast<float *>(s_pflag + 2 * G);
    float *s_seg = s_loss + G;  // [G][2][RT] segment sums and compensations
    // partial of run-cut segment e (slot 2g: the run's first segment, 2g+1:
    // its last, kept in the group's region once the run is done)
    auto part_ptr = [&](int e) -> double * {
        return (e & 1) ? reinterpret_cast<double *>(smem + (size_t)(e >> 1) * gstride)
                       : s_first + (size_t)(e >> 1) * RT;
    };

    const int64_t c0 = (int64_t)blockIdx.x * p.cta_chunk;
    const int64_t c1 = min(c0 + p.cta_chunk, p.nnz);
    const int64_t r0 = min(c0 + (int64_t)g * p.run_len, c1);
    const int64_t r1 = min(r0 + p.run_len, c1);

    // SpTTMc on a 3-way tensor with vector lanes: a lane holds one E-wide
    // piece bq of the last digit and NCH consecutive first digits, so the one
    // row piece it gathers per nonzero serves all its chunks
    constexpr bool KSH = KIND == 2 && NP == 2 && E > 1;
    constexpr int NCL = KSH ? 1 : NCH;  // row pieces gathered per nonzero
    // columns of this lane: chunk c holds columns (c * LPR + lig) * E + 0..E-1,
    // or for KSH first digit (lig / nbp) * NCH + c, last digits from (lig % nbp) * E
    const int nbp = KSH ? p.Rin / E : 1;
    int col[NCH];
    bool act[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        col[c] = KSH ? ((lig / nbp) * NCH + c) * p.Rin + (lig % nbp) * E : (c * LPR + lig) * E;
        act[c] = col[c] < R;
    }
    // loads use a clamped column so that lanes past R read valid memory
    // unconditionally (their sums are never stored)
    int colc[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) colc[c] = act[c] ? col[c] : 0;
    // factor row width: R, or the per-mode rank Rin of SpTTMc, whose last
    // product mode is read at the last digit of the column and whose first
    // (3-way) contributes the single element at the first digit
    const int Rin = KIND == 2 ? p.Rin : R;
    int colL[NCH], colB[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        colL[c] = KIND == 2 ? colc[c] % Rin : colc[c];
        colB[c] = KIND == 2 ? colc[c] / Rin : colc[c];
    }
    const TF *Fl = static_cast<const TF *>(p.F[nprod - 1]);
    const TF *Fb = static_cast<const TF *>(p.F[0]);

    if (lig == 0) {
        s_pseg[2 * g] = -1;
        s_pseg[2 * g + 1] = -1;
        s_pflag[2 * g] = 0;
        s_pflag[2 * g + 1] = 0;
        s_loss[g] = 0.f;
    }
    if (tid == 0 && has_out) {
        p.carry_seg[2 * blockIdx.x] = -1;
        p.carry_seg[2 * blockIdx.x + 1] = -1;
    }

    if (r0 < r1) {
        const int nst = (int)((r1 - r0 + T - 1) / T);
        // ---- stream prefetch: stage s -> ring slot s % NS
        auto issue_stage = [&](int s) {
            if (s < nst) {
                const int64_t base = r0 + (int64_t)s * T;
                unsigned char *slot = ring + (s % NS) * sbytes;
                constexpr int CPA = T / 4;  // 16-byte pieces per 4-byte stream array
                if constexpr (IX == 2) {
                    // NP 16-bit index arrays (T * 2 bytes each), then the values
                    constexpr int CPI = T * 2 / 16;
#pragma unroll
                    for (int c = lig; c < NP * CPI + CPA; c += LPR) {
                        if (c < NP * CPI) {
                            const int a = c / CPI, q = c % CPI;
                            cp_async16(slot + a * T * 2 + q * 16, p.pidx16[a] + base + q * 8);
                        } else {
                            const int q = c - NP * CPI;
                            cp_async16(slot + val_off + q * 16, p.val + base + q * 4);
                        }
                    }
                } else if constexpr (NP > 0 && LPR <= CPA) {
                    // piece i * LPR + lig: the array is the same for every lane
#pragma unroll
                    for (int i = 0; i < (NP + 1 + (KIND == 1 ? 1 : 0)) * CPA / LPR; ++i) {
                        const int a = i * LPR / CPA, q = i * LPR % CPA + lig;
                        if (a == NP + 1 && (!p.dvals || p.dvals_fcoo)) continue;
                        const void *src = a < NP    ? (const void *)(p.pidx[a] + base + q * 4)
                                          : a == NP ? (const void *)(p.val + base + q * 4)
                                                    : (const void *)(p.perm + base + q * 4);
                        cp_async16(slot + a * T * 4 + q * 16, src);
                    }
                } else {
                    const int nchunks = nstream * CPA;
                    for (int c = lig; c < nchunks; c += LPR) {
                        const int a = c / CPA, q = c % CPA;
                        if (a == nprod + 1 && (!p.dvals || p.dvals_fcoo)) continue;
                        const void *src = a < nprod    ? (const void *)(p.pidx[a] + base + q * 4)
                                          : a == nprod ? (const void *)(p.val + base + q * 4)
                                                       : (const void *)(p.perm + base + q * 4);
                        cp_async16(slot + a * T * 4 + q * 16, src);
                    }
                }
                if (lig == 0) cp_async4(slot + flag_off, p.bf + (base >> 5));
            }
            cp_async_commit();
        };
#pragma unroll
        for (int s = 0; s < NS - 1; ++s) issue_stage(s);

        // segment containing r0 and whether r0 opens it (start-flag of the partition)
        const int64_t part = r0 / p.threadlen;
        const bool head0 = (__ldg(p.sf + (part >> 5)) >> (part & 31)) & 1u;
        int64_t seg = heads_before(p, r0, lig, LPR, gmask) + (head0 ? 1 : 0) - 1;
        int64_t row = p.segrow ? (int64_t)__ldg(p.segrow + seg) : seg;
        bool first = true;  // the current segment is the run's first
        float lsum = 0.f;

        // rows between the previous segment's row and this one hold no nonzeros
        auto fill_gap = [&](int64_t from, int64_t to) { zero_rows<E, NCH>(p.out, R, col, from, to); };
        // output row of the current segment
        float *orow = has_out ? p.out + row * R : nullptr;
        if (has_out && p.segrow && head0) fill_gap(seg > 0 ? (int64_t)__ldg(p.segrow + seg - 1) : -1, row);

        // accumulators: the stage sum in registers; once a segment reaches the
        // end of a stage, its running sum and Kahan compensation move to
        // shared memory (folded once per stage); a segment that starts and
        // ends between two folds never leaves registers.  brow = product of
        // the current fibre's non-last product-mode rows
        float acc_st[NCH][E], brow[NCH][E];
        // SpMTTKRP of a 3-way tensor with BF16 rows: the fibre row stays in
        // its BF16 words, and each nonzero multiplies it into the gathered row
        // exactly (bf16_prod2) before the FP32 multiply-add with the value
        constexpr bool RAWB = std::is_same<TF, __nv_bfloat16>::value && KIND == 0 && NP == 2 && E == 8;
        uint32_t brw[RAWB ? NCH : 1][4];
        float trow[KIND == 1 ? NCH : 1][E];
        float *s_acc = s_seg + (size_t)g * 2 * RT;  // [RT] sum, then [RT] compensation
        float *s_cmp = s_acc + RT;
        bool in_smem = false;  // the current segment has a folded part in s_acc / s_cmp
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                acc_st[c][e] = 0.f;
                brow[c][e] = 1.f;
            }
#pragma unroll
        for (int c = 0; c < (RAWB ? NCH : 1); ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i) brw[c][i] = 0x3f803f80u;  // BF16 ones
        auto set_brw = [&](int c, const raw &r) {
            if constexpr (RAWB) {
                brw[c][0] = r.x, brw[c][1] = r.y, brw[c][2] = r.z, brw[c][3] = r.w;
            }
        };
        auto load_target = [&]() {
            if constexpr (KIND == 1) {
                const TF *Tm = static_cast<const TF *>(p.T);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    if (act[c]) {
                        IO::cvt(IO::load(Tm + (size_t)row * R + col[c]), trow[c]);
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) trow[c][e] = 0.f;  // masks the clamped lanes
                    }
                }
            }
        };
        load_target();

        auto sidx = [&](int c, int e) -> int { return acc_slot<E, LPR>(c, e, lig); };
        // Kahan: segment sum += acc_st (the stage sum), acc_st = 0
        auto fold = [&]() {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                if constexpr (E % 4 == 0) {
#pragma unroll
                    for (int h = 0; h < E / 4; ++h) {
                        float4 *pa = reinterpret_cast<float4 *>(s_acc + sidx(c, 4 * h));
                        float4 *pc = reinterpret_cast<float4 *>(s_cmp + sidx(c, 4 * h));
                        const float *st = &acc_st[c][4 * h];
                        if (in_smem) {
                            const float4 A = *pa, C = *pc;
                            const float a[4] = {A.x, A.y, A.z, A.w}, cm[4] = {C.x, C.y, C.z, C.w};
                            float t[4], nc[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float y = st[i] - cm[i];
                                t[i] = a[i] + y;
                                nc[i] = (t[i] - a[i]) - y;
                            }
                            *pa = make_float4(t[0], t[1], t[2], t[3]);
                            *pc = make_float4(nc[0], nc[1], nc[2], nc[3]);
                        } else {
                            *pa = make_float4(st[0], st[1], st[2], st[3]);
                            *pc = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int i = sidx(c, e);
                        if (in_smem) {
                            const float a = s_acc[i];
                            const float y = acc_st[c][e] - s_cmp[i];
                            const float t = a + y;
                            s_cmp[i] = (t - a) - y;
                            s_acc[i] = t;
                        } else {
                            s_acc[i] = acc_st[c][e];
                            s_cmp[i] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < E; ++e) acc_st[c][e] = 0.f;
            }
            in_smem = true;
        };
        // hand a finished (or run-cut) segment to its writer
        auto emit = [&](bool starts_before, bool continues_after) {
            if (!has_out) return;
            const bool cut = starts_before || continues_after;
            if (!cut && !in_smem) {  // the common case: the stage sum is the segment
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (act[c]) store_row<E>(orow + col[c], acc_st[c]);
                return;
            }
            SegAcc<E, NCH> a;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int e = 0; e < E; ++e) a.v[c][e] = acc_st[c][e];
            const int slot = 2 * g + (first ? 0 : 1);
            double *part = cut ? part_ptr(slot) : nullptr;
            if constexpr (NP == 1)  // short segments: emitted often, one out-of-line copy
                emit_segment_outlined<E, NCH, LPR>(a, in_smem, s_acc, s_cmp, lig, col, R, orow, part);
            else  // calls would cost the register-heavy variants spills in the hot loop
                emit_segment_body<E, NCH, LPR>(a, in_smem, s_acc, s_cmp, lig, col, R, orow, part);
            if (cut && lig == 0) {
                s_pseg[slot] = seg;
                s_pflag[slot] = (starts_before ? 1 : 0) | (continues_after ? 2 : 0);
            }
        };
        // a new segment starts at this nonzero
        auto new_segment = [&]() {
            emit(first && !head0, false);
            first = false;
            in_smem = false;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int e = 0; e < E; ++e) acc_st[c][e] = 0.f;
            ++seg;
            if (p.segrow) {
                const int64_t prev = row;
                row = (int64_t)__ldg(p.segrow + seg);
                if (has_out) {
                    fill_gap(prev, row);
                    orow = p.out + row * R;
                }
            } else {
                ++row;
                if (has_out) orow += R;
            }
            load_target();
        };
        // acc_st += w * (brow * row), w = val (KIND 0) or the residual weight
        // (KIND 1); element pairs go through the paired FP32 instructions
        // (u = position in the stage that starts at nonzero `base`)
        auto accumulate = [&](float v, const raw (&cr)[NCL], const unsigned char *slot, int64_t base, int u) {
            float t[NCL][E];
#pragma unroll
            for (int c = 0; c < NCL; ++c) IO::cvt(cr[c], t[c]);
            if constexpr (RAWB) {
                const float2 v2 = make_float2(v, v);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const uint32_t cw[4] = {cr[c].x, cr[c].y, cr[c].z, cr[c].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 a = __ffma2_rn(v2, bf16_prod2(brw[c][i], cw[i]),
                                                    make_float2(acc_st[c][2 * i], acc_st[c][2 * i + 1]));
                        acc_st[c][2 * i] = a.x;
                        acc_st[c][2 * i + 1] = a.y;
                    }
                }
            } else if constexpr (KIND == 0) {
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    if constexpr (E % 2 == 0) {
                        const float2 v2 = make_float2(v, v);
#pragma unroll
                        for (int e = 0; e < E; e += 2) {
                            // one product mode: there is no other row to multiply (brow = 1)
                            const float2 s = NP == 1 ? v2 : __fmul2_rn(v2, make_float2(brow[c][e], brow[c][e + 1]));
                            const float2 a = __ffma2_rn(s, make_float2(t[c][e], t[c][e + 1]),
                                                        make_float2(acc_st[c][e], acc_st[c][e + 1]));
                            acc_st[c][e] = a.x;
                            acc_st[c][e + 1] = a.y;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) acc_st[c][e] = fmaf(v * brow[c][e], t[c][e], acc_st[c][e]);
                    }
                }
            } else if constexpr (KIND == 2) {
                // Kronecker columns: brow is one element per chunk (the
                // non-last product modes' entries at this lane's digits)
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const float sc = v * brow[c][0];
                    const float *tc = t[NCL == 1 ? 0 : c];
                    if constexpr (E % 2 == 0) {
                        const float2 s2 = make_float2(sc, sc);
#pragma unroll
                        for (int e = 0; e < E; e += 2) {
                            const float2 a = __ffma2_rn(s2, make_float2(tc[e], tc[e + 1]),
                                                        make_float2(acc_st[c][e], acc_st[c][e + 1]));
                            acc_st[c][e] = a.x;
                            acc_st[c][e + 1] = a.y;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) acc_st[c][e] = fmaf(sc, tc[e], acc_st[c][e]);
                    }
                }
            } else {
                // h = brow * row; e = <T(row), h> - val; acc_st += e * h
                float h[NCH][E];
                float d = 0.f;
#pragma unroll
                for (int c = 0; c < NCH; ++c)
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        h[c][e] = brow[c][e] * t[c][e];
                        d = fmaf(trow[c][e], h[c][e], d);
                    }
#pragma unroll
                for (int o = 1; o < LPR; o <<= 1) d += __shfl_xor_sync(gmask, d, o);
                const float w = p.sub_val ? d - v : d;
                if (lig == 0) {
                    lsum = fmaf(w, w, lsum);
                    if (p.dvals) {
                        // in F-COO order, or the caller's COO order through the streamed permutation
                        const int64_t at = p.dvals_fcoo ? base + u
                                                        : (int64_t)reinterpret_cast<const uint32_t *>(
                                                              slot + val_off + T * 4)[u];
                        p.dvals[at] = p.dsign * w;
                    }
                }
#pragma unroll
                for (int c = 0; c < NCH; ++c)
#pragma unroll
                    for (int e = 0; e < E; ++e) acc_st[c][e] = fmaf(w, h[c][e], acc_st[c][e]);
            }
        };
        // brow from the rows of the non-last product modes (general N)
        auto set_brow_sync = [&](const unsigned char *slot, int u) {
            if constexpr (KIND == 2) {
                // the product of F_m(k_m, digit m of the column), m < nprod - 1
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    int q = colB[c];
                    float b = 1.f;
                    for (int m = nprod - 2; m >= 0; --m) {
                        const TF *Fm = static_cast<const TF *>(p.F[m]);
                        const uint32_t km = idx_at(slot, m, u);
                        b *= ld_elem(Fm + (size_t)km * Rin + q % Rin);
                        q /= Rin;
                    }
                    brow[c][0] = b;
                }
                return;
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
#pragma unroll
                for (int e = 0; e < E; ++e) brow[c][e] = 1.f;
                for (int m = 0; m < nprod - 1; ++m) {
                    const TF *Fm = static_cast<const TF *>(p.F[m]);
                    const uint32_t km = idx_at(slot, m, u);
                    float t[E];
                    IO::cvt(IO::load(Fm + (size_t)km * R + colc[c]), t);
#pragma unroll
                    for (int e = 0; e < E; ++e) brow[c][e] *= t[e];
                }
            }
        };

        uint32_t jprev = 0xffffffffu;           // fibre key of the previous nonzero (3-way)
        uint32_t lastkey[FCOO_MAX_MODES - 1];  // fibre keys of the previous nonzero (general)
#pragma unroll
        for (int m = 0; m < FCOO_MAX_MODES - 1; ++m) lastkey[m] = 0xffffffffu;

        // Row addresses: one 32 x 32 -> 64-bit multiply-add from a per-lane base.
        const uint32_t Rb = (uint32_t)Rin * (uint32_t)sizeof(TF);
        const char *Flb[NCH];
        const char *Fbb[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            Flb[c] = reinterpret_cast<const char *>(Fl + colL[c]);
            Fbb[c] = reinterpret_cast<const char *>(Fb + colB[c]);
        }

        // ---- software pipeline over quarters of a stage (Q nonzeros): the
        // gathers of quarter h+1 are in flight while quarter h is consumed.  A
        // full stage is walked by a rolled loop over pairs of quarters (two
        // register buffers); the first quarter of the next stage is requested
        // while the last quarter of the current one is consumed.  Q is 4 where
        // a lane holds at most 4 FP32 columns (2 CTAs per SM) and for the BF16
        // value pass (eight columns in four registers per row: measured 3.5-5 %
        // faster SpMTTKRP than Q = 2 at R = 32 and 64, 14 % faster SpTTM at
        // R = 64); 2 otherwise (FP32 rows of eight columns, whose four-nonzero
        // quarters spill, and the 3-CTA variant).
        constexpr bool BF16V = std::is_same<TF, __nv_bfloat16>::value && E == 8 && KIND == 0;
        constexpr int Q = ((E * NCH <= 4 && !stream_three_ctas<E, NCH, NP, KIND>()) || BF16V) ? 4 : 2;
        constexpr int QPS = T / Q;  // quarters per stage (even)
        static_assert(QPS % 2 == 0, "quarters are consumed in pairs");
        // the unrolled pipeline serves the 3-way SpMTTKRP and SpTTM vector
        // variants; the general-N and scalar ones walk nonzeros one at a time
        constexpr bool PIPE = (NP == 1 || NP == 2) && E > 1;
        // first-product-mode operand: a row piece, or one element (SpTTMc)
        using braw = typename std::conditional<KIND == 2, float, raw>::type;
        struct Quarter {
            raw cr[Q][NCL];
            braw br[NP == 2 ? Q : 1][NCH];
            float vv[Q];
            uint32_t fcm;
        };
        // read quarter qt of a full stage from its slot and start its gathers;
        // hw = the stage's segment-start bits
        auto prefetch = [&](Quarter &b, const unsigned char *slot, int qt, uint32_t hw) {
            const int ub = qt * Q;
            uint32_t kk[Q], jj[Q];
            // Q consecutive indices of product-mode stream a
            auto idx_q = [&](int a, uint32_t (&o)[Q]) {
                if constexpr (IX == 4) {
                    if constexpr (Q == 4) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(slot + a * T * 4 + ub * 4);
                        o[0] = w.x, o[1] = w.y, o[2] = w.z, o[3] = w.w;
                    } else {
                        const uint2 w = *reinterpret_cast<const uint2 *>(slot + a * T * 4 + ub * 4);
                        o[0] = w.x, o[1] = w.y;
                    }
                } else {  // two 16-bit indices per word, the lower position in the low half
                    if constexpr (Q == 4) {
                        const uint2 w = *reinterpret_cast<const uint2 *>(slot + a * T * 2 + ub * 2);
                        o[0] = w.x & 0xffffu, o[1] = w.x >> 16, o[2] = w.y & 0xffffu, o[3] = w.y >> 16;
                    } else {
                        const uint32_t w = *reinterpret_cast<const uint32_t *>(slot + a * T * 2 + ub * 2);
                        o[0] = w & 0xffffu, o[1] = w >> 16;
                    }
                }
            };
            idx_q(nprod - 1, kk);
            if constexpr (Q == 4) {
                const float4 v4 = *reinterpret_cast<const float4 *>(slot + val_off + ub * 4);
                b.vv[0] = v4.x, b.vv[1] = v4.y, b.vv[2] = v4.z, b.vv[3] = v4.w;
            } else {
                const float2 v2 = *reinterpret_cast<const float2 *>(slot + val_off + ub * 4);
                b.vv[0] = v2.x, b.vv[1] = v2.y;
            }
            uint32_t fcm = (hw >> ub) & ((1u << Q) - 1u);
            if constexpr (NP == 2) {
                idx_q(0, jj);
#pragma unroll
                for (int q = 0; q < Q; ++q) fcm |= (uint32_t)(jj[q] != (q ? jj[q - 1] : jprev)) << q;
                jprev = jj[Q - 1];
            } else if constexpr (NP != 1) {
                for (int q = 0; q < Q; ++q) {
                    bool ch = false;
                    for (int m = 0; m < nprod - 1; ++m) {
                        const uint32_t k = idx_at(slot, m, ub + q);
                        ch |= k != lastkey[m];
                        lastkey[m] = k;
                    }
                    fcm |= (uint32_t)ch << q;
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
#pragma unroll
                for (int c = 0; c < NCL; ++c)
                    b.cr[q][c] = IO::load(reinterpret_cast<const TF *>(Flb[c] + (uint64_t)kk[q] * Rb));
                if constexpr (NP == 2) {
                    const bool f = (fcm >> q) & 1u;
                    if constexpr (KSH && NCH == 2 && std::is_same<TF, float>::value) {
                        // the lane's two first digits are adjacent: one 8-byte load
                        const float2 *src = reinterpret_cast<const float2 *>(Fbb[0] + (uint64_t)jj[q] * Rb);
                        const float2 v2 = f ? __ldg(src) : make_float2(0.f, 0.f);
                        b.br[q][0] = v2.x;
                        b.br[q][1] = v2.y;
                    } else {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) {
                            const TF *src = reinterpret_cast<const TF *>(Fbb[c] + (uint64_t)jj[q] * Rb);
                            if constexpr (KIND == 2)
                                b.br[q][c] = f ? ld_elem(src) : 0.f;
                            else
                                b.br[q][c] = IO::load_if(src, f);
                        }
                    }
                }
            }
            b.fcm = fcm;
        };
        // consume quarter qt (hdm = its segment-start bits)
        auto consume = [&](const Quarter &b, const unsigned char *slot, int qt, uint32_t hdm, int64_t base) {
            // SpTTM (one product mode, value weights, rows = segments): the
            // quarters of all groups take the same predicated path whether or
            // not they hold a segment start, so a warp does not split on them
            const bool short_path = NP == 1 && KIND == 0 && !p.segrow && has_out && !first && !in_smem;
            if (hdm == 0 && !short_path) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const bool f = (b.fcm >> q) & 1u;
                    if constexpr (NP == 2 && KIND == 2) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) brow[c][0] = f ? b.br[q][c] : brow[c][0];
                    } else if constexpr (RAWB) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) {
                            const raw &r = b.br[q][c];
                            brw[c][0] = f ? r.x : brw[c][0];
                            brw[c][1] = f ? r.y : brw[c][1];
                            brw[c][2] = f ? r.z : brw[c][2];
                            brw[c][3] = f ? r.w : brw[c][3];
                        }
                    } else if constexpr (NP == 2) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) {
                            float t[E];
                            IO::cvt(b.br[q][c], t);
#pragma unroll
                            for (int e = 0; e < E; ++e) brow[c][e] = f ? t[e] : brow[c][e];
                        }
                    } else if constexpr (NP != 1) {
                        if (f) set_brow_sync(slot, qt * Q + q);
                    }
                    accumulate(b.vv[q], b.cr[q], slot, base, qt * Q + q);
                }
            } else if (short_path) {
                // SpTTM: fibres of one or two nonzeros are the norm, so segment
                // starts take predicated stores and selects instead of a branch
                // per nonzero (a warp's groups would diverge on almost every
                // nonzero).  Within a quarter nothing sets `first` or `in_smem`
                // (folds happen at stage ends), so the test is made once per
                // quarter; a run's first segment and segments that reached a
                // fold take the general path.
                // the lane's first column of the current output row, stepped
                // by one multiply-add per nonzero
                char *ocol = reinterpret_cast<char *>(orow + col[0]);
                const uint32_t rbytes = (uint32_t)R * 4u;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const uint32_t hd = (hdm >> q) & 1u;
#pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        if (hd && act[c])
                            store_row<E>(reinterpret_cast<float *>(ocol) + (col[c] - col[0]), acc_st[c]);
#pragma unroll
                        for (int e = 0; e < E; ++e) acc_st[c][e] = hd ? 0.f : acc_st[c][e];
                    }
                    ocol += (uint64_t)(hd * rbytes);
                    accumulate(b.vv[q], b.cr[q], slot, base, qt * Q + q);
                }
                const int nh = __popc(hdm);
                orow += (int64_t)nh * R;
                seg += nh;
                row += nh;
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    if ((hdm >> q) & 1u) new_segment();
                    if ((b.fcm >> q) & 1u) {
                        if constexpr (NP == 2 && KIND == 2) {
#pragma unroll
                            for (int c = 0; c < NCH; ++c) brow[c][0] = b.br[q][c];
                        } else if constexpr (RAWB) {
#pragma unroll
                            for (int c = 0; c < NCH; ++c) set_brw(c, b.br[q][c]);
                        } else if constexpr (NP == 2) {
#pragma unroll
                            for (int c = 0; c < NCH; ++c) IO::cvt(b.br[q][c], brow[c]);
                        } else if constexpr (NP != 1) {
                            set_brow_sync(slot, qt * Q + q);
                        }
                    }
                    accumulate(b.vv[q], b.cr[q], slot, base, qt * Q + q);
                }
            }
        };
        // ragged last stage: nonzeros one at a time, no pipelining
        auto process_tail = [&](const unsigned char *slot, int64_t base, uint32_t hw, int cnt) {
            const float *sv = reinterpret_cast<const float *>(slot + val_off);
            for (int u = 0; u < cnt; ++u) {
                const bool hd = (hw >> u) & 1u;
                bool f = hd;
                const uint32_t sku = idx_at(slot, nprod - 1, u);
                const uint32_t sju = NP == 2 ? idx_at(slot, 0, u) : 0u;
                if constexpr (NP == 2) {
                    f |= sju != jprev;
                    jprev = sju;
                } else if constexpr (NP != 1) {
                    for (int m = 0; m < nprod - 1; ++m) {
                        const uint32_t k = idx_at(slot, m, u);
                        f |= k != lastkey[m];
                        lastkey[m] = k;
                    }
                }
                raw cr[NCL];
#pragma unroll
                for (int c = 0; c < NCL; ++c)
                    cr[c] = IO::load(reinterpret_cast<const TF *>(Flb[c] + (uint64_t)sku * Rb));
                if (hd) new_segment();
                if (f) {
                    if constexpr (NP == 2 && KIND == 2) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c)
                            brow[c][0] = ld_elem(reinterpret_cast<const TF *>(Fbb[c] + (uint64_t)sju * Rb));
                    } else if constexpr (RAWB) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c)
                            set_brw(c, IO::load(reinterpret_cast<const TF *>(Fbb[c] + (uint64_t)sju * Rb)));
                    } else if constexpr (NP == 2) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c)
                            IO::cvt(IO::load(reinterpret_cast<const TF *>(Fbb[c] + (uint64_t)sju * Rb)), brow[c]);
                    } else if constexpr (NP != 1) {
                        set_brow_sync(slot, u);
                    }
                }
                accumulate(sv[u], cr, slot, base, u);
            }
        };

        Quarter qa, qb;
        bool have_first = false;  // qa already holds quarter 0 of the current stage
#pragma unroll 1
        for (int s = 0; s < nst; ++s) {
            __syncwarp(gmask);  // the previous stage's slot is no longer read
            issue_stage(s + NS - 1);
            cp_async_wait<NS - 1>();
            __syncwarp(gmask);
            const unsigned char *slot = ring + (s % NS) * sbytes;
            const int64_t base = r0 + (int64_t)s * T;
            const int cnt = (int)min((int64_t)T, r1 - base);
            uint32_t hw = *reinterpret_cast<const uint32_t *>(slot + flag_off);
            if (s == 0) hw &= ~1u;  // r0 opens the run, not a new segment
            if (PIPE && cnt == T) {
                if (!have_first) prefetch(qa, slot, 0, hw);
                have_first = false;
                // quarters in pairs (qa, qb alternate), the loop kept rolled so
                // that the code stays small
#pragma unroll 1
                for (int qt = 0; qt < QPS; qt += 2) {
                    prefetch(qb, slot, qt + 1, hw);
                    consume(qa, slot, qt, (hw >> (qt * Q)) & ((1u << Q) - 1u), base);
                    if (qt + 2 < QPS) {
                        prefetch(qa, slot, qt + 2, hw);
                    } else if (s + 1 < nst && r1 - (base + T) >= T) {
                        // the next stage is full: request its first quarter now
                        cp_async_wait<NS - 2>();
                        __syncwarp(gmask);
                        const unsigned char *nslot = ring + ((s + 1) % NS) * sbytes;
                        prefetch(qa, nslot, 0, *reinterpret_cast<const uint32_t *>(nslot + flag_off));
                        have_first = true;
                    }
                    consume(qb, slot, qt + 1, (hw >> ((qt + 1) * Q)) & ((1u << Q) - 1u), base);
                }
            } else {
                process_tail(slot, base, hw, cnt);
            }
            // fold where no segment started in this stage: the open segment
            // then began before it, so its register sum holds at most two
            // stages' terms; a segment that started here stays in registers
            // (it has at most 32 terms), which keeps short segments off the
            // folded path
            if ((hw & (cnt == T ? kFull : (1u << cnt) - 1u)) == 0u) fold();
        }
        // ---- end of run: the last segment (its partial may go to the ring
        // region, so every lane of the group must be done with the ring)
        cp_async_wait<0>();
        __syncwarp(gmask);
        const bool ends_here = (r1 == p.nnz) || head_at(p, r1);
        emit(first && !head0, !ends_here);
        if (has_out && p.segrow && r1 == p.nnz) fill_gap(row, p.out_rows);
        if (KIND == 1 && lig == 0) s_loss[g] = lsum;
    }

    // lane groups of one warp leave their runs at different points: reconverge
    // the warp before the CTA barrier
    __syncwarp();
    __syncthreads();
    if (KIND == 1 && p.loss_part) {
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < G; ++q) s += (double)s_loss[q];
            p.loss_part[blockIdx.x] = s;
        }
    }
    if (!has_out) return;
    // ---- combine the run-cut segments of this CTA in run order (FP64)
    const int last_group = (int)min((int64_t)G - 1, (c1 - c0 + p.run_len - 1) / p.run_len - 1);
    for (int t = tid; t < R; t += kThreads) {
        int64_t cur = -1;
        double sum = 0.0;
        int cur_first_e = -1, cur_last_e = -1;
        auto flush = [&]() {
            if (cur < 0) return;
            const bool before = cur_first_e / 2 == 0 && (s_pflag[cur_first_e] & 1);
            const bool after = cur_last_e / 2 == last_group && (s_pflag[cur_last_e] & 2);
            if (before || after) {
                const int64_t slot = 2 * (int64_t)blockIdx.x + (before ? 0 : 1);
                p.carry_val[slot * R + t] = sum;
                if (t == 0) p.carry_seg[slot] = (cur << 2) | (before ? 1 : 0) | (after ? 2 : 0);
            } else {
                const int64_t orow = p.segrow ? (int64_t)__ldg(p.segrow + cur) : cur;
                p.out[orow * R + t] = (float)sum;
            }
        };
        for (int e = 0; e < 2 * G; ++e) {
            const int64_t sg = s_pseg[e];
            if (sg < 0) continue;
            if (sg != cur) {
                flush();
                cur = sg;
                sum = 0.0;
                cur_first_e = e;
            }
            cur_last_e = e;
            sum += part_ptr(e)[t];
        }
        flush();
    }
}

// One block per CTA boundary b (between CTAs b-1 and b).  If a segment crosses
// b and b is the first boundary it crosses, this block adds its carries -- CTA
// b-1's, then CTA b, b+1, ... up to the CTA where it ends -- in CTA order and
// stores the output row.
__global__ void __launch_bounds__(256) k_carry_fixup(const StreamParams p) {
    const int b = blockIdx.x + 1;
    if (b >= p.grid) return;
    const int64_t e1 = p.carry_seg[2 * (b - 1) + 1], e0 = p.carry_seg[2 * (b - 1)];
    int aslot;
    int64_t a;
    if (e1 >= 0 && (e1 & 2)) {
        a = e1;
        aslot = 1;
    } else if (e0 >= 0 && (e0 & 2)) {
        a = e0;
        aslot = 0;
    } else {
        return;  // boundary b cuts no segment
    }
    if (a & 1) return;  // the segment started before CTA b-1: an earlier block owns it
    const int64_t seg = a >> 2;
    __shared__ int s_end;
    if (threadIdx.x == 0) s_end = INT_MAX;
    __syncthreads();
    for (int base = b; base < p.grid; base += blockDim.x) {
        const int j = base + threadIdx.x;
        if (j < p.grid) {
            const int64_t c = p.carry_seg[2 * (int64_t)j];
            if (c < 0 || !(c & 2)) atomicMin(&s_end, j);
        }
        __syncthreads();
        const bool done = s_end != INT_MAX;
        __syncthreads();
        if (done) break;
    }
    const int end = min(s_end, p.grid - 1);
    const int count = end - b + 2;  // (b-1, aslot) then (j, 0) for j = b..end
    const int nw = blockDim.x / 32, w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int R = p.R;
    double acc[FCOO_MAX_RANK / 32];
#pragma unroll
    for (int i = 0; i < FCOO_MAX_RANK / 32; ++i) acc[i] = 0.0;
    for (int k = w; k < count; k += nw) {
        const int64_t slot = k == 0 ? 2 * (int64_t)(b - 1) + aslot : 2 * (int64_t)(b + k - 1);
#pragma unroll
        for (int i = 0; i < FCOO_MAX_RANK / 32; ++i) {
            const int t = lane + 32 * i;
            if (t < R) acc[i] += __ldcg(p.carry_val + slot * R + t);
        }
    }
    __shared__ double s_w[8][FCOO_MAX_RANK];
#pragma unroll
    for (int i = 0; i < FCOO_MAX_RANK / 32; ++i) {
        const int t = lane + 32 * i;
        if (t < R) s_w[w][t] = acc[i];
    }
    __syncthreads();
    const int64_t row = p.segrow ? (int64_t)__ldg(p.segrow + seg) : seg;
    for (int t = threadIdx.x; t < R; t += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += s_w[q][t];
        p.out[row * R + t] = (float)s;
    }
}

// ------------------------------------------------------------ launch

template <typename TF, int E, int LPR, int NCH, int NP, int KIND, int IX = 4>
int launch_variant(StreamParams &p, cudaStream_t s) {
    constexpr int G = kThreads / LPR;
    constexpr int RT = NCH * LPR * E;
    auto kern = k_stream<TF, E, LPR, NCH, NP, KIND, IX>;
    // the shared memory size depends on the number of streams, which the
    // general-N variant (NP = 0) takes at run time: one cache per size
    const int nstream = p.nprod + 1 + (KIND == 1 ? 1 : 0);
    const size_t smem = stream_smem_bytes(nstream, G, RT, p.nprod, IX);
    int dev = 0, occ = 0;
    FCOO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FCOO_ERR_UNSUPPORTED, "device %d above %d", dev, kMaxDevices);
    {
        // per device: the largest shared-memory size the kernel was enabled
        // for (only ever raised, so a launch never finds it lowered by
        // another size), and its residency per stream count
        static std::mutex mu;
        static size_t attr_smem[kMaxDevices];
        static int occ_plus1[kMaxDevices][FCOO_MAX_MODES + 2];
        std::lock_guard<std::mutex> lock(mu);
        if (smem > attr_smem[dev]) {
            FCOO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_smem[dev] = smem;
        }
        if (!occ_plus1[dev][nstream]) {
            FCOO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
            if (occ < 1) return fail(FCOO_ERR_UNSUPPORTED, "stream kernel does not fit on an SM (smem %zu)", smem);
            occ_plus1[dev][nstream] = occ + 1;
        }
        occ = occ_plus1[dev][nstream] - 1;
    }
    const int64_t ra = p.threadlen > 32 ? p.threadlen : 32;
    const int64_t max_ctas =
        std::max<int64_t>(1, std::min<int64_t>((int64_t)device_sms(dev) * occ - p.reserve_ctas, p.grid));
    int64_t grid = std::min<int64_t>(max_ctas, ceil_div(p.nnz, (int64_t)G * ra));
    if (grid < 1) grid = 1;
    p.run_len = round_up(ceil_div(p.nnz, grid * G), ra);
    p.cta_chunk = p.run_len * G;
    grid = ceil_div(p.nnz, p.cta_chunk);
    p.grid = (int)grid;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(p);
    FCOO_CUDA(cudaGetLastError());
    if (p.out && grid > 1) {
        k_carry_fixup<<<(unsigned)(grid - 1), 256, 0, s>>>(p);
        FCOO_CUDA(cudaGetLastError());
    }
    return FCOO_OK;
}

template <typename TF, int E, int LPR, int NCH, int KIND>
int launch_np(StreamParams &p, cudaStream_t s) {
    // a compressed handle's 16-bit index streams serve the value kind with
    // one or two product modes
    const bool ix16 = KIND == 0 && p.pidx16[0] != nullptr;
    switch (p.nprod) {
        case 1:
            if constexpr (KIND == 0) {
                if (ix16) return launch_variant<TF, E, LPR, NCH, 1, KIND, 2>(p, s);
                return launch_variant<TF, E, LPR, NCH, 1, KIND>(p, s);
            }
            return launch_variant<TF, E, LPR, NCH, 0, KIND>(p, s);
        case 2:
            if constexpr (KIND == 0)
                if (ix16) return launch_variant<TF, E, LPR, NCH, 2, KIND, 2>(p, s);
            return launch_variant<TF, E, LPR, NCH, 2, KIND>(p, s);
        default: return launch_variant<TF, E, LPR, NCH, 0, KIND>(p, s);
    }
}

// eight columns per lane (FP32: one 32-byte load per row, BF16: one 16-byte
// load), lane groups of 4..32 lanes for R up to 256
template <typename TF, int KIND>
int launch_v8(StreamParams &p, cudaStream_t s) {
    const int chunks = (p.R + 7) / 8;
    if (chunks <= 4) return launch_np<TF, 8, 4, 1, KIND>(p, s);
    if (chunks <= 8) return launch_np<TF, 8, 8, 1, KIND>(p, s);
    if (chunks <= 16) return launch_np<TF, 8, 16, 1, KIND>(p, s);
    if (chunks <= 32) return launch_np<TF, 8, 32, 1, KIND>(p, s);
    return fail(FCOO_ERR_UNSUPPORTED, "R=%d above the supported rank", p.R);
}

// scalar lanes for ranks that are not a multiple of the vector width
template <typename TF, int KIND>
int launch_scalar(StreamParams &p, cudaStream_t s) {
    const int nch = (p.R + 31) / 32;
    if (nch <= 1) return launch_variant<TF, 1, 32, 1, 0, KIND>(p, s);
    if (nch <= 2) return launch_variant<TF, 1, 32, 2, 0, KIND>(p, s);
    if (nch <= 4) return launch_variant<TF, 1, 32, 4, 0, KIND>(p, s);
    return launch_variant<TF, 1, 32, 8, 0, KIND>(p, s);
}

bool aligned(const void *q, uintptr_t a) { return q == nullptr || ((uintptr_t)q & (a - 1)) == 0; }

// SpTTMc (kind 2): output width R = Rin^nprod.  3-way tensors with Rin = 8
// or 16 (R = 64 or 256) take eight-column lanes (FP32 or BF16 rows), Rin = 4
// (R = 16, FP32) four-column lanes, each lane gathering one row piece per nonzero for all its chunks
// ((LPR / (Rin / E)) * NCH = Rin); every other shape the scalar lanes of the
// general path.
template <typename TF>
int launch_kron(StreamParams &p, cudaStream_t s) {
    auto all_aligned = [&](uintptr_t a) {
        bool ok = aligned(p.out, 16);
        for (int m = 0; m < p.nprod; ++m) ok = ok && aligned(p.F[m], a);
        return ok;
    };
    if (p.nprod == 2 && p.Rin % 8 == 0 && all_aligned(32)) {
        // lanes of (first-digit group, last-digit piece), two first digits
        // per lane: 4 x 1 lanes for Rin = 8, 8 x 2 for Rin = 16 (measured on
        // the skewed 3-way tensor: 9 % and 1.47x faster than one first digit
        // per lane; four digits per lane, at one CTA per SM, gained nothing)
        if (p.Rin == 8) return launch_variant<TF, 8, 4, 2, 2, 2>(p, s);
        if (p.Rin == 16) return launch_variant<TF, 8, 16, 2, 2, 2>(p, s);
    }
    if constexpr (std::is_same<TF, float>::value)  // four-column lanes: FP32 rows only
        if (p.nprod == 2 && p.Rin == 4 && all_aligned(16)) return launch_variant<TF, 4, 4, 1, 2, 2>(p, s);
    const int nch = (p.R + 31) / 32;
    if (nch <= 1) return launch_variant<TF, 1, 32, 1, 0, 2>(p, s);
    if (nch <= 2) return launch_variant<TF, 1, 32, 2, 0, 2>(p, s);
    if (nch <= 4) return launch_variant<TF, 1, 32, 4, 0, 2>(p, s);
    return launch_variant<TF, 1, 32, 8, 0, 2>(p, s);
}

// Lane layout by factor type, rank and alignment: eight columns per lane
// when R is a multiple of 8 (FP32 from R = 24 on; rows 32-byte aligned),
// four FP32 columns per lane in groups of 4 for R <= 16, scalar lanes
// otherwise.
template <typename TF, int KIND>
int launch_typed(StreamParams &p, cudaStream_t s) {
    auto all_aligned = [&](uintptr_t a) {
        bool ok = aligned(p.out, 16) && aligned(p.T, a);
        for (int m = 0; m < p.nprod; ++m) ok = ok && aligned(p.F[m], a);
        return ok;
    };
    if constexpr (std::is_same<TF, float>::value) {
        if (p.R % 4 == 0 && p.R <= 16 && all_aligned(16)) return launch_np<TF, 4, 4, 1, KIND>(p, s);
        if (p.R % 8 == 0 && all_aligned(32)) return launch_v8<TF, KIND>(p, s);
    } else {
        if (p.R % 8 == 0 && all_aligned(16)) return launch_v8<TF, KIND>(p, s);
    }
    return launch_scalar<TF, KIND>(p, s);
}

}  // namespace
}  // namespace fcx
