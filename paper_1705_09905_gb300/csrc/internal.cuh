// internal.cuh -- handle layout, status plumbing and small device helpers
// shared by the libfcoo CUDA sources (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fcoo.h"

namespace fcx {

// Nonzeros per segment-count checkpoint (hcount table).
constexpr int kChunk = 1024;
// Every stream array is padded to a multiple of this many nonzeros, so that
// vector loads of a whole stage never leave the allocation.
constexpr int kPad = 2048;
// Threads per CTA of the streaming kernels.
constexpr int kThreads = 256;
// Upper bound on CTAs per SM the streaming kernels are launched with.
constexpr int kMaxCtasPerSm = 8;

// Record a failure message for fcoo_last_error() and return `status`.
int fail(int status, const char *fmt, ...);
// Map a CUDA error to FCOO_ERR_CUDA / FCOO_ERR_NOMEM with a message.
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Device allocation through the fault-injection hook (FCOO_FAULT_ALLOC).
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p);
void dev_free_async(void *p, cudaStream_t s);

int num_sms();
// SM count of device `dev`, looked up once per device (thread-safe).
int device_sms(int dev);
// Devices a process may use with per-device cached launch data.
constexpr int kMaxDevices = 64;

#define FCOO_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::fcx::cuda_fail(e_, #call);  \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

}  // namespace fcx

// The opaque handle behind fcoo_t (Sec. IV-B layout plus the segment map).
struct fcoo {
    int nmodes, mode, op, threadlen;
    int64_t nnz, npad, nseg, nfib;
    uint32_t dims[FCOO_MAX_MODES];
    int nprod, prod_modes[FCOO_MAX_MODES];
    int nidx, idx_modes[FCOO_MAX_MODES];
    int device;
    // one device allocation, carved into the arrays below
    void *base;
    size_t base_bytes;
    uint32_t *pidx[FCOO_MAX_MODES];  // nprod streams of npad product-mode indices
    float *val;                      // npad values
    uint32_t *bf;                    // npad/32 bit-flag words (1 = segment head)
    uint32_t *sf;                    // start-flag words, one bit per threadlen partition
    uint32_t *segkeys;               // nseg x nidx index-mode tuples
    uint32_t *hcount;                // heads before chunk c (kChunk nonzeros each), nchunk+1
    uint32_t *perm;                  // npad: original COO position of each nonzero
    // 16-bit copies of the product-mode streams (fcoo_compress_indices), in
    // one allocation of nprod * npad uint16; NULL until compressed
    uint16_t *pidx16[FCOO_MAX_MODES];
    void *base16;
    // kernel scratch: carry partials (FP64) and their segment ids, and the
    // arrival counter of the last-CTA combine
    double *carry_val;
    int64_t *carry_seg;
    unsigned int *counter;
    double *red_part;  // max_grid per-CTA partial sums (loss)
    int max_grid;
    // sparse-fit gradient scratch, allocated on first use.  On the handle the
    // residuals are computed on: e in its F-COO order, one other mode's copy
    // of e, and an inverse permutation (npad entries each).  On the other
    // handles: gmap[p] = position in the source handle's order of nonzero p,
    // valid for the handle whose uid is gmap_src.
    float *grad_scratch;
    uint32_t *gmap;
    uint64_t gmap_src;
    uint64_t uid;  // unique per handle built in this process
    int64_t bytes_val, bytes_pidx, bytes_bf, bytes_sf, bytes_segmap, bytes_aux, bytes_scratch;
};

namespace fcx {

// Launch parameters for the streaming segmented-reduction kernels (SpMTTKRP,
// SpTTM, and the adjoint passes, which are SpMTTKRP-shaped).
struct StreamParams {
    const uint32_t *pidx[FCOO_MAX_MODES - 1];  // product-mode streams
    const uint16_t *pidx16[FCOO_MAX_MODES - 1];  // the same in 16 bits, or NULL
    const void *F[FCOO_MAX_MODES - 1];         // matching dense rows (dtype)
    const float *val;                          // values (or per-nonzero weights)
    const uint32_t *bf, *sf, *hcount;
    const uint32_t *segrow;  // segment -> output row; NULL: row = segment id
    float *out;               // output rows, or NULL for a pass that only produces weights / loss
    double *carry_val;        // [2 * grid][R] partials of segments cut by CTA boundaries
    int64_t *carry_seg;       // [2 * grid] (segment << 2) | before(1) | after(2), -1 = empty
    unsigned int *counter;
    // residual weights (sparse CP fit, adjoint of SpMTTKRP): per nonzero
    //   e = <T(row), prod of product-mode rows> - (sub_val ? val : 0)
    const void *T;            // target rows (dtype of F), row = output row of the segment
    const uint32_t *perm;     // F-COO position -> original COO position
    float *dvals;             // dvals[perm[p]] = dsign * e, or NULL
    int dvals_fcoo;           // 1: dvals[p] (F-COO order) instead of dvals[perm[p]]
    float dsign;
    int sub_val;
    double *loss_part;        // per-CTA sum of e^2, or NULL
    int64_t nnz;
    int64_t nseg;
    int64_t out_rows;
    int R;              // output row width (SpTTMc: Rin^nprod)
    int Rin;            // SpTTMc: rank of every factor; unused by the other kinds
    int nprod;
    int threadlen;
    int grid;
    int reserve_ctas;   // CTA slots left free for a kernel running beside this one
    int64_t cta_chunk;  // nonzeros per CTA (multiple of groups * run alignment)
    int64_t run_len;    // nonzeros per group run
};

// Fill the stream part of StreamParams from a handle.
void stream_params_from(const fcoo_t *X, StreamParams &p);

// Launch the segmented-reduction kernel for dtype / R (spmttkrp.cu); kind 0
// weights every nonzero by its value, kind 1 by the residual weight above,
// kind 2 by its value with Kronecker output columns (SpTTMc).
int launch_stream_kernel(StreamParams &p, int dtype, cudaStream_t s, int kind = 0);
// The instantiations, one translation unit each (stream_*.cu).
int launch_stream_f32_k0(StreamParams &p, cudaStream_t s);
int launch_stream_f32_k1(StreamParams &p, cudaStream_t s);
int launch_stream_bf16_k0(StreamParams &p, cudaStream_t s);
int launch_stream_bf16_k1(StreamParams &p, cudaStream_t s);
int launch_stream_f32_k2(StreamParams &p, cudaStream_t s);
int launch_stream_bf16_k2(StreamParams &p, cudaStream_t s);

// G = F^T F (R x R, FP64) of an I x R FP32 matrix: compensated (Dot2) FP32
// partials over 128-row blocks (part: ceil(I/128) * R * R doubles), summed in
// FP64 (cp_als.cu).  R <= 128.
int gram_f32_fp64(const float *F, int64_t I, int R, double *part, double *G, cudaStream_t s);
// *out = sum of val[p]^2 in FP64 (part: 1024 doubles).
int sumsq_fp64(const float *val, int64_t n, double *part, double *out, cudaStream_t s);

}  // namespace fcx
