/*
 * fcoo.h -- C ABI of libfcoo.so, a GB300 (sm_103a) implementation of the
 * F-COO sparse tensor kernels of "A Unified Optimization Approach for Sparse
 * Tensor Operations on GPUs" (Liu, Wen, Sarwate, Mehri Dehnavi, 2017).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Tensors are N-way (2 <= N <= FCOO_MAX_MODES) coordinate lists with
 *    0-based indices (the paper is 1-based, Sec. II).  Index arrays are
 *    uint32, one per mode; values are float32.
 *  - Dense matrices (factor matrices, U, outputs) are row-major with R
 *    contiguous columns per row: element (i, r) lives at ptr[i * R + r].
 *    Device pointers must be 16-byte aligned.
 *  - "host or device" pointers are classified with cudaPointerGetAttributes;
 *    everything else named "device" must be device memory of the current
 *    device.  Nothing is retained after a call returns except inside the
 *    opaque handles, which own their device memory.
 *  - Streams are cudaStream_t values (NULL = legacy default stream).  Compute
 *    entry points are asynchronous on that stream unless documented as
 *    synchronous; argument errors are reported synchronously, kernel errors by
 *    the next synchronous call.
 *  - Every entry point returns FCOO_OK (0) or a negative status; the calling
 *    thread's last error message is available from fcoo_last_error().  No
 *    entry point aborts, traps or prints.
 *  - A handle must not be used by two calls that overlap on the GPU (the
 *    kernels share the handle's scratch memory); issue them on one stream.
 */
#ifndef FCOO_H
#define FCOO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif
#ifdef __cplusplus
extern "C" {
#endif

#define FCOO_MAX_MODES 8
/* Largest rank (columns R) the kernels accept. */
#define FCOO_MAX_RANK 256
/* Largest number of nonzeros one handle holds. */
#define FCOO_MAX_NNZ 2147479552LL

typedef struct CUstream_st *fcoo_stream_t; /* same type as cudaStream_t */
typedef struct fcoo fcoo_t;
typedef struct cp_state cp_state_t;

typedef enum { FCOO_F32 = 0, FCOO_BF16 = 1 } fcoo_dtype;

/* Table I: which modes are product modes and which are index modes. */
typedef enum { FCOO_OP_MTTKRP = 0, FCOO_OP_TTM = 1 } fcoo_op;

enum {
    FCOO_OK = 0,
    FCOO_ERR_INVALID_ARG = -1, /* bad pointer, size, mode, rank, dtype, ...   */
    FCOO_ERR_INDEX_RANGE = -2, /* an index >= its dimension                    */
    FCOO_ERR_DUPLICATE = -3,   /* two nonzeros with identical coordinates      */
    FCOO_ERR_NOMEM = -4,       /* a device or host allocation failed           */
    FCOO_ERR_CUDA = -5,        /* a CUDA runtime call failed                   */
    FCOO_ERR_NOT_PD = -6,      /* normal equations could not be solved         */
    FCOO_ERR_NONFINITE = -7,   /* NaN or Inf met where a finite value is needed */
    FCOO_ERR_TIMEOUT = -8,     /* a bounded device wait gave up                */
    FCOO_ERR_UNSUPPORTED = -9  /* valid request outside this build's limits    */
};

/* Description of a built F-COO handle (fcoo_info). */
typedef struct {
    int nmodes, mode, op, threadlen;
    int64_t nnz;
    int64_t nseg;  /* index-mode tuples = output rows written (SpMTTKRP) or fibres (SpTTM) */
    int64_t nfib;  /* distinct (index modes, all product modes but the last) tuples */
    uint32_t dims[FCOO_MAX_MODES];
    int nprod, prod_modes[FCOO_MAX_MODES]; /* product modes, in stream order (Table I) */
    int nidx, idx_modes[FCOO_MAX_MODES];   /* index modes, in sort order (Table I)     */
    /* Table II terms: val (4 B/nnz), product-mode indices (4 B/nnz each),
     * bit-flags (1 bit/nnz, packed in 32-bit words) and start-flags (1 bit per
     * partition of threadlen nonzeros, packed in 32-bit words). */
    int64_t bytes_val, bytes_pidx, bytes_bf, bytes_sf;
    int64_t bytes_table2;  /* sum of the four terms above                   */
    int64_t bytes_segmap;  /* segment -> output row / fibre index tuples     */
    int64_t bytes_aux;     /* segment counts per 1024 nonzeros, permutation  */
    int64_t bytes_scratch; /* carry buffers used by the kernels              */
    int64_t bytes_pidx16;  /* 16-bit product-mode index streams, 2 B/nnz each
                              (0 unless fcoo_compress_indices was called)   */
} fcoo_info_t;

/* ---------------------------------------------------------------------- */
/* Library                                                                 */
/* ---------------------------------------------------------------------- */

/* Message describing the calling thread's most recent failure ("" if none).
 * The pointer stays valid until the thread's next failing call. */
const char *fcoo_last_error(void);

/* Static name of a status code. */
const char *fcoo_status_string(int status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int fcoo_version(void);

/* Host-only: bytes of the four Table II arrays that fcoo_build allocates for
 * a tensor with `nprod` product modes (Table II; nprod = 2 for 3-way
 * SpMTTKRP, 1 for SpTTM): 4*nnz (val) + 4*nprod*nnz (indices) +
 * 4*ceil(nnz/32) (bf) + 4*ceil(ceil(nnz/threadlen)/32) (sf).  For nnz a
 * multiple of 32*threadlen this is exactly (4 + 4*nprod + 1/8 +
 * 1/(8*threadlen)) * nnz.  Returns -1 on bad arguments. */
int64_t fcoo_table2_bytes(int nprod, int64_t nnz, int threadlen);

/* The same with `index_bytes` (4 or 2) bytes per product-mode index: the
 * Table II arrays of a handle after fcoo_compress_indices (index_bytes = 2)
 * are 4*nnz + 2*nprod*nnz + the two flag arrays.  Returns -1 on bad
 * arguments. */
int64_t fcoo_table2_bytes_ex(int nprod, int64_t nnz, int threadlen, int index_bytes);

/* ---------------------------------------------------------------------- */
/* F-COO construction (Sec. IV-B, Table I, Table II, Fig. 2; host          */
/* preprocessing of Sec. IV-D "Complete tensor-based algorithms")          */
/* ---------------------------------------------------------------------- */

/* Build the F-COO form of an N-way COO tensor for one operation on one
 * mode, on the GPU:
 *   - op = FCOO_OP_MTTKRP: index mode = `mode`, product modes = all others
 *     in ascending order;  op = FCOO_OP_TTM: product mode = `mode`, index
 *     modes = all others in ascending order (Table I);
 *   - nonzeros are sorted lexicographically by (index modes, product modes);
 *   - the stream holds, per nonzero, the product-mode indices and the value
 *     (Table II); the bit-flag array marks with a 1 every nonzero that starts
 *     a new index-mode tuple (a new slice for SpMTTKRP, a new fibre for
 *     SpTTM; the paper's toggling bit changes at exactly these positions,
 *     Fig. 2); the start-flag array holds one bit per partition of
 *     `threadlen` nonzeros, set when the partition starts a new tuple;
 *   - the index-mode tuple of each segment is kept (the output row of an
 *     SpMTTKRP segment, the fibre index of an SpTTM output fibre), so slices
 *     without nonzeros are allowed.
 * Arguments:
 *   nmodes    N, 2..FCOO_MAX_MODES
 *   dims      host array of N dimensions, each >= 1
 *   nnz       0..FCOO_MAX_NNZ
 *   idx       host array of N pointers (host or device), idx[k][p] < dims[k]
 *   val       nnz values (host or device)
 *   mode      0..N-1
 *   op        FCOO_OP_MTTKRP or FCOO_OP_TTM
 *   threadlen nonzeros per partition, a power of two 1..64 (the paper packs
 *             the flags of one partition in a uint8..uint64: 8..64; Fig. 2
 *             illustrates 4)
 *   stream    stream for the device work
 *   out       receives the handle (NULL on failure)
 * The inputs are copied; the caller keeps ownership.  Synchronous: the
 * stream is synchronised before return.  Errors: FCOO_ERR_INVALID_ARG,
 * FCOO_ERR_INDEX_RANGE, FCOO_ERR_DUPLICATE, FCOO_ERR_NOMEM, FCOO_ERR_CUDA.
 * Environment FCOO_FAULT_ALLOC=k makes the k-th device allocation of the
 * process fail (test hook; k counts from 1). */
int fcoo_build(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx, const float *val,
               int mode, int op, int threadlen, fcoo_stream_t stream, fcoo_t **out);

/* Free a handle and its device memory (NULL is accepted).  Synchronises the
 * device first so that no kernel still reads the handle. */
int fcoo_destroy(fcoo_t *X);

/* Fill *info (host struct) from the handle.  Host only, no device work. */
int fcoo_info(const fcoo_t *X, fcoo_info_t *info);

/* Copy parts of the layout to host buffers (any may be NULL).  Synchronous.
 *   perm     nnz uint32: original COO position of the q-th nonzero in F-COO order
 *   bf       ceil(nnz/32) uint32 words, bit (p % 32) of word p/32 = flag of nonzero p
 *   sf       ceil(ceil(nnz/threadlen)/32) uint32 words, bit t%32 of word t/32
 *   segkeys  nseg * nidx uint32: index-mode tuple of each segment
 *   pidx     nprod * nnz uint32: product-mode index streams, one after the other
 *   val      nnz float32 values in F-COO order */
int fcoo_copy_layout(const fcoo_t *X, uint32_t *perm, uint32_t *bf, uint32_t *sf, uint32_t *segkeys,
                     uint32_t *pidx, float *val, fcoo_stream_t stream);

/* Index compression (Table II with 16-bit indices): adds to the handle a copy
 * of every product-mode index stream in 16 bits (2 bytes per nonzero and
 * stream instead of 4), allowed when every product-mode dimension is at most
 * 65,536.  Afterwards spmttkrp and spttm read these streams wherever their
 * kernel takes them: 3-way SpMTTKRP and SpTTM of any order, with factor rows
 * of eight FP32 or BF16 columns per lane (R a multiple of 8, rows 32-byte
 * (FP32) or 16-byte (BF16) aligned) or four FP32 columns per lane (R = 4..16
 * in steps of 4, rows 16-byte aligned).  Other calls and shapes keep reading the
 * 32-bit streams, which stay in the handle.  The results are bitwise equal
 * to those from the 32-bit streams (same reduction order).  Calling it again
 * is a no-op.  Synchronous.  Errors: FCOO_ERR_INVALID_ARG (NULL handle),
 * FCOO_ERR_UNSUPPORTED (a product-mode dimension above 65,536),
 * FCOO_ERR_NOMEM, FCOO_ERR_CUDA. */
int fcoo_compress_indices(fcoo_t *X, fcoo_stream_t stream);

/* Index tuples of the SpTTM output fibres (the semi-sparse result of Eq. 3,
 * Sec. II): nseg rows of (N-1) uint32, in output-row order, written to host
 * or device memory `keys`.  Synchronous.  For an SpMTTKRP handle it returns
 * the output row of each segment (nseg values). */
int fcoo_fibre_indices(const fcoo_t *X, uint32_t *keys, fcoo_stream_t stream);

/* ---------------------------------------------------------------------- */
/* SpMTTKRP (Eq. 5, Eq. 6, Table I row 2; one-shot product of Sec. IV-C;    */
/* segmented reduction of Sec. IV-D)                                        */
/* ---------------------------------------------------------------------- */

/* out(i, :) = sum over nonzeros p with idx_mode(p) = i of
 *             val(p) * prod_{k != mode} F_k(idx_k(p), :)
 * X        handle built with op = FCOO_OP_MTTKRP
 * factors  host array of N device pointers; factors[k] is dims[k] x R of
 *          dtype (FCOO_F32 or FCOO_BF16); factors[mode] is not read (may be NULL)
 * R        1..FCOO_MAX_RANK
 * out      device float32 dims[mode] x R; every element is written (rows
 *          without nonzeros are set to 0); no pre-zeroing needed
 * The reduction order is fixed by the handle and R, so repeated calls give
 * bitwise identical results.  Asynchronous on `stream`. */
int spmttkrp(const fcoo_t *X, const void *const *factors, int dtype, int R, float *out, fcoo_stream_t stream);

/* ---------------------------------------------------------------------- */
/* SpTTM (Eq. 3, Table I row 1; semi-sparse output of Sec. II)              */
/* ---------------------------------------------------------------------- */

/* Y(f, :) = sum over nonzeros p in output fibre f of val(p) * U(idx_mode(p), :)
 * X    handle built with op = FCOO_OP_TTM
 * U    device dims[mode] x R of dtype
 * out  device float32 nseg x R; row f is the fibre whose index tuple is row f
 *      of fcoo_fibre_indices (lexicographic order); every element written.
 * Asynchronous on `stream`. */
int spttm(const fcoo_t *X, const void *U, int dtype, int R, float *out, fcoo_stream_t stream);

/* ---------------------------------------------------------------------- */
/* SpTTMc (Eq. 4, Table I row 3): the tensor times a matrix on every mode  */
/* but one, the core of Tucker decomposition by HOOI (Sec. II)            */
/* ---------------------------------------------------------------------- */

/* out(i, c) = sum over nonzeros p with idx_mode(p) = i of
 *             val(p) * prod_{t} U_{k_t}(idx_{k_t}(p), r_t)
 * where k_0 < k_1 < ... are the modes other than `mode` and the output column
 * c = ((r_0 * R + r_1) * R + ...) holds the digits r_t of the row-vector
 * Kronecker product U_{k_0}(j, :) (x) U_{k_1}(k, :) (x) ... (Eq. 1); the
 * first product mode varies slowest.
 * X        handle built with op = FCOO_OP_MTTKRP (the same handle SpMTTKRP uses)
 * factors  host array of N device pointers; factors[k] is dims[k] x R of
 *          dtype, row-major; factors[mode] is not read (may be NULL)
 * dtype    FCOO_F32 or FCOO_BF16 (BF16 storage, FP32 products and sums)
 * R        per-mode rank, R >= 1 with R^(N-1) <= FCOO_MAX_RANK
 *          (FCOO_ERR_UNSUPPORTED above)
 * out      device float32 dims[mode] x R^(N-1), row-major; every element is
 *          written (rows without nonzeros are set to 0)
 * Deterministic for a given handle and R, like spmttkrp.  Asynchronous on
 * `stream`. */
int spttmc(const fcoo_t *X, const void *const *factors, int dtype, int R, float *out, fcoo_stream_t stream);

/* SpTTMc of a 3-way tensor by fibres: Eq. 4 regrouped, with the same result
 * up to rounding.  For index mode n and product modes a < b, the sum over
 * the mode-b index k runs first, along each fibre (i_n, i_a) of the SpTTM
 * handle along mode b (Eq. 3): T(f, :) = sum_k X U_b(k, :).  Then Eq. 4 runs
 * over the fibres, one term U_a(i_a, :) (x) T(f, :) per fibre.  A nonzero
 * costs R FMAs plus R^2 per fibre, instead of R^2 (fewer wherever fibres
 * hold more than one nonzero).
 *
 * spttmc_plan_create
 *   Xttm      3-way handle built with op = FCOO_OP_TTM along mode b, where b
 *             is the highest mode other than `mode` (b = 2 for mode 0 or 1,
 *             b = 1 for mode 2).  Not copied: it must outlive the plan.
 *   mode      the SpTTMc index mode n, 0..2
 *   R         rank of both factors, 1..16 (R^2 <= FCOO_MAX_RANK)
 *   threadlen partition length of the fibre tensor's F-COO (as fcoo_build)
 *   plan      receives the plan.  It holds the fibre tensor (an F-COO of
 *             nfib nonzeros) and nfib x R FP32 fibre sums in device memory.
 *   Synchronous (it builds an F-COO).  Errors: FCOO_ERR_INVALID_ARG (wrong
 *   handle or mode), FCOO_ERR_UNSUPPORTED (R), FCOO_ERR_NOMEM, FCOO_ERR_CUDA.
 * spttmc_plan_run
 *   factors   host array of 3 device pointers to dims[k] x R FP32 row-major
 *             factors; factors[mode] is not read (may be NULL)
 *   dtype     FCOO_F32 (others: FCOO_ERR_UNSUPPORTED)
 *   out       device float32 dims[mode] x R^2, columns r_a * R + r_b as for
 *             spttmc; every element written
 *   Two kernels and a fix-up, asynchronous on `stream`; deterministic.
 *   Calls on one plan must not overlap (they share the fibre sums).
 * spttmc_plan_info: fibres of the plan and the device bytes it holds.
 * spttmc_plan_destroy: frees the plan (NULL is accepted). */
typedef struct fcoo_ttmc_plan fcoo_ttmc_plan_t;
int spttmc_plan_create(const fcoo_t *Xttm, int mode, int R, int threadlen, fcoo_ttmc_plan_t **plan,
                       fcoo_stream_t stream);
int spttmc_plan_run(const fcoo_ttmc_plan_t *plan, const void *const *factors, int dtype, float *out,
                    fcoo_stream_t stream);
int spttmc_plan_info(const fcoo_ttmc_plan_t *plan, int64_t *nfib, int64_t *device_bytes);
int spttmc_plan_destroy(fcoo_ttmc_plan_t *plan);

/* ---------------------------------------------------------------------- */
/* Tucker decomposition by HOOI around SpTTMc (Sec. II: HOOI's key          */
/* operation is TTMc, Eq. 4)                                                */
/* ---------------------------------------------------------------------- */

/* State of a rank-(R, ..., R) Tucker decomposition: N factors U_k (dims[k] x
 * R, FP32, device).  One iteration (tucker_hooi_iter) updates the modes in
 * order; mode n's update is
 *   Y_(n) = SpTTMc of mode n with the current other factors (dims[n] x W,
 *           W = R^(N-1)),
 *   U_n   = the R leading left singular vectors of Y_(n): eigenvectors q_r of
 *           S = Y^T Y (FP64 Gram of compensated FP32 partials; FP32 parallel
 *           Jacobi) mapped back as Y q_r / sqrt(d_r), each column signed so
 *           that its entry of largest magnitude (first row on ties) is
 *           positive.
 * After the last mode, |G|^2 = sum_r q_r^T S q_r (the core's squared norm)
 * and fit = 1 - sqrt(max(0, |X|^2 - |G|^2)) / |X|.  A direction whose
 * eigenvalue is below 1e-6 of the largest leaves a zero column and is
 * counted (nnull in tucker_state_stats).
 *
 * tucker_state_create
 *   nmodes 2..FCOO_MAX_MODES; dims host array; R 1..12 with R^(N-1) <= 128
 *   (FCOO_ERR_UNSUPPORTED above); init: N pointers (host or device) to
 *   dims[k] x R FP32 start factors (copied).  Synchronous.
 * tucker_hooi_iter
 *   Xn: N SpMTTKRP handles of one tensor, Xn[n] built for mode n.  About
 *   seven launches per mode, asynchronous on `stream`; deterministic.
 * tucker_state_stats: fit, |G|^2, iterations done, null directions met
 *   (synchronous; any pointer may be NULL).
 * tucker_state_copy_factor: U_n to host or device memory (synchronous).
 * tucker_state_destroy: frees the state (NULL is accepted). */
typedef struct tucker_state tucker_state_t;
int tucker_state_create(int nmodes, const uint32_t *dims, int R, const float *const *init, fcoo_stream_t stream,
                        tucker_state_t **out);
int tucker_hooi_iter(const fcoo_t *const *Xn, tucker_state_t *st, fcoo_stream_t stream);
int tucker_state_stats(const tucker_state_t *st, double *fit, double *core_sq, int *iters, int *nnull,
                       fcoo_stream_t stream);
int tucker_state_copy_factor(const tucker_state_t *st, int n, float *dst, fcoo_stream_t stream);
int tucker_state_destroy(tucker_state_t *st);

/* ---------------------------------------------------------------------- */
/* SpMTTKRP for callers that cannot allocate device memory                  */
/* ---------------------------------------------------------------------- */

/* The fixed scratch of spmttkrp_noalloc holds the carry slots of
 * FCOO_NOALLOC_MAX_CTAS CTAs for ranks up to FCOO_NOALLOC_MAX_RANK:
 * 2 * FCOO_NOALLOC_MAX_CTAS * FCOO_NOALLOC_MAX_RANK doubles plus
 * 2 * FCOO_NOALLOC_MAX_CTAS int64 = 2 MiB + 16 KiB.  A larger R is refused;
 * the CTA count is not a caller parameter: the launch uses at most
 * FCOO_NOALLOC_MAX_CTAS CTAs. */
#define FCOO_NOALLOC_MAX_RANK 128
#define FCOO_NOALLOC_MAX_CTAS 1024

/* An F-COO layout for SpMTTKRP held in memory the caller owns.  The arrays
 * are the ones fcoo_copy_layout returns (same meaning, same order), placed
 * by the caller in device memory:
 *   pidx[m]  product-mode indices of stream m (modes ascending, all but
 *            `mode`), val the values: each array 16-byte aligned and readable
 *            for round_up(nnz, 32) entries (entries past nnz are read, unused)
 *   bf       ceil(nnz/32) words of segment-start bits; sf the start-flag words
 *            for partitions of `threadlen` nonzeros
 *   segrow   nseg output rows, one per segment, strictly ascending, each
 *            below dims[mode]
 *   hcount   ceil(nnz/1024)+1 words: hcount[c] = number of set bits in
 *            bf[0 .. 32c-1] (segment starts before nonzero 1024c)
 * No pointer is retained after the call returns.  These buffers are trusted
 * as they are: the call checks pointers, alignment and nseg <= dims[mode], but
 * not the contents.  A layout that breaks the rules above (for example a
 * segrow that is not strictly ascending or holds a row >= dims[mode]) makes
 * the kernel read and write outside the buffers: behaviour is undefined. */
typedef struct {
    int nmodes, mode, threadlen;
    int64_t nnz, nseg;
    uint32_t dims[FCOO_MAX_MODES];
    const uint32_t *pidx[FCOO_MAX_MODES - 1];
    const float *val;
    const uint32_t *bf, *sf, *segrow, *hcount;
} fcoo_view_t;

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory while they run: code whose device
 * memory is reserved up front by a framework allocator or a fixed arena, and
 * real-time or safety-constrained code that forbids allocation after
 * start-up.  spmttkrp (above) allocates nothing per call either, but its
 * scratch lives in the handle that fcoo_build allocates; this variant takes
 * the layout as plain caller-owned buffers and keeps its scratch (the
 * per-CTA carry slots) in a fixed array inside the library.
 *
 * Computes exactly what spmttkrp computes (Eq. 6) for the layout in *view:
 *   out(i, :) = sum over nonzeros p with idx_mode(p) = i of
 *               val(p) * prod_{k != mode} F_k(idx_k(p), :)
 *   factors  host array of nmodes device pointers, dims[k] x R of dtype
 *            (factors[mode] not read); R in 1..FCOO_NOALLOC_MAX_RANK
 *   out      device float32 dims[mode] x R, 4-byte aligned, fully
 *            overwritten
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch (2 MiB + 16 KiB) is a file-scope __device__ array held by every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current) and caches it; make that first call before any stream
 * capture.  Every call uses the same array, so calls that overlap on the GPU
 * (other streams, other threads) race and give wrong results: serialise them.
 * Nothing in the array has to start at zero: each launch initialises the
 * slots it reads.  R above FCOO_NOALLOC_MAX_RANK returns FCOO_ERR_UNSUPPORTED
 * with a message; NULL or misaligned pointers and inconsistent sizes return
 * FCOO_ERR_INVALID_ARG, both before any device work.  Asynchronous on
 * `stream`. */
int spmttkrp_noalloc(const fcoo_view_t *view, const void *const *factors, int dtype, int R, float *out,
                     fcoo_stream_t stream);

/* Gather-only bound of SpMTTKRP on a 3-way tensor (Eq. 6; Sec. IV-D reads
 * the factor rows through the read-only cache).  A measurement aid, not part
 * of any result: it loads exactly the factor rows that spmttkrp on the same
 * handle loads, and nothing else -- per nonzero, in F-COO order along each
 * lane group's range, the row C(k,:) of the last product mode, and the row
 * B(j,:) of the first product mode where j changes, a segment starts or the
 * group's range starts -- with eight columns per lane as spmttkrp's R/8-lane
 * layout, and no products, reduction or output.  Its duration bounds from
 * below what the gathers alone cost SpMTTKRP on this tensor and these
 * factors.
 * Arguments:
 *   X            handle built with FCOO_OP_MTTKRP on a 3-way tensor
 *   factors      as spmttkrp (device rows, dtype FCOO_F32 or FCOO_BF16); the
 *                two product-mode factors must be 32-byte (F32) or 16-byte
 *                (BF16) aligned
 *   R            8, 16, 32, 64, 128 or 256
 *   rows_loaded  device pointer to one 8-byte counter, set to the number of
 *                rows loaded (C rows plus B rows)
 * Asynchronous on `stream`.  Errors (before any device work):
 * FCOO_ERR_INVALID_ARG (NULL or misaligned pointers, wrong op or dtype),
 * FCOO_ERR_UNSUPPORTED (not 3-way, another R, factor rows not aligned). */
int spmttkrp_gather_bound(const fcoo_t *X, const void *const *factors, int dtype, int R,
                          unsigned long long *rows_loaded, fcoo_stream_t stream);

/* ---------------------------------------------------------------------- */
/* CP-ALS (Algorithm 1; Sec. IV-D "Complete tensor-based algorithms")       */
/* ---------------------------------------------------------------------- */

/* Create the device state of a rank-R CP decomposition: factor matrices
 * stored as dtype (FCOO_F32 or FCOO_BF16), lambda, FP64 Gram matrices,
 * the last MTTKRP, iteration count and fit.
 *   init  host array of N pointers (host or device) to float32 dims[k] x R
 *         initial factors (rounded to dtype on copy).
 * Synchronous. */
int cp_state_create(int nmodes, const uint32_t *dims, int R, int dtype, const float *const *init,
                    fcoo_stream_t stream, cp_state_t **out);
int cp_state_destroy(cp_state_t *st);

/* One full sweep of Algorithm 1 over all modes n = 0..N-1:
 *   M   = SpMTTKRP_n(X, F)                       (Eq. 6, FP32 accumulation)
 *   V   = Hadamard product over k != n of F_k^T F_k  (Grams of the stored
 *         factors from compensated FP32 partial sums added in FP64)
 *   F_n = M V^dagger   (FP64 Cholesky; if a pivot is <= 1e-12 * max diag(V),
 *                       the eigen-decomposition pseudo-inverse that drops
 *                       eigenvalues <= 1e-12 * max |eig|; the product with M in
 *                       compensated FP32 against the inverse split in two
 *                       FP32 parts)
 *   lambda = column 2-norms of F_n; F_n columns divided by them (a zero
 *            column keeps lambda 0 and is left as it is)
 * then the fit 1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2<X,Xhat>)) / |X|.
 *   Xn  host array of N handles, Xn[n] built with op = FCOO_OP_MTTKRP, mode n,
 *       all from the same tensor.
 * Asynchronous on `stream`; read results with cp_state_stats. */
int cp_als_iter(const fcoo_t *const *Xn, cp_state_t *st, fcoo_stream_t stream);

/* Synchronous read of lambda (host, R doubles, may be NULL), the last fit,
 * the number of completed sweeps and the number of pseudo-inverse solves. */
int cp_state_stats(const cp_state_t *st, double *lambda, double *fit, int *iters, int *npinv, fcoo_stream_t stream);

/* Fibre reuse for 3-way CP-ALS.  SpMTTKRP of modes 0 and 1 both contract
 * the tensor with the mode-2 factor C, which does not change between their
 * updates.  With this on, mode 0 first forms the mode-2 fibre sums
 *   T(f, :) = sum_k X(i,j,k) C(k, :)      for each fibre f = (i, j)   (Eq. 3)
 * and modes 0 and 1 each run Eq. 6 over the fibres, with factors (B, T) and
 * (A, T), instead of over the nonzeros.  The result is the same up to
 * rounding, and it pays where fibres hold several nonzeros.
 *   Xttm       the SpTTM handle along mode 2 of the same tensor (op =
 *              FCOO_OP_TTM, mode 2).  Not copied: it must outlive its use.
 *              NULL turns the reuse off and frees its buffers.
 *   threadlen  partition length of the fibre tensor's F-COO handles.
 * The state holds two F-COO handles of nfib nonzeros, nfib x R FP32 fibre
 * sums, and an FP32 copy of one factor (for BF16 storage).  Synchronous.
 * Cost: the fibre sums are written once and read twice per sweep (nfib x R
 * x 4 bytes each time).  On a 76M-nonzero Zipf tensor with 13M fibres at
 * R = 64 that made FP32 sweeps 4 % faster and BF16 sweeps slower, so it is
 * off unless asked for.
 * Errors: FCOO_ERR_INVALID_ARG (not 3-way, wrong handle), FCOO_ERR_NOMEM. */
int cp_state_use_fibres(cp_state_t *st, const fcoo_t *Xttm, int threadlen, fcoo_stream_t stream);

/* Change the storage type of the factors (FCOO_F32 <-> FCOO_BF16) in place:
 * BF16 -> FP32 is exact; FP32 -> BF16 rounds to nearest even and recomputes
 * the Grams.  Later cp_als_iter sweeps gather the factors in the new type.
 * This serves a mixed-precision schedule (BF16 sweeps while the fit moves,
 * FP32 sweeps to finish); the paper's Algorithm 1 has one precision
 * throughout.  Asynchronous on `stream`. */
int cp_state_set_dtype(cp_state_t *st, int dtype, fcoo_stream_t stream);

/* Copy factor k as float32 (dims[k] x R) to host or device memory. Synchronous. */
int cp_state_copy_factor(const cp_state_t *st, int k, float *dst, fcoo_stream_t stream);

/* Checkpoint: size of the blob, serialise to host memory, restore from it
 * (same nmodes, dims, R and dtype).  Synchronous. */
int64_t cp_state_blob_size(const cp_state_t *st);
int cp_state_save(const cp_state_t *st, void *blob, int64_t size, fcoo_stream_t stream);
int cp_state_load(cp_state_t *st, const void *blob, int64_t size, fcoo_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Differentiation: loss and adjoints built from the Eq. 6 one-shot product */
/* ---------------------------------------------------------------------- */

/* kind = 0, sparse CP fit over the observed entries:
 *   e(p) = sum_r prod_k F_k(idx_k(p), r) - val(p),  loss = 1/2 sum_p e(p)^2
 *   dfactors[n](i, :) = sum_{p: idx_n(p) = i} e(p) prod_{k != n} F_k(idx_k(p), :)
 *   dvals(p) = -e(p), in the caller's original COO order
 *   Xn: N handles (op MTTKRP, mode n each); `mode` and gradM are ignored;
 *   loss: device double (may be NULL); dfactors[n] device float32 dims[n] x R
 *   (entries may be NULL to skip that mode); dvals device float32 nnz (may be NULL).
 * kind = 1, adjoint of M = SpMTTKRP_mode(X, F) for gradM = dL/dM (device
 * float32 dims[mode] x R):
 *   dfactors[k](j, :) = sum_{p: idx_k(p) = j} val(p) gradM(idx_mode(p), :)
 *                       * prod_{m != mode, k} F_m(idx_m(p), :)     (k != mode)
 *   dvals(p) = sum_r gradM(idx_mode(p), r) prod_{k != mode} F_k(idx_k(p), r)
 *   Xn: N handles as above (Xn[k] is used for dfactors[k]); dvals uses Xn[mode].
 * All outputs are fully overwritten.  Asynchronous on `stream`.
 * Kind 0 with two or more gradients computes e once, on the first requested
 * mode, and reuses it for the others.  For that it keeps, allocated on first
 * use and freed by fcoo_destroy, 12 bytes per padded nonzero with the handle
 * of the first requested mode and a 4-byte position map per padded nonzero
 * with each other handle; calls that share handles must not overlap. */
int spmttkrp_backward(const fcoo_t *const *Xn, const void *const *factors, int dtype, int R, const float *gradM,
                      int kind, int mode, float *const *dfactors, float *dvals, double *loss, fcoo_stream_t stream);

/* Forward value of the kind = 0 loss only (device double *loss). */
int sparse_cp_loss(const fcoo_t *X, const void *const *factors, int dtype, int R, double *loss,
                   fcoo_stream_t stream);

#ifdef __cplusplus
}
#endif
#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#endif /* FCOO_H */
