// tucker.cu -- Tucker decomposition by higher-order orthogonal iteration
// (HOOI), whose TTM chain is SpTTMc (Sec. II, Eq. 4).
//
// One mode update, for factors U_k (I_k x R, orthonormal columns):
//   Y   = SpTTMc_n(X; U_k, k != n)            I_n x W, W = R^(N-1)   (k_stream kind 2)
//   S   = Y^T Y                               W x W, Dot2 partials summed in FP64
//   S   = Q diag(d) Q^T                        parallel cyclic Jacobi: FP32 sweeps
//                                              (from the mode's last eigenvectors
//                                              once there are some), an FP64
//                                              re-orthonormalisation, then FP64
//                                              sweeps on Q^T S Q against the
//                                              2R + 2 leading directions
//   U_n = Y q_r / sqrt(d_r) for the R largest d_r (FP64 sums): the R leading
//         left singular vectors of Y_(n); each column signed so that its
//         largest entry is positive
// After the last mode the core is G = U_n^T Y_(n), |G|^2 = sum_r d_r, and
// fit = 1 - sqrt(max(0, |X|^2 - |G|^2)) / |X|.
// The FP64 stage matters on skewed tensors: there the R leading eigenvalues
// of S can lie 1e-4 below the largest, under the FP32 stage's resolution.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

struct tucker_state {
    int nmodes, R, W;
    uint32_t dims[FCOO_MAX_MODES];
    int64_t max_dim;
    float *U[FCOO_MAX_MODES];  // dims[k] x R
    float *Y;                  // max_dim x W
    double *S;                 // W x W
    double *Qd;                // W x W eigenvectors (columns)
    double *T1, *Aq;           // W x W: S Q1 and Q1^T S Q1
    double *Qprev[FCOO_MAX_MODES];  // W x W: each mode's last eigenvectors (warm start)
    bool have_q[FCOO_MAX_MODES];
    double *part;              // Gram partials / |X|^2 partials
    float *cand;               // per-block sign candidates: [nb][R][3] (|u|, index, u)
    int *sel;                  // R selected eigenpairs
    double *inv_sig;           // R: 1 / sqrt(d) (0 for a null direction)
    double *dsel;              // R selected eigenvalues
    float *sgn;                // R column signs
    double *scal;              // [0] |X|^2, [1] fit, [2] |G|^2
    int *flags;                // [0] null directions met, [1] FP32 Jacobi sweeps of the last solve
    int iters;
    bool have_norm;
    void *base;
};

namespace fcx {
namespace {

constexpr int kMaxW = 128;       // W = R^(N-1) limit (shared-memory Jacobi)
constexpr int kEigThreads = 512;
constexpr int kProjWarps = 8;    // rows in flight per projection CTA

// Parallel cyclic Jacobi sweeps on the symmetric W x W matrix A (shared
// memory), accumulating the rotations into Q (columns are eigenvectors).
// Each step rotates W/2 disjoint pairs at once (round-robin ordering: one
// index fixed, the others on a circle), so the rotations commute and
// A <- J^T A J is two passes over the pairs.  Rotation angles are taken in
// TA.  Stops when the off-diagonal entries are at the rounding level of TA
// (|a_pq| ~ 8 eps |A|_F), or, once near it, when a sweep gains less than 4x;
// at most max_sweeps.  With `act` (shared flags, one per index), only pairs
// with an active index rotate and only their entries count as off-diagonal:
// the leading eigenvectors are refined without touching the rest of the
// spectrum.  Returns the sweeps done.
template <typename TA, typename TQ>
__device__ int jacobi_sweeps(TA *A, TQ *Q, int W, int max_sweeps, double eps, const int *act) {
    __shared__ TA s_c[kMaxW / 2 + 1], s_s[kMaxW / 2 + 1];
    __shared__ int s_p[kMaxW / 2 + 1], s_q[kMaxW / 2 + 1];
    __shared__ double s_red[kEigThreads / 32][2];
    __shared__ int s_done, s_np, s_wc[2];
    __shared__ double s_prev;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_prev = -1.0;
    const int m = W + (W & 1), half = m / 2;
    __syncthreads();
    int sweeps = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < W * W; e += nt) {
            const double a = A[e];
            const int i = e / W, j = e % W;
            tot += a * a;
            if (i != j && (!act || act[i] || act[j])) off += a * a;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) {
            s_red[tid >> 5][0] = off;
            s_red[tid >> 5][1] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            double o2 = 0.0, t2 = 0.0;
            for (int w = 0; w < nt / 32; ++w) {
                o2 += s_red[w][0];
                t2 += s_red[w][1];
            }
            const double floor2 = (double)W * W * 64.0 * eps * eps * t2;
            const bool near = o2 <= 1e6 * floor2;
            s_done = (o2 <= floor2 || (near && s_prev >= 0.0 && o2 > 0.25 * s_prev)) ? 1 : 0;
            s_prev = o2;
        }
        __syncthreads();
        if (s_done) break;
        ++sweeps;
        for (int step = 0; step < m - 1; ++step) {
            // threads k < half (two warps at most) each take pair k of this step
            bool rot = false;
            int p = -1, q = -1;
            TA c = 1, sn = 0;
            if (tid < half) {
                const int k = tid;
                int a, b;
                if (k == 0) {
                    a = m - 1;
                    b = step;
                } else {
                    a = (step + k) % (m - 1);
                    b = (step - k + m - 1) % (m - 1);
                }
                p = min(a, b);
                q = max(a, b);
                if (q < W && (!act || act[p] || act[q])) {
                    const TA apq = A[p * W + q];
                    if (apq != (TA)0) {
                        // t = tan of the rotation angle (the smaller root), in
                        // FP32: a rotation then leaves ~1e-7 of a_pq, which
                        // FP64 sweeps started at FP32 level absorb in two
                        const float theta = (float)(A[q * W + q] - A[p * W + p]) / (float)(2 * apq);
                        const float at = fabsf(theta);
                        const float tf = at > 1e15f ? 0.5f / theta
                                                    : (theta >= 0.f ? 1.f : -1.f) / (at + sqrtf(theta * theta + 1.f));
                        const TA t = (TA)tf, u = t * t + 1;
                        // c = 1/sqrt(u) exactly enough that c^2 + s^2 = 1 in TA:
                        // the FP32 estimate plus one Newton step
                        TA cc = (TA)rsqrtf((float)u);
                        if (sizeof(TA) > 4) cc = cc * ((TA)1.5 - (TA)0.5 * u * cc * cc);
                        c = cc;
                        sn = t * cc;
                        rot = true;
                    }
                }
            }
            if (!act) {
                // every pair in its slot; the update passes skip the idle ones
                if (tid < half) {
                    s_c[tid] = c;
                    s_s[tid] = sn;
                    s_p[tid] = rot ? p : -1;
                    s_q[tid] = q;
                }
            } else if (tid < 64) {
                // pack the rotating pairs (warp ballots; order kept)
                const unsigned bal = __ballot_sync(0xffffffffu, rot);
                if ((tid & 31) == 0) s_wc[tid >> 5] = __popc(bal);
                __syncwarp();
                asm volatile("bar.sync 1, 64;" ::: "memory");  // the two warps of the pair threads
                const int base = (tid >> 5) ? s_wc[0] : 0;
                const int pos = base + __popc(bal & ((1u << (tid & 31)) - 1u));
                if (rot) {
                    s_c[pos] = c;
                    s_s[pos] = sn;
                    s_p[pos] = p;
                    s_q[pos] = q;
                }
                if (tid == 0) s_np = s_wc[0] + s_wc[1];
            }
            __syncthreads();
            const int np = act ? s_np : half;
            // A <- A J (columns p, q of every row)
            for (int e = tid; e < W * np; e += nt) {
                const int r = e / np, k = e % np;
                const int p = s_p[k], q = s_q[k];
                if (p < 0 || s_s[k] == (TA)0) continue;
                const TA c = s_c[k], sn = s_s[k];
                const TA ap = A[r * W + p], aq = A[r * W + q];
                A[r * W + p] = c * ap - sn * aq;
                A[r * W + q] = sn * ap + c * aq;
            }
            __syncthreads();
            // A <- J^T A (rows p, q), Q <- Q J
            for (int e = tid; e < W * np; e += nt) {
                const int col = e / np, k = e % np;
                const int p = s_p[k], q = s_q[k];
                if (p < 0 || s_s[k] == (TA)0) continue;
                const TA c = s_c[k], sn = s_s[k];
                const TA ap = A[p * W + col], aq = A[q * W + col];
                A[p * W + col] = c * ap - sn * aq;
                A[q * W + col] = sn * ap + c * aq;
                const TQ cq = (TQ)s_c[k], sq = (TQ)s_s[k];
                const TQ qp = Q[col * W + p], qq = Q[col * W + q];
                Q[col * W + p] = cq * qp - sq * qq;
                Q[col * W + q] = sq * qp + cq * qq;
            }
            __syncthreads();
        }
    }
    return sweeps;
}

// Stage 1: FP32 Jacobi on S (or on Qp^T S Qp, warm start) from Q = I (A and
// Q in shared memory); the eigenvectors go to Qd in FP64.
__global__ void __launch_bounds__(kEigThreads) k_eig_f32(const double *S, int W, double *Qd, int *flags) {
    extern __shared__ __align__(16) float sm[];
    float *A = sm, *Q = sm + W * W;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        A[e] = (float)S[e];
        Q[e] = (e / W == e % W) ? 1.f : 0.f;
    }
    __syncthreads();
    const int sweeps = jacobi_sweeps<float, float>(A, Q, W, 40, 6e-8, nullptr);
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) Qd[e] = Q[e];
    if (threadIdx.x == 0) flags[1] = sweeps;
}

// W x W FP64 products, one thread per entry of C, spread over many CTAs
// (FP64 is slow per SM).  op 0: C = A B;  op 1: C = A^T B;  op 2: C =
// A (1.5 I - 0.5 B), with B = A^T A: one Newton-Schulz (Lowdin) step that
// makes the nearly orthonormal columns of A orthonormal to second order.
__global__ void k_gemm64(const double *A, const double *B, double *C, int W, int op) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= W * W) return;
    const int i = e / W, j = e % W;
    auto a = [&](int k) { return op == 1 ? A[k * W + i] : A[i * W + k]; };
    auto b = [&](int k) { return op == 2 ? (k == j ? 1.5 : 0.0) - 0.5 * B[k * W + j] : B[k * W + j]; };
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < W; k += 2) {
        s0 = fma(a(k), b(k), s0);
        s1 = fma(a(k + 1), b(k + 1), s1);
    }
    if (k < W) s0 = fma(a(k), b(k), s0);
    C[e] = s0 + s1;
}

// Stage 2: FP64 Jacobi on Aq = Q1^T S Q1 (nearly diagonal after stage 1; Q1
// re-orthonormalised in FP64 first, so that this is a similarity to FP64
// rounding), accumulating into Qd = Q1 (global memory); then the R largest eigenvalues
// (ties: lower index) and their 1 / sqrt(d).  A direction whose eigenvalue
// is below 1e-12 of the largest counts as null (S is accurate to ~1e-13).
__global__ void __launch_bounds__(kEigThreads) k_eig_refine(const double *Aq, int W, int R, double *Qd, int *sel,
                                                            double *dsel, double *inv_sig, int *flags) {
    extern __shared__ __align__(16) double smd[];
    double *A = smd;
    __shared__ int act[kMaxW];
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) A[e] = Aq[e];
    __syncthreads();
    // active set: the 2R + 2 largest diagonal entries (the FP32 stage has
    // ordered the spectrum to ~1e-7 of its largest value)
    if (threadIdx.x == 0) {
        const int K = min(W, 2 * R + 2);
        for (int c = 0; c < W; ++c) act[c] = 0;
        for (int r = 0; r < K; ++r) {
            int best = -1;
            for (int c = 0; c < W; ++c)
                if (!act[c] && (best < 0 || A[c * W + c] > A[best * W + best])) best = c;
            act[best] = 1;
        }
    }
    __syncthreads();
    // from the FP32 stage's off-diagonal level (~1e-7 of the largest entry)
    // each sweep against the active indices cuts it by ~1e-7 (FP32 tangents):
    // two sweeps reach FP64 rounding, three at most
    jacobi_sweeps<double, double>(A, Qd, W, 3, 1.1e-16, act);
    __syncthreads();
    if (threadIdx.x == 0) {
        double dmax = 0.0;
        for (int c = 0; c < W; ++c) dmax = fmax(dmax, A[c * W + c]);
        unsigned long long taken[2] = {0ull, 0ull};
        for (int r = 0; r < R; ++r) {
            int best = -1;
            for (int c = 0; c < W; ++c) {
                if ((taken[c >> 6] >> (c & 63)) & 1ull) continue;
                if (best < 0 || A[c * W + c] > A[best * W + best]) best = c;
            }
            taken[best >> 6] |= 1ull << (best & 63);
            sel[r] = best;
            const double d = A[best * W + best];
            dsel[r] = d;
            if (d > 1e-12 * dmax && d > 0.0) {
                inv_sig[r] = 1.0 / sqrt(d);
            } else {
                inv_sig[r] = 0.0;  // Y has rank < R: this column stays zero
                atomicAdd(&flags[0], 1);
            }
        }
    }
}

// U(i, r) = (sum_c Y(i, c) Q(c, sel_r)) * inv_sig_r in FP64: one warp per
// row, the lanes splitting c.  Each CTA also leaves, per column, its entry
// of largest magnitude (first row on ties) for the sign convention.
__global__ void __launch_bounds__(kProjWarps * 32) k_project(const float *Y, int64_t I, int W, const double *Qd,
                                                             const int *sel, const double *inv_sig, int R,
                                                             float *U, float *cand) {
    __shared__ double Qs[kMaxW * 12];
    __shared__ float s_best[kProjWarps][12][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < W * R; e += blockDim.x) Qs[e] = Qd[(e / R) * W + sel[e % R]];
    __syncthreads();
    float bmag = -1.f, bidx = 0.f, bval = 0.f;  // lane r < R tracks column r
    for (int64_t i = (int64_t)blockIdx.x * kProjWarps + warp; i < I; i += (int64_t)gridDim.x * kProjWarps) {
        double acc[12];
#pragma unroll
        for (int r = 0; r < 12; ++r) acc[r] = 0.0;
        for (int c = lane; c < W; c += 32) {
            const double y = Y[i * W + c];
#pragma unroll
            for (int r = 0; r < 12; ++r)
                if (r < R) acc[r] = fma(y, Qs[c * R + r], acc[r]);
        }
        float mine = 0.f;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            if (r < R) {
                double v = acc[r];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == r) mine = (float)(v * inv_sig[r]);
            }
        }
        if (lane < R) {
            U[i * R + lane] = mine;
            const float mag = fabsf(mine);
            if (mag > bmag) {  // rows of one warp ascend, so the first wins ties
                bmag = mag;
                bidx = (float)i;
                bval = mine;
            }
        }
    }
    if (lane < R) {
        s_best[warp][lane][0] = bmag;
        s_best[warp][lane][1] = bidx;
        s_best[warp][lane][2] = bval;
    }
    __syncthreads();
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        float m = -1.f, ix = 0.f, v = 0.f;
        for (int w = 0; w < kProjWarps; ++w) {
            const float mm = s_best[w][r][0], ii = s_best[w][r][1];
            if (mm > m || (mm == m && mm >= 0.f && ii < ix)) {
                m = mm;
                ix = ii;
                v = s_best[w][r][2];
            }
        }
        cand[((int64_t)blockIdx.x * R + r) * 3 + 0] = m;
        cand[((int64_t)blockIdx.x * R + r) * 3 + 1] = ix;
        cand[((int64_t)blockIdx.x * R + r) * 3 + 2] = v;
    }
}

// sign_r = sign of column r's entry of largest magnitude (first row on
// ties); one CTA per column, the per-CTA candidates reduced in parallel.
__global__ void __launch_bounds__(256) k_sign(const float *cand, int nb, int R, float *sgn) {
    __shared__ float s_m[256], s_i[256], s_v[256];
    const int r = blockIdx.x;
    float m = -1.f, ix = 0.f, v = 0.f;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const float *cb = cand + ((int64_t)b * R + r) * 3;
        if (cb[0] > m || (cb[0] == m && cb[0] >= 0.f && cb[1] < ix)) {
            m = cb[0];
            ix = cb[1];
            v = cb[2];
        }
    }
    s_m[threadIdx.x] = m;
    s_i[threadIdx.x] = ix;
    s_v[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const float m2 = s_m[threadIdx.x + o], i2 = s_i[threadIdx.x + o];
            const float m1 = s_m[threadIdx.x], i1 = s_i[threadIdx.x];
            if (m2 > m1 || (m2 == m1 && m2 >= 0.f && i2 < i1)) {
                s_m[threadIdx.x] = m2;
                s_i[threadIdx.x] = i2;
                s_v[threadIdx.x] = s_v[threadIdx.x + o];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sgn[r] = s_v[0] < 0.f ? -1.f : 1.f;
}

__global__ void k_flip(float *U, int64_t n, int R, const float *sgn) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        U[e] *= sgn[e % R];
}

// |G|^2 = sum_r d_r (the selected eigenvalues of S, FP64) and the fit.
__global__ void k_core_fit(const double *dsel, int R, double *scal) {
    if (threadIdx.x != 0) return;
    double g2 = 0.0;
    for (int r = 0; r < R; ++r) g2 += dsel[r];
    const double x2 = scal[0];
    scal[2] = g2;
    scal[1] = x2 > 0.0 ? 1.0 - sqrt(fmax(0.0, x2 - g2)) / sqrt(x2) : 0.0;
}

int proj_blocks(int64_t I) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, kProjWarps), 2048)); }

}  // namespace
}  // namespace fcx

using namespace fcx;

extern "C" int tucker_state_create(int nmodes, const uint32_t *dims, int R, const float *const *init,
                                   fcoo_stream_t stream, tucker_state_t **out) {
    clear_error();
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_create: out is NULL");
    *out = nullptr;
    if (nmodes < 2 || nmodes > FCOO_MAX_MODES || !dims || !init)
        return fail(FCOO_ERR_INVALID_ARG, "tucker_state_create: bad nmodes/dims/init");
    if (R < 1 || R > 12) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_create: R=%d outside 1..12", R);
    int64_t W = 1;
    for (int k = 0; k < nmodes - 1; ++k) {
        W *= R;
        if (W > kMaxW)
            return fail(FCOO_ERR_UNSUPPORTED, "tucker_state_create: R^%d above %d", nmodes - 1, kMaxW);
    }
    for (int k = 0; k < nmodes; ++k) {
        if (dims[k] == 0) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_create: dims[%d] is 0", k);
        if (!init[k]) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_create: init[%d] is NULL", k);
    }
    tucker_state_t *st = (tucker_state_t *)calloc(1, sizeof(tucker_state_t));
    if (!st) return fail(FCOO_ERR_NOMEM, "tucker_state_create: host allocation failed");
    st->nmodes = nmodes;
    st->R = R;
    st->W = (int)W;
    for (int k = 0; k < nmodes; ++k) {
        st->dims[k] = dims[k];
        st->max_dim = std::max<int64_t>(st->max_dim, dims[k]);
    }
    const int64_t nbg = ceil_div(st->max_dim, 128);
    const int64_t nbp = proj_blocks(st->max_dim);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += round_up((int64_t)b, 256);
        return o;
    };
    size_t oU[FCOO_MAX_MODES];
    for (int k = 0; k < nmodes; ++k) oU[k] = take((size_t)dims[k] * R * 4);
    const size_t oY = take((size_t)st->max_dim * W * 4), oS = take((size_t)W * W * 8), oQ = take((size_t)W * W * 8),
                 oT1 = take((size_t)W * W * 8), oAq = take((size_t)W * W * 8), oDs = take((size_t)R * 8),
                 oQp = take((size_t)nmodes * W * W * 8),
                 oP = take((size_t)std::max<int64_t>(nbg * W * W, 1024) * 8), oC = take((size_t)nbp * R * 3 * 4),
                 oSel = take((size_t)R * 4), oIs = take((size_t)R * 8), oSg = take((size_t)R * 4),
                 oSc = take(4 * 8), oF = take(2 * 4);
    cudaError_t e = dev_alloc(&st->base, off);
    if (e != cudaSuccess) {
        free(st);
        return cuda_fail(e, "tucker_state_create");
    }
    char *b = static_cast<char *>(st->base);
    for (int k = 0; k < nmodes; ++k) st->U[k] = reinterpret_cast<float *>(b + oU[k]);
    st->Y = reinterpret_cast<float *>(b + oY);
    st->S = reinterpret_cast<double *>(b + oS);
    st->Qd = reinterpret_cast<double *>(b + oQ);
    st->T1 = reinterpret_cast<double *>(b + oT1);
    st->Aq = reinterpret_cast<double *>(b + oAq);
    st->dsel = reinterpret_cast<double *>(b + oDs);
    for (int k = 0; k < nmodes; ++k) st->Qprev[k] = reinterpret_cast<double *>(b + oQp) + (size_t)k * W * W;
    st->part = reinterpret_cast<double *>(b + oP);
    st->cand = reinterpret_cast<float *>(b + oC);
    st->sel = reinterpret_cast<int *>(b + oSel);
    st->inv_sig = reinterpret_cast<double *>(b + oIs);
    st->sgn = reinterpret_cast<float *>(b + oSg);
    st->scal = reinterpret_cast<double *>(b + oSc);
    st->flags = reinterpret_cast<int *>(b + oF);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = FCOO_OK;
    for (int k = 0; k < nmodes && rc == FCOO_OK; ++k) {
        e = cudaMemcpyAsync(st->U[k], init[k], (size_t)dims[k] * R * 4, cudaMemcpyDefault, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tucker_state_create: init copy");
    }
    if (rc == FCOO_OK) {
        e = cudaMemsetAsync(st->scal, 0, 4 * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(st->flags, 0, 2 * 4, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tucker_state_create");
    }
    if (rc != FCOO_OK) {
        dev_free(st->base);
        free(st);
        return rc;
    }
    *out = st;
    return FCOO_OK;
}

extern "C" int tucker_state_destroy(tucker_state_t *st) {
    clear_error();
    if (!st) return FCOO_OK;
    cudaDeviceSynchronize();
    dev_free(st->base);
    free(st);
    return FCOO_OK;
}

extern "C" int tucker_hooi_iter(const fcoo_t *const *Xn, tucker_state_t *st, fcoo_stream_t stream) {
    clear_error();
    if (!Xn || !st) return fail(FCOO_ERR_INVALID_ARG, "tucker_hooi_iter: NULL argument");
    for (int n = 0; n < st->nmodes; ++n) {
        const fcoo_t *X = Xn[n];
        if (!X) return fail(FCOO_ERR_INVALID_ARG, "tucker_hooi_iter: Xn[%d] is NULL", n);
        if (X->op != FCOO_OP_MTTKRP || X->mode != n || X->nmodes != st->nmodes)
            return fail(FCOO_ERR_INVALID_ARG, "tucker_hooi_iter: Xn[%d] is not an SpMTTKRP handle for mode %d", n, n);
        for (int k = 0; k < st->nmodes; ++k)
            if (X->dims[k] != st->dims[k]) return fail(FCOO_ERR_INVALID_ARG, "tucker_hooi_iter: Xn[%d] dims differ", n);
        if (X->nnz != Xn[0]->nnz) return fail(FCOO_ERR_INVALID_ARG, "tucker_hooi_iter: handles hold different tensors");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int R = st->R, W = st->W;
    int rc;
    if (!st->have_norm) {
        rc = sumsq_fp64(Xn[0]->val, Xn[0]->nnz, st->part, st->scal, s);
        if (rc) return rc;
        st->have_norm = true;
    }
    const size_t eig_smem = (size_t)2 * W * W * 4, ref_smem = (size_t)W * W * 8;
    FCOO_CUDA(cudaFuncSetAttribute(k_eig_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eig_smem));
    FCOO_CUDA(cudaFuncSetAttribute(k_eig_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ref_smem));
    const unsigned gg = (unsigned)ceil_div(W * W, 128);
    for (int n = 0; n < st->nmodes; ++n) {
        const int64_t I = st->dims[n];
        const void *fac[FCOO_MAX_MODES];
        for (int k = 0; k < st->nmodes; ++k) fac[k] = st->U[k];
        rc = spttmc(Xn[n], fac, FCOO_F32, R, st->Y, stream);
        if (rc) return rc;
        rc = gram_f32_fp64(st->Y, I, W, st->part, st->S, s);
        if (rc) return rc;
        // eigenvectors of S: FP32 Jacobi (on Qp^T S Qp from the mode's last
        // eigenvectors Qp once there are some: nearly diagonal after the first
        // iteration, so few sweeps); Q1 re-orthonormalised in FP64 (Q1 <- Q1
        // (1.5 I - 0.5 Q1^T Q1)); FP64 sweeps on Q1^T S Q1
        if (st->have_q[n]) {
            k_gemm64<<<gg, 128, 0, s>>>(st->S, st->Qprev[n], st->T1, W, 0);
            k_gemm64<<<gg, 128, 0, s>>>(st->Qprev[n], st->T1, st->Aq, W, 1);
            k_eig_f32<<<1, kEigThreads, eig_smem, s>>>(st->Aq, W, st->Qd, st->flags);
            k_gemm64<<<gg, 128, 0, s>>>(st->Qprev[n], st->Qd, st->T1, W, 0);
            std::swap(st->Qd, st->T1);
        } else {
            k_eig_f32<<<1, kEigThreads, eig_smem, s>>>(st->S, W, st->Qd, st->flags);
        }
        k_gemm64<<<gg, 128, 0, s>>>(st->Qd, st->Qd, st->Aq, W, 1);
        k_gemm64<<<gg, 128, 0, s>>>(st->Qd, st->Aq, st->T1, W, 2);
        std::swap(st->Qd, st->T1);
        k_gemm64<<<gg, 128, 0, s>>>(st->S, st->Qd, st->T1, W, 0);
        k_gemm64<<<gg, 128, 0, s>>>(st->Qd, st->T1, st->Aq, W, 1);
        k_eig_refine<<<1, kEigThreads, ref_smem, s>>>(st->Aq, W, R, st->Qd, st->sel, st->dsel, st->inv_sig,
                                                       st->flags);
        FCOO_CUDA(cudaGetLastError());
        FCOO_CUDA(cudaMemcpyAsync(st->Qprev[n], st->Qd, (size_t)W * W * 8, cudaMemcpyDeviceToDevice, s));
        st->have_q[n] = true;
        const int nb = proj_blocks(I);
        k_project<<<nb, kProjWarps * 32, 0, s>>>(st->Y, I, W, st->Qd, st->sel, st->inv_sig, R, st->U[n], st->cand);
        FCOO_CUDA(cudaGetLastError());
        k_sign<<<R, 256, 0, s>>>(st->cand, nb, R, st->sgn);
        const int64_t ne = I * R;
        k_flip<<<(unsigned)std::min<int64_t>(ceil_div(ne, 256), 4096), 256, 0, s>>>(st->U[n], ne, R, st->sgn);
        FCOO_CUDA(cudaGetLastError());
        if (n == st->nmodes - 1) {
            k_core_fit<<<1, 32, 0, s>>>(st->dsel, R, st->scal);
            FCOO_CUDA(cudaGetLastError());
        }
    }
    st->iters++;
    return FCOO_OK;
}

extern "C" int tucker_state_stats(const tucker_state_t *st, double *fit, double *core_sq, int *iters, int *nnull,
                                  fcoo_stream_t stream) {
    clear_error();
    if (!st) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_stats: NULL state");
    cudaStream_t s = (cudaStream_t)stream;
    double scal[3];
    int flags[2];
    FCOO_CUDA(cudaMemcpyAsync(scal, st->scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
    FCOO_CUDA(cudaMemcpyAsync(flags, st->flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    if (fit) *fit = scal[1];
    if (core_sq) *core_sq = scal[2];
    if (iters) *iters = st->iters;
    if (nnull) *nnull = flags[0];
    return FCOO_OK;
}

extern "C" int tucker_state_copy_factor(const tucker_state_t *st, int n, float *dst, fcoo_stream_t stream) {
    clear_error();
    if (!st || !dst) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_copy_factor: NULL argument");
    if (n < 0 || n >= st->nmodes) return fail(FCOO_ERR_INVALID_ARG, "tucker_state_copy_factor: mode %d", n);
    cudaStream_t s = (cudaStream_t)stream;
    FCOO_CUDA(cudaMemcpyAsync(dst, st->U[n], (size_t)st->dims[n] * st->R * 4, cudaMemcpyDefault, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    return FCOO_OK;
}
