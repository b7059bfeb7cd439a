// cp_als.cu -- CP-ALS (Algorithm 1) on the device, N-way, one sweep per call.
//
// Per mode n (all kernels on the caller's stream, no host round trip):
//   M   = SpMTTKRP_n(X, F)                         k_stream (spmttkrp.cu)
//   V   = Hadamard_{k != n} G_k, V^-1 (FP64)         k_solve: Cholesky, or the
//                                                   eigen pseudo-inverse (cyclic
//                                                   Jacobi) when a pivot is tiny
//   Fu  = M * V^-1 (FP32), column sums of squares    k_apply
//   lambda = column 2-norms (FP64)                   k_lambda
//   F_n = Fu / lambda, stored as FP32 or BF16         k_normalize (+ <M, F_n> for the fit)
//   G_n = F_n^T F_n of the stored values (FP64)      k_gram_part + k_gram_reduce
// after the last mode: fit from the Grams, lambda and <M_last, F_last>   k_fit
//
// FP64 is used only for R x R work (Hadamard of Grams, factorisation,
// inverse, lambda, fit) and for the cross-block sums of the Gram / norm
// partials; the I x R work is FP32.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fibre.cuh"

struct cp_state {
    int nmodes, R, dtype;
    uint32_t dims[FCOO_MAX_MODES];
    int64_t max_dim;
    void *F[FCOO_MAX_MODES];        // factors, dims[k] x R, dtype
    double *gram[FCOO_MAX_MODES];   // R x R FP64 Grams of the stored factors
    double *lambda;                 // R
    float *M;                       // max_dim x R: MTTKRP of the current mode
    float *Fu;                      // max_dim x R: unnormalised update
    double *V, *Q, *W;              // R x R FP64 work: normal matrix, eigenvectors, inverse
    float *Wf;                      // R x R FP32 copy of the inverse for the apply
    double *part;                   // block partials
    double *scal;                   // [0] |X|^2, [1] fit, [2] <X, Xhat>, [3] |Xhat|^2
    int *flags;                     // [0] pseudo-inverse solves, [1] non-finite seen
    int iters;
    bool have_norm;
    // the R x R solve of mode n runs on `side` while SpMTTKRP of mode n runs
    // on the caller's stream (it needs only the other modes' Grams)
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    void *base;
    size_t bytes;
    // fibre reuse (3-way): modes 0 and 1 share the mode-2 fibre sums
    // T(f, :) = sum_k X(i,j,k) C(k, :) (C does not change between their
    // updates), each then an SpMTTKRP over the fibre tensor
    const fcoo_t *fib_ttm;  // SpTTM handle along mode 2 (not owned)
    fcoo_t *fib_X[2];       // fibre tensor, SpMTTKRP handles for modes 0 and 1
    float *fib_T;           // nfib x R
    float *fib_f32;         // FP32 copy of a BF16 factor (max(I_0, I_1) x R)
};

namespace fcx {
namespace {

constexpr int kRowsPerBlock = 128;  // rows per CTA in the I x R kernels
constexpr int kSolveThreads = 256;
// Relative size below which a Cholesky pivot or an eigenvalue of V counts as
// zero, as in the FP64 oracle.  It is meaningful here because the Grams are
// compensated (Dot2) sums of the stored factors, accurate to ~1e-13: with
// plain FP32 partial sums (~1e-7) rounding noise passed for rank.
constexpr double kRankTol = 1e-12;

// W (FP64) -> Wf[0 .. R*R) = FP32 high part, Wf[R*R .. 2*R*R) = FP32 remainder.
__device__ __forceinline__ void split_store(float *Wf, int RR, int e, double w) {
    const float hi = (float)w;
    Wf[e] = hi;
    Wf[RR + e] = (float)(w - (double)hi);
}

int64_t max_blocks(int64_t max_dim) { return ceil_div(max_dim, kRowsPerBlock); }

template <typename TF>
__device__ __forceinline__ float ldf(const TF *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// ---------------------------------------------------------------- |X|^2

__global__ void k_sumsq_part(const float *val, int64_t n, double *part) {
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double v = val[p];
        s += v * v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_final(const double *part, int nb, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------- solve

struct GramList {
    const double *g[FCOO_MAX_MODES];
    int n;
};

// Moore-Penrose inverse of the normal matrix held in Q (V is work space) from
// a cyclic Jacobi eigendecomposition, dropping eigenvalues |w| <= kRankTol *
// max |w|; W = the inverse (FP64), Wf = its FP32 split.  Whole CTA.
__device__ void pinv_jacobi(int R, double *V, double *Q, double *W, float *Wf, int *flags) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double s_c, s_s;
    __shared__ int s_done;
    if (tid == 0) atomicAdd(flags, 1);
    // A (in V) <- copy of the normal matrix, Q (eigenvectors) <- I
    for (int e = tid; e < R * R; e += nt) {
        V[e] = Q[e];
        Q[e] = (e / R == e % R) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 100; ++sweep) {
        if (tid == 0) {
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < R; ++i)
                for (int j = 0; j < R; ++j) {
                    double a = V[i * R + j];
                    tot += a * a;
                    if (i != j) off += a * a;
                }
            s_done = (off <= 1e-30 * tot || off == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (s_done) break;
        for (int p = 0; p < R - 1; ++p)
            for (int q = p + 1; q < R; ++q) {
                if (tid == 0) {
                    double apq = V[p * R + q];
                    if (apq == 0.0) {
                        s_c = 1.0;
                        s_s = 0.0;
                    } else {
                        double theta = (V[q * R + q] - V[p * R + p]) / (2.0 * apq);
                        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        s_c = 1.0 / sqrt(t * t + 1.0);
                        s_s = t * s_c;
                    }
                }
                __syncthreads();
                const double c = s_c, s = s_s;
                if (s != 0.0) {
                    for (int k = tid; k < R; k += nt) {  // columns p, q
                        double akp = V[k * R + p], akq = V[k * R + q];
                        V[k * R + p] = c * akp - s * akq;
                        V[k * R + q] = s * akp + c * akq;
                    }
                    __syncthreads();
                    for (int k = tid; k < R; k += nt) {  // rows p, q
                        double apk = V[p * R + k], aqk = V[q * R + k];
                        V[p * R + k] = c * apk - s * aqk;
                        V[q * R + k] = s * apk + c * aqk;
                        double qkp = Q[k * R + p], qkq = Q[k * R + q];
                        Q[k * R + p] = c * qkp - s * qkq;
                        Q[k * R + q] = s * qkp + c * qkq;
                    }
                }
                __syncthreads();
            }
    }
    __shared__ double s_wmax;
    if (tid == 0) {
        double m = 0.0;
        for (int i = 0; i < R; ++i) m = fmax(m, fabs(V[i * R + i]));
        s_wmax = m;
    }
    __syncthreads();
    for (int e = tid; e < R * R; e += nt) {
        int a = e / R, b = e % R;
        double s = 0.0;
        for (int k = 0; k < R; ++k) {
            double w = V[k * R + k];
            if (fabs(w) <= kRankTol * s_wmax || w == 0.0) continue;
            s += Q[a * R + k] * Q[b * R + k] / w;
        }
        W[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < R * R; e += nt) split_store(Wf, R * R, e, W[e]);
}

// One CTA.  V = Hadamard of the listed Grams; W = V^-1 via FP64 Cholesky,
// or, when a pivot d <= kRankTol * max diag(V), the Moore-Penrose inverse from
// a cyclic Jacobi eigendecomposition dropping |w| <= kRankTol * max |w|.
__global__ void __launch_bounds__(kSolveThreads) k_solve(GramList gl, int R, double *V, double *Q, double *W,
                                                         float *Wf, int *flags) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double s_dmax;
    __shared__ int s_ok;
    for (int e = tid; e < R * R; e += nt) {
        double v = 1.0;
        for (int k = 0; k < gl.n; ++k) v *= gl.g[k][e];
        V[e] = v;
        Q[e] = v;  // copy kept for the eigen fallback
    }
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        int finite = 1;
        for (int i = 0; i < R; ++i) m = fmax(m, V[i * R + i]);
        for (int e = 0; e < R * R; ++e) finite &= isfinite(V[e]) ? 1 : 0;
        if (!finite) atomicOr(flags + 1, 1);
        s_dmax = m;
        s_ok = (m > 0.0 && finite) ? 1 : 0;
    }
    __syncthreads();
    // right-looking Cholesky in place (lower triangle)
    for (int j = 0; j < R && s_ok; ++j) {
        if (tid == 0) {
            double d = V[j * R + j];
            if (!(d > kRankTol * s_dmax)) s_ok = 0;
            else V[j * R + j] = sqrt(d);
        }
        __syncthreads();
        if (!s_ok) break;
        const double ljj = V[j * R + j];
        for (int i = j + 1 + tid; i < R; i += nt) V[i * R + j] /= ljj;
        __syncthreads();
        const int m = R - j - 1;
        for (int e = tid; e < m * m; e += nt) {
            int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) V[i * R + k] -= V[i * R + j] * V[k * R + j];
        }
        __syncthreads();
    }
    if (s_ok) {
        // W = L^-T L^-1: column c of L^-1 by forward substitution (thread c),
        // kept in the upper triangle of W transposed: W[c*R + i] = Linv[i][c]
        for (int c = tid; c < R; c += nt) {
            for (int i = 0; i < R; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                if (i < c) {
                    W[c * R + i] = 0.0;
                    continue;
                }
                for (int k = c; k < i; ++k) s -= V[i * R + k] * W[c * R + k];
                W[c * R + i] = s / V[i * R + i];
            }
        }
        __syncthreads();
        // V <- (L^-1)^T L^-1 ; entry (a,b) = sum_k Linv[k][a] Linv[k][b]
        for (int e = tid; e < R * R; e += nt) {
            int a = e / R, b = e % R;
            int k0 = a > b ? a : b;
            double s = 0.0;
            for (int k = k0; k < R; ++k) s += W[a * R + k] * W[b * R + k];
            V[e] = s;
        }
        __syncthreads();
        for (int e = tid; e < R * R; e += nt) {
            W[e] = V[e];
            split_store(Wf, R * R, e, V[e]);
        }
        return;
    }
    pinv_jacobi(R, V, Q, W, Wf, flags);
}

// Largest R whose normal matrix and triangular inverse both fit in shared memory.
constexpr int kSolveSmemMaxR = 112;

// The same solve with the matrices in shared memory (R <= kSolveSmemMaxR),
// for the FP64 rate of GB300 and to keep each step off the memory system:
//  * V = Hadamard of the Grams; max diag(V) and finiteness by block reduction;
//  * right-looking Cholesky, two barriers per column: the pivot's reciprocal
//    square root by one thread, then one FMA per trailing entry (the column
//    is scaled to L a step later);
//  * Y = L^-1 by forward substitution over all columns at once, one barrier
//    per row;
//  * W = Y^T Y on the upper triangle, mirrored, and split to FP32 hi + lo.
// A non-positive pivot d_j <= kRankTol * max diag(V) (or a non-finite V) sends
// the whole CTA to the Jacobi pseudo-inverse, as in k_solve.
__global__ void __launch_bounds__(kSolveThreads) k_solve_smem(GramList gl, int R, double *V, double *Q, double *W,
                                                              float *Wf, int *flags) {
    extern __shared__ double sd[];
    double *A = sd;          // R x R: V, then L in the lower triangle
    double *Y = sd + R * R;  // R x R: L^-1 (lower triangle)
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double s_wmax[kSolveThreads / 32];
    __shared__ int s_wbad[kSolveThreads / 32];
    double dmax = 0.0;
    int bad = 0;
    for (int e = tid; e < R * R; e += nt) {
        double v = 1.0;
        for (int k = 0; k < gl.n; ++k) v *= gl.g[k][e];
        A[e] = v;
        Q[e] = v;  // copy kept for the eigen fallback
        bad |= isfinite(v) ? 0 : 1;
        if (e / R == e % R) dmax = fmax(dmax, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((tid & 31) == 0) {
        s_wmax[tid >> 5] = dmax;
        s_wbad[tid >> 5] = bad;
    }
    __syncthreads();
    dmax = 0.0;
    bad = 0;
    for (int w = 0; w < nt / 32; ++w) {
        dmax = fmax(dmax, s_wmax[w]);
        bad |= s_wbad[w];
    }
    if (bad && tid == 0) atomicOr(flags + 1, 1);
    __shared__ double s_inv[kSolveSmemMaxR];  // 1 / L(j, j)
    __shared__ double s_inv2;
    __shared__ int s_ok;
    if (tid == 0) s_ok = (dmax > 0.0 && !bad) ? 1 : 0;
    __syncthreads();
    // Right-looking Cholesky, two barriers per column.  GB300 runs FP64 with a
    // long latency per dependent operation, so the critical path is kept
    // short: thread 0 takes the pivot with one reciprocal square root
    // (l = d * r, 1 / l = r), and every trailing entry gets one FMA with the
    // still unscaled column, A(i,k) -= (A(i,j) / d) A(k,j) = l_ij l_kj.
    // Column j is scaled to L in the next column's update phase, when nothing
    // reads it any more.
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    for (int j = 0; j < R; ++j) {
        if (tid == 0) {
            const double d = A[j * R + j];
            if (!(d > kRankTol * dmax)) {
                s_ok = 0;
            } else {
                const double r = rsqrt(d);
                s_inv[j] = r;
                s_inv2 = r * r;
            }
        }
        __syncthreads();
        if (!s_ok) break;  // uniform: read after the barrier
        const double r2 = s_inv2;
        if (j > 0) {  // column j-1 -> L
            const double r = s_inv[j - 1];
            for (int i = j + tid; i < R; i += nt) A[i * R + j - 1] *= r;
        }
        for (int i = j + 1 + warp; i < R; i += nwarps) {
            const double t = A[i * R + j] * r2;
            for (int k = j + 1 + lane; k <= i; k += 32) A[i * R + k] = fma(-t, A[k * R + j], A[i * R + k]);
        }
        __syncthreads();
    }
    if (!s_ok) {
        pinv_jacobi(R, V, Q, W, Wf, flags);
        return;
    }
    // the diagonal of L: l_jj = d_j * r_j (the last column has nothing below it)
    for (int i = tid; i < R; i += nt) A[i * R + i] *= s_inv[i];
    // Y = L^-1 by forward substitution, all columns at once and the rows in
    // order: once row k of Y is final, every later row subtracts its multiple
    // of it (one FMA per entry, independent across entries, a barrier per
    // row) -- the dependent chain is R steps long instead of R^2 / 2.
    // Y starts as the identity and holds the running right-hand sides.
    for (int e = tid; e < R * R; e += nt) Y[e] = (e / R == e % R) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < R; ++k) {
        // row k - 1 is final: scale it by 1 / l_(k-1)(k-1)
        if (k > 0)
            for (int c = tid; c < k; c += nt) Y[(k - 1) * R + c] *= s_inv[k - 1];
        // rows i > k (a warp per row), columns c <= k (lanes along the row):
        // Y(i, c) -= l_ik * Y(k, c) / l_kk
        const double rk = s_inv[k];
        for (int i = k + 1 + warp; i < R; i += nwarps) {
            const double t = A[i * R + k] * rk;
            for (int c = lane; c <= k; c += 32) Y[i * R + c] = fma(-t, Y[k * R + c], Y[i * R + c]);
        }
        __syncthreads();
    }
    for (int c = tid; c < R; c += nt) Y[(R - 1) * R + c] *= s_inv[R - 1];
    __syncthreads();
    // W(a, b) = sum_{k >= max(a, b)} Y(k, a) Y(k, b) for a <= b: a warp per
    // row a, lanes along b, four partial sums per entry
    for (int a = warp; a < R; a += nwarps) {
        for (int b = a + lane; b < R; b += 32) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int k = b;
            for (; k + 3 < R; k += 4) {
                s0 = fma(Y[k * R + a], Y[k * R + b], s0);
                s1 = fma(Y[(k + 1) * R + a], Y[(k + 1) * R + b], s1);
                s2 = fma(Y[(k + 2) * R + a], Y[(k + 2) * R + b], s2);
                s3 = fma(Y[(k + 3) * R + a], Y[(k + 3) * R + b], s3);
            }
            for (; k < R; ++k) s0 = fma(Y[k * R + a], Y[k * R + b], s0);
            const double w = (s0 + s1) + (s2 + s3);
            W[a * R + b] = w;
            W[b * R + a] = w;
            split_store(Wf, R * R, a * R + b, w);
            split_store(Wf, R * R, b * R + a, w);
        }
    }
}

// ---------------------------------------------------------------- I x R kernels

// Compensated FP32 dot product (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, algorithm Dot2): the product is split
// exactly with an FMA, the running sum with TwoSum, and all rounding errors
// are collected in c, so s + c carries about twice the FP32 precision.  The
// _rn intrinsics keep the compiler from contracting the error terms.
struct Dot2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);  // a * b == p + pe exactly
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p == t + se
        s = t;
        c = __fadd_rn(c, __fadd_rn(se, pe));
    }
    __device__ __forceinline__ void add_small(float a, float b) { c = fmaf(a, b, c); }
};

// Fu = M * W, one CTA per kRowsPerBlock rows, W = Wf_hi + Wf_lo (the FP64
// inverse split into two FP32 parts) and Dot2 accumulation, so the result is
// accurate to about one FP32 rounding even when V is ill-conditioned (a plain
// FP32 product would lose about cond(V) ulps).  Column sums of squares of Fu
// per CTA into part[blk * R + c] (FP64).
__global__ void k_apply(const float *M, const float *Wf, int64_t I, int R, float *Fu, double *part) {
    extern __shared__ __align__(16) float sm[];
    float *sWh = sm;                // R x R
    float *sWl = sm + R * R;        // R x R
    float *sM = sm + 2 * R * R;     // kRowsPerBlock x R
    const int64_t i0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int rows = (int)min((int64_t)kRowsPerBlock, I - i0);
    for (int e = threadIdx.x; e < 2 * R * R; e += blockDim.x) sWh[e] = Wf[e];
    for (int e = threadIdx.x; e < rows * R; e += blockDim.x) sM[e] = M[i0 * R + e];
    __syncthreads();
    // blockDim.x is a multiple of R: thread (r0, c) handles column c of rows r0, r0 + step, ...
    const int c = threadIdx.x % R, r0 = threadIdx.x / R, step = blockDim.x / R;
    __shared__ double red[1024];
    Dot2 sq;  // compensated FP32: a long FP64 chain is slow at GB300's FP64 rate
    // four rows at a time: four independent compensated chains in flight
    for (int r = r0; r < rows; r += 4 * step) {
        Dot2 d[4];
        int rr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) rr[u] = min(r + u * step, rows - 1);
        for (int k = 0; k < R; ++k) {
            const float wh = sWh[k * R + c], wl = sWl[k * R + c];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float m = sM[rr[u] * R + k];
                d[u].add(m, wh);
                d[u].add_small(m, wl);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (r + u * step >= rows) break;
            const float s = __fadd_rn(d[u].s, d[u].c);
            Fu[(i0 + r + u * step) * R + c] = s;
            sq.add(s, s);
        }
    }
    red[r0 * R + c] = (double)sq.s + (double)sq.c;
    __syncthreads();
    if (r0 == 0) {
        double t = 0.0;
        for (int q = 0; q < step; ++q) t += red[q * R + c];
        part[(int64_t)blockIdx.x * R + c] = t;
    }
}

// sum_b part[b * stride + x] for the x this thread serves, over the blocks
// b = q, q + P, ... ; the P partial sums of each x are then added in q order
// by part_combine.  Short FP64 chains: GB300 runs FP64 at a small fraction of
// its FP32 rate, and a 200-long dependent chain per thread is its latency
// times 200.
__device__ __forceinline__ double part_sum(const double *part, int nb, int64_t stride, int x, int q, int P) {
    double s0 = 0.0, s1 = 0.0;
    int b = q;
    for (; b + P < nb; b += 2 * P) {
        s0 += part[(int64_t)b * stride + x];
        s1 += part[(int64_t)(b + P) * stride + x];
    }
    if (b < nb) s0 += part[(int64_t)b * stride + x];
    return s0 + s1;
}

// lambda_c = sqrt(sum_b part[b][c]); one CTA of kSolveThreads threads, R <= 128.
__global__ void __launch_bounds__(kSolveThreads) k_lambda(const double *part, int nb, int R, double *lambda,
                                                          int *flags) {
    __shared__ double red[kSolveThreads];
    const int P = blockDim.x / R, q = threadIdx.x / R, c = threadIdx.x % R;
    if (q < P) red[threadIdx.x] = part_sum(part, nb, R, c, q, P);
    __syncthreads();
    if (threadIdx.x < R) {
        double s = 0.0;
        for (int t = 0; t < P; ++t) s += red[t * R + c];
        const double l = sqrt(s);
        if (!isfinite(l)) atomicOr(flags + 1, 1);
        lambda[c] = l;
    }
}

// F = Fu / lambda (columns with lambda = 0 kept as they are), stored as TF;
// optional per-CTA partial of sum_i M(i,c) * F(i,c) with the stored F.
template <typename TF>
__global__ void k_normalize(const float *Fu, const double *lambda, int64_t I, int R, TF *F, const float *M,
                            double *dotpart) {
    const int64_t i0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int rows = (int)min((int64_t)kRowsPerBlock, I - i0);
    __shared__ double red[1024];
    const int c = threadIdx.x % R, r0 = threadIdx.x / R, step = blockDim.x / R;
    const double l = lambda[c];
    const float inv = l > 0.0 ? (float)(1.0 / l) : 1.0f;
    Dot2 dot;
    for (int r = r0; r < rows; r += step) {
        const int64_t e = (i0 + r) * R + c;
        float v = Fu[e] * inv;
        TF st;
        if constexpr (sizeof(TF) == 2) st = __float2bfloat16_rn(v);
        else st = v;
        F[e] = st;
        if (dotpart) dot.add(M[e], ldf<TF>(&st));
    }
    if (dotpart) {
        red[r0 * R + c] = (double)dot.s + (double)dot.c;
        __syncthreads();
        if (r0 == 0) {
            double t = 0.0;
            for (int q = 0; q < step; ++q) t += red[q * R + c];
            dotpart[(int64_t)blockIdx.x * R + c] = t;
        }
    }
}

// Per-CTA Gram partial of the stored factor rows [i0, i0 + rows): Dot2
// (compensated FP32) sums of kRowsPerBlock products, written as FP64, so the
// Gram of the stored factor is accurate to ~1e-13 relative and rank decisions
// on V see the factors, not the summation error.
template <typename TF>
__global__ void k_gram_part(const TF *F, int64_t I, int R, double *part) {
    extern __shared__ __align__(16) float sF[];
    const int64_t i0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int rows = (int)min((int64_t)kRowsPerBlock, I - i0);
    for (int e = threadIdx.x; e < rows * R; e += blockDim.x) sF[e] = ldf<TF>(F + i0 * R + e);
    __syncthreads();
    // four entries per pass: four independent compensated chains in flight
    const int RR = R * R, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < RR; e0 += 4 * nt) {
        int a[4], b[4];
        Dot2 d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = min(e0 + u * nt, RR - 1);
            a[u] = e / R;
            b[u] = e % R;
        }
        for (int r = 0; r < rows; ++r) {
            const float *row = sF + r * R;
#pragma unroll
            for (int u = 0; u < 4; ++u) d[u].add(row[a[u]], row[b[u]]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * nt;
            if (e < RR) part[(int64_t)blockIdx.x * RR + e] = (double)d[u].s + (double)d[u].c;
        }
    }
}

// G[e] = sum_b part[b][e]; blocks of 256 threads serve 32 entries, 8 threads each.
__global__ void __launch_bounds__(256) k_gram_reduce(const double *part, int nb, int R, double *G) {
    __shared__ double red[256];
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), q = threadIdx.x >> 5;
    const int RR = R * R;
    red[threadIdx.x] = x < RR ? part_sum(part, nb, RR, x, q, 8) : 0.0;
    __syncthreads();
    if (threadIdx.x < 32 && x < RR) {
        double s = 0.0;
        for (int t = 0; t < 8; ++t) s += red[t * 32 + threadIdx.x];
        G[x] = s;
    }
}

struct GramAll {
    const double *g[FCOO_MAX_MODES];
    int n;
};

// fit = 1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2 <X,Xhat>)) / |X| ; one CTA.
__global__ void k_fit(GramAll ga, const double *lambda, int R, const double *dotpart, int nb, double *scal) {
    __shared__ double red[256];
    double xh = 0.0, inner = 0.0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        double v = lambda[e / R] * lambda[e % R];
        for (int k = 0; k < ga.n; ++k) v *= ga.g[k][e];
        xh += v;
    }
    {
        const int P = blockDim.x / R, q = threadIdx.x / R, c = threadIdx.x % R;
        if (q < P) inner = lambda[c] * part_sum(dotpart, nb, R, c, q, P);
    }
    red[threadIdx.x] = xh;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double xhat2 = red[0];
    __syncthreads();
    red[threadIdx.x] = inner;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double in = red[0], nx = scal[0];
        const double r2 = nx + xhat2 - 2.0 * in;
        scal[1] = 1.0 - sqrt(r2 > 0.0 ? r2 : 0.0) / sqrt(nx);
        scal[2] = in;
        scal[3] = xhat2;
    }
}

__global__ void k_to_dtype(const float *src, int64_t n, __nv_bfloat16 *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_to_f32(const __nv_bfloat16 *src, int64_t n, float *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __bfloat162float(src[i]);
}

unsigned gs(int64_t n) {
    int64_t b = ceil_div(n, 256);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

int gram_of(cp_state_t *st, int k, cudaStream_t s) {
    const int R = st->R;
    const int64_t I = st->dims[k];
    const int nb = (int)ceil_div(I, kRowsPerBlock);
    const size_t smem = (size_t)kRowsPerBlock * R * 4;
    if (st->dtype == FCOO_BF16) {
        FCOO_CUDA(cudaFuncSetAttribute(k_gram_part<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        k_gram_part<__nv_bfloat16><<<nb, 256, smem, s>>>((const __nv_bfloat16 *)st->F[k], I, R, st->part);
    } else {
        FCOO_CUDA(cudaFuncSetAttribute(k_gram_part<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_gram_part<float><<<nb, 256, smem, s>>>((const float *)st->F[k], I, R, st->part);
    }
    FCOO_CUDA(cudaGetLastError());
    k_gram_reduce<<<(unsigned)ceil_div(R * R, 32), 256, 0, s>>>(st->part, nb, R, st->gram[k]);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}

__global__ void k_bf16_to_f32(const __nv_bfloat16 *a, int64_t n, float *b) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = __bfloat162float(a[e]);
}

void fibres_release(cp_state_t *st) {
    for (int k = 0; k < 2; ++k) {
        if (st->fib_X[k]) fcoo_destroy(st->fib_X[k]);
        st->fib_X[k] = nullptr;
    }
    dev_free(st->fib_T);
    dev_free(st->fib_f32);
    st->fib_T = st->fib_f32 = nullptr;
    st->fib_ttm = nullptr;
}

// M = SpMTTKRP of mode n < 2 through the fibre sums: for mode 0 first the
// sums T = SpTTM along mode 2 with the current C (Eq. 3), then Eq. 6 over the
// fibre tensor with factors (B, T) for mode 0 or (A, T) for mode 1, in FP32
// (a BF16 factor is widened first).  Both launches leave one CTA slot for
// the solve on the side stream.
int mode_mttkrp_fibres(cp_state_t *st, int n, cudaStream_t s) {
    const int R = st->R;
    if (n == 0 && st->fib_ttm->nnz > 0) {
        StreamParams q;
        stream_params_from(st->fib_ttm, q);
        q.F[0] = st->F[2];
        q.out = st->fib_T;
        q.R = R;
        q.out_rows = st->fib_ttm->nseg;
        q.reserve_ctas = 1;
        int rc = launch_stream_kernel(q, st->dtype, s);
        if (rc) return rc;
    }
    const fcoo_t *Xf = st->fib_X[n];
    if (Xf->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(st->M, 0, (size_t)st->dims[n] * R * 4, s));
        return FCOO_OK;
    }
    const void *other = st->F[1 - n];
    if (st->dtype == FCOO_BF16) {
        const int64_t ne = (int64_t)st->dims[1 - n] * R;
        k_bf16_to_f32<<<(unsigned)std::min<int64_t>(ceil_div(ne, 256), 4096), 256, 0, s>>>(
            (const __nv_bfloat16 *)other, ne, st->fib_f32);
        FCOO_CUDA(cudaGetLastError());
        other = st->fib_f32;
    }
    StreamParams p;
    stream_params_from(Xf, p);
    p.F[0] = other;      // product modes of the fibre tensor: the other index mode, then f
    p.F[1] = st->fib_T;
    p.out = st->M;
    p.R = R;
    p.out_rows = st->dims[n];
    p.reserve_ctas = 1;
    return launch_stream_kernel(p, FCOO_F32, s);
}

// One mode update of Algorithm 1.
int mode_update(const fcoo_t *X, cp_state_t *st, int n, bool last, cudaStream_t s) {
    const int R = st->R;
    const int64_t I = st->dims[n];
    // V = Hadamard of the other modes' Grams and V^-1: on the side stream,
    // overlapped with SpMTTKRP (one CTA beside a grid that leaves it a slot)
    GramList gl;
    memset(&gl, 0, sizeof(gl));
    for (int k = 0; k < st->nmodes; ++k)
        if (k != n) gl.g[gl.n++] = st->gram[k];
    FCOO_CUDA(cudaEventRecord(st->ev_fork, s));
    FCOO_CUDA(cudaStreamWaitEvent(st->side, st->ev_fork, 0));
    if (R <= kSolveSmemMaxR) {
        const int smem = 2 * R * R * 8;
        FCOO_CUDA(cudaFuncSetAttribute(k_solve_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_solve_smem<<<1, kSolveThreads, smem, st->side>>>(gl, R, st->V, st->Q, st->W, st->Wf, st->flags);
    } else {
        k_solve<<<1, kSolveThreads, 0, st->side>>>(gl, R, st->V, st->Q, st->W, st->Wf, st->flags);
    }
    FCOO_CUDA(cudaGetLastError());
    FCOO_CUDA(cudaEventRecord(st->ev_join, st->side));
    // M = SpMTTKRP_n
    StreamParams p;
    stream_params_from(X, p);
    for (int m = 0; m < X->nprod; ++m) p.F[m] = st->F[X->prod_modes[m]];
    p.out = st->M;
    p.R = R;
    p.out_rows = I;
    p.reserve_ctas = 1;
    if (st->fib_ttm && n < 2) {
        int rc = mode_mttkrp_fibres(st, n, s);
        if (rc) return rc;
    } else if (X->nnz == 0) {
        FCOO_CUDA(cudaMemsetAsync(st->M, 0, (size_t)I * R * 4, s));
    } else {
        int rc = launch_stream_kernel(p, st->dtype, s);
        if (rc) return rc;
    }
    FCOO_CUDA(cudaStreamWaitEvent(s, st->ev_join, 0));
    // Fu = M W, column norms
    const int nb = (int)ceil_div(I, kRowsPerBlock);
    const int threads = R >= 256 ? R : (256 / R) * R;  // a multiple of R
    const size_t smem = ((size_t)2 * R * R + (size_t)kRowsPerBlock * R) * 4;
    FCOO_CUDA(cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_apply<<<nb, threads, smem, s>>>(st->M, st->Wf, I, R, st->Fu, st->part);
    FCOO_CUDA(cudaGetLastError());
    k_lambda<<<1, 256, 0, s>>>(st->part, nb, R, st->lambda, st->flags);
    FCOO_CUDA(cudaGetLastError());
    double *dotpart = last ? st->part : nullptr;
    if (st->dtype == FCOO_BF16)
        k_normalize<__nv_bfloat16><<<nb, threads, 0, s>>>(st->Fu, st->lambda, I, R, (__nv_bfloat16 *)st->F[n],
                                                          st->M, dotpart);
    else
        k_normalize<float><<<nb, threads, 0, s>>>(st->Fu, st->lambda, I, R, (float *)st->F[n], st->M, dotpart);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}

}  // namespace

// Helpers shared with the Tucker solver (tucker.cu).
int gram_f32_fp64(const float *F, int64_t I, int R, double *part, double *G, cudaStream_t s) {
    const int nb = (int)ceil_div(I, kRowsPerBlock);
    const size_t smem = (size_t)kRowsPerBlock * R * 4;
    FCOO_CUDA(cudaFuncSetAttribute(k_gram_part<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gram_part<float><<<nb, 256, smem, s>>>(F, I, R, part);
    FCOO_CUDA(cudaGetLastError());
    k_gram_reduce<<<(unsigned)ceil_div(R * R, 32), 256, 0, s>>>(part, nb, R, G);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}

int sumsq_fp64(const float *val, int64_t n, double *part, double *out, cudaStream_t s) {
    const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, ceil_div(n, 256)));
    k_sumsq_part<<<nb, 256, 0, s>>>(val, n, part);
    k_sum_final<<<1, 256, 0, s>>>(part, nb, out);
    FCOO_CUDA(cudaGetLastError());
    return FCOO_OK;
}

}  // namespace fcx

using namespace fcx;

extern "C" int cp_state_create(int nmodes, const uint32_t *dims, int R, int dtype, const float *const *init,
                               fcoo_stream_t stream, cp_state_t **out) {
    clear_error();
    if (!out) return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: out is NULL");
    *out = nullptr;
    if (nmodes < 2 || nmodes > FCOO_MAX_MODES || !dims || !init)
        return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: bad nmodes/dims/init");
    if (R < 1 || R > 128) return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: R=%d outside 1..128", R);
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: bad dtype");
    for (int k = 0; k < nmodes; ++k) {
        if (dims[k] == 0) return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: dims[%d] is 0", k);
        if (!init[k]) return fail(FCOO_ERR_INVALID_ARG, "cp_state_create: init[%d] is NULL", k);
    }
    cudaStream_t s = (cudaStream_t)stream;
    cp_state_t *st = (cp_state_t *)calloc(1, sizeof(cp_state_t));
    if (!st) return fail(FCOO_ERR_NOMEM, "cp_state_create: host allocation failed");
    st->nmodes = nmodes;
    st->R = R;
    st->dtype = dtype;
    st->max_dim = 0;
    for (int k = 0; k < nmodes; ++k) {
        st->dims[k] = dims[k];
        st->max_dim = std::max<int64_t>(st->max_dim, dims[k]);
    }
    // factor buffers are FP32-sized for either dtype, so that
    // cp_state_set_dtype can change the storage in place
    const size_t es = 4;
    const int64_t nbmax = max_blocks(st->max_dim);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += round_up((int64_t)b, 256);
        return o;
    };
    size_t oF[FCOO_MAX_MODES], oG[FCOO_MAX_MODES];
    for (int k = 0; k < nmodes; ++k) oF[k] = take((size_t)dims[k] * R * es);
    for (int k = 0; k < nmodes; ++k) oG[k] = take((size_t)R * R * 8);
    size_t oL = take(R * 8), oM = take((size_t)st->max_dim * R * 4), oFu = take((size_t)st->max_dim * R * 4);
    size_t oV = take((size_t)R * R * 8), oQ = take((size_t)R * R * 8), oW = take((size_t)R * R * 8);
    size_t oWf = take((size_t)2 * R * R * 4);
    size_t oP = take((size_t)std::max<int64_t>(nbmax * R * R, 4096) * 8);
    size_t oS = take(8 * 8), oFl = take(16);
    cudaError_t e = dev_alloc(&st->base, off);
    if (e != cudaSuccess) {
        free(st);
        return cuda_fail(e, "cp_state_create: cudaMalloc");
    }
    st->bytes = off;
    char *b = (char *)st->base;
    for (int k = 0; k < nmodes; ++k) {
        st->F[k] = b + oF[k];
        st->gram[k] = (double *)(b + oG[k]);
    }
    st->lambda = (double *)(b + oL);
    st->M = (float *)(b + oM);
    st->Fu = (float *)(b + oFu);
    st->V = (double *)(b + oV);
    st->Q = (double *)(b + oQ);
    st->W = (double *)(b + oW);
    st->Wf = (float *)(b + oWf);
    st->part = (double *)(b + oP);
    st->scal = (double *)(b + oS);
    st->flags = (int *)(b + oFl);
    int rc = FCOO_OK;
    auto cu = [&](cudaError_t ce, const char *what) {
        if (ce != cudaSuccess && rc == FCOO_OK) rc = cuda_fail(ce, what);
    };
    cu(cudaMemsetAsync(st->base, 0, off, s), "cudaMemsetAsync");
    for (int k = 0; k < nmodes && rc == FCOO_OK; ++k) {
        const size_t n = (size_t)dims[k] * R;
        if (dtype == FCOO_F32) {
            cu(cudaMemcpyAsync(st->F[k], init[k], n * 4, cudaMemcpyDefault, s), "cudaMemcpyAsync(init)");
        } else {
            cu(cudaMemcpyAsync(st->Fu, init[k], n * 4, cudaMemcpyDefault, s), "cudaMemcpyAsync(init)");
            k_to_dtype<<<gs(n), 256, 0, s>>>(st->Fu, n, (__nv_bfloat16 *)st->F[k]);
            cu(cudaGetLastError(), "k_to_dtype");
        }
        if (rc == FCOO_OK) rc = gram_of(st, k, s);
    }
    if (rc == FCOO_OK) cu(cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking), "cudaStreamCreate");
    if (rc == FCOO_OK) cu(cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    if (rc == FCOO_OK) cu(cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    {
        double ones[FCOO_MAX_RANK];
        for (int r = 0; r < R; ++r) ones[r] = 1.0;
        cu(cudaMemcpyAsync(st->lambda, ones, R * 8, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(lambda)");
        cu(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    if (rc != FCOO_OK) {
        if (st->ev_join) cudaEventDestroy(st->ev_join);
        if (st->ev_fork) cudaEventDestroy(st->ev_fork);
        if (st->side) cudaStreamDestroy(st->side);
        dev_free(st->base);
        free(st);
        return rc;
    }
    *out = st;
    return FCOO_OK;
}

extern "C" int cp_state_set_dtype(cp_state_t *st, int dtype, fcoo_stream_t stream) {
    clear_error();
    if (!st) return fail(FCOO_ERR_INVALID_ARG, "cp_state_set_dtype: NULL state");
    if (dtype != FCOO_F32 && dtype != FCOO_BF16) return fail(FCOO_ERR_INVALID_ARG, "cp_state_set_dtype: bad dtype");
    if (dtype == st->dtype) return FCOO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < st->nmodes; ++k) {
        const int64_t n = (int64_t)st->dims[k] * st->R;
        if (dtype == FCOO_F32) {
            // BF16 -> FP32 is exact: the Grams of the stored factors stay valid
            k_to_f32<<<gs(n), 256, 0, s>>>((const __nv_bfloat16 *)st->F[k], n, st->Fu);
            FCOO_CUDA(cudaGetLastError());
            FCOO_CUDA(cudaMemcpyAsync(st->F[k], st->Fu, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        } else {
            // FP32 -> BF16 rounds: the Grams are recomputed from the rounded factors
            FCOO_CUDA(cudaMemcpyAsync(st->Fu, st->F[k], (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
            k_to_dtype<<<gs(n), 256, 0, s>>>(st->Fu, n, (__nv_bfloat16 *)st->F[k]);
            FCOO_CUDA(cudaGetLastError());
        }
    }
    st->dtype = dtype;
    if (dtype == FCOO_BF16)
        for (int k = 0; k < st->nmodes; ++k) {
            const int rc = gram_of(st, k, s);
            if (rc) return rc;
        }
    return FCOO_OK;
}

extern "C" int cp_state_destroy(cp_state_t *st) {
    clear_error();
    if (!st) return FCOO_OK;
    cudaDeviceSynchronize();
    if (st->ev_join) cudaEventDestroy(st->ev_join);
    if (st->ev_fork) cudaEventDestroy(st->ev_fork);
    if (st->side) cudaStreamDestroy(st->side);
    fibres_release(st);
    dev_free(st->base);
    free(st);
    return FCOO_OK;
}

extern "C" int cp_state_use_fibres(cp_state_t *st, const fcoo_t *Xttm, int threadlen, fcoo_stream_t stream) {
    clear_error();
    if (!st) return fail(FCOO_ERR_INVALID_ARG, "cp_state_use_fibres: NULL state");
    cudaStream_t s = (cudaStream_t)stream;
    FCOO_CUDA(cudaStreamSynchronize(s));
    fibres_release(st);
    if (!Xttm) return FCOO_OK;
    if (st->nmodes != 3 || Xttm->op != FCOO_OP_TTM || Xttm->nmodes != 3 || Xttm->mode != 2)
        return fail(FCOO_ERR_INVALID_ARG, "cp_state_use_fibres: needs a 3-way state and the SpTTM handle along mode 2");
    for (int k = 0; k < 3; ++k)
        if (Xttm->dims[k] != st->dims[k]) return fail(FCOO_ERR_INVALID_ARG, "cp_state_use_fibres: dims differ");
    int rc = FCOO_OK;
    for (int k = 0; k < 2 && rc == FCOO_OK; ++k) rc = fibre_tensor_build(Xttm, k, threadlen, s, &st->fib_X[k]);
    if (rc == FCOO_OK) {
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&st->fib_T), (size_t)std::max<int64_t>(Xttm->nseg, 1) * st->R * 4);
        if (e == cudaSuccess)
            e = dev_alloc(reinterpret_cast<void **>(&st->fib_f32),
                          (size_t)std::max(st->dims[0], st->dims[1]) * st->R * 4);
        if (e != cudaSuccess) rc = cuda_fail(e, "cp_state_use_fibres");
    }
    if (rc != FCOO_OK) {
        fibres_release(st);
        return rc;
    }
    st->fib_ttm = Xttm;
    return FCOO_OK;
}

extern "C" int cp_als_iter(const fcoo_t *const *Xn, cp_state_t *st, fcoo_stream_t stream) {
    clear_error();
    if (!Xn || !st) return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: NULL argument");
    for (int n = 0; n < st->nmodes; ++n) {
        const fcoo_t *X = Xn[n];
        if (!X) return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: Xn[%d] is NULL", n);
        if (X->op != FCOO_OP_MTTKRP || X->mode != n || X->nmodes != st->nmodes)
            return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: Xn[%d] is not an SpMTTKRP handle for mode %d", n, n);
        for (int k = 0; k < st->nmodes; ++k)
            if (X->dims[k] != st->dims[k]) return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: Xn[%d] dims differ", n);
        if (X->nnz != Xn[0]->nnz) return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: handles hold different tensors");
    }
    if (st->fib_ttm && st->fib_ttm->nnz != Xn[0]->nnz)
        return fail(FCOO_ERR_INVALID_ARG, "cp_als_iter: the fibre handle holds a different tensor");
    cudaStream_t s = (cudaStream_t)stream;
    const int R = st->R;
    if (!st->have_norm) {
        const fcoo_t *X = Xn[0];
        const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, ceil_div(X->nnz, 256)));
        k_sumsq_part<<<nb, 256, 0, s>>>(X->val, X->nnz, st->part);
        k_sum_final<<<1, 256, 0, s>>>(st->part, nb, st->scal);
        FCOO_CUDA(cudaGetLastError());
        st->have_norm = true;
    }
    for (int n = 0; n < st->nmodes; ++n) {
        const bool last = n == st->nmodes - 1;
        int rc = mode_update(Xn[n], st, n, last, s);
        if (rc) return rc;
        const int nb = (int)ceil_div(st->dims[n], kRowsPerBlock);
        if (last) {
            // move the <M, F_last> partials out of `part` before the Gram pass reuses it
            FCOO_CUDA(cudaMemcpyAsync(st->Fu, st->part, (size_t)nb * R * 8, cudaMemcpyDeviceToDevice, s));
        }
        rc = gram_of(st, n, s);
        if (rc) return rc;
        if (last) {
            GramAll ga;
            memset(&ga, 0, sizeof(ga));
            for (int k = 0; k < st->nmodes; ++k) ga.g[ga.n++] = st->gram[k];
            k_fit<<<1, 256, 0, s>>>(ga, st->lambda, R, (const double *)st->Fu, nb, st->scal);
            FCOO_CUDA(cudaGetLastError());
        }
    }
    st->iters++;
    return FCOO_OK;
}

extern "C" int cp_state_stats(const cp_state_t *st, double *lambda, double *fit, int *iters, int *npinv,
                              fcoo_stream_t stream) {
    clear_error();
    if (!st) return fail(FCOO_ERR_INVALID_ARG, "cp_state_stats: NULL state");
    cudaStream_t s = (cudaStream_t)stream;
    double scal[4];
    int flags[2];
    FCOO_CUDA(cudaMemcpyAsync(scal, st->scal, sizeof(scal), cudaMemcpyDeviceToHost, s));
    FCOO_CUDA(cudaMemcpyAsync(flags, st->flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    if (lambda) FCOO_CUDA(cudaMemcpyAsync(lambda, st->lambda, st->R * 8, cudaMemcpyDeviceToHost, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    if (fit) *fit = scal[1];
    if (iters) *iters = st->iters;
    if (npinv) *npinv = flags[0];
    if (flags[1]) return fail(FCOO_ERR_NONFINITE, "cp_state_stats: a non-finite value appeared in the normal equations");
    return FCOO_OK;
}

extern "C" int cp_state_copy_factor(const cp_state_t *st, int k, float *dst, fcoo_stream_t stream) {
    clear_error();
    if (!st || !dst || k < 0 || k >= st->nmodes) return fail(FCOO_ERR_INVALID_ARG, "cp_state_copy_factor: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)st->dims[k] * st->R;
    if (st->dtype == FCOO_F32) {
        FCOO_CUDA(cudaMemcpyAsync(dst, st->F[k], n * 4, cudaMemcpyDefault, s));
    } else {
        k_to_f32<<<gs(n), 256, 0, s>>>((const __nv_bfloat16 *)st->F[k], n, st->Fu);
        FCOO_CUDA(cudaGetLastError());
        FCOO_CUDA(cudaMemcpyAsync(dst, st->Fu, n * 4, cudaMemcpyDefault, s));
    }
    FCOO_CUDA(cudaStreamSynchronize(s));
    return FCOO_OK;
}

// ---------------------------------------------------------------- checkpoint

namespace {
struct BlobHeader {
    uint64_t magic;
    int32_t nmodes, R, dtype, iters;
    uint32_t dims[FCOO_MAX_MODES];
    int32_t have_norm, pad;
};
constexpr uint64_t kMagic = 0x31504f4f43464350ull;  // "PCFCOOP1"

int64_t blob_bytes(const cp_state_t *st) {
    const size_t es = st->dtype == FCOO_BF16 ? 2 : 4;
    int64_t b = sizeof(BlobHeader);
    for (int k = 0; k < st->nmodes; ++k) b += (int64_t)st->dims[k] * st->R * es + (int64_t)st->R * st->R * 8;
    b += (int64_t)st->R * 8 + 4 * 8 + 2 * 4;
    return b;
}
}  // namespace

extern "C" int64_t cp_state_blob_size(const cp_state_t *st) { return st ? blob_bytes(st) : -1; }

extern "C" int cp_state_save(const cp_state_t *st, void *blob, int64_t size, fcoo_stream_t stream) {
    clear_error();
    if (!st || !blob || size < blob_bytes(st)) return fail(FCOO_ERR_INVALID_ARG, "cp_state_save: bad argument or size");
    cudaStream_t s = (cudaStream_t)stream;
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kMagic;
    h.nmodes = st->nmodes;
    h.R = st->R;
    h.dtype = st->dtype;
    h.iters = st->iters;
    h.have_norm = st->have_norm;
    for (int k = 0; k < st->nmodes; ++k) h.dims[k] = st->dims[k];
    char *p = (char *)blob;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t es = st->dtype == FCOO_BF16 ? 2 : 4;
    for (int k = 0; k < st->nmodes; ++k) {
        const size_t n = (size_t)st->dims[k] * st->R * es;
        FCOO_CUDA(cudaMemcpyAsync(p, st->F[k], n, cudaMemcpyDeviceToHost, s));
        p += n;
        FCOO_CUDA(cudaMemcpyAsync(p, st->gram[k], (size_t)st->R * st->R * 8, cudaMemcpyDeviceToHost, s));
        p += (size_t)st->R * st->R * 8;
    }
    FCOO_CUDA(cudaMemcpyAsync(p, st->lambda, (size_t)st->R * 8, cudaMemcpyDeviceToHost, s));
    p += (size_t)st->R * 8;
    FCOO_CUDA(cudaMemcpyAsync(p, st->scal, 4 * 8, cudaMemcpyDeviceToHost, s));
    p += 4 * 8;
    FCOO_CUDA(cudaMemcpyAsync(p, st->flags, 2 * 4, cudaMemcpyDeviceToHost, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    return FCOO_OK;
}

extern "C" int cp_state_load(cp_state_t *st, const void *blob, int64_t size, fcoo_stream_t stream) {
    clear_error();
    if (!st || !blob || size < (int64_t)sizeof(BlobHeader)) return fail(FCOO_ERR_INVALID_ARG, "cp_state_load: bad argument");
    BlobHeader h;
    memcpy(&h, blob, sizeof(h));
    if (h.magic != kMagic || h.nmodes != st->nmodes || h.R != st->R || h.dtype != st->dtype)
        return fail(FCOO_ERR_INVALID_ARG, "cp_state_load: blob does not match this state");
    for (int k = 0; k < st->nmodes; ++k)
        if (h.dims[k] != st->dims[k]) return fail(FCOO_ERR_INVALID_ARG, "cp_state_load: dims differ");
    if (size < blob_bytes(st)) return fail(FCOO_ERR_INVALID_ARG, "cp_state_load: blob too small");
    cudaStream_t s = (cudaStream_t)stream;
    const char *p = (const char *)blob + sizeof(h);
    const size_t es = st->dtype == FCOO_BF16 ? 2 : 4;
    for (int k = 0; k < st->nmodes; ++k) {
        const size_t n = (size_t)st->dims[k] * st->R * es;
        FCOO_CUDA(cudaMemcpyAsync(st->F[k], p, n, cudaMemcpyHostToDevice, s));
        p += n;
        FCOO_CUDA(cudaMemcpyAsync(st->gram[k], p, (size_t)st->R * st->R * 8, cudaMemcpyHostToDevice, s));
        p += (size_t)st->R * st->R * 8;
    }
    FCOO_CUDA(cudaMemcpyAsync(st->lambda, p, (size_t)st->R * 8, cudaMemcpyHostToDevice, s));
    p += (size_t)st->R * 8;
    FCOO_CUDA(cudaMemcpyAsync(st->scal, p, 4 * 8, cudaMemcpyHostToDevice, s));
    p += 4 * 8;
    FCOO_CUDA(cudaMemcpyAsync(st->flags, p, 2 * 4, cudaMemcpyHostToDevice, s));
    FCOO_CUDA(cudaStreamSynchronize(s));
    st->iters = h.iters;
    st->have_norm = h.have_norm != 0;
    return FCOO_OK;
}
