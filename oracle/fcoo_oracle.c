/*
 * fcoo_oracle.c -- plain, slow, FP64 CPU oracle for the F-COO sparse tensor
 * operations of "A Unified Optimization Approach for Sparse Tensor Operations
 * on GPUs" (Liu, Wen, Sarwate, Mehri Dehnavi; arXiv 1705.09905).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every function here is the plain definition written out as loops over the
 * coordinate (COO) list, in FP64, with no blocking, fusion or reordering
 * beyond what the definition states.  Indices are 0-based (the paper is
 * 1-based, Sec. II).  Inputs that the GPU path holds in FP32 or BF16 are
 * passed here already upcast to double.
 *
 * Parity status: every function is pinned by tests against brute-force dense
 * algebra (unfolding + explicit Khatri-Rao product), closed forms for Kruskal
 * tensors, special cases and invariants; nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_MODES 8

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_RANGE = -2, ORC_ERR_DUP = -3, ORC_ERR_NOMEM = -4 };

static int check_coo(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx)
{
    if (nmodes < 1 || nmodes > ORC_MAX_MODES || nnz < 0 || !dims || (nnz > 0 && !idx)) return ORC_ERR_ARG;
    for (int k = 0; k < nmodes; ++k) {
        if (dims[k] == 0) return ORC_ERR_ARG;
        for (int64_t p = 0; p < nnz; ++p)
            if (idx[k][p] >= dims[k]) return ORC_ERR_RANGE;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SpMTTKRP, Eq. 5 / Eq. 6 and Table I row 2:                                */
/*   M(i,:) += X(i,j,k) * (B(j,:) .* C(k,:)),                                 */
/* generalised to N modes: for mode n every other mode is a product mode.    */
/*   out[idx_n(p)][r] += val(p) * prod_{k != n} F_k[idx_k(p)][r]              */
/* out is dims[mode] x R row-major and is fully overwritten.                 */
/* factors[k] is dims[k] x R row-major; factors[mode] is not read.           */
/* ------------------------------------------------------------------------ */
int orc_mttkrp(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
               const double *val, const double *const *factors, int R, int mode, double *out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (mode < 0 || mode >= nmodes || R <= 0 || !out) return ORC_ERR_ARG;
    memset(out, 0, sizeof(double) * (size_t)dims[mode] * (size_t)R);
    for (int64_t p = 0; p < nnz; ++p) {
        double *row = out + (size_t)idx[mode][p] * R;
        for (int r = 0; r < R; ++r) {
            double t = val[p];
            for (int k = 0; k < nmodes; ++k)
                if (k != mode) t *= factors[k][(size_t)idx[k][p] * R + r];
            row[r] += t;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SpTTMc along `mode` (Eq. 4, Table I row 3): the tensor times a matrix on  */
/* every other mode, written per nonzero as the row-vector Kronecker product */
/*   Y_(mode)(i_mode, :) += val * (U_a(i_a, :) (x) U_b(i_b, :) (x) ...)      */
/* over the product modes a < b < ... in ascending mode order, all of rank R. */
/* Output column c = (((r_a * R) + r_b) * R + ...) (the first product mode    */
/* varies slowest); out is dims[mode] x R^(nmodes-1), row-major.             */
/* ------------------------------------------------------------------------ */
int orc_ttmc(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
             const double *val, const double *const *factors, int R, int mode, double *out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (mode < 0 || mode >= nmodes || R <= 0 || !out || nmodes < 2) return ORC_ERR_ARG;
    int64_t width = 1;
    for (int k = 0; k < nmodes - 1; ++k) width *= R;
    memset(out, 0, sizeof(double) * (size_t)dims[mode] * (size_t)width);
    int rr[ORC_MAX_MODES];
    for (int64_t p = 0; p < nnz; ++p) {
        double *row = out + (size_t)idx[mode][p] * (size_t)width;
        for (int64_t c = 0; c < width; ++c) {
            /* digits of c in base R, most significant first = first product mode */
            int64_t q = c;
            for (int t = nmodes - 2; t >= 0; --t) {
                rr[t] = (int)(q % R);
                q /= R;
            }
            double v = val[p];
            int t = 0;
            for (int k = 0; k < nmodes; ++k)
                if (k != mode) v *= factors[k][(size_t)idx[k][p] * R + rr[t++]];
            row[c] += v;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Lexicographic comparison of two nonzeros over a list of modes.            */
/* The sort below is a library primitive used only to enumerate the          */
/* distinct index tuples of the semi-sparse output (Sec. II, Eq. 3) and the  */
/* mode-sorted order that F-COO is defined over (Sec. IV-B).                  */
/* ------------------------------------------------------------------------ */
static const uint32_t *const *g_cmp_idx;
static const int *g_cmp_modes;
static int g_cmp_nm;

static int cmp_by_modes(const void *a, const void *b)
{
    int64_t pa = *(const int64_t *)a, pb = *(const int64_t *)b;
    for (int q = 0; q < g_cmp_nm; ++q) {
        uint32_t ia = g_cmp_idx[g_cmp_modes[q]][pa], ib = g_cmp_idx[g_cmp_modes[q]][pb];
        if (ia != ib) return ia < ib ? -1 : 1;
    }
    return (pa > pb) - (pa < pb);
}

static void sort_by_modes(int64_t *perm, int64_t nnz, const uint32_t *const *idx, const int *modes, int nm)
{
    for (int64_t p = 0; p < nnz; ++p) perm[p] = p;
    g_cmp_idx = idx;
    g_cmp_modes = modes;
    g_cmp_nm = nm;
    qsort(perm, (size_t)nnz, sizeof(int64_t), cmp_by_modes);
}

static int same_on_modes(const uint32_t *const *idx, const int *modes, int nm, int64_t a, int64_t b)
{
    for (int q = 0; q < nm; ++q)
        if (idx[modes[q]][a] != idx[modes[q]][b]) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* SpTTM on mode n, Eq. 3 and Table I row 1:                                 */
/*   Y(i,j,:) += X(i,j,k) * U(k,:)                                            */
/* The result is semi-sparse: one dense length-R fibre per distinct tuple of */
/* the index modes (all modes but n, ascending).  Fibres are returned in     */
/* lexicographic order of that tuple: keys_out is nfib x (nmodes-1), out is  */
/* nfib x R.  Both need capacity for nnz fibres.  Returns nfib (>= 0) or a   */
/* negative error code.                                                       */
/* ------------------------------------------------------------------------ */
int64_t orc_ttm(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                const double *val, const double *U, int R, int mode, uint32_t *keys_out, double *out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (mode < 0 || mode >= nmodes || R <= 0 || nmodes < 2) return ORC_ERR_ARG;
    int imodes[ORC_MAX_MODES], ni = 0;
    for (int k = 0; k < nmodes; ++k)
        if (k != mode) imodes[ni++] = k;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!perm) return ORC_ERR_NOMEM;
    sort_by_modes(perm, nnz, idx, imodes, ni);
    int64_t nfib = 0;
    for (int64_t q = 0; q < nnz; ++q) {
        int64_t p = perm[q];
        if (q == 0 || !same_on_modes(idx, imodes, ni, p, perm[q - 1])) {
            for (int t = 0; t < ni; ++t) keys_out[(size_t)nfib * ni + t] = idx[imodes[t]][p];
            memset(out + (size_t)nfib * R, 0, sizeof(double) * (size_t)R);
            ++nfib;
        }
        double *y = out + (size_t)(nfib - 1) * R;
        const double *u = U + (size_t)idx[mode][p] * R;
        for (int r = 0; r < R; ++r) y[r] += val[p] * u[r];
    }
    free(perm);
    return nfib;
}

/* ------------------------------------------------------------------------ */
/* F-COO layout, Sec. IV-B, Table I, Table II and the Fig. 2 caption.        */
/*  - Table I: for SpMTTKRP on mode n the index mode is n and every other    */
/*    mode is a product mode; for SpTTM on mode n the product mode is n and  */
/*    every other mode is an index mode.                                      */
/*  - Nonzeros are ordered lexicographically by (index modes ascending, then  */
/*    product modes ascending).                                              */
/*  - head[p] = 1 iff nonzero p starts a new index-mode tuple (a new slice    */
/*    for SpMTTKRP, a new fibre for SpTTM).  The paper's bit-flag toggles at  */
/*    exactly these positions.                                                */
/*  - sf[t] = 1 iff partition t (nonzeros t*threadlen .. t*threadlen+tl-1)    */
/*    starts a new index-mode tuple; sf[0] = 1.                               */
/*  - segkeys: the index-mode tuple of each segment, in segment order.        */
/* perm_out[q] = original position of the q-th nonzero in F-COO order.       */
/* Returns ORC_ERR_DUP if two nonzeros share all coordinates.                 */
/* ------------------------------------------------------------------------ */
int orc_fcoo_layout(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                    int mode, int op, int threadlen, int64_t *perm_out, uint8_t *head_out,
                    uint8_t *sf_out, uint32_t *segkeys_out, int64_t *nseg_out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (mode < 0 || mode >= nmodes || (op != 0 && op != 1) || threadlen <= 0) return ORC_ERR_ARG;
    int order[ORC_MAX_MODES], nidx = 0;
    if (op == 0) {
        order[nidx++] = mode; /* SpMTTKRP: index mode first */
        for (int k = 0; k < nmodes; ++k)
            if (k != mode) order[k < mode ? k + 1 : k] = k;
    } else {
        for (int k = 0; k < nmodes; ++k)
            if (k != mode) order[nidx++] = k; /* SpTTM: index modes */
        order[nmodes - 1] = mode;
    }
    sort_by_modes(perm_out, nnz, idx, order, nmodes);
    int64_t nseg = 0;
    for (int64_t q = 0; q < nnz; ++q) {
        int64_t p = perm_out[q];
        if (q > 0 && same_on_modes(idx, order, nmodes, p, perm_out[q - 1])) return ORC_ERR_DUP;
        int h = (q == 0) || !same_on_modes(idx, order, nidx, p, perm_out[q - 1]);
        head_out[q] = (uint8_t)h;
        if (h) {
            for (int t = 0; t < nidx; ++t) segkeys_out[(size_t)nseg * nidx + t] = idx[order[t]][p];
            ++nseg;
        }
    }
    int64_t npart = (nnz + threadlen - 1) / threadlen;
    for (int64_t t = 0; t < npart; ++t) sf_out[t] = head_out[t * threadlen];
    *nseg_out = nseg;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers for Algorithm 1 (CP-ALS).                                    */
/* ------------------------------------------------------------------------ */

/* Gram matrix G = F^T F of an I x R row-major matrix. */
void orc_gram(const double *F, int64_t I, int R, double *G)
{
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < I; ++i) s += F[(size_t)i * R + a] * F[(size_t)i * R + b];
            G[a * R + b] = s;
        }
}

/* Cyclic Jacobi eigendecomposition of a symmetric R x R matrix A (Golub and
 * Van Loan, Sec. 8.5): A = Q diag(w) Q^T.  A is destroyed. */
static void jacobi_eig(double *A, int R, double *w, double *Q)
{
    for (int i = 0; i < R; ++i)
        for (int j = 0; j < R; ++j) Q[i * R + j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < R; ++i)
            for (int j = 0; j < R; ++j) {
                tot += A[i * R + j] * A[i * R + j];
                if (i != j) off += A[i * R + j] * A[i * R + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < R - 1; ++p)
            for (int q = p + 1; q < R; ++q) {
                double apq = A[p * R + q];
                if (apq == 0.0) continue;
                double theta = (A[q * R + q] - A[p * R + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < R; ++k) { /* A <- A J (columns p, q) */
                    double akp = A[k * R + p], akq = A[k * R + q];
                    A[k * R + p] = c * akp - s * akq;
                    A[k * R + q] = s * akp + c * akq;
                }
                for (int k = 0; k < R; ++k) { /* A <- J^T A (rows p, q) */
                    double apk = A[p * R + k], aqk = A[q * R + k];
                    A[p * R + k] = c * apk - s * aqk;
                    A[q * R + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < R; ++k) { /* Q <- Q J */
                    double qkp = Q[k * R + p], qkq = Q[k * R + q];
                    Q[k * R + p] = c * qkp - s * qkq;
                    Q[k * R + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < R; ++i) w[i] = A[i * R + i];
}

/* Solve X V = M for X (rows of M independently), V symmetric R x R, i.e.
 * X = M V^dagger as in Algorithm 1.  Reading of the pseudo-inverse: FP64
 * Cholesky V = L L^T; if a pivot is <= 1e-12 * max diag(V) the matrix is
 * treated as singular and the Moore-Penrose pseudo-inverse is formed from the
 * symmetric eigendecomposition, dropping eigenvalues <= 1e-12 * max |eig|.
 * Returns 0 when Cholesky was used, 1 when the pseudo-inverse was used. */
int orc_spd_solve(const double *V, int R, const double *M, int64_t I, double *X)
{
    double *L = (double *)calloc((size_t)R * R, sizeof(double));
    double dmax = 0.0;
    for (int i = 0; i < R; ++i) dmax = fmax(dmax, V[i * R + i]);
    int ok = dmax > 0.0;
    for (int j = 0; j < R && ok; ++j) {
        double d = V[j * R + j];
        for (int k = 0; k < j; ++k) d -= L[j * R + k] * L[j * R + k];
        if (d <= 1e-12 * dmax) { ok = 0; break; }
        L[j * R + j] = sqrt(d);
        for (int i = j + 1; i < R; ++i) {
            double s = V[i * R + j];
            for (int k = 0; k < j; ++k) s -= L[i * R + k] * L[j * R + k];
            L[i * R + j] = s / L[j * R + j];
        }
    }
    if (ok) {
        double *y = (double *)malloc(sizeof(double) * (size_t)R);
        for (int64_t i = 0; i < I; ++i) {
            const double *m = M + (size_t)i * R;
            double *x = X + (size_t)i * R;
            for (int a = 0; a < R; ++a) { /* L y = m */
                double s = m[a];
                for (int k = 0; k < a; ++k) s -= L[a * R + k] * y[k];
                y[a] = s / L[a * R + a];
            }
            for (int a = R - 1; a >= 0; --a) { /* L^T x = y */
                double s = y[a];
                for (int k = a + 1; k < R; ++k) s -= L[k * R + a] * x[k];
                x[a] = s / L[a * R + a];
            }
        }
        free(y);
        free(L);
        return 0;
    }
    free(L);
    double *A = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *Q = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *w = (double *)malloc(sizeof(double) * (size_t)R);
    double *P = (double *)calloc((size_t)R * R, sizeof(double));
    memcpy(A, V, sizeof(double) * (size_t)R * R);
    jacobi_eig(A, R, w, Q);
    double wmax = 0.0;
    for (int i = 0; i < R; ++i) wmax = fmax(wmax, fabs(w[i]));
    for (int e = 0; e < R; ++e) {
        if (fabs(w[e]) <= 1e-12 * wmax || w[e] == 0.0) continue;
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) P[a * R + b] += Q[a * R + e] * Q[b * R + e] / w[e];
    }
    for (int64_t i = 0; i < I; ++i)
        for (int b = 0; b < R; ++b) {
            double s = 0.0;
            for (int a = 0; a < R; ++a) s += M[(size_t)i * R + a] * P[a * R + b];
            X[(size_t)i * R + b] = s;
        }
    free(A);
    free(Q);
    free(w);
    free(P);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* CP-ALS, Algorithm 1, generalised to N modes.  One call runs `iters` full   */
/* sweeps.  For each mode n in order:                                         */
/*   V   = Hadamard product over k != n of F_k^T F_k                          */
/*   F_n = MTTKRP_n(X, F) * V^dagger                                          */
/*   normalise the columns of F_n by their 2-norms; the norms of the last     */
/*   mode are kept as lambda (a column of norm 0 gets lambda 0 and is left    */
/*   as it is).                                                               */
/* After each sweep the fit is computed as                                    */
/*   fit = 1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2 <X, Xhat>)) / |X|             */
/*   |Xhat|^2 = lambda^T (Hadamard_k F_k^T F_k) lambda                        */
/*   <X, Xhat> = sum_r lambda_r sum_i M_last(i,r) F_last(i,r)                 */
/* with M_last the last mode's MTTKRP of this sweep.                          */
/* factors[k] (dims[k] x R) hold the initial factors on entry and the final   */
/* ones on exit; lambda gets R values; fit_out gets `iters` values;          */
/* npinv_out (may be NULL) counts solves that needed the pseudo-inverse.      */
/* ------------------------------------------------------------------------ */
int orc_cp_als(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
               const double *val, int R, int iters, double *const *factors, double *lambda,
               double *fit_out, int *npinv_out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (R <= 0 || iters < 0 || nmodes < 2) return ORC_ERR_ARG;
    uint32_t Imax = 0;
    for (int k = 0; k < nmodes; ++k) Imax = dims[k] > Imax ? dims[k] : Imax;
    double *M = (double *)malloc(sizeof(double) * (size_t)Imax * R);
    double *V = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *G = (double *)malloc(sizeof(double) * (size_t)R * R);
    double normX2 = 0.0;
    for (int64_t p = 0; p < nnz; ++p) normX2 += val[p] * val[p];
    int npinv = 0;
    for (int r = 0; r < R; ++r) lambda[r] = 1.0;
    for (int it = 0; it < iters; ++it) {
        for (int n = 0; n < nmodes; ++n) {
            orc_mttkrp(nmodes, dims, nnz, idx, val, (const double *const *)factors, R, n, M);
            for (int a = 0; a < R * R; ++a) V[a] = 1.0;
            for (int k = 0; k < nmodes; ++k) {
                if (k == n) continue;
                orc_gram(factors[k], dims[k], R, G);
                for (int a = 0; a < R * R; ++a) V[a] *= G[a];
            }
            npinv += orc_spd_solve(V, R, M, dims[n], factors[n]);
            for (int r = 0; r < R; ++r) {
                double s = 0.0;
                for (uint32_t i = 0; i < dims[n]; ++i) s += factors[n][(size_t)i * R + r] * factors[n][(size_t)i * R + r];
                double nr = sqrt(s);
                lambda[r] = nr;
                if (nr > 0.0)
                    for (uint32_t i = 0; i < dims[n]; ++i) factors[n][(size_t)i * R + r] /= nr;
            }
        }
        /* fit after the sweep; M holds the last mode's MTTKRP */
        int last = nmodes - 1;
        for (int a = 0; a < R * R; ++a) V[a] = 1.0;
        for (int k = 0; k < nmodes; ++k) {
            orc_gram(factors[k], dims[k], R, G);
            for (int a = 0; a < R * R; ++a) V[a] *= G[a];
        }
        double xhat2 = 0.0, inner = 0.0;
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) xhat2 += lambda[a] * V[a * R + b] * lambda[b];
        for (int r = 0; r < R; ++r) {
            double s = 0.0;
            for (uint32_t i = 0; i < dims[last]; ++i) s += M[(size_t)i * R + r] * factors[last][(size_t)i * R + r];
            inner += lambda[r] * s;
        }
        double resid2 = normX2 + xhat2 - 2.0 * inner;
        fit_out[it] = 1.0 - sqrt(resid2 > 0.0 ? resid2 : 0.0) / sqrt(normX2);
    }
    if (npinv_out) *npinv_out = npinv;
    free(M);
    free(V);
    free(G);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse CP fit over the observed entries (the differentiable extension of */
/* the one-shot product of Eq. 6):                                           */
/*   model(p) = sum_r prod_k F_k[idx_k(p)][r],  e(p) = model(p) - val(p)      */
/*   loss     = 1/2 sum_p e(p)^2                                              */
/*   dF_n[i][r] = sum_{p: idx_n(p) = i} e(p) prod_{k != n} F_k[idx_k(p)][r]   */
/*   dval(p)  = -e(p)                                                          */
/* dfactors[k] (dims[k] x R) and dvals (nnz) are overwritten; either may be   */
/* NULL to skip it.                                                           */
/* ------------------------------------------------------------------------ */
int orc_sparse_fit(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                   const double *val, const double *const *factors, int R, double *loss,
                   double *const *dfactors, double *dvals)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (R <= 0) return ORC_ERR_ARG;
    if (dfactors)
        for (int k = 0; k < nmodes; ++k)
            if (dfactors[k]) memset(dfactors[k], 0, sizeof(double) * (size_t)dims[k] * R);
    double L = 0.0;
    for (int64_t p = 0; p < nnz; ++p) {
        double model = 0.0;
        for (int r = 0; r < R; ++r) {
            double t = 1.0;
            for (int k = 0; k < nmodes; ++k) t *= factors[k][(size_t)idx[k][p] * R + r];
            model += t;
        }
        double e = model - val[p];
        L += 0.5 * e * e;
        if (dvals) dvals[p] = -e;
        if (!dfactors) continue;
        for (int n = 0; n < nmodes; ++n) {
            if (!dfactors[n]) continue;
            for (int r = 0; r < R; ++r) {
                double t = e;
                for (int k = 0; k < nmodes; ++k)
                    if (k != n) t *= factors[k][(size_t)idx[k][p] * R + r];
                dfactors[n][(size_t)idx[n][p] * R + r] += t;
            }
        }
    }
    *loss = L;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of M = SpMTTKRP_n(X, F) (Eq. 6) for a given G = dL/dM              */
/* (dims[mode] x R):                                                          */
/*   dF_k[idx_k(p)][r] += val(p) G[idx_n(p)][r] prod_{m != n,k} F_m[.][r]     */
/*   dval(p) = sum_r G[idx_n(p)][r] prod_{k != n} F_k[idx_k(p)][r]            */
/* dfactors[mode] is not written; other entries may be NULL to skip them.    */
/* ------------------------------------------------------------------------ */
int orc_mttkrp_adjoint(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                       const double *val, const double *const *factors, int R, int mode,
                       const double *G, double *const *dfactors, double *dvals)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (mode < 0 || mode >= nmodes || R <= 0) return ORC_ERR_ARG;
    if (dfactors)
        for (int k = 0; k < nmodes; ++k)
            if (k != mode && dfactors[k]) memset(dfactors[k], 0, sizeof(double) * (size_t)dims[k] * R);
    for (int64_t p = 0; p < nnz; ++p) {
        const double *g = G + (size_t)idx[mode][p] * R;
        if (dvals) {
            double s = 0.0;
            for (int r = 0; r < R; ++r) {
                double t = g[r];
                for (int k = 0; k < nmodes; ++k)
                    if (k != mode) t *= factors[k][(size_t)idx[k][p] * R + r];
                s += t;
            }
            dvals[p] = s;
        }
        if (!dfactors) continue;
        for (int k = 0; k < nmodes; ++k) {
            if (k == mode || !dfactors[k]) continue;
            for (int r = 0; r < R; ++r) {
                double t = val[p] * g[r];
                for (int m = 0; m < nmodes; ++m)
                    if (m != mode && m != k) t *= factors[m][(size_t)idx[m][p] * R + r];
                dfactors[k][(size_t)idx[k][p] * R + r] += t;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 split into its steps, for checking a device path that rounds  */
/* the factors between steps.                                                 */
/* One mode update of the loop body, for mode n:                             */
/*   V = Hadamard_{k != n} F_k^T F_k;  F_n = MTTKRP_n(X, F) V^dagger;         */
/*   lambda = column 2-norms of F_n; F_n columns divided by them.            */
/* M_out (may be NULL) receives the MTTKRP.  Returns 1 if the                 */
/* pseudo-inverse was used, 0 for Cholesky, < 0 on error.                     */
/* ------------------------------------------------------------------------ */
int orc_cp_als_mode(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx,
                    const double *val, int R, int n, double *const *factors, double *lambda, double *M_out)
{
    int st = check_coo(nmodes, dims, nnz, idx);
    if (st) return st;
    if (R <= 0 || n < 0 || n >= nmodes) return ORC_ERR_ARG;
    double *M = (double *)malloc(sizeof(double) * (size_t)dims[n] * R);
    double *V = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *G = (double *)malloc(sizeof(double) * (size_t)R * R);
    orc_mttkrp(nmodes, dims, nnz, idx, val, (const double *const *)factors, R, n, M);
    for (int a = 0; a < R * R; ++a) V[a] = 1.0;
    for (int k = 0; k < nmodes; ++k) {
        if (k == n) continue;
        orc_gram(factors[k], dims[k], R, G);
        for (int a = 0; a < R * R; ++a) V[a] *= G[a];
    }
    int used = orc_spd_solve(V, R, M, dims[n], factors[n]);
    for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (uint32_t i = 0; i < dims[n]; ++i) s += factors[n][(size_t)i * R + r] * factors[n][(size_t)i * R + r];
        double nr = sqrt(s);
        lambda[r] = nr;
        if (nr > 0.0)
            for (uint32_t i = 0; i < dims[n]; ++i) factors[n][(size_t)i * R + r] /= nr;
    }
    if (M_out) memcpy(M_out, M, sizeof(double) * (size_t)dims[n] * R);
    free(M);
    free(V);
    free(G);
    return used;
}

/* The fit of Algorithm 1's model [lambda; F_0..F_{N-1}] against X, from the  */
/* definition 1 - |X - Xhat| / |X| with                                       */
/* |X - Xhat|^2 = |X|^2 + lambda^T (Hadamard_k F_k^T F_k) lambda              */
/*                - 2 sum_r lambda_r sum_i M_last(i,r) F_last(i,r),           */
/* M_last = MTTKRP of the last mode with the given factors.                   */
double orc_cp_fit(int nmodes, const uint32_t *dims, int64_t nnz, const uint32_t *const *idx, const double *val,
                  int R, const double *const *factors, const double *lambda)
{
    int last = nmodes - 1;
    double *M = (double *)malloc(sizeof(double) * (size_t)dims[last] * R);
    double *V = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *G = (double *)malloc(sizeof(double) * (size_t)R * R);
    orc_mttkrp(nmodes, dims, nnz, idx, val, factors, R, last, M);
    double normX2 = 0.0, xhat2 = 0.0, inner = 0.0;
    for (int64_t p = 0; p < nnz; ++p) normX2 += val[p] * val[p];
    for (int a = 0; a < R * R; ++a) V[a] = 1.0;
    for (int k = 0; k < nmodes; ++k) {
        orc_gram(factors[k], dims[k], R, G);
        for (int a = 0; a < R * R; ++a) V[a] *= G[a];
    }
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) xhat2 += lambda[a] * V[a * R + b] * lambda[b];
    for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (uint32_t i = 0; i < dims[last]; ++i) s += M[(size_t)i * R + r] * factors[last][(size_t)i * R + r];
        inner += lambda[r] * s;
    }
    double resid2 = normX2 + xhat2 - 2.0 * inner;
    free(M);
    free(V);
    free(G);
    return 1.0 - sqrt(resid2 > 0.0 ? resid2 : 0.0) / sqrt(normX2);
}
