/*
 * fcoo_oracle_omp.c -- multi-threaded build of the oracle's SpMTTKRP loop
 * (Eq. 5 / Eq. 6, Table I row 2), for the CPU baseline and for oracle runs
 * too large for one core (20 CP-ALS sweeps on the 76M-nonzero tensor).
 *
 * TEST INFRASTRUCTURE ONLY, like fcoo_oracle.c: only tests/ and bench.py's
 * CPU-baseline leg use it; the product library never links or calls it and
 * shares no code with it.
 *
 * The arithmetic is the oracle's, term for term:
 *   out[idx_n(p)][r] += val(p) * prod_{k != n} F_k[idx_k(p)][r]
 * The only change is who adds which terms: the nonzeros are grouped by their
 * index in `mode` (a stable counting sort, so each row keeps the nonzeros in
 * their input order) and every output row is summed by one thread.  Each row
 * therefore adds the same terms in the same order as the single-threaded
 * loop, and the FP64 result is bitwise equal to orc_mttkrp (tested).  An FP32
 * variant (FP32 values, factors and sums) gives the FP32 CPU baseline.
 * Built with gcc -O3 -fopenmp.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORP_OK = 0, ORP_ERR_ARG = -1, ORP_ERR_RANGE = -2, ORP_ERR_NOMEM = -4 };

int orp_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Group the nonzeros by idx_mode: rowptr (dim + 1 entries) and order (nnz
 * entries) such that order[rowptr[i] .. rowptr[i+1]) lists the nonzeros with
 * index i in increasing position.  Returns ORP_ERR_RANGE for an index >= dim. */
int orp_mode_rows(int64_t nnz, const uint32_t *idx_mode, uint32_t dim, int64_t *rowptr, int64_t *order)
{
    if (nnz < 0 || !rowptr || (nnz > 0 && (!idx_mode || !order))) return ORP_ERR_ARG;
    memset(rowptr, 0, sizeof(int64_t) * ((size_t)dim + 1));
    for (int64_t p = 0; p < nnz; ++p) {
        if (idx_mode[p] >= dim) return ORP_ERR_RANGE;
        rowptr[idx_mode[p] + 1]++;
    }
    for (uint32_t i = 0; i < dim; ++i) rowptr[i + 1] += rowptr[i];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * ((size_t)dim + 1));
    if (!next) return ORP_ERR_NOMEM;
    memcpy(next, rowptr, sizeof(int64_t) * ((size_t)dim + 1));
    for (int64_t p = 0; p < nnz; ++p) order[next[idx_mode[p]]++] = p;
    free(next);
    return ORP_OK;
}

/* FP64: out (dims[mode] x R, row-major) fully overwritten. */
int orp_mttkrp_f64(int nmodes, const uint32_t *dims, const uint32_t *const *idx, const double *val,
                   const double *const *factors, int R, int mode, const int64_t *rowptr, const int64_t *order,
                   double *out)
{
    if (nmodes < 2 || mode < 0 || mode >= nmodes || R <= 0 || !out || !rowptr) return ORP_ERR_ARG;
    const int64_t rows = dims[mode];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < rows; ++i) {
        double *row = out + (size_t)i * R;
        for (int r = 0; r < R; ++r) row[r] = 0.0;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            const int64_t p = order[q];
            for (int r = 0; r < R; ++r) {
                double t = val[p];
                for (int k = 0; k < nmodes; ++k)
                    if (k != mode) t *= factors[k][(size_t)idx[k][p] * R + r];
                row[r] += t;
            }
        }
    }
    return ORP_OK;
}

/* FP32 values, factors and sums; otherwise as orp_mttkrp_f64. */
int orp_mttkrp_f32(int nmodes, const uint32_t *dims, const uint32_t *const *idx, const float *val,
                   const float *const *factors, int R, int mode, const int64_t *rowptr, const int64_t *order,
                   float *out)
{
    if (nmodes < 2 || mode < 0 || mode >= nmodes || R <= 0 || !out || !rowptr) return ORP_ERR_ARG;
    const int64_t rows = dims[mode];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < rows; ++i) {
        float *row = out + (size_t)i * R;
        for (int r = 0; r < R; ++r) row[r] = 0.0f;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            const int64_t p = order[q];
            for (int r = 0; r < R; ++r) {
                float t = val[p];
                for (int k = 0; k < nmodes; ++k)
                    if (k != mode) t *= factors[k][(size_t)idx[k][p] * R + r];
                row[r] += t;
            }
        }
    }
    return ORP_OK;
}
