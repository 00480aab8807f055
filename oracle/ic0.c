/* Oracle incomplete Cholesky IC(0) on CSR (test infrastructure; plain C, FP64).
 *
 * IC(0) (Section 5 remark: "incomplete Cholesky IC0", after Saad): a lower-triangular L with the
 * sparsity pattern of the lower triangle of A such that (L L^T)_ij = A_ij for every (i, j) in
 * that pattern. Computed row by row: for each stored j < i in ascending order,
 *     L_ij = (A_ij - sum_{k < j} L_ik L_jk) / L_jj,
 * then L_ii = sqrt(A_ii - sum_{k < i} L_ik^2), the sums running over k stored in both rows.
 *
 * Input: the lower triangle (diagonal included) in CSR with ascending column indices, so the
 * diagonal is the last entry of each row. The matrix is already in the elimination order the
 * caller wants (natural or multicolour). Nothing here is shared with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* Returns 0 on success; on a non-positive pivot returns -(row + 1). */
int oracle_ic0_factor(int64_t n, const int64_t* indptr, const int32_t* indices,
                      const double* a, double* L) {
  int64_t* pos = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!pos) return -(int)(n + 1);
  for (int64_t k = 0; k < n; ++k) pos[k] = -1;
  int status = 0;
  for (int64_t i = 0; i < n && status == 0; ++i) {
    const int64_t b = indptr[i], e = indptr[i + 1];
    for (int64_t p = b; p < e; ++p) pos[indices[p]] = p;
    double diag_sum = 0.0;
    for (int64_t p = b; p < e - 1; ++p) {        /* off-diagonal entries j < i */
      const int64_t j = indices[p];
      double s = a[p];
      for (int64_t q = indptr[j]; q < indptr[j + 1] - 1; ++q) {  /* k < j in row j */
        const int64_t k = indices[q];
        const int64_t pk = pos[k];
        if (pk >= 0 && pk < p) s -= L[pk] * L[q];
      }
      L[p] = s / L[indptr[j + 1] - 1];
      diag_sum += L[p] * L[p];
    }
    const double d = a[e - 1] - diag_sum;
    if (!(d > 0.0)) status = -(int)(i + 1);
    else L[e - 1] = sqrt(d);
    for (int64_t p = b; p < e; ++p) pos[indices[p]] = -1;
  }
  free(pos);
  return status;
}

/* z = (L L^T)^{-1} r: forward sweep L y = r, then backward sweep L^T z = y. */
void oracle_ic0_solve(int64_t n, const int64_t* indptr, const int32_t* indices, const double* L,
                      const double* r, double* z) {
  for (int64_t i = 0; i < n; ++i) {
    double s = r[i];
    const int64_t e = indptr[i + 1] - 1;
    for (int64_t p = indptr[i]; p < e; ++p) s -= L[p] * z[indices[p]];
    z[i] = s / L[e];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t e = indptr[i + 1] - 1;
    const double zi = z[i] / L[e];
    z[i] = zi;
    for (int64_t p = indptr[i]; p < e; ++p) z[indices[p]] -= L[p] * zi;
  }
}
