/*
 * krylov.c - plain FP64 iterative solve of a sparse system, for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/iterative.py, which only tests/,
 * the smoke check and the CPU-baseline legs of bench.py call.  It shares no
 * code with the CUDA library.
 *
 * The oracle needs the exact solution of the linearised system J d = -R of
 * the paper's Newton iteration (Sec. 3, the system after Eq.
 * fully-coupled-fully-discrete) at sizes where a sparse direct LU runs out of
 * memory.  These routines are the textbook definitions, single-threaded and
 * unblocked, on a CSR matrix whose rows hold sorted column indices and a
 * diagonal entry:
 *   - scalar ILU(0): incomplete LU with the sparsity pattern of the matrix,
 *     in the row-by-row (IKJ) form: for each row i, each earlier column k of
 *     the row is divided by the pivot u_kk and its multiple of row k of U is
 *     subtracted from the entries of row i that exist in the pattern;
 *   - restarted GMRES(m), right preconditioned by that ILU(0), with the
 *     modified Gram-Schmidt Arnoldi process and Givens rotations on the
 *     Hessenberg matrix; the residual norm |g_{j+1}| of the rotated
 *     least-squares problem is the stopping test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* y = A x */
void oracle_csr_matvec(int64_t n, const int64_t* ptr, const int32_t* col, const double* a, const double* x,
                       double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) s += a[p] * x[col[p]];
    y[i] = s;
  }
}

/* ILU(0) of A into lu (same pattern; L unit lower, stored below the
 * diagonal, U on and above it).  diag[i] receives the position of a_ii.
 * Returns 0, or -(i+1) if row i has no diagonal entry or a zero pivot. */
int64_t oracle_ilu0(int64_t n, const int64_t* ptr, const int32_t* col, const double* a, double* lu, int64_t* diag) {
  int64_t* pos = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!pos) return -(n + 1);
  for (int64_t i = 0; i < n; ++i) pos[i] = -1;
  memcpy(lu, a, (size_t)ptr[n] * sizeof(double));
  int64_t status = 0;
  for (int64_t i = 0; i < n && status == 0; ++i) {
    diag[i] = -1;
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
      pos[col[p]] = p;
      if (col[p] == i) diag[i] = p;
    }
    if (diag[i] < 0) {
      status = -(i + 1);
    } else {
      for (int64_t p = ptr[i]; p < diag[i]; ++p) {
        const int64_t k = col[p];
        const double lik = lu[p] / lu[diag[k]];
        lu[p] = lik;
        for (int64_t q = diag[k] + 1; q < ptr[k + 1]; ++q) {
          const int64_t at = pos[col[q]];
          if (at >= 0) lu[at] -= lik * lu[q];
        }
      }
      if (lu[diag[i]] == 0.0 || !isfinite(lu[diag[i]])) status = -(i + 1);
    }
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) pos[col[p]] = -1;
  }
  free(pos);
  return status;
}

/* z = U^-1 L^-1 r with the factors of oracle_ilu0 (z may alias r) */
void oracle_ilu0_solve(int64_t n, const int64_t* ptr, const int32_t* col, const double* lu, const int64_t* diag,
                       const double* r, double* z) {
  for (int64_t i = 0; i < n; ++i) {
    double s = r[i];
    for (int64_t p = ptr[i]; p < diag[i]; ++p) s -= lu[p] * z[col[p]];
    z[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = z[i];
    for (int64_t p = diag[i] + 1; p < ptr[i + 1]; ++p) s -= lu[p] * z[col[p]];
    z[i] = s / lu[diag[i]];
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Restarted GMRES(m) for A x = b, right preconditioned (A M^-1 u = b,
 * x = M^-1 u) with the ILU(0) factors, starting from the x given.  Stops when
 * the residual norm of the least-squares problem falls to tol_abs, or after
 * maxit Arnoldi steps in all.  out[0] = Arnoldi steps taken, out[1] = the
 * last least-squares residual norm.  Returns 0, or -1 if memory ran out. */
int64_t oracle_gmres(int64_t n, const int64_t* ptr, const int32_t* col, const double* a, const double* lu,
                     const int64_t* diag, const double* b, double* x, int64_t m, int64_t maxit, double tol_abs,
                     double* out) {
  double* V = (double*)malloc((size_t)(m + 1) * (size_t)n * sizeof(double));
  double* w = (double*)malloc((size_t)n * sizeof(double));
  double* z = (double*)malloc((size_t)n * sizeof(double));
  double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));  /* H[j*(m+1) + i] = h_ij */
  double* cs = (double*)malloc((size_t)m * sizeof(double));
  double* sn = (double*)malloc((size_t)m * sizeof(double));
  double* g = (double*)malloc((size_t)(m + 1) * sizeof(double));
  double* y = (double*)malloc((size_t)m * sizeof(double));
  if (!V || !w || !z || !H || !cs || !sn || !g || !y) {
    free(V); free(w); free(z); free(H); free(cs); free(sn); free(g); free(y);
    return -1;
  }
  int64_t its = 0;
  double res = 0.0;
  for (;;) {
    /* r0 = b - A x, v_1 = r0 / beta */
    oracle_csr_matvec(n, ptr, col, a, x, w);
    for (int64_t i = 0; i < n; ++i) V[i] = b[i] - w[i];
    const double beta = sqrt(dot(n, V, V));
    res = beta;
    if (beta <= tol_abs || its >= maxit || !(beta > 0.0)) break;
    for (int64_t i = 0; i < n; ++i) V[i] /= beta;
    for (int64_t i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int64_t jl = 0;
    for (int64_t j = 0; j < m && its < maxit; ++j) {
      double* hj = H + j * (m + 1);
      /* w = A M^-1 v_j */
      oracle_ilu0_solve(n, ptr, col, lu, diag, V + j * n, z);
      oracle_csr_matvec(n, ptr, col, a, z, w);
      /* modified Gram-Schmidt */
      for (int64_t i = 0; i <= j; ++i) {
        const double* vi = V + i * n;
        const double h = dot(n, w, vi);
        hj[i] = h;
        for (int64_t t = 0; t < n; ++t) w[t] -= h * vi[t];
      }
      const double hn = sqrt(dot(n, w, w));
      hj[j + 1] = hn;
      if (hn > 0.0)
        for (int64_t t = 0; t < n; ++t) V[(j + 1) * n + t] = w[t] / hn;
      /* earlier rotations on the new column, then the rotation removing h_{j+1,j} */
      for (int64_t i = 0; i < j; ++i) {
        const double p = hj[i], q = hj[i + 1];
        hj[i] = cs[i] * p + sn[i] * q;
        hj[i + 1] = -sn[i] * p + cs[i] * q;
      }
      const double den = hypot(hj[j], hj[j + 1]);
      cs[j] = den > 0.0 ? hj[j] / den : 1.0;
      sn[j] = den > 0.0 ? hj[j + 1] / den : 0.0;
      hj[j] = den;
      hj[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jl = j + 1;
      res = fabs(g[j + 1]);
      if (res <= tol_abs || !(hn > 0.0)) break;
    }
    /* y = R^-1 g, x += M^-1 V y */
    for (int64_t i = jl - 1; i >= 0; --i) {
      double s = g[i];
      for (int64_t k = i + 1; k < jl; ++k) s -= H[k * (m + 1) + i] * y[k];
      y[i] = s / H[i * (m + 1) + i];
    }
    for (int64_t t = 0; t < n; ++t) w[t] = 0.0;
    for (int64_t i = 0; i < jl; ++i)
      for (int64_t t = 0; t < n; ++t) w[t] += y[i] * V[i * n + t];
    oracle_ilu0_solve(n, ptr, col, lu, diag, w, z);
    for (int64_t t = 0; t < n; ++t) x[t] += z[t];
    if (res <= tol_abs || its >= maxit) break;
  }
  out[0] = (double)its;
  out[1] = res;
  free(V); free(w); free(z); free(H); free(cs); free(sn); free(g); free(y);
  return 0;
}
