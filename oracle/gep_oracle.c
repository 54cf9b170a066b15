/*
 * FP64 CPU oracle for the real-symmetric-definite generalized eigenproblem
 *     A y_k = lambda_k B y_k            (Imachi & Hoshi, Eq. 1; matrix form Eq. 2)
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  The GPU solver shares
 * no code, header, table or helper with it.
 *
 * Every routine is a plain, slow, textbook restatement of one step of the
 * paper's formulation (section 3.1):
 *   Eq. 4   B = U^T U (here written B = L L^T with L = U^T lower)   oc_cholesky
 *   Eq. 5   A' = U^-T A U^-1 = L^-1 A L^-T                          oc_two_sided
 *   Eq. 3   A' Z = Z Lambda by Householder tridiagonalisation
 *           ("TRD", Table 3) + implicit QL on the tridiagonal         oc_tridiag, oc_tql
 *           (the paper's D&C stage is replaced by an independent
 *            algorithm on purpose: QL with Wilkinson shifts)
 *           Sturm-sequence bisection (eigenvalue-only mode, T_evo)    oc_bisect
 *   Eq. 6   Y = U^-1 Z = L^-T Z                                      oc_backsub
 *   Eq. 2   full GEP driver, ascending order, sign convention       oc_gep_solve
 *   Eq. 7-9 Cholesky-free reducer: SEP of B, A' = D^-1/2 W^T A W D^-1/2,
 *           Y = W D^-1/2 Z                                          oc_gep_solve_eigenexa
 *   lowest n eigenpairs: bisection + inverse iteration on T          oc_gep_solve_partial
 * Independent pins that do not reuse the pipeline above:
 *   cyclic Jacobi on a small symmetric matrix                       oc_jacobi
 *   Sylvester inertia of A - sigma B (Bunch-Parlett LDL^T)          oc_inertia
 *   first-order perturbation adjoint of eigenvalue / density loss   oc_adjoint
 *
 * Storage: column-major, element (i,j) of X at X[i + j*ld]; only the lower
 * triangle of symmetric inputs is read.  All arithmetic is IEEE FP64, built with
 * -ffp-contract=off so results do not depend on FMA contraction.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static double sym_lower(const double* X, int ld, int i, int j) {
  return i >= j ? X[IX(i, j, ld)] : X[IX(j, i, ld)];
}

/* ---------------------------------------------------------------- Eq. 4 ---
 * Cholesky factorisation B = L L^T, L lower, column-oriented (left-looking).
 * Overwrites the lower triangle of B with L; the strict upper triangle is set
 * to zero.  Returns 0, or k > 0 when the leading minor of order k is not
 * positive definite (pivot <= 0 or not finite). */
int oc_cholesky(int M, double* B, int ldb) {
  for (int j = 0; j < M; ++j) {
    double s = B[IX(j, j, ldb)];
    for (int k = 0; k < j; ++k) s -= B[IX(j, k, ldb)] * B[IX(j, k, ldb)];
    if (!(s > 0.0) || !isfinite(s)) return j + 1;
    double ljj = sqrt(s);
    B[IX(j, j, ldb)] = ljj;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < M; ++i) {
      double t = B[IX(i, j, ldb)];
      for (int k = 0; k < j; ++k) t -= B[IX(i, k, ldb)] * B[IX(j, k, ldb)];
      B[IX(i, j, ldb)] = t / ljj;
    }
  }
  for (int j = 1; j < M; ++j)
    for (int i = 0; i < j; ++i) B[IX(i, j, ldb)] = 0.0;
  return 0;
}

/* ---------------------------------------------------------------- Eq. 5 ---
 * C = L^-1 A L^-T without forming L^-1: X = L^-1 A column by column (forward
 * substitution on the full symmetric A), then C = L^-1 X^T (because
 * (L^-1 A)^T = A L^-T for symmetric A), then C <- (C + C^T)/2.
 * A (lower triangle read) is overwritten by the full symmetric C. */
void oc_two_sided(int M, double* A, int lda, const double* L, int ldl) {
  double* X = (double*)malloc(sizeof(double) * (size_t)M * M);
  /* X(:,j) = L^-1 A(:,j) */
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < M; ++j) {
    double* x = X + (size_t)j * M;
    for (int i = 0; i < M; ++i) x[i] = sym_lower(A, lda, i, j);
    for (int i = 0; i < M; ++i) {
      double t = x[i];
      for (int k = 0; k < i; ++k) t -= L[IX(i, k, ldl)] * x[k];
      x[i] = t / L[IX(i, i, ldl)];
    }
  }
  /* C(:,j) = L^-1 (X^T)(:,j) = L^-1 X(j,:)^T */
  double* C = (double*)malloc(sizeof(double) * (size_t)M * M);
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < M; ++j) {
    double* c = C + (size_t)j * M;
    for (int i = 0; i < M; ++i) c[i] = X[IX(j, i, M)];
    for (int i = 0; i < M; ++i) {
      double t = c[i];
      for (int k = 0; k < i; ++k) t -= L[IX(i, k, ldl)] * c[k];
      c[i] = t / L[IX(i, i, ldl)];
    }
  }
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) A[IX(i, j, lda)] = 0.5 * (C[IX(i, j, M)] + C[IX(j, i, M)]);
  free(C);
  free(X);
}

/* ------------------------------------------------------- SEP solver, TRD ---
 * Unblocked Householder tridiagonalisation C = Q T Q^T (Golub & Van Loan,
 * symmetric tridiagonalisation).  Step k annihilates C(k+2:M, k) with
 * H_k = I - tau_k v_k v_k^T, v_k(0) = 1, and updates the trailing block two-sided
 * (C22 <- H C22 H via p = tau C22 v, w = p - (tau/2)(p.v) v, C22 -= v w^T + w v^T).
 * Reads the lower triangle of C (destroyed).  Outputs d[M], e[M-1] and, if
 * Q != NULL, the explicit orthogonal Q = H_0 H_1 ... H_{M-3}. */
void oc_tridiag(int M, double* C, int ldc, double* d, double* e, double* Q, int ldq) {
  /* work on a full symmetric copy so both triangles stay consistent */
  double* S = (double*)malloc(sizeof(double) * (size_t)M * M);
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) S[IX(i, j, M)] = sym_lower(C, ldc, i, j);
  double* V = (double*)calloc((size_t)M * (M > 0 ? M : 1), sizeof(double)); /* reflectors, column k */
  double* tau = (double*)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
  double* p = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
  for (int k = 0; k + 2 < M; ++k) {
    int n = M - k - 1; /* length of x = S(k+1:M, k) */
    double* x = S + IX(k + 1, k, M);
    double sig = 0.0;
    for (int i = 1; i < n; ++i) sig += x[i] * x[i];
    double* v = V + IX(k + 1, k, M);
    if (sig == 0.0) { /* already zero below the subdiagonal: H_k = I */
      tau[k] = 0.0;
      for (int i = 0; i < n; ++i) v[i] = (i == 0) ? 1.0 : 0.0;
      continue;
    }
    double alpha = x[0];
    double nrm = sqrt(alpha * alpha + sig);
    double beta = alpha >= 0.0 ? -nrm : nrm;  /* H x = beta e_1 */
    tau[k] = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    v[0] = 1.0;
    for (int i = 1; i < n; ++i) v[i] = x[i] * scal;
    /* two-sided update of the trailing block S22 = S(k+1:M, k+1:M) */
    double t = tau[k];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += S[IX(k + 1 + i, k + 1 + j, M)] * v[j];
      p[i] = t * s;
    }
    double pv = 0.0;
    for (int i = 0; i < n; ++i) pv += p[i] * v[i];
    double half = 0.5 * t * pv;
    for (int i = 0; i < n; ++i) p[i] -= half * v[i]; /* p now holds w */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        S[IX(k + 1 + i, k + 1 + j, M)] -= v[i] * p[j] + p[i] * v[j];
    /* column k after the reflection: beta on the subdiagonal, zeros below */
    S[IX(k + 1, k, M)] = beta;
    S[IX(k, k + 1, M)] = beta;
    for (int i = 1; i < n; ++i) { S[IX(k + 1 + i, k, M)] = 0.0; S[IX(k, k + 1 + i, M)] = 0.0; }
  }
  for (int i = 0; i < M; ++i) d[i] = S[IX(i, i, M)];
  for (int i = 0; i + 1 < M; ++i) e[i] = S[IX(i + 1, i, M)];
  if (Q) {
    /* Q = H_0 H_1 ... H_{M-3}: start from I and apply the reflectors from the
     * last to the first on the left, Q <- H_k Q. */
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) Q[IX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
    for (int k = M - 3; k >= 0; --k) {
      if (tau[k] == 0.0) continue;
      int n = M - k - 1;
      const double* v = V + IX(k + 1, k, M);
#pragma omp parallel for schedule(static)
      for (int j = 0; j < M; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += v[i] * Q[IX(k + 1 + i, j, ldq)];
        s *= tau[k];
        for (int i = 0; i < n; ++i) Q[IX(k + 1 + i, j, ldq)] -= s * v[i];
      }
    }
  }
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) C[IX(i, j, ldc)] = S[IX(i, j, M)];
  free(p);
  free(tau);
  free(V);
  free(S);
}

/* ------------------------------------------- tridiagonal eigensolver (QL) ---
 * Implicit QL iteration with Wilkinson-type shift on the symmetric tridiagonal
 * (d, e): d[0..M-1] diagonal, e[0..M-2] off-diagonal (e[i] couples i and i+1).
 * On return d holds the eigenvalues (unsorted) and, if Z != NULL, the columns
 * of Z are post-multiplied by the accumulated rotations (Z <- Z G), so a Z that
 * held Q on entry ends as Q Z_T.  Returns 0, or l+1 if eigenvalue l failed to
 * converge in 60 iterations.  e is destroyed. */
int oc_tql(int M, double* d, double* e_in, double* Z, int ldz) {
  if (M <= 0) return 0;
  double* e = (double*)calloc((size_t)M, sizeof(double));
  for (int i = 0; i + 1 < M; ++i) e[i] = e_in[i];
  double* cs = (double*)malloc(sizeof(double) * (size_t)M);
  double* sn = (double*)malloc(sizeof(double) * (size_t)M);
  const double eps = 0x1p-52;
  int status = 0;
  for (int l = 0; l < M; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m + 1 < M; ++m) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) { status = l + 1; goto done; }
      /* shift from the leading 2x2 block at l (eigenvalue of it closer to d[l]) */
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i, nrot = 0, early = 0;
      for (i = m - 1; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) { /* underflow: the bulge vanished, deflate here */
          d[i + 1] -= p;
          e[m] = 0.0;
          early = 1;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        cs[nrot] = c;
        sn[nrot] = s;
        ++nrot;
      }
      if (Z && nrot > 0) {
        /* apply the rotations of this sweep (columns m-1..l, in order) row by row */
        int i0 = m - 1;
#pragma omp parallel for schedule(static)
        for (int row = 0; row < M; ++row) {
          for (int q = 0; q < nrot; ++q) {
            int col = i0 - q;
            double zi = Z[IX(row, col, ldz)], zi1 = Z[IX(row, col + 1, ldz)];
            Z[IX(row, col + 1, ldz)] = sn[q] * zi + cs[q] * zi1;
            Z[IX(row, col, ldz)] = cs[q] * zi - sn[q] * zi1;
          }
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
done:
  free(sn);
  free(cs);
  free(e);
  return status;
}

/* --------------------------------------------- Sturm count / bisection ---
 * Number of eigenvalues of the tridiagonal (d, e) strictly below sigma, from
 * the signs of the pivots of the LDL^T factorisation of T - sigma I. */
int oc_sturm_count(int M, const double* d, const double* e, double sigma) {
  int cnt = 0;
  double q = 1.0;
  const double tiny = 0x1p-1000;
  for (int i = 0; i < M; ++i) {
    double off = (i > 0) ? e[i - 1] * e[i - 1] / q : 0.0;
    q = (d[i] - sigma) - off;
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

/* Eigenvalues k0 .. k1-1 (ascending order) of the tridiagonal (d, e) into
 * w[0 .. k1-k0) by bisection on the Sturm count, each bracketed until the interval
 * no longer shrinks (width at the level of one ulp).  Independent of oc_tql. */
static void bisect_range(int M, const double* d, const double* e, int k0, int k1, double* w) {
  if (M <= 0 || k1 <= k0) return;
  double lo = d[0], hi = d[0];
  for (int i = 0; i < M; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < M ? fabs(e[i]) : 0.0);
    if (d[i] - r < lo) lo = d[i] - r;
    if (d[i] + r > hi) hi = d[i] + r;
  }
  double span = hi - lo;
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
#pragma omp parallel for schedule(dynamic, 8)
  for (int k = k0; k < k1; ++k) {
    /* smallest x with count(x) > k: the (k+1)-th eigenvalue */
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      if (oc_sturm_count(M, d, e, mid) > k) b = mid; else a = mid;
    }
    w[k - k0] = 0.5 * (a + b);
  }
}

/* All M eigenvalues of (d, e), ascending. */
void oc_bisect(int M, const double* d, const double* e, double* w) { bisect_range(M, d, e, 0, M, w); }

/* ---------------------------------------------------------------- Eq. 6 ---
 * Back-transformation Y = L^-T Z: back substitution with the upper triangular
 * L^T for every column of Z (overwritten by Y). */
void oc_backsub(int M, int ncol, const double* L, int ldl, double* Z, int ldz) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ncol; ++j) {
    double* z = Z + (size_t)j * ldz;
    for (int i = M - 1; i >= 0; --i) {
      double t = z[i];
      for (int k = i + 1; k < M; ++k) t -= L[IX(k, i, ldl)] * z[k];
      z[i] = t / L[IX(i, i, ldl)];
    }
  }
}

/* Sort eigenpairs ascending (stable insertion order by value) and fix each
 * eigenvector's sign: the entry of largest magnitude is made positive, ties go
 * to the lowest row index. */
static void sort_and_sign(int M, double* w, double* Y, int ldy) {
  int* idx = (int*)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
  for (int i = 0; i < M; ++i) idx[i] = i;
  for (int i = 1; i < M; ++i) { /* insertion sort of indices by w */
    int t = idx[i], j = i - 1;
    while (j >= 0 && w[idx[j]] > w[t]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = t;
  }
  double* w2 = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
  for (int i = 0; i < M; ++i) w2[i] = w[idx[i]];
  if (Y) {
    double* Y2 = (double*)malloc(sizeof(double) * (size_t)M * (M > 0 ? M : 1));
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) Y2[IX(i, j, M)] = Y[IX(i, idx[j], ldy)];
    for (int j = 0; j < M; ++j) {
      int im = 0;
      double best = -1.0;
      for (int i = 0; i < M; ++i) {
        double a = fabs(Y2[IX(i, j, M)]);
        if (a > best) { best = a; im = i; }
      }
      double sgn = (Y2[IX(im, j, M)] < 0.0) ? -1.0 : 1.0;
      for (int i = 0; i < M; ++i) Y[IX(i, j, ldy)] = sgn * Y2[IX(i, j, M)];
    }
    free(Y2);
  }
  for (int i = 0; i < M; ++i) w[i] = w2[i];
  free(w2);
  free(idx);
}

/* ---------------------------------------------------------------- Eq. 2 ---
 * Full GEP solve A Y = B Y Lambda, Y^T B Y = I, following section 3.1:
 * Cholesky (Eq. 4), reduction (Eq. 5), SEP by tridiagonalisation + QL (Eq. 3),
 * back-transformation (Eq. 6).  A and B are read (lower triangles) and not
 * modified.  w[M] receives the eigenvalues ascending; if Y != NULL and
 * want_vectors, Y receives the B-orthonormal eigenvectors with the sign
 * convention of sort_and_sign.  want_vectors == 0 takes the eigenvalue-only
 * route (Sturm bisection, no Q, no back-transformation).
 * Returns 0, k in 1..M if B is not positive definite (leading minor k), or
 * M + l if QL failed on eigenvalue l. */
int oc_gep_solve(int M, const double* A, int lda, const double* B, int ldb, double* w, double* Y,
                 int ldy, int want_vectors) {
  if (M <= 0) return 0;
  size_t n2 = (size_t)M * M;
  double* L = (double*)malloc(sizeof(double) * n2);
  double* C = (double*)malloc(sizeof(double) * n2);
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      L[IX(i, j, M)] = B[IX(i, j, ldb)];
      C[IX(i, j, M)] = A[IX(i, j, lda)];
    }
  int info = oc_cholesky(M, L, M);
  if (info) { free(C); free(L); return info; }
  oc_two_sided(M, C, M, L, M);
  double* d = (double*)malloc(sizeof(double) * (size_t)M);
  double* e = (double*)calloc((size_t)M, sizeof(double));
  int status = 0;
  if (want_vectors && Y) {
    double* Q = (double*)malloc(sizeof(double) * n2);
    oc_tridiag(M, C, M, d, e, Q, M);
    status = oc_tql(M, d, e, Q, M);
    if (!status) {
      oc_backsub(M, M, L, M, Q, M);
      for (int j = 0; j < M; ++j)
        for (int i = 0; i < M; ++i) Y[IX(i, j, ldy)] = Q[IX(i, j, M)];
      for (int i = 0; i < M; ++i) w[i] = d[i];
      sort_and_sign(M, w, Y, ldy);
    }
    free(Q);
  } else {
    oc_tridiag(M, C, M, d, e, NULL, 0);
    oc_bisect(M, d, e, w);
  }
  free(e);
  free(d);
  free(C);
  free(L);
  return status ? M + status : 0;
}

/* ----------------------------------------------------------- Eq. 7 - 9 ---
 * Cholesky-free ("EigenExa style") GEP solve, section 3.1:
 *   B W = W D                       standard eigenproblem of B (Eq. 7),
 *   A' = (D^-1/2 W^T) A (W D^-1/2)  reduced standard problem (Eq. 8),
 *   A' Z = Z Lambda,  Y = W D^-1/2 Z (Eq. 9),
 * each standard problem solved by the same TRD + QL route as oc_gep_solve.  Same
 * arguments, outputs and conventions as oc_gep_solve; returns 0, n in 1..M when B has
 * n eigenvalues <= 0 (B not positive definite), or M + l if QL failed. */
int oc_gep_solve_eigenexa(int M, const double* A, int lda, const double* B, int ldb, double* w, double* Y,
                          int ldy, int want_vectors) {
  if (M <= 0) return 0;
  size_t n2 = (size_t)M * M;
  double* S = (double*)malloc(sizeof(double) * n2);
  double* X = (double*)malloc(sizeof(double) * n2);
  double* d = (double*)malloc(sizeof(double) * (size_t)M);
  double* e = (double*)calloc((size_t)M, sizeof(double));
  int status = 0;
  /* Eq. 7: W (into X) and D (into d) */
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) S[IX(i, j, M)] = B[IX(i, j, ldb)];
  oc_tridiag(M, S, M, d, e, X, M);
  status = oc_tql(M, d, e, X, M);
  if (status) goto done;
  {
    int nonpos = 0;
    for (int i = 0; i < M; ++i) nonpos += !(d[i] > 0.0);
    if (nonpos) { status = -nonpos; goto done; }
  }
  /* X = W D^-1/2 */
  for (int j = 0; j < M; ++j) {
    double s = 1.0 / sqrt(d[j]);
    for (int i = 0; i < M; ++i) X[IX(i, j, M)] *= s;
  }
  /* Eq. 8: A' = X^T (A X), A read through its lower triangle */
  {
    double* T = (double*)malloc(sizeof(double) * n2);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        double t = 0.0;
        for (int k = 0; k < M; ++k) t += sym_lower(A, lda, i, k) * X[IX(k, j, M)];
        T[IX(i, j, M)] = t;
      }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        double t = 0.0;
        for (int k = 0; k < M; ++k) t += X[IX(k, i, M)] * T[IX(k, j, M)];
        S[IX(i, j, M)] = t;
      }
    free(T);
  }
  /* Eq. 9: A' Z = Z Lambda, Y = X Z */
  for (int i = 0; i < M; ++i) e[i] = 0.0;
  if (want_vectors && Y) {
    double* Z = (double*)malloc(sizeof(double) * n2);
    oc_tridiag(M, S, M, d, e, Z, M);
    status = oc_tql(M, d, e, Z, M);
    if (!status) {
#pragma omp parallel for schedule(static)
      for (int j = 0; j < M; ++j)
        for (int i = 0; i < M; ++i) {
          double t = 0.0;
          for (int k = 0; k < M; ++k) t += X[IX(i, k, M)] * Z[IX(k, j, M)];
          Y[IX(i, j, ldy)] = t;
        }
      for (int i = 0; i < M; ++i) w[i] = d[i];
      sort_and_sign(M, w, Y, ldy);
    }
    free(Z);
  } else {
    oc_tridiag(M, S, M, d, e, NULL, 0);
    oc_bisect(M, d, e, w);
  }
done:
  free(e);
  free(d);
  free(X);
  free(S);
  if (status < 0) return -status;
  return status ? M + status : 0;
}

/* ------------------------------------------------------ partial spectrum ---
 * The n_want lowest eigenpairs only (the occupied states of the electronic-structure
 * use case): Cholesky (Eq. 4), reduction (Eq. 5), tridiagonalisation with explicit Q,
 * Sturm bisection for eigenvalues 0 .. n_want-1, inverse iteration on T for their
 * vectors (Golub & Van Loan, inverse iteration: LU with partial pivoting of T - sigma I,
 * a fixed number of solves from a deterministic start; vectors whose eigenvalues lie
 * within 1e-3 ||T|| of the previous one form a cluster and are re-orthogonalised against
 * its earlier members; shifts of equal eigenvalues are separated by 10 eps ||T||),
 * Z = Q X and Y = L^-T Z (Eq. 6).  w[n_want] ascending; Y (M x n_want, ldy) B-orthonormal
 * with the sign convention of sort_and_sign.  Returns 0 or k in 1..M as oc_gep_solve. */

/* x <- (T - sigma I)^-1 x using the factors of tri_lu. */
static void tri_solve(int n, const double* u0, const double* u1, const double* u2, const double* l,
                      const int* piv, double* x) {
  for (int i = 0; i + 1 < n; ++i) {
    if (piv[i]) { double t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
    x[i + 1] -= l[i] * x[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = x[i];
    if (i + 1 < n) t -= u1[i] * x[i + 1];
    if (i + 2 < n) t -= u2[i] * x[i + 2];
    x[i] = t / u0[i];
  }
}

/* Gaussian elimination with partial pivoting of the tridiagonal T - sigma I: row i of U
 * is (u0, u1, u2) on columns i, i+1, i+2; l[i], piv[i] record step i.  A zero pivot is
 * replaced by tiny (the shift is an eigenvalue to working accuracy). */
static void tri_lu(int n, const double* d, const double* e, double sigma, double tiny, double* u0,
                   double* u1, double* u2, double* l, int* piv) {
  double c0 = d[0] - sigma, c1 = (n > 1) ? e[0] : 0.0, c2 = 0.0;  /* current row */
  for (int i = 0; i + 1 < n; ++i) {
    double s0 = e[i], s1 = d[i + 1] - sigma, s2 = (i + 2 < n) ? e[i + 1] : 0.0;  /* next row */
    if (fabs(c0) >= fabs(s0)) {
      if (c0 == 0.0) c0 = tiny;
      double m = s0 / c0;
      u0[i] = c0; u1[i] = c1; u2[i] = c2; l[i] = m; piv[i] = 0;
      c0 = s1 - m * c1;
      c1 = s2 - m * c2;
    } else {
      double m = c0 / s0;
      u0[i] = s0; u1[i] = s1; u2[i] = s2; l[i] = m; piv[i] = 1;
      c0 = c1 - m * s1;
      c1 = c2 - m * s2;
    }
    c2 = 0.0;
  }
  if (c0 == 0.0) c0 = tiny;
  u0[n - 1] = c0;
}

int oc_gep_solve_partial(int M, const double* A, int lda, const double* B, int ldb, int n_want, double* w,
                         double* Y, int ldy) {
  if (M <= 0 || n_want <= 0) return 0;
  if (n_want > M) n_want = M;
  size_t n2 = (size_t)M * M;
  double* L = (double*)malloc(sizeof(double) * n2);
  double* C = (double*)malloc(sizeof(double) * n2);
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      L[IX(i, j, M)] = B[IX(i, j, ldb)];
      C[IX(i, j, M)] = A[IX(i, j, lda)];
    }
  int info = oc_cholesky(M, L, M);
  if (info) { free(C); free(L); return info; }
  oc_two_sided(M, C, M, L, M);
  double* Q = (double*)malloc(sizeof(double) * n2);
  double* d = (double*)malloc(sizeof(double) * (size_t)M);
  double* e = (double*)calloc((size_t)M, sizeof(double));
  oc_tridiag(M, C, M, d, e, Q, M);
  bisect_range(M, d, e, 0, n_want, w);
  double tnorm = 0.0;
  for (int i = 0; i < M; ++i) {
    double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < M ? fabs(e[i]) : 0.0);
    if (r > tnorm) tnorm = r;
  }
  if (tnorm == 0.0) tnorm = 1.0;
  const double eps = 0x1p-53, sep = 10.0 * eps * tnorm, ortol = 1e-3 * tnorm;
  double* X = (double*)calloc((size_t)M * n_want, sizeof(double));
  double *u0 = (double*)malloc(sizeof(double) * M), *u1 = (double*)malloc(sizeof(double) * M);
  double *u2 = (double*)malloc(sizeof(double) * M), *lm = (double*)malloc(sizeof(double) * M);
  int* piv = (int*)malloc(sizeof(int) * (size_t)M);
  int cl0 = 0;               /* first index of the current cluster */
  double prev_shift = 0.0;
  for (int j = 0; j < n_want; ++j) {
    double sigma = w[j];
    if (j > 0 && w[j] - w[j - 1] > ortol) cl0 = j;
    if (j > cl0 && sigma - prev_shift < sep) sigma = prev_shift + sep;
    prev_shift = sigma;
    tri_lu(M, d, e, sigma, eps * tnorm, u0, u1, u2, lm, piv);
    double* x = X + (size_t)j * M;
    unsigned long long st = 0x9E3779B97F4A7C15ull * (unsigned long long)(j + 1);
    for (int i = 0; i < M; ++i) {  /* deterministic start in [-1, 1] (splitmix64) */
      st += 0x9E3779B97F4A7C15ull;
      unsigned long long z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      x[i] = (double)(z >> 11) * 0x1p-52 - 1.0;
    }
    for (int it = 0; it < 4; ++it) {
      tri_solve(M, u0, u1, u2, lm, piv, x);
      for (int k = cl0; k < j; ++k) {  /* re-orthogonalise within the cluster */
        const double* y = X + (size_t)k * M;
        double dot = 0.0;
        for (int i = 0; i < M; ++i) dot += y[i] * x[i];
        for (int i = 0; i < M; ++i) x[i] -= dot * y[i];
      }
      double nrm = 0.0;
      for (int i = 0; i < M; ++i) nrm += x[i] * x[i];
      nrm = sqrt(nrm);
      for (int i = 0; i < M; ++i) x[i] /= nrm;
    }
  }
  /* Z = Q X, then Y = L^-T Z */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n_want; ++j)
    for (int i = 0; i < M; ++i) {
      double t = 0.0;
      for (int k = 0; k < M; ++k) t += Q[IX(i, k, M)] * X[IX(k, j, M)];
      Y[IX(i, j, ldy)] = t;
    }
  oc_backsub(M, n_want, L, M, Y, ldy);
  for (int j = 0; j < n_want; ++j) {  /* largest-magnitude entry positive, lowest row on ties */
    int im = 0;
    double best = -1.0;
    for (int i = 0; i < M; ++i) {
      double a = fabs(Y[IX(i, j, ldy)]);
      if (a > best) { best = a; im = i; }
    }
    if (Y[IX(im, j, ldy)] < 0.0)
      for (int i = 0; i < M; ++i) Y[IX(i, j, ldy)] = -Y[IX(i, j, ldy)];
  }
  free(piv); free(lm); free(u2); free(u1); free(u0); free(X);
  free(e); free(d); free(Q); free(C); free(L);
  return 0;
}

/* ---------------------------------------------- independent pin: Jacobi ---
 * Cyclic two-sided Jacobi on a symmetric S (full, both triangles used; lower
 * read and mirrored first).  Sweeps until off(S) <= 1e-15 ||S||_F or 100
 * sweeps.  w receives the diagonal (unsorted), V (if non-NULL) the rotations'
 * product.  Returns the number of sweeps, or -1 on non-convergence. */
int oc_jacobi(int M, double* S, int lds, double* w, double* V, int ldv) {
  for (int j = 0; j < M; ++j)
    for (int i = j + 1; i < M; ++i) S[IX(j, i, lds)] = S[IX(i, j, lds)];
  if (V)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) V[IX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) fro += S[IX(i, j, lds)] * S[IX(i, j, lds)];
  fro = sqrt(fro);
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i)
        if (i != j) off += S[IX(i, j, lds)] * S[IX(i, j, lds)];
    if (sqrt(off) <= 1e-15 * fro) break;
    for (int p = 0; p < M - 1; ++p)
      for (int q = p + 1; q < M; ++q) {
        double apq = S[IX(p, q, lds)];
        if (apq == 0.0) continue;
        double theta = (S[IX(q, q, lds)] - S[IX(p, p, lds)]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* S <- J^T S J with J the rotation in the (p, q) plane */
        for (int k = 0; k < M; ++k) {
          double skp = S[IX(k, p, lds)], skq = S[IX(k, q, lds)];
          S[IX(k, p, lds)] = c * skp - s * skq;
          S[IX(k, q, lds)] = s * skp + c * skq;
        }
        for (int k = 0; k < M; ++k) {
          double spk = S[IX(p, k, lds)], sqk = S[IX(q, k, lds)];
          S[IX(p, k, lds)] = c * spk - s * sqk;
          S[IX(q, k, lds)] = s * spk + c * sqk;
        }
        if (V)
          for (int k = 0; k < M; ++k) {
            double vkp = V[IX(k, p, ldv)], vkq = V[IX(k, q, ldv)];
            V[IX(k, p, ldv)] = c * vkp - s * vkq;
            V[IX(k, q, ldv)] = s * vkp + c * vkq;
          }
      }
  }
  for (int i = 0; i < M; ++i) w[i] = S[IX(i, i, lds)];
  return sweep < 100 ? sweep : -1;
}

/* ------------------------------------------ independent pin: inertia ---
 * Sylvester's law of inertia: with B positive definite, the number of
 * eigenvalues of the pencil (A, B) below sigma equals the number of negative
 * eigenvalues of the symmetric matrix A - sigma B.  That inertia is read off a
 * symmetric LDL^T factorisation with Bunch-Parlett complete pivoting (1x1 or
 * 2x2 pivots; a 2x2 pivot chosen by the rule has a negative determinant and so
 * contributes one negative and one positive eigenvalue).  Uses neither the
 * Cholesky factor nor any eigen-routine. */
void oc_inertia(int M, const double* A, int lda, const double* B, int ldb, double sigma, int* nneg,
                int* nzero, int* npos) {
  double* S = (double*)malloc(sizeof(double) * (size_t)M * (M > 0 ? M : 1));
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) S[IX(i, j, M)] = sym_lower(A, lda, i, j) - sigma * sym_lower(B, ldb, i, j);
  int* perm = (int*)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1)); /* active index set */
  for (int i = 0; i < M; ++i) perm[i] = i;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int neg = 0, zer = 0, pos = 0;
  int n = M;
  while (n > 0) {
    /* largest diagonal and off-diagonal magnitudes in the active block */
    int id = 0, oi = 0, oj = 0;
    double mu1 = -1.0, mu0 = -1.0;
    for (int a = 0; a < n; ++a) {
      double v = fabs(S[IX(perm[a], perm[a], M)]);
      if (v > mu1) { mu1 = v; id = a; }
      for (int b = a + 1; b < n; ++b) {
        double o = fabs(S[IX(perm[b], perm[a], M)]);
        if (o > mu0) { mu0 = o; oi = a; oj = b; }
      }
    }
    if (n == 1 || mu1 >= alpha * mu0) {
      int p = perm[id];
      double piv = S[IX(p, p, M)];
      if (piv < 0.0) ++neg; else if (piv > 0.0) ++pos; else ++zer;
      if (piv != 0.0)
        for (int b = 0; b < n; ++b) {
          if (b == id) continue;
          int j = perm[b];
          double f = S[IX(j, p, M)] / piv;
          for (int a = 0; a < n; ++a) {
            if (a == id) continue;
            int i = perm[a];
            S[IX(i, j, M)] -= f * S[IX(i, p, M)];
          }
        }
      perm[id] = perm[n - 1];
      --n;
    } else {
      int p = perm[oi], q = perm[oj];
      double a11 = S[IX(p, p, M)], a22 = S[IX(q, q, M)], a21 = S[IX(q, p, M)];
      double det = a11 * a22 - a21 * a21; /* < 0 by the pivot rule */
      ++neg;
      ++pos;
      /* S_rest -= [s_p s_q] E^-1 [s_p s_q]^T, E = [[a11 a21];[a21 a22]] */
      double i11 = a22 / det, i22 = a11 / det, i21 = -a21 / det;
      for (int b = 0; b < n; ++b) {
        if (b == oi || b == oj) continue;
        int j = perm[b];
        double sjp = S[IX(j, p, M)], sjq = S[IX(j, q, M)];
        double fp = i11 * sjp + i21 * sjq, fq = i21 * sjp + i22 * sjq;
        for (int a = 0; a < n; ++a) {
          if (a == oi || a == oj) continue;
          int i = perm[a];
          S[IX(i, j, M)] -= S[IX(i, p, M)] * fp + S[IX(i, q, M)] * fq;
        }
      }
      /* remove positions oi < oj from the active set */
      perm[oj] = perm[n - 1];
      --n;
      perm[oi] = perm[n - 1];
      --n;
    }
  }
  *nneg = neg;
  *nzero = zer;
  *npos = pos;
  free(perm);
  free(S);
}

/* ------------------------------------------------ adjoint (derivative) ---
 * Reverse-mode derivative of  loss = sum_k lbar_k lambda_k + <W, P>,
 * P = Y_o Y_o^T over the n_occ lowest eigenpairs, from first-order
 * perturbation of Eq. 2 (d lambda_k = y_k^T (dA - lambda_k dB) y_k and the
 * standard eigenvector perturbation with the B-normalisation term).  With
 * What = Y^T W Y, o = occupied, v = virtual and F_kj = 1/(lambda_k - lambda_j):
 *   Abar = Y G Y^T:  G_oo = diag(lbar_o), G_ov = G_vo^T = What_ov o F_ov, G_vv = 0
 *   Bbar = Y H Y^T:  H_oo = -diag(lbar_o lambda_o) - What_oo,
 *                    H_ov = H_vo^T = -diag(lambda_o) (What_ov o F_ov), H_vv = 0
 * Only occupied/virtual gaps are divided by.  lbar has n_occ entries (the
 * loss's eigenvalue weights); W may be NULL (eigenvalue part only).  Y is the
 * full M x M B-orthonormal eigenvector matrix, w ascending.  Plain triple loops. */
void oc_adjoint(int M, int n_occ, const double* w, const double* Y, int ldy, const double* lbar,
                const double* W, int ldw, double* Abar, double* Bbar, int ldab) {
  size_t n2 = (size_t)M * (M > 0 ? M : 1);
  double* Wh = (double*)calloc(n2, sizeof(double));
  if (W) {
    double* T = (double*)calloc(n2, sizeof(double)); /* T = W Y */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int k = 0; k < M; ++k) s += sym_lower(W, ldw, i, k) * Y[IX(k, j, ldy)];
        T[IX(i, j, M)] = s;
      }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int k = 0; k < M; ++k) s += Y[IX(k, i, ldy)] * T[IX(k, j, M)];
        Wh[IX(i, j, M)] = s;
      }
    free(T);
  }
  double* G = (double*)calloc(n2, sizeof(double));
  double* H = (double*)calloc(n2, sizeof(double));
  for (int k = 0; k < n_occ; ++k) {
    G[IX(k, k, M)] += lbar ? lbar[k] : 0.0;
    H[IX(k, k, M)] -= (lbar ? lbar[k] : 0.0) * w[k];
    for (int j = 0; j < n_occ; ++j) H[IX(k, j, M)] -= 0.5 * (Wh[IX(k, j, M)] + Wh[IX(j, k, M)]);
    for (int j = n_occ; j < M; ++j) {
      double wkj = 0.5 * (Wh[IX(k, j, M)] + Wh[IX(j, k, M)]);
      double g = wkj / (w[k] - w[j]);
      G[IX(k, j, M)] = g;
      G[IX(j, k, M)] = g;
      H[IX(k, j, M)] = -w[k] * g;
      H[IX(j, k, M)] = -w[k] * g;
    }
  }
  /* Abar = Y G Y^T, Bbar = Y H Y^T */
  double* TG = (double*)calloc(n2, sizeof(double));
  double* TH = (double*)calloc(n2, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      double sg = 0.0, sh = 0.0;
      for (int k = 0; k < M; ++k) {
        sg += Y[IX(i, k, ldy)] * G[IX(k, j, M)];
        sh += Y[IX(i, k, ldy)] * H[IX(k, j, M)];
      }
      TG[IX(i, j, M)] = sg;
      TH[IX(i, j, M)] = sh;
    }
#pragma omp parallel for schedule(static)
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      double sg = 0.0, sh = 0.0;
      for (int k = 0; k < M; ++k) {
        sg += TG[IX(i, k, M)] * Y[IX(j, k, ldy)];
        sh += TH[IX(i, k, M)] * Y[IX(j, k, ldy)];
      }
      Abar[IX(i, j, ldab)] = sg;
      Bbar[IX(i, j, ldab)] = sh;
    }
  free(TH);
  free(TG);
  free(H);
  free(G);
  free(Wh);
}
