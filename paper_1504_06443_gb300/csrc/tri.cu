// Reducer stages (section 3.1 (b)):
//   Eq. 4  B = L L^T              blocked right-looking Cholesky
//   Eq. 5  C = L^-1 A L^-T         "ScaLAPACK style" (triangular solves, L^-1 never formed)
//                                  "ELPA style" (R = L^-1 formed, then C = R A R^T)
//   Eq. 6  Y = L^-T Z              blocked back-substitution
// plus the triangular building blocks they share.  Every nb x nb diagonal block
// of L is factored and inverted by one CTA in shared memory; everything else is
// a dense product on the GEMM engine, so the O(M^3) work runs as matrix products.
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int NB = 128;  // diagonal block order

// In-place inverse of the r x r lower triangular S (shared, leading dim NB),
// from the bottom-right: column j of L^-1 is -(1/l_jj) * L22^-1 * l(j+1:, j).
__device__ void tri_inv_smem(double* S, double* tmp, int r) {
  // X = L^-1 column by column from the last: X(i, j) = -X(j, j) sum_{q=j+1..i} X(i, q) L(q, j),
  // columns q > j already inverted in place.  Two threads per row i (lanes 2i, 2i + 1 take
  // alternate q) halve the dependent FMA chain of each dot product.
  __shared__ double ajj_s;
  const int i = threadIdx.x >> 1, part = threadIdx.x & 1;
  for (int j = r - 1; j >= 0; --j) {
    __syncthreads();
    if (threadIdx.x == 0) ajj_s = 1.0 / S[j + j * NB];  // one division per column
    double s = 0.0, s2 = 0.0;  // two independent FMA chains per thread
    if (i > j && i < r) {
      int q = j + 1 + part;
      for (; q + 2 <= i; q += 4) {
        s = fma(S[i + q * NB], S[q + j * NB], s);
        s2 = fma(S[i + (q + 2) * NB], S[q + 2 + j * NB], s2);
      }
      if (q <= i) s = fma(S[i + q * NB], S[q + j * NB], s);
    }
    s += s2;
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (part == 0 && i > j && i < r) tmp[i] = s;
    __syncthreads();
    const double ajj = ajj_s;
    if (part == 0 && i > j && i < r) S[i + j * NB] = -ajj * tmp[i];
    if (threadIdx.x == 0) S[j + j * NB] = ajj;
  }
  __syncthreads();
}

// Writes the r x r lower inverse from shared memory into an NB x NB block (identity
// padding for r < NB, zero strict upper triangle).
__device__ void store_inv(const double* S, int r, double* out) {
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int i = idx % NB, j = idx / NB;
    double v;
    if (i < r && j < r) v = (i >= j) ? S[i + j * NB] : 0.0;
    else v = (i == j) ? 1.0 : 0.0;
    out[idx] = v;
  }
}

// Factor the diagonal block B(kb:kb+r, kb:kb+r) (already updated by earlier trailing
// products) and store L_kk in place plus L_kk^-1 into invD.
__global__ void __launch_bounds__(256) k_potrf_diag(int r, double* B, int ldb, double* invD, int kb,
                                                    int* st) {
  extern __shared__ double sm[];
  double* S = sm;
  double* tmp = sm + NB * NB;
  __shared__ int fail;
  if (status_bad(st)) return;
  if (threadIdx.x == 0) fail = 0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    int i = idx % r, j = idx / r;
    S[i + j * NB] = (i >= j) ? B[GEP_IX(i, j, ldb)] : 0.0;
  }
  // right-looking, one column per step; thread t owns row i = t mod 128 of the trailing
  // triangle, columns of parity t / 128 (no index division, no idle upper half)
  __shared__ double rinv;
  const int i = threadIdx.x & (NB - 1), h = threadIdx.x / NB;
  for (int j = 0; j < r; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      double p = S[j + j * NB];
      if (!(p > 0.0) || !isfinite(p)) fail = j + 1;
      else {
        const double l = sqrt(p);
        S[j + j * NB] = l;
        rinv = 1.0 / l;
      }
    }
    __syncthreads();
    if (fail) break;
    if (h == 0 && i > j && i < r) S[i + j * NB] *= rinv;
    __syncthreads();
    if (i > j && i < r) {
      const double lij = S[i + j * NB];
      int c = j + 1;
      if ((c & 1) != h) ++c;
      for (; c + 6 <= i; c += 8) {  // four columns at a time: loads issued before the stores
        const double l0 = S[c + j * NB], l1 = S[c + 2 + j * NB], l2 = S[c + 4 + j * NB], l3 = S[c + 6 + j * NB];
        double* x = S + i + c * NB;
        const double x0 = x[0], x1 = x[2 * NB], x2 = x[4 * NB], x3 = x[6 * NB];
        x[0] = fma(-lij, l0, x0);
        x[2 * NB] = fma(-lij, l1, x1);
        x[4 * NB] = fma(-lij, l2, x2);
        x[6 * NB] = fma(-lij, l3, x3);
      }
      for (; c <= i; c += 2) S[i + c * NB] = fma(-lij, S[c + j * NB], S[i + c * NB]);
    }
  }
  __syncthreads();
  if (fail) {
    if (threadIdx.x == 0) atomicCAS(st, 0, kb + fail);
    return;
  }
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    int i = idx % r, j = idx / r;
    if (i >= j) B[GEP_IX(i, j, ldb)] = S[i + j * NB];
  }
  tri_inv_smem(S, tmp, r);
  store_inv(S, r, invD);
}

// One CTA per diagonal block of an existing lower triangular L: invert it.
__global__ void __launch_bounds__(256) k_inv_diag(int M, const double* L, int ldl, double* invD,
                                                  const int* st) {
  extern __shared__ double sm[];
  if (status_bad(st)) return;
  double* S = sm;
  double* tmp = sm + NB * NB;
  int b = blockIdx.x, kb = b * NB;
  int r = min(NB, M - kb);
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    int i = idx % r, j = idx / r;
    S[i + j * NB] = (i >= j) ? L[GEP_IX(kb + i, kb + j, ldl)] : 0.0;
  }
  tri_inv_smem(S, tmp, r);
  store_inv(S, r, invD + (size_t)b * NB * NB);
}

constexpr size_t kSmemDiag = (size_t)NB * NB * sizeof(double) + NB * sizeof(double);

int set_smem_attr() {
  static unsigned long long devices = 0;
  if (first_use_on_device(devices)) {
    cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDiag);
    cudaFuncSetAttribute(k_inv_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDiag);
  }
  return GEP_OK;
}

}  // namespace

size_t trsm_tmp_elems(int M, int n, int nb) { (void)M; return (size_t)nb * (size_t)(n > 0 ? n : 1); }

int tri_inv_diag_blocks(gep_handle_t h, int M, const double* L, int ldl, double* invD, int nb) {
  if (nb != NB) return GEP_ERR_UNSUPPORTED;
  if (M <= 0) return GEP_OK;
  set_smem_attr();
  int nblk = (M + NB - 1) / NB;
  k_inv_diag<<<nblk, 256, kSmemDiag, h->stream>>>(M, L, ldl, invD, h->d_status);
  return check_launch(h);
}

// All triangular solves and the Cholesky factorisation below recurse on halves whose
// split points are multiples of NB, down to the NB x NB diagonal blocks (leaf o covers
// rows o .. o+NB-1 and uses invD block o/NB).  The off-diagonal work is then a few
// products with a long inner dimension (n/2, n/4, ...), which the tensor-core engine
// runs near its best rate, instead of many rank-NB updates.
namespace {

int split_nb(int n) { return ((n / NB + 1) / 2) * NB; }

// rows [o, o+n) of X (X points at row o) := L(o:o+n, o:o+n)^-1 X
int lln_rec(gep_handle_t h, int o, int n, int ncol, const double* L, int ldl, const double* invD, double* X, int ldx,
            double* tmp, int engine) {
  if (n <= NB) {
    const double* Dk = invD + (size_t)(o / NB) * NB * NB;
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', n, ncol, n, 1.0, Dk, NB, X, ldx, 0.0, tmp, n, engine));
    return copy_matrix(h, n, ncol, tmp, n, X, ldx);
  }
  int n1 = split_nb(n), n2 = n - n1;
  GEP_CHECK(lln_rec(h, o, n1, ncol, L, ldl, invD, X, ldx, tmp, engine));
  GEP_CHECK(dgemm(h, 'N', 'N', 'F', n2, ncol, n1, -1.0, L + GEP_IX(o + n1, o, ldl), ldl, X, ldx, 1.0, X + n1, ldx,
                  engine));
  return lln_rec(h, o + n1, n2, ncol, L, ldl, invD, X + n1, ldx, tmp, engine);
}

// rows [o, o+n) of X := L(o:o+n, o:o+n)^-T X
int llt_rec(gep_handle_t h, int o, int n, int ncol, const double* L, int ldl, const double* invD, double* X, int ldx,
            double* tmp, int engine) {
  if (n <= NB) {
    const double* Dk = invD + (size_t)(o / NB) * NB * NB;
    GEP_CHECK(dgemm(h, 'T', 'N', 'F', n, ncol, n, 1.0, Dk, NB, X, ldx, 0.0, tmp, n, engine));
    return copy_matrix(h, n, ncol, tmp, n, X, ldx);
  }
  int n1 = split_nb(n), n2 = n - n1;
  GEP_CHECK(llt_rec(h, o + n1, n2, ncol, L, ldl, invD, X + n1, ldx, tmp, engine));
  GEP_CHECK(dgemm(h, 'T', 'N', 'F', n1, ncol, n2, -1.0, L + GEP_IX(o + n1, o, ldl), ldl, X + n1, ldx, 1.0, X, ldx,
                  engine));
  return llt_rec(h, o, n1, ncol, L, ldl, invD, X, ldx, tmp, engine);
}

// X (m x n, columns o .. o+n of the factor) := X L(o:o+n, o:o+n)^-T
int rlt_rec(gep_handle_t h, int o, int n, int m, const double* L, int ldl, const double* invD, double* X, int ldx,
            double* tmp, int engine) {
  if (n <= NB) {
    const double* Dk = invD + (size_t)(o / NB) * NB * NB;
    GEP_CHECK(dgemm(h, 'N', 'T', 'F', m, n, n, 1.0, X, ldx, Dk, NB, 0.0, tmp, m, engine));
    return copy_matrix(h, m, n, tmp, m, X, ldx);
  }
  int n1 = split_nb(n), n2 = n - n1;
  GEP_CHECK(rlt_rec(h, o, n1, m, L, ldl, invD, X, ldx, tmp, engine));
  GEP_CHECK(dgemm(h, 'N', 'T', 'F', m, n2, n1, -1.0, X, ldx, L + GEP_IX(o + n1, o, ldl), ldl, 1.0,
                  X + (size_t)n1 * ldx, ldx, engine));
  return rlt_rec(h, o + n1, n2, m, L, ldl, invD, X + (size_t)n1 * ldx, ldx, tmp, engine);
}

// Eq. 4 on the diagonal block (o, o) of order n; B points at the full matrix.
int potrf_rec(gep_handle_t h, int o, int n, double* B, int ldb, double* invD, double* tmp, int engine) {
  if (n <= NB) {
    k_potrf_diag<<<1, 256, kSmemDiag, h->stream>>>(n, B + GEP_IX(o, o, ldb), ldb, invD + (size_t)(o / NB) * NB * NB, o,
                                                   h->d_status);
    return check_launch(h);
  }
  int n1 = split_nb(n), n2 = n - n1;
  GEP_CHECK(potrf_rec(h, o, n1, B, ldb, invD, tmp, engine));
  double* L21 = B + GEP_IX(o + n1, o, ldb);
  GEP_CHECK(rlt_rec(h, o, n1, n2, B, ldb, invD, L21, ldb, tmp, engine));   // L21 = A21 L11^-T
  GEP_CHECK(dgemm(h, 'N', 'T', 'L', n2, n2, n1, -1.0, L21, ldb, L21, ldb, 1.0, B + GEP_IX(o + n1, o + n1, ldb), ldb,
                  engine));                                                 // A22 -= L21 L21^T
  return potrf_rec(h, o + n1, n2, B, ldb, invD, tmp, engine);
}

}  // namespace

// X := L^-1 X (forward substitution); tmp holds max(NB x n) doubles.
int trsm_lln(gep_handle_t h, int M, int n, const double* L, int ldl, const double* invD, int nb,
             double* X, int ldx, double* tmp, int engine) {
  if (nb != NB) return GEP_ERR_UNSUPPORTED;
  if (M <= 0 || n <= 0) return GEP_OK;
  return lln_rec(h, 0, M, n, L, ldl, invD, X, ldx, tmp, engine);
}

// X := L^-T X (backward substitution with the upper triangular L^T).
int trsm_llt(gep_handle_t h, int M, int n, const double* L, int ldl, const double* invD, int nb,
             double* X, int ldx, double* tmp, int engine) {
  if (nb != NB) return GEP_ERR_UNSUPPORTED;
  if (M <= 0 || n <= 0) return GEP_OK;
  return llt_rec(h, 0, M, n, L, ldl, invD, X, ldx, tmp, engine);
}

// Eq. 4: recursive Cholesky.  invD receives the inverses of the NB x NB diagonal
// blocks (reused by the reduction and the back-substitution).  tmp (M x NB doubles)
// follows invD in the caller's workspace.
int cholesky(gep_handle_t h, int M, double* B, int ldb, double* invD, int engine) {
  if (M <= 0) return GEP_OK;
  set_smem_attr();
  int nblk = (M + NB - 1) / NB;
  double* tmp = invD + (size_t)nblk * NB * NB;
  return potrf_rec(h, 0, M, B, ldb, invD, tmp, engine);
}

// Eq. 5, "ScaLAPACK style": C = L^-1 A L^-T without forming L^-1, blocked over panels of
// nb columns and exploiting the symmetry of A and C (the blocking of ScaLAPACK's pdsygst):
// with the leading panel A11 (nb x nb), A21 below it and the trailing A22,
//     C11 = L11^-1 A11 L11^-T                       (two triangular solves of order nb)
//     A21 <- A21 L11^-T - 1/2 L21 C11
//     A22 <- A22 - A21 L21^T - L21 A21^T            (lower triangle, one product of depth 2 nb)
//     C21 = L22^-1 (A21 - 1/2 L21 C11)              (triangular solve with the trailing factor)
// and the trailing matrix is reduced the same way.  About M^3 flops in products (two
// thirds in the symmetric rank-2nb updates, one third in the solves), against 2 M^3 for two
// full triangular solves.  A (lower) is overwritten by the full symmetric C; X is an M x M
// scratch matrix, tmp an NB x M one.
int reduce_twosided(gep_handle_t h, int M, double* A, int lda, const double* L, int ldl,
                    const double* invD, double* X, double* tmp, int engine) {
  if (M <= 0) return GEP_OK;
  // panel width: a multiple of NB (the triangular recursions split at multiples of NB)
  int nbp = (M / 8) / NB * NB;
  if (nbp < NB) nbp = NB;
  if (nbp > 1024) nbp = 1024;
  for (int k = 0; k < M; k += nbp) {
    const int nb = (M - k) < nbp ? (M - k) : nbp, n2 = M - k - nb;
    double* A11 = A + GEP_IX(k, k, lda);
    double* A21 = A + GEP_IX(k + nb, k, lda);
    double* A22 = A + GEP_IX(k + nb, k + nb, lda);
    const double* L21 = L + GEP_IX(k + nb, k, ldl);
    // C11 = L11^-1 (L11^-1 A11)^T, full symmetric in A11
    double* T1 = X;
    GEP_CHECK(symmetrize_lower(h, nb, A11, lda));
    GEP_CHECK(lln_rec(h, k, nb, nb, L, ldl, invD, A11, lda, tmp, engine));
    GEP_CHECK(transpose(h, nb, nb, A11, lda, T1, nb));
    GEP_CHECK(lln_rec(h, k, nb, nb, L, ldl, invD, T1, nb, tmp, engine));
    GEP_CHECK(copy_lower(h, nb, T1, nb, A11, lda));
    GEP_CHECK(symmetrize_lower(h, nb, A11, lda));
    if (n2 == 0) break;
    // A21 <- A21 L11^-T - 1/2 L21 C11
    GEP_CHECK(rlt_rec(h, k, nb, n2, L, ldl, invD, A21, lda, tmp, engine));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', n2, nb, nb, -0.5, L21, ldl, A11, lda, 1.0, A21, lda, engine));
    // A22 <- A22 - [A21 L21] [L21 A21]^T (lower triangle)
    double* AA = X;
    double* BB = X + (size_t)n2 * 2 * nb;
    GEP_CHECK(copy_matrix(h, n2, nb, A21, lda, AA, n2));
    GEP_CHECK(copy_matrix(h, n2, nb, L21, ldl, AA + (size_t)n2 * nb, n2));
    GEP_CHECK(copy_matrix(h, n2, nb, L21, ldl, BB, n2));
    GEP_CHECK(copy_matrix(h, n2, nb, A21, lda, BB + (size_t)n2 * nb, n2));
    GEP_CHECK(dgemm(h, 'N', 'T', 'L', n2, n2, 2 * nb, -1.0, AA, n2, BB, n2, 1.0, A22, lda, engine));
    // C21 = L22^-1 (A21 - 1/2 L21 C11)
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', n2, nb, nb, -0.5, L21, ldl, A11, lda, 1.0, A21, lda, engine));
    GEP_CHECK(lln_rec(h, k + nb, n2, nb, L, ldl, invD, A21, lda, tmp, engine));
  }
  return symmetrize_lower(h, M, A, lda);
}

// Eq. 5, "ELPA style": R = L^-1 formed explicitly (R2), then C = (R A) R^T (R3, R4).
// L (lower of B) is overwritten by R.  X and T are M x M scratch matrices (T = tmp2).
int reduce_explicit_inv(gep_handle_t h, int M, double* A, int lda, double* L, int ldl,
                        const double* invD, double* X, double* tmp, int engine) {
  if (M <= 0) return GEP_OK;
  double* T = tmp;                    // M x M
  double* tmp_small = tmp + (size_t)M * M;  // NB x M
  GEP_CHECK(set_matrix(h, M, M, 0.0, 1.0, X, M));
  GEP_CHECK(trsm_lln(h, M, M, L, ldl, invD, NB, X, M, tmp_small, engine));  // X = R = L^-1
  GEP_CHECK(symmetrize_lower(h, M, A, lda));
  GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, X, M, A, lda, 0.0, T, M, engine));   // T = R A
  GEP_CHECK(dgemm(h, 'N', 'T', 'L', M, M, M, 1.0, T, M, X, M, 0.0, A, lda, engine));   // C = T R^T
  GEP_CHECK(symmetrize_lower(h, M, A, lda));
  return copy_lower(h, M, X, M, L, ldl);  // lower(B) <- R
}

}  // namespace gep
