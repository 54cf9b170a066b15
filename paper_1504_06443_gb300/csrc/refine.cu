// FP64 refinement of all eigenpairs of the pencil (A, B) (mixed-precision path).
//
// From an approximate X (columns ~ eigenvectors, X^T B X ~ I) of a lower-precision
// solve, one step forms, with FP64-accurate products,
//     S = X^T A X,   R = X^T B X,   lambda_i = S_ii / R_ii  (B-Rayleigh quotients),
// and the first-order correction X <- X (I + E) that makes X^T B X = I and X^T A X
// diagonal to first order:
//     E_ii = (1 - R_ii) / 2,
//     E_ij = (S_ij - lambda_j R_ij) / (lambda_j - lambda_i)      (i != j),
//     E_ij = -R_ij / 2   when |lambda_j - lambda_i| <= delta (numerically degenerate
//                        pair: only B-orthogonality is restored inside such a pair).
// This is the Ogita-Aishima refinement for the symmetric eigenproblem written in the
// B inner product; it converges quadratically for well-separated eigenvalues, so two
// steps take eigenpairs of FP32-grade accuracy to FP64 accuracy.
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

// lambda_i = S_ii / R_ii; also max |lambda| into lmax[0] (block reduction, one CTA).
__global__ void __launch_bounds__(1024) k_rayleigh(int M, const double* __restrict__ S, const double* __restrict__ R,
                                                   double* __restrict__ lam, double* __restrict__ lmax,
                                                   const int* st) {
  __shared__ double red[32];
  if (status_bad(st)) return;
  double m = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double l = S[GEP_IX(i, i, M)] / R[GEP_IX(i, i, M)];
    lam[i] = l;
    m = fmax(m, fabs(l));
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) r = fmax(r, red[w]);
    lmax[0] = r;
  }
}

// E from the lower triangles of S and R (both symmetric).
__global__ void k_refine_E(int M, const double* __restrict__ S, const double* __restrict__ R,
                           const double* __restrict__ lam, const double* __restrict__ lmax, double rel_delta,
                           double* __restrict__ E, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double delta = rel_delta * lmax[0];
  for (int j = blockIdx.y; j < M; j += gridDim.y) {
    if (i >= M) continue;
    double e;
    int a = i > j ? i : j, b = i > j ? j : i;  // lower-triangle index
    double rij = R[GEP_IX(a, b, M)];
    if (i == j) {
      e = 0.5 * (1.0 - rij);
    } else {
      double gap = lam[j] - lam[i];
      if (fabs(gap) <= delta) e = -0.5 * rij;
      else e = (S[GEP_IX(a, b, M)] - lam[j] * rij) / gap;
    }
    E[GEP_IX(i, j, M)] = e;
  }
}

}  // namespace

size_t refine_ws_elems(int M) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  return 4 * r((size_t)M * M) + r((size_t)M) + 32;
}

// Af, Bf: full symmetric A and B (M x M, ld M).  X (ld ldx) refined in place, w <- lambda.
int refine_eigenpairs(gep_handle_t h, int M, const double* Af, const double* Bf, double* X, int ldx, double* w,
                      double* ws, int iters, int engine) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  double* T1 = ws;                        // A X, then B X, then X E
  double* S = T1 + r((size_t)M * M);
  double* R = S + r((size_t)M * M);
  double* E = R + r((size_t)M * M);
  double* lmax = E + r((size_t)M * M);
  for (int it = 0; it < iters; ++it) {
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Af, M, X, ldx, 0.0, T1, M, engine));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, X, ldx, T1, M, 0.0, S, M, engine));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Bf, M, X, ldx, 0.0, T1, M, engine));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, X, ldx, T1, M, 0.0, R, M, engine));
    k_rayleigh<<<1, 1024, 0, h->stream>>>(M, S, R, w, lmax, h->d_status);
    GEP_CHECK(check_launch(h));
    dim3 g((M + 255) / 256, M < 65535 ? M : 65535);
    k_refine_E<<<g, 256, 0, h->stream>>>(M, S, R, w, lmax, 1e-12, E, h->d_status);
    GEP_CHECK(check_launch(h));
    GEP_CHECK(copy_matrix(h, M, M, X, ldx, T1, M));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, T1, M, E, M, 1.0, X, ldx, engine));   // X <- X + X E
  }
  return GEP_OK;
}

}  // namespace gep
