// Block-Jacobi SEP solver (GEP_SEP_JACOBI): the parallel block-Jacobi method the paper names
// as future work (section 6), a third SEP variant beside the 1-stage and 2-stage
// tridiagonal routes.  C (order M, symmetric) is cut into column blocks of NBJ; a sweep
// takes every pair of blocks once, in round-robin order, so the nblk/2 pairs of a round are
// disjoint and are treated in parallel:
//   1. each pair (I, J) diagonalises its 2NBJ x 2NBJ submatrix [C_II C_IJ; C_JI C_JJ] = Q D Q^T
//      exactly with the one-CTA Jacobi solver (one CTA per pair);
//   2. C <- Q^T C Q and V <- V Q, Q the block rotation of all pairs: first the columns I u J
//      of C and V (C(:, IJ) Q), then the rows (Q^T C(IJ, :)).
// Sweeps continue until the off-diagonal part of C is ~1e-14 of C (FP64 level, checked on
// the host after each sweep; a fixed number of sweeps while the stream is being captured).
// The eigenvalues are diag(C), sorted ascending with the columns of V.  Work per sweep is
// about 8 M^3 FP64 flops on the CUDA cores (against ~9 M^3 for the whole tridiagonal route),
// so on this part the variant pays only for small orders; it exists as the paper's third
// SEP method and as the route of the small batched pencils.
#include <math.h>

#include "cta_eig.cuh"

namespace gep {
namespace {

constexpr int NBJ = 32;          // block width: subproblems of order <= 64
constexpr int KSUB = 2 * NBJ;

__device__ __forceinline__ int bj_block_size(int M, int I) { return min(NBJ, M - I * NBJ); }

// Players of a round-robin round r over n (even) blocks: pair t = (player(t), player(n-1-t)),
// player 0 fixed, the others rotating by one place per round.
__device__ __forceinline__ int bj_player(int pos, int r, int n) { return pos == 0 ? 0 : ((pos - 1 + r) % (n - 1)) + 1; }

// Pair t of round r: its two blocks and the order k of its submatrix (0: a dummy pair).
// A matrix of one block (M <= NBJ) is its own subproblem (paired with the dummy block).
__device__ __forceinline__ int bj_pair(int M, int nreal, int n, int r, int t, int& I, int& J) {
  int a = bj_player(t, r, n), b = bj_player(n - 1 - t, r, n);
  I = min(a, b);
  J = max(a, b);
  if (J >= nreal) return (nreal == 1 && I == 0) ? bj_block_size(M, 0) : 0;
  return bj_block_size(M, I) + bj_block_size(M, J);
}

// global index of subproblem row/column i of the pair (I, J)
__device__ __forceinline__ int bj_index(int M, int I, int J, int i) {
  const int kI = bj_block_size(M, I);
  return i < kI ? I * NBJ + i : J * NBJ + (i - kI);
}

// 1. one CTA per pair: gather the submatrix, diagonalise it, leave Q (k x k) in Qs.
__global__ void __launch_bounds__(256) k_bj_solve(int M, int nreal, int n, int r, const double* __restrict__ C,
                                                  int ldc, double* __restrict__ scratch, const int* st) {
  __shared__ CtaEigShared sh;
  if (status_bad(st)) return;
  int I, J;
  const int k = bj_pair(M, nreal, n, r, blockIdx.x, I, J);
  if (k == 0) return;
  double* L = scratch + (size_t)blockIdx.x * 3 * KSUB * KSUB;
  double* Cm = L + KSUB * KSUB;
  double* V = Cm + KSUB * KSUB;  // Q of this pair (ld k)
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int p = idx % k, q = idx / k;
    L[idx] = (p == q) ? 1.0 : 0.0;
    Cm[idx] = C[GEP_IX(bj_index(M, I, J, p), bj_index(M, I, J, q), ldc)];
  }
  __syncthreads();
  cta_pencil_eig(k, L, Cm, V, sh, false);
}

// 2a. X(:, IJ) <- X(:, IJ) Q for X = C and X = V: CTA (16 rows, one pair).
__global__ void __launch_bounds__(256) k_bj_cols(int M, int nreal, int n, int r, double* __restrict__ C, int ldc,
                                                 double* __restrict__ V, int ldv, const double* __restrict__ scratch,
                                                 const int* st) {
  __shared__ double Qs[KSUB * KSUB];
  __shared__ double T[16][KSUB + 1];
  if (status_bad(st)) return;
  int I, J;
  const int k = bj_pair(M, nreal, n, r, blockIdx.y, I, J);
  if (k == 0) return;
  const double* Q = scratch + (size_t)blockIdx.y * 3 * KSUB * KSUB + 2 * KSUB * KSUB;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) Qs[idx] = Q[idx];
  const int r0 = blockIdx.x * 16;
  for (int which = 0; which < 2; ++which) {
    double* X = which ? V : C;
    const int ldx = which ? ldv : ldc;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 16 * k; idx += blockDim.x) {
      const int i = idx % 16, c = idx / 16;
      T[i][c] = (r0 + i < M) ? X[GEP_IX(r0 + i, bj_index(M, I, J, c), ldx)] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 16 * k; idx += blockDim.x) {
      const int i = idx % 16, c = idx / 16;
      if (r0 + i >= M) continue;
      double s = 0.0;
      for (int p = 0; p < k; ++p) s = fma(T[i][p], Qs[p + c * k], s);
      X[GEP_IX(r0 + i, bj_index(M, I, J, c), ldx)] = s;
    }
  }
}

// 2b. C(IJ, :) <- Q^T C(IJ, :): CTA (16 columns, one pair).
__global__ void __launch_bounds__(256) k_bj_rows(int M, int nreal, int n, int r, double* __restrict__ C, int ldc,
                                                 const double* __restrict__ scratch, const int* st) {
  __shared__ double Qs[KSUB * KSUB];
  __shared__ double T[KSUB][17];
  if (status_bad(st)) return;
  int I, J;
  const int k = bj_pair(M, nreal, n, r, blockIdx.y, I, J);
  if (k == 0) return;
  const double* Q = scratch + (size_t)blockIdx.y * 3 * KSUB * KSUB + 2 * KSUB * KSUB;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) Qs[idx] = Q[idx];
  const int c0 = blockIdx.x * 16;
  for (int idx = threadIdx.x; idx < 16 * k; idx += blockDim.x) {
    const int p = idx % k, j = idx / k;
    T[p][j] = (c0 + j < M) ? C[GEP_IX(bj_index(M, I, J, p), c0 + j, ldc)] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 16 * k; idx += blockDim.x) {
    const int p = idx % k, j = idx / k;
    if (c0 + j >= M) continue;
    double s = 0.0;
    for (int q = 0; q < k; ++q) s = fma(Qs[q + p * k], T[q][j], s);
    C[GEP_IX(bj_index(M, I, J, p), c0 + j, ldc)] = s;
  }
}

// out[0] += sum of squares of the off-diagonal entries, out[1] += of all entries.
__global__ void k_bj_offnorm(int M, const double* __restrict__ C, int ldc, double* out, const int* st) {
  __shared__ double red[2][8];
  if (status_bad(st)) return;
  double off = 0.0, tot = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < M; j += gridDim.y) {
    if (i >= M) continue;
    const double x = C[GEP_IX(i, j, ldc)];
    tot += x * x;
    if (i != j) off += x * x;
  }
  for (int o = 16; o; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = off;
    red[1][threadIdx.x >> 5] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
  }
}

// w ascending from diag(C), Z(:, rank) = V(:, i): rank of i = #{j: d_j < d_i, or equal and j < i}.
__global__ void k_bj_sort(int M, const double* __restrict__ C, int ldc, const double* __restrict__ V, int ldv,
                          double* __restrict__ w, double* __restrict__ Z, int ldz, const int* st) {
  if (status_bad(st)) return;
  const int i = blockIdx.x;
  const double di = C[GEP_IX(i, i, ldc)];
  __shared__ int rank_s;
  int cnt = 0;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const double dj = C[GEP_IX(j, j, ldc)];
    cnt += (dj < di || (dj == di && j < i)) ? 1 : 0;
  }
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (threadIdx.x == 0) rank_s = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicAdd(&rank_s, cnt);
  __syncthreads();
  const int rk = rank_s;
  if (threadIdx.x == 0) w[rk] = di;
  for (int rr = threadIdx.x; rr < M; rr += blockDim.x) Z[GEP_IX(rr, rk, ldz)] = V[GEP_IX(rr, i, ldv)];
}

}  // namespace

size_t jacobi_ws_elems(int M) {
  const size_t nblk = (size_t)(M + NBJ - 1) / NBJ + 1;
  return 2 * (size_t)M * M + (nblk / 2 + 1) * 3 * KSUB * KSUB + 64;
}

// Block-Jacobi eigensolver of the symmetric C (lower triangle read; overwritten): w
// ascending, Z its orthonormal eigenvectors (ldz; Z = nullptr: eigenvalues only).
// ws: jacobi_ws_elems(M) doubles.
int jacobi_sep(gep_handle_t h, int M, double* C, int ldc, double* w, double* Z, int ldz, double* ws) {
  if (M <= 0) return GEP_OK;
  const int nreal = (M + NBJ - 1) / NBJ, n = nreal + (nreal & 1), npairs = n / 2;
  double* V = ws;                              // M x M, ld M
  if (!Z) {                                    // eigenvalues only: the sorted vectors go here
    Z = ws + (size_t)M * M;
    ldz = M;
  }
  double* scratch = ws + 2 * (size_t)M * M;    // per pair: L, Cm, Q (KSUB^2 each)
  double* norms = scratch + (size_t)(npairs + 1) * 3 * KSUB * KSUB;  // off, total
  GEP_CHECK(symmetrize_lower(h, M, C, ldc));
  GEP_CHECK(set_matrix(h, M, M, 0.0, 1.0, V, M));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return GEP_ERR_CUDA;
  const bool adaptive = cs == cudaStreamCaptureStatusNone;
  const int max_sweeps = adaptive ? 30 : 12;
  const dim3 gn((M + 255) / 256, M < 1024 ? M : 1024);
  for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
    if (adaptive) {
      GEP_CUDA(cudaMemsetAsync(norms, 0, 2 * sizeof(double), h->stream));
      k_bj_offnorm<<<gn, 256, 0, h->stream>>>(M, C, ldc, norms, h->d_status);
      GEP_CHECK(check_launch(h));
      double nv[2] = {0.0, 0.0};
      GEP_CUDA(cudaMemcpyAsync(nv, norms, sizeof(nv), cudaMemcpyDeviceToHost, h->stream));
      GEP_CUDA(cudaStreamSynchronize(h->stream));
      if (!(nv[0] > 1e-28 * nv[1])) break;  // also stops on NaN
    }
    for (int r = 0; r < n - 1; ++r) {
      k_bj_solve<<<npairs, 256, 0, h->stream>>>(M, nreal, n, r, C, ldc, scratch, h->d_status);
      GEP_CHECK(check_launch(h));
      k_bj_cols<<<dim3((M + 15) / 16, npairs), 256, 0, h->stream>>>(M, nreal, n, r, C, ldc, V, M, scratch,
                                                                    h->d_status);
      GEP_CHECK(check_launch(h));
      k_bj_rows<<<dim3((M + 15) / 16, npairs), 256, 0, h->stream>>>(M, nreal, n, r, C, ldc, scratch, h->d_status);
      GEP_CHECK(check_launch(h));
    }
  }
  k_bj_sort<<<M, 256, 0, h->stream>>>(M, C, ldc, V, M, w, Z, ldz, h->d_status);
  return check_launch(h);
}

}  // namespace gep
