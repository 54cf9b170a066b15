// FP64 FMA matrix product C = alpha op(A) op(B) + beta C (column-major); op(A) may also
// be a symmetric matrix given by its lower triangle (transa 'S', m = k).
//
// The dense contraction under every blocked stage (trailing updates of the
// Cholesky factorisation, triangular solves, the SYR2K update of the
// tridiagonalisation, the compact-WY back-transformation and the divide-and-
// conquer merge).  64 x 64 output tile per 256-thread CTA, 16-deep k slices
// staged through shared memory, 4 x 4 register micro-tile per thread; the row
// index is the fast thread index so C is read and written coalesced.
// uplo 'L' skips tiles strictly above the diagonal and stores only i >= j
// (SYRK / SYR2K shaped updates of a symmetric lower triangle).
#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool TA, bool TB, bool SA = false>
__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int k, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb, double beta,
                                               double* __restrict__ C, int ldc, int lower,
                                               const int* __restrict__ st) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (lower && bi < bj) return;
  if (status_bad(st)) return;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = bi * BM, col0 = bj * BN;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + r * 256;
      int i, kk;
      if (!TA) { i = idx & 63; kk = idx >> 6; }
      else { kk = idx & 15; i = idx >> 4; }
      int gi = row0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < m && gk < k) {
        if (SA) v = gi >= gk ? A[GEP_IX(gi, gk, lda)] : A[GEP_IX(gk, gi, lda)];  // symmetric, lower stored
        else v = TA ? A[GEP_IX(gk, gi, lda)] : A[GEP_IX(gi, gk, lda)];
      }
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + r * 256;
      int j, kk;
      if (!TB) { kk = idx & 15; j = idx >> 4; }
      else { j = idx & 63; kk = idx >> 6; }
      int gj = col0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < n && gk < k) v = TB ? B[GEP_IX(gj, gk, ldb)] : B[GEP_IX(gk, gj, ldb)];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int j = col0 + ty + 16 * c;
    if (j >= n) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i = row0 + tx + 16 * r;
      if (i >= m || (lower && i < j)) continue;
      double v = alpha * acc[r][c];
      if (beta != 0.0) v = fma(beta, C[GEP_IX(i, j, ldc)], v);
      C[GEP_IX(i, j, ldc)] = v;
    }
  }
}

// Split-K partial products for small outputs with long K: CTA (bi, bj, z) computes the
// 64 x 64 tile over k in [z*kc, (z+1)*kc) into P[z] (m x n, leading dimension m).
template <bool TA, bool TB, bool SA = false>
__global__ void __launch_bounds__(256) k_dgemm_splitk(int m, int n, int k, int kc, const double* __restrict__ A,
                                                      int lda, const double* __restrict__ B, int ldb,
                                                      double* __restrict__ P, const int* __restrict__ st) {
  if (status_bad(st)) return;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int bi = blockIdx.x, bj = blockIdx.y, z = blockIdx.z;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = bi * BM, col0 = bj * BN;
  const int kb = z * kc, ke = min(k, kb + kc);
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + r * 256;
      int i, kk;
      if (!TA) { i = idx & 63; kk = idx >> 6; }
      else { kk = idx & 15; i = idx >> 4; }
      int gi = row0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < m && gk < ke) {
        if (SA) v = gi >= gk ? A[GEP_IX(gi, gk, lda)] : A[GEP_IX(gk, gi, lda)];
        else v = TA ? A[GEP_IX(gk, gi, lda)] : A[GEP_IX(gi, gk, lda)];
      }
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + r * 256;
      int j, kk;
      if (!TB) { kk = idx & 15; j = idx >> 4; }
      else { j = idx & 63; kk = idx >> 6; }
      int gj = col0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < n && gk < ke) v = TB ? B[GEP_IX(gj, gk, ldb)] : B[GEP_IX(gk, gj, ldb)];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  double* Pz = P + (size_t)z * m * n;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int j = col0 + ty + 16 * c;
    if (j >= n) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int i = row0 + tx + 16 * r;
      if (i < m) Pz[(size_t)i + (size_t)j * m] = acc[r][c];
    }
  }
}

// C = alpha * sum_z P[z] + beta * C, summed in a fixed order (deterministic).
__global__ void k_splitk_reduce(int m, int n, int nz, const double* __restrict__ P, double alpha, double beta,
                                double* __restrict__ C, int ldc, int lower, const int* __restrict__ st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= m || j >= n || (lower && i < j)) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += P[(size_t)z * m * n + (size_t)i + (size_t)j * m];
  double v = alpha * s;
  if (beta != 0.0) v = fma(beta, C[GEP_IX(i, j, ldc)], v);
  C[GEP_IX(i, j, ldc)] = v;
}

__global__ void k_scale(int m, int n, double beta, double* C, int ldc, int lower,
                        const int* __restrict__ st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= m || j >= n || (lower && i < j)) return;
  C[GEP_IX(i, j, ldc)] = beta == 0.0 ? 0.0 : beta * C[GEP_IX(i, j, ldc)];
}

}  // namespace

int dgemm_f64(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  if (m <= 0 || n <= 0) return GEP_OK;
  int lower = (uplo == 'L' || uplo == 'l');
  if (k <= 0 || alpha == 0.0) {
    if (beta == 1.0) return GEP_OK;
    dim3 g((m + 255) / 256, n);
    k_scale<<<g, 256, 0, h->stream>>>(m, n, beta, C, ldc, lower, h->d_status);
    return check_launch(h);
  }
  bool TA = (ta == 'T' || ta == 't'), TB = (tb == 'T' || tb == 't');
  const bool SA = (ta == 'S' || ta == 's');  // A symmetric (m x m, k = m), lower triangle stored
  if (SA && (TB || k != m)) return GEP_ERR_UNSUPPORTED;
  dim3 grid((m + BM - 1) / BM, (n + BN - 1) / BN);
  long long tiles = (long long)grid.x * grid.y;
  // A few output tiles with a long K leave most SMs idle: split K across CTAs.
  if (tiles < h->sm_count && k >= 1024 && h->d_splitk != nullptr) {
    long long nz = (2LL * h->sm_count + tiles - 1) / tiles;
    nz = nz < k / 64 ? nz : k / 64;  // slices of at least 64: the FP64 pipe, not the loads, is the limit
    long long cap = (long long)(h->splitk_bytes / (sizeof(double) * (size_t)m * n));
    nz = nz < cap ? nz : cap;
    if (nz >= 2) {
      int kc = (int)((k + nz - 1) / nz);
      kc = (kc + BK - 1) / BK * BK;
      int z = (k + kc - 1) / kc;
      dim3 g3(grid.x, grid.y, z);
      double* P = h->d_splitk;
      if (SA) k_dgemm_splitk<false, false, true><<<g3, 256, 0, h->stream>>>(m, n, k, kc, A, lda, B, ldb, P, h->d_status);
      else if (!TA && !TB) k_dgemm_splitk<false, false><<<g3, 256, 0, h->stream>>>(m, n, k, kc, A, lda, B, ldb, P, h->d_status);
      else if (!TA && TB) k_dgemm_splitk<false, true><<<g3, 256, 0, h->stream>>>(m, n, k, kc, A, lda, B, ldb, P, h->d_status);
      else if (TA && !TB) k_dgemm_splitk<true, false><<<g3, 256, 0, h->stream>>>(m, n, k, kc, A, lda, B, ldb, P, h->d_status);
      else k_dgemm_splitk<true, true><<<g3, 256, 0, h->stream>>>(m, n, k, kc, A, lda, B, ldb, P, h->d_status);
      GEP_CHECK(check_launch(h));
      dim3 gr((m + 255) / 256, n);
      k_splitk_reduce<<<gr, 256, 0, h->stream>>>(m, n, z, P, alpha, beta, C, ldc, lower, h->d_status);
      return check_launch(h);
    }
  }
  if (SA)
    k_dgemm<false, false, true><<<grid, 256, 0, h->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower,
                                                              h->d_status);
  else if (!TA && !TB)
    k_dgemm<false, false><<<grid, 256, 0, h->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, h->d_status);
  else if (!TA && TB)
    k_dgemm<false, true><<<grid, 256, 0, h->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, h->d_status);
  else if (TA && !TB)
    k_dgemm<true, false><<<grid, 256, 0, h->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, h->d_status);
  else
    k_dgemm<true, true><<<grid, 256, 0, h->stream>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, h->d_status);
  return check_launch(h);
}

int dgemm(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
          int engine, const OzKRange* kr) {
  // Products too small to fill 128 x 64 tensor-core tiles stay on the FP64 FMA kernel, and
  // so do outputs of one or two tiles with a long K (split K over many CTAs there).
  bool big = m >= 128 && n >= 64 && k >= 16;
  const long long oz_tiles = (long long)((m + 127) / 128) * ((n + 63) / 64);
  if (big && oz_tiles <= 2 && k >= 2048) big = false;
  if (engine == GEP_PREC_FP64_EMULATED && big)
    return dgemm_oz(h, ta, tb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 9, kr);
  if (engine == GEP_PREC_MIXED_REFINED && big)
    return dgemm_oz(h, ta, tb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 4, kr);
  return dgemm_f64(h, ta, tb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

}  // namespace gep
