// Elementwise helpers on column-major FP64 matrices (copies, fills, symmetric
// mirroring, transposition, non-finite scan, eigenvector sign convention).
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

__global__ void k_copy(int m, int n, const double* __restrict__ s, int lds, double* __restrict__ d,
                       int ldd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < n; j += gridDim.y)
    if (i < m) d[GEP_IX(i, j, ldd)] = s[GEP_IX(i, j, lds)];
}

__global__ void k_copy_lower(int m, const double* __restrict__ s, int lds, double* __restrict__ d,
                             int ldd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < m; j += gridDim.y)
    if (i < m && i >= j) d[GEP_IX(i, j, ldd)] = s[GEP_IX(i, j, lds)];
}

__global__ void k_set(int m, int n, double off, double dia, double* A, int lda) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < n; j += gridDim.y)
    if (i < m) A[GEP_IX(i, j, lda)] = (i == j) ? dia : off;
}

// 32 x 32 tiles through shared memory so both sides are coalesced.
__global__ void k_transpose(int m, int n, const double* __restrict__ s, int lds, double* __restrict__ d,
                            int ldd) {
  __shared__ double t[32][33];
  int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + threadIdx.x, j = j0 + r;
    if (i < m && j < n) t[r][threadIdx.x] = s[GEP_IX(i, j, lds)];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + threadIdx.x, i = i0 + r;  // d(j, i) = s(i, j)
    if (i < m && j < n) d[GEP_IX(j, i, ldd)] = t[threadIdx.x][r];
  }
}

// upper(A) := lower(A)^T, tile-wise (tile (bi, bj) with bi > bj mirrored into (bj, bi)).
__global__ void k_symmetrize(int M, double* A, int lda) {
  __shared__ double t[32][33];
  int bi = blockIdx.x, bj = blockIdx.y;
  if (bi < bj) return;
  int i0 = bi * 32, j0 = bj * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + threadIdx.x, j = j0 + r;
    if (i < M && j < M) t[r][threadIdx.x] = A[GEP_IX(i, j, lda)];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + threadIdx.x, i = i0 + r;  // write A(j, i) = A(i, j) for i > j
    if (i < M && j < M && i > j) A[GEP_IX(j, i, lda)] = t[threadIdx.x][r];
  }
}

// X = (W + W^T) / 2: tile (bi, bj) of W and the transposed tile (bj, bi), both read
// through shared memory so every access is coalesced.
__global__ void k_sym_part(int M, const double* __restrict__ W, int ldw, double* __restrict__ X, int ldx) {
  __shared__ double t[32][33];
  int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {  // t[c][r'] = W(j0 + r, i0 + c)
    int i = j0 + threadIdx.x, j = i0 + r;
    if (i < M && j < M) t[threadIdx.x][r] = W[GEP_IX(i, j, ldw)];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + threadIdx.x, j = j0 + r;  // X(i, j) = (W(i, j) + W(j, i)) / 2
    if (i < M && j < M) X[GEP_IX(i, j, ldx)] = 0.5 * (W[GEP_IX(i, j, ldw)] + t[r][threadIdx.x]);
  }
}

// Number of d_i <= 0 (or not finite): recorded as the numerical status when nonzero.
__global__ void k_count_nonpositive(int M, const double* __restrict__ d, int* st) {
  __shared__ int cnt;
  if (status_bad(st)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) c += (d[i] > 0.0 && isfinite(d[i])) ? 0 : 1;
  if (c) atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0 && cnt > 0) atomicCAS(st, 0, cnt);
}

// X(:, j) *= 1 / sqrt(d_j)
__global__ void k_scale_cols_rsqrt(int m, int n, const double* __restrict__ d, double* X, int ldx, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < n; j += gridDim.y)
    if (i < m) X[GEP_IX(i, j, ldx)] /= sqrt(d[j]);
}

__global__ void k_zero_upper(int M, double* A, int lda) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < M; j += gridDim.y)
    if (i < j) A[GEP_IX(i, j, lda)] = 0.0;
}

__global__ void k_scan_nonfinite(int M, const double* __restrict__ A, int lda, int* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < M; j += gridDim.y)
    if (i < M && i >= j && !isfinite(A[GEP_IX(i, j, lda)])) st[1] = GEP_ERR_NONFINITE;
}

// One warp per column: find the entry of largest magnitude (lowest row on ties) and
// flip the column so that entry is positive.
__global__ void k_sign(int M, int ncol, double* Y, int ldy, const int* __restrict__ st) {
  if (status_bad(st)) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ncol) return;
  double* y = Y + (size_t)warp * ldy;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = lane; i < M; i += 32) {
    double a = fabs(y[i]);
    if (a > best) { best = a; bi = i; }
  }
  for (int o = 16; o; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (bi >= M) return;
  double s = y[bi] < 0.0 ? -1.0 : 1.0;
  if (s < 0.0)
    for (int i = lane; i < M; i += 32) y[i] = -y[i];
}

inline dim3 grid2(int m, int n) { return dim3((m + 255) / 256, n < 65535 ? (n > 0 ? n : 1) : 65535); }

}  // namespace

int copy_matrix(gep_handle_t h, int m, int n, const double* src, int lds, double* dst, int ldd) {
  if (m <= 0 || n <= 0) return GEP_OK;
  k_copy<<<grid2(m, n), 256, 0, h->stream>>>(m, n, src, lds, dst, ldd);
  return check_launch(h);
}

int copy_lower(gep_handle_t h, int M, const double* src, int lds, double* dst, int ldd) {
  if (M <= 0) return GEP_OK;
  k_copy_lower<<<grid2(M, M), 256, 0, h->stream>>>(M, src, lds, dst, ldd);
  return check_launch(h);
}

int set_matrix(gep_handle_t h, int m, int n, double off, double dia, double* A, int lda) {
  if (m <= 0 || n <= 0) return GEP_OK;
  k_set<<<grid2(m, n), 256, 0, h->stream>>>(m, n, off, dia, A, lda);
  return check_launch(h);
}

int transpose(gep_handle_t h, int m, int n, const double* src, int lds, double* dst, int ldd) {
  if (m <= 0 || n <= 0) return GEP_OK;
  dim3 g((m + 31) / 32, (n + 31) / 32);
  k_transpose<<<g, dim3(32, 8), 0, h->stream>>>(m, n, src, lds, dst, ldd);
  return check_launch(h);
}

int symmetrize_lower(gep_handle_t h, int M, double* A, int lda) {
  if (M <= 1) return GEP_OK;
  dim3 g((M + 31) / 32, (M + 31) / 32);
  k_symmetrize<<<g, dim3(32, 8), 0, h->stream>>>(M, A, lda);
  return check_launch(h);
}

int symmetric_part(gep_handle_t h, int M, const double* W, int ldw, double* X, int ldx) {
  if (M <= 0) return GEP_OK;
  dim3 g((M + 31) / 32, (M + 31) / 32);
  k_sym_part<<<g, dim3(32, 8), 0, h->stream>>>(M, W, ldw, X, ldx);
  return check_launch(h);
}

int scale_cols_rsqrt_checked(gep_handle_t h, int m, int n, const double* d, double* X, int ldx) {
  if (m <= 0 || n <= 0) return GEP_OK;
  k_count_nonpositive<<<1, 256, 0, h->stream>>>(n, d, h->d_status);
  GEP_CHECK(check_launch(h));
  k_scale_cols_rsqrt<<<grid2(m, n), 256, 0, h->stream>>>(m, n, d, X, ldx, h->d_status);
  return check_launch(h);
}

int zero_upper(gep_handle_t h, int M, double* A, int lda) {
  if (M <= 1) return GEP_OK;
  k_zero_upper<<<grid2(M, M), 256, 0, h->stream>>>(M, A, lda);
  return check_launch(h);
}

int scan_nonfinite(gep_handle_t h, int M, const double* A, int lda) {
  if (M <= 0) return GEP_OK;
  k_scan_nonfinite<<<grid2(M, M), 256, 0, h->stream>>>(M, A, lda, h->d_status);
  return check_launch(h);
}

int sign_convention(gep_handle_t h, int M, int ncol, double* Y, int ldy) {
  if (M <= 0 || ncol <= 0) return GEP_OK;
  int warps_per_block = 8;
  k_sign<<<(ncol + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, h->stream>>>(
      M, ncol, Y, ldy, h->d_status);
  return check_launch(h);
}

}  // namespace gep
