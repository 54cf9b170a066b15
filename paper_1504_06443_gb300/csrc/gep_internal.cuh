// Internal declarations shared by the solver's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "gep.h"

#define GEP_IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

struct gep_handle_s {
  cudaStream_t stream = nullptr;
  int* d_status = nullptr;   // [0] numerical info, [1] error code (timeouts etc.)
  char* ws = nullptr;        // caller workspace
  size_t ws_bytes = 0;
  char* eng_ws = nullptr;    // scratch of the split-BF16 product engine
  size_t eng_bytes = 0;
  double* d_splitk = nullptr;  // handle-owned partial sums of split-K FP64 products
  size_t splitk_bytes = 0;
  long long launches = 0;
  int sm_count = 152;
  // bounded device-side waits: their limit, and a test hook that drops the progress
  // releases of one bulge-chasing sweep so that the waits behind it run out
  unsigned long long wait_limit_ns = 4000000000ull;
  int fault_drop_sweep = -1;
  // test hook: rows per CTA of the single-launch panel QR (64, 128 or 256), -1 for the
  // one-launch-per-column kernel, 0 for the automatic choice
  int pqr_rows = 0;
  int band_group_min = -1;  // trailing order from which S1b takes panels in groups of four (-1: default)
  int magic = 0x6e70;
  cudaEvent_t ev[8] = {};
  cudaEvent_t ev_band = nullptr;  // between full->band and bulge chasing (two-stage, timers on)
  // second stream of the solve: the dense Q2 tiles are built there while the tridiagonal
  // eigensolver runs on the handle's stream (fork/join by events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool band_recorded = false;
  bool timers_recorded = false;
  // optional per-launch timing of the tensor-core product kernel
  int prof_on = 0;
  int prof_cap = 0, prof_used = 0;
  long long prof_skipped = 0;
  cudaEvent_t* prof_ev = nullptr;   // 2 * prof_cap events
  double* prof_flops = nullptr;     // tensor flops of each recorded launch
  double* prof_f64eq = nullptr;     // FP64-equivalent flops of each recorded launch
  int* prof_mnk = nullptr;          // m, n, k of each recorded launch
  // batched solves: child handles, one per concurrent stream (created on first use)
  int nchild = 0;
  gep_handle_s* child[64] = {};
  cudaStream_t child_stream[64] = {};
  cudaEvent_t child_done[64] = {};
  cudaEvent_t fork_ev = nullptr;
  int* d_batch_info = nullptr;  // 2 ints per pencil of the last batched call
  int* d_small_next = nullptr;  // work-queue counter of the one-CTA small-pencil launch
  int batch_count = 0;
  int refine_steps = 0;  // FP64 refinement steps taken by the last mixed-precision solve
};

namespace gep {

// Bump allocator over the caller's workspace.
struct Arena {
  char* base;
  size_t cap, off = 0;
  bool ok = true;
  Arena(void* b, size_t c) : base((char*)b), cap(c) {}
  template <class T>
  T* take(size_t n) {
    size_t a = (off + 255) & ~(size_t)255;
    size_t need = a + n * sizeof(T);
    if (need > cap || base == nullptr) { ok = false; off = need; return nullptr; }
    off = need;
    return (T*)(base + a);
  }
};

// Counting-only arena: used by workspace queries to size the same carving.
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Kernel attributes (the dynamic shared-memory limit) belong to a device context, so
// one-time settings are made once per device: `mask` (one per call site) records the
// devices already done.  Returns true on the first call for the current device.
inline bool first_use_on_device(unsigned long long& mask) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return true;
  const unsigned long long bit = 1ull << d;
  if (mask & bit) return false;
  mask |= bit;
  return true;
}

inline int check_launch(gep_handle_t h) {
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "gep: kernel launch failed: %s\n", cudaGetErrorString(e));
    return GEP_ERR_CUDA;
  }
  return GEP_OK;
}

#define GEP_CHECK(x)                        \
  do {                                      \
    int _r = (x);                           \
    if (_r != GEP_OK) return _r;            \
  } while (0)

#define GEP_CUDA(x)                                                                  \
  do {                                                                               \
    cudaError_t _e = (x);                                                            \
    if (_e != cudaSuccess) {                                                         \
      fprintf(stderr, "gep: %s failed: %s (%s:%d)\n", #x, cudaGetErrorString(_e), __FILE__, \
              __LINE__);                                                             \
      return GEP_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)

// ---- dense contraction engines (gemm_f64.cu, gemm_oz.cu) ----
// Structure of op(A) a product may exploit: rows [128 r, 128 r + 128) of op(A) are exactly
// zero outside the columns [lo[r], hi[r]) for r < n (the other row blocks are dense).  The
// split-BF16 engine skips the zero part (same result bits); the FP64 engine ignores it.
constexpr int OZ_KR_MAX = 32;
struct OzKRange {
  int n = 0;
  int lo[OZ_KR_MAX], hi[OZ_KR_MAX];
};
// C = alpha op(A) op(B) + beta C; uplo 'L' restricts computation/storage to i >= j.
int dgemm(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
          int engine, const OzKRange* kr = nullptr);
int dgemm_f64(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc);
int dgemm_oz(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
             int levels, const OzKRange* kr = nullptr);
size_t oz_workspace_bytes(int m, int n, int k);
// Digit planes of a symmetric operand (the lower triangle of an m x m matrix), split once
// for all its K panels so that several products can share them (the two C22 products of a
// panel pair in the full -> band reduction).  Panel p: planes + p * S * m * OZ_SYM_KP,
// its row exponent fields at ea + p * m.
constexpr int OZ_SYM_KP = 4096;
struct OzSymPlanes {
  unsigned short* planes = nullptr;
  int* ea = nullptr;
  int m = 0, levels = 0;
};
size_t oz_sym_planes_bytes(int m, int levels);
int oz_split_sym(gep_handle_t h, int m, const double* A, int lda, int levels, void* buf, size_t bytes,
                 OzSymPlanes* P);
// C (m - row0 x n) = alpha A(row0:m, 0:m) B + beta C with A given by its planes P (B is
// m x n, column-major, ld ldb): rows row0.. of the symmetric operand against all of K.
int dgemm_oz_sym_planes(gep_handle_t h, const OzSymPlanes& P, int row0, int n, double alpha, const double* B,
                        int ldb, double beta, double* C, int ldc);

// ---- small dense helpers (blas_util.cu) ----
int copy_matrix(gep_handle_t h, int m, int n, const double* src, int lds, double* dst, int ldd);
int copy_lower(gep_handle_t h, int M, const double* src, int lds, double* dst, int ldd);
int set_matrix(gep_handle_t h, int m, int n, double offdiag, double diag, double* A, int lda);
int symmetrize_lower(gep_handle_t h, int M, double* A, int lda);  // upper := lower^T
int transpose(gep_handle_t h, int m, int n, const double* src, int lds, double* dst, int ldd);
int zero_upper(gep_handle_t h, int M, double* A, int lda);          // strict upper := 0
int symmetric_part(gep_handle_t h, int M, const double* W, int ldw, double* X, int ldx);  // X = (W + W^T) / 2
// X(:, j) *= d_j^-1/2 (m x n); first records the number of d_j <= 0 as numerical status k > 0
int scale_cols_rsqrt_checked(gep_handle_t h, int m, int n, const double* d, double* X, int ldx);
int scan_nonfinite(gep_handle_t h, int M, const double* A, int lda);  // lower triangle

// ---- triangular building blocks (tri.cu) ----
// Inverts every nb x nb diagonal block of the lower triangular L into invD
// (block b at invD + b*nb*nb, column-major nb x nb, lower; ragged last block padded
// with identity).
int tri_inv_diag_blocks(gep_handle_t h, int M, const double* L, int ldl, double* invD, int nb);
// X (M x n) := L^-1 X  (left, lower, no transpose)
int trsm_lln(gep_handle_t h, int M, int n, const double* L, int ldl, const double* invD, int nb,
             double* X, int ldx, double* tmp, int engine);
// X (M x n) := L^-T X  (left, lower, transpose)
int trsm_llt(gep_handle_t h, int M, int n, const double* L, int ldl, const double* invD, int nb,
             double* X, int ldx, double* tmp, int engine);
size_t trsm_tmp_elems(int M, int n, int nb);

// ---- stages ----
int cholesky(gep_handle_t h, int M, double* B, int ldb, double* ws_invdiag, int engine);
int reduce_twosided(gep_handle_t h, int M, double* A, int lda, const double* L, int ldl,
                    const double* invD, double* X, double* tmp, int engine);
int reduce_explicit_inv(gep_handle_t h, int M, double* A, int lda, double* L, int ldl,
                        const double* invD, double* X, double* tmp, int engine);
int tridiag_1stage(gep_handle_t h, int M, double* C, int ldc, double* d, double* e, double* tau,
                   double* ws, size_t ws_elems, int engine);
size_t tridiag_ws_elems(int M);
int backtransform_q(gep_handle_t h, int M, int ncol, const double* C, int ldc, const double* tau,
                    double* Z, int ldz, double* ws, size_t ws_elems, int engine, int off = 1);
// T (nb x nb, upper) of the block reflector whose Gram matrix is G = V^T V (backtrans.cu).
int larft_rec(gep_handle_t h, int nb, const double* G, int ldg, const double* tau, double* T, int ldt,
              double* tmp);
// two-stage SEP path (band.cu)
size_t q2_elems(int M, int b);
size_t band_ws_elems(int M, int b);
int band_reduce(gep_handle_t h, int M, double* C, int ldc, int b, double* tau1, double* ws, size_t ws_elems,
                int eng);
int band_to_tridiag(gep_handle_t h, int M, const double* C, int ldc, int b, double* d, double* e, double* q2,
                    double* ws, size_t ws_elems);
size_t q2_tile_ws_elems(int M, int b);
int apply_q2(gep_handle_t h, int M, int b, const double* q2, double* Z, int ldz, int ncol, int engine, double* ws,
             size_t ws_elems, const double* U_all = nullptr);
// every dense Q2 tile at once (tensor-core engines), e.g. on a second stream
size_t q2_all_tiles_elems(int M, int b);
int build_q2_tiles(gep_handle_t h, cudaStream_t stream, int M, int b, const double* q2, double* U);
size_t backtransform_ws_elems(int M, int ncol);
int tridiag_eig_dc(gep_handle_t h, int M, const double* d, const double* e, double* w, double* Z,
                   int ldz, double* ws, size_t ws_elems, int engine);
size_t dc_ws_bytes(int M);
int tridiag_eig_bisect(gep_handle_t h, int M, const double* d, const double* e, double* w, int n = -1);
int sign_convention(gep_handle_t h, int M, int ncol, double* Y, int ldy);
size_t refine_ws_elems(int M);
int refine_eigenpairs(gep_handle_t h, int M, const double* Af, const double* Bf, double* X, int ldx, double* w,
                      double* ws, int iters, int engine);
size_t adjoint_ws_elems(int M, int no);
int adjoint(gep_handle_t h, int M, int no, const double* w, const double* Y, int ldy, const double* lbar,
            const double* W, int ldw, double* Abar, double* Bbar, int ldab, double* ws, int engine);

// block-Jacobi SEP solver (jacobi.cu)
size_t jacobi_ws_elems(int M);
int jacobi_sep(gep_handle_t h, int M, double* C, int ldc, double* w, double* Z, int ldz, double* ws);

// small pencils of a batched solve, one CTA each in one persistent launch (batched.cu)
constexpr int SMALL_MAX = 128;         // largest order solved by one CTA
constexpr int SMALL_PER_LAUNCH = 256;  // pencils whose table one launch carries in its parameters
size_t small_gep_scratch_bytes(int ctas);
int small_gep_batched(gep_handle_t h, cudaStream_t s, int count, const int* M, double* const* A, double* const* B,
                      double* const* w, double* const* Y, const int* order, double* scratch, int ctas, int* next,
                      int* info);

// Kernel-side helper: returns true when an earlier stage recorded an error.
__device__ __forceinline__ bool status_bad(const int* st) { return st != nullptr && (st[0] != 0 || st[1] != 0); }

}  // namespace gep
