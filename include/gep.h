/*
 * gep.h - C ABI of a one-GPU (sm_103a) dense solver for the real symmetric-
 * definite generalized eigenproblem
 *
 *     A y_k = lambda_k B y_k,   A Y = B Y Lambda,   Y^T B Y = I      (Eq. 1, Eq. 2)
 *
 * organised as Imachi & Hoshi decompose it (section 3.1): a *reducer*
 * (Cholesky B = L L^T, Eq. 4 with L = U^T; two-sided reduction C = L^-1 A L^-T,
 * Eq. 5; back-substitution Y = L^-T Z, Eq. 6) and an *SEP solver* (reduction
 * of C to tridiagonal form, "TRD" in Table 3; a tridiagonal divide-and-conquer
 * eigensolver, "D&C"; the Householder back-transformation, "BACK").  Each
 * stage offers the variants of the paper's hybrid workflows (Table 1).
 *
 * Conventions shared by every entry point
 *  - Matrices are FP64, column-major, element (i,j) at X[i + j*ld], ld >= max(1,M).
 *    Symmetric inputs are read from their LOWER triangle only.
 *  - Every matrix/vector pointer is DEVICE memory owned by the caller; the library
 *    never frees it.  Inputs documented as "overwritten" are modified in place.
 *  - All calls enqueue work on the handle's stream and return without waiting
 *    for the GPU, except gep_get_info() and the host-buffer variant
 *    gep_solve_host(), which synchronise the stream.
 *  - Return value: GEP_OK (0) on success; -i if argument i (1-based) is illegal
 *    (checked on the host before anything is enqueued, LAPACK info < 0
 *    convention); GEP_ERR_* codes below for other failures.
 *  - Numerical status (B not positive definite, D&C not converged) and device-side
 *    failures (non-finite input, a bounded wait that gave up: GEP_ERR_NONFINITE,
 *    GEP_ERR_TIMEOUT) are written to device memory and read with gep_get_info();
 *    once it is non-zero, later stages of the same handle become no-ops until
 *    gep_reset_info().
 */
#ifndef GEP_H
#define GEP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gep_handle_s* gep_handle_t;

/* Return codes (negative values -1..-20 are "illegal argument i"). */
#define GEP_OK 0
#define GEP_ERR_CUDA (-100)        /* a CUDA runtime call failed                    */
#define GEP_ERR_ALLOC (-101)       /* workspace too small / allocation failed      */
#define GEP_ERR_NONFINITE (-102)   /* NaN or Inf found in an input matrix           */
#define GEP_ERR_TIMEOUT (-103)     /* a bounded device-side wait gave up            */
#define GEP_ERR_HANDLE (-104)      /* NULL or destroyed handle                      */
#define GEP_ERR_UNSUPPORTED (-105) /* option combination not implemented            */
#define GEP_ERR_TOO_LARGE (-106)   /* exceeds the fixed scratch of gep_dgemm_emulated_noalloc */

/* Reducer variants (section 3.1, "ScaLAPACK style" / "ELPA style" / "EigenExa style"). */
#define GEP_RED_TWOSIDED 0     /* C = L^-1 A L^-T by triangular solves, L^-1 never formed */
#define GEP_RED_EXPLICIT_INV 1 /* R = L^-1 formed explicitly, then C = R A R^T           */
#define GEP_RED_EIGENEXA 2     /* Cholesky-free (Eq. 7-9): B W = W D by the SEP solver,
                                  C = A' = D^-1/2 W^T A W D^-1/2, Y = W D^-1/2 Z          */

/* SEP-solver variants (section 3.1: conventional tridiagonalisation, or
 * narrow-band reduction followed by band -> tridiagonal; section 6: the parallel
 * block-Jacobi method named as future work). */
#define GEP_SEP_1STAGE 0
#define GEP_SEP_2STAGE 1
#define GEP_SEP_JACOBI 2 /* block Jacobi on C itself (no tridiagonal form, no back-transformation
                            of Householder reflectors): blocks of 32 columns, every pair of blocks
                            diagonalised exactly by one CTA per round (round-robin order), the
                            block rotations applied to C and to the eigenvectors; FP64 on the
                            CUDA cores, about 8 M^3 flops per sweep.  Stage times: t[3] holds it. */

/* Arithmetic of the dense contractions. */
#define GEP_PREC_FP64 0          /* FP64 throughout                                     */
#define GEP_PREC_FP64_EMULATED 1 /* FP64-accurate products from split-BF16 tensor cores  */
#define GEP_PREC_MIXED_REFINED 2 /* FP32-grade split-BF16 reducer + full->band, then FP64 refinement */

typedef struct gep_options {
  int reducer;      /* GEP_RED_*                                                  */
  int sep;          /* GEP_SEP_*                                                  */
  int bandwidth;    /* band width b for GEP_SEP_2STAGE, 1..64 (0 = library default, 64) */
  int precision;    /* GEP_PREC_*                                                 */
  int want_vectors; /* 1: eigenpairs (T_full); 0: eigenvalues only (T_evo)        */
  int overwrite;    /* 1: A and B may be destroyed by gep_solve (saves two copies) */
  int timers;       /* 1: record per-stage CUDA-event times (gep_get_stage_times) */
  int refine_iters; /* GEP_PREC_MIXED_REFINED: FP64 refinement steps; 0 = until converged;
                       -1 = none (the FP32-grade first pass alone, for error studies) */
  int n_want;       /* 0: all M eigenpairs; 1..M: only the n_want lowest (section 2: the occupied
                       states), w[0..n_want) and Y M x n_want.  Eigenvalues only: bisection for
                       those indices; with vectors: divide and conquer gives every eigenvector of
                       T, and only the n_want wanted columns are back-transformed (Q2, Q1, Eq. 6
                       or Eq. 9 on n_want columns).  Not with GEP_PREC_MIXED_REFINED nor in
                       gep_solve_batched (GEP_ERR_UNSUPPORTED). */
  int batch_small;  /* gep_solve_batched only: pencils of order <= batch_small (at most 128) are
                       each solved whole by one CTA (Cholesky, C = L^-1 A L^-T, cyclic Jacobi,
                       Y = L^-T Q, all FP64), all of them in one persistent launch that takes
                       them from a device work queue, largest order first; 0 = none. */
} gep_options;

/* Fills *o with the defaults: TWOSIDED, 1STAGE, b = 0, FP64, vectors, no overwrite, no timers.
 * GEP_RED_EIGENEXA runs the SEP solver twice with the same options (sep, bandwidth, precision):
 * first on B with eigenvectors (Eq. 7), then on A' (Eq. 8); the stage times of
 * gep_get_stage_times then read t[0] = SEP of B (Eq. 7), t[1] = forming A' (Eq. 8),
 * t[5] = Y = W D^-1/2 Z (Eq. 9).  If B has k > 0 eigenvalues that are not positive,
 * gep_get_info reports k and the later stages become no-ops.
 * GEP_PREC_MIXED_REFINED (needs want_vectors = 1): every dense product of the solve runs
 * on the FP32-grade split-BF16 engine and the SYMVs in FP32; FP64 stays in the diagonal
 * blocks, the secular equations and deflation; then all eigenpairs are refined in FP64
 * (B-Rayleigh quotients and the first-order correction X <- X (I + E) from S = X^T A X,
 * R = X^T B X formed with FP64-accurate products; pairs whose gap is below
 * max(64 |S_ij - lambda_j R_ij|, 16 max_ij |S_ij - lambda_j R_ij|, 1e-6 max|lambda|) are
 * grouped into clusters whose k x k pencil (S_CC, R_CC) is solved exactly: by one thread
 * up to 32 eigenpairs, by one CTA up to 256; inside larger clusters a pair takes the
 * first-order step where its own gap is safe, else -R_ij / 2). */
void gep_default_options(gep_options* o);

/* Creates a handle bound to `stream` (a cudaStream_t passed as void*; NULL = legacy
 * default stream).  The handle owns a small device status block (allocated here). */
int gep_create(gep_handle_t* h, void* stream);
int gep_destroy(gep_handle_t h);
int gep_set_stream(gep_handle_t h, void* stream);

/* Bytes of device workspace gep_solve needs for order M with options o. */
int gep_workspace_size(gep_handle_t h, int M, const gep_options* o, size_t* bytes);
/* Bytes of device workspace that every stage entry point below (gep_cholesky ..
 * sep_backtransform_2stage) needs for order M and ncol right-hand columns. */
int gep_stage_workspace_size(gep_handle_t h, int M, int ncol, size_t* bytes);
/* Hands the library caller-owned device workspace (256-byte aligned).  If none is
 * set, or it is too small, gep_solve returns GEP_ERR_ALLOC. */
int gep_set_workspace(gep_handle_t h, void* dptr, size_t bytes);

/* ---- reducer (section 3.1 (b)) ------------------------------------------------
 * gep_cholesky: Eq. 4.  B (lower) is overwritten by L with B = L L^T; the strict
 *   upper triangle is not referenced.  Status k > 0 (gep_get_info) when the leading
 *   minor of order k is not positive definite.
 * gep_reduce: Eq. 5.  Expects L from gep_cholesky in B.  A (lower) is overwritten
 *   by the full symmetric C = L^-1 A L^-T (both triangles written).
 *   variant GEP_RED_EXPLICIT_INV additionally overwrites B's lower triangle with
 *   R = L^-1 (ELPA style "R2"), which gep_backtransform then multiplies by.
 * gep_backtransform: Eq. 6.  Z (M x ncol) is overwritten by Y = L^-T Z
 *   (variant TWOSIDED: triangular solve with L in B) or Y = R^T Z (EXPLICIT_INV).
 * Variant GEP_RED_EIGENEXA (Eq. 7-9, no Cholesky factor): gep_reduce takes the original B
 *   (lower triangle read; do not call gep_cholesky first), solves B W = W D with the 1-stage
 *   SEP solver and overwrites B (all M x M entries) with X = W D^-1/2 and A (both triangles)
 *   with A' = X^T A X; status k > 0 when k eigenvalues of B are not positive.
 *   gep_backtransform then forms Y = X Z with X in B. */
int gep_cholesky(gep_handle_t h, int M, double* B, int ldb);
int gep_reduce(gep_handle_t h, int M, double* A, int lda, double* B, int ldb, int variant);
int gep_backtransform(gep_handle_t h, int M, int ncol, const double* B, int ldb, double* Z, int ldz,
                      int variant);

/* ---- SEP solver (section 3.1 (a); TRD / D&C / BACK of Table 3) ---------------
 * sep_tridiag_1stage: Householder reduction C = Q T Q^T.  C (lower) is overwritten:
 *   its strictly-lower part below the subdiagonal holds the reflectors v_k (unit
 *   leading entry implied); d[M], e[M-1], tau[M-1] receive T and the reflector
 *   scalars (H_k = I - tau_k v_k v_k^T, Q = H_0 H_1 ... H_{M-2}).
 * sep_tridiag_eig: divide and conquer on (d, e).  w[M] receives the eigenvalues in
 *   ascending order; if want_vectors, Z (M x M) receives the orthonormal eigenvectors
 *   of T.  d and e are not modified.  want_vectors = 0 uses Sturm bisection.
 * sep_backtransform: Z (M x ncol) is overwritten by Q Z using the reflectors left
 *   in C by sep_tridiag_1stage (blocked compact-WY products). */
int sep_tridiag_1stage(gep_handle_t h, int M, double* C, int ldc, double* d, double* e, double* tau);
int sep_tridiag_eig(gep_handle_t h, int M, const double* d, const double* e, double* w, double* Z,
                    int ldz, int want_vectors);
int sep_backtransform(gep_handle_t h, int M, int ncol, const double* C, int ldc, const double* tau,
                      double* Z, int ldz);

/* ---- two-stage SEP solver (section 3: the narrow-band reduction solvers ELPA2 and
 * Eigen_sx; "TRD/BAND" and "BACK" of Table 3) --------------------------------------
 * sep_q2_elems: number of doubles of the bulge-chasing reflector storage q2 for order M
 *   and bandwidth b (1 <= b <= 64; 0 for invalid arguments).
 * sep_tridiag_2stage: C = Q1 Q2 T Q2^T Q1^T in two stages.  Full -> band: C (lower
 *   triangle read and overwritten, upper not referenced) becomes a matrix of bandwidth b, whose
 *   lower band (offsets 0..b) is kept, with the panel reflectors stored below the band
 *   (reflector j has its implied unit entry at row j+b) and their scalars in tau1[M]
 *   (tau1[j] = 0 where no reflector exists).  Band -> tridiagonal by bulge chasing:
 *   d[M], e[M-1] receive T; q2 (device, sep_q2_elems(M, b) doubles, caller-owned;
 *   NULL when only eigenvalues are wanted) receives the bulge-chasing reflectors.
 *   C's band itself is not modified by the second stage.
 * sep_backtransform_2stage: Z (M x ncol) is overwritten by Q1 (Q2 Z) using C, tau1 and
 *   q2 from sep_tridiag_2stage with the same M and b.
 * Both take their scratch from the handle workspace (size it with gep_workspace_size
 * and sep = GEP_SEP_2STAGE, bandwidth = b); products run in FP64. */
size_t sep_q2_elems(int M, int b);
int sep_tridiag_2stage(gep_handle_t h, int M, double* C, int ldc, int b, double* d, double* e, double* tau1,
                       double* q2);
int sep_backtransform_2stage(gep_handle_t h, int M, int ncol, int b, const double* C, int ldc,
                             const double* tau1, const double* q2, double* Z, int ldz);

/* ---- whole workflow ------------------------------------------------------------
 * gep_solve: Eq. 2 for all M eigenpairs (or the n = o->n_want lowest).  A, B (lower) are
 *   read and preserved unless o->overwrite.  w[n] receives eigenvalues ascending; if
 *   o->want_vectors, Y (M x n, ldy) receives B-orthonormal eigenvectors whose
 *   largest-magnitude entry is positive (ties: lowest row index).  Uses the workspace set
 *   with gep_set_workspace.  Returns -10 for o == NULL or o->n_want outside [0, M]. */
int gep_solve(gep_handle_t h, int M, double* A, int lda, double* B, int ldb, double* w, double* Y,
              int ldy, const gep_options* o);

/* Same as gep_solve but A, B, w, Y are HOST pointers (pinned or pageable): copies
 * in, solves, copies out and synchronises.  Device memory comes from the workspace,
 * which must be sized with gep_workspace_size(..., o) plus 2*M*M*8 + M*8 + M*M*8 bytes
 * (gep_workspace_size_host gives the exact figure). */
int gep_workspace_size_host(gep_handle_t h, int M, const gep_options* o, size_t* bytes);
int gep_solve_host(gep_handle_t h, int M, const double* A, int lda, const double* B, int ldb,
                   double* w, double* Y, int ldy, const gep_options* o);

/* ---- adjoint (reverse-mode derivative of Eq. 2) ---------------------------------
 * For loss = sum_k lbar_k lambda_k + <W, P>, P = Y_o Y_o^T over the n_occ lowest
 * eigenpairs, writes Abar = d loss / dA and Bbar = d loss / dB (full symmetric M x M,
 * leading dimension ldab) from the output (w ascending, Y B-orthonormal) of gep_solve.
 * First-order perturbation of Eq. 2: Abar = Y G Y^T, Bbar = Y H Y^T with G, H built from
 * lbar, lambda and What = Y^T W Y on the occupied/virtual blocks (only occupied/virtual
 * gaps are divided by).  lbar: M weights (NULL = 1 for occupied, 0 for virtual); W:
 * M x M, both triangles read (NULL = no density term); since P is symmetric only the
 * symmetric part (W + W^T) / 2 enters the loss, and that is what the library forms, so a
 * raw gradient with respect to P can be passed as it is.  All pointers are device memory;
 * the workspace must hold gep_adjoint_workspace_size bytes.  Dense products run on the
 * FP64-accurate tensor-core engine. */
int gep_adjoint_workspace_size(gep_handle_t h, int M, int n_occ, size_t* bytes);
int gep_adjoint(gep_handle_t h, int M, int n_occ, const double* w, const double* Y, int ldy, const double* lbar,
                const double* W, int ldw, double* Abar, double* Bbar, int ldab);

/* ---- batched solves (many independent pencils of uneven order) -------------------
 * Solves count pencils (A_i, B_i) of order M[i] with the workflow of gep_solve; host
 * arrays of device pointers.  Pencils of order <= o->batch_small go to one persistent
 * launch on the handle's stream (one CTA per pencil, see gep_options).  The others are
 * spread over nstreams (1..64) concurrent child streams (largest M^3 first, each to the
 * least loaded stream), forked from and joined back into the handle's stream with events,
 * so the whole call can be captured into one CUDA graph (call it once outside capture
 * first: that call creates the child streams and their status blocks).  precision[i] (may be NULL: o->precision for all)
 * selects the product engine per pencil (the autotuned choice per size bucket).
 * The workspace (gep_solve_batched_workspace_size) holds one solve workspace per
 * stream, sized for the largest pencil that stream receives.  Numerical status of
 * pencil i is not reported separately: gep_get_info covers the handle's own stream;
 * check each child with gep_batched_info. */
int gep_solve_batched_workspace_size(gep_handle_t h, int count, const int* M, const gep_options* o,
                                     const int* precision, int nstreams, size_t* bytes);
int gep_solve_batched(gep_handle_t h, int count, const int* M, double* const* A, double* const* B, double* const* w,
                      double* const* Y, const gep_options* o, const int* precision, int nstreams);
/* As gep_solve_batched / gep_solve_batched_workspace_size, with one gep_options per pencil
 * (opts[0..count), host memory): pencil i runs its own workflow (reducer, SEP solver,
 * bandwidth, precision, want_vectors; the autotuned route of its size bucket) and takes the
 * one-CTA route when M[i] <= opts[i].batch_small.  timers are ignored and n_want must be 0.
 * Returns -2 (count outside 0..4096), -3 (a null array or a negative order), -4 (opts null
 * or a negative batch_small; -8 in gep_solve_batched_opts), -5 / -9 (nstreams outside
 * 1..64), -6 (bytes null), GEP_ERR_UNSUPPORTED for an unsupported option set,
 * GEP_ERR_ALLOC for a workspace smaller than the query's answer. */
int gep_solve_batched_opts_workspace_size(gep_handle_t h, int count, const int* M, const gep_options* opts,
                                          int nstreams, size_t* bytes);
int gep_solve_batched_opts(gep_handle_t h, int count, const int* M, double* const* A, double* const* B,
                           double* const* w, double* const* Y, const gep_options* opts, int nstreams);
/* Synchronises and returns max over child streams of their numerical status. */
int gep_batched_info(gep_handle_t h, int* info);

/* Synchronises the stream and returns the numerical status in *info:
 *   0 ok; k in 1..M: leading minor k of B not positive definite (Eq. 4 failed);
 *   M + j: divide and conquer failed on a subproblem; GEP_ERR_NONFINITE / GEP_ERR_TIMEOUT. */
int gep_get_info(gep_handle_t h, int* info);
int gep_reset_info(gep_handle_t h);

/* Failure-detection hook (tests).  Every device-side wait of the bulge chasing (S1c: step k
 * of sweep s waits for step k+1 of sweep s-1) gives up after wait_limit_s seconds
 * (0 < wait_limit_s <= 4; default 4), records GEP_ERR_TIMEOUT for gep_get_info and returns;
 * the waits behind it see the error and return too, so the launch ends and the context stays
 * usable.  drop_sweep >= 0 makes that sweep publish no progress (a message dropped on
 * purpose, so that the next sweep's wait runs out); -1 (the default) injects nothing.
 * Returns -2 / -3 for an out-of-range drop_sweep / wait_limit_s.  Clear the recorded error
 * with gep_reset_info. */
int gep_set_wait_fault(gep_handle_t h, int drop_sweep, double wait_limit_s);

/* Test hook for the panel QR of the full -> band reduction (S1b).  By default each panel
 * is factorised in one cooperative launch whose CTAs keep 64, 128 or 256 panel rows each
 * in shared memory (the fewest rows whose grid is resident at once), and by one launch
 * per column step when no such grid exists.  rows = 64, 128 or 256 forces that CTA height
 * (a panel whose grid would not be resident then returns GEP_ERR_UNSUPPORTED), rows = -1
 * forces the per-column-step kernel, rows = 0 restores the automatic choice.  Returns -2
 * for any other value. */
int gep_set_panel_qr(gep_handle_t h, int rows);

/* Test hook for the panel grouping of the full -> band reduction (S1b).  Panels are taken in
 * groups of four (their trailing updates deferred and applied as one product) while the
 * trailing matrix has order >= min_order, in pairs below it; by default min_order = 8192.
 * min_order = 0 groups every panel it can (so that small matrices exercise the grouped
 * path), -1 restores the default.  Returns -2 for min_order < -1. */
int gep_set_band_group(gep_handle_t h, int min_order);

/* Per-stage times (ms) of the last gep_solve with o->timers = 1:
 * t[0] Cholesky (R1), t[1] reduction (R2), t[2] tridiagonalisation (TRD/BAND),
 * t[3] tridiagonal eigensolver (D&C), t[4] Householder back-transform (BACK),
 * t[5] back-substitution (R5 / Eq. 6), t[6] FP64 refinement (mixed precision only, else ~0).
 * Synchronises. */
int gep_get_stage_times(gep_handle_t h, double t[7]);

/* FP64 refinement steps the last GEP_PREC_MIXED_REFINED gep_solve on h took (or
 * GEP_ERR_HANDLE).  With refine_iters = 0 the refinement stops after the step whose
 * size (largest first-order correction |E_ij|, B-orthogonality defect inside clusters,
 * |1 - y_i^T B y_i|) is at most 1e-8, and after 8 steps at most; that test synchronises
 * the stream once per step, so while h's stream is being captured into a CUDA graph a
 * fixed 4 steps run instead.  (No counterpart in the paper: the refinement is this
 * library's mixed-precision extension.) */
int gep_refine_steps(gep_handle_t h);

/* Split of the SEP reduction time t[2] of the last GEP_SEP_2STAGE gep_solve with
 * timers: t[0] full -> band, t[1] band -> tridiagonal (bulge chasing), in ms.
 * Synchronises with that solve; GEP_ERR_UNSUPPORTED when none was recorded. */
int gep_get_band_times(gep_handle_t h, double t[2]);

/* Number of kernels the library launched since gep_create / last reset (for
 * gep_solve_batched: every kernel of the batch, the child streams' included). */
long long gep_launch_count(gep_handle_t h, int reset);

/* Per-launch timing of the split-BF16 tensor-core product kernel (measurement aid;
 * no counterpart in the paper).  gep_profile_enable(h, cap) records a CUDA event
 * pair around each of the next `cap` launches (cap = 0 switches recording off and
 * releases the events).  gep_profile_read synchronises the stream and returns the
 * summed kernel time (ms), the tensor-core flops those launches performed (all
 * digit-plane products), their FP64-equivalent flops (2mnk), the number of timed
 * launches and of launches not timed because the pool was full; reset != 0 clears
 * the counters. */
int gep_profile_enable(gep_handle_t h, int cap);
int gep_profile_read(gep_handle_t h, double* ms, double* tensor_flops, double* fp64_flops, long long* launches,
                     long long* skipped, int reset);
/* Recorded launch i (0 <= i < launches of gep_profile_read, before a reset): its product
 * shape (m, n, k of that K panel) and CUDA-event time in ms.  Synchronises the stream. */
int gep_profile_entry(gep_handle_t h, int i, int mnk[3], double* ms);

const char* gep_status_string(int code);

/* ---- FP64 matrix product (the dense contraction every stage is built on) ------
 * C = alpha op(A) op(B) + beta C, op = 'N' or 'T'; transa 'S': A is symmetric (m x m,
 * k = m, transb 'N') and only its lower triangle is read.  uplo 'F' (full) or 'L' (only
 * entries i >= j of C are computed and written).  engine: GEP_PREC_FP64 (FP64 FMA)
 * or GEP_PREC_FP64_EMULATED (split-BF16 tensor cores, FP64-accurate). */
int gep_dgemm(gep_handle_t h, char transa, char transb, char uplo, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
              int engine);

/* ---- allocation-free product (no counterpart in the paper) ---------------------
 * For callers that cannot call cudaMalloc, e.g. a framework that owns the whole
 * device-memory budget through its own pool, or a latency-critical loop that must
 * not let a library grow its footprint or enter the allocator mid-run.
 * Computes the same product as gep_dgemm(..., GEP_PREC_FP64_EMULATED) without a
 * handle or workspace: its scratch (digit planes, exponents, a status word) is a
 * fixed 64 MiB device array inside this library, which every GPU that loads the
 * library keeps until the process exits.  The caller passes A, B, C (device memory)
 * and the stream (a cudaStream_t as void*, NULL = legacy default stream).
 *  - Sizes: requires 2*8*(m+n)*32 + 4*(m+n) bytes plus ~1.3 KB to fit in 64 MiB,
 *    i.e. m + n <= 130,000 or so; larger problems return GEP_ERR_TOO_LARGE before
 *    anything is enqueued.  Long K is processed in panels sized to the array.
 *  - The first call on a device resolves the array's device address for that device
 *    (cudaGetSymbolAddress with the caller's current device); make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents; calls that
 *    overlap on the GPU (other streams, other threads) race on it.  Serialise them.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *  - A failure on the GPU after the call has returned (a bounded wait inside the product
 *    kernel that gave up) cannot be a return code: the last kernel of the call then fills
 *    every element of C the call writes with NaN, so such a failure shows in C.
 * Returns 0, -i for an illegal argument i, GEP_ERR_TOO_LARGE or GEP_ERR_CUDA. */
int gep_dgemm_emulated_noalloc(char transa, char transb, char uplo, int m, int n, int k, double alpha,
                               const double* A, int lda, const double* B, int ldb, double beta, double* C,
                               int ldc, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GEP_H */
