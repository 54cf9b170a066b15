// C ABI (include/gep.h): handle, workspace, stage entry points and the whole
// GEP workflow of section 3.1 (reducer -> SEP solver -> back-transformation).
// Host code here only validates arguments, carves the caller's workspace and
// enqueues kernels; no step of the method runs on the host.
#include <string.h>

#include "gep_internal.cuh"

using namespace gep;

namespace {

constexpr int NB = 128;  // diagonal block order of the triangular kernels (tri.cu)

bool handle_ok(gep_handle_t h) { return h != nullptr && h->magic == 0x6e70; }

struct SolveLayout {
  size_t Cw, Lw, invD, vec, uni, eng, af, q2, xw, zt, q2u, end;  // byte offsets
  size_t uni_bytes, eng_bytes;
};

constexpr int kDefaultBand = 64;  // bandwidth of the two-stage reduction when o->bandwidth = 0

int band_of(const gep_options* o) { return o->bandwidth > 0 ? o->bandwidth : kDefaultBand; }
bool two_stage(const gep_options* o) { return o->sep == GEP_SEP_2STAGE; }
bool jacobi(const gep_options* o) { return o->sep == GEP_SEP_JACOBI; }
bool eigenexa(const gep_options* o) { return o->reducer == GEP_RED_EIGENEXA; }
// the SEP solver runs with eigenvectors: for the caller's pencil, or on B (Eq. 7)
bool sep_vectors(const gep_options* o) { return o->want_vectors || eigenexa(o); }
// only the lowest n_want eigenpairs, with vectors: D&C writes all eigenvectors of T to a
// workspace matrix first
bool partial_vectors(int M, const gep_options* o) { return o->want_vectors && o->n_want > 0 && o->n_want < M; }
// the tensor-core engines apply Q2 as dense tiles, all built ahead on the second stream
bool q2_tiles_ahead(const gep_options* o) {
  return two_stage(o) && sep_vectors(o) && o->precision != GEP_PREC_FP64;
}

size_t r256(size_t x) { return align256(x); }

size_t invd_bytes(int M) {
  size_t nblk = (M + NB - 1) / NB;
  return (nblk * NB * NB + (size_t)M * NB) * sizeof(double);
}

size_t union_bytes(int M, const gep_options* o) {
  size_t mm = (size_t)M * M * sizeof(double);
  size_t tmpb = (size_t)NB * M * sizeof(double);
  size_t red = (o->reducer == GEP_RED_EXPLICIT_INV) ? r256(mm) + r256(mm) + r256(tmpb)
               : eigenexa(o) ? r256(mm)  // A X of Eq. 8
                             : r256(mm) + r256(tmpb);
  size_t tri = two_stage(o) ? band_ws_elems(M, band_of(o)) * sizeof(double)
               : jacobi(o)  ? jacobi_ws_elems(M) * sizeof(double)
                            : tridiag_ws_elems(M) * sizeof(double);
  size_t dc = sep_vectors(o) ? dc_ws_bytes(M) : 0;
  size_t bt = sep_vectors(o) ? backtransform_ws_elems(M, M) * sizeof(double) : 0;
  if (two_stage(o) && sep_vectors(o)) {
    size_t q2t = q2_tile_ws_elems(M, band_of(o)) * sizeof(double);
    if (q2t > bt) bt = q2t;
  }
  size_t r3 = (o->want_vectors && !eigenexa(o))
                  ? (r256(tmpb) + (o->reducer == GEP_RED_EXPLICIT_INV ? r256(mm) : 0))
                  : 0;
  size_t rf = (o->precision == GEP_PREC_MIXED_REFINED) ? r256(refine_ws_elems(M) * sizeof(double)) : 0;
  size_t u = red;
  if (rf > u) u = rf;
  if (tri > u) u = tri;
  if (dc > u) u = dc;
  if (bt > u) u = bt;
  if (r3 > u) u = r3;
  return r256(u);
}

SolveLayout layout(int M, const gep_options* o) {
  SolveLayout L;
  size_t mm = (size_t)M * M * sizeof(double);
  size_t off = 0;
  L.Cw = off; off += o->overwrite ? 0 : r256(mm);
  L.Lw = off; off += o->overwrite ? 0 : r256(mm);
  L.invD = off; off += r256(invd_bytes(M));
  L.vec = off; off += r256((size_t)5 * (M + 1) * sizeof(double));
  L.uni = off;
  L.uni_bytes = union_bytes(M, o);
  off += L.uni_bytes;
  L.eng = off;
  L.eng_bytes = (o->precision == GEP_PREC_FP64) ? 0 : r256(oz_workspace_bytes(M, M, M));
  off += L.eng_bytes;
  L.af = off;  // full symmetric A and B kept for the FP64 refinement
  off += (o->precision == GEP_PREC_MIXED_REFINED) ? 2 * r256(mm) : 0;
  L.q2 = off;  // bulge-chasing reflectors, kept from S1c to the back-transformation
  off += (two_stage(o) && sep_vectors(o)) ? r256(q2_elems(M, band_of(o)) * sizeof(double)) : 0;
  L.xw = off;  // X = W D^-1/2 of the Cholesky-free reducer (Eq. 7-9)
  off += eigenexa(o) ? r256(mm) : 0;
  L.zt = off;  // all eigenvectors of T when only the lowest n_want are back-transformed
  off += partial_vectors(M, o) ? r256(mm) : 0;
  L.q2u = off;  // every dense Q2 tile, built on the second stream during divide and conquer
  off += q2_tiles_ahead(o) ? r256(q2_all_tiles_elems(M, band_of(o)) * sizeof(double)) : 0;
  L.end = off;
  return L;
}

int check_opts(const gep_options* o) {
  if (!o) return -1;
  if (o->reducer != GEP_RED_TWOSIDED && o->reducer != GEP_RED_EXPLICIT_INV && o->reducer != GEP_RED_EIGENEXA)
    return GEP_ERR_UNSUPPORTED;
  if (o->sep != GEP_SEP_1STAGE && o->sep != GEP_SEP_2STAGE && o->sep != GEP_SEP_JACOBI) return GEP_ERR_UNSUPPORTED;
  if (o->sep == GEP_SEP_2STAGE && (o->bandwidth < 0 || o->bandwidth > 64)) return GEP_ERR_UNSUPPORTED;
  if (o->precision != GEP_PREC_FP64 && o->precision != GEP_PREC_FP64_EMULATED &&
      o->precision != GEP_PREC_MIXED_REFINED)
    return GEP_ERR_UNSUPPORTED;
  if (o->precision == GEP_PREC_MIXED_REFINED && !o->want_vectors) return GEP_ERR_UNSUPPORTED;
  if (o->refine_iters < -1) return -10;
  if (o->n_want < 0) return -10;
  if (o->n_want > 0 && o->precision == GEP_PREC_MIXED_REFINED) return GEP_ERR_UNSUPPORTED;
  return GEP_OK;
}

int reset_status(gep_handle_t h) {
  GEP_CUDA(cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), h->stream));
  return GEP_OK;
}

void mark(gep_handle_t h, const gep_options* o, int i) {
  if (o->timers) cudaEventRecord(h->ev[i], h->stream);
}

// SEP solver of section 3.1 (a) on the symmetric C (lower triangle read, overwritten by the
// reflectors): tridiagonalisation (1-stage, or full -> band -> tridiagonal), then either the
// eigenvalues w by bisection (Z == nullptr) or divide and conquer with the eigenvectors of T
// written to Z and back-transformed.  n < M: only the n lowest eigenpairs (w[0..n), Z M x n);
// with vectors D&C then writes all eigenvalues to wt and all eigenvectors of T to Zt (M x M)
// and only the first n columns are copied to Z and back-transformed.  timed: record marks 3
// (after TRD/BAND) and 4 (after D&C) and the S1b/S1c split of the caller's timers.
int sep_solve(gep_handle_t h, int M, double* C, int ldc, const gep_options* o, double* dvec, double* evec,
              double* tvec, double* q2, char* uni, size_t uni_bytes, int eng, double* w, double* Z, int ldz,
              bool timed, int n = 0, double* Zt = nullptr, double* wt = nullptr, double* q2u = nullptr) {
  if (n <= 0 || n > M) n = M;
  const int bw = band_of(o);
  if (jacobi(o)) {  // no tridiagonal form: the block-Jacobi solver works on C itself
    if (timed) mark(h, o, 3);
    double* wj = (n < M) ? wt : w;
    double* Zj = (n < M) ? Zt : Z;
    if (n < M && Z && (!Zt || !wt)) return GEP_ERR_ALLOC;
    if (n < M && !Z && !wt) return GEP_ERR_ALLOC;
    GEP_CHECK(jacobi_sep(h, M, C, ldc, wj, Zj, (n < M) ? M : ldz, (double*)uni));
    if (n < M) {
      GEP_CHECK(copy_matrix(h, n, 1, wt, n, w, n));
      if (Z) GEP_CHECK(copy_matrix(h, M, n, Zt, M, Z, ldz));
    }
    if (timed) mark(h, o, 4);
    return GEP_OK;
  }
  if (two_stage(o)) {
    GEP_CHECK(band_reduce(h, M, C, ldc, bw, tvec, (double*)uni, uni_bytes / sizeof(double), eng));  // S1b
    if (timed && o->timers) cudaEventRecord(h->ev_band, h->stream);
    GEP_CHECK(band_to_tridiag(h, M, C, ldc, bw, dvec, evec, Z ? q2 : nullptr, (double*)uni,
                              uni_bytes / sizeof(double)));  // S1c
  } else {
    GEP_CHECK(tridiag_1stage(h, M, C, ldc, dvec, evec, tvec, (double*)uni, uni_bytes / sizeof(double), eng));
  }
  if (timed) mark(h, o, 3);
  if (!Z) {
    GEP_CHECK(tridiag_eig_bisect(h, M, dvec, evec, w, n));
    if (timed) mark(h, o, 4);
    return GEP_OK;
  }
  // the Q2 tiles depend only on the bulge-chasing reflectors: build them on the second
  // stream while divide and conquer runs here
  const bool ahead = q2u != nullptr && two_stage(o) && eng != GEP_PREC_FP64;
  if (ahead) {
    GEP_CUDA(cudaEventRecord(h->ev_fork, h->stream));
    GEP_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    GEP_CHECK(build_q2_tiles(h, h->side, M, band_of(o), q2, q2u));
    GEP_CUDA(cudaEventRecord(h->ev_join, h->side));
  }
  if (n < M) {
    if (!Zt || !wt) return GEP_ERR_ALLOC;
    GEP_CHECK(tridiag_eig_dc(h, M, dvec, evec, wt, Zt, M, (double*)uni, uni_bytes, eng));  // D&C
    GEP_CHECK(copy_matrix(h, n, 1, wt, n, w, n));
    GEP_CHECK(copy_matrix(h, M, n, Zt, M, Z, ldz));  // the n lowest eigenvectors of T
  } else {
    GEP_CHECK(tridiag_eig_dc(h, M, dvec, evec, w, Z, ldz, (double*)uni, uni_bytes, eng));  // D&C
  }
  if (timed) mark(h, o, 4);
  if (ahead) GEP_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  if (two_stage(o)) {
    GEP_CHECK(apply_q2(h, M, bw, q2, Z, ldz, n, eng, (double*)uni, uni_bytes / sizeof(double),
                       ahead ? q2u : nullptr));
    return backtransform_q(h, M, n, C, ldc, tvec, Z, ldz, (double*)uni, uni_bytes / sizeof(double), eng, bw);
  }
  return backtransform_q(h, M, n, C, ldc, tvec, Z, ldz, (double*)uni, uni_bytes / sizeof(double), eng);
}

}  // namespace

extern "C" {

void gep_default_options(gep_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->reducer = GEP_RED_TWOSIDED;
  o->sep = GEP_SEP_1STAGE;
  o->precision = GEP_PREC_FP64;
  o->want_vectors = 1;
}

int gep_create(gep_handle_t* out, void* stream) {
  if (!out) return -1;
  *out = nullptr;
  gep_handle_t h = new gep_handle_s();
  h->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc((void**)&h->d_status, 256) != cudaSuccess) { delete h; return GEP_ERR_CUDA; }
  if (cudaMemset(h->d_status, 0, 256) != cudaSuccess) { cudaFree(h->d_status); delete h; return GEP_ERR_CUDA; }
  h->splitk_bytes = (size_t)32 << 20;
  if (cudaMalloc((void**)&h->d_splitk, h->splitk_bytes) != cudaSuccess) {
    cudaFree(h->d_status);
    delete h;
    return GEP_ERR_CUDA;
  }
  for (int i = 0; i < 8; ++i) cudaEventCreate(&h->ev[i]);
  cudaEventCreate(&h->ev_band);
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    gep_destroy(h);
    return GEP_ERR_CUDA;
  }
  *out = h;
  return GEP_OK;
}

int gep_destroy(gep_handle_t h) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  gep_profile_enable(h, 0);
  for (int c = 0; c < h->nchild; ++c) {
    gep_destroy(h->child[c]);
    cudaEventDestroy(h->child_done[c]);
    cudaStreamDestroy(h->child_stream[c]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  cudaFree(h->d_batch_info);
  cudaFree(h->d_small_next);
  for (int i = 0; i < 8; ++i) cudaEventDestroy(h->ev[i]);
  cudaEventDestroy(h->ev_band);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  cudaFree(h->d_status);
  cudaFree(h->d_splitk);
  h->magic = 0;
  delete h;
  return GEP_OK;
}

int gep_set_stream(gep_handle_t h, void* stream) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  h->stream = (cudaStream_t)stream;
  return GEP_OK;
}

int gep_workspace_size(gep_handle_t h, int M, const gep_options* o, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (!o) return -3;
  if (!bytes) return -4;
  *bytes = layout(M, o).end;
  return GEP_OK;
}

int gep_stage_workspace_size(gep_handle_t h, int M, int ncol, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (ncol < 0) return -3;
  if (!bytes) return -4;
  const size_t slack = 4 * 256;  // arena alignment of up to four carvings
  const size_t d = sizeof(double), mm = (size_t)M * M;
  size_t need = invd_bytes(M);                                                        // gep_cholesky
  size_t red = invd_bytes(M) + d * mm + d * (mm + (size_t)NB * M);                    // gep_reduce
  size_t bks = invd_bytes(M) + d * (size_t)NB * (ncol > M ? ncol : M) + d * mm;       // gep_backtransform
  size_t tri = d * tridiag_ws_elems(M);
  size_t dc = dc_ws_bytes(M);
  size_t bt = d * backtransform_ws_elems(M, ncol > 0 ? ncol : 1);
  size_t band = d * band_ws_elems(M, 64);                                              // largest bandwidth
  // gep_reduce, Cholesky-free variant: copy of B, four vectors, then the largest SEP stage
  size_t sep_max = tri;
  for (size_t x : {dc, d * backtransform_ws_elems(M, M), d * mm})
    if (x > sep_max) sep_max = x;
  size_t ee = d * mm + d * 4 * ((size_t)M + 1) + sep_max;
  size_t bke = d * mm;  // gep_backtransform, Cholesky-free variant: X Z
  if (ncol > M) bke = d * (size_t)M * ncol;
  for (size_t x : {red, bks, tri, dc, bt, band, ee, bke})
    if (x > need) need = x;
  *bytes = need + slack;
  return GEP_OK;
}

int gep_set_workspace(gep_handle_t h, void* dptr, size_t bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (dptr == nullptr && bytes != 0) return -2;
  if (((uintptr_t)dptr & 255) != 0) return -2;
  h->ws = (char*)dptr;
  h->ws_bytes = bytes;
  return GEP_OK;
}

int gep_get_info(gep_handle_t h, int* info) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (!info) return -2;
  int st[2] = {0, 0};
  GEP_CUDA(cudaStreamSynchronize(h->stream));
  GEP_CUDA(cudaMemcpy(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  *info = st[1] != 0 ? st[1] : st[0];
  return GEP_OK;
}

int gep_reset_info(gep_handle_t h) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  return reset_status(h);
}

int gep_set_wait_fault(gep_handle_t h, int drop_sweep, double wait_limit_s) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (drop_sweep < -1) return -2;
  if (!(wait_limit_s > 0.0 && wait_limit_s <= 4.0)) return -3;
  h->fault_drop_sweep = drop_sweep;
  h->wait_limit_ns = (unsigned long long)(wait_limit_s * 1e9);
  return GEP_OK;
}

int gep_set_panel_qr(gep_handle_t h, int rows) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (rows != 0 && rows != -1 && rows != 64 && rows != 128 && rows != 256) return -2;
  h->pqr_rows = rows;
  return GEP_OK;
}

int gep_set_band_group(gep_handle_t h, int min_order) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (min_order < -1) return -2;
  h->band_group_min = min_order;
  return GEP_OK;
}

long long gep_launch_count(gep_handle_t h, int reset) {
  if (!handle_ok(h)) return -1;
  long long n = h->launches;
  if (reset) h->launches = 0;
  return n;
}

int gep_refine_steps(gep_handle_t h) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  return h->refine_steps;
}

int gep_profile_enable(gep_handle_t h, int cap) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (cap < 0) return -2;
  GEP_CUDA(cudaStreamSynchronize(h->stream));
  if (h->prof_ev) {
    for (int i = 0; i < 2 * h->prof_cap; ++i) cudaEventDestroy(h->prof_ev[i]);
    delete[] h->prof_ev;
    delete[] h->prof_flops;
    delete[] h->prof_f64eq;
    delete[] h->prof_mnk;
    h->prof_mnk = nullptr;
    h->prof_ev = nullptr;
    h->prof_flops = h->prof_f64eq = nullptr;
  }
  h->prof_on = 0;
  h->prof_cap = h->prof_used = 0;
  h->prof_skipped = 0;
  if (cap == 0) return GEP_OK;
  h->prof_ev = new cudaEvent_t[2 * (size_t)cap];
  h->prof_flops = new double[cap];
  h->prof_f64eq = new double[cap];
  h->prof_mnk = new int[3 * (size_t)cap];
  for (int i = 0; i < 2 * cap; ++i) GEP_CUDA(cudaEventCreate(&h->prof_ev[i]));
  h->prof_cap = cap;
  h->prof_on = 1;
  return GEP_OK;
}

int gep_profile_read(gep_handle_t h, double* ms, double* tensor_flops, double* fp64_flops, long long* launches,
                     long long* skipped, int reset) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  GEP_CUDA(cudaStreamSynchronize(h->stream));
  double t = 0.0, f = 0.0, f64 = 0.0;
  for (int i = 0; i < h->prof_used; ++i) {
    float e = 0.f;
    GEP_CUDA(cudaEventElapsedTime(&e, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    t += e;
    f += h->prof_flops[i];
    f64 += h->prof_f64eq[i];
  }
  if (ms) *ms = t;
  if (tensor_flops) *tensor_flops = f;
  if (fp64_flops) *fp64_flops = f64;
  if (launches) *launches = h->prof_used;
  if (skipped) *skipped = h->prof_skipped;
  if (reset) {
    h->prof_used = 0;
    h->prof_skipped = 0;
  }
  return GEP_OK;
}

int gep_profile_entry(gep_handle_t h, int i, int mnk[3], double* ms) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (i < 0 || i >= h->prof_used) return -2;
  if (!mnk || !ms) return -3;
  GEP_CUDA(cudaStreamSynchronize(h->stream));
  float e = 0.f;
  GEP_CUDA(cudaEventElapsedTime(&e, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
  for (int q = 0; q < 3; ++q) mnk[q] = h->prof_mnk[3 * i + q];
  *ms = e;
  return GEP_OK;
}

int gep_get_stage_times(gep_handle_t h, double t[7]) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (!t) return -2;
  if (!h->timers_recorded) return GEP_ERR_UNSUPPORTED;
  GEP_CUDA(cudaEventSynchronize(h->ev[7]));
  for (int i = 0; i < 7; ++i) {
    float ms = 0.f;
    GEP_CUDA(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
    t[i] = ms;
  }
  return GEP_OK;
}

int gep_get_band_times(gep_handle_t h, double t[2]) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (!t) return -2;
  if (!h->timers_recorded || !h->band_recorded) return GEP_ERR_UNSUPPORTED;
  GEP_CUDA(cudaEventSynchronize(h->ev[3]));
  float a = 0.f, b = 0.f;
  GEP_CUDA(cudaEventElapsedTime(&a, h->ev[2], h->ev_band));
  GEP_CUDA(cudaEventElapsedTime(&b, h->ev_band, h->ev[3]));
  t[0] = a;
  t[1] = b;
  return GEP_OK;
}

const char* gep_status_string(int code) {
  switch (code) {
    case GEP_OK: return "ok";
    case GEP_ERR_CUDA: return "CUDA runtime error";
    case GEP_ERR_ALLOC: return "workspace missing or too small";
    case GEP_ERR_NONFINITE: return "NaN or Inf in an input matrix";
    case GEP_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case GEP_ERR_HANDLE: return "invalid handle";
    case GEP_ERR_UNSUPPORTED: return "option combination not implemented";
    case GEP_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the allocation-free entry point";
    default: break;
  }
  if (code < 0 && code >= -20) return "illegal argument";
  if (code > 0) return "numerical failure (see gep_get_info)";
  return "unknown status";
}

int gep_dgemm(gep_handle_t h, char transa, char transb, char uplo, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
              int engine) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  bool sa = (transa == 'S' || transa == 's');
  if (!ta && !sa && transa != 'N' && transa != 'n') return -2;
  if (!tb && transb != 'N' && transb != 'n') return -3;
  if (sa && tb) return -3;
  if (uplo != 'F' && uplo != 'f' && uplo != 'L' && uplo != 'l') return -4;
  if (m < 0) return -5;
  if (n < 0) return -6;
  if (k < 0 || (sa && k != m)) return -7;
  if (lda < (ta ? (k > 1 ? k : 1) : (m > 1 ? m : 1))) return -10;
  if (ldb < (tb ? (n > 1 ? n : 1) : (k > 1 ? k : 1))) return -12;
  if (ldc < (m > 1 ? m : 1)) return -15;
  if (engine != GEP_PREC_FP64 && engine != GEP_PREC_FP64_EMULATED && engine != GEP_PREC_MIXED_REFINED) return -16;
  h->eng_ws = h->ws;  // the whole caller workspace serves as product-engine scratch
  h->eng_bytes = h->ws_bytes;
  return dgemm(h, transa, transb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine);
}

int gep_cholesky(gep_handle_t h, int M, double* B, int ldb) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !B) return -3;
  if (ldb < (M > 1 ? M : 1)) return -4;
  if (M == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  double* invD = ar.take<double>(invd_bytes(M) / sizeof(double));
  if (!ar.ok) return GEP_ERR_ALLOC;
  return cholesky(h, M, B, ldb, invD, GEP_PREC_FP64);
}

int gep_reduce(gep_handle_t h, int M, double* A, int lda, double* B, int ldb, int variant) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !A) return -3;
  if (lda < (M > 1 ? M : 1)) return -4;
  if (M > 0 && !B) return -5;
  if (ldb < (M > 1 ? M : 1)) return -6;
  if (variant != GEP_RED_TWOSIDED && variant != GEP_RED_EXPLICIT_INV && variant != GEP_RED_EIGENEXA) return -7;
  if (M == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  if (variant == GEP_RED_EIGENEXA) {
    // Eq. 7 with the 1-stage SEP solver: S = copy of B -> reflectors, W into B, X = W D^-1/2
    double* S = ar.take<double>((size_t)M * M);
    double* v = ar.take<double>((size_t)4 * (M + 1));
    const size_t mm = (size_t)M * M;
    size_t n = tridiag_ws_elems(M);
    if (dc_ws_bytes(M) / sizeof(double) + 1 > n) n = dc_ws_bytes(M) / sizeof(double) + 1;
    if (backtransform_ws_elems(M, M) > n) n = backtransform_ws_elems(M, M);
    if (mm > n) n = mm;
    double* ws = ar.take<double>(n);
    if (!ar.ok) return GEP_ERR_ALLOC;
    double *dv = v, *ev = v + (M + 1), *tv = v + 2 * (M + 1), *wB = v + 3 * (M + 1);
    GEP_CHECK(copy_lower(h, M, B, ldb, S, M));
    GEP_CHECK(tridiag_1stage(h, M, S, M, dv, ev, tv, ws, n, GEP_PREC_FP64));
    GEP_CHECK(tridiag_eig_dc(h, M, dv, ev, wB, B, ldb, ws, n * sizeof(double), GEP_PREC_FP64));
    GEP_CHECK(backtransform_q(h, M, M, S, M, tv, B, ldb, ws, n, GEP_PREC_FP64));
    GEP_CHECK(scale_cols_rsqrt_checked(h, M, M, wB, B, ldb));
    // Eq. 8: A' = X^T (A X) into A (both triangles)
    GEP_CHECK(dgemm(h, 'S', 'N', 'F', M, M, M, 1.0, A, lda, B, ldb, 0.0, ws, M, GEP_PREC_FP64));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, B, ldb, ws, M, 0.0, A, lda, GEP_PREC_FP64));
    return symmetrize_lower(h, M, A, lda);
  }
  double* invD = ar.take<double>(invd_bytes(M) / sizeof(double));
  double* X = ar.take<double>((size_t)M * M);
  double* tmp = ar.take<double>((size_t)M * M + (size_t)NB * M);
  if (!ar.ok) return GEP_ERR_ALLOC;
  GEP_CHECK(tri_inv_diag_blocks(h, M, B, ldb, invD, NB));
  if (variant == GEP_RED_TWOSIDED) return reduce_twosided(h, M, A, lda, B, ldb, invD, X, tmp, GEP_PREC_FP64);
  return reduce_explicit_inv(h, M, A, lda, B, ldb, invD, X, tmp, GEP_PREC_FP64);
}

int gep_backtransform(gep_handle_t h, int M, int ncol, const double* B, int ldb, double* Z, int ldz,
                      int variant) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (ncol < 0) return -3;
  if (M > 0 && !B) return -4;
  if (ldb < (M > 1 ? M : 1)) return -5;
  if (M > 0 && ncol > 0 && !Z) return -6;
  if (ldz < (M > 1 ? M : 1)) return -7;
  if (variant != GEP_RED_TWOSIDED && variant != GEP_RED_EXPLICIT_INV && variant != GEP_RED_EIGENEXA) return -8;
  if (M == 0 || ncol == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  if (variant == GEP_RED_EIGENEXA) {  // Eq. 9: Y = X Z with X = W D^-1/2 in B (full)
    double* T = ar.take<double>((size_t)M * ncol);
    if (!ar.ok) return GEP_ERR_ALLOC;
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, ncol, M, 1.0, B, ldb, Z, ldz, 0.0, T, M, GEP_PREC_FP64));
    return copy_matrix(h, M, ncol, T, M, Z, ldz);
  }
  if (variant == GEP_RED_TWOSIDED) {
    double* invD = ar.take<double>(invd_bytes(M) / sizeof(double));
    double* tmp = ar.take<double>((size_t)NB * ncol);
    if (!ar.ok) return GEP_ERR_ALLOC;
    GEP_CHECK(tri_inv_diag_blocks(h, M, B, ldb, invD, NB));
    return trsm_llt(h, M, ncol, B, ldb, invD, NB, Z, ldz, tmp, GEP_PREC_FP64);
  }
  double* T = ar.take<double>((size_t)M * ncol);
  double* R = ar.take<double>((size_t)M * M);
  if (!ar.ok) return GEP_ERR_ALLOC;
  // Y = R^T Z with R the lower triangle of B (its upper part is not referenced)
  GEP_CHECK(set_matrix(h, M, M, 0.0, 0.0, R, M));
  GEP_CHECK(copy_lower(h, M, B, ldb, R, M));
  GEP_CHECK(dgemm(h, 'T', 'N', 'F', M, ncol, M, 1.0, R, M, Z, ldz, 0.0, T, M, GEP_PREC_FP64));
  return copy_matrix(h, M, ncol, T, M, Z, ldz);
}

int sep_tridiag_1stage(gep_handle_t h, int M, double* C, int ldc, double* d, double* e, double* tau) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !C) return -3;
  if (ldc < (M > 1 ? M : 1)) return -4;
  if (M > 0 && !d) return -5;
  if (M > 1 && !e) return -6;
  if (M > 1 && !tau) return -7;
  if (M == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  size_t n = tridiag_ws_elems(M);
  double* ws = ar.take<double>(n);
  if (!ar.ok) return GEP_ERR_ALLOC;
  return tridiag_1stage(h, M, C, ldc, d, e, tau, ws, n, GEP_PREC_FP64);
}

int sep_tridiag_eig(gep_handle_t h, int M, const double* d, const double* e, double* w, double* Z,
                    int ldz, int want_vectors) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !d) return -3;
  if (M > 1 && !e) return -4;
  if (M > 0 && !w) return -5;
  if (want_vectors && M > 0 && !Z) return -6;
  if (want_vectors && ldz < (M > 1 ? M : 1)) return -7;
  if (M == 0) return GEP_OK;
  if (!want_vectors) return tridiag_eig_bisect(h, M, d, e, w);
  Arena ar(h->ws, h->ws_bytes);
  size_t nb = dc_ws_bytes(M);
  double* ws = (double*)ar.take<char>(nb);
  if (!ar.ok) return GEP_ERR_ALLOC;
  return tridiag_eig_dc(h, M, d, e, w, Z, ldz, ws, nb, GEP_PREC_FP64);
}

int sep_backtransform(gep_handle_t h, int M, int ncol, const double* C, int ldc, const double* tau,
                      double* Z, int ldz) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (ncol < 0) return -3;
  if (M > 0 && !C) return -4;
  if (ldc < (M > 1 ? M : 1)) return -5;
  if (M > 1 && !tau) return -6;
  if (M > 0 && ncol > 0 && !Z) return -7;
  if (ldz < (M > 1 ? M : 1)) return -8;
  if (M <= 1 || ncol == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  size_t n = backtransform_ws_elems(M, ncol);
  double* ws = ar.take<double>(n);
  if (!ar.ok) return GEP_ERR_ALLOC;
  return backtransform_q(h, M, ncol, C, ldc, tau, Z, ldz, ws, n, GEP_PREC_FP64);
}

size_t sep_q2_elems(int M, int b) {
  if (M < 0 || b < 1 || b > 64) return 0;
  return q2_elems(M, b);
}

int sep_tridiag_2stage(gep_handle_t h, int M, double* C, int ldc, int b, double* d, double* e, double* tau1,
                       double* q2) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !C) return -3;
  if (ldc < (M > 1 ? M : 1)) return -4;
  if (b < 1 || b > 64) return -5;
  if (M > 0 && !d) return -6;
  if (M > 1 && !e) return -7;
  if (M > 0 && !tau1) return -8;
  if (M == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  size_t n = band_ws_elems(M, b);
  double* ws = ar.take<double>(n);
  if (!ar.ok) return GEP_ERR_ALLOC;
  GEP_CHECK(band_reduce(h, M, C, ldc, b, tau1, ws, n, GEP_PREC_FP64));
  return band_to_tridiag(h, M, C, ldc, b, d, e, q2, ws, n);
}

int sep_backtransform_2stage(gep_handle_t h, int M, int ncol, int b, const double* C, int ldc, const double* tau1,
                             const double* q2, double* Z, int ldz) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (ncol < 0) return -3;
  if (b < 1 || b > 64) return -4;
  if (M > 0 && !C) return -5;
  if (ldc < (M > 1 ? M : 1)) return -6;
  if (M > 0 && !tau1) return -7;
  if (M > 2 && !q2) return -8;
  if (M > 0 && ncol > 0 && !Z) return -9;
  if (ldz < (M > 1 ? M : 1)) return -10;
  if (M <= 1 || ncol == 0) return GEP_OK;
  Arena ar(h->ws, h->ws_bytes);
  size_t n = backtransform_ws_elems(M, ncol);
  double* ws = ar.take<double>(n);
  if (!ar.ok) return GEP_ERR_ALLOC;
  GEP_CHECK(apply_q2(h, M, b, q2, Z, ldz, ncol, GEP_PREC_FP64, nullptr, 0));
  return backtransform_q(h, M, ncol, C, ldc, tau1, Z, ldz, ws, n, GEP_PREC_FP64, b);
}

int gep_solve(gep_handle_t h, int M, double* A, int lda, double* B, int ldb, double* w, double* Y,
              int ldy, const gep_options* o) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !A) return -3;
  if (lda < (M > 1 ? M : 1)) return -4;
  if (M > 0 && !B) return -5;
  if (ldb < (M > 1 ? M : 1)) return -6;
  if (M > 0 && !w) return -7;
  if (!o) return -10;
  if (o->n_want < 0 || o->n_want > M) return -10;
  if (o->want_vectors && M > 0 && !Y) return -8;
  if (o->want_vectors && ldy < (M > 1 ? M : 1)) return -9;
  GEP_CHECK(check_opts(o));
  if (M == 0) return GEP_OK;
  const int n = o->n_want > 0 ? o->n_want : M;  // eigenpairs wanted (the lowest n)
  SolveLayout Ly = layout(M, o);
  if (h->ws == nullptr || h->ws_bytes < Ly.end) return GEP_ERR_ALLOC;
  const int eng = o->precision;
  char* base = h->ws;
  double* Cw = o->overwrite ? A : (double*)(base + Ly.Cw);
  int ldcw = o->overwrite ? lda : M;
  double* Lw = o->overwrite ? B : (double*)(base + Ly.Lw);
  int ldlw = o->overwrite ? ldb : M;
  double* invD = (double*)(base + Ly.invD);
  double* dvec = (double*)(base + Ly.vec);
  double* evec = dvec + (M + 1);
  double* tvec = evec + (M + 1);
  char* uni = base + Ly.uni;
  h->eng_ws = Ly.eng_bytes ? base + Ly.eng : nullptr;
  h->eng_bytes = Ly.eng_bytes;
  h->timers_recorded = false;

  GEP_CHECK(reset_status(h));
  GEP_CHECK(scan_nonfinite(h, M, A, lda));
  GEP_CHECK(scan_nonfinite(h, M, B, ldb));
  const bool mixed = o->precision == GEP_PREC_MIXED_REFINED;
  double* Af = (double*)(base + Ly.af);
  double* Bf = Af + align256((size_t)M * M * sizeof(double)) / sizeof(double);
  if (mixed) {  // the refinement needs the original pencil, as full symmetric matrices
    GEP_CHECK(copy_lower(h, M, A, lda, Af, M));
    GEP_CHECK(symmetrize_lower(h, M, Af, M));
    GEP_CHECK(copy_lower(h, M, B, ldb, Bf, M));
    GEP_CHECK(symmetrize_lower(h, M, Bf, M));
  }
  if (!o->overwrite) {
    GEP_CHECK(copy_lower(h, M, A, lda, Cw, ldcw));
    GEP_CHECK(copy_lower(h, M, B, ldb, Lw, ldlw));
  }
  double* wB = tvec + (M + 1);  // eigenvalues D of B (Cholesky-free reducer)
  double* wT = wB + (M + 1);     // all eigenvalues of T when only the lowest n are wanted
  double* Zt = partial_vectors(M, o) ? (double*)(base + Ly.zt) : nullptr;
  double* q2u = q2_tiles_ahead(o) ? (double*)(base + Ly.q2u) : nullptr;
  h->band_recorded = two_stage(o) && o->timers;
  double* q2 = (two_stage(o) && sep_vectors(o)) ? (double*)(base + Ly.q2) : nullptr;
  mark(h, o, 0);
  if (eigenexa(o)) {
    // Eq. 7: B W = W D by the SEP solver (B's copy becomes its reflectors), X = W D^-1/2
    double* Xw = (double*)(base + Ly.xw);
    GEP_CHECK(sep_solve(h, M, Lw, ldlw, o, dvec, evec, tvec, q2, uni, Ly.uni_bytes, eng, wB, Xw, M, false, 0, nullptr,
                        nullptr, q2u));
    GEP_CHECK(scale_cols_rsqrt_checked(h, M, M, wB, Xw, M));  // status k: k eigenvalues of B <= 0
    mark(h, o, 1);
    // Eq. 8: A' = X^T (A X), lower triangle (all the SEP solver reads)
    double* T = (double*)uni;
    GEP_CHECK(dgemm(h, 'S', 'N', 'F', M, M, M, 1.0, Cw, ldcw, Xw, M, 0.0, T, M, eng));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, Xw, M, T, M, 0.0, Cw, ldcw, eng));
    mark(h, o, 2);
    // A' Z = Z Lambda (Z into B's buffer, no longer needed), then Eq. 9: Y = X Z
    double* Z = o->want_vectors ? Lw : nullptr;
    GEP_CHECK(sep_solve(h, M, Cw, ldcw, o, dvec, evec, tvec, q2, uni, Ly.uni_bytes, eng, w, Z, ldlw, true, n, Zt,
                        wT, q2u));
    if (!o->want_vectors) {
      mark(h, o, 5);
      mark(h, o, 6);
      mark(h, o, 7);
      h->timers_recorded = o->timers != 0;
      return GEP_OK;
    }
    mark(h, o, 5);
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, n, M, 1.0, Xw, M, Z, ldlw, 0.0, Y, ldy, eng));
    mark(h, o, 6);
  } else {
    GEP_CHECK(cholesky(h, M, Lw, ldlw, invD, eng));  // R1
    mark(h, o, 1);
    {
      double* X = (double*)uni;
      double* tmp = (double*)(uni + r256((size_t)M * M * sizeof(double)));
      if (o->reducer == GEP_RED_TWOSIDED)
        GEP_CHECK(reduce_twosided(h, M, Cw, ldcw, Lw, ldlw, invD, X, tmp, eng));  // R2
      else {
        GEP_CHECK(reduce_explicit_inv(h, M, Cw, ldcw, Lw, ldlw, invD, X, tmp, eng));
        GEP_CHECK(zero_upper(h, M, Lw, ldlw));  // R is used as a full matrix by Eq. 6 below
      }
    }
    mark(h, o, 2);
    GEP_CHECK(sep_solve(h, M, Cw, ldcw, o, dvec, evec, tvec, q2, uni, Ly.uni_bytes, eng, w,
                        o->want_vectors ? Y : nullptr, ldy, true, n, Zt, wT, q2u));
    if (!o->want_vectors) {
      mark(h, o, 5);
      mark(h, o, 6);
      mark(h, o, 7);
      h->timers_recorded = o->timers != 0;
      return GEP_OK;
    }
    mark(h, o, 5);
    if (o->reducer == GEP_RED_TWOSIDED) {
      GEP_CHECK(trsm_llt(h, M, n, Lw, ldlw, invD, NB, Y, ldy, (double*)uni, eng));  // Eq. 6
    } else {
      double* T = (double*)uni;
      GEP_CHECK(dgemm(h, 'T', 'N', 'F', M, n, M, 1.0, Lw, ldlw, Y, ldy, 0.0, T, M, eng));  // Y = R^T Z
      GEP_CHECK(copy_matrix(h, M, n, T, M, Y, ldy));
    }
    mark(h, o, 6);
  }
  h->refine_steps = 0;
  if (mixed && o->refine_iters >= 0) {
    GEP_CHECK(refine_eigenpairs(h, M, Af, Bf, Y, ldy, w, (double*)uni, o->refine_iters, GEP_PREC_FP64_EMULATED));
  }
  mark(h, o, 7);
  GEP_CHECK(sign_convention(h, M, n, Y, ldy));
  h->timers_recorded = o->timers != 0;
  return GEP_OK;
}

int gep_adjoint_workspace_size(gep_handle_t h, int M, int n_occ, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (n_occ < 0 || n_occ > M) return -3;
  if (!bytes) return -4;
  *bytes = r256(adjoint_ws_elems(M, n_occ) * sizeof(double)) + r256(oz_workspace_bytes(M, M, M));
  return GEP_OK;
}

int gep_adjoint(gep_handle_t h, int M, int n_occ, const double* w, const double* Y, int ldy, const double* lbar,
                const double* W, int ldw, double* Abar, double* Bbar, int ldab) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (n_occ < 0 || n_occ > M) return -3;
  if (M > 0 && !w) return -4;
  if (M > 0 && !Y) return -5;
  if (ldy < (M > 1 ? M : 1)) return -6;
  if (W && ldw < (M > 1 ? M : 1)) return -9;
  if (M > 0 && (!Abar || !Bbar)) return -10;
  if (ldab < (M > 1 ? M : 1)) return -12;
  if (M == 0) return GEP_OK;
  size_t need = 0;
  GEP_CHECK(gep_adjoint_workspace_size(h, M, n_occ, &need));
  if (h->ws == nullptr || h->ws_bytes < need) return GEP_ERR_ALLOC;
  size_t main = r256(adjoint_ws_elems(M, n_occ) * sizeof(double));
  h->eng_ws = h->ws + main;
  h->eng_bytes = h->ws_bytes - main;
  return adjoint(h, M, n_occ, w, Y, ldy, lbar, W, ldw, Abar, Bbar, ldab, (double*)h->ws, GEP_PREC_FP64_EMULATED);
}

// ---------------------------------------------------------------- batched solves
namespace {

constexpr int kMaxBatch = 4096;

struct BatchPlan {
  int ns;
  int assign[kMaxBatch];  // child stream of pencil i, -1 for the one-CTA small-pencil launch
  int small_order[kMaxBatch], nsmall, small_ctas;
  size_t need[64], off[64], total, small_off;
};

int small_limit(const gep_options* o) { return o->batch_small < SMALL_MAX ? o->batch_small : SMALL_MAX; }

// Options of pencil i: opts[i] when given, else o with precision[i] (when given).
gep_options pencil_opts(const gep_options* o, const int* prec, const gep_options* opts, int i) {
  if (opts) return opts[i];
  gep_options oi = *o;
  if (prec) oi.precision = prec[i];
  return oi;
}

int make_plan(gep_handle_t h, int count, const int* M, const gep_options* o, const int* prec,
              const gep_options* opts, int nstreams, BatchPlan* p) {
  if (count < 0 || count > kMaxBatch) return -2;
  if (nstreams < 1 || nstreams > 64) return -7;
  int order[kMaxBatch];
  bool small_of[kMaxBatch];
  for (int i = 0; i < count; ++i) {
    const gep_options oi = pencil_opts(o, prec, opts, i);
    if (oi.batch_small < 0) return -4;
    if (M[i] < 0) return -3;
    order[i] = i;
    small_of[i] = M[i] >= 1 && M[i] <= small_limit(&oi);
  }
  for (int a = 1; a < count; ++a) {  // stable insertion sort, M descending
    int t = order[a], b = a - 1;
    while (b >= 0 && M[order[b]] < M[t]) { order[b + 1] = order[b]; --b; }
    order[b + 1] = t;
  }
  p->nsmall = 0;
  for (int a = 0; a < count; ++a)
    if (small_of[order[a]]) p->small_order[p->nsmall++] = order[a];
  const int nbig = count - p->nsmall;
  p->ns = nstreams < nbig ? nstreams : (nbig > 0 ? nbig : 1);
  double load[64] = {};
  for (int s = 0; s < 64; ++s) p->need[s] = 0;
  for (int a = 0; a < count; ++a) {
    int i = order[a];
    if (small_of[i]) {
      p->assign[i] = -1;
      continue;
    }
    int best = 0;
    for (int s = 1; s < p->ns; ++s)
      if (load[s] < load[best]) best = s;
    p->assign[i] = best;
    load[best] += (double)M[i] * M[i] * M[i];
    const gep_options oi = pencil_opts(o, prec, opts, i);
    size_t need = layout(M[i], &oi).end;
    if (need > p->need[best]) p->need[best] = need;
  }
  size_t off = 0;
  for (int s = 0; s < p->ns; ++s) {
    p->off[s] = off;
    off += r256(p->need[s]);
  }
  p->small_off = off;
  p->small_ctas = p->nsmall < 2 * h->sm_count ? p->nsmall : 2 * h->sm_count;
  off += p->nsmall ? r256(small_gep_scratch_bytes(p->small_ctas)) : 0;
  p->total = off;
  return GEP_OK;
}

int batched_workspace_size(gep_handle_t h, int count, const int* M, const gep_options* o, const int* prec,
                           const gep_options* opts, int nstreams, size_t* bytes) {
  static BatchPlan plan;
  GEP_CHECK(make_plan(h, count, M, o, prec, opts, nstreams, &plan));
  *bytes = plan.total;
  return GEP_OK;
}

int solve_batched(gep_handle_t h, int count, const int* M, double* const* A, double* const* B, double* const* w,
                  double* const* Y, const gep_options* o, const int* precision, const gep_options* opts,
                  int nstreams) {
  for (int i = 0; i < count; ++i) {
    const gep_options oi = pencil_opts(o, precision, opts, i);
    GEP_CHECK(check_opts(&oi));
    if (oi.n_want != 0) return GEP_ERR_UNSUPPORTED;
  }
  if (count == 0) return GEP_OK;
  static BatchPlan plan;
  GEP_CHECK(make_plan(h, count, M, o, precision, opts, nstreams, &plan));
  if (h->ws == nullptr || h->ws_bytes < plan.total) return GEP_ERR_ALLOC;
  // child handles, streams and events are created once (outside any stream capture)
  if (!h->fork_ev) GEP_CUDA(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
  if (!h->d_batch_info) GEP_CUDA(cudaMalloc((void**)&h->d_batch_info, sizeof(int) * 2 * kMaxBatch));
  if (!h->d_small_next) GEP_CUDA(cudaMalloc((void**)&h->d_small_next, 256));
  while (h->nchild < plan.ns) {
    int c = h->nchild;
    GEP_CUDA(cudaStreamCreateWithFlags(&h->child_stream[c], cudaStreamNonBlocking));
    GEP_CUDA(cudaEventCreateWithFlags(&h->child_done[c], cudaEventDisableTiming));
    GEP_CHECK(gep_create(&h->child[c], (void*)h->child_stream[c]));
    h->nchild++;
  }
  GEP_CUDA(cudaEventRecord(h->fork_ev, h->stream));
  for (int s = 0; s < plan.ns; ++s) GEP_CUDA(cudaStreamWaitEvent(h->child_stream[s], h->fork_ev, 0));
  if (plan.nsmall > 0)  // the small pencils, on the handle's stream while the children run
    GEP_CHECK(small_gep_batched(h, h->stream, plan.nsmall, M, A, B, w, Y, plan.small_order,
                                (double*)(h->ws + plan.small_off), plan.small_ctas, h->d_small_next,
                                h->d_batch_info));
  for (int i = 0; i < count; ++i) {
    int s = plan.assign[i];
    if (s < 0) continue;
    gep_handle_t c = h->child[s];
    c->ws = h->ws + plan.off[s];
    c->ws_bytes = plan.need[s];
    gep_options oi = pencil_opts(o, precision, opts, i);
    oi.timers = 0;
    GEP_CHECK(gep_solve(c, M[i], A[i], M[i] > 1 ? M[i] : 1, B[i], M[i] > 1 ? M[i] : 1, w[i], Y[i],
                        M[i] > 1 ? M[i] : 1, &oi));
    GEP_CUDA(cudaMemcpyAsync(h->d_batch_info + 2 * i, c->d_status, 2 * sizeof(int), cudaMemcpyDeviceToDevice,
                             c->stream));
    h->launches += c->launches;  // the children's kernel launches count as the batch's
    c->launches = 0;
  }
  for (int s = 0; s < plan.ns; ++s) {
    GEP_CUDA(cudaEventRecord(h->child_done[s], h->child_stream[s]));
    GEP_CUDA(cudaStreamWaitEvent(h->stream, h->child_done[s], 0));
  }
  h->batch_count = count;
  return GEP_OK;
}

}  // namespace

int gep_solve_batched_workspace_size(gep_handle_t h, int count, const int* M, const gep_options* o,
                                     const int* precision, int nstreams, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (count > 0 && !M) return -3;
  if (!o) return -4;
  if (!bytes) return -7;
  return batched_workspace_size(h, count, M, o, precision, nullptr, nstreams, bytes);
}

int gep_solve_batched(gep_handle_t h, int count, const int* M, double* const* A, double* const* B, double* const* w,
                      double* const* Y, const gep_options* o, const int* precision, int nstreams) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (count < 0 || count > kMaxBatch) return -2;
  if (count > 0 && (!M || !A || !B || !w || !Y)) return -3;
  if (!o) return -8;
  if (nstreams < 1 || nstreams > 64) return -10;
  return solve_batched(h, count, M, A, B, w, Y, o, precision, nullptr, nstreams);
}

int gep_solve_batched_opts_workspace_size(gep_handle_t h, int count, const int* M, const gep_options* opts,
                                          int nstreams, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (count < 0 || count > kMaxBatch) return -2;
  if (count > 0 && !M) return -3;
  if (count > 0 && !opts) return -4;
  if (nstreams < 1 || nstreams > 64) return -5;
  if (!bytes) return -6;
  return batched_workspace_size(h, count, M, nullptr, nullptr, opts, nstreams, bytes);
}

int gep_solve_batched_opts(gep_handle_t h, int count, const int* M, double* const* A, double* const* B,
                           double* const* w, double* const* Y, const gep_options* opts, int nstreams) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (count < 0 || count > kMaxBatch) return -2;
  if (count > 0 && (!M || !A || !B || !w || !Y)) return -3;
  if (count > 0 && !opts) return -8;
  if (nstreams < 1 || nstreams > 64) return -9;
  return solve_batched(h, count, M, A, B, w, Y, nullptr, nullptr, opts, nstreams);
}

int gep_batched_info(gep_handle_t h, int* info) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (!info) return -2;
  *info = 0;
  if (!h->d_batch_info || h->batch_count == 0) return GEP_OK;
  static int st[2 * kMaxBatch];
  GEP_CUDA(cudaStreamSynchronize(h->stream));
  GEP_CUDA(cudaMemcpy(st, h->d_batch_info, sizeof(int) * 2 * h->batch_count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < h->batch_count; ++i) {
    int v = st[2 * i + 1] != 0 ? st[2 * i + 1] : st[2 * i];
    if (v != 0) { *info = v; break; }
  }
  return GEP_OK;
}

int gep_workspace_size_host(gep_handle_t h, int M, const gep_options* o, size_t* bytes) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (!o) return -3;
  if (!bytes) return -4;
  gep_options oo = *o;
  oo.overwrite = 1;
  size_t mm = (size_t)M * M * sizeof(double);
  *bytes = layout(M, &oo).end + 3 * r256(mm) + r256((size_t)(M + 1) * sizeof(double));
  return GEP_OK;
}

int gep_solve_host(gep_handle_t h, int M, const double* A, int lda, const double* B, int ldb, double* w,
                   double* Y, int ldy, const gep_options* o) {
  if (!handle_ok(h)) return GEP_ERR_HANDLE;
  if (M < 0) return -2;
  if (M > 0 && !A) return -3;
  if (lda < (M > 1 ? M : 1)) return -4;
  if (M > 0 && !B) return -5;
  if (ldb < (M > 1 ? M : 1)) return -6;
  if (M > 0 && !w) return -7;
  if (!o) return -10;
  if (o->n_want < 0 || o->n_want > M) return -10;
  if (o->want_vectors && M > 0 && !Y) return -8;
  if (o->want_vectors && ldy < (M > 1 ? M : 1)) return -9;
  GEP_CHECK(check_opts(o));
  if (M == 0) return GEP_OK;
  const int n = o->n_want > 0 ? o->n_want : M;
  size_t need = 0;
  GEP_CHECK(gep_workspace_size_host(h, M, o, &need));
  if (h->ws == nullptr || h->ws_bytes < need) return GEP_ERR_ALLOC;
  gep_options oo = *o;
  oo.overwrite = 1;
  size_t mm = (size_t)M * M * sizeof(double);
  size_t inner = layout(M, &oo).end;
  char* base = h->ws;
  double* dA = (double*)(base + inner);
  double* dB = (double*)(base + inner + r256(mm));
  double* dY = (double*)(base + inner + 2 * r256(mm));
  double* dw = (double*)(base + inner + 3 * r256(mm));
  cudaStream_t s = h->stream;
  GEP_CUDA(cudaMemcpy2DAsync(dA, (size_t)M * sizeof(double), A, (size_t)lda * sizeof(double), (size_t)M * sizeof(double),
                             M, cudaMemcpyHostToDevice, s));
  GEP_CUDA(cudaMemcpy2DAsync(dB, (size_t)M * sizeof(double), B, (size_t)ldb * sizeof(double), (size_t)M * sizeof(double),
                             M, cudaMemcpyHostToDevice, s));
  // the inner solve must not see the H2D buffers as workspace
  char* saved_ws = h->ws;
  size_t saved_b = h->ws_bytes;
  h->ws_bytes = inner;
  int rc = gep_solve(h, M, dA, M, dB, M, dw, dY, M, &oo);
  h->ws = saved_ws;
  h->ws_bytes = saved_b;
  if (rc != GEP_OK) return rc;
  GEP_CUDA(cudaMemcpyAsync(w, dw, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (o->want_vectors)
    GEP_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * sizeof(double), dY, (size_t)M * sizeof(double), (size_t)M * sizeof(double),
                               n, cudaMemcpyDeviceToHost, s));
  GEP_CUDA(cudaStreamSynchronize(s));
  return GEP_OK;
}

}  // extern "C"
