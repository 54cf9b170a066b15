// FP64 refinement of all eigenpairs of the pencil (A, B) (mixed-precision path).
//
// From an approximate X (columns ~ eigenvectors, X^T B X ~ I) of a lower-precision
// solve, one step forms, with FP64-accurate products,
//     S = X^T A X,   R = X^T B X,   lambda_i = S_ii / R_ii  (B-Rayleigh quotients),
// and the first-order correction X <- X (I + E) that makes X^T B X = I and X^T A X
// diagonal to first order:
//     E_ii = (1 - R_ii) / 2,
//     E_ij = (S_ij - lambda_j R_ij) / (lambda_j - lambda_i)      (i != j).
// This is the Ogita-Aishima refinement for the symmetric eigenproblem written in the
// B inner product; it converges quadratically for well-separated eigenvalues.  A pair
// whose gap is below max(THETA res_ij, OMEGA_GLOBAL max res, OMEGA_FLOOR max|lambda|),
// res_ij = |S_ij - lambda_j R_ij|, cannot take the first-order formula (its E_ij would
// not be small, or its second-order remainder would exceed FP64 rounding); such pairs
// are joined into clusters of consecutive indices.  Inside a cluster C the k x k pencil
// (S_CC, R_CC) is solved exactly (Cholesky + cyclic Jacobi, one thread per cluster),
// W_C = its B-orthonormal eigenvectors, and the block update is
//     E_CC = W_C - I,   E_{out,C} <- E_{out,C} W_C
// (the corrections from outside the cluster follow the rotated cluster basis).
#include <math.h>

#include "gep_internal.cuh"
#include "cta_eig.cuh"

namespace gep {
namespace {

// lambda_i = S_ii / R_ii; also conv[0] = max |lambda| (block reduction, one CTA);
// conv[2], conv[3] <- 0 for the atomic maxima that follow.
__global__ void __launch_bounds__(1024) k_rayleigh(int M, const double* __restrict__ S, const double* __restrict__ R,
                                                   double* __restrict__ lam, double* __restrict__ conv,
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
    conv[0] = r;
    conv[2] = 0.0;
    conv[3] = 0.0;
  }
}

constexpr int KMAX = 32;              // largest cluster solved by one thread, also the pair window
constexpr int KBIG = 256;             // largest cluster solved exactly (one CTA above KMAX)
constexpr double THETA = 64;          // |gap| < THETA res_ij: first-order step not small
constexpr double OMEGA_GLOBAL = 16;   // |gap| < 16 max res: below the current error level
constexpr double OMEGA_FLOOR = 1e-6;  // |gap| < 1e-6 max|lambda|: unresolvable at FP64

// conv[3] (bits of a non-negative double, ordered by an integer atomicMax) =
// max over i != j of |S_ij - lambda_j R_ij|.
__global__ void k_offmax(int M, const double* __restrict__ S, const double* __restrict__ R,
                         const double* __restrict__ lam, unsigned long long* off, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  for (int j = blockIdx.y; j < M; j += gridDim.y) {
    if (i >= M || i <= j) continue;  // strictly lower: (i, j) and (j, i) both checked
    double s = S[GEP_IX(i, j, M)], r = R[GEP_IX(i, j, M)];
    m = fmax(m, fmax(fabs(s - lam[j] * r), fabs(s - lam[i] * r)));
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(off, (unsigned long long)__double_as_longlong(m));
}

// far[i] = largest j in (i, i + KMAX] whose pair with i the first-order formula cannot
// take (far[i] = i when there is none).
__global__ void k_pair_far(int M, const double* __restrict__ S, const double* __restrict__ R,
                           const double* __restrict__ lam, const double* __restrict__ conv, int* __restrict__ far,
                           const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double omega = fmax(OMEGA_GLOBAL * __longlong_as_double(((const long long*)conv)[3]), OMEGA_FLOOR * conv[0]);
  int f = i;
  double li = lam[i];
  int jend = i + KMAX < M - 1 ? i + KMAX : M - 1;
  for (int j = i + 1; j <= jend; ++j) {
    double s = S[GEP_IX(j, i, M)], r = R[GEP_IX(j, i, M)], lj = lam[j];
    double res = fmax(fabs(s - lj * r), fabs(s - li * r));
    if (fabs(lj - li) < fmax(THETA * res, omega)) f = j;
  }
  far[i] = f;
}

// Clusters = unions of the overlapping index ranges [i, far[i]] (serial scan, one
// thread): cstart/csize/coff (scratch offset) per cluster, ncl[0] = number of clusters,
// cid[i] = the cluster of index i when that cluster is solved exactly (k <= KBIG),
// -2 - c when i lies in cluster c of more than KBIG members (chained near-degenerate
// eigenvalues; its inner pairs take the first-order step where their own gap is safe and
// only get their B-orthogonality restored otherwise), else -1.
// Scratch use is sum 3 k^2 <= 3 M min(M, KBIG).
__global__ void k_clusters(int M, const int* __restrict__ far, int* cstart, int* csize, long long* coff, int* cid,
                           int* ncl, const int* st) {
  if (status_bad(st)) return;
  int nc = 0, i = 0;
  long long used = 0;
  while (i < M) {
    int end = far[i], j = i + 1;
    while (j <= end) {
      end = max(end, far[j]);
      ++j;
    }
    int k = end - i + 1;
    if (k > 1) {
      cstart[nc] = i;
      csize[nc] = k;
      coff[nc] = used;
      if (k <= KBIG) used += 3LL * k * k;
    }
    for (int q = i; q <= end; ++q) cid[q] = (k > 1 && k <= KBIG) ? nc : (k > KBIG ? -2 - nc : -1);
    if (k > 1) ++nc;
    i = end + 1;
  }
  ncl[0] = nc;
}

// E from the lower triangles of S and R (both symmetric).  Numerically degenerate pairs
// (|gap| <= delta) only get their B-orthogonality restored: E_ij = -R_ij / 2.  Pairs
// inside an exactly solved cluster are written by k_cluster_solve.  conv[2] (bits,
// integer atomicMax) = the size of this step: max of |E_ij| over first-order pairs,
// |R_ij| over pairs inside clusters and |1 - R_ii| (the rotation inside a degenerate
// cluster is arbitrary and does not count).
__global__ void k_refine_E(int M, const double* __restrict__ S, const double* __restrict__ R,
                           const double* __restrict__ lam, const int* __restrict__ cid, double* __restrict__ conv,
                           double rel_delta, double* __restrict__ E, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double delta = rel_delta * conv[0];
  double m = 0.0;
  for (int j = blockIdx.y; j < M; j += gridDim.y) {
    if (i >= M) continue;
    double e;
    int a = i > j ? i : j, b = i > j ? j : i;  // lower-triangle index
    double rij = R[GEP_IX(a, b, M)];
    if (i == j) {
      e = 0.5 * (1.0 - rij);
      m = fmax(m, fabs(2.0 * e));
    } else if (cid[i] >= 0 && cid[i] == cid[j]) {
      e = 0.0;
      m = fmax(m, fabs(rij));
    } else if (cid[i] <= -2 && cid[i] == cid[j]) {
      // inside a cluster too large to solve exactly (a chain formed through the global
      // threshold): the first-order step where the pair's own gap allows it, else restore
      // B-orthogonality only
      const double gap = lam[j] - lam[i], sij = S[GEP_IX(a, b, M)];
      const double res = fmax(fabs(sij - lam[j] * rij), fabs(sij - lam[i] * rij));
      if (fabs(gap) > fmax(THETA * res, delta)) {
        e = (sij - lam[j] * rij) / gap;
        m = fmax(m, fabs(e));
      } else {
        e = -0.5 * rij;
        m = fmax(m, fabs(rij));
      }
    } else {
      double gap = lam[j] - lam[i];
      if (fabs(gap) <= delta) e = -0.5 * rij;
      else e = (S[GEP_IX(a, b, M)] - lam[j] * rij) / gap;
      m = fmax(m, fabs(e));
    }
    E[GEP_IX(i, j, M)] = e;
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(conv + 2), (unsigned long long)__double_as_longlong(m));
}

// E_{j,C} <- E_{j,C} W_C for every row j outside each exactly solved cluster C (one
// thread per row; W_C is left in the cluster's scratch by k_cluster_solve).
__global__ void k_cluster_rotate(int M, const int* __restrict__ cstart, const int* __restrict__ csize,
                                 const long long* __restrict__ coff, const int* ncl,
                                 const double* __restrict__ scratch, double* __restrict__ E, const int* st) {
  if (status_bad(st)) return;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int nc = ncl[0];
  double row[KMAX];
  for (int c = 0; c < nc; ++c) {
    int s0 = cstart[c], k = csize[c];
    if (k > KMAX || (j >= s0 && j < s0 + k)) continue;
    const double* W = scratch + coff[c] + 2 * k * k;
    for (int q = 0; q < k; ++q) row[q] = E[GEP_IX(j, s0 + q, M)];
    for (int q = 0; q < k; ++q) {
      double t = 0.0;
      for (int p = 0; p < k; ++p) t = fma(row[p], W[p + q * k], t);
      E[GEP_IX(j, s0 + q, M)] = t;
    }
  }
}

// One thread per cluster of size k <= KMAX: solve S_CC v = mu R_CC v exactly
// (R_CC = L L^T, C = L^-1 S_CC L^-T, cyclic Jacobi on C, V = L^-T Q), write
// E_CC = W - I, keep W in the cluster's scratch (in place of V) and write the cluster's
// eigenvalues.  Larger clusters keep the first-order entries.
__global__ void k_cluster_solve(int M, const double* __restrict__ S, const double* __restrict__ R,
                                const int* __restrict__ cstart, const int* __restrict__ csize,
                                const long long* __restrict__ coff, const int* ncl, double* __restrict__ lam,
                                double* __restrict__ E, double* __restrict__ scratch,
                                const int* st) {
  if (status_bad(st)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncl[0]) return;
  int s0 = cstart[c], k = csize[c];
  if (k > KMAX) return;
  const int ld = k;  // L, Cm, V: k x k each, column-major
  double* L = scratch + coff[c];
  double* Cm = L + k * k;
  double* V = Cm + k * k;
  for (int q = 0; q < k; ++q)
    for (int p = 0; p < k; ++p) {
      int a = max(s0 + p, s0 + q), b = min(s0 + p, s0 + q);
      L[p + q * ld] = R[GEP_IX(a, b, M)];
      Cm[p + q * ld] = S[GEP_IX(a, b, M)];
    }
  // Cholesky R_CC = L L^T (lower, in place)
  for (int j = 0; j < k; ++j) {
    double d = L[j + j * ld];
    for (int q = 0; q < j; ++q) d -= L[j + q * ld] * L[j + q * ld];
    d = sqrt(fmax(d, 1e-300));
    L[j + j * ld] = d;
    for (int i = j + 1; i < k; ++i) {
      double t = L[i + j * ld];
      for (int q = 0; q < j; ++q) t -= L[i + q * ld] * L[j + q * ld];
      L[i + j * ld] = t / d;
    }
  }
  // Cm <- L^-1 Cm L^-T (two forward substitutions)
  for (int q = 0; q < k; ++q)
    for (int i = 0; i < k; ++i) {
      double t = Cm[i + q * ld];
      for (int p = 0; p < i; ++p) t -= L[i + p * ld] * Cm[p + q * ld];
      Cm[i + q * ld] = t / L[i + i * ld];
    }
  for (int i = 0; i < k; ++i)
    for (int q = 0; q < k; ++q) {
      double t = Cm[i + q * ld];
      for (int p = 0; p < q; ++p) t -= Cm[i + p * ld] * L[q + p * ld];
      Cm[i + q * ld] = t / L[q + q * ld];
    }
  for (int q = 0; q < k; ++q)
    for (int p = 0; p < k; ++p) V[p + q * ld] = (p == q) ? 1.0 : 0.0;
  // cyclic Jacobi on the symmetric Cm, rotations accumulated in V
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int q = 0; q < k; ++q)
      for (int p = 0; p < k; ++p) {
        double x = Cm[p + q * ld];
        tot += x * x;
        if (p != q) off += x * x;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double apq = 0.5 * (Cm[p + q * ld] + Cm[q + p * ld]);
        if (apq == 0.0) continue;
        double th = (Cm[q + q * ld] - Cm[p + p * ld]) / (2.0 * apq);
        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < k; ++r) {
          double x = Cm[r + p * ld], y = Cm[r + q * ld];
          Cm[r + p * ld] = cs * x - sn * y;
          Cm[r + q * ld] = sn * x + cs * y;
        }
        for (int r = 0; r < k; ++r) {
          double x = Cm[p + r * ld], y = Cm[q + r * ld];
          Cm[p + r * ld] = cs * x - sn * y;
          Cm[q + r * ld] = sn * x + cs * y;
        }
        for (int r = 0; r < k; ++r) {
          double x = V[r + p * ld], y = V[r + q * ld];
          V[r + p * ld] = cs * x - sn * y;
          V[r + q * ld] = sn * x + cs * y;
        }
      }
  }
  // ascending order of the cluster's eigenvalues (selection sort on columns of V)
  for (int a = 0; a < k; ++a) {
    int m = a;
    for (int b = a + 1; b < k; ++b)
      if (Cm[b + b * ld] < Cm[m + m * ld]) m = b;
    if (m != a) {
      double t = Cm[a + a * ld];
      Cm[a + a * ld] = Cm[m + m * ld];
      Cm[m + m * ld] = t;
      for (int r = 0; r < k; ++r) {
        double x = V[r + a * ld];
        V[r + a * ld] = V[r + m * ld];
        V[r + m * ld] = x;
      }
    }
  }
  // W = L^-T V (back substitution), E_CC = W - I
  for (int q = 0; q < k; ++q) {
    for (int i = k - 1; i >= 0; --i) {
      double t = V[i + q * ld];
      for (int p = i + 1; p < k; ++p) t -= L[p + i * ld] * V[p + q * ld];
      V[i + q * ld] = t / L[i + i * ld];
    }
    for (int p = 0; p < k; ++p) E[GEP_IX(s0 + p, s0 + q, M)] = V[p + q * ld] - (p == q ? 1.0 : 0.0);
    lam[s0 + q] = Cm[q + q * ld];
  }
}

// One CTA per cluster of KMAX < k <= KBIG members (a chain of near-degenerate eigenvalues):
// the exact solve of k_cluster_solve with its steps spread over the CTA (cta_pencil_eig).
__global__ void __launch_bounds__(256) k_cluster_solve_big(int M, const double* __restrict__ S,
                                                           const double* __restrict__ R,
                                                           const int* __restrict__ cstart,
                                                           const int* __restrict__ csize,
                                                           const long long* __restrict__ coff, const int* ncl,
                                                           double* __restrict__ lam, double* __restrict__ E,
                                                           double* __restrict__ scratch, const int* st) {
  __shared__ CtaEigShared sh;
  if (status_bad(st)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = blockIdx.x; c < ncl[0]; c += gridDim.x) {
    const int s0 = cstart[c], k = csize[c];
    if (k <= KMAX || k > KBIG) continue;
    double* L = scratch + coff[c];
    double* Cm = L + (size_t)k * k;
    double* V = Cm + (size_t)k * k;
    for (int idx = tid; idx < k * k; idx += nt) {
      int p = idx % k, q = idx / k;
      int a = max(s0 + p, s0 + q), b = min(s0 + p, s0 + q);
      L[idx] = R[GEP_IX(a, b, M)];
      Cm[idx] = S[GEP_IX(a, b, M)];
    }
    __syncthreads();
    cta_pencil_eig(k, L, Cm, V, sh, false);  // R_CC: Gram matrix of nearly B-orthonormal vectors
    for (int q = tid; q < k; q += nt) {
      for (int p = 0; p < k; ++p) E[GEP_IX(s0 + p, s0 + q, M)] = V[p + q * k] - (p == q ? 1.0 : 0.0);
      lam[s0 + q] = Cm[q + q * k];
    }
    __syncthreads();
  }
}

// E_{j,C} <- E_{j,C} W_C for the rows j outside every cluster C of KMAX < k <= KBIG members
// (W_C left in the cluster's scratch by k_cluster_solve_big); CTA: 8 rows, staged in shared
// memory, one loop over the clusters.
__global__ void __launch_bounds__(256) k_cluster_rotate_big(int M, const int* __restrict__ cstart,
                                                            const int* __restrict__ csize,
                                                            const long long* __restrict__ coff, const int* ncl,
                                                            const double* __restrict__ scratch, double* __restrict__ E,
                                                            const int* st) {
  __shared__ double rows[8][KBIG];
  if (status_bad(st)) return;
  const int j0 = blockIdx.x * 8, tid = threadIdx.x;
  const int nc = ncl[0];
  for (int c = 0; c < nc; ++c) {
    const int s0 = cstart[c], k = csize[c];
    if (k <= KMAX || k > KBIG) continue;
    const double* W = scratch + coff[c] + 2 * (size_t)k * k;
    for (int idx = tid; idx < 8 * k; idx += blockDim.x) {
      int r = idx / k, p = idx % k, j = j0 + r;
      rows[r][p] = (j < M) ? E[GEP_IX(j, s0 + p, M)] : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < 8 * k; idx += blockDim.x) {
      int r = idx / k, q = idx % k, j = j0 + r;
      if (j >= M || (j >= s0 && j < s0 + k)) continue;
      double t = 0.0;
      for (int p = 0; p < k; ++p) t = fma(rows[r][p], W[p + (size_t)q * k], t);
      E[GEP_IX(j, s0 + q, M)] = t;
    }
    __syncthreads();
  }
}

}  // namespace

size_t refine_ws_elems(int M) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  size_t kmax = M < KBIG ? (size_t)M : (size_t)KBIG;
  // T1, S, R, E; conv; far, cstart, csize, cid (ints) and coff (int64) per index; cluster scratch
  return 4 * r((size_t)M * M) + 32 + 2 * r((size_t)M) + r((size_t)M) + r(3 * (size_t)M * kmax) + 32;
}

// Af, Bf: full symmetric A and B (M x M, ld M).  X (ld ldx) refined in place, w <- lambda.
// iters > 0: exactly that many steps.  iters = 0: steps until converged (at most
// REFINE_MAX_STEPS): the step whose size (k_refine_E) is at most 1e-8 is the last, its
// second-order remainder being at FP64 rounding level; that test reads the size back to
// the host, so under stream capture a fixed REFINE_CAPTURE_STEPS steps run instead.
// The number of steps taken is left in h->refine_steps.
int refine_eigenpairs(gep_handle_t h, int M, const double* Af, const double* Bf, double* X, int ldx, double* w,
                      double* ws, int iters, int engine) {
  constexpr int REFINE_MAX_STEPS = 8, REFINE_CAPTURE_STEPS = 4;
  constexpr double REFINE_STOP = 1e-8;
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  double* T1 = ws;                        // A X, then B X, then X E
  double* S = T1 + r((size_t)M * M);
  double* R = S + r((size_t)M * M);
  double* E = R + r((size_t)M * M);
  double* conv = E + r((size_t)M * M);    // max|lambda|, -, step size (bits), max res (bits)
  int* far = reinterpret_cast<int*>(conv + 32);
  int* cstart = far + M;
  int* csize = cstart + M;
  int* cid = csize + M;  // four int arrays fit in 2 r(M) doubles
  long long* coff = reinterpret_cast<long long*>(conv + 32 + 2 * r((size_t)M));
  double* scratch = conv + 32 + 3 * r((size_t)M);
  int* ncl = reinterpret_cast<int*>(scratch + r(3 * (size_t)M * (M < KBIG ? M : KBIG)));
  bool adaptive = iters == 0;
  if (adaptive) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return GEP_ERR_CUDA;
    adaptive = cs == cudaStreamCaptureStatusNone;
    iters = adaptive ? REFINE_MAX_STEPS : REFINE_CAPTURE_STEPS;
  }
  h->refine_steps = 0;
  for (int it = 0; it < iters; ++it) {
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Af, M, X, ldx, 0.0, T1, M, engine));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, X, ldx, T1, M, 0.0, S, M, engine));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Bf, M, X, ldx, 0.0, T1, M, engine));
    GEP_CHECK(dgemm(h, 'T', 'N', 'L', M, M, M, 1.0, X, ldx, T1, M, 0.0, R, M, engine));
    k_rayleigh<<<1, 1024, 0, h->stream>>>(M, S, R, w, conv, h->d_status);
    GEP_CHECK(check_launch(h));
    dim3 g((M + 255) / 256, M < 65535 ? M : 65535);
    k_offmax<<<g, 256, 0, h->stream>>>(M, S, R, w, reinterpret_cast<unsigned long long*>(conv + 3), h->d_status);
    GEP_CHECK(check_launch(h));
    k_pair_far<<<(M + 127) / 128, 128, 0, h->stream>>>(M, S, R, w, conv, far, h->d_status);
    GEP_CHECK(check_launch(h));
    k_clusters<<<1, 1, 0, h->stream>>>(M, far, cstart, csize, coff, cid, ncl, h->d_status);
    GEP_CHECK(check_launch(h));
    k_refine_E<<<g, 256, 0, h->stream>>>(M, S, R, w, cid, conv, 1e-12, E, h->d_status);
    GEP_CHECK(check_launch(h));
    k_cluster_solve<<<(M / 2 + 64) / 64, 64, 0, h->stream>>>(M, S, R, cstart, csize, coff, ncl, w, E, scratch,
                                                             h->d_status);
    GEP_CHECK(check_launch(h));
    k_cluster_rotate<<<(M + 127) / 128, 128, 0, h->stream>>>(M, cstart, csize, coff, ncl, scratch, E, h->d_status);
    GEP_CHECK(check_launch(h));
    if (M > KMAX) {  // clusters of KMAX < k <= KBIG members (chains of near-degenerate eigenvalues)
      k_cluster_solve_big<<<h->sm_count, 256, 0, h->stream>>>(M, S, R, cstart, csize, coff, ncl, w, E, scratch,
                                                              h->d_status);
      GEP_CHECK(check_launch(h));
      k_cluster_rotate_big<<<(M + 7) / 8, 256, 0, h->stream>>>(M, cstart, csize, coff, ncl, scratch, E,
                                                               h->d_status);
      GEP_CHECK(check_launch(h));
    }
    GEP_CHECK(copy_matrix(h, M, M, X, ldx, T1, M));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, T1, M, E, M, 1.0, X, ldx, engine));   // X <- X + X E
    h->refine_steps = it + 1;
    if (adaptive) {
      double c[3];
      int sv[2] = {0, 0};
      if (cudaMemcpyAsync(c, conv, sizeof(c), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaMemcpyAsync(sv, h->d_status, sizeof(sv), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        return GEP_ERR_CUDA;
      if (sv[0] != 0 || sv[1] != 0) break;  // reported through the status word
      double e = c[2];
      if (!(e == e) || e <= REFINE_STOP) break;  // NaN: nothing more to gain
    }
  }
  return GEP_OK;
}

}  // namespace gep
