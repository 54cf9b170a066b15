// One-CTA exact solver of a small symmetric-definite pencil (S, R), S y = mu R y, of order
// k <= CTA_EIG_KMAX, shared by the FP64 refinement (clusters of near-degenerate eigenpairs)
// and the fused solver of small batched pencils.  Every step is spread over the CTA's
// threads; the matrices live in global scratch (column-major, ld k):
//   L = R on entry -> Cholesky factor L (R = L L^T, lower triangle);
//   Cm = S on entry -> C = L^-1 S L^-T -> diagonal (mu ascending) after cyclic Jacobi;
//   V -> W = L^-T Q: R-orthonormal eigenvectors, column j for mu_j = Cm(j, j).
// The Jacobi rotations run in round-robin order: the k/2 rotations of a round act on
// disjoint index pairs and are applied together (columns of C and V, then rows of C).
#pragma once

#include "gep_internal.cuh"

namespace gep {

constexpr int CTA_EIG_KMAX = 256;

struct CtaEigShared {
  double csv[CTA_EIG_KMAX / 2], snv[CTA_EIG_KMAX / 2], red[32];
  int pa[CTA_EIG_KMAX / 2], pb[CTA_EIG_KMAX / 2], pos[CTA_EIG_KMAX];
  int done, fail;
};

// Sum over the CTA (blockDim.x a multiple of 32, at most 1024); every thread gets the total.
__device__ __forceinline__ double cta_sum(double v, CtaEigShared& sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh.red[w];
  __syncthreads();
  return t;
}

// Returns 0, or j + 1 when the Cholesky pivot j of R is not positive (detect = true; then
// nothing else is computed).  With detect = false such a pivot is clamped to 1e-150 (R is a
// Gram matrix of nearly R-orthonormal vectors there and cannot lose definiteness).
__device__ __forceinline__ int cta_pencil_eig(int k, double* L, double* Cm, double* V, CtaEigShared& sh, bool detect) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) sh.fail = 0;
  for (int idx = tid; idx < k * k; idx += nt) V[idx] = (idx % k == idx / k) ? 1.0 : 0.0;
  __syncthreads();
  // Cholesky R = L L^T (right-looking, lower triangle)
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double p = L[j + j * k];
      if (!(p > 0.0) || !isfinite(p)) {
        if (detect) sh.fail = j + 1;
        L[j + j * k] = 1e-150;
      } else {
        L[j + j * k] = sqrt(p);
      }
    }
    __syncthreads();
    if (sh.fail) return sh.fail;
    const double d = L[j + j * k];
    for (int i = j + 1 + tid; i < k; i += nt) L[i + j * k] /= d;
    __syncthreads();
    const int w = k - j - 1;
    for (int t = tid; t < w * w; t += nt) {
      int i = j + 1 + t % w, q = j + 1 + t / w;
      if (i >= q) L[i + q * k] -= L[i + j * k] * L[q + j * k];
    }
    __syncthreads();
  }
  // Cm <- L^-1 Cm (each column a forward substitution), then Cm <- Cm L^-T (each row)
  for (int q = tid; q < k; q += nt)
    for (int i = 0; i < k; ++i) {
      double t = Cm[i + q * k];
      for (int p = 0; p < i; ++p) t -= L[i + p * k] * Cm[p + q * k];
      Cm[i + q * k] = t / L[i + i * k];
    }
  __syncthreads();
  for (int i = tid; i < k; i += nt)
    for (int q = 0; q < k; ++q) {
      double t = Cm[i + q * k];
      for (int p = 0; p < q; ++p) t -= Cm[i + p * k] * L[q + p * k];
      Cm[i + q * k] = t / L[q + q * k];
    }
  __syncthreads();
  // parallel cyclic Jacobi: n = k rounded up to even (index k, if present, is a dummy)
  const int n = (k + 1) & ~1, half = n / 2;
  for (int i = tid; i < n; i += nt) sh.pos[i] = i;
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < k * k; idx += nt) {
      const double x = Cm[idx];
      tot += x * x;
      if (idx % k != idx / k) off += x * x;
    }
    off = cta_sum(off, sh);
    tot = cta_sum(tot, sh);
    if (off <= 1e-28 * tot) break;  // off-diagonal entries ~1e-14 of the matrix: FP64 level
    for (int round = 0; round < n - 1; ++round) {
      for (int t = tid; t < half; t += nt) {
        const int a = sh.pos[t], b = sh.pos[n - 1 - t];
        const int p = min(a, b), q = max(a, b);
        double cs = 1.0, sn = 0.0;
        if (q < k) {
          const double apq = 0.5 * (Cm[p + q * k] + Cm[q + p * k]);
          if (apq != 0.0) {
            const double th = (Cm[q + q * k] - Cm[p + p * k]) / (2.0 * apq);
            const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            cs = 1.0 / sqrt(tt * tt + 1.0);
            sn = tt * cs;
          }
        }
        sh.pa[t] = p;
        sh.pb[t] = q;
        sh.csv[t] = cs;
        sh.snv[t] = sn;
      }
      __syncthreads();
      for (int idx = tid; idx < half * k; idx += nt) {  // columns of Cm and V
        const int t = idx / k, r = idx % k;
        if (sh.pb[t] >= k || sh.snv[t] == 0.0) continue;
        const int p = sh.pa[t], q = sh.pb[t];
        const double cs = sh.csv[t], sn = sh.snv[t];
        double x = Cm[r + p * k], y = Cm[r + q * k];
        Cm[r + p * k] = cs * x - sn * y;
        Cm[r + q * k] = sn * x + cs * y;
        x = V[r + p * k];
        y = V[r + q * k];
        V[r + p * k] = cs * x - sn * y;
        V[r + q * k] = sn * x + cs * y;
      }
      __syncthreads();
      for (int idx = tid; idx < half * k; idx += nt) {  // rows of Cm
        const int t = idx / k, r = idx % k;
        if (sh.pb[t] >= k || sh.snv[t] == 0.0) continue;
        const int p = sh.pa[t], q = sh.pb[t];
        const double cs = sh.csv[t], sn = sh.snv[t];
        const double x = Cm[p + r * k], y = Cm[q + r * k];
        Cm[p + r * k] = cs * x - sn * y;
        Cm[q + r * k] = sn * x + cs * y;
      }
      __syncthreads();
      if (tid == 0) {  // round-robin: position 0 stays, the others rotate by one
        const int last = sh.pos[n - 1];
        for (int i = n - 1; i > 1; --i) sh.pos[i] = sh.pos[i - 1];
        sh.pos[1] = last;
      }
      __syncthreads();
    }
  }
  // ascending order of the eigenvalues (selection sort; column swaps in parallel)
  for (int a = 0; a < k; ++a) {
    if (tid == 0) {
      int m = a;
      for (int b = a + 1; b < k; ++b)
        if (Cm[b + b * k] < Cm[m + m * k]) m = b;
      sh.pos[0] = m;
    }
    __syncthreads();
    const int m = sh.pos[0];
    if (m != a) {
      for (int r = tid; r < k; r += nt) {
        const double x = V[r + a * k];
        V[r + a * k] = V[r + m * k];
        V[r + m * k] = x;
      }
      if (tid == 0) {
        const double t = Cm[a + a * k];
        Cm[a + a * k] = Cm[m + m * k];
        Cm[m + m * k] = t;
      }
    }
    __syncthreads();
  }
  // W = L^-T V (each column a back substitution)
  for (int q = tid; q < k; q += nt)
    for (int i = k - 1; i >= 0; --i) {
      double t = V[i + q * k];
      for (int p = i + 1; p < k; ++p) t -= L[p + i * k] * V[p + q * k];
      V[i + q * k] = t / L[i + i * k];
    }
  __syncthreads();
  return 0;
}

}  // namespace gep
