// Small pencils of a batched solve, each solved whole by one CTA in one persistent launch.
//
// A batch of uneven orders (per-k-point or per-fragment Hamiltonians) holds many small
// pencils whose solve through the staged workflow costs hundreds of kernel launches for
// little arithmetic.  Pencils of order k <= SMALL_MAX are instead taken from a device work
// queue (largest k^3 first, the order the host sorted them in) by the CTAs of one launch;
// each CTA solves its pencil exactly in FP64 with the shared one-CTA solver (Cholesky of
// B, C = L^-1 A L^-T, cyclic Jacobi, Y = L^-T Q, Eq. 4-6), applies the sign convention and
// writes w and Y.  The pencil table travels by value in the kernel parameters, so a CUDA
// graph that captured the launch carries it too.
#include "cta_eig.cuh"

namespace gep {
namespace {

struct SmallTable {
  const double* A[SMALL_PER_LAUNCH];
  const double* B[SMALL_PER_LAUNCH];
  double* w[SMALL_PER_LAUNCH];
  double* Y[SMALL_PER_LAUNCH];
  int M[SMALL_PER_LAUNCH];
  int idx[SMALL_PER_LAUNCH];  // position in the caller's batch (status slot)
  int count;
};

// info[2 idx] = k > 0 when B's leading minor k is not positive definite, info[2 idx + 1] =
// GEP_ERR_NONFINITE for a NaN or Inf in the lower triangle of A or B; both 0 otherwise.
__global__ void __launch_bounds__(256) k_small_gep(const __grid_constant__ SmallTable T, int* next,
                                                   double* __restrict__ scratch, size_t per_cta, int* info) {
  __shared__ CtaEigShared sh;
  __shared__ int q, bad;
  double* L = scratch + (size_t)blockIdx.x * per_cta;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    if (tid == 0) {
      q = atomicAdd(next, 1);
      bad = 0;
    }
    __syncthreads();
    const int i = q;
    if (i >= T.count) break;
    const int k = T.M[i];
    const double* A = T.A[i];
    const double* B = T.B[i];
    double* Cm = L + (size_t)k * k;
    double* V = Cm + (size_t)k * k;
    int nonfinite = 0;
    for (int idx = tid; idx < k * k; idx += nt) {  // symmetric from the lower triangles
      const int r = idx % k, c = idx / k;
      const int a = max(r, c), b = min(r, c);
      const double bv = B[a + (size_t)b * k], av = A[a + (size_t)b * k];
      nonfinite |= !isfinite(bv) || !isfinite(av);
      L[idx] = bv;
      Cm[idx] = av;
    }
    if (nonfinite) atomicOr(&bad, 1);
    __syncthreads();
    const int slot = T.idx[i];
    if (bad) {
      if (tid == 0) {
        info[2 * slot] = 0;
        info[2 * slot + 1] = GEP_ERR_NONFINITE;
      }
      __syncthreads();
      continue;
    }
    const int fail = cta_pencil_eig(k, L, Cm, V, sh, true);
    if (tid == 0) {
      info[2 * slot] = fail;
      info[2 * slot + 1] = 0;
    }
    if (fail) {
      __syncthreads();
      continue;
    }
    // sign convention (largest-magnitude entry positive, lowest row on ties); one warp per column
    double* w = T.w[i];
    double* Y = T.Y[i];
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < k; j += nt >> 5) {
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int r = lane; r < k; r += 32) {
        const double a = fabs(V[r + (size_t)j * k]);
        if (a > best) { best = a; bi = r; }
      }
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const double s = (bi < k && V[bi + (size_t)j * k] < 0.0) ? -1.0 : 1.0;
      for (int r = lane; r < k; r += 32) Y[r + (size_t)j * k] = s * V[r + (size_t)j * k];
      if (lane == 0) w[j] = Cm[j + (size_t)j * k];
    }
    __syncthreads();
  }
}

}  // namespace

size_t small_gep_scratch_bytes(int ctas) { return (size_t)ctas * 3 * SMALL_MAX * SMALL_MAX * sizeof(double); }

int small_gep_batched(gep_handle_t h, cudaStream_t s, int count, const int* M, double* const* A, double* const* B,
                      double* const* w, double* const* Y, const int* order, double* scratch, int ctas, int* next,
                      int* info) {
  const size_t per_cta = (size_t)3 * SMALL_MAX * SMALL_MAX;
  for (int first = 0; first < count; first += SMALL_PER_LAUNCH) {
    SmallTable T;
    T.count = count - first < SMALL_PER_LAUNCH ? count - first : SMALL_PER_LAUNCH;
    for (int t = 0; t < T.count; ++t) {
      const int i = order[first + t];
      if (M[i] < 1 || M[i] > SMALL_MAX) return GEP_ERR_UNSUPPORTED;
      T.A[t] = A[i];
      T.B[t] = B[i];
      T.w[t] = w[i];
      T.Y[t] = Y[i];
      T.M[t] = M[i];
      T.idx[t] = i;
    }
    GEP_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
    const int grid = T.count < ctas ? T.count : ctas;
    k_small_gep<<<grid, 256, 0, s>>>(T, next, scratch, per_cta, info);
    GEP_CHECK(check_launch(h));
  }
  return GEP_OK;
}

}  // namespace gep
