// SEP solver, stage "BACK" (Table 3): Z <- Q Z with Q = H_0 H_1 ... H_{M-2} left
// in C by the tridiagonalisation.  Reflectors are grouped in panels of NBB and
// applied from the last panel to the first in compact-WY form,
//     H_j ... H_{j+nb-1} = I - V T V^T    (T upper triangular, forward/columnwise),
//     Z(j+1:, :) -= V (T (V^T Z(j+1:, :))),
// so all O(M^3) work is three matrix products per panel.
#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int NBB = 64;

// Explicit V (rows j0+1 .. M-1, nb columns): unit entry at local row q, reflector below.
__global__ void k_build_v(int rows, int nb, int j0, const double* __restrict__ C, int ldc,
                          double* __restrict__ V, const int* st) {
  if (status_bad(st)) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int q = blockIdx.y;
  if (t >= rows || q >= nb) return;
  double val;
  if (t < q) val = 0.0;
  else if (t == q) val = 1.0;
  else val = C[GEP_IX(j0 + 1 + t, j0 + q, ldc)];
  V[GEP_IX(t, q, rows)] = val;
}

// T factor from G = V^T V:  T(i,i) = tau_i,  T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i).
__global__ void k_larft(int nb, const double* __restrict__ G, const double* __restrict__ tau,
                        double* __restrict__ T, const int* st) {
  __shared__ double Ts[NBB][NBB + 1];
  __shared__ double col[NBB];
  if (status_bad(st)) return;
  int t = threadIdx.x;
  for (int idx = t; idx < NBB * NBB; idx += blockDim.x) Ts[idx % NBB][idx / NBB] = 0.0;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    double ti = tau[i];
    if (t < i) {
      double s = 0.0;
      for (int u = t; u < i; ++u) s = fma(Ts[t][u], G[GEP_IX(u, i, nb)], s);
      col[t] = -ti * s;
    }
    __syncthreads();
    if (t < i) Ts[t][i] = col[t];
    if (t == 0) Ts[i][i] = ti;
    __syncthreads();
  }
  for (int idx = t; idx < nb * nb; idx += blockDim.x) T[idx] = Ts[idx % nb][idx / nb];
}

}  // namespace

size_t backtransform_ws_elems(int M, int ncol) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  return r((size_t)M * NBB) + r((size_t)NBB * NBB) * 2 + r((size_t)NBB * (ncol > 0 ? ncol : 1)) * 2;
}

int backtransform_q(gep_handle_t h, int M, int ncol, const double* C, int ldc, const double* tau,
                    double* Z, int ldz, double* ws, size_t ws_elems, int engine) {
  if (M <= 1 || ncol <= 0) return GEP_OK;
  if (ws_elems < backtransform_ws_elems(M, ncol)) return GEP_ERR_ALLOC;
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  double* V = ws;
  double* G = V + r((size_t)M * NBB);
  double* T = G + r((size_t)NBB * NBB);
  double* W1 = T + r((size_t)NBB * NBB);
  double* W2 = W1 + r((size_t)NBB * ncol);
  int nref = M - 1;  // reflectors exist for columns 0 .. M-2
  int last = ((nref - 1) / NBB) * NBB;
  for (int j0 = last; j0 >= 0; j0 -= NBB) {
    int nb = min(NBB, nref - j0);
    int rows = M - j0 - 1;
    dim3 g((rows + 255) / 256, nb);
    k_build_v<<<g, 256, 0, h->stream>>>(rows, nb, j0, C, ldc, V, h->d_status);
    GEP_CHECK(check_launch(h));
    GEP_CHECK(dgemm(h, 'T', 'N', 'F', nb, nb, rows, 1.0, V, rows, V, rows, 0.0, G, nb, engine));
    k_larft<<<1, NBB, 0, h->stream>>>(nb, G, tau + j0, T, h->d_status);
    GEP_CHECK(check_launch(h));
    double* Zs = Z + (j0 + 1);
    // transposed products keep the long dimension (ncol) as the row dimension of
    // each product, so all three fill full tensor-core tiles:
    //   W1^T = Z^T V,  W2^T = W1^T T^T,  Z -= V W2 = V (W2^T)^T
    GEP_CHECK(dgemm(h, 'T', 'N', 'F', ncol, nb, rows, 1.0, Zs, ldz, V, rows, 0.0, W1, ncol, engine));
    GEP_CHECK(dgemm(h, 'N', 'T', 'F', ncol, nb, nb, 1.0, W1, ncol, T, nb, 0.0, W2, ncol, engine));
    GEP_CHECK(dgemm(h, 'N', 'T', 'F', rows, ncol, nb, -1.0, V, rows, W2, ncol, 1.0, Zs, ldz, engine));
  }
  return GEP_OK;
}

}  // namespace gep
