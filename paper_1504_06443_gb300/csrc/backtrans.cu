// SEP solver, stage "BACK" (Table 3): Z <- Q Z with Q = H_0 H_1 ... H_{M-off-1} left
// in C by the tridiagonalisation (off = 1: reflector j on rows j+1..M-1) or by the
// full-to-band reduction (off = b: reflector j on rows j+b..M-1).  Reflectors are
// grouped in panels of NBB and applied from the last panel to the first in compact-WY
// form,
//     H_j ... H_{j+nb-1} = I - V T V^T    (T upper triangular, forward/columnwise),
//     Z(j+1:, :) -= V (T (V^T Z(j+1:, :))),
// so all O(M^3) work is three matrix products per panel.  Panels are NBB = 1024
// reflectors wide (the update product then has depth 1024); their T factor is built
// recursively, T = [T1, -T1 (V1^T V2) T2; 0, T2], from 64-wide leaves.
#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int NBB = 1024;
constexpr int LB = 64;  // leaf order of the T-factor recursion

// Explicit V (rows j0+off .. M-1, nb columns): unit entry at local row q, reflector below.
__global__ void k_build_v(int rows, int nb, int j0, int off, const double* __restrict__ C, int ldc,
                          double* __restrict__ V, const int* st) {
  if (status_bad(st)) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int q = blockIdx.y;
  if (t >= rows || q >= nb) return;
  double val;
  if (t < q) val = 0.0;
  else if (t == q) val = 1.0;
  else val = C[GEP_IX(j0 + off + t, j0 + q, ldc)];
  V[GEP_IX(t, q, rows)] = val;
}

// T factor from G = V^T V:  T(i,i) = tau_i,  T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i).
// (leaf, nb <= LB; G and T with leading dimensions ldg, ldt)
__global__ void k_larft(int nb, const double* __restrict__ G, int ldg, const double* __restrict__ tau,
                        double* __restrict__ T, int ldt, const int* st) {
  __shared__ double Ts[LB][LB + 1];
  __shared__ double col[LB];
  if (status_bad(st)) return;
  int t = threadIdx.x;
  for (int idx = t; idx < LB * LB; idx += blockDim.x) Ts[idx % LB][idx / LB] = 0.0;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    double ti = tau[i];
    if (t < i) {
      double s = 0.0;
      for (int u = t; u < i; ++u) s = fma(Ts[t][u], G[GEP_IX(u, i, ldg)], s);
      col[t] = -ti * s;
    }
    __syncthreads();
    if (t < i) Ts[t][i] = col[t];
    if (t == 0) Ts[i][i] = ti;
    __syncthreads();
  }
  for (int idx = t; idx < nb * nb; idx += blockDim.x) T[GEP_IX(idx % nb, idx / nb, ldt)] = Ts[idx % nb][idx / nb];
}

}  // namespace

// T (nb x nb, upper) of the block reflector whose Gram matrix is G = V^T V.
int larft_rec(gep_handle_t h, int nb, const double* G, int ldg, const double* tau, double* T, int ldt,
              double* tmp) {
  if (nb <= LB) {
    k_larft<<<1, LB, 0, h->stream>>>(nb, G, ldg, tau, T, ldt, h->d_status);
    return check_launch(h);
  }
  int n1 = ((nb / 2 + LB - 1) / LB) * LB, n2 = nb - n1;
  GEP_CHECK(larft_rec(h, n1, G, ldg, tau, T, ldt, tmp));
  GEP_CHECK(larft_rec(h, n2, G + GEP_IX(n1, n1, ldg), ldg, tau + n1, T + GEP_IX(n1, n1, ldt), ldt, tmp));
  GEP_CHECK(set_matrix(h, n2, n1, 0.0, 0.0, T + n1, ldt));  // strictly lower block
  // T12 = -T1 (G12 T2)
  GEP_CHECK(dgemm_f64(h, 'N', 'N', 'F', n1, n2, n2, 1.0, G + GEP_IX(0, n1, ldg), ldg, T + GEP_IX(n1, n1, ldt), ldt,
                      0.0, tmp, n1));
  return dgemm_f64(h, 'N', 'N', 'F', n1, n2, n1, -1.0, T, ldt, tmp, n1, 0.0, T + GEP_IX(0, n1, ldt), ldt);
}

size_t backtransform_ws_elems(int M, int ncol) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  return r((size_t)M * NBB) + r((size_t)NBB * NBB) * 3 + r((size_t)NBB * (ncol > 0 ? ncol : 1)) * 2;
}

int backtransform_q(gep_handle_t h, int M, int ncol, const double* C, int ldc, const double* tau,
                    double* Z, int ldz, double* ws, size_t ws_elems, int engine, int off) {
  if (M <= off || ncol <= 0) return GEP_OK;
  if (ws_elems < backtransform_ws_elems(M, ncol)) return GEP_ERR_ALLOC;
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  double* V = ws;
  double* G = V + r((size_t)M * NBB);
  double* T = G + r((size_t)NBB * NBB);
  double* Tt = T + r((size_t)NBB * NBB);  // recursion scratch
  double* W1 = Tt + r((size_t)NBB * NBB);
  double* W2 = W1 + r((size_t)NBB * ncol);
  int nref = M - off;  // reflectors exist for columns 0 .. M-off-1 (reflector j on rows j+off ..)
  int last = ((nref - 1) / NBB) * NBB;
  for (int j0 = last; j0 >= 0; j0 -= NBB) {
    int nb = min(NBB, nref - j0);
    int rows = M - j0 - off;
    dim3 g((rows + 255) / 256, nb);
    k_build_v<<<g, 256, 0, h->stream>>>(rows, nb, j0, off, C, ldc, V, h->d_status);
    GEP_CHECK(check_launch(h));
    GEP_CHECK(dgemm(h, 'T', 'N', 'F', nb, nb, rows, 1.0, V, rows, V, rows, 0.0, G, nb, engine));
    GEP_CHECK(larft_rec(h, nb, G, nb, tau + j0, T, nb, Tt));
    double* Zs = Z + (j0 + off);
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
