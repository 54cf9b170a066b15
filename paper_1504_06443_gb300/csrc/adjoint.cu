// Reverse-mode derivative (adjoint) of the generalized eigenproblem A Y = B Y Lambda,
// Y^T B Y = I (Eq. 2), for losses built from eigenvalues and from the
// gauge-invariant occupied-subspace density matrix P = Y_o Y_o^T:
//     loss = sum_k lbar_k lambda_k + <W, P>.
// First-order perturbation of Eq. 2 (d lambda_k = y_k^T (dA - lambda_k dB) y_k, and the
// eigenvector perturbation with its B-normalisation term) gives, with What = Y^T W Y,
// o = occupied (first n_occ, ascending), v = virtual, F_kj = 1/(lambda_k - lambda_j):
//     Abar = Y G Y^T,  G_kk = lbar_k,  G_ov = G_vo^T = What_ov o F_ov, other entries 0
//     Bbar = Y H Y^T,  H_kk = -lbar_k lambda_k - [k in o] What_kk,
//                      H_oo(k != j) = -What_kj,  H_ov = H_vo^T = -diag(lambda_o) G_ov
// Only occupied/virtual gaps are divided by, so degenerate eigenvalues inside either
// block are harmless; the occupied/virtual gap must be nonzero.
#include "gep_internal.cuh"

namespace gep {
namespace {

__global__ void k_adj_build(int M, int no, const double* __restrict__ w, const double* __restrict__ lbar,
                            const double* __restrict__ Wh, int ldwh, double* __restrict__ G,
                            double* __restrict__ H, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < M; j += gridDim.y) {
    if (i >= M) continue;
    double g = 0.0, hv = 0.0;
    bool io = i < no, jo = j < no;
    if (i == j) {
      double lb = lbar ? lbar[i] : (io ? 1.0 : 0.0);
      g = lb;
      hv = -lb * w[i] - ((io && Wh) ? Wh[GEP_IX(i, i, ldwh)] : 0.0);
    } else if (io && jo) {
      hv = Wh ? -0.5 * (Wh[GEP_IX(i, j, ldwh)] + Wh[GEP_IX(j, i, ldwh)]) : 0.0;
    } else if (io && !jo) {
      g = Wh ? Wh[GEP_IX(i, j, ldwh)] / (w[i] - w[j]) : 0.0;
      hv = -w[i] * g;
    } else if (!io && jo) {
      g = Wh ? Wh[GEP_IX(j, i, ldwh)] / (w[j] - w[i]) : 0.0;
      hv = -w[j] * g;
    }
    G[GEP_IX(i, j, M)] = g;
    H[GEP_IX(i, j, M)] = hv;
  }
}

}  // namespace

size_t adjoint_ws_elems(int M, int no) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  return 3 * r((size_t)M * M) + r((size_t)(no > 0 ? no : 1) * M);
}

int adjoint(gep_handle_t h, int M, int no, const double* w, const double* Y, int ldy, const double* lbar,
            const double* W, int ldw, double* Abar, double* Bbar, int ldab, double* ws, int engine) {
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  double* X1 = ws;                         // (W + W^T) / 2, then G
  double* X2 = X1 + r((size_t)M * M);      // W Y then H
  double* X3 = X2 + r((size_t)M * M);      // G Y^T / H Y^T
  double* Wh = X3 + r((size_t)M * M);      // Y_o^T W Y  (no x M)
  const double* Whp = nullptr;
  if (W && no > 0) {
    // <W, P> with P symmetric only sees the symmetric part of W: both triangles are read
    GEP_CHECK(symmetric_part(h, M, W, ldw, X1, M));
    GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, X1, M, Y, ldy, 0.0, X2, M, engine));     // W Y
    GEP_CHECK(dgemm(h, 'T', 'N', 'F', no, M, M, 1.0, Y, ldy, X2, M, 0.0, Wh, no, engine));   // Y_o^T W Y
    Whp = Wh;
  }
  dim3 g((M + 255) / 256, M < 65535 ? M : 65535);
  k_adj_build<<<g, 256, 0, h->stream>>>(M, no, w, lbar, Whp, no > 0 ? no : 1, X1, X2, h->d_status);
  GEP_CHECK(check_launch(h));
  GEP_CHECK(dgemm(h, 'N', 'T', 'F', M, M, M, 1.0, X1, M, Y, ldy, 0.0, X3, M, engine));    // G Y^T
  GEP_CHECK(dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Y, ldy, X3, M, 0.0, Abar, ldab, engine));
  GEP_CHECK(dgemm(h, 'N', 'T', 'F', M, M, M, 1.0, X2, M, Y, ldy, 0.0, X3, M, engine));    // H Y^T
  return dgemm(h, 'N', 'N', 'F', M, M, M, 1.0, Y, ldy, X3, M, 0.0, Bbar, ldab, engine);
}

}  // namespace gep
