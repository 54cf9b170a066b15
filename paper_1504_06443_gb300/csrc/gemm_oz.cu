// FP64-accurate matrix product on the BF16 tensor cores (split-BF16 / Ozaki-style).
#include "gep_internal.cuh"

namespace gep {

size_t oz_workspace_bytes(int m, int n, int k) { (void)m; (void)n; (void)k; return 0; }

int dgemm_oz(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha,
             const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
             int levels) {
  (void)h; (void)ta; (void)tb; (void)uplo; (void)m; (void)n; (void)k; (void)alpha; (void)A; (void)lda;
  (void)B; (void)ldb; (void)beta; (void)C; (void)ldc; (void)levels;
  return GEP_ERR_UNSUPPORTED;
}

}  // namespace gep
