// SEP solver, stage "TRD" (Table 3): one-stage Householder reduction of the
// symmetric C to tridiagonal form, C = Q T Q^T, Q = H_0 H_1 ... H_{M-2}.
//
// Blocked in panels of NBT columns (the conventional algorithm of the
// ScaLAPACK/ELPA1/EigenExa "eigen_s" solvers of section 3.1).  Inside a panel,
// column c needs one symmetric matrix-vector product with the trailing matrix
// as it stood before the panel, corrected by the panel's earlier reflectors
// (V) and their companions (W):  A_cur v = A v - V (W^T v) - W (V^T v).  After
// the panel, the trailing matrix takes the rank-2*NBT update A -= V W^T + W V^T
// on the GEMM engine.  Half of the flops are in the memory-bound SYMVs.
//
// The SYMV reads only the lower triangle (each 64-wide column strip once) and
// is deterministic: every strip writes its partial sums to its own slots, and a
// second kernel adds them in a fixed order.
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int NBT = 64;     // panel width
constexpr int SW = 64;      // SYMV strip width
constexpr int SCH = 1024;   // SYMV rows per CTA
constexpr int DCH = 128;    // panel dot-product rows per CTA

struct TWs {
  double *Vp, *W, *y, *Pd, *Pt, *part, *part2, *WV, *tq;
  float2* S2;  // float-pair copy of the trailing matrix (lower triangle) for the SYMVs
  int M, nblk, maxch, ndch;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  red must hold 32 doubles.
__device__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) s = warp_sum(s);
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// Householder reflector of x = C(c+1:M, c):  H x = beta e_1, H = I - tau v v^T, v(0) = 1.
// Writes d[c], e[c], tau[c], the reflector into C below the subdiagonal, and the
// explicit column i of the panel V (zeros above row c+1).
__global__ void __launch_bounds__(1024) k_householder(int M, int c, int i, double* C, int ldc, double* d,
                                                      double* e, double* tau, double* Vp, int ldp,
                                                      const int* st) {
  __shared__ double red[32];
  if (status_bad(st)) return;
  int n = M - c - 1;
  double* x = C + GEP_IX(c + 1, c, ldc);
  double s = 0.0;
  for (int t = 1 + threadIdx.x; t < n; t += blockDim.x) s = fma(x[t], x[t], s);
  double sig = block_sum(s, red);
  double alpha = x[0];
  double beta, tv, scal;
  if (sig == 0.0) {
    tv = 0.0; beta = alpha; scal = 0.0;
  } else {
    double nrm = sqrt(alpha * alpha + sig);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tv = (beta - alpha) / beta;
    scal = 1.0 / (alpha - beta);
  }
  double* v = Vp + (size_t)i * ldp;
  for (int r = threadIdx.x; r <= c; r += blockDim.x) v[r] = 0.0;
  for (int t = 1 + threadIdx.x; t < n; t += blockDim.x) {
    double vt = (sig == 0.0) ? 0.0 : x[t] * scal;
    x[t] = vt;
    v[c + 1 + t] = vt;
  }
  if (threadIdx.x == 0) {
    d[c] = C[GEP_IX(c, c, ldc)];
    e[c] = beta;
    tau[c] = tv;
    x[0] = beta;
    v[c + 1] = 1.0;
  }
}

__global__ void k_last_diag(int M, const double* C, int ldc, double* d, const int* st) {
  if (status_bad(st)) return;
  d[M - 1] = C[GEP_IX(M - 1, M - 1, ldc)];
}

// ---- compensated single-precision arithmetic for the SYMV ----------------------
// The SYMV needs two multiply-adds per matrix element; at this part's FP64 rate that
// is ~3x slower than streaming the element from HBM.  The trailing matrix is kept
// as an unevaluated float pair (hi, lo) with hi + lo = a to ~2^-48 relative, the
// vector is split the same way, and every term is formed as an exact product
// (FMA error term) plus the two cross terms, summed with TwoSum, so each partial
// sum carries ~46 significant bits and the kernel stays bound by memory.
struct ff {
  float h, l;
};

// x = h + l with h = x rounded to 24 significant bits and l = x - h (|l| <= 2^-25 |x|,
// itself rounded to float), built from the IEEE bits with integer instructions (on
// this part the float<->double conversions run on the slow FP64 pipe).  Values whose
// exponent is outside a comfortable float range take the conversion path.
__device__ __forceinline__ ff ff_split(double x) {
  long long b = __double_as_longlong(x);
  int E = (int)((b >> 52) & 0x7FF);
  if (E < 1023 - 70 || E > 1023 + 120) {
    if (E == 0) return {0.f, 0.f};
    float h = (float)x;
    return {h, (float)(x - (double)h)};
  }
  unsigned sign = (unsigned)((unsigned long long)b >> 63);
  long long m53 = (long long)(((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  long long m24 = (m53 + (1ll << 28)) >> 29;       // rounded 24-bit significand (may carry to 2^24)
  long long lo_int = m53 - (m24 << 29);            // |lo_int| <= 2^28, exact
  unsigned hb;
  if (m24 >> 24) hb = (sign << 31) | ((unsigned)(E - 1023 + 128) << 23);  // rounded up to 2^(E-1022)
  else hb = (sign << 31) | ((unsigned)(E - 1023 + 127) << 23) | ((unsigned)m24 & 0x7FFFFFu);
  float scale = __int_as_float((E - 1075 + 127) << 23);  // 2^(E-1075), a normal float here
  float l = __ll2float_rn(lo_int) * scale;
  return {__int_as_float((int)hb), sign ? -l : l};
}

// s += x with both parts TwoSum'ed and the pair renormalised (accurate double-float
// addition, relative error ~3 * 2^-48 per step): used where hundreds of partial sums
// of one row are added, so the error does not grow with their number.
__device__ __forceinline__ void ff_add_acc(ff& s, ff x) {
  float hs = s.h + x.h;
  float z = hs - s.h;
  float eh = (s.h - (hs - z)) + (x.h - z);
  float ls = s.l + x.l;
  float z2 = ls - s.l;
  float el = (s.l - (ls - z2)) + (x.l - z2);
  eh += ls;
  float h2 = hs + eh;
  eh = eh - (h2 - hs);
  eh += el;
  s.h = h2 + eh;
  s.l = eh - (s.h - h2);
}

__device__ __forceinline__ ff ff_warp_sum(ff v) {
  for (int o = 16; o; o >>= 1) {
    ff u = {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    ff_add_acc(v, u);
  }
  return v;
}

// s += a * v (a, v float pairs), TwoSum on the leading parts.
__device__ __forceinline__ void ff_madd(ff& s, float ah, float al, float vh, float vl) {
  float p = ah * vh;
  float e = fmaf(ah, vh, -p);
  e = fmaf(ah, vl, e);
  e = fmaf(al, vh, e);
  float t = s.h + p;
  float z = t - s.h;
  float err = (s.h - (t - z)) + (p - z);
  s.h = t;
  s.l += err + e;
}

// Matrix element types of the single-precision SYMV: a float pair (FP64-grade path)
// or a single float (the FP32-grade mixed-precision path, half the traffic).
__device__ __forceinline__ float2 as_pair(float2 a) { return a; }
__device__ __forceinline__ float2 as_pair(float a) { return make_float2(a, 0.f); }
__device__ __forceinline__ void put(float2* p, ff x) { *p = make_float2(x.h, x.l); }
__device__ __forceinline__ void put(float* p, ff x) { *p = x.h; }

// Lower triangle of the n x n block at A (FP64) -> float pairs / floats at S (same indexing).
template <class T>
__global__ void k_to_ff(int n, const double* __restrict__ A, int lda, T* __restrict__ S, int lds, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = blockIdx.y; j < n; j += gridDim.y) {
    if (i < n && i >= j) put(&S[GEP_IX(i, j, lds)], ff_split(A[GEP_IX(i, j, lda)]));
  }
}

// Same partial-product scheme as k_symv_partial below, on the single-precision matrix.
template <class T>
__global__ void __launch_bounds__(256) k_symv_partial_ff(int n, const T* __restrict__ A, int lda,
                                                         const double* __restrict__ v, double* __restrict__ Pd,
                                                         double* __restrict__ Pt, int maxch, const int* st) {
  __shared__ float vsh[SW], vsl[SW];
  __shared__ float2 dsum[4][SCH];
  __shared__ float2 tsum[4][2][16];
  if (status_bad(st)) return;
  int jb = blockIdx.x, ch = blockIdx.y;
  int c0 = jb * SW;
  int R0 = c0 + ch * SCH;
  if (R0 >= n) return;
  int rl = threadIdx.x & 63, cq = threadIdx.x >> 6;
  if (threadIdx.x < SW) {
    ff t = ff_split((c0 + threadIdx.x < n) ? v[c0 + threadIdx.x] : 0.0);
    vsh[threadIdx.x] = t.h;
    vsl[threadIdx.x] = t.l;
  }
  __syncthreads();
  int cbase = c0 + cq * 16;
  int ncols = min(16, n - cbase);
  ff acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = {0.f, 0.f};
  int rend = min(n, R0 + SCH);
  for (int p = 0; p < SCH / 64; ++p) {
    int r = R0 + p * 64 + rl;
    ff dir = {0.f, 0.f};
    if (r < rend && ncols > 0) {
      ff vr = ff_split(v[r]);
      const T* arow = A + r;
      if (r >= cbase + 16 && ncols == 16) {
        // full quarter strictly below the diagonal: issue all 16 loads, then compute
        float2 a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = as_pair(__ldg(arow + (size_t)(cbase + q) * lda));
        ff dir2 = {0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          ff_madd(dir, a[q].x, a[q].y, vsh[cq * 16 + q], vsl[cq * 16 + q]);
          ff_madd(dir2, a[q + 1].x, a[q + 1].y, vsh[cq * 16 + q + 1], vsl[cq * 16 + q + 1]);
          ff_madd(acc[q], a[q].x, a[q].y, vr.h, vr.l);
          ff_madd(acc[q + 1], a[q + 1].x, a[q + 1].y, vr.h, vr.l);
        }
        ff_madd(dir, dir2.h, 0.f, 1.f, 0.f);
        dir.l += dir2.l;
      } else if (r >= cbase + 16) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q < ncols) {
            float2 a = as_pair(arow[(size_t)(cbase + q) * lda]);
            ff_madd(dir, a.x, a.y, vsh[cq * 16 + q], vsl[cq * 16 + q]);
            ff_madd(acc[q], a.x, a.y, vr.h, vr.l);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          int col = cbase + q;
          if (q < ncols && r >= col) {
            float2 a = as_pair(arow[(size_t)col * lda]);
            ff_madd(dir, a.x, a.y, vsh[cq * 16 + q], vsl[cq * 16 + q]);
            if (r > col) ff_madd(acc[q], a.x, a.y, vr.h, vr.l);
          }
        }
      }
    }
    dsum[cq][p * 64 + rl] = make_float2(dir.h, dir.l);
  }
  int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 1;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    ff s = ff_warp_sum(acc[q]);
    if (lane == 0) tsum[cq][wq][q] = make_float2(s.h, s.l);
  }
  __syncthreads();
  // partials stay float pairs; k_w_compute adds them up and converts once per row
  float2* Pd2 = reinterpret_cast<float2*>(Pd);
  float2* Pt2 = reinterpret_cast<float2*>(Pt);
  for (int t = threadIdx.x; t < SCH; t += blockDim.x) {
    int r = R0 + t;
    if (r < rend) {
      ff s = {dsum[0][t].x, dsum[0][t].y};
      ff_add_acc(s, {dsum[1][t].x, dsum[1][t].y});
      ff_add_acc(s, {dsum[2][t].x, dsum[2][t].y});
      ff_add_acc(s, {dsum[3][t].x, dsum[3][t].y});
      Pd2[(size_t)jb * n + r] = make_float2(s.h, s.l);
    }
  }
  if (threadIdx.x < SW) {
    int q4 = threadIdx.x >> 4, q = threadIdx.x & 15;
    ff s = {tsum[q4][0][q].x, tsum[q4][0][q].y};
    ff_add_acc(s, {tsum[q4][1][q].x, tsum[q4][1][q].y});
    Pt2[((size_t)jb * maxch + ch) * SW + threadIdx.x] = make_float2(s.h, s.l);
  }
}

// Partial products of the symmetric SYMV y = A v over strip jb (columns 64 jb ..),
// rows [R0, R0 + SCH) of the lower triangle.  256 threads = 64 row lanes x 4 column
// quarters of 16 columns.  Direct terms A(r,c) v(c) (r >= c) go to Pd[jb][r];
// transposed terms A(r,c) v(r) (r > c) are summed per column into Pt[jb][ch][.].
__global__ void __launch_bounds__(256) k_symv_partial(int n, const double* __restrict__ A, int lda,
                                                      const double* __restrict__ v, double* __restrict__ Pd,
                                                      double* __restrict__ Pt, int maxch, const int* st) {
  __shared__ double vs[SW];
  __shared__ double dsum[4][SCH];
  __shared__ double tsum[4][2][16];
  if (status_bad(st)) return;
  int jb = blockIdx.x, ch = blockIdx.y;
  int c0 = jb * SW;
  int R0 = c0 + ch * SCH;
  if (R0 >= n) return;
  int rl = threadIdx.x & 63, cq = threadIdx.x >> 6;
  if (threadIdx.x < SW) vs[threadIdx.x] = (c0 + threadIdx.x < n) ? v[c0 + threadIdx.x] : 0.0;
  __syncthreads();
  int cbase = c0 + cq * 16;
  int ncols = min(16, n - cbase);  // may be <= 0 at the ragged end
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  int rend = min(n, R0 + SCH);
  for (int p = 0; p < SCH / 64; ++p) {
    int r = R0 + p * 64 + rl;
    double dir = 0.0;
    if (r < rend && ncols > 0) {
      double vr = v[r];
      const double* arow = A + r;
      if (r >= cbase + 16 && ncols == 16) {  // full quarter below the diagonal: loads first
        double a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = __ldg(arow + (size_t)(cbase + q) * lda);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          dir = fma(a[q], vs[cq * 16 + q], dir);
          acc[q] = fma(a[q], vr, acc[q]);
        }
      } else if (r >= cbase + 16) {  // strictly below every column of this quarter
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q < ncols) {
            double a = arow[(size_t)(cbase + q) * lda];
            dir = fma(a, vs[cq * 16 + q], dir);
            acc[q] = fma(a, vr, acc[q]);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          int col = cbase + q;
          if (q < ncols && r >= col) {
            double a = arow[(size_t)col * lda];
            dir = fma(a, vs[cq * 16 + q], dir);
            if (r > col) acc[q] = fma(a, vr, acc[q]);
          }
        }
      }
    }
    dsum[cq][p * 64 + rl] = dir;
  }
  // transposed terms: reduce over the 64 row lanes (2 warps per quarter)
  int lane = threadIdx.x & 31, wq = (threadIdx.x >> 5) & 1;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    double s = warp_sum(acc[q]);
    if (lane == 0) tsum[cq][wq][q] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SCH; t += blockDim.x) {
    int r = R0 + t;
    if (r < rend) Pd[(size_t)jb * n + r] = (dsum[0][t] + dsum[1][t]) + (dsum[2][t] + dsum[3][t]);
  }
  if (threadIdx.x < SW) {
    int q4 = threadIdx.x >> 4, q = threadIdx.x & 15;
    Pt[((size_t)jb * maxch + ch) * SW + threadIdx.x] = tsum[q4][0][q] + tsum[q4][1][q];
  }
}

// Partial dots over rows [ch*DCH, ...) of t1 = W(:,0:i)^T v and t2 = V(:,0:i)^T v
// (rows c+1 .. M-1 of the panel).  One warp per (matrix, column).
__global__ void __launch_bounds__(256) k_panel_dots(int n, int i, const double* __restrict__ Vp,
                                                    const double* __restrict__ W, int ldp,
                                                    const double* __restrict__ v, double* __restrict__ part,
                                                    const int* st) {
  if (status_bad(st)) return;
  int ch = blockIdx.x;
  int r0 = ch * DCH, r1 = min(n, r0 + DCH);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < 2 * i; q += 8) {
    const double* col = (q < i) ? (W + (size_t)q * ldp) : (Vp + (size_t)(q - i) * ldp);
    double s = 0.0;
    for (int r = r0 + lane; r < r1; r += 32) s = fma(col[r], v[r], s);
    s = warp_sum(s);
    if (lane == 0) part[(size_t)ch * 2 * NBT + q] = s;
  }
}

// t[q] = sum over chunks of the panel dot partials (one CTA per q, fixed order).
__global__ void __launch_bounds__(256) k_dots_reduce(int nch, const double* __restrict__ part,
                                                     double* __restrict__ tq, const int* st) {
  __shared__ double red[32];
  if (status_bad(st)) return;
  int q = blockIdx.x;
  double s = 0.0;
  for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) s += part[(size_t)ch * 2 * NBT + q];
  s = block_sum(s, red);
  if (threadIdx.x == 0) tq[q] = s;
}

// y = A v from the SYMV partials (same fixed order as k_symv_reduce), then
// w = tau (y - V t1 - W t2) on rows [blk*256, ...); also writes partial w.v.
__global__ void __launch_bounds__(256) k_w_compute(int n, int i, const double* __restrict__ Vp,
                                                   const double* __restrict__ W, int ldp,
                                                   const double* __restrict__ v, const double* __restrict__ Pd,
                                                   const double* __restrict__ Pt, int maxch, int pairs,
                                                   double* __restrict__ y, const double* __restrict__ tq,
                                                   const double* tau_c, double* __restrict__ part2, const int* st) {
  __shared__ double t[2 * NBT];
  __shared__ double red[32];
  if (status_bad(st)) return;
  if (threadIdx.x < 2 * i) t[threadIdx.x] = tq[threadIdx.x];
  __syncthreads();
  double tv = *tau_c;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  double dotp = 0.0;
  if (r < n) {
    int jr = r / SW;
    int nch = (n - jr * SW + SCH - 1) / SCH;
    double s;
    if (pairs) {  // float-pair partials from k_symv_partial_ff
      const float2* Pd2 = reinterpret_cast<const float2*>(Pd);
      const float2* Pt2 = reinterpret_cast<const float2*>(Pt);
      ff sd = {0.f, 0.f}, stt = {0.f, 0.f};
      for (int jb = 0; jb <= jr; ++jb) {
        float2 p = Pd2[(size_t)jb * n + r];
        ff_add_acc(sd, {p.x, p.y});
      }
      for (int ch = 0; ch < nch; ++ch) {
        float2 p = Pt2[((size_t)jr * maxch + ch) * SW + (r - jr * SW)];
        ff_add_acc(stt, {p.x, p.y});
      }
      ff_add_acc(sd, stt);
      s = (double)sd.h + (double)sd.l;
    } else {
      double sd = 0.0;
      for (int jb = 0; jb <= jr; ++jb) sd += Pd[(size_t)jb * n + r];
      double stt = 0.0;
      for (int ch = 0; ch < nch; ++ch) stt += Pt[((size_t)jr * maxch + ch) * SW + (r - jr * SW)];
      s = sd + stt;
    }
    for (int q = 0; q < i; ++q) s -= Vp[GEP_IX(r, q, ldp)] * t[q] + W[GEP_IX(r, q, ldp)] * t[i + q];
    double w = tv * s;
    y[r] = w;
    dotp = w * v[r];
  }
  double tot = block_sum(dotp, red);
  if (threadIdx.x == 0) part2[blockIdx.x] = tot;
}

// alpha = -tau/2 (w.v);  W(:, i) = w + alpha v  (rows c+1 ..).  With `next`, the same
// kernel also applies the panel update to column c+1 (rows c+1 ..), which needs the
// new W(:, i): every CTA recomputes W(c+1, i) from y(0), v(0) and alpha.
__global__ void __launch_bounds__(256) k_w_finish(int n, int nblk, const double* __restrict__ y,
                                                  const double* __restrict__ v, const double* __restrict__ part2,
                                                  const double* tau_c, int c, int i, int next, double* C, int ldc,
                                                  const double* __restrict__ Vp, double* __restrict__ W, int ldp,
                                                  const int* st) {
  __shared__ double red[32];
  __shared__ double vc[NBT], wc[NBT];
  if (status_bad(st)) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part2[b];
  double dot = block_sum(s, red);
  double alpha = -0.5 * (*tau_c) * dot;
  if (next && threadIdx.x <= i) {
    int q = threadIdx.x;
    vc[q] = Vp[GEP_IX(c + 1, q, ldp)];
    wc[q] = (q < i) ? W[GEP_IX(c + 1, q, ldp)] : fma(alpha, v[0], y[0]);
  }
  __syncthreads();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double wnew = fma(alpha, v[r], y[r]);
  W[GEP_IX(c + 1 + r, i, ldp)] = wnew;
  if (next) {
    int R = c + 1 + r;
    double sum = 0.0;
    for (int q = 0; q < i; ++q)
      sum = fma(Vp[GEP_IX(R, q, ldp)], wc[q], fma(W[GEP_IX(R, q, ldp)], vc[q], sum));
    sum = fma(Vp[GEP_IX(R, i, ldp)], wc[i], fma(wnew, vc[i], sum));
    C[GEP_IX(R, c + 1, ldc)] -= sum;
  }
}

TWs carve(double* ws, int M) {
  TWs t;
  t.M = M;
  t.nblk = (M + SW - 1) / SW;
  t.maxch = (M + SCH - 1) / SCH;
  t.ndch = (M + DCH - 1) / DCH;
  size_t o = 0;
  auto take = [&](size_t n) { double* p = ws + o; o += (n + 31) & ~(size_t)31; return p; };
  t.Vp = take((size_t)M * NBT);
  t.W = take((size_t)M * NBT);
  t.y = take((size_t)M);
  t.Pd = take((size_t)t.nblk * M);
  t.Pt = take((size_t)t.nblk * t.maxch * SW);
  t.part = take((size_t)t.ndch * 2 * NBT);
  t.part2 = take((size_t)(M + 255) / 256 + 1);
  t.WV = take((size_t)M * 2 * NBT);
  t.S2 = (float2*)take((size_t)M * M);
  t.tq = take((size_t)2 * NBT);
  return t;
}

}  // namespace

size_t tridiag_ws_elems(int M) {
  size_t nblk = (M + SW - 1) / SW, maxch = (M + SCH - 1) / SCH, ndch = (M + DCH - 1) / DCH;
  auto r = [](size_t n) { return (n + 31) & ~(size_t)31; };
  return r((size_t)M * NBT) * 2 + r(M) + r(nblk * M) + r(nblk * maxch * SW) + r(ndch * 2 * NBT) +
         r((M + 255) / 256 + 1) + r((size_t)M * 2 * NBT) + r((size_t)M * M) + r(2 * NBT);
}

int tridiag_1stage(gep_handle_t h, int M, double* C, int ldc, double* d, double* e, double* tau,
                   double* ws, size_t ws_elems, int engine) {
  if (M <= 0) return GEP_OK;
  if (ws_elems < tridiag_ws_elems(M)) return GEP_ERR_ALLOC;
  TWs t = carve(ws, M);
  const int ldp = M;
  cudaStream_t s = h->stream;
  const int* st = h->d_status;
  // FP64 engine: plain FP64 SYMVs.  Tensor-core engines: compensated float-pair SYMVs.
  const bool pairs = engine != GEP_PREC_FP64;
  // FP32-grade engine: the SYMV matrix is a single float per element (half the traffic).
  const bool single = engine == GEP_PREC_MIXED_REFINED;
  float* S1 = reinterpret_cast<float*>(t.S2);
  for (int j0 = 0; j0 < M; j0 += NBT) {
    int nbp = min(NBT, M - j0);
    int done = 0;
    if (pairs && M - j0 > 1) {
      int nt = M - j0;
      dim3 g((nt + 255) / 256, nt < 65535 ? nt : 65535);
      if (single)
        k_to_ff<float><<<g, 256, 0, s>>>(nt, C + GEP_IX(j0, j0, ldc), ldc, S1 + GEP_IX(j0, j0, M), M, st);
      else
        k_to_ff<float2><<<g, 256, 0, s>>>(nt, C + GEP_IX(j0, j0, ldc), ldc, t.S2 + GEP_IX(j0, j0, M), M, st);
      GEP_CHECK(check_launch(h));
    }
    for (int i = 0; i < nbp; ++i) {
      int c = j0 + i;
      // (columns i > 0 of the panel were already updated by the previous column's k_w_finish)
      if (c == M - 1) {
        k_last_diag<<<1, 1, 0, s>>>(M, C, ldc, d, st);
        GEP_CHECK(check_launch(h));
        done = 1;
        break;
      }
      k_householder<<<1, 1024, 0, s>>>(M, c, i, C, ldc, d, e, tau, t.Vp, ldp, st);
      GEP_CHECK(check_launch(h));
      int n = M - c - 1;
      const double* v = t.Vp + GEP_IX(c + 1, i, ldp);
      const double* A = C + GEP_IX(c + 1, c + 1, ldc);
      int nblk = (n + SW - 1) / SW, maxch = (n + SCH - 1) / SCH;
      if (pairs && single)
        k_symv_partial_ff<float><<<dim3(nblk, maxch), 256, 0, s>>>(n, S1 + GEP_IX(c + 1, c + 1, M), M, v, t.Pd,
                                                                   t.Pt, maxch, st);
      else if (pairs)
        k_symv_partial_ff<float2><<<dim3(nblk, maxch), 256, 0, s>>>(n, t.S2 + GEP_IX(c + 1, c + 1, M), M, v, t.Pd,
                                                                    t.Pt, maxch, st);
      else
        k_symv_partial<<<dim3(nblk, maxch), 256, 0, s>>>(n, A, ldc, v, t.Pd, t.Pt, maxch, st);
      GEP_CHECK(check_launch(h));
      int ndch = (n + DCH - 1) / DCH;
      if (i > 0) {
        k_panel_dots<<<ndch, 256, 0, s>>>(n, i, t.Vp + (c + 1), t.W + (c + 1), ldp, v, t.part, st);
        GEP_CHECK(check_launch(h));
        k_dots_reduce<<<2 * i, 256, 0, s>>>(ndch, t.part, t.tq, st);
        GEP_CHECK(check_launch(h));
      }
      int nb256 = (n + 255) / 256;
      k_w_compute<<<nb256, 256, 0, s>>>(n, i, t.Vp + (c + 1), t.W + (c + 1), ldp, v, t.Pd, t.Pt, maxch,
                                        pairs ? 1 : 0, t.y, t.tq, tau + c, t.part2, st);
      GEP_CHECK(check_launch(h));
      int next = (i + 1 < nbp) ? 1 : 0;
      k_w_finish<<<nb256, 256, 0, s>>>(n, nb256, t.y, v, t.part2, tau + c, c, i, next, C, ldc, t.Vp, t.W, ldp,
                                       st);
      GEP_CHECK(check_launch(h));
    }
    if (done) break;
    int jn = j0 + nbp;
    int n2 = M - jn;
    if (n2 > 0) {
      // A(jn:, jn:) -= V W^T + W V^T on the lower triangle
      if (nbp == NBT) {
        // one product of depth 2*NBT: [V W] [W V]^T (V and W are adjacent in the workspace)
        GEP_CHECK(copy_matrix(h, n2, NBT, t.W + jn, ldp, t.WV + jn, ldp));
        GEP_CHECK(copy_matrix(h, n2, NBT, t.Vp + jn, ldp, t.WV + jn + (size_t)NBT * ldp, ldp));
        GEP_CHECK(dgemm(h, 'N', 'T', 'L', n2, n2, 2 * NBT, -1.0, t.Vp + jn, ldp, t.WV + jn, ldp, 1.0,
                        C + GEP_IX(jn, jn, ldc), ldc, engine));
      } else {
        GEP_CHECK(dgemm(h, 'N', 'T', 'L', n2, n2, nbp, -1.0, t.Vp + jn, ldp, t.W + jn, ldp, 1.0,
                        C + GEP_IX(jn, jn, ldc), ldc, engine));
        GEP_CHECK(dgemm(h, 'N', 'T', 'L', n2, n2, nbp, -1.0, t.W + jn, ldp, t.Vp + jn, ldp, 1.0,
                        C + GEP_IX(jn, jn, ldc), ldc, engine));
      }
    }
  }
  return GEP_OK;
}

}  // namespace gep
