// SEP solver, two-stage path: the narrow-band reduction SEP solvers of section 3
// (ELPA2 / Eigen_sx), stages "TRD/BAND" and "BACK" of Table 3.
//
// S1b full -> band.  C = Q1 C_b Q1^T with C_b of bandwidth b.  For each panel of b
// columns the n x b block below the band is QR-factorised with Householder
// reflectors (Q_p = I - V T V^T), R stays in the band and the trailing matrix takes
// the two-sided update
//     X = C22 V T,  W = X - V (T^T V^T X) / 2,  C22 <- C22 - W V^T - V W^T,
// i.e. all O(M^3) work is matrix products (split-BF16 tensor-core engine).  Only the
// lower triangle of C22 is stored and updated; C22 V reads it as a symmetric operand.
//
// S1c band -> tridiagonal (bulge chasing).  Sweep s annihilates column s below the
// subdiagonal with a reflector H(s,0) on rows s+1..s+b, then chases the bulge that
// the right-application creates one b x b block further down per step:
//     step k: B = C(st_k:, st_{k-1}:) <- B H(s,k-1);  H(s,k) annihilates B(1:, 0);
//             B <- H(s,k) B;  D = C(st_k:, st_k:) <- H(s,k) D H(s,k),
// st_k = s + 1 + k b.  Step k of sweep s+1 only needs step k+1 of sweep s to be done,
// so sweeps run concurrently on different CTAs, each one step-pipelined behind the
// previous sweep (progress counters with acquire/release, bounded waits).
//
// Back-transformation.  Z = Q1 (Q2 Z_T), Q2 = prod_s prod_k H(s,k).  The reflectors
// H(s,k) of the b sweeps s0..s0+b-1 of group j (s0 = j b) at the same step k occupy a
// (2b-1)-row "diamond" G(j,k) = H(s0,k) ... H(s0+b-1,k), and
//     Q2 = prod_{j ascending} prod_{k descending} G(j,k),
// because H(s,k) commutes with every H(s',k') (s' < s, k' < k) it has to pass.  The
// diamonds are applied in wavefronts t = (J - j) + k: diamonds of one wavefront touch
// disjoint rows and every diamond that must precede one of them lies in an earlier
// wavefront.  Q1 is applied with the compact-WY back-transformation of the 1-stage
// path, its reflectors starting b rows (instead of one) below their column.
#include <math.h>

#include <algorithm>
#include <vector>

#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int BMAX = 64;      // largest bandwidth
constexpr int BULGE_CTAS_PER_SM = 1;  // resident bulge-chasing CTAs per SM
constexpr int BAND_GROUP = 4;  // panels per group of the full -> band reduction (trailing update depth 2 G b)
constexpr int BAND_GROUP_MIN_N = 8192;  // trailing order from which groups of BAND_GROUP are used
constexpr int PQ_ROWS = 256;  // panel rows per CTA in the panel QR (one per thread)
constexpr int PQ_CH = 16;     // columns per reduction chunk in the panel QR

size_t rr(size_t n) { return (n + 31) & ~(size_t)31; }

// ------------------------------------------------------------------ S1b panel QR

// One Householder step (column c) of the QR factorisation of the n x nb panel P (ld ldp),
// fused with the partial dot products the next step needs.  part_in[j][g] (g over the
// CTAs) = sum over rows r > c of P(r,c) P(r,j), prow_in[j] = P(c,j): the pivot row is
// kept out of the sums so that the norm of the tail is never formed by cancellation.
// c = -1 only produces part/prow for column 0.  The reflector follows LAPACK's dlarfg:
// beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta, v = [1; x(1:) / (alpha - beta)].
__global__ void __launch_bounds__(PQ_ROWS) k_pqr_step(int n, int nb, int c, double* __restrict__ P, int ldp,
                                                      const double* __restrict__ part_in,
                                                      const double* __restrict__ prow_in,
                                                      double* __restrict__ part_out, double* __restrict__ prow_out,
                                                      double* __restrict__ tau, const int* st) {
  __shared__ double sd[BMAX], sw[BMAX], sc[3];
  __shared__ double prod[PQ_ROWS][PQ_CH + 1];
  __shared__ double seg[PQ_ROWS / PQ_CH][PQ_CH];
  if (status_bad(st)) return;
  const int t = threadIdx.x, G = gridDim.x;
  const int r = blockIdx.x * PQ_ROWS + t;
  double tk = 0.0, scale = 0.0, beta = 0.0;
  if (c >= 0) {
    {  // column j's partials part_in[j * G + g]: one warp per column, fixed-order tree
      const int w = t >> 5, lane = t & 31;
      for (int j = c + w; j < nb; j += PQ_ROWS / 32) {
        double s = 0.0;
        for (int g = lane; g < G; g += 32) s += part_in[(size_t)j * G + g];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sd[j] = s;
      }
    }
    __syncthreads();
    if (t == 0) {
      double alpha = prow_in[c], xn2 = sd[c];
      double tt = 0.0, sl = 0.0, be = alpha;
      if (xn2 > 0.0) {
        be = -copysign(sqrt(alpha * alpha + xn2), alpha);
        tt = (be - alpha) / be;
        sl = 1.0 / (alpha - be);
      }
      sc[0] = tt;
      sc[1] = sl;
      sc[2] = be;
      if (blockIdx.x == 0) tau[c] = tt;
    }
    __syncthreads();
    tk = sc[0];
    scale = sc[1];
    beta = sc[2];
    if (t < nb && t > c) sw[t] = prow_in[t] + scale * sd[t];  // v^T P(:, t)
    __syncthreads();
  }
  const int nc = c + 1;  // pivot column of the next step
  // this row: reflector entry and the new value of P(r, nc)
  double vr = 0.0, pn = 0.0;
  bool live = r < n && r >= (c < 0 ? 0 : c);
  if (live && c >= 0) {
    if (r == c) {
      P[r + (size_t)c * ldp] = beta;
    } else {
      vr = P[r + (size_t)c * ldp] * scale;
      P[r + (size_t)c * ldp] = vr;
    }
  }
  if (live && nc < nb) {
    double x = (c >= 0 && r == c) ? prow_in[nc] : P[r + (size_t)nc * ldp];
    if (c >= 0) x -= tk * (r == c ? 1.0 : vr) * sw[nc];
    pn = x;
  }
  for (int cb = (nc < 0 ? 0 : nc); cb < nb; cb += PQ_CH) {
    for (int q = 0; q < PQ_CH; ++q) {
      int j = cb + q;
      double pr = 0.0;
      if (live && j < nb) {
        double x = (c >= 0 && r == c) ? prow_in[j] : P[r + (size_t)j * ldp];
        if (c >= 0) {
          x -= tk * (r == c ? 1.0 : vr) * sw[j];
          P[r + (size_t)j * ldp] = x;
        }
        if (r == nc) prow_out[j] = x;
        if (r > nc) pr = pn * x;
      }
      prod[t][q] = pr;
    }
    __syncthreads();
    {
      int q = t % PQ_CH, sg = t / PQ_CH;
      double s = 0.0;
      for (int i = 0; i < PQ_CH; ++i) s += prod[sg * PQ_CH + i][q];
      seg[sg][q] = s;
    }
    __syncthreads();
    if (t < PQ_CH && cb + t < nb) {
      double s = 0.0;
      for (int sg = 0; sg < PQ_ROWS / PQ_CH; ++sg) s += seg[sg][t];
      part_out[(size_t)(cb + t) * G + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned long long gclock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The whole panel QR in one cooperative launch: CTA g keeps panel rows [rp g, rp g + rp)
// (rp = 64, 128 or 256: the per-SM FP64 rate bounds a step, so short panels take more
// CTAs of fewer rows) in shared memory for all column steps.  Each step is k_pqr_step's
// Householder step; the partial dot products of the next step are accumulated per column
// with FMAs down the CTA's rows (four row quarters, then three adds).  The partial sums and
// the next pivot row go through part/prow (ping-pong) across a grid barrier.  bar[0]
// counts barrier arrivals (zero on entry); a barrier that does not complete within 4 s
// records GEP_ERR_TIMEOUT and the CTA returns.
__global__ void __launch_bounds__(PQ_ROWS) k_pqr_coop(int n, int nb, int rp, double* __restrict__ P, int ldp,
                                                      double* __restrict__ part0, double* __restrict__ part1,
                                                      double* __restrict__ prow0, double* __restrict__ prow1,
                                                      double* __restrict__ tau, int* bar, int* st) {
  extern __shared__ double Ps[];  // [rp][nb + 1]
  __shared__ double sd[BMAX], sw[BMAX], sc[3];
  __shared__ double pnv[PQ_ROWS];      // P(r, nc) of the rows below the next pivot, else 0
  __shared__ double red4[4][BMAX];     // per-column partial dots of the four row quarters
  __shared__ int gok;
  if (status_bad(st)) return;
  const int t = threadIdx.x, G = gridDim.x, blk = blockIdx.x;
  const bool mine = t < rp;
  const int r = blk * rp + t;
  const int ld = nb + 1;
  if (mine)
    for (int j = 0; j < nb; ++j) Ps[t * ld + j] = (r < n) ? P[r + (size_t)j * ldp] : 0.0;
  const int nref = n < nb ? n : nb;
  double *pin = part0, *pout = part1, *rin = prow0, *rout = prow1;
  int epoch = 0;
  __syncthreads();
  for (int c = -1; c < nref; ++c) {
    double tk = 0.0, scale = 0.0, beta = 0.0;
    if (c >= 0) {
      {  // column j's partials pin[j * G + g], one warp per column, fixed-order tree
        const int w = t >> 5, lane = t & 31;
        for (int j = c + w; j < nb; j += PQ_ROWS / 32) {
          double s = 0.0;
          for (int g = lane; g < G; g += 32) s += __ldcg(pin + (size_t)j * G + g);
          for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) sd[j] = s;
        }
      }
      __syncthreads();
      if (t == 0) {
        double alpha = __ldcg(rin + c), xn2 = sd[c];
        double tt = 0.0, sl = 0.0, be = alpha;
        if (xn2 > 0.0) {
          be = -copysign(sqrt(alpha * alpha + xn2), alpha);
          tt = (be - alpha) / be;
          sl = 1.0 / (alpha - be);
        }
        sc[0] = tt;
        sc[1] = sl;
        sc[2] = be;
        if (blk == 0) tau[c] = tt;
      }
      __syncthreads();
      tk = sc[0];
      scale = sc[1];
      beta = sc[2];
      if (t < nb && t > c) sw[t] = __ldcg(rin + t) + scale * sd[t];  // v^T P(:, t)
      __syncthreads();
    }
    const int nc = c + 1;
    const bool live = mine && r < n && r >= (c < 0 ? 0 : c);
    double* row = Ps + t * ld;
    if (live && c >= 0) {
      const double vr = (r == c) ? 1.0 : row[c] * scale;
      row[c] = (r == c) ? beta : vr;
      for (int j = c + 1; j < nb; ++j) row[j] -= tk * vr * sw[j];
    }
    if (nc < nb) {
      // partial dots of column nc with columns j >= nc over this CTA's rows below the pivot:
      // thread (j = t mod 64, quarter t / 64) accumulates with FMAs down its rows, then the
      // four quarters are added (the FP64 pipe, not the loads, bounds this phase)
      if (mine) {
        pnv[t] = (live && r > nc) ? row[nc] : 0.0;
        if (live && r == nc)
          for (int j = nc; j < nb; ++j) rout[j] = row[j];
      }
      __syncthreads();
      {
        const int j = t & (BMAX - 1), qtr = t >> 6;
        double sum = 0.0;
        if (j >= nc && j < nb)
          for (int i = qtr; i < rp; i += 4) sum = fma(pnv[i], Ps[i * ld + j], sum);
        red4[qtr][j] = sum;
      }
      __syncthreads();
      if (t >= nc && t < nb) pout[(size_t)t * G + blk] = (red4[0][t] + red4[1][t]) + (red4[2][t] + red4[3][t]);
    }
    if (c + 1 >= nref) break;  // the last step needs no exchange
    // grid barrier: this CTA's pout / rout are complete and visible before any CTA reads them
    __syncthreads();
    if (t == 0) {
      __threadfence();
      const int target = (epoch + 1) * G;
      int ok = 1;
      if (atomicAdd(bar, 1) + 1 < target) {
        unsigned long long t0 = gclock();
        for (;;) {
          if (ld_acquire(bar) >= target) break;
          if (*(volatile int*)(st + 1) != 0) { ok = 0; break; }
          if (gclock() - t0 > 4000000000ull) {
            atomicExch(st + 1, GEP_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
      gok = ok;
    }
    __syncthreads();
    if (!gok) return;
    ++epoch;
    double* tp = pin; pin = pout; pout = tp;
    tp = rin; rin = rout; rout = tp;
  }
  __syncthreads();
  if (mine && r < n)
    for (int j = 0; j < nb; ++j) P[r + (size_t)j * ldp] = Ps[t * ld + j];
}

size_t pqr_coop_smem_bytes(int rp, int nb) { return (size_t)rp * (nb + 1) * sizeof(double); }

// V (n x nb, ld n): unit lower trapezoidal factor of the panel QR stored in P.
__global__ void k_panel_v(int n, int nb, const double* __restrict__ P, int ldp, double* __restrict__ V,
                          const int* st) {
  if (status_bad(st)) return;
  int r = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (r >= n || q >= nb) return;
  V[r + (size_t)q * n] = r < q ? 0.0 : (r == q ? 1.0 : P[r + (size_t)q * ldp]);
}

// ------------------------------------------------------------------ S1c bulge chasing

// Lower band storage with room for the bulge: AB[o + j*ldab] = C(j + o, j), 0 <= o < 2b.
__global__ void k_band_copy(int M, int b, const double* __restrict__ C, int ldc, double* __restrict__ AB, int ldab,
                            const int* st) {
  if (status_bad(st)) return;
  int o = threadIdx.x, j = blockIdx.x;
  if (o >= ldab || j >= M) return;
  AB[o + (size_t)j * ldab] = (o <= b && j + o < M) ? C[(j + o) + (size_t)j * ldc] : 0.0;
}

__device__ __forceinline__ int bulge_steps(int M, int b, int s) { return (M - 2 - s) / b + 1; }

struct BulgeArgs {
  int M, b, ldab, Q;  // Q = (M - 2) / b: groups 0..Q of b sweeps
  double* AB;
  int* prog;          // prog[s] = steps of sweep s completed
  double* q2;         // diamond storage (or null)
  int* st;
  unsigned long long wait_ns;  // limit of each progress wait
  int drop_sweep;              // test hook: this sweep publishes no progress (-1: none)
};

// Diamond (j, k) base in the reflector storage: [V: 2b x b][tau: b][T: b x b].
__host__ __device__ __forceinline__ size_t diamond_elems(int b) { return (size_t)3 * b * b + b; }
__host__ __device__ __forceinline__ size_t diamond_index(int Q, int j, int k) {
  return (size_t)j * (Q + 1) - (size_t)j * (j - 1) / 2 + k;
}

// dlarfg on x[0..len) (shared): v[0] = 1, v[i] = x[i] / (alpha - beta); returns tau, beta in out[0..1].
__device__ void house(const double* x, int len, double* v, double* out, int b) {
  const int t = threadIdx.x;
  if (t < 32) {
    double s = 0.0;
    for (int i = 1 + t; i < len; i += 32) s += x[i] * x[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (t < 2) {  // lane 0 forms tau, lane 1 the scale: one division sequence for both
      double alpha = x[0], be = alpha, q = 0.0;
      if (s > 0.0) {
        be = -copysign(sqrt(alpha * alpha + s), alpha);
        const double num = (t == 0) ? be - alpha : 1.0, den = (t == 0) ? be : alpha - be;
        q = num / den;
      }
      out[t == 0 ? 0 : 2] = q;
      if (t == 0) out[1] = be;
    }
  }
  __syncthreads();
  double sl = out[2];
  for (int i = t; i < b; i += blockDim.x) v[i] = (i == 0) ? 1.0 : (i < len ? x[i] * sl : 0.0);
  __syncthreads();
}

// D (len x len, full on entry, ld BMAX+1) <- H D H, H = I - tau v v^T; only the lower
// triangle of the result is formed.
__device__ void two_sided(double* D, int len, const double* v, double tau, double* p, double* red) {
  const int t = threadIdx.x, i = t & 63, part = t >> 6;
  double s = 0.0;
  if (i < len)
    for (int q = part; q < len; q += 4) s += D[i * (BMAX + 1) + q] * v[q];
  red[part * BMAX + i] = s;
  __syncthreads();
  if (t < len) p[t] = tau * (red[t] + red[BMAX + t] + red[2 * BMAX + t] + red[3 * BMAX + t]);
  __syncthreads();
  if (t < 32) {  // K = tau/2 p^T v
    double k = 0.0;
    for (int q = t; q < len; q += 32) k += p[q] * v[q];
    for (int o = 16; o; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if (t == 0) red[4 * BMAX] = 0.5 * tau * k;
  }
  __syncthreads();
  double K = red[4 * BMAX];
  if (t < len) p[t] -= K * v[t];  // w
  __syncthreads();
  // lower triangle only: the block is stored back as its lower part and re-read (and
  // mirrored) from the band at every step
  for (int idx = t; idx < len * len; idx += blockDim.x) {
    int a = idx % len, c = idx / len;
    if (a >= c) D[a * (BMAX + 1) + c] -= v[a] * p[c] + p[a] * v[c];
  }
  __syncthreads();
}

// One chasing step k >= 1 of a full block (b = len = BMAX = 64, 256 threads), the same
// arithmetic as the general step below with a fixed thread map: thread t owns row
// i = t mod 64 and columns q = t / 64 + 4 r (r < 16) of B and of the diagonal block D.
// B and the lower triangle of D are fetched in one round of coalesced loads.
__device__ __forceinline__ void bulge_step_full(const BulgeArgs& a, int stp, int st_k, double* Bm, double* Dm,
                                                const double* vp, double* vc, double* xv, double* pw, double* red,
                                                double* hs, double taup) {
  constexpr int N = BMAX, LD = BMAX + 1, R = N / 4;
  const int t = threadIdx.x, i = t & (N - 1), part = t >> 6;
  const int ldab = a.ldab;
  const double* AB = a.AB;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int q = part + 4 * r;
    Bm[i * LD + q] = __ldcg(AB + (N + i - q) + (size_t)(stp + q) * ldab);
    if (q <= i) Dm[i * LD + q] = __ldcg(AB + (i - q) + (size_t)(st_k + q) * ldab);
  }
  __syncthreads();
  {  // B <- B H(s, k-1): y = B vp, B -= taup y vp^T (the thread's own row: no barrier between)
    double y = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) y += Bm[i * LD + part + 4 * r] * vp[part + 4 * r];
    red[part * N + i] = y;
    __syncthreads();
    const double yi = taup * (red[i] + red[N + i] + red[2 * N + i] + red[3 * N + i]);
#pragma unroll
    for (int r = 0; r < R; ++r) Bm[i * LD + part + 4 * r] -= yi * vp[part + 4 * r];
    if (part == 0) xv[i] = Bm[i * LD];
  }
  __syncthreads();
  house(xv, N, vc, hs, N);
  const double tk = hs[0];
  {  // B(:, 1:) <- H B(:, 1:): u = tau B^T v over rows i = part + 4 r
    const int q = i;
    double u = 0.0;
    if (q >= 1)
#pragma unroll
      for (int r = 0; r < R; ++r) u += vc[part + 4 * r] * Bm[(part + 4 * r) * LD + q];
    red[part * N + q] = u;
    __syncthreads();
    if (t < N) pw[t] = tk * (red[t] + red[N + t] + red[2 * N + t] + red[3 * N + t]);
    __syncthreads();
    const double beta = hs[1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int qq = part + 4 * r;
      const double x = (qq == 0) ? (i == 0 ? beta : 0.0) : Bm[i * LD + qq] - vc[i] * pw[qq];
      a.AB[(N + i - qq) + (size_t)(stp + qq) * ldab] = x;
    }
  }
  {  // D <- H D H on the lower triangle (D read symmetric from its lower half)
    double y = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int q = part + 4 * r;
      y += (q <= i ? Dm[i * LD + q] : Dm[q * LD + i]) * vc[q];
    }
    red[part * N + i] = y;
    __syncthreads();
    if (t < N) pw[t] = tk * (red[t] + red[N + t] + red[2 * N + t] + red[3 * N + t]);
    __syncthreads();
    if (t < 32) {  // K = tau/2 p^T v
      double kk = 0.0;
      for (int q = t; q < N; q += 32) kk += pw[q] * vc[q];
      for (int o = 16; o; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
      if (t == 0) red[4 * N] = 0.5 * tk * kk;
    }
    __syncthreads();
    const double K = red[4 * N];
    if (t < N) pw[t] -= K * vc[t];
    __syncthreads();
    const double vi = vc[i], wi = pw[i];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int q = part + 4 * r;
      if (q <= i) {
        const double x = Dm[i * LD + q] - (vi * pw[q] + wi * vc[q]);
        a.AB[(i - q) + (size_t)(st_k + q) * ldab] = x;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_bulge(BulgeArgs a) {
  extern __shared__ double sm[];
  double* Bm = sm;                          // BMAX x (BMAX+1), [row][col]
  double* Dm = Bm + BMAX * (BMAX + 1);
  double* vp = Dm + BMAX * (BMAX + 1);      // previous reflector
  double* vc = vp + BMAX;                   // current reflector
  double* xv = vc + BMAX;                   // column to annihilate / scratch
  double* pw = xv + BMAX;
  double* red = pw + BMAX;                  // 4*BMAX + 1
  double* hs = red + 4 * BMAX + 8;          // tau, beta, scale
  __shared__ int abort_flag;
  const int t = threadIdx.x, M = a.M, b = a.b, ldab = a.ldab;
  if (t == 0) abort_flag = 0;
  __syncthreads();
  if (status_bad(a.st)) return;
  for (int s = blockIdx.x; s <= M - 2; s += gridDim.x) {
    const int ns = bulge_steps(M, b, s);
    double taup = 0.0;
    for (int k = 0; k < ns; ++k) {
      if (s > 0 && t == 0) {  // step k of sweep s needs step k+1 of sweep s-1
        int pns = bulge_steps(M, b, s - 1);
        int need = k + 2 < pns ? k + 2 : pns;
        unsigned long long t0 = gclock();
        while (ld_acquire(a.prog + (s - 1)) < need) {
          if (*(volatile int*)(a.st + 1) != 0) { abort_flag = 1; break; }
          if (gclock() - t0 > a.wait_ns) {
            atomicExch(a.st + 1, GEP_ERR_TIMEOUT);
            abort_flag = 1;
            break;
          }
        }
      }
      __syncthreads();
      if (abort_flag) return;
      const int st_k = s + 1 + k * b;
      const int len = (M - st_k) < b ? (M - st_k) : b;
      if (k > 0 && b == BMAX && len == BMAX) {
        bulge_step_full(a, st_k - b, st_k, Bm, Dm, vp, vc, xv, pw, red, hs, taup);
      } else {
        if (k == 0) {
          for (int i = t; i < len; i += blockDim.x) xv[i] = __ldcg(a.AB + (1 + i) + (size_t)s * ldab);
          __syncthreads();
          house(xv, len, vc, hs, b);
          if (t < len) a.AB[(1 + t) + (size_t)s * ldab] = (t == 0) ? hs[1] : 0.0;
        } else {
          const int stp = st_k - b;  // previous block's first row/column (its length is b)
          for (int idx = t; idx < len * b; idx += blockDim.x) {
            int i = idx % len, q = idx / len;
            Bm[i * (BMAX + 1) + q] = __ldcg(a.AB + (b + i - q) + (size_t)(stp + q) * ldab);
          }
          __syncthreads();
          {  // B <- B H(s,k-1): y = B vp, B -= taup y vp^T
            int i = t & 63, part = t >> 6;
            double y = 0.0;
            if (i < len)
              for (int q = part; q < b; q += 4) y += Bm[i * (BMAX + 1) + q] * vp[q];
            red[part * BMAX + i] = y;
            __syncthreads();
            if (t < len) pw[t] = taup * (red[t] + red[BMAX + t] + red[2 * BMAX + t] + red[3 * BMAX + t]);
            __syncthreads();
            for (int idx = t; idx < len * b; idx += blockDim.x) {
              int ii = idx % len, q = idx / len;
              Bm[ii * (BMAX + 1) + q] -= pw[ii] * vp[q];
            }
            __syncthreads();
          }
          for (int i = t; i < len; i += blockDim.x) xv[i] = Bm[i * (BMAX + 1)];
          __syncthreads();
          house(xv, len, vc, hs, b);
          {  // B(:, 1:) <- H B(:, 1:): u = tau B^T v
            double tk = hs[0];
            int q = t & 63, part = t >> 6;
            double u = 0.0;
            if (q >= 1 && q < b)
              for (int i = part; i < len; i += 4) u += vc[i] * Bm[i * (BMAX + 1) + q];
            red[part * BMAX + q] = u;
            __syncthreads();
            if (t < b) pw[t] = tk * (red[t] + red[BMAX + t] + red[2 * BMAX + t] + red[3 * BMAX + t]);
            __syncthreads();
            for (int idx = t; idx < len * b; idx += blockDim.x) {
              int i = idx % len, qq = idx / len;
              double x;
              if (qq == 0) x = (i == 0) ? hs[1] : 0.0;
              else x = Bm[i * (BMAX + 1) + qq] - vc[i] * pw[qq];
              a.AB[(b + i - qq) + (size_t)(stp + qq) * ldab] = x;
            }
          }
        }
        // D = C(st_k : st_k+len, same) <- H D H
        for (int idx = t; idx < len * len; idx += blockDim.x) {
          int i = idx % len, q = idx / len;
          int lo = i > q ? i : q, hi = i > q ? q : i;
          Dm[i * (BMAX + 1) + q] = __ldcg(a.AB + (lo - hi) + (size_t)(st_k + hi) * ldab);
        }
        __syncthreads();
        double tk = hs[0];
        two_sided(Dm, len, vc, tk, pw, red);
        for (int idx = t; idx < len * len; idx += blockDim.x) {
          int i = idx % len, q = idx / len;
          if (i >= q) a.AB[(i - q) + (size_t)(st_k + q) * ldab] = Dm[i * (BMAX + 1) + q];
        }
      }
      const double tk = hs[0];
      if (a.q2) {  // reflector into diamond (j, k), column c
        int j = s / b, c = s - j * b;
        double* D0 = a.q2 + diamond_index(a.Q, j, k) * diamond_elems(b);
        for (int i = t; i < len; i += blockDim.x) D0[(c + i) + (size_t)c * 2 * b] = vc[i];
        if (t == 0) D0[(size_t)2 * b * b + c] = tk;
      }
      if (t < b) vp[t] = vc[t];
      taup = tk;
      __syncthreads();  // every thread's stores of this step precede the release below
      if (t == 0 && s != a.drop_sweep) {
        __threadfence();
        st_release(a.prog + s, k + 1);
      }
    }
  }
}

__global__ void k_band_diag(int M, const double* __restrict__ AB, int ldab, double* __restrict__ d,
                            double* __restrict__ e, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  d[i] = AB[(size_t)i * ldab];
  if (i + 1 < M) e[i] = AB[1 + (size_t)i * ldab];
}

// ------------------------------------------------------------------ Q2 application

constexpr int Q2_COLS = 64;  // Z columns per CTA

// Z <- G(j,k) Z for every diamond of wavefront t (blockIdx.x) on a slab of Q2_COLS
// columns (blockIdx.y).  G(j,k) = H(s0,k) ... H(s0+b-1,k) is applied reflector by
// reflector, the last one first.  Each Z column is owned by four lanes of one warp.
__global__ void __launch_bounds__(256) k_q2_apply(int M, int b, int Q, int wt, const double* __restrict__ q2,
                                                  double* __restrict__ Z, int ldz, int ncol, const int* st) {
  extern __shared__ double sm[];
  if (status_bad(st)) return;
  const int kmin = wt - Q > 0 ? wt - Q : 0;
  const int k = kmin + blockIdx.x;
  if (2 * k > wt) return;  // k <= wt / 2 keeps j + k <= Q
  const int j = Q - wt + k;
  if (j < 0 || j > Q || k > Q - j) return;
  const int L = 2 * b - 1;
  const int r0 = 1 + (j + k) * b;
  const int c0 = blockIdx.y * Q2_COLS;
  double* Vs = sm;                      // [c][2b]
  double* Zs = Vs + (size_t)2 * b * b;  // [row][Q2_COLS + 1]
  double* ts = Zs + (size_t)L * (Q2_COLS + 1);
  const double* D0 = q2 + diamond_index(Q, j, k) * diamond_elems(b);
  const int t = threadIdx.x;
  for (int idx = t; idx < 2 * b * b; idx += blockDim.x) Vs[idx] = D0[idx];
  if (t < b) ts[t] = D0[(size_t)2 * b * b + t];
  for (int idx = t; idx < L * Q2_COLS; idx += blockDim.x) {
    int r = idx % L, cc = idx / L;
    int gr = r0 + r, gc = c0 + cc;
    Zs[r * (Q2_COLS + 1) + cc] = (gr < M && gc < ncol) ? Z[gr + (size_t)gc * ldz] : 0.0;
  }
  __syncthreads();
  const int col = t >> 2, part = t & 3;
  for (int c = b - 1; c >= 0; --c) {
    double tc = ts[c];
    if (tc == 0.0) continue;
    const double* v = Vs + (size_t)c * 2 * b;
    double u = 0.0;
    for (int r = c + part; r < c + b; r += 4) u += v[r] * Zs[r * (Q2_COLS + 1) + col];
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u *= tc;
    for (int r = c + part; r < c + b; r += 4) Zs[r * (Q2_COLS + 1) + col] -= u * v[r];
    __syncwarp();
  }
  __syncthreads();
  for (int idx = t; idx < L * Q2_COLS; idx += blockDim.x) {
    int r = idx % L, cc = idx / L;
    int gr = r0 + r, gc = c0 + cc;
    if (gr < M && gc < ncol) Z[gr + (size_t)gc * ldz] = Zs[r * (Q2_COLS + 1) + cc];
  }
}

// Dense tiles of Q2.  Tile (J, K) holds the diamonds (j, k) with j in [J TQ, (J+1) TQ)
// and k in [K TQ, (K+1) TQ); diamond (j, k) acts on rows 1 + (j + k) b .. + 2b - 2, so
// the tile acts on the W = 2 TQ b rows starting at 1 + (J + K) TQ b.  A diamond must
// precede (j, k+1) and, where rows overlap, the diamonds (j-1, k'), k' >= k of the next
// lower group: every dependency keeps or lowers j and keeps or raises k, so tiles are
// applied with J descending and K ascending, and inside a tile with j descending and k
// ascending.  U(J, K) is the product of its diamonds in that order, built by applying
// them to the identity, W x TB_COLS columns per CTA, and stored as U - I so that a tile
// is applied as Z(rows) += (U - I) Z(rows).
constexpr int TQ = 4;
constexpr int TB_COLS = 32;  // tile columns per CTA in the build (8 lanes per column)

__global__ void __launch_bounds__(256) k_q2_tile_build(int M, int b, int Q, int J, const double* __restrict__ q2,
                                                       double* __restrict__ U, const int* st) {
  extern __shared__ double sm[];
  if (status_bad(st)) return;
  const int K = blockIdx.x;
  const int W = 2 * TQ * b;
  const int J0 = J * TQ, K0 = K * TQ;
  const int r0 = 1 + (J0 + K0) * b;  // global row of tile row 0
  const int c0 = blockIdx.y * TB_COLS;
  double* Us = sm;  // [row][TB_COLS + 1]
  const int t = threadIdx.x;
  for (int idx = t; idx < W * TB_COLS; idx += blockDim.x) {
    int r = idx % W, cc = idx / W;
    Us[r * (TB_COLS + 1) + cc] = (r == c0 + cc) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int col = t >> 3, part = t & 7;
  const int jhi = min(J0 + TQ - 1, Q);
  // rows [rmin, rmax] hold every nonzero of this CTA's columns (identity columns at
  // first): a reflector whose rows miss that range leaves them unchanged and is skipped
  int rmin = c0, rmax = c0 + TB_COLS - 1;
  for (int j = jhi; j >= J0; --j) {
    for (int k = K0; k < K0 + TQ; ++k) {
      if (k > Q - j) continue;
      const double* D0 = q2 + diamond_index(Q, j, k) * diamond_elems(b);
      const int lo = (j + k - J0 - K0) * b;  // tile row of the diamond's row 0
      for (int c = b - 1; c >= 0; --c) {
        if (lo + c + b - 1 < rmin || lo + c > rmax) continue;
        double tc = D0[(size_t)2 * b * b + c];
        if (tc == 0.0) continue;
        rmin = min(rmin, lo + c);
        rmax = max(rmax, lo + c + b - 1);
        const double* v = D0 + (size_t)c * 2 * b;
        double u = 0.0;
        for (int r = c + part; r < c + b; r += 8)
          if (r0 + lo + r < M) u += v[r] * Us[(lo + r) * (TB_COLS + 1) + col];
        u += __shfl_xor_sync(0xffffffffu, u, 1);
        u += __shfl_xor_sync(0xffffffffu, u, 2);
        u += __shfl_xor_sync(0xffffffffu, u, 4);
        u *= tc;
        for (int r = c + part; r < c + b; r += 8)
          if (r0 + lo + r < M) Us[(lo + r) * (TB_COLS + 1) + col] -= u * v[r];
        __syncwarp();
      }
    }
  }
  __syncthreads();
  double* Ut = U + (size_t)K * W * W;  // U - I, W x W column-major
  for (int idx = t; idx < W * TB_COLS; idx += blockDim.x) {
    int r = idx % W, cc = idx / W;
    if (c0 + cc < W) Ut[r + (size_t)(c0 + cc) * W] = Us[r * (TB_COLS + 1) + cc] - (r == c0 + cc ? 1.0 : 0.0);
  }
}

size_t q2_tile_smem_bytes(int b) { return (size_t)2 * TQ * b * (TB_COLS + 1) * sizeof(double); }

size_t q2_smem_bytes(int b) {
  return ((size_t)2 * b * b + (size_t)(2 * b - 1) * (Q2_COLS + 1) + b) * sizeof(double);
}
size_t bulge_smem_bytes() { return ((size_t)2 * BMAX * (BMAX + 1) + 4 * BMAX + 4 * BMAX + 16) * sizeof(double); }

}  // namespace

// CTAs whose partial sums the panel-QR buffers hold: the per-step kernel's ceil(M / 256),
// or up to 1024 CTAs of 64 rows for the single-launch form.
static size_t pqr_partial_ctas(int M) {
  size_t g256 = ((size_t)M + PQ_ROWS - 1) / PQ_ROWS, g64 = ((size_t)M + 63) / 64;
  if (g64 > 1024) g64 = 1024;
  return g256 > g64 ? g256 : g64;
}

size_t q2_elems(int M, int b) {
  if (M < 2 || b < 1) return 0;
  size_t Q = (size_t)(M - 2) / b;
  return (Q + 1) * (Q + 2) / 2 * diamond_elems(b);
}

size_t band_ws_elems(int M, int b) {
  size_t G = pqr_partial_ctas(M);
  // + the digit planes of the trailing matrix (shared by the C22 products of a panel group)
  size_t reduce = 2 * rr(G * BMAX) + 2 * rr(BMAX) + rr(32) + 4 * rr((size_t)M * b) +
                  2 * rr((size_t)M * 2 * BAND_GROUP * b) + 5 * rr((size_t)2 * b * b) +
                  rr((size_t)2 * BAND_GROUP * b * b) + rr(oz_sym_planes_bytes(M, 9) / sizeof(double) + 1);
  size_t chase = rr((size_t)2 * b * M) + rr((size_t)M);  // band + progress counters
  return reduce > chase ? reduce : chase;
}

namespace {

struct BandWs {
  double *part0, *part1, *prow0, *prow1;
  long long gcap;  // CTAs the partial-sum buffers hold
  int* bar;
  double *V, *CV, *V1, *W1;
  double *WV, *VW;     // n x 2 G b: [W_0 V_0 W_1 V_1 ...] and [V_0 W_0 V_1 W_1 ...] of a panel group
  double *GV, *T, *Tt, *Pm, *Ym, *Zs;
  void* planes;        // digit planes of C22
  size_t planes_bytes;
};

// QR of the n x b panel P (ld ldp): reflectors stay in P, tau[0..b), explicit V (n x b,
// unit lower trapezoidal) and the compact-WY factor T (b x b).
int panel_factor(gep_handle_t h, int n, int b, double* P, int ldp, double* tau, const BandWs& w, double* V,
                 int eng) {
  const int G = (n + PQ_ROWS - 1) / PQ_ROWS;
  const int nref = n < b ? n : b;
  double *pin = w.part0, *pout = w.part1, *rin = w.prow0, *rout = w.prow1;
  // one cooperative launch when every CTA of the panel can be resident at once
  static int per_sm_of[64];
  static unsigned long long devices = 0;
  int dev = 0;
  GEP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GEP_ERR_UNSUPPORTED;
  if (first_use_on_device(devices)) {
    const size_t smax = pqr_coop_smem_bytes(PQ_ROWS, BMAX);
    GEP_CUDA(cudaFuncSetAttribute(k_pqr_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    GEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_of[dev], k_pqr_coop, PQ_ROWS, smax));
  }
  const int coop_per_sm = per_sm_of[dev];
  // fewest rows per CTA whose grid is resident at once and fits the partial-sum buffers
  // (a test may force 64, 128 or 256 rows, or the per-column kernel with -1)
  const long long cap = (long long)coop_per_sm * h->sm_count;
  int rp = 0;
  if (h->pqr_rows > 0) {
    const long long g = (n + h->pqr_rows - 1) / h->pqr_rows;
    if (g > cap || g > w.gcap) return GEP_ERR_UNSUPPORTED;
    rp = h->pqr_rows;
  } else if (h->pqr_rows == 0) {
    for (int c = 64; c <= PQ_ROWS; c *= 2) {
      long long g = (n + c - 1) / c;
      if (g <= cap && g <= w.gcap) { rp = c; break; }
    }
  }
  if (rp > 0) {
    const int Gc = (n + rp - 1) / rp;
    const size_t smem = pqr_coop_smem_bytes(rp, BMAX);
    GEP_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(int), h->stream));
    int nn = n, nbb = b, rpp = rp, ld = ldp;
    int* bar = w.bar;
    int* st = h->d_status;
    void* args[] = {&nn, &nbb, &rpp, &P, &ld, &pin, &pout, &rin, &rout, &tau, &bar, &st};
    GEP_CUDA(cudaLaunchCooperativeKernel((void*)k_pqr_coop, dim3(Gc), dim3(PQ_ROWS), args, smem, h->stream));
    GEP_CHECK(check_launch(h));
  } else {
    k_pqr_step<<<G, PQ_ROWS, 0, h->stream>>>(n, b, -1, P, ldp, pin, rin, pout, rout, tau, h->d_status);
    GEP_CHECK(check_launch(h));
    for (int c = 0; c < nref; ++c) {
      double* tp = pin; pin = pout; pout = tp;
      tp = rin; rin = rout; rout = tp;
      k_pqr_step<<<G, PQ_ROWS, 0, h->stream>>>(n, b, c, P, ldp, pin, rin, pout, rout, tau, h->d_status);
      GEP_CHECK(check_launch(h));
    }
  }
  k_panel_v<<<dim3((n + 255) / 256, b), 256, 0, h->stream>>>(n, b, P, ldp, V, h->d_status);
  GEP_CHECK(check_launch(h));
  GEP_CHECK(dgemm(h, 'T', 'N', 'F', b, b, n, 1.0, V, n, V, n, 0.0, w.GV, b, eng));
  return larft_rec(h, b, w.GV, b, tau, w.T, b, w.Tt);
}

// W = X - V (T^T V^T X) / 2 with X = CV T (CV = C22 V, n x b): the two-sided update of
// the trailing matrix is then C22 - W V^T - V W^T.
int panel_w(gep_handle_t h, int n, int b, const double* V, const double* CV, double* W, const BandWs& w, int eng) {
  GEP_CHECK(dgemm(h, 'N', 'N', 'F', n, b, b, 1.0, CV, n, w.T, b, 0.0, W, n, eng));    // X = C22 V T
  GEP_CHECK(dgemm(h, 'T', 'N', 'F', b, b, n, 1.0, V, n, W, n, 0.0, w.Pm, b, eng));    // V^T X
  GEP_CHECK(dgemm(h, 'T', 'N', 'F', b, b, b, 1.0, w.T, b, w.Pm, b, 0.0, w.Ym, b, eng));  // T^T V^T X
  return dgemm(h, 'N', 'N', 'F', n, b, b, -0.5, V, n, w.Ym, b, 1.0, W, n, eng);
}

}  // namespace

// S1b.  C (M x M, lower triangle) -> band of width b in C (lower), reflectors below the
// band, tau1[j] for columns j < M - b (zero where no reflector).  The upper triangle is
// not referenced.  Panels are taken in groups of up to BAND_GROUP: panel j of a group first
// receives the pending updates of panels 0..j-1 on its columns and diagonal block, its
// C^(j) V_j is formed from the group's not yet updated trailing matrix minus the low-rank
// corrections sum_i W_i (V_i^T V_j) + V_i (W_i^T V_j), and all the group's updates are
// applied together as one product of depth 2 G b (512 for G = 4, b = 64: one full exact
// chunk of the product kernel, and one digit split of the trailing matrix per group).
int band_reduce(gep_handle_t h, int M, double* C, int ldc, int b, double* tau1, double* ws, size_t ws_elems,
                int eng) {
  if (b < 1 || b > BMAX) return GEP_ERR_UNSUPPORTED;
  if (ws_elems < band_ws_elems(M, b)) return GEP_ERR_ALLOC;
  if (M <= 0) return GEP_OK;
  GEP_CHECK(set_matrix(h, M, 1, 0.0, 0.0, tau1, M));
  if (M <= b + 1) return GEP_OK;
  size_t Gmax = pqr_partial_ctas(M);
  BandWs w;
  w.gcap = (long long)Gmax;
  double* q = ws;
  auto take = [&](size_t n) { double* p = q; q += rr(n); return p; };
  w.part0 = take(Gmax * BMAX);
  w.part1 = take(Gmax * BMAX);
  w.prow0 = take(BMAX);
  w.prow1 = take(BMAX);
  w.bar = reinterpret_cast<int*>(take(32));
  w.V = take((size_t)M * b);
  w.CV = take((size_t)M * b);
  w.V1 = take((size_t)M * b);
  w.W1 = take((size_t)M * b);
  w.WV = take((size_t)M * 2 * BAND_GROUP * b);
  w.VW = take((size_t)M * 2 * BAND_GROUP * b);
  w.GV = take((size_t)2 * b * b);
  w.T = take((size_t)2 * b * b);
  w.Tt = take((size_t)2 * b * b);
  w.Pm = take((size_t)2 * b * b);
  w.Ym = take((size_t)2 * b * b);
  w.Zs = take((size_t)2 * BAND_GROUP * b * b);
  w.planes_bytes = oz_sym_planes_bytes(M, 9);
  w.planes = take(w.planes_bytes / sizeof(double) + 1);
  const int levels = eng == GEP_PREC_MIXED_REFINED ? 4 : 9;
  for (int pb = 0; M - pb - b >= 2;) {
    const int n = M - pb - b;
    // panels of this group: panel j (j >= 1) owns columns [(j-1) b, j b) of C22 and its
    // reflectors act on rows [j b, n), which needs n - j b >= 2
    // (groups pay where the trailing matrix is large; below that pairs, whose two C22 products
    // need no cross-panel corrections beyond one pair of small products)
    const int gmin = h->band_group_min >= 0 ? h->band_group_min : BAND_GROUP_MIN_N;
    const int g = std::min(n >= gmin ? BAND_GROUP : 2, (n - 2) / b + 1);
    double* P = C + (pb + b) + (size_t)pb * ldc;
    double* C22 = C + (pb + b) + (size_t)(pb + b) * ldc;
    // V_j and W_j are kept at full height n (zero above row j b) in WV / VW, so that the
    // pending update of panel i on any block of C22 is the same slice of one product.
    auto wv = [&](int blk) { return w.WV + (size_t)blk * b * n; };
    auto vw = [&](int blk) { return w.VW + (size_t)blk * b * n; };
    // C22 is split into digit planes once for the group on the tensor-core engines: every
    // C^(j) V_j below reads rows j b.. of the planes against the full-height V_j.  The columns
    // the group updates in between (those of panels 1..g-1) meet V_j's zero rows.
    OzSymPlanes planes;
    const bool use_planes = eng != GEP_PREC_FP64 && n >= 128 && b >= 64;
    if (use_planes) GEP_CHECK(oz_split_sym(h, n, C22, ldc, levels, w.planes, w.planes_bytes, &planes));
    for (int j = 0; j < g; ++j) {
      const int r0 = j * b, nr = n - r0;  // panel j's reflectors act on rows [r0, n) of C22
      double* Vj;
      if (j == 0) {
        GEP_CHECK(panel_factor(h, n, b, P, ldc, tau1 + pb, w, w.V, eng));
        Vj = w.V;
      } else {
        // panel j = C22 columns [(j-1) b, j b), rows [(j-1) b, n): the pending updates of
        // panels 0..j-1 first (its diagonal block on the lower triangle only), then its QR
        const int c0 = r0 - b;
        double* Dj = C22 + c0 + (size_t)c0 * ldc;
        GEP_CHECK(dgemm(h, 'N', 'T', 'L', b, b, 2 * j * b, -1.0, w.WV + c0, n, w.VW + c0, n, 1.0, Dj, ldc, eng));
        GEP_CHECK(dgemm(h, 'N', 'T', 'F', nr, b, 2 * j * b, -1.0, w.WV + r0, n, w.VW + c0, n, 1.0, Dj + b, ldc,
                        eng));
        GEP_CHECK(panel_factor(h, nr, b, Dj + b, ldc, tau1 + pb + r0, w, w.V1, eng));
        Vj = w.V1;
      }
      // V_j at full height into both group buffers (zero rows above r0)
      if (r0 > 0) {
        GEP_CHECK(set_matrix(h, r0, b, 0.0, 0.0, wv(2 * j + 1), n));
        GEP_CHECK(set_matrix(h, r0, b, 0.0, 0.0, vw(2 * j), n));
        GEP_CHECK(set_matrix(h, r0, b, 0.0, 0.0, wv(2 * j), n));
        GEP_CHECK(set_matrix(h, r0, b, 0.0, 0.0, vw(2 * j + 1), n));
      }
      GEP_CHECK(copy_matrix(h, nr, b, Vj, nr, wv(2 * j + 1) + r0, n));
      GEP_CHECK(copy_matrix(h, nr, b, Vj, nr, vw(2 * j) + r0, n));
      // C^(j) V_j = C22(r0:, r0:) V_j - sum_{i<j} (W_i V_i^T + V_i W_i^T)(r0:, r0:) V_j
      if (use_planes && nr >= 128) {
        GEP_CHECK(dgemm_oz_sym_planes(h, planes, r0, b, 1.0, vw(2 * j), n, 0.0, w.CV, nr));
      } else {
        GEP_CHECK(dgemm(h, 'S', 'N', 'F', nr, b, nr, 1.0, C22 + r0 + (size_t)r0 * ldc, ldc, Vj, nr, 0.0, w.CV, nr,
                        eng));
      }
      if (j > 0) {
        // Zs = [V_0 W_0 .. V_{j-1} W_{j-1}](r0:)^T V_j, CV -= [W_0 V_0 ..](r0:) Zs
        GEP_CHECK(dgemm(h, 'T', 'N', 'F', 2 * j * b, b, nr, 1.0, w.VW + r0, n, Vj, nr, 0.0, w.Zs, 2 * j * b, eng));
        GEP_CHECK(dgemm(h, 'N', 'N', 'F', nr, b, 2 * j * b, -1.0, w.WV + r0, n, w.Zs, 2 * j * b, 1.0, w.CV, nr,
                        eng));
      }
      GEP_CHECK(panel_w(h, nr, b, Vj, w.CV, w.W1, w, eng));
      GEP_CHECK(copy_matrix(h, nr, b, w.W1, nr, wv(2 * j) + r0, n));
      GEP_CHECK(copy_matrix(h, nr, b, w.W1, nr, vw(2 * j + 1) + r0, n));
    }
    // trailing matrix after the group: C22(t0:, t0:) -= [W_0 V_0 ..][V_0 W_0 ..]^T (lower
    // triangle, depth 2 g b), t0 = (g-1) b
    const int t0 = (g - 1) * b, nt = n - t0;
    GEP_CHECK(dgemm(h, 'N', 'T', 'L', nt, nt, 2 * g * b, -1.0, w.WV + t0, n, w.VW + t0, n, 1.0,
                    C22 + t0 + (size_t)t0 * ldc, ldc, eng));
    pb += g * b;
  }
  return GEP_OK;
}

// S1c.  Band of width b in the lower triangle of C -> d, e; reflectors into q2 (may be null).
int band_to_tridiag(gep_handle_t h, int M, const double* C, int ldc, int b, double* d, double* e, double* q2,
                    double* ws, size_t ws_elems) {
  if (b < 1 || b > BMAX) return GEP_ERR_UNSUPPORTED;
  if (ws_elems < band_ws_elems(M, b)) return GEP_ERR_ALLOC;
  if (M <= 0) return GEP_OK;
  const int ldab = 2 * b;
  double* AB = ws;
  int* prog = reinterpret_cast<int*>(ws + rr((size_t)2 * b * M));
  k_band_copy<<<M, ldab, 0, h->stream>>>(M, b, C, ldc, AB, ldab, h->d_status);
  GEP_CHECK(check_launch(h));
  if (M >= 2) {
    GEP_CUDA(cudaMemsetAsync(prog, 0, sizeof(int) * (size_t)M, h->stream));
    const int Q = (M - 2) / b;
    if (q2) GEP_CUDA(cudaMemsetAsync(q2, 0, q2_elems(M, b) * sizeof(double), h->stream));
    size_t smem = bulge_smem_bytes();
    static unsigned long long attr_devices = 0;
    if (first_use_on_device(attr_devices))
      GEP_CUDA(cudaFuncSetAttribute(k_bulge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bulge, 256, smem));
    if (per_sm < 1) return GEP_ERR_UNSUPPORTED;
    // The sweeps form a dependency chain (step k of sweep s waits for step k+1 of sweep
    // s-1): the time is set by the latency of one step, which co-resident CTAs stretch.
    if (per_sm > BULGE_CTAS_PER_SM) per_sm = BULGE_CTAS_PER_SM;
    int grid = per_sm * h->sm_count;
    // Sweep s starts two steps after sweep s-1 and lasts about (M - 2) / b + 1 steps, so
    // about half that many sweeps are in flight at once: CTAs beyond that would only wait,
    // holding SMs that concurrent solves on other streams could use.
    const int in_flight = ((M - 2) / b + 1) / 2 + 2;
    if (grid > in_flight) grid = in_flight;
    if (grid > M - 1) grid = M - 1;
    BulgeArgs a;
    a.M = M; a.b = b; a.ldab = ldab; a.Q = Q; a.AB = AB; a.prog = prog; a.q2 = q2; a.st = h->d_status;
    a.wait_ns = h->wait_limit_ns;
    a.drop_sweep = h->fault_drop_sweep;
    void* args[] = {&a};
    GEP_CUDA(cudaLaunchCooperativeKernel((void*)k_bulge, dim3(grid), dim3(256), args, smem, h->stream));
    GEP_CHECK(check_launch(h));
  }
  k_band_diag<<<(M + 255) / 256, 256, 0, h->stream>>>(M, AB, ldab, d, e, h->d_status);
  return check_launch(h);
}

size_t q2_tile_ws_elems(int M, int b) {
  if (M < 3 || b < 1) return 0;
  size_t Q = (size_t)(M - 2) / b;
  size_t nK = Q / TQ + 1, W = (size_t)2 * TQ * b;
  return rr(nK * W * W) + rr(W * (size_t)M);
}

namespace {

// Tiles of every tile row J, one after the other (tile (J, K) at all_tiles_offset(Q, J) + K).
size_t all_tiles_offset(int Q, int J) {
  size_t off = 0;
  for (int j = 0; j < J; ++j) off += (size_t)((Q - j * TQ) / TQ + 1);
  return off;
}

int set_tile_build_attr() {
  static unsigned long long attr_devices = 0;
  if (first_use_on_device(attr_devices))
    GEP_CUDA(cudaFuncSetAttribute(k_q2_tile_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)q2_tile_smem_bytes(BMAX)));
  return GEP_OK;
}

}  // namespace

size_t q2_all_tiles_elems(int M, int b) {
  if (M < 3 || b < 1) return 0;
  const int Q = (M - 2) / b;
  const size_t W = (size_t)2 * TQ * b;
  return all_tiles_offset(Q, Q / TQ + 1) * W * W;
}

// Builds every dense tile U(J, K) - I of Q2 into U (q2_all_tiles_elems doubles) on `stream`,
// for apply_q2 to use later; it only reads q2, so it may run on a second stream while the
// tridiagonal eigensolver runs on the first.
int build_q2_tiles(gep_handle_t h, cudaStream_t stream, int M, int b, const double* q2, double* U) {
  if (b < 1 || b > BMAX) return GEP_ERR_UNSUPPORTED;
  if (M < 3) return GEP_OK;
  GEP_CHECK(set_tile_build_attr());
  const int Q = (M - 2) / b;
  const int W = 2 * TQ * b, nJ = Q / TQ + 1;
  const size_t smem = q2_tile_smem_bytes(b);
  for (int J = 0; J < nJ; ++J) {
    const int nK = (Q - J * TQ) / TQ + 1;
    double* UJ = U + all_tiles_offset(Q, J) * (size_t)W * W;
    k_q2_tile_build<<<dim3(nK, (W + TB_COLS - 1) / TB_COLS), 256, smem, stream>>>(M, b, Q, J, q2, UJ, h->d_status);
    GEP_CHECK(check_launch(h));
  }
  return GEP_OK;
}

// Where U(J, K) - I can be nonzero, per 128-row block of a W x W tile: the reflectors of the
// tile's diamonds, taken in the order k_q2_tile_build applies them, spread each column's
// nonzero rows over an interval (a reflector whose rows miss the interval leaves the
// column alone, one that meets it widens it to the union).  Row block r then needs only
// the columns whose interval meets its rows.  Every tile has this structure or a subset
// of it (tiles at the edge hold fewer diamonds).
static void q2_tile_kranges(int b, OzKRange* kr) {
  const int W = 2 * TQ * b;
  std::vector<int> rmin(W), rmax(W);
  for (int c = 0; c < W; ++c) rmin[c] = rmax[c] = c;
  for (int jj = TQ - 1; jj >= 0; --jj)
    for (int kk = 0; kk < TQ; ++kk)
      for (int c = b - 1; c >= 0; --c) {
        const int r0 = (jj + kk) * b + c, r1 = r0 + b - 1;
        for (int x = 0; x < W; ++x)
          if (r0 <= rmax[x] && r1 >= rmin[x]) {
            rmin[x] = std::min(rmin[x], r0);
            rmax[x] = std::max(rmax[x], r1);
          }
      }
  kr->n = std::min((W + 127) / 128, OZ_KR_MAX);
  for (int r = 0; r < kr->n; ++r) {
    const int a = 128 * r, e = std::min(W, a + 128) - 1;
    int lo = W, hi = 0;
    for (int x = 0; x < W; ++x)
      if (rmin[x] <= e && rmax[x] >= a) {
        lo = std::min(lo, x);
        hi = std::max(hi, x + 1);
      }
    kr->lo[r] = lo < hi ? lo : 0;
    kr->hi[r] = lo < hi ? hi : 0;
  }
}

// Z (M x ncol) <- Q2 Z.  engine FP64: diamonds applied directly on the FP64 cores.
// Otherwise the diamonds are merged into dense W x W tiles U(J, R) and every tile is
// applied as one product Z(rows) <- U Z(rows) on the engine (ws: q2_tile_ws_elems).
// U_all != null: the tiles were built by build_q2_tiles (on the caller's stream order).
int apply_q2(gep_handle_t h, int M, int b, const double* q2, double* Z, int ldz, int ncol, int engine, double* ws,
             size_t ws_elems, const double* U_all) {
  if (b < 1 || b > BMAX) return GEP_ERR_UNSUPPORTED;
  if (M < 3 || ncol <= 0) return GEP_OK;  // M = 2: the only reflector is the identity
  const int Q = (M - 2) / b;
  if (engine != GEP_PREC_FP64) {
    if (ws_elems < q2_tile_ws_elems(M, b)) return GEP_ERR_ALLOC;
    const int W = 2 * TQ * b;
    const int nJ = Q / TQ + 1;
    double* Ubuf = ws;
    double* Tmp = ws + rr((size_t)(Q / TQ + 1) * W * W);
    size_t smem = q2_tile_smem_bytes(b);
    OzKRange kr;
    q2_tile_kranges(b, &kr);
    GEP_CHECK(set_tile_build_attr());
    for (int J = nJ - 1; J >= 0; --J) {
      const int nK = (Q - J * TQ) / TQ + 1;  // tiles (J, K) with a diamond: K TQ <= Q - J TQ
      const double* U = Ubuf;
      if (U_all) {
        U = U_all + all_tiles_offset(Q, J) * (size_t)W * W;
      } else {
        k_q2_tile_build<<<dim3(nK, (W + TB_COLS - 1) / TB_COLS), 256, smem, h->stream>>>(M, b, Q, J, q2, Ubuf,
                                                                                        h->d_status);
        GEP_CHECK(check_launch(h));
      }
      for (int K = 0; K < nK; ++K) {
        const int r0 = 1 + (J + K) * TQ * b;
        if (r0 >= M) break;
        const int Wc = (M - r0) < W ? (M - r0) : W;
        const double* Ut = U + (size_t)K * W * W;
        // one K panel of the split-BF16 engine: all of Z(rows) is split into digit planes
        // before its product kernel writes C, so the update may run in place
        const size_t one_panel = (size_t)16 * (Wc + ncol) * ((Wc + 31) / 32 * 32) + (size_t)4 * (Wc + ncol) + 4096;
        if (Wc >= 128 && ncol >= 64 && Wc <= 4096 && one_panel <= h->eng_bytes) {
          GEP_CHECK(dgemm(h, 'N', 'N', 'F', Wc, ncol, Wc, 1.0, Ut, W, Z + r0, ldz, 1.0, Z + r0, ldz, engine, &kr));
        } else {  // Z(rows) += (U - I) copy(Z(rows))
          GEP_CHECK(copy_matrix(h, Wc, ncol, Z + r0, ldz, Tmp, Wc));
          GEP_CHECK(dgemm(h, 'N', 'N', 'F', Wc, ncol, Wc, 1.0, Ut, W, Tmp, Wc, 1.0, Z + r0, ldz, engine, &kr));
        }
      }
    }
    return GEP_OK;
  }
  size_t smem = q2_smem_bytes(b);
  static unsigned long long attr_devices = 0;
  if (first_use_on_device(attr_devices))
    GEP_CUDA(cudaFuncSetAttribute(k_q2_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)q2_smem_bytes(BMAX)));
  const int slabs = (ncol + Q2_COLS - 1) / Q2_COLS;
  for (int wt = 0; wt <= 2 * Q; ++wt) {
    int kmin = wt - Q > 0 ? wt - Q : 0, kmax = wt / 2;
    if (kmax < kmin) continue;
    k_q2_apply<<<dim3(kmax - kmin + 1, slabs), 256, smem, h->stream>>>(M, b, Q, wt, q2, Z, ldz, ncol,
                                                                      h->d_status);
    GEP_CHECK(check_launch(h));
  }
  return GEP_OK;
}

}  // namespace gep
