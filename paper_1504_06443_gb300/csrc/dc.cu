// SEP solver, stage "D&C" (Table 3): eigenvalues and eigenvectors of the
// symmetric tridiagonal T = tridiag(e, d, e) by divide and conquer.
//
// T is torn at every multiple of LEAF (Cuppen): at split point p the coupling
// beta = e[p-1] is removed from the diagonal on both sides, leaving independent
// leaves solved one warp each (implicit QL with Wilkinson shift in shared
// memory).  Leaves are merged bottom-up, level by level.  Merging two solved
// halves is the rank-one problem D + rho z z^T (z = last row of Q1 and first row
// of Q2 scaled by sign(beta)/sqrt(2), rho = 2|beta|), handled as:
//   1. deflation of negligible z_i and of nearly equal d_i (Givens rotation),
//   2. one root per non-deflated pole of the secular equation
//        f(lambda) = 1 + rho sum_i z_i^2 / (d_i - lambda) = 0,
//      found by a bracketed iteration on a two-pole rational model, with the root
//      stored as (nearest pole, offset) so every d_i - lambda_j is accurate,
//   3. z recomputed from the roots (Loewner formula, Gu & Eisenstat) so the
//      eigenvectors u_j ~ z_i / (d_i - lambda_j) are numerically orthogonal,
//   4. the merged eigenvectors Q [u_j] as one product per child on the GEMM engine
//      (the deflation rotations are folded into the rows of [u_j], so Q stays
//      block diagonal).
// Eigenvalues of every block are kept sorted ascending.
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int LEAF = 32;
constexpr double EPS = 0x1p-53;

struct DcWs {
  double *Qt, *U, *D, *dd, *zs, *dv, *ndd, *ndz, *dfv, *rc, *rs, *tauR, *lam, *zhat, *newD, *rho;
  double *ptau, *pc, *ps;  // the Givens deflation test of each adjacent pair, from the undeflated values
  int *perm, *ndx, *dfx, *ra, *rb, *org, *posr, *posd, *cnt;
  int *nsl, *prot;         // positions (in perm) with z not negligible; pair test outcome
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

__device__ double block_max(double v, double* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// Tearing: dd = d with |e[p-1]| removed on both sides of every split point p.
__global__ void k_tear(int M, const double* __restrict__ d, const double* __restrict__ e,
                       double* __restrict__ dd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double v = d[i];
  if (i > 0 && i % LEAF == 0) v -= fabs(e[i - 1]);
  if ((i + 1) % LEAF == 0 && i + 1 < M) v -= fabs(e[i]);
  dd[i] = v;
}

// One warp per leaf: implicit QL with Wilkinson shift; eigenvectors accumulated in
// shared memory (lane r owns row r), then sorted ascending and written to Z/D.
__global__ void __launch_bounds__(128) k_leaf(int M, const double* __restrict__ dd,
                                              const double* __restrict__ e, double* __restrict__ D,
                                              double* __restrict__ Z, int ldz, int* st) {
  __shared__ double Zs[4][LEAF][LEAF + 1];
  __shared__ double dl[4][LEAF], el[4][LEAF], rcs[4][LEAF], rsn[4][LEAF];
  __shared__ int ord[4][LEAF];
  __shared__ int sh_m[4], sh_n[4], sh_stop[4];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int leaf = blockIdx.x * 4 + w;
  int lo = leaf * LEAF;
  if (lo >= M) return;
  int n = min(LEAF, M - lo);
  for (int c = 0; c < LEAF; ++c) Zs[w][lane][c] = (lane == c) ? 1.0 : 0.0;
  dl[w][lane] = (lane < n) ? dd[lo + lane] : 0.0;
  el[w][lane] = (lane < n - 1) ? e[lo + lane] : 0.0;
  __syncwarp();
  int bad = 0;
  for (int l = 0; l < n && !bad; ++l) {
    int iter = 0;
    for (;;) {
      if (lane == 0) {
        int m = l;
        for (; m + 1 < n; ++m) {
          double s = fabs(dl[w][m]) + fabs(dl[w][m + 1]);
          if (fabs(el[w][m]) <= 2.0 * EPS * s) break;
        }
        sh_m[w] = m;
        sh_stop[w] = 0;
        if (m != l) {
          if (++iter > 40) {
            sh_stop[w] = 2;
          } else {
            double g = (dl[w][l + 1] - dl[w][l]) / (2.0 * el[w][l]);
            double r = hypot(g, 1.0);
            g = dl[w][m] - dl[w][l] + el[w][l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int nr = 0, early = 0;
            for (int i = m - 1; i >= l; --i) {
              double f = s * el[w][i], b = c * el[w][i];
              r = hypot(f, g);
              el[w][i + 1] = r;
              if (r == 0.0) {
                dl[w][i + 1] -= p;
                el[w][m] = 0.0;
                early = 1;
                break;
              }
              s = f / r;
              c = g / r;
              g = dl[w][i + 1] - p;
              r = (dl[w][i] - g) * s + 2.0 * c * b;
              p = s * r;
              dl[w][i + 1] = g + p;
              g = c * r - b;
              rcs[w][nr] = c;
              rsn[w][nr] = s;
              ++nr;
            }
            if (!early) {
              dl[w][l] -= p;
              el[w][l] = g;
              el[w][m] = 0.0;
            }
            sh_n[w] = nr;
            sh_stop[w] = 1;
          }
        }
      }
      __syncwarp();
      int m = sh_m[w], stop = sh_stop[w];
      if (m == l) break;
      if (stop == 2) { bad = 1; break; }
      int nr = sh_n[w];
      for (int q = 0; q < nr; ++q) {
        int col = m - 1 - q;
        double zi = Zs[w][lane][col], zi1 = Zs[w][lane][col + 1];
        Zs[w][lane][col + 1] = rsn[w][q] * zi + rcs[w][q] * zi1;
        Zs[w][lane][col] = rcs[w][q] * zi - rsn[w][q] * zi1;
      }
      __syncwarp();
    }
  }
  if (bad) {
    if (lane == 0) atomicCAS(st, 0, M + lo + 1);
    return;
  }
  if (lane == 0) {
    for (int j = 0; j < n; ++j) ord[w][j] = j;
    for (int a = 1; a < n; ++a) {  // insertion sort of indices by eigenvalue
      int t = ord[w][a], b = a - 1;
      while (b >= 0 && dl[w][ord[w][b]] > dl[w][t]) { ord[w][b + 1] = ord[w][b]; --b; }
      ord[w][b + 1] = t;
    }
  }
  __syncwarp();
  if (lane < n)
    for (int j = 0; j < n; ++j) Z[GEP_IX(lo + lane, lo + j, ldz)] = Zs[w][lane][ord[w][j]];
  if (lane < n) D[lo + lane] = dl[w][ord[w][lane]];
}

// Merge set-up (one CTA): z, sort of the two halves' eigenvalues, deflation.  The
// deflation scan is sequential (a Givens rotation changes the next pair's operands), but
// only a rotated pair's successor needs its test re-evaluated: every pair's test is first
// formed in parallel from the undeflated values, and the scan takes those results wherever
// the previous pair was not rotated, which gives the sequential outcome exactly.
__global__ void __launch_bounds__(1024) k_prep(int lo, int mid, int hi, const double* __restrict__ e,
                                               const double* __restrict__ D, const double* __restrict__ Z,
                                               int ldz, DcWs w, const int* st) {
  __shared__ double red[32];
  __shared__ int scnt[1024];
  if (status_bad(st)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  int n = hi - lo, n1 = mid - lo;
  double beta = e[mid - 1];
  double sg = beta < 0.0 ? -1.0 : 1.0;
  double rho = 2.0 * fabs(beta);
  double zmax = 0.0, dmax = 0.0;
  for (int t = tid; t < n; t += nt) {
    double z = (t < n1) ? Z[GEP_IX(mid - 1, lo + t, ldz)] : sg * Z[GEP_IX(mid, lo + t, ldz)];
    z *= 0.70710678118654752440;
    w.zs[t] = z;
    double dv = D[lo + t];
    w.dv[t] = dv;
    zmax = fmax(zmax, fabs(z));
    dmax = fmax(dmax, fabs(dv));
  }
  zmax = block_max(zmax, red);
  dmax = block_max(dmax, red);
  __syncthreads();
  const double tol = 8.0 * EPS * 2.0 * fmax(dmax, zmax);
  // merge the two ascending runs [0, n1) and [n1, n), the first run's entry first on ties
  for (int x = tid; x < n; x += nt) {
    const double v = w.dv[x];
    int a = (x < n1) ? n1 : 0, b = (x < n1) ? n : n1;  // search the other run
    while (a < b) {
      int c = (a + b) >> 1;
      bool before = (x < n1) ? (w.dv[c] < v) : (w.dv[c] <= v);
      if (before) a = c + 1; else b = c;
    }
    w.perm[(x < n1) ? x + (a - n1) : (x - n1) + a] = x;
  }
  __syncthreads();
  // positions whose z is not negligible, in order (chunk counts, then a scan)
  const int chunk = (n + nt - 1) / nt, c0 = tid * chunk, c1 = min(n, c0 + chunk);
  int cnt = 0;
  for (int q = c0; q < c1; ++q) cnt += !(rho * fabs(w.zs[w.perm[q]]) <= tol);
  scnt[tid] = cnt;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    int v = tid >= o ? scnt[tid - o] : 0;
    __syncthreads();
    scnt[tid] += v;
    __syncthreads();
  }
  const int nns = scnt[nt - 1];
  for (int q = c0, o = scnt[tid] - cnt; q < c1; ++q)
    if (!(rho * fabs(w.zs[w.perm[q]]) <= tol)) w.nsl[o++] = q;
  __syncthreads();
  // the rotation test of every adjacent pair, from the undeflated values
  for (int m = 1 + tid; m < nns; m += nt) {
    const int pj = w.perm[w.nsl[m - 1]], t = w.perm[w.nsl[m]];
    double zs_ = w.zs[pj], zc = w.zs[t];
    double tau = hypot(zc, zs_);
    double c = zc / tau, sn = -zs_ / tau;
    double tdiff = w.dv[t] - w.dv[pj];
    w.prot[m] = fabs(tdiff * c * sn) <= tol;
    w.ptau[m] = tau;
    w.pc[m] = c;
    w.ps[m] = sn;
  }
  __syncthreads();
  if (tid != 0) return;
  int k = 0, nd = 0, nr = 0, pj = -1, mi = -1;
  bool prev_rot = false;
  for (int s = 0; s < n; ++s) {
    int t = w.perm[s];
    if (rho * fabs(w.zs[t]) <= tol) {
      w.dfx[nd] = t;
      w.dfv[nd] = w.dv[t];
      ++nd;
      continue;
    }
    ++mi;
    if (pj < 0) { pj = t; continue; }
    double tau, c, sn;
    bool rot;
    if (prev_rot) {  // pj was rotated into: its z and d changed
      double zs_ = w.zs[pj], zc = w.zs[t];
      tau = hypot(zc, zs_);
      c = zc / tau;
      sn = -zs_ / tau;
      double tdiff = w.dv[t] - w.dv[pj];
      rot = fabs(tdiff * c * sn) <= tol;
    } else {
      tau = w.ptau[mi];
      c = w.pc[mi];
      sn = w.ps[mi];
      rot = w.prot[mi] != 0;
    }
    if (rot) {
      w.zs[t] = tau;
      w.zs[pj] = 0.0;
      w.ra[nr] = pj; w.rb[nr] = t; w.rc[nr] = c; w.rs[nr] = sn; ++nr;
      double dp = w.dv[pj], dt = w.dv[t];
      double t2 = dp * c * c + dt * sn * sn;
      w.dv[t] = dp * sn * sn + dt * c * c;
      w.dv[pj] = t2;
      w.dfx[nd] = pj;
      w.dfv[nd] = t2;
      ++nd;
    } else {
      w.ndx[k] = pj; w.ndd[k] = w.dv[pj]; w.ndz[k] = w.zs[pj]; ++k;
    }
    prev_rot = rot;
    pj = t;
  }
  if (pj >= 0) { w.ndx[k] = pj; w.ndd[k] = w.dv[pj]; w.ndz[k] = w.zs[pj]; ++k; }
  // both lists ascending (they are nearly sorted already)
  for (int x = 1; x < nd; ++x) {
    double v = w.dfv[x];
    int ix = w.dfx[x], y = x - 1;
    while (y >= 0 && w.dfv[y] > v) { w.dfv[y + 1] = w.dfv[y]; w.dfx[y + 1] = w.dfx[y]; --y; }
    w.dfv[y + 1] = v; w.dfx[y + 1] = ix;
  }
  for (int x = 1; x < k; ++x) {
    double v = w.ndd[x], zz = w.ndz[x];
    int ix = w.ndx[x], y = x - 1;
    while (y >= 0 && w.ndd[y] > v) { w.ndd[y + 1] = w.ndd[y]; w.ndz[y + 1] = w.ndz[y]; w.ndx[y + 1] = w.ndx[y]; --y; }
    w.ndd[y + 1] = v; w.ndz[y + 1] = zz; w.ndx[y + 1] = ix;
  }
  w.cnt[0] = k;
  w.cnt[1] = nd;
  w.cnt[2] = nr;
  w.rho[0] = rho;
}

// The deflation rotations applied to the rows of U instead of the columns of Q:
// Q G_0 ... G_{nr-1} U = Q (G_0 (... (G_{nr-1} U))), so Q keeps its block-diagonal
// form and the merge product splits into one product per child.  One thread per column.
__global__ void k_rot_u(int lo, int n, double* U, int ldu, DcWs w, const int* st) {
  if (status_bad(st)) return;
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  double* u = U + GEP_IX(lo, lo + col, ldu);
  for (int q = w.cnt[2] - 1; q >= 0; --q) {
    int a = w.ra[q], b = w.rb[q];
    double x = u[a], y = u[b], c = w.rc[q], s = w.rs[q];
    u[a] = c * x - s * y;
    u[b] = s * x + c * y;
  }
}

// One warp per root j of the secular equation on the k non-deflated poles.
__global__ void __launch_bounds__(256) k_secular(DcWs w, const int* st) {
  if (status_bad(st)) return;
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  int k = w.cnt[0];
  if (j >= k) return;
  const double rho = w.rho[0];
  const double* dd = w.ndd;
  const double* zz = w.ndz;
  int org;
  double lo, hi;
  if (j < k - 1) {
    double gap = dd[j + 1] - dd[j];
    double s = 0.0;
    for (int i = lane; i < k; i += 32) {
      double del = (dd[i] - dd[j]) - 0.5 * gap;
      s += zz[i] * zz[i] / del;
    }
    double fmid = 1.0 + rho * warp_sum(s);
    if (fmid >= 0.0) { org = j; lo = 0.0; hi = 0.5 * gap; }
    else { org = j + 1; lo = -0.5 * gap; hi = 0.0; }
  } else {
    double s = 0.0;
    for (int i = lane; i < k; i += 32) s += zz[i] * zz[i];
    org = j; lo = 0.0; hi = rho * warp_sum(s);
  }
  const double dorg = dd[org];
  const double DL = dd[j] - dorg;                          // left pole (relative)
  const double DR = (j < k - 1) ? dd[j + 1] - dorg : 0.0;  // right pole (relative)
  double tau = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    double pL = 0.0, dpL = 0.0, pR = 0.0, dpR = 0.0;
    for (int i = lane; i < k; i += 32) {  // one reciprocal per pole (the FP64 pipe is the bound)
      double r = 1.0 / ((dd[i] - dorg) - tau);
      double t = zz[i] * zz[i] * r;
      if (i <= j) { pL += t; dpL += t * r; }
      else { pR += t; dpR += t * r; }
    }
    pL = rho * warp_sum(pL);
    dpL = rho * warp_sum(dpL);
    pR = rho * warp_sum(pR);
    dpR = rho * warp_sum(dpR);
    double f = 1.0 + pL + pR;
    if (f == 0.0) break;
    if (f > 0.0) hi = tau; else lo = tau;
    double errf = EPS * (8.0 * (1.0 + fabs(pL) + fabs(pR)) + fabs(tau) * (dpL + dpR));
    if (fabs(f) <= errf) break;
    if (hi - lo <= 4.0 * EPS * fmax(fabs(lo), fabs(hi))) break;
    // two-pole rational model around tau, solved for the step eta
    double a = DL - tau;
    double sL = dpL * a * a, cL = pL - dpL * a;
    double eta = NAN;
    if (j < k - 1) {
      double b = DR - tau;
      double sR = dpR * b * b, cR = pR - dpR * b;
      double C0 = 1.0 + cL + cR;
      double B2 = C0 * (a + b) + sL + sR;
      double C2 = C0 * a * b + sL * b + sR * a;
      if (C0 == 0.0) {
        eta = C2 / B2;
      } else {
        double disc = fmax(B2 * B2 - 4.0 * C0 * C2, 0.0);
        double q = 0.5 * (B2 + copysign(sqrt(disc), B2));
        double e1 = q / C0, e2 = (q != 0.0) ? C2 / q : NAN;
        bool ok1 = (tau + e1 > lo) && (tau + e1 < hi);
        bool ok2 = (tau + e2 > lo) && (tau + e2 < hi);
        if (ok1 && ok2) eta = fabs(e1) < fabs(e2) ? e1 : e2;
        else if (ok1) eta = e1;
        else if (ok2) eta = e2;
      }
    } else {
      double C0 = 1.0 + cL;
      if (C0 > 0.0) eta = a + sL / C0;
    }
    double tn = tau + eta;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (tn == tau) break;
    tau = tn;
  }
  if (lane == 0) {
    w.org[j] = org;
    w.tauR[j] = tau;
    w.lam[j] = dorg + tau;
  }
}

// x <- x 2^-s with |x 2^-s| in [1, 2) (sign kept), e += s; zero and subnormal x are left as
// they are (a zero product stays zero).
__device__ __forceinline__ void renorm_exp(double& x, int& e) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return;
  x = __longlong_as_double((bits & ~(0x7FFll << 52)) | (1023ll << 52));
  e += E - 1023;
}

// Loewner formula: zhat_i^2 = ((lam_i - d_i)/rho) prod_{j != i} (lam_j - d_i)/(d_j - d_i).
__global__ void k_zhat(DcWs w, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int k = w.cnt[0];
  if (i >= k) return;
  const double di = w.ndd[i];
  // numerator and denominator products kept apart (one division at the end); every eighth
  // factor both are brought back to [1, 2) in magnitude, their binary exponents counted in
  // en, ed, so that neither over- nor underflows
  double pn = -((di - w.ndd[w.org[i]]) - w.tauR[i]) / w.rho[0], pd = 1.0;
  int en = 0, ed = 0, c = 0;
  for (int j = 0; j < k; ++j) {
    if (j == i) continue;
    pn *= -((di - w.ndd[w.org[j]]) - w.tauR[j]);
    pd *= w.ndd[j] - di;
    if (++c == 8) {
      c = 0;
      renorm_exp(pn, en);
      renorm_exp(pd, ed);
    }
  }
  const double prod = ldexp(pn / pd, en - ed);
  w.zhat[i] = copysign(sqrt(fmax(prod, 0.0)), w.ndz[i]);
}

// Final ascending order of the merged eigenvalues (roots and deflated values).
__global__ void k_order(int n, DcWs w, const int* st) {
  if (status_bad(st)) return;
  int k = w.cnt[0], nd = w.cnt[1];
  int a = 0, b = 0, o = 0;
  while (a < k && b < nd) {
    if (w.lam[a] <= w.dfv[b]) { w.posr[a] = o; w.newD[o++] = w.lam[a++]; }
    else { w.posd[b] = o; w.newD[o++] = w.dfv[b++]; }
  }
  while (a < k) { w.posr[a] = o; w.newD[o++] = w.lam[a++]; }
  while (b < nd) { w.posd[b] = o; w.newD[o++] = w.dfv[b++]; }
}

// Column pos_root[j] of U: normalised z_hat_i / (d_i - lam_j) at rows ndx[i].
__global__ void __launch_bounds__(256) k_ucols(int lo, double* U, int ldu, DcWs w, const int* st) {
  __shared__ double red[32];
  if (status_bad(st)) return;
  int j = blockIdx.x;
  int k = w.cnt[0];
  if (j >= k) return;
  const double dorg = w.ndd[w.org[j]], tj = w.tauR[j];
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double u = w.zhat[i] / ((w.ndd[i] - dorg) - tj);
    s = fma(u, u, s);
  }
  double inv = 1.0 / sqrt(block_sum(s, red));
  double* col = U + GEP_IX(lo, lo + w.posr[j], ldu);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double u = w.zhat[i] / ((w.ndd[i] - dorg) - tj);
    col[w.ndx[i]] = u * inv;
  }
}

__global__ void k_udefl(int lo, double* U, int ldu, DcWs w, const int* st) {
  if (status_bad(st)) return;
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= w.cnt[1]) return;
  U[GEP_IX(lo + w.dfx[m], lo + w.posd[m], ldu)] = 1.0;
}

__global__ void k_copy_vec(int n, const double* __restrict__ s, double* __restrict__ d, const int* st) {
  if (status_bad(st)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = s[i];
}

DcWs carve(char* base, int M, size_t* used) {
  DcWs w;
  size_t off = 0;
  auto takeD = [&](size_t n) { off = align256(off); double* p = (double*)(base + off); off += n * sizeof(double); return p; };
  auto takeI = [&](size_t n) { off = align256(off); int* p = (int*)(base + off); off += n * sizeof(int); return p; };
  size_t mm = (size_t)M * M, m = (size_t)M;
  w.Qt = takeD(mm); w.U = takeD(mm);
  w.D = takeD(m); w.dd = takeD(m); w.zs = takeD(m); w.dv = takeD(m); w.ndd = takeD(m); w.ndz = takeD(m);
  w.dfv = takeD(m); w.rc = takeD(m); w.rs = takeD(m); w.tauR = takeD(m); w.lam = takeD(m); w.zhat = takeD(m);
  w.newD = takeD(m); w.rho = takeD(4);
  w.ptau = takeD(m); w.pc = takeD(m); w.ps = takeD(m);
  w.perm = takeI(m); w.ndx = takeI(m); w.dfx = takeI(m); w.ra = takeI(m); w.rb = takeI(m); w.org = takeI(m);
  w.posr = takeI(m); w.posd = takeI(m); w.cnt = takeI(8);
  w.nsl = takeI(m); w.prot = takeI(m);
  *used = align256(off);
  return w;
}

}  // namespace

size_t dc_ws_bytes(int M) {
  size_t used = 0;
  carve(nullptr, M, &used);
  return used;
}

int tridiag_eig_dc(gep_handle_t h, int M, const double* d, const double* e, double* wout, double* Z,
                   int ldz, double* ws, size_t ws_bytes, int engine) {
  if (M <= 0) return GEP_OK;
  size_t used = 0;
  DcWs w = carve((char*)ws, M, &used);
  if (ws_bytes < used) return GEP_ERR_ALLOC;
  cudaStream_t s = h->stream;
  const int* stc = h->d_status;
  GEP_CHECK(set_matrix(h, M, M, 0.0, 0.0, Z, ldz));
  k_tear<<<(M + 255) / 256, 256, 0, s>>>(M, d, e, w.dd);
  GEP_CHECK(check_launch(h));
  int nleaf = (M + LEAF - 1) / LEAF;
  k_leaf<<<(nleaf + 3) / 4, 128, 0, s>>>(M, w.dd, e, w.D, Z, ldz, h->d_status);
  GEP_CHECK(check_launch(h));
  for (int half = LEAF; half < M; half *= 2) {
    int width = 2 * half;
    for (int lo = 0; lo < M; lo += width) {
      int mid = lo + half;
      if (mid >= M) break;
      int hi = min(M, lo + width);
      int n = hi - lo;
      k_prep<<<1, 1024, 0, s>>>(lo, mid, hi, e, w.D, Z, ldz, w, stc);
      GEP_CHECK(check_launch(h));
      k_secular<<<(n + 7) / 8, 256, 0, s>>>(w, stc);
      GEP_CHECK(check_launch(h));
      k_zhat<<<(n + 127) / 128, 128, 0, s>>>(w, stc);
      GEP_CHECK(check_launch(h));
      k_order<<<1, 1, 0, s>>>(n, w, stc);
      GEP_CHECK(check_launch(h));
      GEP_CHECK(set_matrix(h, n, n, 0.0, 0.0, w.U + GEP_IX(lo, lo, M), M));
      k_ucols<<<n, 256, 0, s>>>(lo, w.U, M, w, stc);
      GEP_CHECK(check_launch(h));
      k_udefl<<<(n + 255) / 256, 256, 0, s>>>(lo, w.U, M, w, stc);
      GEP_CHECK(check_launch(h));
      k_rot_u<<<(n + 255) / 256, 256, 0, s>>>(lo, n, w.U, M, w, stc);
      GEP_CHECK(check_launch(h));
      // Q = diag(Q1, Q2): one product per child (half the flops of a dense n x n product)
      const int n1 = mid - lo, n2 = hi - mid;
      GEP_CHECK(dgemm(h, 'N', 'N', 'F', n1, n, n1, 1.0, Z + GEP_IX(lo, lo, ldz), ldz, w.U + GEP_IX(lo, lo, M), M,
                      0.0, w.Qt + GEP_IX(lo, lo, M), M, engine));
      GEP_CHECK(dgemm(h, 'N', 'N', 'F', n2, n, n2, 1.0, Z + GEP_IX(mid, mid, ldz), ldz, w.U + GEP_IX(mid, lo, M), M,
                      0.0, w.Qt + GEP_IX(mid, lo, M), M, engine));
      GEP_CHECK(copy_matrix(h, n, n, w.Qt + GEP_IX(lo, lo, M), M, Z + GEP_IX(lo, lo, ldz), ldz));
      k_copy_vec<<<(n + 255) / 256, 256, 0, s>>>(n, w.newD, w.D + lo, stc);
      GEP_CHECK(check_launch(h));
    }
  }
  k_copy_vec<<<(M + 255) / 256, 256, 0, s>>>(M, w.D, wout, stc);
  return check_launch(h);
}

// ---------------------------------------------------------------- T_evo path
namespace {

__global__ void k_gersh(int M, const double* __restrict__ d, const double* __restrict__ e, double* out) {
  __shared__ double red[32];
  double lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < M ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
  }
  double mlo = -block_max(-lo, red);
  double mhi = block_max(hi, red);
  if (threadIdx.x == 0) {
    double span = mhi - mlo;
    out[0] = mlo - 1e-12 * span - 1e-300;
    out[1] = mhi + 1e-12 * span + 1e-300;
  }
}

// Sturm count: eigenvalues of T strictly below x (signs of the LDL^T pivots of T - xI).
__device__ int sturm(int M, const double* __restrict__ d, const double* __restrict__ e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < M; ++i) {
    double off = (i > 0) ? e[i - 1] * e[i - 1] / q : 0.0;
    q = (d[i] - x) - off;
    if (q == 0.0) q = -0x1p-1000;
    cnt += (q < 0.0);
  }
  return cnt;
}

// w[k], k < n: the (k+1)-th smallest eigenvalue of T (order M) by bisection on Sturm counts.
__global__ void k_bisect(int n, int M, const double* __restrict__ d, const double* __restrict__ e,
                         const double* __restrict__ gb, double* __restrict__ w, const int* st) {
  if (status_bad(st)) return;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double a = gb[0], b = gb[1];
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (a + b);
    if (mid <= a || mid >= b) break;
    if (sturm(M, d, e, mid) > k) b = mid; else a = mid;
  }
  w[k] = 0.5 * (a + b);
}

}  // namespace

int tridiag_eig_bisect(gep_handle_t h, int M, const double* d, const double* e, double* w, int n) {
  if (M <= 0) return GEP_OK;
  if (n < 0 || n > M) n = M;  // the n lowest eigenvalues w[0..n)
  if (n == 0) return GEP_OK;
  double* gb = (double*)(h->d_status + 8);  // two doubles of the handle's status block
  k_gersh<<<1, 1024, 0, h->stream>>>(M, d, e, gb);
  GEP_CHECK(check_launch(h));
  k_bisect<<<(n + 127) / 128, 128, 0, h->stream>>>(n, M, d, e, gb, w, h->d_status);
  return check_launch(h);
}

}  // namespace gep
