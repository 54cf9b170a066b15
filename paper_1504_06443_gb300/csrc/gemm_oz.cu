// FP64-accurate matrix product C = alpha op(A) op(B) + beta C on the BF16 tensor
// cores of sm_103a (tcgen05 + TMEM + TMA), by exact splitting of the operands.
//
// Splitting (per K panel): every row i of op(A) is scaled by 2^-e_i with
// max_k |A_ik| < 2^(e_i - 1) and cut into S signed 7-bit digits,
//     A_ik 2^-e_i = sum_s d_s 2^-7s + r,   every d_s in [-64,64],
// (the FP32-grade setting keeps max_k |A_ik| < 2^e_i, its leading digit in [-128,128]),
// each digit an integer held exactly in BF16; likewise every column j of op(B)
// with 2^-f_j.  Then
//     (op(A) op(B))_ij = 2^(e_i+f_j) sum_l 2^-7l L_l,   L_l = sum_{s+t=l} D^A_s D^B_t,
// and only levels l <= LMAX are kept.  With S = 8 planes and LMAX = 9 (36 plane
// products, the FP64 setting) the dropped levels and the digit remainders sit
// near 2^-54 of the row/column scale; S = 3, LMAX = 4 (6 products) is the
// FP32-grade setting of the mixed-precision path.  Each L_l is an integer
// matrix product: with balanced leading digits a digit product is at most 2^12 in
// magnitude and a level holds at most 8 of them (the FP32-grade levels at most
// 2^13 + 2^12 + 2^13), so over a 512-deep K chunk every partial sum stays within 2^24
// and the FP32 accumulation in tensor memory is exact.  After each
// chunk the level sums are drained from TMEM into two 64-bit integer fixed-point
// accumulators per output (levels 2..4 and 5..LMAX); FP64 arithmetic appears only
// once per output element, in the final epilogue.
//
// Kernel: persistent, grid = min(output tiles, SMs); each CTA walks 128 x 64 output
// tiles (its TMA ring and barrier phases continue from one tile to the next), 10 warps:
// warp 0 issues TMA loads of all S digit planes of a 32-deep K step (3-D boxes, 64-byte
// swizzle) into a two-stage ring; warp 1 issues tcgen05.mma (M=128, K=16, N up to 256 covering
// several levels at once: for fixed s the planes B_1..B_{LMAX-s} are contiguous in
// shared memory and their levels are contiguous TMEM columns); warps 2-9 drain
// TMEM (warp w reads lane quarter w%4, column half (w-2)/4).  Every mbarrier wait
// is bounded; on expiry the kernel records GEP_ERR_TIMEOUT in the status block,
// waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "gep_internal.cuh"

namespace gep {
namespace {

constexpr int TM = 128, TN = 64, TK = 32, KCH = 512, STAGES = 2, MAXS = 8;
// warp 0 issues the TMA loads, warp 1 the MMAs; EPI_WARPS warps drain the accumulators
// (four per 32-lane quarter of TMEM, each with CPW of the tile's TN columns): the drain
// stalls the MMAs, and more warps per scheduler hide its TMEM-load and conversion latency
constexpr int EPI_WARPS = 16, CPW = TN / (EPI_WARPS / 4);
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int KP_MAX = 4096;  // K panel per launch (integer accumulators sized for <= 16 chunks)

// ------------------------------------------------------------------ splitting

// Both splitting kernels work on the IEEE bit patterns with integer instructions
// only: the FP64 pipe of this part is far slower than its integer ALUs, and with
// FP64 arithmetic the split would cost more than the tensor-core product it feeds.

// Biased exponent field of |x| (0 for zero / subnormal).
__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// Row scale exponent from the largest biased exponent m of the row: e with max |x| < 2^(e-1)
// when xbit = 1 (for a normal x with biased exponent E, |x| < 2^(E-1022)), so that the
// leading digit lies in [-64, 64] like the others; xbit = 0 (the FP32-grade setting, whose
// few levels stay exact with a leading digit in [-128, 128]) keeps max |x| < 2^e.  0 for an
// all-zero row.
__device__ __forceinline__ int scale_exp(int m, int xbit) { return m ? m - 1022 + xbit : 0; }

// The exponent arrays of the engine hold, per row of op(A) and per column of op(B), the
// largest biased exponent field of the K panel (raw); scale_exp turns it into the scale.
//
// raw[r] = max over the K panel of exp_field(X(r, kk)), X(r,kk) = X[r*sr + kk*sk], for an
// operand whose K is strided (consecutive rows contiguous): block (256 rows, one 128-deep
// slab of K), atomicMax into raw (zero on entry), so that short-and-wide panels spread over
// many CTAs.
__global__ void k_rowexp_slab(int R, int K, const double* __restrict__ X, long long sr, long long sk,
                              int* __restrict__ raw, const int* st) {
  if (status_bad(st)) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int k0 = blockIdx.y * 128, k1 = min(K, k0 + 128);
  int m = 0;
  for (int kk = k0; kk < k1; ++kk) m = max(m, exp_field(X[r * sr + kk * sk]));
  if (m) atomicMax(raw + r, m);
}

// F = round(x 2^(7S - e)) as a signed integer (|F| < 2^(7S)), from the IEEE bits: the
// magnitude is rounded half away from zero (error at most half a unit of the last digit).
// The row's own exponent e keeps the left shift at most 3.
__device__ __forceinline__ long long to_fixed(double x, int e, int S) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0) return 0;
  const unsigned long long m = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1075 + 7 * S - e;
  unsigned long long qv;
  if (sh >= 0) qv = m << sh;
  else if (sh > -54) qv = (m + (1ull << (-sh - 1))) >> (-sh);
  else qv = 0;  // below half a unit of the last digit
  return (bits < 0) ? -(long long)qv : (long long)qv;
}

// 64 in every digit position below the leading one: F + this has base-128 digits
// d_s + 64 in [0, 127] for s >= 2 (d_s in [-64, 63]) and d_1 above them.
template <int S>
__device__ __forceinline__ constexpr long long digit_offset() {
  long long o = 0;
  for (int i = 0; i < S - 1; ++i) o = o * 128 + 64;
  return o;
}

// FP32 bit pattern of the small integer d + bias (|d + bias| <= 256): 1.5 * 2^23 + d is a
// float of the binade [2^23, 2^24) whose last bits are d, and subtracting 1.5 * 2^23 leaves
// d exactly; with at most 9 significant bits its upper half is its BF16 pattern.
__device__ __forceinline__ unsigned f32_bits_of_int(int d, int bias) {
  return (unsigned)__float_as_int(__int_as_float(0x4B400000 + bias + d) - 12582912.0f);
}

// Balanced base-128 digits of the fixed-point integer F (|F| < 2^(7S)): d_S..d_2 in
// [-64, 63] and the leading d_1 (the same digits the peel "d = F mod 128 in [-64, 63],
// F <- (F - d) / 128" gives, from the least significant end).  With the offset above they
// are plain bit fields of Fp = F + offset, so no carries are propagated: d_1 = Fp >> 7(S-1)
// and d_s + 64 = (Fp >> 7(S-s)) & 127 for s >= 2.

// BF16 pair (lo, hi halves) of the digits d' - 64 from p = 0x4300 + d' in each half, d' in
// [0, 128]: 0x4300 + d' is the BF16 pattern of 128 + d' (exponent 2^7, mantissa d'), and
// subtracting 192 leaves d' - 64 exactly, two digits per instruction.
__device__ __forceinline__ unsigned bf16x2_minus192(unsigned p) {
  unsigned r;
  asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(p), "r"(0x43404340u));
  return r;
}

// Digits of 4 consecutive elements x[0..3] of row r (columns kk .. kk+3, all < Kpad;
// columns >= K are zero) written as one 8-byte store per plane.  The leading digit (range
// [-128, 128] in the FP32-grade setting) goes through the FP32 pattern above, paired by byte
// permutes; the others, 7-bit fields d_s + 64 of F + offset, through the BF16 pair trick.
template <int SC>
__device__ __forceinline__ void split4_store_t(const double* x, int kk, int K, int e, size_t base, size_t plane,
                                               unsigned short* __restrict__ out) {
  long long Fp[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) Fp[u] = ((kk + u < K) ? to_fixed(x[u], e, SC) : 0ll) + digit_offset<SC>();
  {
    unsigned f[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) f[u] = f32_bits_of_int((int)(Fp[u] >> (7 * (SC - 1))), 0);
    uint2 w;
    w.x = __byte_perm(f[0], f[1], 0x7632);
    w.y = __byte_perm(f[2], f[3], 0x7632);
    *reinterpret_cast<uint2*>(out + base) = w;
  }
#pragma unroll
  for (int s = 1; s < SC; ++s) {
    const int sh = 7 * (SC - 1 - s);
    unsigned a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = (unsigned)(Fp[u] >> sh) & 127u;
    uint2 w;
    w.x = bf16x2_minus192(0x43004300u + (a[0] | (a[1] << 16)));
    w.y = bf16x2_minus192(0x43004300u + (a[2] | (a[3] << 16)));
    *reinterpret_cast<uint2*>(out + base + (size_t)s * plane) = w;
  }
}

__device__ __forceinline__ void split4_store(const double* x, int kk, int K, int e, int S, size_t base,
                                             size_t plane, unsigned short* __restrict__ out) {
  switch (S) {
    case 8: split4_store_t<8>(x, kk, K, e, base, plane, out); break;
    case 3: split4_store_t<3>(x, kk, K, e, base, plane, out); break;
    case 1: split4_store_t<1>(x, kk, K, e, base, plane, out); break;
    case 2: split4_store_t<2>(x, kk, K, e, base, plane, out); break;
    case 4: split4_store_t<4>(x, kk, K, e, base, plane, out); break;
    case 5: split4_store_t<5>(x, kk, K, e, base, plane, out); break;
    case 6: split4_store_t<6>(x, kk, K, e, base, plane, out); break;
    default: split4_store_t<7>(x, kk, K, e, base, plane, out); break;
  }
}

// Digit planes out[s][r][kk] (bf16, kk contiguous, Kpad columns, zero padding).
// x 2^-e[r] is rounded to the integer F = round(x 2^(7S-e)) (|F| <= 2^(7S-1)), whose
// balanced base-128 digits are peeled off from the least significant end:
// d_S..d_2 in [-64, 63], the leading d_1 in [-64, 64].  Plane s-1 holds d_s.
__global__ void __launch_bounds__(256) k_split(int R, int K, int Kpad, const double* __restrict__ X, long long sr,
                                               long long sk, const int* __restrict__ e, int S, int xbit,
                                               unsigned short* __restrict__ out, const int* st) {
  __shared__ double t[32][33];
  if (status_bad(st)) return;
  int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int q = ty; q < 32; q += 8) {
    int r, kk;
    if (sk == 1) { r = r0 + q; kk = k0 + tx; }
    else { r = r0 + tx; kk = k0 + q; }
    double v = 0.0;
    if (r < R && kk < K) v = X[r * sr + kk * sk];
    if (sk == 1) t[q][tx] = v; else t[tx][q] = v;
  }
  __syncthreads();
  {  // thread: row r0 + (tid >> 3), columns k0 + 4 (tid & 7) .. + 3
    const int q = threadIdx.x >> 3, c4 = (threadIdx.x & 7) * 4;
    const int r = r0 + q;
    if (r < R) {
      double x[4] = {t[q][c4], t[q][c4 + 1], t[q][c4 + 2], t[q][c4 + 3]};
      split4_store(x, k0 + c4, K, scale_exp(e[r], xbit), S, (size_t)r * Kpad + k0 + c4, (size_t)R * Kpad, out);
    }
  }
}

// Exponent pass and digit split in one kernel for an operand whose K runs contiguously
// along each row (sk = 1): one warp per row, lane l taking columns 4 l + 128 i .. + 3; the
// row is read twice (largest exponent, then digits), the second time from cache.
__global__ void __launch_bounds__(256) k_split_rows(int R, int K, int Kpad, const double* __restrict__ X,
                                                    long long sr, int* __restrict__ e_out, int S, int xbit,
                                                    unsigned short* __restrict__ out, const int* st) {
  if (status_bad(st)) return;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= R) return;
  const double* x = X + (size_t)r * sr;
  int m = 0;
  for (int kk = lane; kk < K; kk += 32) m = max(m, exp_field(x[kk]));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = scale_exp(m, xbit);
  if (lane == 0) e_out[r] = m;
  const size_t plane = (size_t)R * Kpad;
  for (int k0 = 4 * lane; k0 < Kpad; k0 += 128) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (k0 + u < K) ? x[k0 + u] : 0.0;
    split4_store(v, k0, K, e, S, (size_t)r * Kpad + k0, plane, out);
  }
}

// The same for few rows (fewer than can fill the GPU one warp per row): one CTA per row,
// the exponent pass reduced over the CTA.
__global__ void __launch_bounds__(256) k_split_row_blk(int R, int K, int Kpad, const double* __restrict__ X,
                                                       long long sr, int* __restrict__ e_out, int S, int xbit,
                                                       unsigned short* __restrict__ out, const int* st) {
  __shared__ int red[8];
  if (status_bad(st)) return;
  const int r = blockIdx.x;
  if (r >= R) return;
  const double* x = X + (size_t)r * sr;
  int m = 0;
  for (int kk = threadIdx.x; kk < K; kk += 256) m = max(m, exp_field(x[kk]));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max(m, red[w]);
  const int e = scale_exp(m, xbit);
  if (threadIdx.x == 0) e_out[r] = m;
  const size_t plane = (size_t)R * Kpad;
  for (int k0 = 4 * threadIdx.x; k0 < Kpad; k0 += 1024) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (k0 + u < K) ? x[k0 + u] : 0.0;
    split4_store(v, k0, K, e, S, (size_t)r * Kpad + k0, plane, out);
  }
}

// Symmetric operand given by its lower triangle (op(A) = A, A(i, kk) = C(max, min)), K
// panel [kb, kb + kc): exponents in two passes (the part of row i left of the diagonal,
// read down the rows; then the part of column i below it, read along the column), and
// digit planes with the same arithmetic as k_split.
__global__ void k_rowexp_sym_row(int R, int kb, int kc, const double* __restrict__ C, long long ldc,
                                 int* __restrict__ raw, const int* st) {
  // block (x: 256 rows, y: 64-deep slab of the panel); raw[r] must start at 0
  if (status_bad(st)) return;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int k0 = kb + blockIdx.y * 64, kend = min(min(r, kb + kc - 1), k0 + 63);
  int m = 0;
  for (int kk = k0; kk <= kend; ++kk) m = max(m, exp_field(C[r + kk * ldc]));
  if (m) atomicMax(raw + r, m);
}

__global__ void k_rowexp_sym_col(int R, int kb, int kc, const double* __restrict__ C, long long ldc,
                                 int* __restrict__ e, const int* st) {
  if (status_bad(st)) return;
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= R) return;
  int m = 0;
  for (int kk = max(r + 1, kb) + lane; kk < kb + kc; kk += 32) m = max(m, exp_field(C[kk + r * ldc]));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    e[r] = max(m, e[r]);
  }
}

__global__ void __launch_bounds__(256) k_split_sym(int R, int K, int Kpad, int kb, const double* __restrict__ C,
                                                   long long ldc, const int* __restrict__ e, int S, int xbit,
                                                   unsigned short* __restrict__ out, const int* st) {
  __shared__ double t[32][33];
  if (status_bad(st)) return;
  int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const bool kfast = r0 + 31 < kb + k0;  // tile strictly above the diagonal: read along columns of C
  for (int q = ty; q < 32; q += 8) {
    int r, kk;
    if (kfast) { r = r0 + q; kk = k0 + tx; }
    else { r = r0 + tx; kk = k0 + q; }
    double v = 0.0;
    if (r < R && kk < K) {
      int g = kb + kk;
      v = r >= g ? C[r + (long long)g * ldc] : C[g + (long long)r * ldc];
    }
    if (kfast) t[q][tx] = v; else t[tx][q] = v;
  }
  __syncthreads();
  {
    const int q = threadIdx.x >> 3, c4 = (threadIdx.x & 7) * 4;
    const int r = r0 + q;
    if (r < R) {
      double x[4] = {t[q][c4], t[q][c4 + 1], t[q][c4 + 2], t[q][c4 + 3]};
      split4_store(x, k0 + c4, K, scale_exp(e[r], xbit), S, (size_t)r * Kpad + k0 + c4, (size_t)R * Kpad, out);
    }
  }
}

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after ~4 s of wall time and records a timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* st) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > 4000000000ull) {
      atomicExch(st + 1, GEP_ERR_TIMEOUT);
      return false;
    }
    if (*(volatile int*)(st + 1) != 0) return false;  // another CTA already gave up
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)map) : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                   // layout: SWIZZLE_64B
  return d;
}

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns of TMEM from taddr; waits for the load
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
  if constexpr (N == 16) tmem_ld16(taddr, v);
  else tmem_ld32(taddr, v);
}

// T = hi * 2^D + lo as a 128-bit two's-complement integer (0 <= D < 64), returned
// as the double nearest to T * 2^adj (round to nearest even), built with integer
// operations only: the FP64 pipe of this part is ~60x slower than its integer ALUs.
// Falls back to FP64 arithmetic when the result would be subnormal or overflow.
__device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int D, int adj) {
  unsigned long long tl, th;
  if (D == 0) {
    tl = (unsigned long long)hi + (unsigned long long)lo;
    unsigned long long c = tl < (unsigned long long)hi ? 1ull : 0ull;
    th = (unsigned long long)(hi >> 63) + (unsigned long long)(lo >> 63) + c;
  } else {
    unsigned long long a = (unsigned long long)hi << D;
    unsigned long long ah = (unsigned long long)(hi >> (64 - D));
    tl = a + (unsigned long long)lo;
    unsigned long long c = tl < a ? 1ull : 0ull;
    th = ah + (unsigned long long)(lo >> 63) + c;
  }
  unsigned long long sign = th >> 63;
  if (sign) {  // magnitude of the 128-bit value
    tl = ~tl + 1ull;
    th = ~th + (tl == 0ull ? 1ull : 0ull);
  }
  if ((th | tl) == 0ull) return 0.0;
  int p;  // position of the leading one
  if (th) p = 127 - __clzll((long long)th);
  else p = 63 - __clzll((long long)tl);
  unsigned long long m;
  if (p <= 52) {
    m = tl << (52 - p);
  } else {
    int sh = p - 52;  // 1 .. 75
    unsigned long long rem_hi, rem_lo, half_hi, half_lo;
    if (sh < 64) {
      m = (tl >> sh) | (sh ? (th << (64 - sh)) : 0ull);
      rem_lo = tl & ((1ull << sh) - 1ull);
      rem_hi = 0ull;
      half_lo = 1ull << (sh - 1);
      half_hi = 0ull;
    } else {
      int s2 = sh - 64;
      m = th >> s2;
      rem_lo = tl;
      rem_hi = s2 ? (th & ((1ull << s2) - 1ull)) : 0ull;
      if (s2 == 0) { half_hi = 0ull; half_lo = 1ull << 63; }
      else { half_hi = 1ull << (s2 - 1); half_lo = 0ull; }
    }
    bool gt = (rem_hi > half_hi) || (rem_hi == half_hi && rem_lo > half_lo);
    bool eq = (rem_hi == half_hi) && (rem_lo == half_lo);
    if (gt || (eq && (m & 1ull))) {
      ++m;
      if (m >> 53) { m >>= 1; ++p; }
    }
  }
  int ex = p + adj + 1023;
  if (ex <= 0 || ex >= 2047) {  // outside the normal range: let FP64 arithmetic handle it
    double v = ldexp((double)(m & ((1ull << 53) - 1ull)), p - 52 + adj);
    return sign ? -v : v;
  }
  unsigned long long bits = (sign << 63) | ((unsigned long long)ex << 52) | (m & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)bits);
}

constexpr int GROUP_M = 8;  // row tiles per group of the tile order (L2 reuse of the A planes)

struct OzArgs {
  int m, n, kpad, S, lmax, lower, xbit;
  int gx, gy, ntiles;  // tile grid gx x gy (128-row x 64-column tiles), in grouped order
  // kr_n > 0: row tile r < kr_n runs only the k-steps [kr_lo[r], kr_hi[r]) of this panel
  // (op(A) is exactly zero elsewhere in its rows); other row tiles run all of them
  int kr_n;
  short kr_lo[OZ_KR_MAX], kr_hi[OZ_KR_MAX];
  const int* ea;
  const int* eb;
  double alpha, beta;
  double* C;
  int ldc;
  int* st;
};

// SC, LC > 0 fix the plane and level counts at compile time (the two settings the
// solver uses): the MMA sequence of a k-step is then straight-line code whose
// descriptors are a per-stage base plus constants.  SC = LC = 0 reads them from p.
template <int SC, int LC>
__global__ void __launch_bounds__(NTHREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, OzArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[2 * STAGES + 3];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int skip;
  __shared__ short kr_lo[OZ_KR_MAX], kr_hi[OZ_KR_MAX];
  // persistent: in wave i CTA b takes tile i G + (b + i) mod G (G = gridDim.x; the last,
  // partial wave unrotated), so a CTA does not meet the same row tile in every wave when G
  // is a multiple of the row-tile count (row tiles may differ in work, see kr_lo / kr_hi);
  // tiles strictly above the diagonal of a lower-triangle product are skipped by every
  // role alike.  Tiles are
  // numbered in groups of GROUP_M row tiles, row fastest inside a group: the tiles that run
  // at the same time cover a near-square block of C (8 rows x ~19 columns on 152 SMs), so
  // their A and B planes are read from DRAM about once and then hit in L2.
  auto tile_rc = [&](int t, int& tm, int& tn) {
    const int per_group = GROUP_M * p.gy;
    const int first = (t / per_group) * GROUP_M;
    const int gm = min(p.gx - first, GROUP_M);
    const int local = t - (first / GROUP_M) * per_group;
    tm = (first + local % gm) * TM;
    tn = (local / gm) * TN;
    return !(p.lower && tm + TM - 1 < tn);
  };
  auto tile_of = [&](int i) {
    const int G = gridDim.x, base = i * G;
    return base + G <= p.ntiles ? base + (int)((blockIdx.x + i) % G) : base + (int)blockIdx.x;
  };
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = SC > 0 ? SC : p.S, LMAX = LC > 0 ? LC : p.lmax;
  const uint32_t a_bytes = (uint32_t)S * TM * TK * 2, b_bytes = (uint32_t)S * TN * TK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[STAGES]);
  const uint32_t bar_accf = smem_u32(&bars[2 * STAGES]), bar_acce = smem_u32(&bars[2 * STAGES + 1]);
  const uint32_t bar_done = smem_u32(&bars[2 * STAGES + 2]);
  const int nsteps = p.kpad / TK;
  const int nlev = LMAX - 1;  // levels 2..LMAX
  // the k-steps [s0, s1) of the tile whose first row is tm (every role takes the same)
  auto tile_steps = [&](int tm, int& s0, int& s1) {
    s0 = 0;
    s1 = nsteps;
    const int r = tm / TM;
    if (r < p.kr_n) {
      s0 = kr_lo[r];
      s1 = kr_hi[r];
    }
  };
  constexpr int SPC = KCH / TK;  // k-steps per exactly accumulated chunk

  if (threadIdx.x == 0) {
    skip = status_bad(p.st) ? 1 : 0;
#pragma unroll
    for (int i = 0; i < OZ_KR_MAX; ++i) {
      kr_lo[i] = p.kr_lo[i];
      kr_hi[i] = p.kr_hi[i];
    }
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_accf, 1);
    mbar_init(bar_acce, EPI_WARPS);
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    prefetch_map(&tmA);
    prefetch_map(&tmB);
  }
  __syncthreads();
  if (skip) return;  // one decision for the whole CTA
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;  // k-steps issued by this CTA over all its tiles
      bool ok = true;
      for (int i = 0, t; ok && (t = tile_of(i)) < p.ntiles; ++i) {
        int tm, tn, s0, s1;
        if (!tile_rc(t, tm, tn)) continue;
        tile_steps(tm, s0, s1);
        for (int step = s0; step < s1 && ok; ++step, ++g) {
          int sidx = g % STAGES;
          uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          ok = mbar_wait(bar_empty + 8 * sidx, ph ^ 1u, p.st);
          if (!ok) break;
          uint32_t dst = smem_u32(smem + (size_t)sidx * stage_bytes);
          mbar_expect_tx(bar_full + 8 * sidx, stage_bytes);
          tma_load_3d(dst, &tmA, step * TK, tm, 0, bar_full + 8 * sidx);
          tma_load_3d(dst + a_bytes, &tmB, step * TK, tn, 0, bar_full + 8 * sidx);
        }
      }
      // make sure every copy this thread started has landed before the CTA retires
      for (int s2 = (g > STAGES ? g - STAGES : 0); s2 < g; ++s2)
        mbar_wait(bar_full + 8 * (s2 % STAGES), (uint32_t)(s2 / STAGES) & 1u, p.st);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int g = 0, gc = 0;  // k-steps and chunks consumed over all tiles
      for (int i = 0, t; ok && (t = tile_of(i)) < p.ntiles; ++i) {
      int tm, tn, s0, s1;
      if (!tile_rc(t, tm, tn)) continue;
      tile_steps(tm, s0, s1);
      const int nch = (s1 - s0 + SPC - 1) / SPC;
      int step = s0;
      for (int c = 0; c < nch && ok; ++c, ++gc) {
        ok = mbar_wait(bar_acce, ((uint32_t)gc & 1u) ^ 1u, p.st);
        if (!ok) break;
        tc_fence_after();
        int send = min(s1, s0 + (c + 1) * SPC);
        for (int sic = 0; step < send; ++step, ++sic, ++g) {
          int sidx = g % STAGES;
          ok = mbar_wait(bar_full + 8 * sidx, (uint32_t)(g / STAGES) & 1u, p.st);
          if (!ok) break;
          tc_fence_after();
          uint32_t abase = smem_u32(smem + (size_t)sidx * stage_bytes);
          const uint64_t a0 = sdesc_sw64(abase), b0 = sdesc_sw64(abase + a_bytes);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
            for (int s = 1; s <= MAXS; ++s) {
              if (s > S) break;
              const int tmax = min(S, LMAX - s);
              if (tmax < 1) break;
              // descriptor start field = byte address / 16: offsets add to it directly
              const uint64_t adesc = a0 + (uint64_t)((((s - 1) * TM * TK * 2) + kk * 32) >> 4);
#pragma unroll
              for (int t0 = 1; t0 <= MAXS; t0 += 4) {
                if (t0 > tmax) break;
                const int nt = min(4, tmax - t0 + 1);
                const uint64_t bdesc = b0 + (uint64_t)((((t0 - 1) * TN * TK * 2) + kk * 32) >> 4);
                const uint32_t col = (uint32_t)(s + t0 - 2) * TN;
                const uint32_t acc = (sic == 0 && kk == 0 && s == 1) ? 0u : 1u;
                umma(tmem + col, adesc, bdesc, idesc_bf16(nt * TN), acc);
              }
            }
          }
          umma_commit(bar_empty + 8 * sidx);  // frees the stage once these MMAs are done
        }
        if (!ok) break;
        umma_commit(bar_accf);
      }
      }
      umma_commit(bar_done);
      mbar_wait(bar_done, 0, p.st);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4).., columns CPW*((w-2)/4)..
    const int q = warp & 3, cg = (warp - 2) >> 2;
    bool ok = true;
    int gc = 0;
    for (int i = 0, t; ok && (t = tile_of(i)) < p.ntiles; ++i) {
    int tm, tn, s0, s1;
    if (!tile_rc(t, tm, tn)) continue;
    tile_steps(tm, s0, s1);
    const int nch = (s1 - s0 + SPC - 1) / SPC;
    const int row = tm + q * 32 + lane;
    long long hi[CPW], lo[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) { hi[j] = 0; lo[j] = 0; }
    for (int c = 0; c < nch; ++c, ++gc) {
      ok = mbar_wait(bar_accf, (uint32_t)gc & 1u, p.st);
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int lv = 0; lv < nlev; ++lv) {
        int l = lv + 2;
        float v[CPW];
        tmem_ld<CPW>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(lv * TN + cg * CPW), v);
        if (l <= 4) {
          int sh = 7 * (4 - l);
#pragma unroll
          for (int j = 0; j < CPW; ++j) hi[j] += (long long)__float2int_rn(v[j]) * (1ll << sh);
        } else {
          int sh = 7 * (LMAX - l);
#pragma unroll
          for (int j = 0; j < CPW; ++j) lo[j] += (long long)__float2int_rn(v[j]) * (1ll << sh);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_acce);
    }
    if (ok && row < p.m) {
      const int ea = scale_exp(p.ea[row], p.xbit);
      const bool two = LMAX >= 5;  // a second (low) accumulator is in use
      const int D = two ? 7 * LMAX - 28 : 0;
      const int base_adj = ea - (two ? 7 * LMAX : 28);
      const double alpha = p.alpha, beta = p.beta;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        int col = tn + cg * CPW + j;
        if (col >= p.n || (p.lower && row < col)) continue;
        double v = fixed_to_double(hi[j], two ? lo[j] : 0ll, D, base_adj + scale_exp(p.eb[col], p.xbit));
        double* cp = p.C + (size_t)row + (size_t)col * p.ldc;
        double out = (alpha == 1.0) ? v : (alpha == -1.0 ? -v : alpha * v);
        if (beta != 0.0) out = fma(beta, *cp, out);
        *cp = out;
      }
    }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

size_t smem_bytes_for(int S) { return (size_t)STAGES * S * (TM + TN) * TK * 2 + 1024; }

// cuTensorMapEncodeTiled is a driver-API call; it is resolved at run time through the
// runtime's entry-point query so the library does not link libcuda directly (it then
// loads on machines without a GPU driver, e.g. for symbol checks).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// plane_rows: rows between consecutive planes (0: rows), for a view of the last rows of
// a plane set
int encode_map(CUtensorMap* map, const void* base, int kpad, int rows, int S, int box_rows, int plane_rows = 0) {
  if (plane_rows <= 0) plane_rows = rows;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * (cuuint64_t)plane_rows};
  cuuint32_t box[3] = {(cuuint32_t)TK, (cuuint32_t)box_rows, (cuuint32_t)S};
  cuuint32_t estr[3] = {1, 1, 1};
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    fprintf(stderr, "gep: cuTensorMapEncodeTiled not available from the driver\n");
    return GEP_ERR_CUDA;
  }
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "gep: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
    return GEP_ERR_CUDA;
  }
  return GEP_OK;
}

}  // namespace

namespace {

// Exponent pass and split of an operand with contiguous K: one warp per row, or one CTA per
// row when the rows are too few to fill the GPU that way.
int split_rows(gep_handle_t h, int R, int K, int Kpad, const double* X, long long sr, int* e, int S, int xbit,
               unsigned short* out) {
  if (R < 16 * h->sm_count)
    k_split_row_blk<<<R, 256, 0, h->stream>>>(R, K, Kpad, X, sr, e, S, xbit, out, h->d_status);
  else
    k_split_rows<<<(R * 32 + 255) / 256, 256, 0, h->stream>>>(R, K, Kpad, X, sr, e, S, xbit, out, h->d_status);
  return check_launch(h);
}

// Product-kernel launch for one K panel (kc deep, planes padded to a.kpad): dynamic shared
// memory attribute, optional per-launch timing, template dispatch on the plane/level counts.
int oz_launch(gep_handle_t h, const CUtensorMap& mA, const CUtensorMap& mB, const OzArgs& a, int kc) {
  static unsigned long long attr_devices = 0;
  if (first_use_on_device(attr_devices)) {
    cudaFuncSetAttribute(k_oz_gemm<8, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_for(MAXS));
    cudaFuncSetAttribute(k_oz_gemm<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_for(MAXS));
    cudaFuncSetAttribute(k_oz_gemm<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_for(MAXS));
  }
  const int S = a.S, levels = a.lmax;
  dim3 grid(a.ntiles < h->sm_count ? a.ntiles : h->sm_count);  // persistent CTAs
  int slot = -1;
  if (h->prof_on) {
    if (h->prof_used < h->prof_cap) {
      slot = h->prof_used++;
      cudaEventRecord(h->prof_ev[2 * slot], h->stream);
      int npairs = 0;
      for (int s = 1; s <= S; ++s) npairs += max(0, min(S, levels - s));
      double f = 2.0 * a.m * a.n * (double)kc * (a.lower ? 0.5 : 1.0);
      h->prof_f64eq[slot] = f;
      h->prof_flops[slot] = f * npairs;
      h->prof_mnk[3 * slot] = a.m;
      h->prof_mnk[3 * slot + 1] = a.n;
      h->prof_mnk[3 * slot + 2] = kc;
    } else {
      h->prof_skipped++;
    }
  }
  if (S == 8 && levels == 9) k_oz_gemm<8, 9><<<grid, NTHREADS, smem_bytes_for(S), h->stream>>>(mA, mB, a);
  else if (S == 3 && levels == 4) k_oz_gemm<3, 4><<<grid, NTHREADS, smem_bytes_for(S), h->stream>>>(mA, mB, a);
  else k_oz_gemm<0, 0><<<grid, NTHREADS, smem_bytes_for(S), h->stream>>>(mA, mB, a);
  GEP_CHECK(check_launch(h));
  if (slot >= 0) cudaEventRecord(h->prof_ev[2 * slot + 1], h->stream);
  return GEP_OK;
}

void oz_args_init(OzArgs& a, int m, int n, int kpad, int S, int levels, int lower, int xbit, const int* ea,
                  const int* eb, double alpha, double beta, double* C, int ldc, int* st) {
  a.m = m; a.n = n; a.kpad = kpad; a.S = S; a.lmax = levels; a.lower = lower; a.xbit = xbit;
  a.ea = ea; a.eb = eb; a.alpha = alpha; a.beta = beta; a.C = C; a.ldc = ldc; a.st = st;
  a.gx = (m + TM - 1) / TM;
  a.gy = (n + TN - 1) / TN;
  a.ntiles = a.gx * a.gy;
  a.kr_n = 0;
  for (int r = 0; r < OZ_KR_MAX; ++r) a.kr_lo[r] = a.kr_hi[r] = 0;
}

}  // namespace

size_t oz_sym_planes_bytes(int m, int levels) {
  if (m <= 0) return 0;
  const size_t S = (size_t)(levels - 1), np = (m + OZ_SYM_KP - 1) / OZ_SYM_KP;
  const size_t kpad_last = (size_t)((m - (np - 1) * OZ_SYM_KP + TK - 1) / TK) * TK;
  return align256((size_t)2 * S * m * ((np - 1) * OZ_SYM_KP + kpad_last)) + align256(sizeof(int) * np * m) + 256;
}

int oz_split_sym(gep_handle_t h, int m, const double* A, int lda, int levels, void* buf, size_t bytes,
                 OzSymPlanes* P) {
  const int S = levels - 1;
  if (S < 1 || S > MAXS || m <= 0) return GEP_ERR_UNSUPPORTED;
  if (buf == nullptr || bytes < oz_sym_planes_bytes(m, levels)) return GEP_ERR_ALLOC;
  const int np = (m + OZ_SYM_KP - 1) / OZ_SYM_KP;
  const int kpad_last = (m - (np - 1) * OZ_SYM_KP + TK - 1) / TK * TK;
  P->planes = (unsigned short*)buf;
  P->ea = (int*)((char*)buf + align256((size_t)2 * S * m * ((size_t)(np - 1) * OZ_SYM_KP + kpad_last)));
  P->m = m;
  P->levels = levels;
  const int xbit = levels >= 8 ? 1 : 0;
  GEP_CUDA(cudaMemsetAsync(P->ea, 0, sizeof(int) * (size_t)np * m, h->stream));
  for (int p = 0; p < np; ++p) {
    const int kb = p * OZ_SYM_KP, kc = min(OZ_SYM_KP, m - kb), kpad = (kc + TK - 1) / TK * TK;
    int* ea = P->ea + (size_t)p * m;
    unsigned short* As = P->planes + (size_t)p * S * m * OZ_SYM_KP;
    k_rowexp_sym_row<<<dim3((m + 255) / 256, (kc + 63) / 64), 256, 0, h->stream>>>(m, kb, kc, A, lda, ea,
                                                                                  h->d_status);
    GEP_CHECK(check_launch(h));
    k_rowexp_sym_col<<<(m * 32 + 255) / 256, 256, 0, h->stream>>>(m, kb, kc, A, lda, ea, h->d_status);
    GEP_CHECK(check_launch(h));
    k_split_sym<<<dim3(kpad / 32, (m + 31) / 32), 256, 0, h->stream>>>(m, kc, kpad, kb, A, lda, ea, S, xbit, As,
                                                                       h->d_status);
    GEP_CHECK(check_launch(h));
  }
  return GEP_OK;
}

int dgemm_oz_sym_planes(gep_handle_t h, const OzSymPlanes& P, int row0, int n, double alpha, const double* B,
                        int ldb, double beta, double* C, int ldc) {
  const int m = P.m - row0, S = P.levels - 1, K = P.m;
  if (row0 < 0 || m <= 0 || n <= 0) return GEP_OK;
  if (S < 1 || S > MAXS || !P.planes) return GEP_ERR_UNSUPPORTED;
  const int kp_max = K < OZ_SYM_KP ? K : OZ_SYM_KP;
  const int kpad_max = (kp_max + TK - 1) / TK * TK;
  const size_t need = align256((size_t)2 * S * n * kpad_max) + align256(sizeof(int) * (size_t)n) + 256;
  if (h->eng_ws == nullptr || h->eng_bytes < need) return GEP_ERR_ALLOC;
  unsigned short* Bs = (unsigned short*)h->eng_ws;
  int* eb = (int*)(h->eng_ws + align256((size_t)2 * S * n * kpad_max));
  const int xbit = P.levels >= 8 ? 1 : 0;
  const int np = (K + OZ_SYM_KP - 1) / OZ_SYM_KP;
  for (int p = 0; p < np; ++p) {
    const int kb = p * OZ_SYM_KP, kc = min(OZ_SYM_KP, K - kb), kpad = (kc + TK - 1) / TK * TK;
    const unsigned short* As = P.planes + (size_t)p * S * P.m * OZ_SYM_KP;
    GEP_CHECK(split_rows(h, n, kc, kpad, B + kb, ldb, eb, S, xbit, Bs));
    CUtensorMap mA, mB;
    GEP_CHECK(encode_map(&mA, As + (size_t)row0 * kpad, kpad, m, S, TM, P.m));  // rows row0.. of each plane
    GEP_CHECK(encode_map(&mB, Bs, kpad, n, S, TN));
    OzArgs a;
    oz_args_init(a, m, n, kpad, S, P.levels, 0, xbit, P.ea + (size_t)p * P.m + row0, eb, alpha,
                 p == 0 ? beta : 1.0, C, ldc, h->d_status);
    GEP_CHECK(oz_launch(h, mA, mB, a, kc));
  }
  return GEP_OK;
}

size_t oz_workspace_bytes(int m, int n, int k) {
  int kp = k < KP_MAX ? k : KP_MAX;
  size_t kpad = (size_t)((kp + TK - 1) / TK) * TK;
  return align256((size_t)MAXS * (m + n) * kpad * 2) + align256((size_t)(m + n) * 4) + 1024;
}

int dgemm_oz(gep_handle_t h, char ta, char tb, char uplo, int m, int n, int k, double alpha, const double* A,
             int lda, const double* B, int ldb, double beta, double* C, int ldc, int levels, const OzKRange* kr) {
  if (m <= 0 || n <= 0) return GEP_OK;
  if (k <= 0 || alpha == 0.0) return dgemm_f64(h, ta, tb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  const int S = levels - 1;
  if (S < 1 || S > MAXS) return GEP_ERR_UNSUPPORTED;
  bool TA = (ta == 'T' || ta == 't'), TB = (tb == 'T' || tb == 't');
  const bool SA = (ta == 'S' || ta == 's');  // A symmetric (m x m, k = m), lower triangle stored
  if (SA && k != m) return GEP_ERR_UNSUPPORTED;
  // view of op(A) as rows i, depth kk: element at A[i*sra + kk*ska]
  long long sra = TA ? lda : 1, ska = TA ? 1 : lda;
  // view of op(B)^T as rows j, depth kk
  long long srb = TB ? 1 : ldb, skb = TB ? ldb : 1;
  // scratch
  size_t cap = h->eng_bytes;
  char* base = h->eng_ws;
  size_t per_k = (size_t)S * (m + n) * 2;
  size_t fixed = align256((size_t)(m + n) * 4) + 1024;
  if (base == nullptr || cap <= fixed) return GEP_ERR_ALLOC;
  long long kp_fit = (long long)((cap - fixed) / per_k) / TK * TK;
  int KP = (int)(kp_fit < KP_MAX ? kp_fit : KP_MAX);
  if (KP < TK) return GEP_ERR_ALLOC;
  int lower = (uplo == 'L' || uplo == 'l');
  // balanced leading digits where a level may hold up to 8 digit products (see the top)
  const int xbit = levels >= 8 ? 1 : 0;
  for (int kb = 0; kb < k; kb += KP) {
    int kc = min(KP, k - kb);
    int kpad = (kc + TK - 1) / TK * TK;
    char* p = base;
    unsigned short* As = (unsigned short*)p;  // bf16 bit patterns
    p += align256((size_t)S * m * kpad * 2);
    unsigned short* Bs = (unsigned short*)p;
    p += align256((size_t)S * n * kpad * 2);
    int* ea = (int*)p;
    int* eb = ea + m;
    const double* Ap = A + (size_t)kb * ska;
    const double* Bp = B + (size_t)kb * skb;
    // operands whose K is contiguous take the fused exponent-and-split kernel; the others
    // (K strided) an exponent pass down the rows, then the tile-transposing split
    if (SA) {
      GEP_CUDA(cudaMemsetAsync(ea, 0, sizeof(int) * (size_t)m, h->stream));
      k_rowexp_sym_row<<<dim3((m + 255) / 256, (kc + 63) / 64), 256, 0, h->stream>>>(m, kb, kc, A, lda, ea,
                                                                                    h->d_status);
      GEP_CHECK(check_launch(h));
      k_rowexp_sym_col<<<(m * 32 + 255) / 256, 256, 0, h->stream>>>(m, kb, kc, A, lda, ea, h->d_status);
      GEP_CHECK(check_launch(h));
      k_split_sym<<<dim3(kpad / 32, (m + 31) / 32), 256, 0, h->stream>>>(m, kc, kpad, kb, A, lda, ea, S, xbit, As,
                                                                         h->d_status);
      GEP_CHECK(check_launch(h));
    } else if (ska == 1) {
      GEP_CHECK(split_rows(h, m, kc, kpad, Ap, sra, ea, S, xbit, As));
    } else {
      GEP_CUDA(cudaMemsetAsync(ea, 0, sizeof(int) * (size_t)m, h->stream));
      k_rowexp_slab<<<dim3((m + 255) / 256, (kc + 127) / 128), 256, 0, h->stream>>>(m, kc, Ap, sra, ska, ea,
                                                                                   h->d_status);
      GEP_CHECK(check_launch(h));
      k_split<<<dim3(kpad / 32, (m + 31) / 32), 256, 0, h->stream>>>(m, kc, kpad, Ap, sra, ska, ea, S, xbit, As,
                                                                     h->d_status);
      GEP_CHECK(check_launch(h));
    }
    if (skb == 1) {
      GEP_CHECK(split_rows(h, n, kc, kpad, Bp, srb, eb, S, xbit, Bs));
    } else {
      GEP_CUDA(cudaMemsetAsync(eb, 0, sizeof(int) * (size_t)n, h->stream));
      k_rowexp_slab<<<dim3((n + 255) / 256, (kc + 127) / 128), 256, 0, h->stream>>>(n, kc, Bp, srb, skb, eb,
                                                                                   h->d_status);
      GEP_CHECK(check_launch(h));
      k_split<<<dim3(kpad / 32, (n + 31) / 32), 256, 0, h->stream>>>(n, kc, kpad, Bp, srb, skb, eb, S, xbit, Bs,
                                                                     h->d_status);
      GEP_CHECK(check_launch(h));
    }
    CUtensorMap mA, mB;
    GEP_CHECK(encode_map(&mA, As, kpad, m, S, TM));
    GEP_CHECK(encode_map(&mB, Bs, kpad, n, S, TN));
    OzArgs a;
    oz_args_init(a, m, n, kpad, S, levels, lower, xbit, ea, eb, alpha, (kb == 0) ? beta : 1.0, C, ldc, h->d_status);
    if (kr && kr->n > 0) {  // this panel's k-steps of each listed row tile
      a.kr_n = min(min(kr->n, OZ_KR_MAX), a.gx);
      for (int r = 0; r < a.kr_n; ++r) {
        int lo = max(kr->lo[r] - kb, 0), hi = min(kr->hi[r] - kb, kc);
        if (hi <= lo) lo = hi = 0;
        a.kr_lo[r] = (short)(lo / TK);
        a.kr_hi[r] = (short)((hi + TK - 1) / TK);
      }
    }
    GEP_CHECK(oz_launch(h, mA, mB, a, kc));
  }
  return GEP_OK;
}

}  // namespace gep

// ---------------------------------------------------------------------------
// Allocation-free variant of the split-BF16 product (gep_dgemm_emulated_noalloc).
//
// Some callers cannot call cudaMalloc: a framework that owns the whole device-memory
// budget through its own pool, or a latency-critical loop that must not let a
// library grow its footprint or hit the allocator mid-run.  This entry point needs
// neither a handle nor a workspace: the digit planes, row/column exponents and the
// status word live in the fixed device array below, which every GPU that loads this
// library holds until the process exits.  The product is the same as gep_dgemm with
// GEP_PREC_FP64_EMULATED; only the K-panel length differs (it is chosen to fit the
// array), so results agree to rounding.
static __device__ __align__(256) unsigned char g_noalloc_scratch[64u << 20];

namespace {
constexpr size_t kNoallocBytes = 64u << 20;
constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};
int g_noalloc_ready[kNoallocMaxDevices] = {};

// The call returns before the GPU runs the product, so a device-side failure (a bounded
// wait of the product kernel that gave up and set the status word) cannot be a return
// code.  This kernel runs last in the call and, only when the status word is set, fills
// every element of C that the call writes with NaN: the failure then shows in C itself.
__global__ void k_noalloc_poison(int m, int n, double* __restrict__ C, int ldc, int lower, const int* st) {
  if (st[0] == 0 && st[1] == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const long long total = (long long)m * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (lower && i < j) continue;
    C[(size_t)i + (size_t)j * ldc] = nan;
  }
}
}  // namespace

extern "C" int gep_dgemm_emulated_noalloc(char transa, char transb, char uplo, int m, int n, int k, double alpha,
                                          const double* A, int lda, const double* B, int ldb, double beta, double* C,
                                          int ldc, void* stream) {
  bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (uplo != 'F' && uplo != 'f' && uplo != 'L' && uplo != 'l') return -3;
  if (m < 0) return -4;
  if (n < 0) return -5;
  if (k < 0) return -6;
  if (lda < (ta ? (k > 1 ? k : 1) : (m > 1 ? m : 1))) return -9;
  if (ldb < (tb ? (n > 1 ? n : 1) : (k > 1 ? k : 1))) return -11;
  if (ldc < (m > 1 ? m : 1)) return -14;
  // The array holds a 256-byte status block, then the planes of a K panel of at least
  // 32 (8 planes x 2 bytes x (m + n) x 32) and the (m + n) exponents.
  const size_t status_bytes = 256;
  const size_t need_min = status_bytes + gep::align256((size_t)8 * 2 * ((size_t)m + n) * 32) +
                          gep::align256((size_t)4 * ((size_t)m + n)) + 1024;
  if (need_min > kNoallocBytes) return GEP_ERR_TOO_LARGE;
  if (m == 0 || n == 0) return GEP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return GEP_ERR_CUDA;
  if (!g_noalloc_ready[dev]) {  // first call on this device (the device is current here)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fprintf(stderr, "gep: cudaGetSymbolAddress of the no-allocation scratch failed: %s\n", cudaGetErrorString(e));
      return GEP_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
    g_noalloc_ready[dev] = 1;
  }
  char* base = (char*)g_noalloc_ptr[dev];
  gep_handle_s h;  // stack-only view: no events, no split-K buffer, no allocation
  h.stream = (cudaStream_t)stream;
  h.d_status = (int*)base;
  h.eng_ws = base + status_bytes;
  h.eng_bytes = kNoallocBytes - status_bytes;
  cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, dev);
  // the status words must start at zero; the digit planes are fully rewritten per panel
  if (cudaMemsetAsync(h.d_status, 0, status_bytes, h.stream) != cudaSuccess) return GEP_ERR_CUDA;
  int rc = gep::dgemm_oz(&h, transa, transb, uplo, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 9);
  h.magic = 0;
  if (rc != GEP_OK) return rc;
  const long long total = (long long)m * n;
  const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
  k_noalloc_poison<<<blocks, 256, 0, h.stream>>>(m, n, C, ldc, (uplo == 'L' || uplo == 'l') ? 1 : 0, h.d_status);
  if (cudaGetLastError() != cudaSuccess) return GEP_ERR_CUDA;
  return GEP_OK;
}
