// Complex128 GEMM at FP64 accuracy on the BF16 tensor cores (tcgen05 kind::f16) by exact operand
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications", Numerical
// Algorithms 59, 2012).
//
// C = alpha op(A) op(B) + beta D. The complex product is taken as three real products (3M):
//     T0 = Ar Br,  T1 = Ai Bi,  T2 = (Ar + Ai)(Br + Bi),   AB = (T0 - T1) + i (T2 - T0 - T1);
// for K <= 192 as four, Re = Ar Br + (-Ai) Bi and Im = Ar Bi + Ai Br, each accumulated whole in one
// set of tensor-memory accumulators (two drains per output tile instead of three: there the drain,
// not the tensor pipe, bounds the kernel).
// Each real product X Y (X: M x K, Y: K x N) is evaluated exactly up to a bounded truncation:
//   * row i of the three real operands Ar, Ai, Ar + Ai gets one power of two sigma_i > 2 max |.|
//     over the row (columns j of Br, Bi, Br + Bi likewise tau_j), so that the three products are
//     integers in the same units;
//   * X_ik / sigma_i, a number in (-1/2, 1/2), is truncated towards zero to 56 fraction bits and
//     written in balanced base-128 digits: X_ik = sigma_i (sum_s t_s 2^(-7 s) + delta), |delta| <
//     2^-56, with OZ_S = 8 digits t_s in [-64, 63] (the leading one in [-65, 65]), each exact in
//     BF16; the slicing works on the FP64 bit pattern (integer operations only: GB300's FP64 pipe is
//     slow); the fixed-point value of Ar + Ai is the exact sum of those of Ar and Ai (|delta| <
//     2^-55), so T2 - T0 - T1 is exactly the cross term of the truncated operands;
//   * a digit product t_s u_r has |t_s u_r| <= 65^2 and carries the weight 2^(-7 (s + r)); the
//     products of one diagonal d = s + r (d <= OZ_S + 1: 36 pairs) accumulate in one FP32 tensor-
//     memory accumulator, exact for 384 K values (at most 8 pairs: 8 * 65^2 * 384 < 2^24); every
//     384 K values the 8 accumulators are drained exactly, on the integer pipe (GB300's FP64 pipe
//     would otherwise bound the kernel), and added to or subtracted from the two 96-bit integers
//     X 2^63 = H 2^32 + L (int64 H, uint32 L; diagonal d carries the weight 2^(63 - 7 d)) of the
//     complex result's real and imaginary parts (Re = T0 - T1, Im = T2 - T0 - T1, exact);
//   * for alpha = +-2^a and beta = 0 or +-2^b (real: every product of the solver) the chunks are
//     added with alpha's sign, beta D / 2^a rounded to the sums' units (2^-63 sigma_i tau_j) is
//     added after the last one, and once per output element each part is rounded to the nearest
//     double on the integer pipe (the scales are powers of two): C = alpha X + beta D with one
//     rounding. Other
//     alpha, beta (and D beyond 2^31 sigma_i tau_j, a zero scale, a non-finite D) round X and apply
//     alpha and beta D in FP64; C is written once;
//   * per K value and real product the error is below 2^-54.5 sigma_i tau_j: 2^-56 from the
//     truncations (|X_ik| < sigma_i / 2) and 2^-55.18 from the dropped diagonals d >= 10
//     (7 * 64^2 * 2^-70 for d = 10, less beyond); the real part carries two such errors, the
//     imaginary part three.
// Pass 1 (k_oz_pack) computes the scales and the slice images: per K step of 16, a 128 x 16 block of
// op(A) (all 8 slices, 32 KB) and a 32 x 16 block of op(B)^T (8 KB) in the K-major core-matrix
// layout the MMA reads, for each of the three real operands (re, im, re + im), reading each complex
// element once per pass and writing 16-byte runs.
// Pass 2 (k_gemm_oz), persistent, one CTA per SM over the items (energy, 128 x 32 output tile):
// warp 0 streams the slice blocks of the three real products one after another through a 5-stage
// ring (cp.async.bulk, mbarrier transaction counts); warp 1 issues the 36 digit products of each K
// step as 8 MMAs of N = 32..256 (for each A digit, the B digit planes it pairs with are contiguous
// along N and their column blocks are the diagonal accumulators it feeds) into one of two sets of 8
// diagonal accumulators (2 x 256 TMEM columns, so the drain of one chunk overlaps the MMAs of the
// next); warps 2-17 drain them every 24 K steps (8 columns of exact complex state per thread) and
// write each output once (read-modify-write by the owning thread, so C may alias D). Every mbarrier
// wait is bounded; on expiry the kernel raises the flag, waits (bounded) for its own copies, frees
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace hsc {
namespace {

constexpr int OZ_S = 8;                  // slices per operand
constexpr int OZ_BITS = 7;               // bits per slice
constexpr int OZ_FRAC = OZ_S * OZ_BITS;  // fraction bits kept (56)
constexpr int OZ_ND = OZ_S;              // accumulated diagonals d = 2 .. OZ_S + 1
constexpr int OZ_BM = 128, OZ_BN = 32, OZ_BK = 16;
constexpr int OZ_ABLK = OZ_S * OZ_BM * OZ_BK;   // bf16 values of one A block (all slices)
constexpr int OZ_BBLK = OZ_S * OZ_BN * OZ_BK;
constexpr int OZ_STAGES = 5;
constexpr int OZ_DRAIN = 24;             // K steps per drain (384 K values)
constexpr int OZ_M4_KS = 12;             // K steps up to which a product takes four real products:
                                         // Re and Im each accumulated whole (2 x 192 K values)
constexpr int OZ_TMAX = 65;              // largest |digit|
constexpr int OZ_ACC = OZ_ND * OZ_BN;     // TMEM columns of one set of accumulators
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr int OZ_NBUF = 2 * OZ_ACC <= (int)OZ_TMEM_COLS ? 2 : 1;   // sets (2: drain overlaps MMAs)
constexpr unsigned long long OZ_WAIT_NS = 2000000000ull;
constexpr int OZ_DRAIN_WARPS = 16;     // four per TMEM lane quadrant
constexpr int OZ_DCOLS = OZ_BN / (OZ_DRAIN_WARPS / 4);   // columns of exact state per drain thread
constexpr int OZ_THREADS = 64 + 32 * OZ_DRAIN_WARPS;
constexpr int OZP_THREADS = 256;
constexpr int OZ_EG = 2;                 // output columns per group of epilogue loads

static_assert(OZ_NBUF * OZ_ACC <= (int)OZ_TMEM_COLS, "accumulators exceed tensor memory");
static_assert((long long)OZ_S * OZ_TMAX * OZ_TMAX * OZ_DRAIN * OZ_BK < (1ll << 24), "FP32 accumulation not exact");
static_assert(OZ_ND == 8 && OZ_BITS == 7, "the drain's diagonal weights assume 8 diagonals of 7 bits");

__device__ __forceinline__ uint32_t oz_su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long oz_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, unsigned long long limit = OZ_WAIT_NS) {
  const unsigned long long t0 = oz_timer();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (oz_timer() - t0 > limit) return false;
  }
}

// The double nearest to (H 2^32 + L) 2^es (H 2^32 + L: a signed 96-bit integer), built on the
// integer pipe: normalise by the leading bit, round to 53 bits (ties away from zero), place the
// exponent. Falls back to FP64 arithmetic when the result would leave the normal range.
__device__ __forceinline__ double oz_fix_to_double(long long H, unsigned int L, int es) {
  if (H == 0 && L == 0u) return 0.0;
  const bool neg = H < 0;
  unsigned long long mh = (unsigned long long)H;
  unsigned int ml = L;
  if (neg) {   // two's complement of the 96-bit value
    ml = ~L + 1u;
    mh = ~mh + (ml == 0u ? 1ull : 0ull);
  }
  unsigned long long top;   // the 64 bits below and including the leading one
  int lead;                 // position of the leading one in the 96-bit magnitude
  if (mh != 0ull) {
    const int lz = __clzll((long long)mh);
    top = lz == 0 ? mh : ((mh << lz) | (lz <= 32 ? (((unsigned long long)ml << lz) >> 32)
                                                 : ((unsigned long long)ml << (lz - 32))));
    lead = 95 - lz;
  } else {
    const int lz = __clz((int)ml);
    top = (unsigned long long)ml << (32 + lz);
    lead = 31 - lz;
  }
  unsigned long long m = (top >> 11) + ((top >> 10) & 1ull);   // 53 bits, rounded
  int ex = lead + es;
  if (m >> 53) { m >>= 1; ++ex; }
  const int biased = ex + 1023;
  if (biased < 1 || biased > 2046)   // not representable as a normal double: the slow, exact way
    return ldexp(fma((double)L, 0x1p-32, (double)H), es + 32);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                          ((unsigned long long)biased << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// x = +-2^k exactly (x normal): k and the sign
__device__ __forceinline__ bool oz_pow2(double x, int& k, bool& neg) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF || (bits & 0xFFFFFFFFFFFFFull) != 0ull) return false;
  k = ex - 1023;
  neg = (bits >> 63) != 0ull;
  return true;
}

// (-1)^neg d / 2^es rounded to the nearest integer (ties away from zero), as the 96-bit H 2^32 + L;
// false for a d that is not finite or whose value does not fit in 94 bits
__device__ __forceinline__ bool oz_double_to_fix(double d, int es, bool neg, long long& H, unsigned int& L) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0x7FF) return false;
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (ex) m |= 1ull << 52;
  if (m == 0ull) { H = 0; L = 0u; return true; }
  const int sh = (ex ? ex : 1) - 1075 - es;   // d = m 2^(sh + es)
  if (sh > 41) return false;
  long long h;
  unsigned int l;
  if (sh >= 32) {
    h = (long long)(m << (sh - 32));
    l = 0u;
  } else if (sh >= 0) {
    h = (long long)(m >> (32 - sh));
    l = (unsigned int)(m << sh);
  } else if (sh > -54) {
    const unsigned long long v = (m + (1ull << (-sh - 1))) >> (-sh);
    h = (long long)(v >> 32);
    l = (unsigned int)v;
  } else {
    h = 0;
    l = 0u;
  }
  if (neg != ((bits >> 63) != 0ull)) {   // two's complement of the 96-bit value
    l = ~l + 1u;
    h = ~h + (l == 0u ? 1 : 0);
  }
  H = h;
  L = l;
  return true;
}

// element (r, k) of a rows x 16 K-major BF16 block: core matrices of 8 rows x 16 B (8 values); the
// two K-adjacent core matrices are 128 B apart, adjacent 8-row groups 256 B apart
__device__ __forceinline__ int oz_cidx(int r, int k) {
  return (((r >> 3) * 2 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);   // no swizzle, version 1
}

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// two FP32 values as one word of two BF16 (round to nearest even; a in the low half)
__device__ __forceinline__ uint32_t oz_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ int oz_expo(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// One CTA per (problem, side, tile): side A = 128 rows of op(A), side B = 64 rows of op(B)^T
// (columns of op(B)), all three real operands (re, im, re + im) from one read of each complex
// element per pass. A thread task is (row, run of 8 consecutive k): its slices of one plane are 16
// contiguous bytes of the core-matrix layout, written as one 16-byte store. Layout per problem and
// energy (BF16 values):
//   A images at pa: [v][tile_m][kstep][slice][128 x 16],  B images at pb: [v][tile_n][kstep][slice][64 x 16];
//   scales (doubles) at sa: [v][tiles_m * 128],  at sb: [v][tiles_n * 64].
template <int OPA, int OPB>
__global__ void __launch_bounds__(OZP_THREADS) k_oz_pack(GemmArgs g, uint16_t* slices, int64_t slice_es,
                                                         double* scales, int64_t scale_es) {
  const int e = blockIdx.y;
  const int blk = blockIdx.x;
  int lo = 0, hi = g.nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.probs[mid].pack_start <= blk) lo = mid;
    else hi = mid - 1;
  }
  const GemmProb P = g.probs[lo];
  int tile = blk - P.pack_start;
  const bool isA = tile < P.tiles_m;
  if (!isA) tile -= P.tiles_m;
  const int rows = isA ? OZ_BM : OZ_BN;
  const int row0 = tile * rows;
  const int nrow = isA ? P.M : P.N;
  const int K = P.K, ks = P.ksteps;
  // products of up to OZ_M4_KS K steps take four real products: no Ar + Ai operand
  const bool m4 = ks <= OZ_M4_KS;
  const int nv = m4 ? 2 : 3;
  const c64* X = reinterpret_cast<const c64*>(isA ? g.A : g.B) + e * (isA ? g.a_es : g.b_es) + (isA ? P.a : P.b);
  const int ld = isA ? P.lda : P.ldb;
  // row r of op(A) (or of op(B)^T) is contiguous in memory for op(A) in {N, C} and op(B) in {T, H}
  const bool krun = isA ? (OPA == OP_N || OPA == OP_C) : (OPB == OP_T || OPB == OP_H);
  const bool conj = isA ? (OPA == OP_C || OPA == OP_H) : (OPB == OP_C || OPB == OP_H);
  auto load = [&](int r, int k) -> c64 {   // element (r, k) after the op's conjugation, 0 outside
    if (row0 + r >= nrow || k >= K) return make_double2(0.0, 0.0);
    c64 x = krun ? X[(int64_t)(row0 + r) * ld + k] : X[(int64_t)k * ld + row0 + r];
    if (conj) x.y = -x.y;
    return x;
  };
  const int64_t blkv = isA ? OZ_ABLK : OZ_BBLK;
  const int64_t vstride = (int64_t)(isA ? P.tiles_m : P.tiles_n) * ks * blkv;   // between real operands
  uint16_t* dst = slices + e * slice_es + (isA ? P.pa + (int64_t)tile * ks * OZ_ABLK : P.pb + (int64_t)tile * ks * OZ_BBLK);
  double* sc = scales + e * scale_es + (isA ? P.sa : P.sb) + row0;
  const int64_t sstride = (int64_t)(isA ? P.tiles_m * OZ_BM : P.tiles_n * OZ_BN);
  __shared__ int s_e[3][OZ_BM];
  const int tid = threadIdx.x;
  for (int r = tid; r < 3 * OZ_BM; r += OZP_THREADS) s_e[r / OZ_BM][r % OZ_BM] = 0;
  __syncthreads();
  const int ngrp = ks * (OZ_BK / 8);        // runs of 8 k per row
  const int ntask = rows * ngrp;            // lanes run over rows: coalesced for either orientation
  // pass 1: largest biased exponent per row and real operand (0 for a row of zeros)
  for (int t = tid; t < ntask; t += OZP_THREADS) {
    const int r = t % rows, k0 = (t / rows) * 8;
    if (row0 + r >= nrow || k0 >= K) continue;
    int e0 = 0, e1 = 0, e2 = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const c64 x = load(r, k0 + q);
      e0 = max(e0, oz_expo(x.x));
      e1 = max(e1, oz_expo(x.y));
      if (!m4) e2 = max(e2, oz_expo(x.x + x.y));
    }
    // one scale per row for all three real operands, so that their products are exact integers in
    // the same units and the complex result can be combined before any rounding
    const int em = max(e0, max(e1, e2));
    if (em) atomicMax(&s_e[0][r], em);
  }
  __syncthreads();
  // sigma = 2^(E - 1021) > 2 |x| for every x of the row with biased exponent <= E
  for (int i = tid; i < 3 * rows; i += OZP_THREADS) {
    const int v = i / rows, r = i % rows;
    sc[v * sstride + r] = s_e[0][r] > 0 ? ldexp(1.0, s_e[0][r] - 1021) : 0.0;
  }
  // pass 2: slices, 8 consecutive k of one row per task
  for (int t = tid; t < ntask; t += OZP_THREADS) {
    const int r = t % rows, k0 = (t / rows) * 8;
    c64 x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = load(r, k0 + q);
    uint16_t* o = dst + (int64_t)(k0 / OZ_BK) * blkv + oz_cidx(r, k0 % OZ_BK);
    // the fixed-point values of re and im; that of re + im is their exact sum, so that the three
    // real operands satisfy A2 = A0 + A1 exactly (|A0 + A1| < 2^55 + 2: the row's scale covers
    // re + im, and each truncation is below one unit)
    long long m01[2][8];
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double val = v == 0 ? x[q].x : x[q].y;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(val);
        const int ex = (int)((bits >> 52) & 0x7FF);
        // floor(|x| / sigma * 2^56) < 2^55: |x| = mant 2^(ex - 1075), sigma = 2^(E - 1021), so the
        // 53-bit significand moves right by E - ex + 52 - 56 + 2 (a left shift of at most 2)
        const int shift = s_e[0][r] - ex + (52 - OZ_FRAC + 2);
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const long long mag = (ex > 0 && shift < 64) ? (long long)(shift >= 0 ? mant >> shift : mant << (-shift)) : 0ll;
        m01[v][q] = (bits >> 63) ? -mag : mag;
      }
#pragma unroll
    for (int v = 0; v < nv; ++v) {
      long long m[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) m[q] = v < 2 ? m01[v][q] : m01[0][q] + m01[1][q];
      // balanced base-128 digits, least significant first: t = ((m + 64) mod 128) - 64, m = (m - t) / 128,
      // in 32-bit halves: the low 28 bits m mod 2^28 give digits 7..4 and a carry (0 or 1) into
      // the high part floor(m / 2^28) (|.| < 2^27), which gives digits 3..1 and the leading digit.
      // A digit t becomes FP32 through the bit pattern of 1.5 2^23 + t (unit spacing there: exact
      // for |t| < 2^22), and two of them become one word of two BF16 (exact: |t| <= 65 has 7 bits).
      uint32_t wd[OZ_S][4];   // slice sl, k pair p: the BF16 digits of k0 + 2p and k0 + 2p + 1
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float f[2][OZ_S];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long mq = m[2 * p + h];
          int lo = (int)(mq & ((1ll << 28) - 1));
          int hi = (int)(mq >> 28);
#pragma unroll
          for (int sl = OZ_S - 1; sl >= OZ_S - 4; --sl) {
            const int t = ((lo + 64) & 127) - 64;
            f[h][sl] = __int_as_float(0x4B400000 + t) - 12582912.0f;
            lo = (lo - t) >> 7;   // exact: lo - t is a multiple of 128
          }
          hi += lo;
#pragma unroll
          for (int sl = OZ_S - 5; sl > 0; --sl) {
            const int t = ((hi + 64) & 127) - 64;
            f[h][sl] = __int_as_float(0x4B400000 + t) - 12582912.0f;
            hi = (hi - t) >> 7;
          }
          f[h][0] = __int_as_float(0x4B400000 + hi) - 12582912.0f;   // the leading digit, |t| <= 65
        }
#pragma unroll
        for (int sl = 0; sl < OZ_S; ++sl) wd[sl][p] = oz_bf16x2(f[0][sl], f[1][sl]);
      }
#pragma unroll
      for (int sl = 0; sl < OZ_S; ++sl)
        *reinterpret_cast<uint4*>(o + v * vstride + sl * (rows * OZ_BK)) = make_uint4(wd[sl][0], wd[sl][1], wd[sl][2], wd[sl][3]);
    }
  }
}

struct __align__(128) OzSmem {
  uint16_t a[OZ_STAGES][OZ_ABLK];
  uint16_t b[OZ_STAGES][OZ_BBLK];
  unsigned long long full[OZ_STAGES];
  unsigned long long empty[OZ_STAGES];
  unsigned long long acc_full[2];    // MMA -> drain: a chunk of K steps is in accumulator set b
  unsigned long long acc_empty[2];   // drain -> MMA: set b read
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void oz_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void oz_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// Persistent: each CTA takes the items (energy, output tile) idx = blockIdx.x, blockIdx.x + gridDim.x,
// ... in turn, with its stage ring, accumulator hand-off and barrier phases running on across items.
// The producer therefore streams the next item's slice blocks while the drain warps finish the
// current one, and the next item's MMAs start as soon as the accumulators are read, overlapping the
// current item's epilogue (read-modify-write of C).
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_gemm_oz(GemmArgs g, const uint16_t* slices, int64_t slice_es, const double* scales, int64_t scale_es,
          int* flag, int n_items) {
  extern __shared__ unsigned char smem_raw[];
  OzSmem& sm = *reinterpret_cast<OzSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // item idx: energy idx / total_tiles, tile idx % total_tiles of problem P (binary search on the
  // problems' first tiles)
  struct Item {
    GemmProb P;
    int e, tm, tn, ks, nchunk, m4, nch, nst;
  };
  auto item = [&](int idx) {
    Item it;
    it.e = idx / g.total_tiles;
    const int tile = idx - it.e * g.total_tiles;
    int lo = 0, hi = g.nprob - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (g.probs[mid].tile_start <= tile) lo = mid;
      else hi = mid - 1;
    }
    it.P = g.probs[lo];
    const int t = tile - it.P.tile_start;
    it.tm = t / it.P.tiles_n;
    it.tn = t % it.P.tiles_n;
    it.ks = it.P.ksteps;
    it.nchunk = (it.ks + OZ_DRAIN - 1) / OZ_DRAIN;   // per real product
    // K <= 192: four real products, Re = ArBr + (-Ai)Bi and Im = ArBi + AiBr accumulated in one
    // chunk each (2 drains per tile instead of 3); larger K: three (3M), a chunk per 384 K values
    it.m4 = it.ks > 0 && it.ks <= OZ_M4_KS;
    it.nch = it.m4 ? 2 : 3 * it.nchunk;
    it.nst = it.m4 ? 4 * it.ks : 3 * it.ks;
    return it;
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz_su32(&sm.tmem)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&sm.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&sm.empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&sm.acc_full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oz_su32(&sm.acc_empty[b])), "r"(OZ_DRAIN_WARPS));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    sm.abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  // kind::f16 with BF16 A and B, FP32 D, both K-major, M = 128, N = 64 q (q = 1..4 digit planes of B)
  const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BM >> 4) << 24);
  auto idesc_n = [&](int q) { return idesc0 | ((uint32_t)((q * OZ_BN) >> 3) << 17); };
  constexpr uint32_t ABYTES = OZ_ABLK * 2, BBYTES = OZ_BBLK * 2;
  volatile int* abort_flag = &sm.abort;

  if (warp == 0) {
    if (lane == 0) {   // producer: per item, the K steps of the three real products in sequence
      int sg = 0;      // stages issued so far (all items)
      bool ok = true;
      for (int idx = blockIdx.x; idx < n_items && ok; idx += gridDim.x) {
        const Item it = item(idx);
        const uint16_t* sl = slices + it.e * slice_es;
        for (int s = 0; s < it.nst; ++s, ++sg) {
          const int st = sg % OZ_STAGES;
          if (sg >= OZ_STAGES && !oz_wait(oz_su32(&sm.empty[st]), (uint32_t)((sg / OZ_STAGES - 1) & 1))) {
            atomicExch(flag, 3);
            *abort_flag = 1;
            ok = false;
            break;
          }
          // operand pair of the stage: 3M (v, v); four products (re, re), (im, im), (re, im), (im, re)
          const int q = s / it.ks, kk = s % it.ks;
          const int va = it.m4 ? (q & 1) : q, vb = it.m4 ? (q == 1 || q == 2) : q;
          const uint16_t* pa = sl + it.P.pa + (((int64_t)va * it.P.tiles_m + it.tm) * it.ks + kk) * OZ_ABLK;
          const uint16_t* pb = sl + it.P.pb + (((int64_t)vb * it.P.tiles_n + it.tn) * it.ks + kk) * OZ_BBLK;
          const uint32_t fb = oz_su32(&sm.full[st]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(ABYTES + BBYTES)
                       : "memory");
          oz_bulk(oz_su32(&sm.a[st][0]), pa, ABYTES, fb);
          oz_bulk(oz_su32(&sm.b[st][0]), pb, BBYTES, fb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      int sg = 0, cg = 0;   // stages consumed, chunks issued (all items)
      bool ok = true;
      for (int idx = blockIdx.x; idx < n_items && ok; idx += gridDim.x) {
        const Item it = item(idx);
        for (int c = 0; c < it.nch && ok; ++c, ++cg) {
          const int ab = cg % OZ_NBUF;   // accumulator set of this chunk; its previous use was cg - OZ_NBUF
          if (cg >= OZ_NBUF && !oz_wait(oz_su32(&sm.acc_empty[ab]), (uint32_t)((cg / OZ_NBUF - 1) & 1))) {
            atomicExch(flag, 3);
            *abort_flag = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int v = c / it.nchunk, cc = c % it.nchunk;
          const int s0 = it.m4 ? 2 * c * it.ks : v * it.ks + cc * OZ_DRAIN;
          const int s1 = it.m4 ? s0 + 2 * it.ks : v * it.ks + min(it.ks, (cc + 1) * OZ_DRAIN);
          for (int s = s0; s < s1; ++s, ++sg) {
            const int st = sg % OZ_STAGES;
            if (!oz_wait(oz_su32(&sm.full[st]), (uint32_t)((sg / OZ_STAGES) & 1))) {
              atomicExch(flag, 3);
              *abort_flag = 1;
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = oz_su32(&sm.a[st][0]), b0 = oz_su32(&sm.b[st][0]);
            // The B digit planes r = 1..8 lie one after another along N (32 rows each, the same core-
            // matrix strides), so A digit s times planes 1..(9 - s) is one MMA of N = 32 (9 - s) <= 256:
            // its column block r lands in the accumulator of diagonal s + r, which starts at TMEM
            // column 32 (s + r - 2). 8 MMAs per K step instead of 36, the same products.
            // The product (-Ai) Bi of Re takes the instruction descriptor's negate-A bit (BF16
            // negation is exact).
            const uint32_t neg = (it.m4 && c == 0 && s >= s0 + it.ks) ? (1u << 13) : 0u;
            for (int si = 0; si < OZ_S; ++si) {
              // the first MMA of a chunk (si = 0) covers every diagonal and starts the accumulation
              const uint32_t acc = (s > s0 || si > 0) ? 1u : 0u;
              oz_mma(tmem + ab * OZ_ACC + si * OZ_BN, oz_desc(a0 + si * (OZ_BM * OZ_BK * 2)), oz_desc(b0),
                     idesc_n(OZ_S - si) | neg, acc);
            }
            oz_commit(oz_su32(&sm.empty[st]));
          }
          oz_commit(oz_su32(&sm.acc_full[ab]));   // also releases the drain warps after an abort
        }
      }
    }
  } else {   // warps 2..: drain, TMEM lane quadrant = warp % 4, column part = (warp - 2) / 4
    const int quad = warp & 3, part = (warp - 2) >> 2;
    // Integer epilogue when alpha = +-2^ka and beta = 0 or +-2^kb (real; every product of the solver):
    // the sums hold alpha X / 2^ka (chunks added with alpha's sign), beta D / 2^ka is added to them
    // in their units (rounded to 2^-63 sigma_i tau_j) after the last chunk, and the output is one
    // rounding of the whole expression, on the integer pipe.
    int ka = 0, kb = 0;
    bool aneg = false, bneg = false;
    const bool iep = g.ai == 0.0 && g.bi == 0.0 && oz_pow2(g.ar, ka, aneg) &&
                     (g.br == 0.0 || oz_pow2(g.br, kb, bneg));
    const bool xneg = iep && aneg;
    int cg = 0;   // chunks drained (all items)
    bool ok = true;
    for (int idx = blockIdx.x; idx < n_items && ok; idx += gridDim.x) {
      const Item it = item(idx);
      const GemmProb& P = it.P;
      const int e = it.e;
      const int row = it.tm * OZ_BM + quad * 32 + lane;
      c64* C = reinterpret_cast<c64*>(g.C) + e * g.c_es + P.c;
      const c64* D = g.D ? reinterpret_cast<const c64*>(g.D) + e * g.d_es + P.d : nullptr;
      const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0) && !(row >= P.zr0 && row < P.zr1);
      const int col0 = it.tn * OZ_BN + part * OZ_DCOLS;
      const bool in_row = row < P.M;
      const int last = it.nch - 1;
      if (it.ks == 0 && in_row) {   // C = beta D
        for (int j = 0; j < OZ_DCOLS && col0 + j < P.N; ++j) {
          c64 o = make_double2(0.0, 0.0);
          if (use_d) {
            const c64 dv = D[(int64_t)row * P.ldd + col0 + j];
            o = make_double2(g.br * dv.x - g.bi * dv.y, g.br * dv.y + g.bi * dv.x);
          }
          C[(int64_t)row * P.ldc + col0 + j] = o;
        }
      }
      // exact running sums of the complex result, Re = T0 - T1 and Im = T2 - T0 - T1 (3M): the three
      // real operands of a row (and of a column) share one power-of-two scale, so the digit products
      // of the three real products are integers in the same units. Each sum is the 96-bit integer
      // H 2^32 + L (int64 H, uint32 L); the products contribute |H| < 3 nchunk 2^42 and beta D at
      // most 2^62 (larger D takes the FP64 path).
      long long Hr[OZ_DCOLS], Hi[OZ_DCOLS];
      unsigned int Lr[OZ_DCOLS], Li[OZ_DCOLS];
#pragma unroll
      for (int j = 0; j < OZ_DCOLS; ++j) { Hr[j] = 0; Hi[j] = 0; Lr[j] = 0u; Li[j] = 0u; }
      for (int c = 0; c < it.nch; ++c, ++cg) {
        const int ab = cg % OZ_NBUF;
        bool got = oz_wait(oz_su32(&sm.acc_full[ab]), (uint32_t)((cg / OZ_NBUF) & 1));
        got = __all_sync(0xffffffffu, got);   // warp-uniform before the .sync.aligned TMEM loads
        if (!got) {
          if (lane == 0) atomicExch(flag, 3);
          ok = false;
          break;
        }
        if (__any_sync(0xffffffffu, *abort_flag != 0)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (c == last && in_row) {   // the epilogue's operands into L1 while the last chunk drains
          const c64* dp = use_d ? D + (int64_t)row * P.ldd + col0 : nullptr;
          const double* sp = scales + e * scale_es + P.sb + col0;
          asm volatile("prefetch.global.L1 [%0];" ::"l"(scales + e * scale_es + P.sa + row));
          asm volatile("prefetch.global.L1 [%0];" ::"l"(sp));
          asm volatile("prefetch.global.L1 [%0];" ::"l"(sp + OZ_DCOLS - 1));
          if (dp) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(dp));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(dp + OZ_DCOLS - 1));
          }
        }
        // real product v of the chunk: T0 adds to Re and subtracts from Im, T1 subtracts from both,
        // T2 adds to Im (each chunk value negated first for a negative alpha on the integer path)
        const int v = it.m4 ? 3 + c : c / it.nchunk;   // 3M products 0..2; four products: Re 3, Im 4
#pragma unroll
        for (int c0 = 0; c0 < OZ_DCOLS; c0 += 2) {
          // all 8 diagonals of 2 columns behind one wait
          uint32_t r[OZ_ND][2];
          const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + ab * OZ_ACC + part * OZ_DCOLS + c0;
#pragma unroll
          for (int dg = 0; dg < OZ_ND; ++dg)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                         : "=r"(r[dg][0]), "=r"(r[dg][1])
                         : "r"(ta + dg * OZ_BN));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            // weight of accumulator dg (diagonal dg + 2) in X 2^63: 2^(49 - 7 dg); the chunk is
            // Hc 2^32 + Lc with b = sum_{dg >= 3} v_dg 2^(49 - 7 dg) (|b| < 2^52.3) split at bit 32
            int x[OZ_ND];
#pragma unroll
            for (int dg = 0; dg < OZ_ND; ++dg) x[dg] = __float2int_rn(__uint_as_float(r[dg][j]));   // exact
            const long long b = (long long)x[3] * (1ll << 28) + (long long)x[4] * (1ll << 21) +
                                (long long)x[5] * (1ll << 14) + (long long)(x[6] * 128 + x[7]);
            unsigned int lc = (unsigned int)b;
            long long hc = (long long)x[0] * (1ll << 17) + (long long)x[1] * (1ll << 10) +
                           (long long)x[2] * (1ll << 3) + (b >> 32);
            if (xneg) {   // alpha < 0: the chunk's value negated (96-bit two's complement)
              hc = -hc - (lc != 0u ? 1 : 0);
              lc = 0u - lc;
            }
            const int q = c0 + j;
            if (v == 0 || v == 3) {   // Re += T0, Re += the four-product Re
              const unsigned int ln = Lr[q] + lc;
              Hr[q] += hc + (ln < lc ? 1 : 0);
              Lr[q] = ln;
            } else if (v == 1) {      // Re -= T1
              const unsigned int ln = Lr[q] - lc;
              Hr[q] -= hc + (Lr[q] < lc ? 1 : 0);
              Lr[q] = ln;
            }
            if (v == 2 || v == 4) {   // Im += T2, Im += the four-product Im
              const unsigned int ln = Li[q] + lc;
              Hi[q] += hc + (ln < lc ? 1 : 0);
              Li[q] = ln;
            } else if (v <= 1) {      // Im -= T0, Im -= T1
              const unsigned int ln = Li[q] - lc;
              Hi[q] -= hc + (Li[q] < lc ? 1 : 0);
              Li[q] = ln;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_su32(&sm.acc_empty[ab])) : "memory");
        if (c == last && in_row) {   // the result, rounded once per part
          c64* crow = C + (int64_t)row * P.ldc + col0;
          const c64* drow = use_d ? D + (int64_t)row * P.ldd + col0 : nullptr;
          // units of the sums of column j: 2^es, es = (row exponent - 1023 - 63) + (column exponent -
          // 1023) (+ ka); a zero scale (an all-zero row or column) makes the product 0 and the element
          // takes the FP64 path, as do a D beyond 2^31 sigma_i tau_j and a non-finite D
          const int er2 = oz_expo(scales[e * scale_es + P.sa + row]);
          const double* scn = scales + e * scale_es + P.sb + col0;
          // in groups of 4 columns, every load of a group before any store: the compiler must assume
          // that C aliases D and the scales, so loads interleaved with the stores would be one
          // memory round trip per column
#pragma unroll
          for (int j0 = 0; j0 < OZ_DCOLS; j0 += OZ_EG) {
            int ecs[OZ_EG];
            c64 dvs[OZ_EG];
#pragma unroll
            for (int q = 0; q < OZ_EG; ++q) {
              const bool in = col0 + j0 + q < P.N;
              ecs[q] = in ? oz_expo(scn[j0 + q]) : 0;
              dvs[q] = (in && use_d) ? drow[j0 + q] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int q = 0; q < OZ_EG; ++q) {
              const int j = j0 + q;
              if (col0 + j >= P.N) continue;
              const int es = er2 - 1023 - 63 + ecs[q] - 1023 + (iep ? ka : 0);
              bool f = !iep || er2 == 0 || ecs[q] == 0;
              if (!f && use_d) {   // fold beta D / 2^ka into the sums
                long long h0, h1;
                unsigned int l0, l1;
                f = !oz_double_to_fix(dvs[q].x, es - kb, bneg, h0, l0) ||
                    !oz_double_to_fix(dvs[q].y, es - kb, bneg, h1, l1);
                if (!f) {
                  unsigned int ln = Lr[j] + l0;
                  Hr[j] += h0 + (ln < l0 ? 1 : 0);
                  Lr[j] = ln;
                  ln = Li[j] + l1;
                  Hi[j] += h1 + (ln < l1 ? 1 : 0);
                  Li[j] = ln;
                }
              }
              const double xr = oz_fix_to_double(Hr[j], Lr[j], es), xi = oz_fix_to_double(Hi[j], Li[j], es);
              c64 o = make_double2(xr, xi);
              if (f) {
                const bool real_ab = g.ai == 0.0 && g.bi == 0.0;
                if (!iep) o = real_ab ? make_double2(g.ar * xr, g.ar * xi)
                                      : make_double2(g.ar * xr - g.ai * xi, g.ar * xi + g.ai * xr);
                if (use_d) {
                  const c64 d = dvs[q];
                  if (real_ab) {
                    o.x = fma(g.br, d.x, o.x);
                    o.y = fma(g.br, d.y, o.y);
                  } else {
                    o.x += g.br * d.x - g.bi * d.y;
                    o.y += g.br * d.y + g.bi * d.x;
                  }
                }
              }
              crow[j] = o;
            }
          }
        }
      }
    }
  }
  // copies still in flight after an abort: wait (bounded) for the stages the producer armed
  if (tid == 0 && *abort_flag)
    for (int s = 0; s < OZ_STAGES; ++s) oz_wait(oz_su32(&sm.full[s]), 0u, 100000000ull);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

}  // namespace

void oz_layout(GemmProb& p, int& pack_blocks, int& tiles, int64_t& slice_vals, int64_t& scale_vals) {
  p.tiles_m = (p.M + OZ_BM - 1) / OZ_BM;
  p.tiles_n = (p.N + OZ_BN - 1) / OZ_BN;
  p.ksteps = (p.K + OZ_BK - 1) / OZ_BK;
  p.tile_start = tiles;
  tiles += p.tiles_m * p.tiles_n;
  p.pack_start = pack_blocks;
  pack_blocks += p.ksteps > 0 ? p.tiles_m + p.tiles_n : 0;
  p.pa = slice_vals;
  p.pb = slice_vals + 3LL * p.tiles_m * p.ksteps * OZ_ABLK;
  slice_vals = p.pb + 3LL * p.tiles_n * p.ksteps * OZ_BBLK;
  p.sa = scale_vals;
  p.sb = scale_vals + 3LL * p.tiles_m * OZ_BM;
  scale_vals = p.sb + 3LL * p.tiles_n * OZ_BN;
}

cudaError_t gemm_oz(const GemmArgs& g, int n_energy, uint16_t* slices, int64_t slice_es, double* scales,
                    int64_t scale_es, int* flag, cudaStream_t s) {
  if (g.total_tiles <= 0 || n_energy <= 0) return cudaSuccess;
  if (g.pack_blocks > 0) {
    dim3 pgrid(g.pack_blocks, n_energy);
#define HSC_OZ_CASE(a, b)                                                                       \
    if (g.opa == a && g.opb == b)                                                               \
      k_oz_pack<a, b><<<pgrid, OZP_THREADS, 0, s>>>(g, slices, slice_es, scales, scale_es); else
    HSC_OZ_CASE(OP_N, OP_N)
    HSC_OZ_CASE(OP_T, OP_N)
    HSC_OZ_CASE(OP_N, OP_T)
    HSC_OZ_CASE(OP_N, OP_C)
    HSC_OZ_CASE(OP_N, OP_H)
    return cudaErrorInvalidValue;
#undef HSC_OZ_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t sm = sizeof(OzSmem) + 128;
  cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  static int sms[64] = {0};   // SM count per device (one resident CTA per SM: all of TMEM, ~200 KB)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  const long long items = (long long)g.total_tiles * n_energy;
  if (items > 0x7fffffffll) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(items, std::max(sms[dev], 1));
  k_gemm_oz<<<grid, OZ_THREADS, sm, s>>>(g, slices, slice_es, scales, scale_es, flag, (int)items);
  return cudaGetLastError();
}

}  // namespace hsc
