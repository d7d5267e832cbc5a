// Grouped complex GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) with split
// precision: C = alpha op(A) op(B) + beta D, operands stored as complex128 in HBM.
//
// Each 128x128 output tile keeps two FP32 accumulators (Re, Im) in tensor memory (TMEM, 256
// columns). Operand tiles (128 x 16 complex) are read from HBM, split into TF32 hi/lo parts
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) for the real and imaginary planes and written to
// shared memory in the K-major core-matrix layout the MMA reads. One thread issues, per 8-wide K
// slice, the 3xTF32 products of the four real products of the complex product
//     Re += Ar Br - Ai Bi,   Im += Ar Bi + Ai Br,   X Y ~ Xhi Yhi + Xhi Ylo + Xlo Yhi
// (12 MMAs; the minus sign comes from the instruction descriptor's negate-A bit). Shared-memory
// buffers form a ring; the next tile is converted while the tensor core works on the
// current one (tcgen05.commit -> mbarrier): warps 0-3 stage the A tile and warps 4-7 the B tile,
// the next tile's global loads are in flight in registers while the current one is converted, and a
// 3-stage shared-memory ring lets the tensor core run two steps behind. Every mbarrier wait is
// bounded: on expiry the kernel
// raises a flag, waits (bounded) for its own MMAs, frees TMEM and returns.
//
// These are the Schur-update and downward block products of Algorithms 1-2 in the mixed-precision
// mode (FP32 accumulation), used below the top levels of the tree.
#include <cstdint>

#include "common.cuh"

namespace hsc {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 16, TC_THREADS = 256, NSTAGE = 3;
constexpr int PLANE = TBM * TBK;               // tf32 words per plane buffer (128 x 16)
constexpr uint32_t TMEM_COLS = 256;            // Re accumulator cols [0,128), Im [128,256)
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s bound on any mbarrier wait

struct __align__(128) TcSmem {
  uint32_t a[NSTAGE][4][PLANE];   // [stage][Re_hi, Re_lo, Im_hi, Im_lo]
  uint32_t b[NSTAGE][4][PLANE];
  unsigned long long mbar[NSTAGE];
  uint32_t tmem;
  int abort;
  int issued;   // MMA groups committed (steps)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi, lo representable in TF32 (lo rounded again by the tensor core)
__device__ __forceinline__ void split(double x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(static_cast<float>(x));
  lo = to_tf32(static_cast<float>(x - static_cast<double>(__uint_as_float(hi))));
}

// element (r, k) of a 128 x 16 K-major tile: 8x(16 B) core matrices, K-adjacent ones 128 B apart,
// row-group-adjacent ones 512 B apart
__device__ __forceinline__ int cidx(int r, int k) {
  return (((r >> 3) * (TBK / 4) + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 512;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);   // no swizzle, version 1
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns = WAIT_NS) {
  const unsigned long long t0 = gtimer();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ int find_prob_tc(const GemmProb* probs, int nprob, int tile) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_start <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int OPA, int OPB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc(GemmArgs g, int* flag) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = blockIdx.y;
  const GemmProb P = g.probs[find_prob_tc(g.probs, g.nprob, blockIdx.x)];
  const int t = blockIdx.x - P.tile_start;
  const int m0 = (t / P.tiles_n) * TBM, n0 = (t % P.tiles_n) * TBN;
  const c64* A = reinterpret_cast<const c64*>(g.A) + e * g.a_es + P.a;
  const c64* B = reinterpret_cast<const c64*>(g.B) + e * g.b_es + P.b;
  c64* C = reinterpret_cast<c64*>(g.C) + e * g.c_es + P.c;
  const c64* D = g.D ? reinterpret_cast<const c64*>(g.D) + e * g.d_es + P.d : nullptr;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sm.abort = 0;
    sm.issued = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                         ((uint32_t)(TBM >> 4) << 24);
  const uint32_t idesc_nega = idesc | (1u << 13);

  // warps 0-3 stage row r of the A tile, warps 4-7 row r of the (K-major) B tile
  const bool isA = tid < 128;
  const int r = tid & 127;
  const int grow = isA ? m0 + r : n0 + r;
  const bool row_ok = isA ? grow < P.M : grow < P.N;
  auto fetch = [&](int s, c64* v) {
    const int k0 = s * TBK;
#pragma unroll
    for (int k = 0; k < TBK; ++k) {
      const int gk = k0 + k;
      c64 x = make_double2(0.0, 0.0);
      if (row_ok && gk < P.K) {
        if (isA)
          x = (OPA == OP_N || OPA == OP_C) ? A[(int64_t)grow * P.lda + gk] : A[(int64_t)gk * P.lda + grow];
        else
          x = (OPB == OP_N || OPB == OP_C) ? B[(int64_t)gk * P.ldb + grow] : B[(int64_t)grow * P.ldb + gk];
      }
      v[k] = x;
    }
  };
  const bool conj = isA ? (OPA == OP_C || OPA == OP_H) : (OPB == OP_C || OPB == OP_H);

  const int nk = (P.K + TBK - 1) / TBK;
  c64 cur[TBK], nxt[TBK];
  if (nk > 0) fetch(0, cur);
  bool ok = true;
  for (int s = 0; s < nk; ++s) {
    const int st = s % NSTAGE;
    if (s + 1 < nk) fetch(s + 1, nxt);   // in flight while this step is converted and multiplied
    if (s >= NSTAGE) {   // stage st was last read by the MMAs of step s - NSTAGE
      if (!mbar_wait(smem_u32(&sm.mbar[st]), (uint32_t)((s / NSTAGE - 1) & 1))) {
        atomicExch(flag, 3);
        sm.abort = 1;
      }
    }
    __syncthreads();
    if (sm.abort) { ok = false; break; }
    {
      uint32_t* pl = isA ? &sm.a[st][0][0] : &sm.b[st][0][0];
#pragma unroll
      for (int k = 0; k < TBK; ++k) {
        c64 v = cur[k];
        if (conj) v.y = -v.y;
        uint32_t rh, rl, ih, il;
        split(v.x, rh, rl);
        split(v.y, ih, il);
        const int c = cidx(r, k);
        pl[0 * PLANE + c] = rh;
        pl[1 * PLANE + c] = rl;
        pl[2 * PLANE + c] = ih;
        pl[3 * PLANE + c] = il;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t dr = tmem, di = tmem + 128;
      const uint32_t a0 = smem_u32(&sm.a[st][0][0]), b0 = smem_u32(&sm.b[st][0][0]);
      const uint32_t pl = PLANE * 4;   // bytes per plane
#pragma unroll
      for (int kk = 0; kk < TBK; kk += 8) {
        const uint32_t ko = kk * 32;   // K slice kk starts at core-matrix column kk/4 (128 B each)
        const uint64_t arh = sdesc(a0 + 0 * pl + ko), arl = sdesc(a0 + 1 * pl + ko);
        const uint64_t aih = sdesc(a0 + 2 * pl + ko), ail = sdesc(a0 + 3 * pl + ko);
        const uint64_t brh = sdesc(b0 + 0 * pl + ko), brl = sdesc(b0 + 1 * pl + ko);
        const uint64_t bih = sdesc(b0 + 2 * pl + ko), bil = sdesc(b0 + 3 * pl + ko);
        const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
        // Re += Ar Br - Ai Bi
        mma_tf32(dr, arl, brh, idesc, acc);
        mma_tf32(dr, arh, brl, idesc, 1);
        mma_tf32(dr, arh, brh, idesc, 1);
        mma_tf32(dr, ail, bih, idesc_nega, 1);
        mma_tf32(dr, aih, bil, idesc_nega, 1);
        mma_tf32(dr, aih, bih, idesc_nega, 1);
        // Im += Ar Bi + Ai Br
        mma_tf32(di, arl, bih, idesc, acc);
        mma_tf32(di, arh, bil, idesc, 1);
        mma_tf32(di, arh, bih, idesc, 1);
        mma_tf32(di, ail, brh, idesc, 1);
        mma_tf32(di, aih, brl, idesc, 1);
        mma_tf32(di, aih, brh, idesc, 1);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sm.mbar[st])));
      sm.issued = s + 1;
    }
#pragma unroll
    for (int k = 0; k < TBK; ++k) cur[k] = nxt[k];
  }
  __syncthreads();
  // wait for the last commit of every stage (each covers all MMAs issued before it)
  const int nissued = sm.issued;
  if (nissued < nk) ok = false;
  for (int b = 0; b < NSTAGE; ++b) {
    int last = -1;
    for (int q = nissued - 1; q >= 0 && q >= nissued - NSTAGE; --q)
      if (q % NSTAGE == b) { last = q; break; }
    if (last >= 0 && !mbar_wait(smem_u32(&sm.mbar[b]), (uint32_t)((last / NSTAGE) & 1))) {
      atomicExch(flag, 3);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (sm.abort) ok = false;

  if (ok) {
    const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0);
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + lane;
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
      uint32_t vr[16], vi[16];
      if (nk > 0) {
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]),
              "=r"(vr[6]), "=r"(vr[7]), "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]),
              "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]), "=r"(vr[15])
            : "r"(ta));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]),
              "=r"(vi[6]), "=r"(vi[7]), "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]),
              "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
            : "r"(ta + 128));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) vr[j] = vi[j] = 0u;
      }
      if (row < P.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < P.N) {
            const double cr = (double)__uint_as_float(vr[j]), ci = (double)__uint_as_float(vi[j]);
            double re = g.ar * cr - g.ai * ci;
            double im = g.ar * ci + g.ai * cr;
            if (use_d && !(row >= P.zr0 && row < P.zr1)) {
              c64 dv = D[(int64_t)row * P.ldd + col];
              re += g.br * dv.x - g.bi * dv.y;
              im += g.br * dv.y + g.bi * dv.x;
            }
            C[(int64_t)row * P.ldc + col] = make_double2(re, im);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}


// ---- packed-operand engine ---------------------------------------------------------------------
// Pass 1 (k_tc_pack): every 128 x 16 block of op(A) (rows = M) and of op(B) (rows = N, K-major) of
// every problem is converted once into its shared-memory image: 4 planes (Re_hi, Re_lo, Im_hi,
// Im_lo) of 2048 TF32 words in the core-matrix layout, 32 KB contiguous.
// Pass 2 (k_gemm_tc_packed): warp 0 streams the images of each K step into a 3-stage ring with
// cp.async.bulk (the TMA engine, completion counted by mbarrier transaction bytes), warp 1 issues
// the tcgen05 MMAs and releases stages by tcgen05.commit, warps 2-5 drain the TMEM accumulators.

constexpr int PK_BLOCK = 4 * PLANE;     // words per packed 128 x 16 block
constexpr int PK_THREADS = 256;

template <int OPA, int OPB>
__global__ void __launch_bounds__(PK_THREADS) k_tc_pack(GemmArgs g, uint32_t* pack, int64_t pack_es) {
  const int e = blockIdx.y;
  const int blk = blockIdx.x;
  int lo = 0, hi = g.nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.probs[mid].pack_start <= blk) lo = mid;
    else hi = mid - 1;
  }
  const GemmProb P = g.probs[lo];
  int b = blk - P.pack_start;
  const bool isA = b < P.tiles_m * P.ksteps;
  if (!isA) b -= P.tiles_m * P.ksteps;
  const int tile = b / P.ksteps, ks = b % P.ksteps;
  const int row0 = tile * 128, k0 = ks * TBK;
  uint32_t* dst = pack + e * pack_es + (isA ? P.pa : P.pb) + (int64_t)b * PK_BLOCK;
  const c64* A = reinterpret_cast<const c64*>(g.A) + e * g.a_es + P.a;
  const c64* B = reinterpret_cast<const c64*>(g.B) + e * g.b_es + P.b;
  const int op = isA ? OPA : OPB;
  // contiguous-in-memory index runs along k for (A, N/C) and (B, T/H), along rows otherwise
  const bool krun = isA ? (OPA == OP_N || OPA == OP_C) : (OPB == OP_T || OPB == OP_H);
  for (int i = threadIdx.x; i < 128 * TBK; i += PK_THREADS) {
    const int r = krun ? i / TBK : i % 128;
    const int k = krun ? i % TBK : i / 128;
    const int gr = row0 + r, gk = k0 + k;
    c64 v = make_double2(0.0, 0.0);
    if (isA) {
      if (gr < P.M && gk < P.K)
        v = (OPA == OP_N || OPA == OP_C) ? A[(int64_t)gr * P.lda + gk] : A[(int64_t)gk * P.lda + gr];
    } else {
      if (gr < P.N && gk < P.K)
        v = (OPB == OP_N || OPB == OP_C) ? B[(int64_t)gk * P.ldb + gr] : B[(int64_t)gr * P.ldb + gk];
    }
    if (op == OP_C || op == OP_H) v.y = -v.y;
    uint32_t rh, rl, ih, il;
    split(v.x, rh, rl);
    split(v.y, ih, il);
    const int c = cidx(r, k);
    dst[0 * PLANE + c] = rh;
    dst[1 * PLANE + c] = rl;
    dst[2 * PLANE + c] = ih;
    dst[3 * PLANE + c] = il;
  }
}

struct __align__(128) TcPkSmem {
  uint32_t a[NSTAGE][PK_BLOCK];
  uint32_t b[NSTAGE][PK_BLOCK];
  unsigned long long full[NSTAGE];
  unsigned long long empty[NSTAGE];
  unsigned long long done;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

constexpr int TCP_THREADS = 192;

__global__ void __launch_bounds__(TCP_THREADS, 1)
k_gemm_tc_packed(GemmArgs g, const uint32_t* pack, int64_t pack_es, int* flag) {
  extern __shared__ unsigned char smem_raw[];
  TcPkSmem& sm = *reinterpret_cast<TcPkSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = blockIdx.y;
  const GemmProb P = g.probs[find_prob_tc(g.probs, g.nprob, blockIdx.x)];
  const int t = blockIdx.x - P.tile_start;
  const int tm = t / P.tiles_n, tn = t % P.tiles_n;
  const int m0 = tm * TBM, n0 = tn * TBN;
  c64* C = reinterpret_cast<c64*>(g.C) + e * g.c_es + P.c;
  const c64* D = g.D ? reinterpret_cast<const c64*>(g.D) + e * g.d_es + P.d : nullptr;
  const uint32_t* pa = pack + e * pack_es + P.pa + (int64_t)tm * P.ksteps * PK_BLOCK;
  const uint32_t* pb = pack + e * pack_es + P.pb + (int64_t)tn * P.ksteps * PK_BLOCK;
  const int nk = P.ksteps;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int b = 0; b < NSTAGE; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sm.abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                         ((uint32_t)(TBM >> 4) << 24);
  const uint32_t idesc_nega = idesc | (1u << 13);
  constexpr uint32_t BLK_BYTES = PK_BLOCK * 4;

  if (warp == 0) {
    if (lane == 0) {   // producer
      for (int s = 0; s < nk; ++s) {
        const int st = s % NSTAGE;
        if (s >= NSTAGE && !mbar_wait(smem_u32(&sm.empty[st]), (uint32_t)((s / NSTAGE - 1) & 1))) {
          atomicExch(flag, 3);
          sm.abort = 1;
          break;
        }
        const uint32_t fb = smem_u32(&sm.full[st]);
        arrive_expect(fb, 2 * BLK_BYTES);
        bulk_g2s(smem_u32(&sm.a[st][0]), pa + (int64_t)s * PK_BLOCK, BLK_BYTES, fb);
        bulk_g2s(smem_u32(&sm.b[st][0]), pb + (int64_t)s * PK_BLOCK, BLK_BYTES, fb);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      bool ok = true;
      for (int s = 0; s < nk && ok; ++s) {
        const int st = s % NSTAGE;
        if (!mbar_wait(smem_u32(&sm.full[st]), (uint32_t)((s / NSTAGE) & 1))) {
          atomicExch(flag, 3);
          sm.abort = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dr = tmem, di = tmem + 128;
        const uint32_t a0 = smem_u32(&sm.a[st][0]), b0 = smem_u32(&sm.b[st][0]);
        const uint32_t pl = PLANE * 4;
#pragma unroll
        for (int kk = 0; kk < TBK; kk += 8) {
          const uint32_t ko = kk * 32;
          const uint64_t arh = sdesc(a0 + 0 * pl + ko), arl = sdesc(a0 + 1 * pl + ko);
          const uint64_t aih = sdesc(a0 + 2 * pl + ko), ail = sdesc(a0 + 3 * pl + ko);
          const uint64_t brh = sdesc(b0 + 0 * pl + ko), brl = sdesc(b0 + 1 * pl + ko);
          const uint64_t bih = sdesc(b0 + 2 * pl + ko), bil = sdesc(b0 + 3 * pl + ko);
          const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(dr, arl, brh, idesc, acc);
          mma_tf32(dr, arh, brl, idesc, 1);
          mma_tf32(dr, arh, brh, idesc, 1);
          mma_tf32(dr, ail, bih, idesc_nega, 1);
          mma_tf32(dr, aih, bil, idesc_nega, 1);
          mma_tf32(dr, aih, bih, idesc_nega, 1);
          mma_tf32(di, arl, bih, idesc, acc);
          mma_tf32(di, arh, bil, idesc, 1);
          mma_tf32(di, arh, bih, idesc, 1);
          mma_tf32(di, ail, brh, idesc, 1);
          mma_tf32(di, aih, brl, idesc, 1);
          mma_tf32(di, aih, brh, idesc, 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sm.empty[st])));
      }
      // done fires when every MMA issued above has completed (also after an abort)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sm.done)));
    }
  } else {   // warps 2-5: epilogue, TMEM lane quadrant = warp % 4
    bool fin = mbar_wait(smem_u32(&sm.done), 0u);
    fin = __all_sync(0xffffffffu, fin);   // warp-uniform before the .sync.aligned TMEM loads
    if (!fin && lane == 0) atomicExch(flag, 3);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (fin && !sm.abort) {
      const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0);
      const int quad = warp & 3;
      const int row = m0 + quad * 32 + lane;
      for (int c0 = 0; c0 < TBN; c0 += 16) {
        uint32_t vr[16], vi[16];
        if (nk > 0) {
          const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + c0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]),
                "=r"(vr[6]), "=r"(vr[7]), "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]),
                "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]), "=r"(vr[15])
              : "r"(ta));
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]),
                "=r"(vi[6]), "=r"(vi[7]), "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]),
                "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
              : "r"(ta + 128));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) vr[j] = vi[j] = 0u;
        }
        if (row < P.M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            if (col < P.N) {
              const double cr = (double)__uint_as_float(vr[j]), ci = (double)__uint_as_float(vi[j]);
              double re = g.ar * cr - g.ai * ci;
              double im = g.ar * ci + g.ai * cr;
              if (use_d && !(row >= P.zr0 && row < P.zr1)) {
                c64 dv = D[(int64_t)row * P.ldd + col];
                re += g.br * dv.x - g.bi * dv.y;
                im += g.br * dv.y + g.bi * dv.x;
              }
              C[(int64_t)row * P.ldc + col] = make_double2(re, im);
            }
          }
        }
      }
    }
  }
  // outstanding bulk copies of an aborted producer: wait (bounded) for each stage it armed
  if (tid == 0 && sm.abort)
    for (int b = 0; b < NSTAGE; ++b) mbar_wait(smem_u32(&sm.full[b]), 0u, 100000000ull);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Waits on an mbarrier that no thread or copy ever arrives at; the bounded wait must give up after
// limit_ns and report through the flag (the failure path every bounded wait of the library uses).
__global__ void k_wait_probe(unsigned long long limit_ns, int* flag) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (!mbar_wait(smem_u32(&bar), 0u, limit_ns) && threadIdx.x == 0) atomicExch(flag, 3);
}

}  // namespace

cudaError_t gemm_tc_packed(const GemmArgs& g, int n_energy, uint32_t* pack, int64_t pack_es, int* flag,
                           cudaStream_t s) {
  if (g.total_tiles <= 0 || n_energy <= 0) return cudaSuccess;
  if (g.pack_blocks > 0) {   // no blocks when every problem of the list has K = 0
    dim3 pgrid(g.pack_blocks, n_energy);
#define HSC_PK_CASE(a, b)                                                       \
    if (g.opa == a && g.opb == b) k_tc_pack<a, b><<<pgrid, PK_THREADS, 0, s>>>(g, pack, pack_es); else
    HSC_PK_CASE(OP_N, OP_N)
    HSC_PK_CASE(OP_T, OP_N)
    HSC_PK_CASE(OP_N, OP_T)
    HSC_PK_CASE(OP_N, OP_C)
    HSC_PK_CASE(OP_N, OP_H)
    return cudaErrorInvalidValue;
#undef HSC_PK_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t sm = sizeof(TcPkSmem) + 128;
  cudaFuncSetAttribute(k_gemm_tc_packed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gemm_tc_packed<<<dim3(g.total_tiles, n_energy), TCP_THREADS, sm, s>>>(g, pack, pack_es, flag);
  return cudaGetLastError();
}

cudaError_t launch_wait_probe(double seconds, int* flag, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>((unsigned long long)(seconds * 1e9), flag);
  return cudaGetLastError();
}

size_t gemm_tc_smem() { return sizeof(TcSmem) + 128; }

cudaError_t gemm_tc(const GemmArgs& g, int n_energy, int* flag, cudaStream_t s) {
  if (g.total_tiles <= 0 || n_energy <= 0) return cudaSuccess;
  dim3 grid(g.total_tiles, n_energy);
  const size_t sm = gemm_tc_smem();
#define HSC_TC_CASE(a, b)                                                               \
  if (g.opa == a && g.opb == b) {                                                       \
    cudaFuncSetAttribute(k_gemm_tc<a, b>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                         (int)sm);                                                      \
    k_gemm_tc<a, b><<<grid, TC_THREADS, sm, s>>>(g, flag);                              \
    return cudaGetLastError();                                                          \
  }
  HSC_TC_CASE(OP_N, OP_N)
  HSC_TC_CASE(OP_T, OP_N)
  HSC_TC_CASE(OP_N, OP_T)
  HSC_TC_CASE(OP_N, OP_C)
  HSC_TC_CASE(OP_N, OP_H)
#undef HSC_TC_CASE
  return cudaErrorInvalidValue;
}

}  // namespace hsc
