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
// buffers are double buffered; the next tile is converted while the tensor core works on the
// current one (tcgen05.commit -> mbarrier). Every mbarrier wait is bounded: on expiry the kernel
// raises a flag, waits (bounded) for its own MMAs, frees TMEM and returns.
//
// These are the Schur-update and downward block products of Algorithms 1-2 in the mixed-precision
// mode (FP32 accumulation), used below the top levels of the tree.
#include <cstdint>

#include "common.cuh"

namespace hsc {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 16, TC_THREADS = 128;
constexpr int PLANE = TBM * TBK;               // tf32 words per plane buffer (128 x 16)
constexpr uint32_t TMEM_COLS = 256;            // Re accumulator cols [0,128), Im [128,256)
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s bound on any mbarrier wait

struct __align__(128) TcSmem {
  uint32_t a[2][4][PLANE];   // [stage][Re_hi, Re_lo, Im_hi, Im_lo]
  uint32_t b[2][4][PLANE];
  unsigned long long mbar[2];
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
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
    if (gtimer() - t0 > WAIT_NS) return false;
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[1])));
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

  const int nk = (P.K + TBK - 1) / TBK;
  bool ok = true;
  for (int s = 0; s < nk && ok; ++s) {
    const int st = s & 1;
    if (s >= 2) {   // buffer st was last read by the MMAs of step s-2
      if (!mbar_wait(smem_u32(&sm.mbar[st]), (uint32_t)(((s - 2) >> 1) & 1))) {
        atomicExch(flag, 3);
        sm.abort = 1;
      }
    }
    __syncthreads();
    if (sm.abort) { ok = false; break; }
    const int k0 = s * TBK;
    // A tile: row m of the tile per thread
    {
      const int r = tid, gm = m0 + r;
      uint32_t* pa = &sm.a[st][0][0];
#pragma unroll 4
      for (int k = 0; k < TBK; ++k) {
        const int gk = k0 + k;
        c64 v = make_double2(0.0, 0.0);
        if (gm < P.M && gk < P.K)
          v = (OPA == OP_N || OPA == OP_C) ? A[(int64_t)gm * P.lda + gk] : A[(int64_t)gk * P.lda + gm];
        if (OPA == OP_C || OPA == OP_H) v.y = -v.y;
        uint32_t rh, rl, ih, il;
        split(v.x, rh, rl);
        split(v.y, ih, il);
        const int c = cidx(r, k);
        pa[0 * PLANE + c] = rh;
        pa[1 * PLANE + c] = rl;
        pa[2 * PLANE + c] = ih;
        pa[3 * PLANE + c] = il;
      }
    }
    // B tile: column n of op(B) per thread, stored as row n (K-major)
    {
      const int r = tid, gn = n0 + r;
      uint32_t* pb = &sm.b[st][0][0];
#pragma unroll 4
      for (int k = 0; k < TBK; ++k) {
        const int gk = k0 + k;
        c64 v = make_double2(0.0, 0.0);
        if (gn < P.N && gk < P.K)
          v = (OPB == OP_N || OPB == OP_C) ? B[(int64_t)gk * P.ldb + gn] : B[(int64_t)gn * P.ldb + gk];
        if (OPB == OP_C || OPB == OP_H) v.y = -v.y;
        uint32_t rh, rl, ih, il;
        split(v.x, rh, rl);
        split(v.y, ih, il);
        const int c = cidx(r, k);
        pb[0 * PLANE + c] = rh;
        pb[1 * PLANE + c] = rl;
        pb[2 * PLANE + c] = ih;
        pb[3 * PLANE + c] = il;
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
  }
  __syncthreads();
  // wait for every committed MMA group of this CTA (the last commit of each buffer)
  const int nissued = sm.issued;
  if (nissued < nk) ok = false;
  if (nissued > 0) {
    const int last = nissued - 1;
    bool done = mbar_wait(smem_u32(&sm.mbar[last & 1]), (uint32_t)((last >> 1) & 1));
    if (last > 0 && done) done = mbar_wait(smem_u32(&sm.mbar[(last - 1) & 1]), (uint32_t)(((last - 1) >> 1) & 1));
    if (!done) {
      atomicExch(flag, 3);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (sm.abort) ok = false;

  if (ok) {
    const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0);
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t vr[16], vi[16];
      if (nk > 0) {
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + c0;
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

}  // namespace

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
