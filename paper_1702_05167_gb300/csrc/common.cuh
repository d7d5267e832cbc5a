// Device-side shared definitions for the HSC kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hsc {

typedef double2 c64;   // complex128 (x = re, y = im)
typedef float2 c32;    // complex64

__host__ __device__ inline c64 cmul(c64 a, c64 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline c64 cadd(c64 a, c64 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline c64 csub(c64 a, c64 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline c64 cconj(c64 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline c64 cneg(c64 a) { return make_double2(-a.x, -a.y); }
// a + f p in four fused multiply-adds
__host__ __device__ inline c64 cfma(c64 a, c64 f, c64 p) {
  return make_double2(fma(f.x, p.x, fma(-f.y, p.y, a.x)), fma(f.x, p.y, fma(f.y, p.x, a.y)));
}
// a - f p in four fused multiply-adds (two roundings per part instead of three)
__host__ __device__ inline c64 cfms(c64 a, c64 f, c64 p) {
  return make_double2(fma(-f.x, p.x, fma(f.y, p.y, a.x)), fma(-f.x, p.y, fma(-f.y, p.x, a.y)));
}

// One problem of a grouped GEMM:  C = alpha * op(A) op(B) + beta * D   (D rows in [zr0, zr1) are
// treated as zero). Offsets are element offsets inside the per-energy slice of each operand array.
struct GemmProb {
  int M, N, K;
  int lda, ldb, ldc, ldd;
  int zr0, zr1;
  int use_d;          // 0: drop the beta * D term for this problem
  int tiles_n;        // ceil(N / BN)
  int tile_start;     // first tile index of this problem in the flattened tile space
  int64_t a, b, c, d; // element offsets
  // tensor-core engine only: operand images packed once per launch (TF32 hi/lo planes, 128 x 16
  // core-matrix blocks of 32 KB); word offsets of the A and B images in the per-energy pack buffer
  int tiles_m, ksteps, pack_start;   // pack_start: first pack block of this problem
  int64_t pa, pb;
  // FP64-emulation engine only: offsets of the row scales of op(A) and column scales of op(B)
  int64_t sa, sb;
};

enum Op { OP_N = 0, OP_T = 1, OP_C = 2, OP_H = 3 };   // none, transpose, conjugate, adjoint

struct GemmArgs {
  const GemmProb* probs;
  int nprob;
  int total_tiles;
  const void* A; int64_t a_es;    // base pointers and per-energy strides (elements)
  const void* B; int64_t b_es;
  void* C; int64_t c_es;
  const void* D; int64_t d_es;
  double ar, ai, br, bi;          // alpha, beta
  int opa, opb;
  double flops;                   // algorithmic real flops per energy (host bookkeeping)
  int pack_blocks;                // tensor-core engine: 128x16 operand blocks to pack per energy
  int64_t pack_words;             // tensor-core engine: pack buffer words needed per energy
                                  // (FP64-emulation engine: BF16 slice values per energy)
  int64_t scale_vals;             // FP64-emulation engine: scale doubles per energy
};

// launchers (gemm_f64.cu, gemm_tc.cu)
cudaError_t gemm_z(const GemmArgs& g, int n_energy, cudaStream_t s, bool four_products = false);
cudaError_t gemm_tc(const GemmArgs& g, int n_energy, int* flag, cudaStream_t s);
cudaError_t gemm_tc_packed(const GemmArgs& g, int n_energy, uint32_t* pack, int64_t pack_es, int* flag,
                           cudaStream_t s);
cudaError_t launch_wait_probe(double seconds, int* flag, cudaStream_t s);
// FP64-emulation engine (gemm_oz.cu): oz_layout fills the tile, pack and scale layout of a problem
// and advances the list's running totals; gemm_oz packs the slices and runs the GEMM.
void oz_layout(GemmProb& p, int& pack_blocks, int& tiles, int64_t& slice_vals, int64_t& scale_vals);
cudaError_t gemm_oz(const GemmArgs& g, int n_energy, uint16_t* slices, int64_t slice_es, double* scales,
                    int64_t scale_es, int* flag, cudaStream_t s);

// Gauss-Jordan inversion problem: n x n matrix at element offset `off` (row stride ld) of a
// per-energy array; pivots at piv_off of the per-energy pivot array; panel copy M (n x nb, row
// stride nb) and row block R (nb x n, row stride n) at mt_off / rt_off of per-energy temporaries.
struct GJProb {
  int n, ld;
  int64_t off, piv_off, mt_off, rt_off;
  int band;   // > 0: the block is banded, |r - c| <= band where non-zero (a leaf's stencil in its local
              // order); Gauss-Jordan with partial pivoting then leaves the rows at positions >= k + band
              // untouched until pivot k, and pivot row j has no non-zero beyond column j + 2 band.
              // 0: dense
  int wide;   // > 0: nested blocking with wide panels of this width whose rows above the wide panel
              // are deferred: the panels and their products touch rows >= k1 (the wide panel's
              // start) only; the trailing product applies T R (at bp_off, ld n) to the rows above,
              // T = -P^{-1} the wide panel's transform of a non-pivot row (P its pivot block)
  int64_t bp_off;
};

// Per-level description of the clusters for the element-wise kernels.
struct LevelCluster {
  int n, m, lesser;
  int child[2];          // cluster ids or -1
  int64_t aug, sq;       // per-energy offsets of the cluster's aug (n x (n+m)) / square (m x m) blocks
  int64_t x;             // offset of X = D^{-1} A_iU (n x m)
  int64_t tt, tz, tn;    // level-temporary offsets: n x m, m x m, n x (n+m)
  int64_t map0, map1;    // child front maps
  int64_t h0, h1;        // H-entry range
  int64_t own0;          // own-unknown range start (own_contact, pivots)
  int64_t u0, pm0;       // update-set gather arrays
  int nseg, depth;
  int64_t elem_start;    // flattened element prefix inside the level (kernel-specific)
  int64_t sp_cp;         // leaf with a sparse coupling block: start of its column pointers (m + 1,
                         // absolute indices into the row list), -1 otherwise
};

// A DENSE contact's self-energy block (Section 3.1.2) and where it goes: the owner cluster's front
// (offset aug, row length ld = n + m), nu x nu values at offset blk of each energy's block array,
// the local row of slot k at loc[k].
struct DenseBlock {
  int64_t aug = 0, blk = 0, loc = 0;
  int32_t ld = 0, nu = 0, lesser = 0;
};

struct ClusterGlobal {   // per-cluster data needed when another cluster reads this one's blocks
  int n, m, depth, lesser;
  int64_t aug, sq;
};

}  // namespace hsc
