// Grouped complex128 GEMM on the FP64 tensor cores (mma.sync m8n8k4 f64).
//
// C = alpha * op(A) op(B) + beta * D for a list of problems (one per cluster of a tree level) and a
// batch of energies (grid.y). A complex product is formed from three real products (3M) on
// shared-memory planes: Re = Ar Br - Ai Bi, Im = (Ar + Ai)(Br + Bi) - Ar Br - Ai Bi.
// These are the dense block products of Algorithms 1-2 (Psi, Schur update, downward G^r / G^<).
#include "common.cuh"

namespace hsc {
namespace {

constexpr int BM = 64, BN = 64, BK = 8, PAD = 4, THREADS = 256, THREADS4 = 128;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ int find_prob(const GemmProb* probs, int nprob, int tile) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_start <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// 3 real products per complex product (3M): T1 = Ar Br, T2 = Ai Bi, T3 = (Ar + Ai)(Br + Bi);
// Re = T1 - T2, Im = T3 - T1 - T2. Shared memory holds the planes (Ar, Ai, Ar + Ai) and
// (Br, Bi, Br + Bi); 8 warps, each a 32 x 16 sub-tile of the 64 x 64 CTA tile.
template <int OPA, int OPB>
__global__ void __launch_bounds__(THREADS) k_gemm_z(GemmArgs g) {
  __shared__ double As[3][BK][BM + PAD];
  __shared__ double Bs[3][BK][BN + PAD];
  const int e = blockIdx.y;
  const int tile = blockIdx.x;
  const GemmProb P = g.probs[find_prob(g.probs, g.nprob, tile)];
  const int t = tile - P.tile_start;
  const int m0 = (t / P.tiles_n) * BM, n0 = (t % P.tiles_n) * BN;
  const c64* A = reinterpret_cast<const c64*>(g.A) + e * g.a_es + P.a;
  const c64* B = reinterpret_cast<const c64*>(g.B) + e * g.b_es + P.b;
  c64* C = reinterpret_cast<c64*>(g.C) + e * g.c_es + P.c;
  const c64* D = g.D ? reinterpret_cast<const c64*>(g.D) + e * g.d_es + P.d : nullptr;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;
  const int gq = lane >> 2, tq = lane & 3;
  double t1[4][2][2], t2[4][2][2], t3[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) t1[i][j][h] = t2[i][j][h] = t3[i][j][h] = 0.0;

  for (int k0 = 0; k0 < P.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / THREADS; ++r) {
      int i = tid + r * THREADS;
      int m, k;
      if (OPA == OP_N || OPA == OP_C) { m = i / BK; k = i % BK; }
      else { m = i % BM; k = i / BM; }
      int gm = m0 + m, gk = k0 + k;
      c64 v = make_double2(0.0, 0.0);
      if (gm < P.M && gk < P.K)
        v = (OPA == OP_N || OPA == OP_C) ? A[(int64_t)gm * P.lda + gk] : A[(int64_t)gk * P.lda + gm];
      if (OPA == OP_C || OPA == OP_H) v.y = -v.y;
      As[0][k][m] = v.x;
      As[1][k][m] = v.y;
      As[2][k][m] = v.x + v.y;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / THREADS; ++r) {
      int i = tid + r * THREADS;
      int n, k;
      if (OPB == OP_N || OPB == OP_C) { n = i % BN; k = i / BN; }
      else { n = i / BK; k = i % BK; }
      int gn = n0 + n, gk = k0 + k;
      c64 v = make_double2(0.0, 0.0);
      if (gn < P.N && gk < P.K)
        v = (OPB == OP_N || OPB == OP_C) ? B[(int64_t)gk * P.ldb + gn] : B[(int64_t)gn * P.ldb + gk];
      if (OPB == OP_C || OPB == OP_H) v.y = -v.y;
      Bs[0][k][n] = v.x;
      Bs[1][k][n] = v.y;
      Bs[2][k][n] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double a[3][4], b[3][2];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[q][i] = As[q][kk + tq][wm + i * 8 + gq];
#pragma unroll
        for (int j = 0; j < 2; ++j) b[q][j] = Bs[q][kk + tq][wn + j * 8 + gq];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          dmma(t1[i][j][0], t1[i][j][1], a[0][i], b[0][j]);
          dmma(t2[i][j][0], t2[i][j][1], a[1][i], b[1][j]);
          dmma(t3[i][j][0], t3[i][j][1], a[2][i], b[2][j]);
        }
    }
    __syncthreads();
  }

  const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int row = m0 + wm + i * 8 + gq;
        int col = n0 + wn + j * 8 + tq * 2 + h;
        if (row < P.M && col < P.N) {
          const double cre = t1[i][j][h] - t2[i][j][h];
          const double cim = t3[i][j][h] - t1[i][j][h] - t2[i][j][h];
          double re = g.ar * cre - g.ai * cim;
          double im = g.ar * cim + g.ai * cre;
          if (use_d && !(row >= P.zr0 && row < P.zr1)) {
            c64 d = D[(int64_t)row * P.ldd + col];
            re += g.br * d.x - g.bi * d.y;
            im += g.br * d.y + g.bi * d.x;
          }
          C[(int64_t)row * P.ldc + col] = make_double2(re, im);
        }
      }
}

template <int OPA, int OPB>
__global__ void __launch_bounds__(THREADS4) k_gemm_z4(GemmArgs g) {
  __shared__ double As[2][BK][BM + PAD];  // 4 real products: Re += ArBr - AiBi, Im += ArBi + AiBr
  __shared__ double Bs[2][BK][BN + PAD];
  const int e = blockIdx.y;
  const int tile = blockIdx.x;
  const GemmProb P = g.probs[find_prob(g.probs, g.nprob, tile)];
  const int t = tile - P.tile_start;
  const int m0 = (t / P.tiles_n) * BM, n0 = (t % P.tiles_n) * BN;
  const c64* A = reinterpret_cast<const c64*>(g.A) + e * g.a_es + P.a;
  const c64* B = reinterpret_cast<const c64*>(g.B) + e * g.b_es + P.b;
  c64* C = reinterpret_cast<c64*>(g.C) + e * g.c_es + P.c;
  const c64* D = g.D ? reinterpret_cast<const c64*>(g.D) + e * g.d_es + P.d : nullptr;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  double cr[4][4][2], ci[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j][0] = cr[i][j][1] = ci[i][j][0] = ci[i][j][1] = 0.0;

  for (int k0 = 0; k0 < P.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / THREADS4; ++r) {
      int i = tid + r * THREADS4;
      int m, k;
      if (OPA == OP_N || OPA == OP_C) { m = i / BK; k = i % BK; }
      else { m = i % BM; k = i / BM; }
      int gm = m0 + m, gk = k0 + k;
      c64 v = make_double2(0.0, 0.0);
      if (gm < P.M && gk < P.K)
        v = (OPA == OP_N || OPA == OP_C) ? A[(int64_t)gm * P.lda + gk] : A[(int64_t)gk * P.lda + gm];
      if (OPA == OP_C || OPA == OP_H) v.y = -v.y;
      As[0][k][m] = v.x;
      As[1][k][m] = v.y;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / THREADS4; ++r) {
      int i = tid + r * THREADS4;
      int n, k;
      if (OPB == OP_N || OPB == OP_C) { n = i % BN; k = i / BN; }
      else { n = i / BK; k = i % BK; }
      int gn = n0 + n, gk = k0 + k;
      c64 v = make_double2(0.0, 0.0);
      if (gn < P.N && gk < P.K)
        v = (OPB == OP_N || OPB == OP_C) ? B[(int64_t)gk * P.ldb + gn] : B[(int64_t)gn * P.ldb + gk];
      if (OPB == OP_C || OPB == OP_H) v.y = -v.y;
      Bs[0][k][n] = v.x;
      Bs[1][k][n] = v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double ar[4], ai[4], nai[4], br[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = As[0][kk + tq][wm + i * 8 + gq];
        ai[i] = As[1][kk + tq][wm + i * 8 + gq];
        nai[i] = -ai[i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        br[j] = Bs[0][kk + tq][wn + j * 8 + gq];
        bi[j] = Bs[1][kk + tq][wn + j * 8 + gq];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          dmma(cr[i][j][0], cr[i][j][1], ar[i], br[j]);
          dmma(cr[i][j][0], cr[i][j][1], nai[i], bi[j]);
          dmma(ci[i][j][0], ci[i][j][1], ar[i], bi[j]);
          dmma(ci[i][j][0], ci[i][j][1], ai[i], br[j]);
        }
    }
    __syncthreads();
  }

  const bool use_d = D != nullptr && P.use_d && (g.br != 0.0 || g.bi != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int row = m0 + wm + i * 8 + gq;
        int col = n0 + wn + j * 8 + tq * 2 + h;
        if (row < P.M && col < P.N) {
          double re = g.ar * cr[i][j][h] - g.ai * ci[i][j][h];
          double im = g.ar * ci[i][j][h] + g.ai * cr[i][j][h];
          if (use_d && !(row >= P.zr0 && row < P.zr1)) {
            c64 d = D[(int64_t)row * P.ldd + col];
            re += g.br * d.x - g.bi * d.y;
            im += g.br * d.y + g.bi * d.x;
          }
          C[(int64_t)row * P.ldc + col] = make_double2(re, im);
        }
      }
}

}  // namespace

cudaError_t gemm_z(const GemmArgs& g, int n_energy, cudaStream_t s, bool four_products) {
  if (g.total_tiles <= 0 || n_energy <= 0) return cudaSuccess;
  dim3 grid(g.total_tiles, n_energy);
#define HSC_GEMM_CASE(a, b)                                         \
  if (g.opa == a && g.opb == b) {                                   \
    if (four_products) k_gemm_z4<a, b><<<grid, THREADS4, 0, s>>>(g); \
    else k_gemm_z<a, b><<<grid, THREADS, 0, s>>>(g);                \
    return cudaGetLastError();                                      \
  }
  HSC_GEMM_CASE(OP_N, OP_N)
  HSC_GEMM_CASE(OP_T, OP_N)
  HSC_GEMM_CASE(OP_N, OP_T)
  HSC_GEMM_CASE(OP_N, OP_C)
  HSC_GEMM_CASE(OP_N, OP_H)
#undef HSC_GEMM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace hsc
