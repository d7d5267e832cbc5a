/* hsc_debug.h -- inspection hook of libhsc for tests and debugging (not part of the solve path).
 *
 * hsc_debug_blocks copies one per-energy block array of the most recent hsc_solve wave back to the
 * host, so that intermediate quantities of Algorithms 1-2 can be compared with a reference:
 *   which 0: F  (per cluster n x (n+m): [D_i^{-1} | A_iU])     1: L  ([Sigma^<-front rows of i])
 *         2: G  ([G_ii | G_iU])                               3: P  ([G^<_ii | G^<_iU])
 *         4: S  (m x m Schur updates)                         5: LS (m x m lesser updates)
 *         6: X  (n x m, D_i^{-1} A_iU)
 *   energy: index inside the last wave; out: host buffer of *count complex values (query with
 *   out = NULL first). Cluster i's block starts at the offset returned by hsc_debug_offset.
 * Errors: HSC_ERR_STATE (no solve yet), HSC_ERR_ARG, HSC_ERR_CUDA. */
#ifndef HSC_DEBUG_H
#define HSC_DEBUG_H
#include "hsc.h"
#ifdef __cplusplus
extern "C" {
#endif
int hsc_debug_blocks(hsc_t h, int32_t which, int32_t energy, hsc_c128* out, int64_t* count);
/* element offsets of cluster i inside the aug arrays (F, L, G, P), square arrays (S, LS) and X */
int hsc_debug_offset(hsc_t h, int32_t i, int64_t* aug, int64_t* sq, int64_t* x);
/* hsc_debug_gemm -- one complex GEMM C = alpha op(A) op(B) + beta D on device buffers (row-major,
 *   complex128) through one of the solve's engines: engine 0 = FP64 tensor pipe (mma.sync f64),
 *   1 = tcgen05 3xTF32 (FP32 accumulation, operands converted per tile), 2 = the same products
 *   from operands packed once into TF32 tile images and streamed by bulk async copies, 3 = FP64
 *   tensor pipe with 4 real products per complex product, 4 = FP64 emulation on the BF16 tensor
 *   cores (tcgen05 kind::f16, operands split exactly into eight 7-bit slices, error below
 *   2^-50 K max|row of op(A)| max|column of op(B)| per real product). op: 0 none, 1 transpose, 2 conjugate, 3 adjoint
 *   (engines support (opa, opb) in {(0,0), (1,0), (0,1), (0,2), (0,3)}). D may be NULL.
 *   Synchronises the stream. Errors: HSC_ERR_ARG, HSC_ERR_CUDA, HSC_ERR_TIMEOUT. */
int hsc_debug_gemm(int32_t engine, int32_t opa, int32_t opb, int32_t M, int32_t N, int32_t K,
                   const hsc_c128* A, int32_t lda, const hsc_c128* B, int32_t ldb, hsc_c128* C,
                   int32_t ldc, const hsc_c128* D, int32_t ldd, double ar, double ai, double br,
                   double bi, void* stream);
/* hsc_debug_wait_timeout -- run one kernel that waits on an mbarrier nothing ever completes, with
 *   the same bounded-wait code as the tensor-core GEMM but a limit of `seconds` (0 < s <= 2). The
 *   wait must expire: returns HSC_ERR_TIMEOUT, and the CUDA context stays usable. */
int hsc_debug_wait_timeout(double seconds);
#ifdef __cplusplus
}
#endif
#endif
