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
#ifdef __cplusplus
}
#endif
#endif
