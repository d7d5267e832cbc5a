// Launchers of the complex128 HSC kernels (kernels.cu, gemm_f64.cu).
#pragma once
#include <algorithm>

#include "common.cuh"

namespace hsc {

cudaError_t launch_assemble(const LevelCluster* lc, int nl, int64_t total, const ClusterGlobal* cg,
                            const int32_t* maps, c64* F, c64* S, c64* L, c64* LS, int64_t aug_es,
                            int64_t sq_es, int ne, int do_lesser, cudaStream_t s);
cudaError_t launch_add_a(const LevelCluster* lc, int nl, int64_t max_h, int max_n, const int32_t* h_rq,
                         const int64_t* h_vi, const c64* hval, const int32_t* own_contact,
                         const double* E, double eta, const c64* sr, const c64* sl, int64_t ncs,
                         c64* F, c64* L, int64_t aug_es, int ne, cudaStream_t s);
cudaError_t launch_gj_panel(const GJProb* probs, int nmat, c64* F, int64_t f_es, int32_t* piv,
                            int64_t piv_es, c64* Mt, c64* Rt, int64_t t_es, int k0, int nb, int ne,
                            int* flag, cudaStream_t s, int cluster = 1);
cudaError_t launch_gj_swap(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es,
                           const int32_t* piv, int64_t piv_es, c64* Rt, int64_t t_es, int k0, int nb,
                           int ne, cudaStream_t s, int c_lo = 0, int c_hi = 1 << 30);
cudaError_t launch_leaf_x(const LevelCluster* lc, int nl, int max_n, const int32_t* colptr,
                          const int32_t* rows, const c64* F, int64_t aug_es, c64* X, int64_t x_es, int ne,
                          cudaStream_t s);
cudaError_t launch_leaf_schur(const LevelCluster* lc, int nl, int max_m, const int32_t* colptr,
                              const int32_t* rows, const c64* F, int64_t aug_es, const c64* X, int64_t x_es,
                              c64* S, int64_t sq_es, int ne, cudaStream_t s);
cudaError_t launch_gj_move(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es, c64* Mt,
                           c64* Rt, int64_t t_es, int k0, int nb, int ne, cudaStream_t s);
cudaError_t launch_gj_colperm(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es,
                              const int32_t* piv, int64_t piv_es, int ne, cudaStream_t s, float* growth = nullptr,
                              float* cond = nullptr, int64_t cond_es = 0);
cudaError_t launch_residual(int64_t n, const int64_t* rowptr, const c64* hval, const int64_t* loc,
                           const int64_t* doff, const int32_t* unk_slot, const double* E, double eta,
                           const c64* sr, int64_t ncs, const c64* G, int64_t aug_es, float* resid,
                           int ne, cudaStream_t s);
cudaError_t launch_fold(const LevelCluster* lc, int nl, int64_t max_sq, c64* LS, int64_t sq_es,
                        const c64* Z, int64_t tz_es, int ne, cudaStream_t s);
cudaError_t launch_gather(const LevelCluster* lc, int nl, int64_t max_sq, const ClusterGlobal* cg,
                          const int32_t* u_owner, const int32_t* u_local, const int32_t* u_seg,
                          const int32_t* posmap, const c64* G, const c64* P, int64_t aug_es,
                          c64* GUU, c64* PUU, int64_t tz_es, int ne, int* flag, cudaStream_t s);
cudaError_t launch_out(const int64_t* doff, int64_t n, const int64_t* poff, int64_t npair,
                       const c64* G, const c64* P, int64_t aug_es, c64* ogr, c64* ogl, c64* pgr,
                       c64* pgl, int ne, cudaStream_t s);

cudaError_t launch_add_dense(const DenseBlock* db, int nb, int64_t max_nn, const int32_t* loc,
                             const c64* dr, const c64* dl, int64_t des, c64* F, c64* L, int64_t aug_es,
                             int ne, cudaStream_t s);

cudaError_t launch_scba_mix(int64_t n_E, int64_t n, int64_t ncs, const int64_t* slot_unknown,
                            const c64* gr, const c64* gl, const c64* cr, const c64* cl, double d0,
                            double mix, c64* s_r, c64* s_l, c64* sig_r, c64* sig_l,
                            unsigned long long* dmax, cudaStream_t s);

cudaError_t launch_observables(int64_t n_E, int64_t n, const c64* gr, const c64* gl, const c64* sr,
                               int64_t ncs, const int64_t* slot_unknown, const int32_t* slot_contact,
                               int contact, double* out, cudaStream_t s);

}  // namespace hsc
