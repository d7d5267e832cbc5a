// Element-wise and factorisation kernels of the HSC / HSC-extension path (complex128):
//   * front assembly by gather (extend-add of the children's Schur and lesser updates),
//   * insertion of A(E) = (E + i eta) I - H - Sigma^r and of Sigma^< into the fronts (Eq. 1-2),
//   * blocked Gauss-Jordan inversion of the cluster blocks A_ii with partial pivoting inside the
//     block (the D_i^{-1} of Eq. 3 / Algorithm 1),
//   * the anti-Hermitian completion of the lesser fold (Algorithm 2),
//   * gathers of G_UU and P_UU from the ancestors' stored blocks (Algorithms 1-2, downward pass),
//   * scatter of diag G^r, diag G^< and requested entries to user order.
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace hsc {
namespace {

__device__ __forceinline__ c64 crecip(c64 d) {
  double s = d.x * d.x + d.y * d.y;
  return make_double2(d.x / s, -d.y / s);
}

// ---- assembly -------------------------------------------------------------------------------

__global__ void k_assemble(const LevelCluster* lc, int nl, int64_t total, const ClusterGlobal* cg,
                           const int32_t* maps, c64* F, c64* S, c64* L, c64* LS, int64_t aug_es,
                           int64_t sq_es, int ne, int do_lesser) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (lc[mid].elem_start <= g) lo = mid;
      else hi = mid - 1;
    }
    const LevelCluster& C = lc[lo];
    const int64_t n = C.n, m = C.m, idx = g - C.elem_start;
    int64_t rpos, cpos, dst;
    bool aug = idx < n * (n + m);
    if (aug) {
      rpos = idx / (n + m);
      cpos = idx % (n + m);
      dst = C.aug + idx;
    } else {
      int64_t j = idx - n * (n + m);
      rpos = n + j / m;
      cpos = n + j % m;
      dst = C.sq + j;
    }
    int64_t src[2] = {-1, -1};
    int les[2] = {0, 0};
    for (int k = 0; k < 2; ++k) {
      int c = C.child[k];
      if (c < 0) continue;
      const int32_t* mp = maps + (k == 0 ? C.map0 : C.map1);
      int32_t a = mp[rpos], b = mp[cpos];
      if (a >= 0 && b >= 0) {
        src[k] = cg[c].sq + (int64_t)a * cg[c].m + b;
        les[k] = cg[c].lesser;
      }
    }
    const bool wl = do_lesser && C.lesser;
    for (int e = 0; e < ne; ++e) {
      c64 v = make_double2(0.0, 0.0), lv = make_double2(0.0, 0.0);
      for (int k = 0; k < 2; ++k)
        if (src[k] >= 0) {
          v = cadd(v, S[e * sq_es + src[k]]);
          if (wl && les[k]) lv = cadd(lv, LS[e * sq_es + src[k]]);
        }
      if (aug) {
        F[e * aug_es + dst] = v;
        if (wl) L[e * aug_es + dst] = lv;
      } else {
        S[e * sq_es + dst] = v;
        if (wl) LS[e * sq_es + dst] = lv;
      }
    }
  }
}

// F -= H on the original entries of each front (rows own, columns own or ancestors)
__global__ void k_add_h(const LevelCluster* lc, const int32_t* h_rq, const int64_t* h_vi,
                        const c64* hval, c64* F, int64_t aug_es, int ne) {
  const LevelCluster& C = lc[blockIdx.y];
  int64_t k = C.h0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= C.h1) return;
  int64_t r = h_rq[2 * k], q = h_rq[2 * k + 1];
  c64 h = hval[h_vi[k]];
  int64_t dst = C.aug + r * (C.n + C.m) + q;
  for (int e = 0; e < ne; ++e) {
    atomicAdd(&F[e * aug_es + dst].x, -h.x);
    atomicAdd(&F[e * aug_es + dst].y, -h.y);
  }
}

// diagonal: (E + i eta) - Sigma^r on A, Sigma^< on the lesser front (Eq. 1-2)
__global__ void k_add_diag(const LevelCluster* lc, const int32_t* own_contact, const double* E,
                           double eta, const c64* sr, const c64* sl, int64_t ncs, c64* F, c64* L,
                           int64_t aug_es, int ne) {
  const LevelCluster& C = lc[blockIdx.y];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= C.n) return;
  int32_t slot = own_contact[C.own0 + r];
  int64_t dst = C.aug + (int64_t)r * (C.n + C.m) + r;
  for (int e = 0; e < ne; ++e) {
    c64 v = F[e * aug_es + dst];
    v.x += E[e];
    v.y += eta;
    if (slot >= 0) v = csub(v, sr[e * ncs + slot]);
    F[e * aug_es + dst] = v;
    if (sl && C.lesser) {
      c64 l = L[e * aug_es + dst];
      if (slot >= 0) l = cadd(l, sl[e * ncs + slot]);
      L[e * aug_es + dst] = l;
    }
  }
}

// ---- Gauss-Jordan -----------------------------------------------------------------------------

constexpr int GJ_THREADS = 128;   // more resident panels per SM: a pivot step is latency-bound

// Unblocked Gauss-Jordan on the panel columns [k0, k0+w), with the pivot of column j chosen as the
// largest |re|+|im| among rows j..n-1 and the swap confined to the panel; then the panel is moved
// to M (and zeroed in place) and the identity part of R is written. Rows taken: all of them, or
// with a wide panel [k1, k1 + wide) (GJProb::wide) rows >= k1 (the rows above take the wide
// panel's whole transform in its trailing product); on a banded block only rows < k0 + w + band
// (the rest are untouched and zero in these columns).
__global__ void __launch_bounds__(GJ_THREADS)
k_gj_panel(const GJProb* probs, c64* F, int64_t f_es, int32_t* piv, int64_t piv_es, c64* Mt,
           c64* Rt, int64_t t_es, int k0, int nb, int* flag) {
  const GJProb P = probs[blockIdx.x];
  const int e = blockIdx.y, n = P.n, ld = P.ld, tid = threadIdx.x;
  if (k0 >= n) return;
  const int w = min(nb, n - k0);
  // banded block: rows at positions >= k0 + w + band are untouched and zero in the panel's columns
  const int nr = P.band > 0 ? min(n, k0 + w + P.band) : n;
  // deferred rows: only rows >= k1 (the wide panel's start) are eliminated here
  const int k1 = P.wide > 0 ? (k0 / P.wide) * P.wide : 0;
  c64* A = F + e * f_es + P.off;
  int32_t* pv = piv + e * piv_es + P.piv_off;
  __shared__ double s_v[GJ_THREADS / 32];
  __shared__ int s_i[GJ_THREADS / 32];
  __shared__ int s_p;
  __shared__ c64 s_inv;
  __shared__ c64 s_pr[64];   // the scaled new row j (panel width <= 64)
  for (int j = k0; j < k0 + w; ++j) {
    double best = -1.0;
    int bi = n;
    for (int r = j + tid; r < nr; r += GJ_THREADS) {
      c64 v = A[(int64_t)r * ld + j];
      double a = fabs(v.x) + fabs(v.y);
      if (a > best) { best = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { s_v[tid >> 5] = best; s_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = s_v[0];
      int ix = s_i[0];
      for (int k = 1; k < GJ_THREADS / 32; ++k)
        if (s_v[k] > b || (s_v[k] == b && s_i[k] < ix)) { b = s_v[k]; ix = s_i[k]; }
      if (ix >= n) ix = j;
      s_p = ix;
      pv[j] = ix;
      c64 d = A[(int64_t)ix * ld + j];
      if (d.x == 0.0 && d.y == 0.0) {
        atomicExch(flag, 1);
        d = make_double2(1.0, 0.0);
      }
      s_inv = crecip(d);
    }
    __syncthreads();
    const int p = s_p;
    const c64 inv = s_inv;
    // swap rows j and p inside the panel and scale the new row j (each thread owns its columns)
    for (int c = tid; c < w; c += GJ_THREADS) {
      const c64 a = A[(int64_t)p * ld + k0 + c];
      if (p != j) A[(int64_t)p * ld + k0 + c] = A[(int64_t)j * ld + k0 + c];
      const c64 nv = (k0 + c == j) ? inv : cmul(a, inv);
      A[(int64_t)j * ld + k0 + c] = nv;
      s_pr[c] = nv;
    }
    __syncthreads();
    for (int r = k1 + tid; r < nr; r += GJ_THREADS) {
      if (r == j) continue;
      c64* row = A + (int64_t)r * ld + k0;
      const int jc = j - k0;
      const c64 f = row[jc];
      for (int c = 0; c < w; ++c) {
        if (c == jc) continue;
        row[c] = cfms(row[c], f, s_pr[c]);
      }
      row[jc] = cneg(cmul(f, inv));
    }
    __syncthreads();
  }
  c64* M = Mt + e * t_es + P.mt_off;
  c64* R = Rt + e * t_es + P.rt_off;
  for (int idx = k1 * w + tid; idx < nr * w; idx += GJ_THREADS) {   // M's rows < k1, >= nr are not read
    int r = idx / w, c = idx % w;
    M[(int64_t)r * nb + c] = A[(int64_t)r * ld + k0 + c];
    A[(int64_t)r * ld + k0 + c] = make_double2(0.0, 0.0);
  }
  for (int idx = tid; idx < w * w; idx += GJ_THREADS) {
    int t = idx / w, c = idx % w;
    R[(int64_t)t * n + k0 + c] = make_double2(t == c ? 1.0 : 0.0, 0.0);
  }
}

// The same panel step spread over a cluster of CS CTAs (CS = 2, 4) when a level has too few
// (matrix, energy) pairs to fill the GPU: CTA q of the cluster owns the rows r with
// (r / GJ_THREADS) % CS == q. Per column: each CTA publishes its best pivot candidate; after a cluster
// barrier every CTA reads all candidates from distributed shared memory and takes the same pivot
// (largest |re|+|im|, then smallest row: the single-CTA choice); every CTA reads rows j and p and
// forms the scaled pivot row; after a second barrier the owners write rows j and p; each CTA
// eliminates its own rows. No barrier closes the column: the next candidate search reads only the
// CTA's own rows, the next cross-CTA reads of pivot rows follow the next column's first barrier
// (release/acquire at cluster scope), and every read of another CTA's shared memory precedes the
// column's second barrier. The arithmetic of every row is the single-CTA kernel's, so the results
// are bitwise identical. Cluster barriers are hardware barriers that every thread of every CTA
// reaches the same number of times.
template <int CS>
__global__ void __launch_bounds__(GJ_THREADS)
k_gj_panel_cl(const GJProb* probs, c64* F, int64_t f_es, int32_t* piv, int64_t piv_es, c64* Mt,
              c64* Rt, int64_t t_es, int k0, int nb, int* flag) {
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const GJProb P = probs[blockIdx.x / CS];
  const int e = blockIdx.y, n = P.n, ld = P.ld, tid = threadIdx.x;
  if (k0 >= n) return;   // uniform over the cluster
  const int w = min(nb, n - k0);
  const int nr = P.band > 0 ? min(n, k0 + w + P.band) : n;   // as in k_gj_panel
  const int k1 = P.wide > 0 ? (k0 / P.wide) * P.wide : 0;    // deferred rows, as in k_gj_panel
  c64* A = F + e * f_es + P.off;
  int32_t* pv = piv + e * piv_es + P.piv_off;
  __shared__ double s_v[GJ_THREADS / 32];
  __shared__ int s_i[GJ_THREADS / 32];
  __shared__ double s_cbest;   // this CTA's candidate, read by the whole cluster
  __shared__ int s_cidx;
  __shared__ int s_p;
  __shared__ c64 s_inv;
  __shared__ c64 s_pr[64], s_old[64];   // scaled new row j, old row j (panel width <= 64)
  auto owner = [&](int r) { return (r / GJ_THREADS) % CS; };
  const int r_first = q * GJ_THREADS + tid, r_step = CS * GJ_THREADS;

  for (int j = k0; j < k0 + w; ++j) {
    double best = -1.0;
    int bi = n;
    for (int r = r_first; r < nr; r += r_step) {
      if (r < j) continue;
      c64 v = A[(int64_t)r * ld + j];
      double a = fabs(v.x) + fabs(v.y);
      if (a > best) { best = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { s_v[tid >> 5] = best; s_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = s_v[0];
      int ix = s_i[0];
      for (int k = 1; k < GJ_THREADS / 32; ++k)
        if (s_v[k] > b || (s_v[k] == b && s_i[k] < ix)) { b = s_v[k]; ix = s_i[k]; }
      s_cbest = b;
      s_cidx = ix;
    }
    cluster.sync();   // 1: every candidate published
    if (tid == 0) {
      double b = -1.0;
      int ix = n;
      for (int k = 0; k < CS; ++k) {
        const double ob = *cluster.map_shared_rank(&s_cbest, k);
        const int oi = *cluster.map_shared_rank(&s_cidx, k);
        if (ob > b || (ob == b && oi < ix)) { b = ob; ix = oi; }
      }
      if (ix >= n) ix = j;
      s_p = ix;
      if (q == 0) pv[j] = ix;
      c64 d = A[(int64_t)ix * ld + j];
      if (d.x == 0.0 && d.y == 0.0) {
        if (q == 0) atomicExch(flag, 1);
        d = make_double2(1.0, 0.0);
      }
      s_inv = crecip(d);
    }
    __syncthreads();
    const int p = s_p;
    const c64 inv = s_inv;
    for (int c = tid; c < w; c += GJ_THREADS) {
      const c64 a = A[(int64_t)p * ld + k0 + c];   // becomes row j
      s_old[c] = A[(int64_t)j * ld + k0 + c];      // becomes row p
      s_pr[c] = (k0 + c == j) ? inv : cmul(a, inv);
    }
    cluster.sync();   // 2: rows j and p read everywhere before their owners overwrite them
    if (owner(j) == q)
      for (int c = tid; c < w; c += GJ_THREADS) A[(int64_t)j * ld + k0 + c] = s_pr[c];
    if (p != j && owner(p) == q)
      for (int c = tid; c < w; c += GJ_THREADS) A[(int64_t)p * ld + k0 + c] = s_old[c];
    __syncthreads();
    for (int r = r_first; r < nr; r += r_step) {
      if (r == j || r < k1) continue;
      c64* row = A + (int64_t)r * ld;
      const c64 f = row[j];
      for (int c = 0; c < w; ++c) {
        if (k0 + c == j) continue;
        row[k0 + c] = cfms(row[k0 + c], f, s_pr[c]);
      }
      row[j] = cneg(cmul(f, inv));
    }

    __syncthreads();   // this CTA's rows are complete before its next candidate search
  }
  c64* M = Mt + e * t_es + P.mt_off;
  c64* R = Rt + e * t_es + P.rt_off;
  for (int r = r_first; r < nr; r += r_step)
    for (int c = 0; c < w && r >= k1; ++c) {
      M[(int64_t)r * nb + c] = A[(int64_t)r * ld + k0 + c];
      A[(int64_t)r * ld + k0 + c] = make_double2(0.0, 0.0);
    }
  if (q == 0)
    for (int idx = tid; idx < w * w; idx += GJ_THREADS) {
      int t = idx / w, c = idx % w;
      R[(int64_t)t * n + k0 + c] = make_double2(t == c ? 1.0 : 0.0, 0.0);
    }
}

// apply the panel's row swaps to the columns [c_lo, c_hi) outside the panel and copy its pivot
// rows there to R (all columns for a whole-matrix step; the enclosing wide panel's columns for a
// step nested inside it)
__global__ void k_gj_swap(const GJProb* probs, c64* F, int64_t f_es, const int32_t* piv,
                          int64_t piv_es, c64* Rt, int64_t t_es, int k0, int nb, int c_lo, int c_hi) {
  const GJProb P = probs[blockIdx.y];
  const int e = blockIdx.z, n = P.n, ld = P.ld;
  const int c = c_lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= n || c >= n || c >= c_hi) return;
  const int w = min(nb, n - k0);
  if (c >= k0 && c < k0 + w) return;
  c64* A = F + e * f_es + P.off;
  const int32_t* pv = piv + e * piv_es + P.piv_off;
  if (P.band > 0 && c >= k0 + w + 2 * P.band) {   // banded: the pivot rows are zero in this column
    c64* R = Rt + e * t_es + P.rt_off;
    for (int t = 0; t < w; ++t) R[(int64_t)t * n + c] = make_double2(0.0, 0.0);
    return;
  }
  for (int j = k0; j < k0 + w; ++j) {
    int p = pv[j];
    if (p != j) {
      c64 t = A[(int64_t)j * ld + c];
      A[(int64_t)j * ld + c] = A[(int64_t)p * ld + c];
      A[(int64_t)p * ld + c] = t;
    }
  }
  c64* R = Rt + e * t_es + P.rt_off;
  for (int t = 0; t < w; ++t) R[(int64_t)t * n + c] = A[(int64_t)(k0 + t) * ld + c];
}

// The wide panel [k0, k0 + w) of each block, whose columns the nested steps have reduced, moves to
// M (n x nb, leading dimension nb) and is zeroed in place; R (nb x n) gets the identity in those
// columns, so that the trailing product M R restores them.
__global__ void k_gj_move(const GJProb* probs, c64* F, int64_t f_es, c64* Mt, c64* Rt, int64_t t_es,
                          int k0, int nb) {
  const GJProb P = probs[blockIdx.y];
  const int e = blockIdx.z, n = P.n, ld = P.ld;
  if (k0 >= n) return;
  const int w = min(nb, n - k0);
  c64* A = F + e * f_es + P.off;
  c64* M = Mt + e * t_es + P.mt_off;
  c64* R = Rt + e * t_es + P.rt_off;
  const int64_t tot = (int64_t)n * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / w), c = (int)(idx % w);
    M[(int64_t)r * nb + c] = A[(int64_t)r * ld + k0 + c];
    A[(int64_t)r * ld + k0 + c] = make_double2(0.0, 0.0);
    if (r < w) R[(int64_t)r * n + k0 + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// undo the row interchanges on the columns of the in-place inverse: A^{-1} = Y P
// Also records the growth of the energy: the largest |Re| + |Im| of any entry of D_i^{-1}, and,
// per (energy, block), ||D_i^{-1}||_F in cond[e * cond_es + block]. The Frobenius norm bounds
// 1 / sigma_min(D_i) from above and below within sqrt(n): a level of the block delta from E shows
// up as ~1/delta, which the largest entry (weighted by the level's eigenvector, ~1/n per entry)
// understates.
__global__ void k_gj_colperm(const GJProb* probs, c64* F, int64_t f_es, const int32_t* piv,
                             int64_t piv_es, float* growth, float* cond, int64_t cond_es) {
  extern __shared__ unsigned char smem[];
  const GJProb P = probs[blockIdx.x];
  const int e = blockIdx.y, n = P.n, ld = P.ld, tid = threadIdx.x;
  c64* buf = reinterpret_cast<c64*>(smem);
  int* idx = reinterpret_cast<int*>(buf + n);
  c64* A = F + e * f_es + P.off;
  const int32_t* pv = piv + e * piv_es + P.piv_off;
  for (int c = tid; c < n; c += blockDim.x) idx[c] = c;
  __syncthreads();
  if (tid == 0)
    for (int j = n - 1; j >= 0; --j) {
      int p = pv[j];
      if (p != j) { int t = idx[j]; idx[j] = idx[p]; idx[p] = t; }
    }
  __syncthreads();
  double mx = 0.0, ss = 0.0;
  for (int r = 0; r < n; ++r) {
    c64* row = A + (int64_t)r * ld;
    for (int c = tid; c < n; c += blockDim.x) {
      buf[c] = row[c];
      mx = fmax(mx, fabs(buf[c].x) + fabs(buf[c].y));
      ss = fma(buf[c].x, buf[c].x, fma(buf[c].y, buf[c].y, ss));
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) row[c] = buf[idx[c]];
    __syncthreads();
  }
  if (cond) {   // block sum of squares: warp shuffles, then one slot per warp (buf is free now)
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    double* red = reinterpret_cast<double*>(smem);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      const double f = sqrt(t);
      cond[e * cond_es + blockIdx.x] = (f == f && f < 3.0e38) ? (float)f : __int_as_float(0x7f800000);
    }
  }
  if (growth) {
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // positive floats order as their bit patterns; NaN or overflow records +inf
    const float f = (mx == mx && mx < 3.0e38) ? (float)mx : __int_as_float(0x7f800000);
    if ((tid & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(growth + e), __float_as_uint(f));
  }
}

// ---- leaves: products with the sparse coupling block A_iU -------------------------------------
// A leaf has no children, so its front's coupling block A_iU holds only the H entries between its
// sites and U_i: column k has the few rows j coupled to U_i[k] (CSC pattern from the analysis).
// X = D^{-1} A_iU is then a gather of D^{-1}'s columns, X[r, k] = sum_j D^{-1}[r, j] A[j, k], and the
// Schur update S -= A_iU^T X a gather of X's rows, S[k, l] -= sum_j A[j, k] X[j, l]: the same sums as
// the dense products (whose other terms are exact zeros), in FP64 on the CUDA cores.
__global__ void k_leaf_x(const LevelCluster* lc, const int32_t* colptr, const int32_t* rows,
                         const c64* F, int64_t aug_es, c64* X, int64_t x_es) {
  const LevelCluster& C = lc[blockIdx.y];
  const int r = blockIdx.x;
  if (C.sp_cp < 0 || r >= C.n) return;
  const int e = blockIdx.z;
  const int64_t ld = C.n + C.m;
  const c64* Fe = F + e * aug_es + C.aug;
  const c64* dr = Fe + (int64_t)r * ld;   // row r of D^{-1}
  c64* xr = X + e * x_es + C.x + (int64_t)r * C.m;
  const int32_t* cp = colptr + C.sp_cp;
  for (int k = threadIdx.x; k < C.m; k += blockDim.x) {
    c64 acc = make_double2(0.0, 0.0);
    for (int t = cp[k]; t < cp[k + 1]; ++t) {
      const int j = rows[t];
      acc = cfma(acc, dr[j], Fe[(int64_t)j * ld + C.n + k]);
    }
    xr[k] = acc;
  }
}

__global__ void k_leaf_schur(const LevelCluster* lc, const int32_t* colptr, const int32_t* rows,
                             const c64* F, int64_t aug_es, const c64* X, int64_t x_es, c64* S,
                             int64_t sq_es) {
  const LevelCluster& C = lc[blockIdx.y];
  const int k = blockIdx.x;
  if (C.sp_cp < 0 || k >= C.m) return;
  const int e = blockIdx.z;
  const int64_t ld = C.n + C.m;
  const c64* Fe = F + e * aug_es + C.aug;
  const c64* Xe = X + e * x_es + C.x;
  c64* sr = S + e * sq_es + C.sq + (int64_t)k * C.m;
  const int32_t* cp = colptr + C.sp_cp;
  const int t0 = cp[k], t1 = cp[k + 1];
  for (int l = threadIdx.x; l < C.m; l += blockDim.x) {
    c64 acc = sr[l];
    for (int t = t0; t < t1; ++t) {
      const int j = rows[t];
      acc = cfms(acc, Fe[(int64_t)j * ld + C.n + k], Xe[(int64_t)j * C.m + l]);
    }
    sr[l] = acc;
  }
}

// ---- a-posteriori check: diagonal residual of A G^r = I ---------------------------------------
// Every non-zero A_uv joins two unknowns whose G^r entry lies in a stored block (same cluster, or
// one in the other's update set; G^r = (G^r)^T for the complex-symmetric A of Eq. 1), so
//   r_u = (E + i eta - Sigma^r_u) G_uu - sum_v H_uv G_uv - 1
// is computable from the solve's own output; the energy's record is max_u |Re r_u| + |Im r_u|.
__global__ void k_residual(int64_t n, const int64_t* rowptr, const c64* hval, const int64_t* loc,
                           const int64_t* doff, const int32_t* unk_slot, const double* E, double eta,
                           const c64* sr, int64_t ncs, const c64* G, int64_t aug_es, float* resid) {
  const int e = blockIdx.y;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (u < n) {
    const c64* Ge = G + e * aug_es;
    c64 a = make_double2(E[e], eta);
    const int slot = unk_slot[u];
    if (slot >= 0) a = csub(a, sr[e * ncs + slot]);
    c64 r = cmul(a, Ge[doff[u]]);
    r.x -= 1.0;
    for (int64_t k = rowptr[u]; k < rowptr[u + 1]; ++k) r = csub(r, cmul(hval[k], Ge[loc[k]]));
    mx = fabs(r.x) + fabs(r.y);
    if (!(mx == mx)) mx = 3.0e38;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float f = mx < 3.0e38 ? (float)mx : __int_as_float(0x7f800000);
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(resid + e), __float_as_uint(f));
}

// ---- lesser fold completion: LS += Z - Z^dagger --------------------------------------------

__global__ void k_fold(const LevelCluster* lc, c64* LS, int64_t sq_es, const c64* Z, int64_t tz_es,
                       int ne) {
  const LevelCluster& C = lc[blockIdx.y];
  const int64_t m = C.m;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!C.lesser || idx >= m * m) return;
  int64_t a = idx / m, b = idx % m;
  for (int e = 0; e < ne; ++e) {
    c64 z = Z[e * tz_es + C.tz + a * m + b];
    c64 zt = Z[e * tz_es + C.tz + b * m + a];
    c64 v = LS[e * sq_es + C.sq + idx];
    v.x += z.x - zt.x;
    v.y += z.y + zt.y;
    LS[e * sq_es + C.sq + idx] = v;
  }
}

// ---- downward gathers --------------------------------------------------------------------------

__global__ void k_gather(const LevelCluster* lc, const ClusterGlobal* cg, const int32_t* u_owner,
                         const int32_t* u_local, const int32_t* u_seg, const int32_t* posmap,
                         const c64* G, const c64* P, int64_t aug_es, c64* GUU, c64* PUU,
                         int64_t tz_es, int ne, int* flag) {
  const LevelCluster& C = lc[blockIdx.y];
  const int64_t m = C.m;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int64_t k1 = idx / m, k2 = idx % m;
  const int p1 = u_owner[C.u0 + k1], p2 = u_owner[C.u0 + k2];
  const int64_t l1 = u_local[C.u0 + k1], l2 = u_local[C.u0 + k2];
  int64_t src;
  bool trans = false;
  if (p1 == p2) {
    src = cg[p1].aug + l1 * (cg[p1].n + cg[p1].m) + l2;
  } else if (cg[p2].depth < cg[p1].depth) {
    int32_t k = posmap[C.pm0 + k2 * C.nseg + u_seg[C.u0 + k1]];
    if (k < 0) { atomicExch(flag, 2); return; }
    src = cg[p1].aug + l1 * (cg[p1].n + cg[p1].m) + cg[p1].n + k;
  } else {
    int32_t k = posmap[C.pm0 + k1 * C.nseg + u_seg[C.u0 + k2]];
    if (k < 0) { atomicExch(flag, 2); return; }
    src = cg[p2].aug + l2 * (cg[p2].n + cg[p2].m) + cg[p2].n + k;
    trans = true;
  }
  for (int e = 0; e < ne; ++e) {
    GUU[e * tz_es + C.tz + idx] = G[e * aug_es + src];
    if (PUU) {
      c64 p = P[e * aug_es + src];
      if (trans) p = make_double2(-p.x, p.y);   // P_ab = -conj(P_ba)
      PUU[e * tz_es + C.tz + idx] = p;
    }
  }
}

// ---- outputs -----------------------------------------------------------------------------------

__global__ void k_out_diag(const int64_t* doff, int64_t n, const c64* G, const c64* P,
                           int64_t aug_es, c64* ogr, c64* ogl, int ne) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int64_t s = doff[u];
  for (int e = 0; e < ne; ++e) {
    ogr[e * n + u] = G[e * aug_es + s];
    if (ogl) ogl[e * n + u] = P[e * aug_es + s];
  }
}

__global__ void k_out_pairs(const int64_t* poff, int64_t npair, const c64* G, const c64* P,
                            int64_t aug_es, c64* ogr, c64* ogl, int ne) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npair) return;
  int64_t s = poff[k];
  bool trans = s < 0;
  if (trans) s = -s - 1;
  for (int e = 0; e < ne; ++e) {
    ogr[e * npair + k] = G[e * aug_es + s];
    if (ogl) {
      c64 p = P[e * aug_es + s];
      if (trans) p = make_double2(-p.x, p.y);
      ogl[e * npair + k] = p;
    }
  }
}

// ---- observables: DOS = -(1/pi) sum_u Im G^r_uu, lesser trace = sum_u Im G^<_uu,
//      T = sum over the slots of one contact of Gamma_slot Im G^<_(slot unknown), Gamma = -2 Im Sigma^r
__global__ void k_observables(int64_t n, const c64* gr, const c64* gl, const c64* sr, int64_t ncs,
                              const int64_t* slot_unknown, const int32_t* slot_contact, int contact,
                              double* out) {
  const int e = blockIdx.x;
  __shared__ double red[3][256];
  double dos = 0, ltr = 0, tr = 0;
  for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
    dos += gr[e * n + u].y;
    if (gl) ltr += gl[e * n + u].y;
  }
  if (gl && sr)
    for (int64_t k = threadIdx.x; k < ncs; k += blockDim.x)
      if (slot_contact[k] == contact) tr += -2.0 * sr[e * ncs + k].y * gl[e * n + slot_unknown[k]].y;
  red[0][threadIdx.x] = dos;
  red[1][threadIdx.x] = tr;
  red[2][threadIdx.x] = ltr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[3 * e + 0] = -red[0][0] / 3.14159265358979323846;
    out[3 * e + 1] = red[1][0];
    out[3 * e + 2] = red[2][0];
  }
}

// ---- DENSE contact self-energies (Section 3.1.2): A_ii -= Sigma^r block and, for the lesser
//      front, L_ii += Sigma^< block on the own rows of each dense contact's cluster; runs after the
//      diagonal terms and before the cluster's Gauss-Jordan. Distinct (a, b) hit distinct front
//      entries (loc is a permutation of the cluster's rows), so there are no races.
__global__ void k_add_dense(const DenseBlock* db, const int32_t* loc, const c64* dr, const c64* dl,
                            int64_t des, c64* F, c64* L, int64_t aug_es, int ne) {
  const DenseBlock& B = db[blockIdx.y];
  const int64_t nn = (int64_t)B.nu * B.nu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = k / B.nu, b = k - a * B.nu;
    const int64_t dst = B.aug + (int64_t)loc[B.loc + a] * B.ld + loc[B.loc + b];
    for (int e = 0; e < ne; ++e) {
      F[e * aug_es + dst] = csub(F[e * aug_es + dst], dr[e * des + B.blk + k]);
      if (dl && B.lesser) L[e * aug_es + dst] = cadd(L[e * aug_es + dst], dl[e * des + B.blk + k]);
    }
  }
}

// ---- self-consistent dephasing (the scattering part of Sigma^r in Eq. 1, local elastic model):
//      on every contact slot k of energy e, with u its unknown, F^r = d0 G^r_uu and F^< = i d0 Im G^<_uu
//      (G^< is anti-Hermitian, Algorithm 2: a real part of its diagonal is rounding error, and fed
//      back it would be a Hermitian part of Sigma^< that the lesser recurrences do not carry);
//      delta = max |F - S| and scale = max |F| over all slots (atomicMax on the bit patterns of
//      non-negative doubles, whose unsigned order is their numeric order); then S += mix (F - S)
//      and the next solve's self-energy Sigma = Sigma_contact + S.
__global__ void k_scba_mix(int64_t total, int64_t n, int64_t ncs, const int64_t* slot_unknown,
                           const c64* gr, const c64* gl, const c64* cr, const c64* cl, double d0,
                           double mix, c64* s_r, c64* s_l, c64* sig_r, c64* sig_l,
                           unsigned long long* dmax) {
  double dm = 0.0, sc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / ncs;
    const int64_t u = e * n + slot_unknown[i - e * ncs];
    const c64 fr = make_double2(d0 * gr[u].x, d0 * gr[u].y);
    const c64 fl = make_double2(0.0, d0 * gl[u].y);
    c64 a = s_r[i], b = s_l[i];
    const c64 dr = csub(fr, a), dl = csub(fl, b);
    dm = fmax(dm, fmax(hypot(dr.x, dr.y), hypot(dl.x, dl.y)));
    sc = fmax(sc, fmax(hypot(fr.x, fr.y), hypot(fl.x, fl.y)));
    a = make_double2(a.x + mix * dr.x, a.y + mix * dr.y);
    b = make_double2(b.x + mix * dl.x, b.y + mix * dl.y);
    s_r[i] = a;
    s_l[i] = b;
    sig_r[i] = cadd(cr[i], a);
    sig_l[i] = cadd(cl[i], b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&dmax[0], (unsigned long long)__double_as_longlong(dm));
    atomicMax(&dmax[1], (unsigned long long)__double_as_longlong(sc));
  }
}

}  // namespace

cudaError_t launch_add_dense(const DenseBlock* db, int nb, int64_t max_nn, const int32_t* loc,
                             const c64* dr, const c64* dl, int64_t des, c64* F, c64* L, int64_t aug_es,
                             int ne, cudaStream_t s) {
  if (nb <= 0 || max_nn <= 0) return cudaSuccess;
  const int64_t bx = std::min<int64_t>((max_nn + 255) / 256, 1024);
  k_add_dense<<<dim3((unsigned)bx, (unsigned)nb), 256, 0, s>>>(db, loc, dr, dl, des, F, L, aug_es, ne);
  return cudaGetLastError();
}

cudaError_t launch_scba_mix(int64_t n_E, int64_t n, int64_t ncs, const int64_t* slot_unknown,
                            const c64* gr, const c64* gl, const c64* cr, const c64* cl, double d0,
                            double mix, c64* s_r, c64* s_l, c64* sig_r, c64* sig_l,
                            unsigned long long* dmax, cudaStream_t s) {
  const int64_t total = n_E * ncs;
  if (total <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 8);
  k_scba_mix<<<(unsigned)blocks, 256, 0, s>>>(total, n, ncs, slot_unknown, gr, gl, cr, cl, d0, mix, s_r,
                                               s_l, sig_r, sig_l, dmax);
  return cudaGetLastError();
}

cudaError_t launch_observables(int64_t n_E, int64_t n, const c64* gr, const c64* gl, const c64* sr,
                               int64_t ncs, const int64_t* slot_unknown, const int32_t* slot_contact,
                               int contact, double* out, cudaStream_t s) {
  if (n_E <= 0) return cudaSuccess;
  k_observables<<<(unsigned)n_E, 256, 0, s>>>(n, gr, gl, sr, ncs, slot_unknown, slot_contact, contact, out);
  return cudaGetLastError();
}

// ---- launchers -----------------------------------------------------------------------------------

static int blocks_for(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 1 << 20); }

cudaError_t launch_assemble(const LevelCluster* lc, int nl, int64_t total, const ClusterGlobal* cg,
                            const int32_t* maps, c64* F, c64* S, c64* L, c64* LS, int64_t aug_es,
                            int64_t sq_es, int ne, int do_lesser, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  int b = std::min(blocks_for(total, 256), 152 * 16);
  k_assemble<<<b, 256, 0, s>>>(lc, nl, total, cg, maps, F, S, L, LS, aug_es, sq_es, ne, do_lesser);
  return cudaGetLastError();
}

cudaError_t launch_add_a(const LevelCluster* lc, int nl, int64_t max_h, int max_n, const int32_t* h_rq,
                         const int64_t* h_vi, const c64* hval, const int32_t* own_contact,
                         const double* E, double eta, const c64* sr, const c64* sl, int64_t ncs,
                         c64* F, c64* L, int64_t aug_es, int ne, cudaStream_t s) {
  if (max_h > 0) {
    dim3 g(blocks_for(max_h, 256), nl);
    k_add_h<<<g, 256, 0, s>>>(lc, h_rq, h_vi, hval, F, aug_es, ne);
  }
  if (max_n > 0) {   // a level of pass-through clusters alone (merged trees) has no own unknowns
    dim3 g2(blocks_for(max_n, 256), nl);
    k_add_diag<<<g2, 256, 0, s>>>(lc, own_contact, E, eta, sr, sl, ncs, F, L, aug_es, ne);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(int64_t n, const int64_t* rowptr, const c64* hval, const int64_t* loc,
                           const int64_t* doff, const int32_t* unk_slot, const double* E, double eta,
                           const c64* sr, int64_t ncs, const c64* G, int64_t aug_es, float* resid,
                           int ne, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_residual<<<dim3((unsigned)((n + 255) / 256), ne), 256, 0, s>>>(n, rowptr, hval, loc, doff, unk_slot, E, eta,
                                                                   sr, ncs, G, aug_es, resid);
  return cudaGetLastError();
}

cudaError_t launch_gj_panel(const GJProb* probs, int nmat, c64* F, int64_t f_es, int32_t* piv,
                            int64_t piv_es, c64* Mt, c64* Rt, int64_t t_es, int k0, int nb, int ne,
                            int* flag, cudaStream_t s, int cluster) {
  if (cluster <= 0) {   // clusters of 2 or 4 CTAs where the (matrix, energy) pairs leave SMs idle
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long pairs = (long long)nmat * ne;
    cluster = pairs >= sms ? 1 : (2 * pairs >= sms ? 2 : 4);
  }
  if (cluster == 1) {
    k_gj_panel<<<dim3(nmat, ne), GJ_THREADS, 0, s>>>(probs, F, f_es, piv, piv_es, Mt, Rt, t_es, k0, nb, flag);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nmat * cluster, ne);
  cfg.blockDim = dim3(GJ_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cluster == 2)
    return cudaLaunchKernelEx(&cfg, k_gj_panel_cl<2>, probs, F, f_es, piv, piv_es, Mt, Rt, t_es, k0, nb, flag);
  return cudaLaunchKernelEx(&cfg, k_gj_panel_cl<4>, probs, F, f_es, piv, piv_es, Mt, Rt, t_es, k0, nb, flag);
}

cudaError_t launch_gj_swap(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es,
                           const int32_t* piv, int64_t piv_es, c64* Rt, int64_t t_es, int k0, int nb,
                           int ne, cudaStream_t s, int c_lo, int c_hi) {
  const int hi = std::min(c_hi, max_n);
  if (hi <= c_lo) return cudaSuccess;
  k_gj_swap<<<dim3(blocks_for(hi - c_lo, 128), nmat, ne), 128, 0, s>>>(probs, F, f_es, piv, piv_es, Rt,
                                                                       t_es, k0, nb, c_lo, hi);
  return cudaGetLastError();
}

cudaError_t launch_gj_move(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es, c64* Mt,
                           c64* Rt, int64_t t_es, int k0, int nb, int ne, cudaStream_t s) {
  if (k0 >= max_n) return cudaSuccess;
  const int64_t tot = (int64_t)max_n * std::min(nb, max_n - k0);
  k_gj_move<<<dim3(blocks_for(tot, 256), nmat, ne), 256, 0, s>>>(probs, F, f_es, Mt, Rt, t_es, k0, nb);
  return cudaGetLastError();
}

cudaError_t launch_leaf_x(const LevelCluster* lc, int nl, int max_n, const int32_t* colptr,
                          const int32_t* rows, const c64* F, int64_t aug_es, c64* X, int64_t x_es, int ne,
                          cudaStream_t s) {
  if (nl <= 0 || max_n <= 0 || ne <= 0) return cudaSuccess;
  k_leaf_x<<<dim3(max_n, nl, ne), 128, 0, s>>>(lc, colptr, rows, F, aug_es, X, x_es);
  return cudaGetLastError();
}

cudaError_t launch_leaf_schur(const LevelCluster* lc, int nl, int max_m, const int32_t* colptr,
                              const int32_t* rows, const c64* F, int64_t aug_es, const c64* X, int64_t x_es,
                              c64* S, int64_t sq_es, int ne, cudaStream_t s) {
  if (nl <= 0 || max_m <= 0 || ne <= 0) return cudaSuccess;
  k_leaf_schur<<<dim3(max_m, nl, ne), 128, 0, s>>>(lc, colptr, rows, F, aug_es, X, x_es, S, sq_es);
  return cudaGetLastError();
}

cudaError_t launch_gj_colperm(const GJProb* probs, int nmat, int max_n, c64* F, int64_t f_es,
                              const int32_t* piv, int64_t piv_es, int ne, cudaStream_t s, float* growth,
                              float* cond, int64_t cond_es) {
  // row buffer and column map; at least 8 doubles for the norm reduction of the 8 warps
  size_t sm = std::max<size_t>((size_t)max_n * (sizeof(c64) + sizeof(int)), 8 * sizeof(double));
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_gj_colperm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gj_colperm<<<dim3(nmat, ne), 256, sm, s>>>(probs, F, f_es, piv, piv_es, growth, cond, cond_es);
  return cudaGetLastError();
}

cudaError_t launch_fold(const LevelCluster* lc, int nl, int64_t max_sq, c64* LS, int64_t sq_es,
                        const c64* Z, int64_t tz_es, int ne, cudaStream_t s) {
  if (max_sq <= 0) return cudaSuccess;
  k_fold<<<dim3(blocks_for(max_sq, 256), nl), 256, 0, s>>>(lc, LS, sq_es, Z, tz_es, ne);
  return cudaGetLastError();
}

cudaError_t launch_gather(const LevelCluster* lc, int nl, int64_t max_sq, const ClusterGlobal* cg,
                          const int32_t* u_owner, const int32_t* u_local, const int32_t* u_seg,
                          const int32_t* posmap, const c64* G, const c64* P, int64_t aug_es,
                          c64* GUU, c64* PUU, int64_t tz_es, int ne, int* flag, cudaStream_t s) {
  if (max_sq <= 0) return cudaSuccess;
  k_gather<<<dim3(blocks_for(max_sq, 256), nl), 256, 0, s>>>(lc, cg, u_owner, u_local, u_seg, posmap,
                                                             G, P, aug_es, GUU, PUU, tz_es, ne, flag);
  return cudaGetLastError();
}

cudaError_t launch_out(const int64_t* doff, int64_t n, const int64_t* poff, int64_t npair,
                       const c64* G, const c64* P, int64_t aug_es, c64* ogr, c64* ogl, c64* pgr,
                       c64* pgl, int ne, cudaStream_t s) {
  k_out_diag<<<blocks_for(n, 256), 256, 0, s>>>(doff, n, G, P, aug_es, ogr, ogl, ne);
  if (npair > 0)
    k_out_pairs<<<blocks_for(npair, 256), 256, 0, s>>>(poff, npair, G, P, aug_es, pgr, pgl, ne);
  return cudaGetLastError();
}

}  // namespace hsc
