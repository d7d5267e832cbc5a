// Device driver of hsc_solve: uploads the analysis, builds the per-level launch schedules and runs
// Algorithm 1 (upward Schur fold, root inverse, downward selected inverse) and Algorithm 2 (the
// lesser fold and its downward pass) for waves of energies, complex128 throughout.
//
// Per cluster i (n own unknowns, m update-set unknowns U_i), per energy:
//   front     [A_ii | A_iU] = original entries + children's Schur updates (extend-add)
//   D_i^{-1}  Gauss-Jordan with partial pivoting inside the block, in place of A_ii (Eq. 3)
//   X_i       = D_i^{-1} A_iU  (= -Psi_iU of Algorithm 1)
//   S_i      += -A_iU^T X_i    (the Schur update A_jk + Psi_ij^T A_ik of Algorithm 1)
//   lesser    T = (1/2) L_ii conj(X) - L_iU,  Z = X^T T,  LS_i += Z - Z^dagger   (Algorithm 2's fold
//             with the (G^r)^dagger factor of N = Sigma^< (G^r)^dagger applied in the downward pass)
//   downward  G_iU = -X G_UU;  G_ii = D^{-1} - X G_iU^T                        (Algorithm 1)
//             W = D^{-1} [L_ii conj(G_ii) + L_iU conj(G_Ui) | L_ii conj(G_iU) + L_iU conj(G_UU)]
//             P_iU = W_iU - X P_UU;  P_ii = W_ii + X P_iU^dagger              (Algorithm 2)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "ctx.h"
#include "kernels.cuh"

namespace hsc {

struct GemmPair {
  GemmArgs z;    // 64x64 tiles, FP64 tensor pipe (gemm_z)
  GemmArgs tc;   // 128x128 tiles, tcgen05 3xTF32 (gemm_tc)
  GemmArgs oz;   // 128x32 tiles, FP64 emulation on the BF16 tensor cores (gemm_oz)
  bool oz_faster = false;   // cost model: the emulation beats the FP64 pipe on this list
};

// One Gauss-Jordan step of a level: kind 0 = a panel of width nb over the whole block (panel,
// swap on every column, trailing product with K = nb); kind 1 = a panel of width nb nested in the
// wide panel [k1, k1 + nbo) (swap and product restricted to the wide panel's columns); kind 2 = the
// wide panel's own step (move it to M, swap every other column, trailing product with K = nbo).
struct GjStep {
  int kind = 0, k0 = 0, k1 = 0;
};

struct UpLevel {
  int nl = 0;
  int64_t lc = 0;           // index into the LevelCluster array
  int64_t total = 0, max_h = 0, max_sq = 0;
  double asm_bytes = 0, gather_bytes = 0;   // algorithmic bytes per energy
  int max_n = 0;
  bool any_lesser = false;
  GemmPair u1{}, u2{}, u3{}, u4{};
  int64_t gj = 0;           // index into the GJProb array
  int nmat = 0;
  std::vector<GemmPair> steps;
  std::vector<GemmPair> vsteps;  // per step, a product on the Gauss-Jordan scratch (deferred rows):
                                 // T R before a wide panel's trailing product, else empty
  std::vector<GjStep> sdesc;     // what each entry of steps is
  int64_t gji = 0;               // index into the nested-panel GJProb array
  int dense0 = 0, dense_n = 0;   // DENSE contact blocks of this level's clusters (dense_dev range)
  int64_t dense_max = 0;         // largest nu^2 among them
  int sp_count = 0, sp_max_m = 0;   // leaves whose X and Schur products use the sparse A_iU
};

struct DownLevel {
  int nl = 0;
  int64_t lc = 0;
  int64_t max_sq = 0;
  bool any_lesser = false;
  double gather_bytes = 0;
  GemmPair d[9]{};
};

enum KClass { K_GEMM = 0, K_GEMM_TC, K_SCHUR, K_SCHUR_TC, K_GJ_PANEL, K_GJ_SWAP, K_GJ_PERM, K_ASSEMBLE, K_ADD_A, K_FOLD, K_GATHER,
              K_OUT, K_GEMM_OZ, K_SCHUR_OZ, K_RESID, K_GJU, K_GJU_TC, K_GJU_OZ, K_LEAF, K_NCLASS };
static const char* kClassName[K_NCLASS] = {"gemm_z_dmma", "gemm_tc_tf32x3", "schur_z_dmma",
                                           "schur_tc_tf32x3", "gj_panel", "gj_swap", "gj_colperm",
                                           "assemble", "add_a", "lesser_fold", "gather", "out",
                                           "gemm_z_ozaki", "schur_z_ozaki", "residual",
                                           "gj_update_dmma", "gj_update_tc", "gj_update_ozaki", "leaf_sparse"};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // pairs (start, stop)
  size_t used = 0;                 // pairs in use
  std::vector<int> cls;
  std::vector<double> flops, bytes;
  int64_t launches[K_NCLASS] = {0};
  hsc_kernel_stat extra[K_NCLASS] = {};   // kernels of alternate-tree re-solves, merged in
};

static uint64_t g_generation = 0;   // distinguishes device states across re-creation

struct DeviceState {
  int device = -1;
  uint64_t gen = ++g_generation;
  Prof prof;
  bool planned = false;
  int nb = 32;                       // Gauss-Jordan panel width
  int nbo = 0;                       // wide-panel width of the nested blocking (0: not nested)
  int fp64_levels = 2;               // mixed mode: top tree levels kept on the FP64 pipe
  bool gj_fp64 = false;              // mixed mode: Gauss-Jordan trailing updates on the FP64 pipe
  bool four_products = false;        // FP64 engine: 4 real products per complex product (else 3M)
  int fp64_engine = 0;               // 0 cost model, 1 FP64 pipe only, 2 emulation wherever K > 0
  int gj_cluster = 0;                // Gauss-Jordan panel: CTAs per (matrix, energy), 0 = by occupancy
  // energy-independent device arrays
  ClusterGlobal* cg = nullptr;
  LevelCluster* lcs = nullptr;
  GJProb* gjp = nullptr;
  GJProb* gjpi = nullptr;            // the same blocks with the nested panels' M and R buffers
  GemmProb* gp = nullptr;
  GemmProb* gp128 = nullptr;
  GemmProb* gpoz = nullptr;
  int32_t *maps = nullptr, *h_rq = nullptr, *own_contact = nullptr;
  int64_t *h_vi = nullptr, *doff = nullptr;
  int64_t *res_rowptr = nullptr, *res_loc = nullptr;   // residual check: CSR rows, G location per entry
  int32_t* unk_slot = nullptr;                          // contact slot of each unknown, or -1
  c64* hval = nullptr;
  int32_t *u_owner = nullptr, *u_local = nullptr, *u_seg = nullptr, *posmap = nullptr;
  int* flag = nullptr;
  std::vector<UpLevel> up;
  std::vector<DownLevel> down;
  // per-energy strides (elements)
  int64_t aug_es = 0, sq_es = 0, x_es = 0, tt_es = 0, tz_es = 0, tn_es = 0, gjt_es = 0, piv_es = 0;
  int64_t pk_es = 1;                 // tensor-core operand pack buffer (32-bit words per energy)
  int64_t oz_es = 0;                 // the same for the FP64-emulation slices and scales
  bool any_oz = false;               // some list runs on the FP64 emulation
  bool use_pack = true;              // HSC_MIXED: pack operands once per launch (else per tile)
  // workspace for `cap` energies
  int64_t cap = 0;
  void* arena = nullptr;             // owned workspace (nullptr while borrowing)
  size_t arena_bytes = 0;
  void* borrow = nullptr;            // alternate-tree handles: the main handle's idle workspace
  size_t borrow_bytes = 0;
  c64 *F = nullptr, *L = nullptr, *G = nullptr, *P = nullptr, *S = nullptr, *LS = nullptr,
      *X = nullptr, *T = nullptr, *Z = nullptr, *GUU = nullptr, *PUU = nullptr, *N = nullptr,
      *GJT = nullptr;
  int32_t* piv = nullptr;
  uint32_t* PK = nullptr;
  int64_t pk_cur = 0;                // words per energy of PK (its per-energy stride)
  // host-io staging, requested-pair offsets, batch branch stream
  int64_t io_cap = 0;
  void* io = nullptr;
  int64_t* poff = nullptr;
  int64_t pair_cap = 0;
  int32_t *sp_colptr = nullptr, *sp_rows = nullptr;   // sparse A_iU of leaves (CSC, per cluster)
  DenseBlock* dense_dev = nullptr;   // DENSE contact blocks, grouped by upward level
  int32_t* dense_loc = nullptr;      // their slot -> local row maps
  const c64* dense_r = nullptr;      // set by hsc_solve_dense for one call: per-energy blocks,
  const c64* dense_l = nullptr;      //   stride dense_es elements; dense_e0 = the wave's first energy
  int64_t dense_es = 0, dense_e0 = 0;
  int64_t* slot_unknown = nullptr;   // contact slot -> unknown (observables)
  int32_t* slot_contact = nullptr;   // contact slot -> contact id
  cudaStream_t branch = nullptr;
  // per energy of the last solve: growth (largest |Re| + |Im| of any D_i^{-1} entry) and residual
  // (largest |(A G^r - I)_uu|); one allocation, resid = growth + growth_cap
  float* growth = nullptr;
  float* resid = nullptr;
  float* cond = nullptr;             // per (energy, block in gj order): ||D_i^{-1}||_F, after resid
  int64_t growth_cap = 0, growth_n = 0;
  float* growth_wave = nullptr;      // the current wave's slices
  float* resid_wave = nullptr;
  float* cond_wave = nullptr;
  int ncl = 0;                       // clusters (blocks per energy of the cond record)
  std::vector<int> gj_owner;         // cluster id of each Gauss-Jordan block (gj order)
  void* rs_buf = nullptr;            // device staging of re-solved energies (device-io solves)
  size_t rs_cap = 0;
  std::vector<void*> fixed;          // energy-independent allocations
};

void device_state_free(DeviceState* d) {
  if (!d) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (d->device >= 0) cudaSetDevice(d->device);
  for (void* p : d->fixed) cudaFree(p);
  for (cudaEvent_t e : d->prof.pool) cudaEventDestroy(e);
  if (d->arena) cudaFree(d->arena);
  if (d->io) cudaFree(d->io);
  if (d->poff) cudaFree(d->poff);
  if (d->slot_unknown) cudaFree(d->slot_unknown);
  if (d->slot_contact) cudaFree(d->slot_contact);
  if (d->branch) cudaStreamDestroy(d->branch);
  if (d->growth) cudaFree(d->growth);
  if (d->rs_buf) cudaFree(d->rs_buf);
  if (cur >= 0) cudaSetDevice(cur);
  delete d;
}

namespace {

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess)                                                        \
      return hsc_fail(h, HSC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

template <class T>
cudaError_t upload(DeviceState* d, T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  d->fixed.push_back(*dst);
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

constexpr int TILE = 64;

// Per-SM cost model of the two FP64-accurate engines in FP64-pipe operations (DFMA equivalents,
// 1.9 DFMA per clock and SM): the FP64 pipe does 3 (4) K DFMA per element of a 64x64 tile; the
// emulation does, per 128x32 tile and real product, 8 MMAs of 128x(32..256)x16 per 16 K values (the
// 36 digit products, ~600 clocks per K step), one integer drain per 384 K values overlapped with
// the MMAs, one epilogue of ~6 FP64-pipe operations per element, plus the slicing pass (about 9
// DFMA-times per operand element at HBM speed).
constexpr double OZ_TILE = 128 * 32, OZ_DRAIN_DFMA = OZ_TILE * 0.3 * 1.9, OZ_MMA_DFMA = 17 * 1.9,
                 OZ_EPI_DFMA = OZ_TILE * 6.0, OZ_PACK_DFMA = 9.0;

struct GemmList {
  std::vector<GemmProb>& all;      // 64x64-tile problem lists
  std::vector<GemmProb>& all128;   // 128x128-tile problem lists
  std::vector<GemmProb>& alloz;    // 128x32-tile problem lists (FP64 emulation)
  size_t start, start128, startoz;
  int tiles = 0, tiles128 = 0, tilesoz = 0;
  int count = 0;
  double flops = 0;
  int pack_blocks = 0, oz_blocks = 0;
  int64_t pack_words = 0, oz_slices = 0, oz_scales = 0;
  double cost_z = 0, cost_oz = 0;
  GemmList(std::vector<GemmProb>& a, std::vector<GemmProb>& b, std::vector<GemmProb>& c)
      : all(a), all128(b), alloz(c), start(a.size()), start128(b.size()), startoz(c.size()) {}
  void add(int M, int N, int K, int64_t a, int lda, int64_t b, int ldb, int64_t c, int ldc,
           int64_t dd = 0, int ldd = 0, int use_d = 0, int zr0 = 0, int zr1 = 0) {
    if (M <= 0 || N <= 0) return;
    if (all.size() != start + (size_t)count || all128.size() != start128 + (size_t)count ||
        alloz.size() != startoz + (size_t)count)
      throw std::logic_error("interleaved GEMM lists");
    ++count;
    GemmProb p{};
    p.M = M; p.N = N; p.K = K;
    p.a = a; p.lda = lda; p.b = b; p.ldb = ldb; p.c = c; p.ldc = ldc; p.d = dd; p.ldd = ldd;
    p.use_d = use_d; p.zr0 = zr0; p.zr1 = zr1;
    GemmProb q = p, o = p;
    p.tiles_n = (N + TILE - 1) / TILE;
    p.tile_start = tiles;
    tiles += ((M + TILE - 1) / TILE) * p.tiles_n;
    q.tiles_n = (N + 127) / 128;
    q.tile_start = tiles128;
    tiles128 += ((M + 127) / 128) * q.tiles_n;
    q.tiles_m = (M + 127) / 128;
    q.ksteps = (K + 15) / 16;
    q.pack_start = pack_blocks;
    q.pa = pack_words;
    q.pb = pack_words + (int64_t)q.tiles_m * q.ksteps * 8192;
    pack_blocks += (q.tiles_m + q.tiles_n) * q.ksteps;
    pack_words += (int64_t)(q.tiles_m + q.tiles_n) * q.ksteps * 8192;
    const int t0 = tilesoz;
    oz_layout(o, oz_blocks, tilesoz, oz_slices, oz_scales);
    flops += 8.0 * M * N * K;
    const double tz = (double)((M + TILE - 1) / TILE) * p.tiles_n * TILE * TILE;
    cost_z += tz * 3.0 * K;
    const double nt = tilesoz - t0;
    cost_oz += nt * (3.0 * (std::ceil(K / 384.0) * OZ_DRAIN_DFMA + std::ceil(K / 16.0) * 36 * OZ_MMA_DFMA) +
                     OZ_EPI_DFMA) +
               ((double)M * K + (double)K * N) * OZ_PACK_DFMA;
    all.push_back(p);
    all128.push_back(q);
    alloz.push_back(o);
  }
  // records the lists; device pointers are patched after upload (index stored in probs)
  GemmPair args(int opa, int opb, double ar, double ai, double br, double bi) const {
    GemmPair r{};
    GemmArgs g{};
    g.nprob = count;
    g.opa = opa; g.opb = opb;
    g.ar = ar; g.ai = ai; g.br = br; g.bi = bi;
    g.flops = flops;
    r.z = g;
    r.z.probs = reinterpret_cast<const GemmProb*>(start);
    r.z.total_tiles = tiles;
    r.tc = g;
    r.tc.probs = reinterpret_cast<const GemmProb*>(start128);
    r.tc.total_tiles = tiles128;
    r.tc.pack_blocks = pack_blocks;
    r.tc.pack_words = pack_words;
    r.oz = g;
    r.oz.probs = reinterpret_cast<const GemmProb*>(startoz);
    r.oz.total_tiles = tilesoz;
    r.oz.pack_blocks = oz_blocks;
    r.oz.pack_words = oz_slices;
    r.oz.scale_vals = oz_scales;
    r.oz_faster = oz_blocks > 0 && cost_oz < 0.7 * cost_z;
    return r;
  }
};

// words of the pack buffer an emulated list needs per energy: slices, then the scales at the next
// 16-byte boundary
int64_t oz_scale_word(const GemmArgs& g) { return ((g.pack_words + 1) / 2 + 3) / 4 * 4; }
int64_t oz_words(const GemmArgs& g) { return oz_scale_word(g) + 2 * g.scale_vals; }

int locate_pair(const Plan& P, int64_t a, int64_t b, int64_t* out);

int build_schedule(hsc_ctx* h) {
  DeviceState* d = h->dev;
  const Plan& P = h->plan;
  const int nc = (int)P.cl.size();
  const int nb = d->nb;
  const int nbo = d->nbo > nb ? d->nbo : 0;   // nested blocking when the wide panel is wider
  std::vector<ClusterGlobal> cg(nc);
  std::vector<int64_t> xoff(nc);
  int64_t xs = 0;
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = P.cl[i];
    cg[i] = ClusterGlobal{(int)c.n, (int)c.m, c.depth, c.lesser ? 1 : 0, P.off[i].aug, P.off[i].sq};
    xoff[i] = xs;
    xs += c.n * c.m;
  }
  d->aug_es = P.tot_aug;
  d->sq_es = P.tot_sq;
  d->ncl = nc;
  d->gj_owner.clear();
  d->x_es = std::max<int64_t>(xs, 1);
  d->piv_es = std::max<int64_t>(P.n, 1);

  std::vector<LevelCluster> lcs;
  std::vector<GJProb> gjs, gjs_in;
  std::vector<GemmProb> gps, gps128, gpsoz;
  int64_t tt_max = 1, tz_max = 1, tn_max = 1, gjt_max = 1;

  // leaves: the lesser front is diag(Sigma^<) on the own contact rows and L_iU = 0, so the leaf's
  // lesser products only need the hull [c0, c1) of those rows (rows outside are exactly zero)
  std::vector<int> hc0(nc, 0), hc1(nc, 0);
  std::vector<char> leafl(nc, 0);
  for (int i = 0; i < nc; ++i) {
    const Cluster& c = P.cl[i];
    hc0[i] = 0;
    hc1[i] = (int)c.n;
    if (c.nchild == 0 && c.lesser) {
      int lo = (int)c.n, hi = -1;
      for (int64_t r = 0; r < c.n; ++r)
        if (P.own_contact[P.own_off[i] + r] >= 0) { lo = std::min(lo, (int)r); hi = (int)r; }
      if (hi >= lo) { hc0[i] = lo; hc1[i] = hi + 1; leafl[i] = 1; }
    }
  }

  auto base_lc = [&](int i) {
    const Cluster& c = P.cl[i];
    LevelCluster L{};
    L.n = (int)c.n; L.m = (int)c.m; L.lesser = c.lesser ? 1 : 0;
    L.child[0] = c.child[0]; L.child[1] = c.child[1];
    L.aug = P.off[i].aug; L.sq = P.off[i].sq; L.x = xoff[i];
    L.map0 = P.map_off[2 * i] < 0 ? 0 : P.map_off[2 * i];
    L.map1 = P.map_off[2 * i + 1] < 0 ? 0 : P.map_off[2 * i + 1];
    L.h0 = P.h_off[i]; L.h1 = P.h_off[i + 1];
    L.sp_cp = -1;
    L.own0 = P.own_off[i];
    L.u0 = P.u_off[i]; L.pm0 = P.pm_off[i]; L.nseg = P.nseg[i]; L.depth = c.depth;
    return L;
  };

  // leaves whose X = D^{-1} A_iU and Schur update use A_iU's sparsity (the H couplings only)
  std::vector<int32_t> spc, spr;
  const bool leaf_sparse = h->opt_leaf_sparse != 0;
  const bool leaf_band_gj = h->opt_leaf_sparse != 0;   // banded Gauss-Jordan of the leaves' blocks

  // upward levels
  d->up.assign(P.by_height.size(), UpLevel());
  for (size_t hl = 0; hl < P.by_height.size(); ++hl) {
    UpLevel& U = d->up[hl];
    const auto& ids = P.by_height[hl];
    U.lc = (int64_t)lcs.size();
    U.nl = (int)ids.size();
    int64_t el = 0, tt = 0, tz = 0, gjt = 0;
    for (int i : ids) {
      LevelCluster L = base_lc(i);
      if (leaf_sparse && P.cl[i].nchild == 0 && L.m > 0) {
        // a leaf's front holds no children's Schur complements: A_iU is the H entries (r, q >= n)
        std::vector<std::vector<int32_t>> colr(L.m);
        for (int64_t t = L.h0; t < L.h1; ++t) {
          const int32_t r = P.h_rq[2 * t], q = P.h_rq[2 * t + 1];
          if (q >= L.n) colr[q - L.n].push_back(r);
        }
        L.sp_cp = (int64_t)spc.size();
        for (int k = 0; k < L.m; ++k) {
          auto& v = colr[k];
          std::sort(v.begin(), v.end());
          v.erase(std::unique(v.begin(), v.end()), v.end());
          spc.push_back((int32_t)spr.size());
          spr.insert(spr.end(), v.begin(), v.end());
        }
        spc.push_back((int32_t)spr.size());
        U.sp_count++;
        U.sp_max_m = std::max(U.sp_max_m, L.m);
      }
      L.elem_start = el;
      L.tt = tt; L.tz = tz; L.tn = 0;
      el += (int64_t)L.n * (L.n + L.m) + (int64_t)L.m * L.m;
      tt += (int64_t)L.n * L.m;
      tz += (int64_t)L.m * L.m;
      U.max_h = std::max(U.max_h, L.h1 - L.h0);
      U.max_n = std::max(U.max_n, L.n);
      U.max_sq = std::max(U.max_sq, (int64_t)L.m * L.m);
      U.any_lesser |= L.lesser != 0;
      {
        double b = 16.0 * ((double)L.n * (L.n + L.m) + (double)L.m * L.m);
        for (int k = 0; k < 2; ++k)
          if (L.child[k] >= 0) b += 16.0 * (double)P.cl[L.child[k]].m * P.cl[L.child[k]].m;
        U.asm_bytes += L.lesser ? 2 * b : b;
      }
      lcs.push_back(L);
      d->gj_owner.push_back(i);
      GJProb g{};
      g.n = L.n; g.ld = L.n + L.m; g.off = L.aug; g.piv_off = L.own0;
      // a leaf's diagonal block is the H pattern (plus the diagonal) unless a DENSE contact block is
      // added to it: its bandwidth in the local order bounds the Gauss-Jordan steps (nested path)
      if (nbo && leaf_band_gj && P.cl[i].nchild == 0) {
        bool dense_here = false;
        for (const auto& Dn : P.dense) dense_here |= Dn.cluster == i;
        int64_t b = 0;
        for (int64_t t = L.h0; t < L.h1; ++t) {
          const int32_t r = P.h_rq[2 * t], q = P.h_rq[2 * t + 1];
          if (q < L.n) b = std::max<int64_t>(b, r > q ? r - q : q - r);
        }
        if (!dense_here && b > 0 && 2 * b < L.n) g.band = (int)b;
      }
      const int wo = nbo ? nbo : nb;   // M: n x wo, R: wo x n
      g.mt_off = gjt; g.rt_off = gjt + (int64_t)L.n * wo;
      gjt += 2 * (int64_t)L.n * wo;
      if (nbo && L.n > nbo) {   // deferred rows above each wide panel: T R (wo x n) on the scratch
        g.wide = nbo;
        g.bp_off = gjt; gjt += (int64_t)nbo * L.n;
      }
      gjs.push_back(g);
      if (nbo) {   // the nested panels' M (n x nb) and R (nb x n)
        GJProb gi = g;
        gi.mt_off = gjt; gi.rt_off = gjt + (int64_t)L.n * nb;
        gjt += 2 * (int64_t)L.n * nb;
        gjs_in.push_back(gi);
      }
    }
    U.total = el;
    tt_max = std::max(tt_max, tt);
    tz_max = std::max(tz_max, tz);
    gjt_max = std::max(gjt_max, gjt);
    U.gj = (int64_t)gjs.size() - U.nl;
    U.gji = nbo ? (int64_t)gjs_in.size() - U.nl : 0;
    U.nmat = U.nl;
    const LevelCluster* lv = lcs.data() + U.lc;
    {
      GemmList g1(gps, gps128, gpsoz);
      for (int k = 0; k < U.nl; ++k) {
        const auto& L = lv[k];
        if (L.sp_cp >= 0) continue;   // sparse A_iU: k_leaf_x
        g1.add(L.n, L.m, L.n, L.aug, L.n + L.m, L.aug + L.n, L.n + L.m, L.x, L.m);
      }
      U.u1 = g1.args(OP_N, OP_N, 1, 0, 0, 0);
      GemmList g2(gps, gps128, gpsoz);
      for (int k = 0; k < U.nl; ++k) {
        const auto& L = lv[k];
        if (L.sp_cp >= 0) continue;   // sparse A_iU: k_leaf_schur
        g2.add(L.m, L.m, L.n, L.aug + L.n, L.n + L.m, L.x, L.m, L.sq, L.m, L.sq, L.m, 1);
      }
      U.u2 = g2.args(OP_T, OP_N, -1, 0, 1, 0);
      GemmList g3(gps, gps128, gpsoz);
      for (int k = 0; k < U.nl; ++k) {
        const auto& L = lv[k];
        const int i = ids[k], c0 = hc0[i], w = hc1[i] - hc0[i];
        if (!L.lesser) continue;
        if (leafl[i])
          g3.add(w, L.m, w, L.aug + (int64_t)c0 * (L.n + L.m) + c0, L.n + L.m, L.x + (int64_t)c0 * L.m, L.m,
                 L.tt + (int64_t)c0 * L.m, L.m);
        else
          g3.add(L.n, L.m, L.n, L.aug, L.n + L.m, L.x, L.m, L.tt, L.m, L.aug + L.n, L.n + L.m, 1);
      }
      U.u3 = g3.args(OP_N, OP_C, 0.5, 0, -1, 0);
      GemmList g4(gps, gps128, gpsoz);
      for (int k = 0; k < U.nl; ++k) {
        const auto& L = lv[k];
        const int i = ids[k], c0 = hc0[i], w = hc1[i] - hc0[i];
        if (!L.lesser) continue;
        if (leafl[i])
          g4.add(L.m, L.m, w, L.x + (int64_t)c0 * L.m, L.m, L.tt + (int64_t)c0 * L.m, L.m, L.tz, L.m);
        else
          g4.add(L.m, L.m, L.n, L.x, L.m, L.tt, L.m, L.tz, L.m);
      }
      U.u4 = g4.args(OP_T, OP_N, 1, 0, 0, 0);
      const GJProb* gl = gjs.data() + U.gj;
      if (!nbo) {
        for (int k0 = 0; k0 < U.max_n; k0 += nb) {
          GemmList gs(gps, gps128, gpsoz);
          for (int k = 0; k < U.nl; ++k) {
            const GJProb& q = gl[k];
            if (q.n <= k0) continue;
            int w = std::min(nb, q.n - k0);
            gs.add(q.n, q.n, w, q.mt_off, nb, q.rt_off, q.n, q.off, q.ld, q.off, q.ld, 1, k0, k0 + w);
          }
          U.steps.push_back(gs.args(OP_N, OP_N, 1, 0, 1, 0));
          U.vsteps.push_back(GemmList(gps, gps128, gpsoz).args(OP_N, OP_N, 1, 0, 1, 0));
          U.sdesc.push_back(GjStep{0, k0, 0});
        }
      } else {
        const GJProb* gi = gjs_in.data() + U.gji;
        for (int k1 = 0; k1 < U.max_n; k1 += nbo) {
          // nested panels: products restricted to the wide panel's columns [k1, k1 + wo)
          for (int k0 = k1; k0 < std::min(k1 + nbo, U.max_n); k0 += nb) {
            GemmList gs(gps, gps128, gpsoz);
            for (int k = 0; k < U.nl; ++k) {
              const GJProb& q = gi[k];
              if (q.n <= k0) continue;
              const int w = std::min(nb, q.n - k0), wo = std::min(nbo, q.n - k1);
              // banded leaf: rows >= k0 + w + band are untouched by the panel's pivots
              const int mr = q.band > 0 ? std::min(q.n, k0 + w + q.band) : q.n;
              // deferred rows: rows >= k1 here, the rows above in the wide panel's trailing product
              const int r0 = q.wide > 0 ? k1 : 0;
              const int64_t ro = (int64_t)r0 * q.ld;
              gs.add(mr - r0, wo, w, q.mt_off + (int64_t)r0 * nb, nb, q.rt_off + k1, q.n, q.off + ro + k1, q.ld,
                     q.off + ro + k1, q.ld, 1, k0 - r0, k0 + w - r0);
            }
            U.steps.push_back(gs.args(OP_N, OP_N, 1, 0, 1, 0));
            U.vsteps.push_back(GemmList(gps, gps128, gpsoz).args(OP_N, OP_N, 1, 0, 1, 0));
            U.sdesc.push_back(GjStep{1, k0, k1});
          }
          // the wide panel's trailing product over the whole block, K = wo
          // banded leaf: rows >= k1 + wo + band untouched, pivot rows zero from column k1 + wo + 2 band
          auto bounds = [&](const GJProb& q, int wo, int& mr, int& nc) {
            mr = q.band > 0 ? std::min(q.n, k1 + wo + q.band) : q.n;
            nc = q.band > 0 ? std::min(q.n, k1 + wo + 2 * q.band) : q.n;
          };
          GemmList gs(gps, gps128, gpsoz);
          for (int k = 0; k < U.nl; ++k) {
            const GJProb& q = gl[k];
            if (q.n <= k1) continue;
            const int wo = std::min(nbo, q.n - k1);
            int mr, nc;
            bounds(q, wo, mr, nc);
            if (q.wide > 0 && k1 > 0) {
              // rows below k1 as before; the rows above, still untransformed in the wide panel's
              // columns, take (their wide-panel part) x (T R), formed first on the scratch: the wide
              // panel's transform of a non-pivot row is T = -P^{-1}, P its pivot block, and its pivot
              // rows hold P^{-1} in the wide panel's columns (moved to M rows k1..k1 + wo)
              const int64_t ro = (int64_t)k1 * q.ld;
              gs.add(mr - k1, nc, wo, q.mt_off + (int64_t)k1 * nbo, nbo, q.rt_off, q.n, q.off + ro, q.ld,
                     q.off + ro, q.ld, 1, 0, wo);
              gs.add(k1, nc, wo, q.mt_off, nbo, q.bp_off, q.n, q.off, q.ld, q.off, q.ld, 1);
            } else {
              gs.add(mr, nc, wo, q.mt_off, nbo, q.rt_off, q.n, q.off, q.ld, q.off, q.ld, 1, k1, k1 + wo);
            }
          }
          U.steps.push_back(gs.args(OP_N, OP_N, 1, 0, 1, 0));
          GemmList gv(gps, gps128, gpsoz);   // T R = -P^{-1} R
          for (int k = 0; k < U.nl; ++k) {
            const GJProb& q = gl[k];
            if (q.n <= k1 || q.wide <= 0 || k1 == 0) continue;
            const int wo = std::min(nbo, q.n - k1);
            int mr, nc;
            bounds(q, wo, mr, nc);
            gv.add(wo, nc, wo, q.mt_off + (int64_t)k1 * nbo, nbo, q.rt_off, q.n, q.bp_off, q.n);
          }
          U.vsteps.push_back(gv.args(OP_N, OP_N, -1, 0, 0, 0));
          U.sdesc.push_back(GjStep{2, k1, k1});
        }
      }
    }
  }

  // residual check: location of G_uv for every non-zero (u, v) (also the leaf bands below)
  std::vector<int64_t> rloc(h->col.size());
  for (int64_t u = 0; u < P.n; ++u)
    for (int64_t k = h->rowptr[u]; k < h->rowptr[u + 1]; ++k) {
      int64_t off = 0;
      if (!locate_pair(P, u, h->col[k], &off))
        return hsc_fail(h, HSC_ERR_ARG, "an H entry lies outside the selected pattern");
      rloc[k] = off >= 0 ? off : -off - 1;   // G^r is complex symmetric
    }

  // Leaf clusters (no children) are nobody's ancestors, so their diagonal blocks G_ii and G^<_ii
  // are read afterwards only at: the diagonal (outputs), the H neighbours of the residual check
  // (G^r), requested pairs inside the block, and, on a lesser leaf, every column of G_ii's contact
  // rows [c0, c1) (the lesser products). Per leaf and row, the first and last column read.
  const bool band = h->opt_leaf_band != 0;
  std::vector<std::vector<int>> gmin(nc), gmax(nc), pmin(nc), pmax(nc);
  std::vector<std::pair<int64_t, int>> aug_start;   // (block start, leaf)
  if (band) {
    for (int i = 0; i < nc; ++i) {
      const Cluster& c = P.cl[i];
      if (c.nchild != 0) continue;
      gmin[i].resize(c.n); gmax[i].resize(c.n); pmin[i].resize(c.n); pmax[i].resize(c.n);
      for (int r = 0; r < (int)c.n; ++r) gmin[i][r] = gmax[i][r] = pmin[i][r] = pmax[i][r] = r;
      aug_start.push_back({P.off[i].aug, i});
    }
    std::sort(aug_start.begin(), aug_start.end());
    // (row, column) of position p if it lies in a leaf's diagonal block
    auto in_leaf = [&](int64_t p, int& leaf, int& r, int& col) {
      auto it = std::upper_bound(aug_start.begin(), aug_start.end(), std::make_pair(p, nc));
      if (it == aug_start.begin()) return false;
      --it;
      const Cluster& c = P.cl[it->second];
      const int64_t w = c.n + c.m, q = p - it->first;
      if (q < 0 || q >= c.n * w || q % w >= c.n) return false;
      leaf = it->second;
      r = (int)(q / w);
      col = (int)(q % w);
      return true;
    };
    int lf, r, col;
    for (int64_t p : rloc)
      if (in_leaf(p, lf, r, col)) {
        gmin[lf][r] = std::min(gmin[lf][r], col);
        gmax[lf][r] = std::max(gmax[lf][r], col);
      }
    for (int64_t p : h->band_pairs)
      if (in_leaf(p, lf, r, col)) {
        gmin[lf][r] = std::min(gmin[lf][r], col);
        gmax[lf][r] = std::max(gmax[lf][r], col);
        pmin[lf][r] = std::min(pmin[lf][r], col);
        pmax[lf][r] = std::max(pmax[lf][r], col);
      }
  }
  // Rows [r0, r1) of a leaf's block per product: segments of <= 128 rows (cut also at c0 and c1
  // when whole contact rows are read), each with the column span [lo, hi) of the entries read.
  struct Band { int r0, r1, lo, hi; };
  auto bands = [&](int i, bool g) {
    std::vector<Band> out;
    const int n = (int)P.cl[i].n;
    const bool rows_whole = g && P.cl[i].lesser;   // lesser leaf: contact rows of G_ii entire
    const int c0 = rows_whole ? hc0[i] : n, c1 = rows_whole ? hc1[i] : n;
    const auto& mn = g ? gmin[i] : pmin[i];
    const auto& mx = g ? gmax[i] : pmax[i];
    int r0 = 0;
    while (r0 < n) {
      int r1 = std::min(n, r0 + 128);
      if (r0 < c0 && r1 > c0) r1 = c0;
      if (r0 >= c0 && r0 < c1) r1 = std::min(r1, c1);
      int lo = n, hi = 0;
      if (r0 >= c0 && r0 < c1) { lo = 0; hi = n; }
      else
        for (int r = r0; r < r1; ++r) { lo = std::min(lo, mn[r]); hi = std::max(hi, mx[r] + 1); }
      out.push_back(Band{r0, r1, lo, hi});
      r0 = r1;
    }
    return out;
  };
  // a lesser leaf without contact rows of its own reads its whole G_ii block (general lesser path)
  auto banded = [&](int i, bool g) {
    return band && P.cl[i].nchild == 0 && !(g && P.cl[i].lesser && !leafl[i]);
  };

  // downward levels
  d->down.assign(P.by_depth.size(), DownLevel());
  for (size_t dl = 0; dl < P.by_depth.size(); ++dl) {
    DownLevel& D = d->down[dl];
    const auto& ids = P.by_depth[dl];
    D.lc = (int64_t)lcs.size();
    D.nl = (int)ids.size();
    int64_t tz = 0, tn = 0;
    for (int i : ids) {
      LevelCluster L = base_lc(i);
      L.tz = tz; L.tn = tn; L.tt = 0; L.elem_start = 0;
      tz += (int64_t)L.m * L.m;
      tn += (int64_t)L.n * (L.n + L.m);
      D.max_sq = std::max(D.max_sq, (int64_t)L.m * L.m);
      D.any_lesser |= L.lesser != 0;
      D.gather_bytes += 2 * 32.0 * (double)L.m * L.m;
      lcs.push_back(L);
    }
    tz_max = std::max(tz_max, tz);
    tn_max = std::max(tn_max, tn);
    const LevelCluster* lv = lcs.data() + D.lc;
    GemmList g1(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      g1.add(L.n, L.m, L.m, L.x, L.m, L.tz, L.m, L.aug + L.n, L.n + L.m);
    }
    D.d[0] = g1.args(OP_N, OP_N, -1, 0, 0, 0);
    GemmList g2(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      const int64_t w = L.n + L.m;
      if (banded(ids[k], true))
        for (const Band& b : bands(ids[k], true))
          g2.add(b.r1 - b.r0, b.hi - b.lo, L.m, L.x + (int64_t)b.r0 * L.m, L.m, L.aug + L.n + b.lo * w, w,
                 L.aug + b.r0 * w + b.lo, w, L.aug + b.r0 * w + b.lo, w, 1);
      else
        g2.add(L.n, L.n, L.m, L.x, L.m, L.aug + L.n, w, L.aug, w, L.aug, w, 1);
    }
    D.d[1] = g2.args(OP_N, OP_T, -1, 0, 1, 0);
    GemmList g3(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      const int i = ids[k], c0 = hc0[i], w = hc1[i] - hc0[i];
      const int64_t ro = (int64_t)c0 * (L.n + L.m);
      if (!L.lesser) continue;
      if (leafl[i])
        g3.add(w, L.m, w, L.aug + ro + c0, L.n + L.m, L.aug + ro + L.n, L.n + L.m, L.tn + ro + L.n, L.n + L.m);
      else
        g3.add(L.n, L.m, L.n, L.aug, L.n + L.m, L.aug + L.n, L.n + L.m, L.tn + L.n, L.n + L.m);
    }
    D.d[2] = g3.args(OP_N, OP_C, 1, 0, 0, 0);
    GemmList g4(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      if (L.lesser && !leafl[ids[k]])   // L_iU = 0 on leaves
        g4.add(L.n, L.m, L.m, L.aug + L.n, L.n + L.m, L.tz, L.m, L.tn + L.n, L.n + L.m, L.tn + L.n, L.n + L.m, 1);
    }
    D.d[3] = g4.args(OP_N, OP_C, 1, 0, 1, 0);
    GemmList g5(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      const int i = ids[k], c0 = hc0[i], w = hc1[i] - hc0[i];
      const int64_t ro = (int64_t)c0 * (L.n + L.m);
      if (!L.lesser) continue;
      if (leafl[i])
        g5.add(w, L.n, w, L.aug + ro + c0, L.n + L.m, L.aug + ro, L.n + L.m, L.tn + ro, L.n + L.m);
      else
        g5.add(L.n, L.n, L.n, L.aug, L.n + L.m, L.aug, L.n + L.m, L.tn, L.n + L.m);
    }
    D.d[4] = g5.args(OP_N, OP_C, 1, 0, 0, 0);
    GemmList g6(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      if (L.lesser && !leafl[ids[k]])   // L_iU = 0 on leaves
        g6.add(L.n, L.n, L.m, L.aug + L.n, L.n + L.m, L.aug + L.n, L.n + L.m, L.tn, L.n + L.m, L.tn, L.n + L.m, 1);
    }
    D.d[5] = g6.args(OP_N, OP_H, 1, 0, 1, 0);
    GemmList g7(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      const int i = ids[k], c0 = hc0[i], w = hc1[i] - hc0[i];
      if (!L.lesser) continue;
      if (leafl[i] && banded(i, false)) {   // W = D^{-1}[:, c0:c1) N[c0:c1, :]: W_iU whole, W_ii banded
        const int64_t ld = L.n + L.m, nro = L.tn + (int64_t)c0 * ld;
        g7.add(L.n, L.m, w, L.aug + c0, ld, nro + L.n, ld, L.aug + L.n, ld);
        for (const Band& b : bands(i, false))
          g7.add(b.r1 - b.r0, b.hi - b.lo, w, L.aug + b.r0 * ld + c0, ld, nro + b.lo, ld, L.aug + b.r0 * ld + b.lo, ld);
      } else if (leafl[i])
        g7.add(L.n, L.n + L.m, w, L.aug + c0, L.n + L.m, L.tn + (int64_t)c0 * (L.n + L.m), L.n + L.m, L.aug,
               L.n + L.m);
      else
        g7.add(L.n, L.n + L.m, L.n, L.aug, L.n + L.m, L.tn, L.n + L.m, L.aug, L.n + L.m);
    }
    D.d[6] = g7.args(OP_N, OP_N, 1, 0, 0, 0);
    GemmList g8(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      g8.add(L.n, L.m, L.m, L.x, L.m, L.tz, L.m, L.aug + L.n, L.n + L.m, L.aug + L.n, L.n + L.m, L.lesser);
    }
    D.d[7] = g8.args(OP_N, OP_N, -1, 0, 1, 0);
    GemmList g9(gps, gps128, gpsoz);
    for (int k = 0; k < D.nl; ++k) {
      const auto& L = lv[k];
      const int64_t w = L.n + L.m;
      if (banded(ids[k], false))
        for (const Band& b : bands(ids[k], false))
          g9.add(b.r1 - b.r0, b.hi - b.lo, L.m, L.x + (int64_t)b.r0 * L.m, L.m, L.aug + L.n + b.lo * w, w,
                 L.aug + b.r0 * w + b.lo, w, L.aug + b.r0 * w + b.lo, w, L.lesser);
      else
        g9.add(L.n, L.n, L.m, L.x, L.m, L.aug + L.n, w, L.aug, w, L.aug, w, L.lesser);
    }
    D.d[8] = g9.args(OP_N, OP_H, 1, 0, 1, 0);
  }
  {
    int64_t pk = 1;
    int64_t oz = 0;
    d->any_oz = false;
    auto upd = [&](GemmPair& g) {
      pk = std::max(pk, g.tc.pack_words);
      if (d->fp64_engine == 1) g.oz_faster = false;
      if (d->fp64_engine == 2) g.oz_faster = g.oz.pack_blocks > 0;
      if (g.oz_faster) {
        oz = std::max(oz, oz_words(g.oz));
        d->any_oz = true;
      }
    };
    for (auto& U : d->up) {
      upd(U.u1); upd(U.u2); upd(U.u3); upd(U.u4);
      for (auto& st : U.steps) upd(st);
      for (auto& st : U.vsteps) upd(st);
    }
    for (auto& D : d->down)
      for (auto& g : D.d) upd(g);
    d->pk_es = (pk + 3) / 4 * 4;
    d->oz_es = (oz + 3) / 4 * 4;
  }
  d->tt_es = tt_max;
  d->tz_es = tz_max;
  d->tn_es = tn_max;
  d->gjt_es = gjt_max;

  // diag output offsets
  std::vector<int64_t> doff(P.n);
  for (int64_t u = 0; u < P.n; ++u) {
    int c = P.unk_cluster[u];
    int64_t l = P.unk_local[u];
    doff[u] = P.off[c].aug + l * (P.cl[c].n + P.cl[c].m) + l;
  }
  std::vector<c64> hv(h->val.size());
  for (size_t k = 0; k < hv.size(); ++k) hv[k] = make_double2(h->val[k].re, h->val[k].im);
  // contact slot of every unknown (residual check)
  std::vector<int32_t> uslot(P.n, -1);
  for (int64_t u = 0; u < P.n; ++u)
    uslot[u] = P.own_contact[P.own_off[P.unk_cluster[u]] + P.unk_local[u]];

  cudaError_t e = cudaSuccess;
#define UP(dst, v) if ((e = upload(d, dst, v)) != cudaSuccess) return hsc_fail(h, HSC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e))
  UP(&d->cg, cg);
  UP(&d->lcs, lcs);
  UP(&d->gjp, gjs);
  UP(&d->gjpi, gjs_in);
  UP(&d->gp, gps);
  UP(&d->gp128, gps128);
  UP(&d->gpoz, gpsoz);
  UP(&d->maps, P.map_child);
  UP(&d->h_rq, P.h_rq);
  UP(&d->h_vi, P.h_vi);
  UP(&d->hval, hv);
  UP(&d->own_contact, P.own_contact);
  UP(&d->u_owner, P.u_owner);
  UP(&d->u_local, P.u_local);
  UP(&d->u_seg, P.u_seg);
  UP(&d->posmap, P.posmap);
  UP(&d->doff, doff);
  UP(&d->res_rowptr, h->rowptr);
  UP(&d->res_loc, rloc);
  UP(&d->unk_slot, uslot);
  if (spc.empty()) spc.push_back(0);
  if (spr.empty()) spr.push_back(0);
  UP(&d->sp_colptr, spc);
  UP(&d->sp_rows, spr);
  {
    // DENSE contact blocks grouped by the upward level of their cluster
    std::vector<DenseBlock> db;
    for (size_t hl = 0; hl < d->up.size(); ++hl) {
      UpLevel& U = d->up[hl];
      U.dense0 = (int)db.size();
      for (const auto& D : P.dense) {
        if (P.cl[D.cluster].height != (int)hl) continue;
        DenseBlock b;
        b.aug = P.off[D.cluster].aug;
        b.blk = D.blk;
        b.loc = D.loc;
        b.ld = (int32_t)(P.cl[D.cluster].n + P.cl[D.cluster].m);
        b.nu = (int32_t)D.nu;
        b.lesser = P.cl[D.cluster].lesser ? 1 : 0;
        db.push_back(b);
        U.dense_max = std::max<int64_t>(U.dense_max, D.nu * D.nu);
      }
      U.dense_n = (int)db.size() - U.dense0;
    }
    UP(&d->dense_dev, db);
    UP(&d->dense_loc, P.dense_local);
  }
#undef UP
  if ((e = cudaMalloc((void**)&d->flag, 4 * sizeof(int))) != cudaSuccess)
    return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc flag");
  d->fixed.push_back(d->flag);
  // patch problem-list pointers
  auto patch = [&](GemmPair& g) {
    g.z.probs = d->gp + reinterpret_cast<size_t>(g.z.probs);
    g.tc.probs = d->gp128 + reinterpret_cast<size_t>(g.tc.probs);
    g.oz.probs = d->gpoz + reinterpret_cast<size_t>(g.oz.probs);
  };
  for (auto& U : d->up) {
    patch(U.u1); patch(U.u2); patch(U.u3); patch(U.u4);
    for (auto& s : U.steps) patch(s);
    for (auto& s : U.vsteps) patch(s);
  }
  for (auto& D : d->down)
    for (auto& g : D.d) patch(g);
  d->planned = true;
  return HSC_OK;
}

// pack-buffer words per energy a solve in this precision needs (0: no pack buffer)
int64_t pack_words_needed(const DeviceState* d, int precision) {
  int64_t w = d->any_oz ? d->oz_es : 0;   // the emulation runs in both precisions (FP64 levels)
  if (precision == HSC_MIXED && d->use_pack) w = std::max(w, d->pk_es);
  return w;
}

int64_t bytes_per_energy(const DeviceState* d, int64_t pack_words = 0) {
  int64_t c = 4 * d->aug_es + 2 * d->sq_es + d->x_es + d->tt_es + 3 * d->tz_es + d->tn_es + d->gjt_es;
  return c * (int64_t)sizeof(c64) + d->piv_es * 4 + pack_words * 4;
}

int ensure_arena(hsc_ctx* h, int64_t want, int64_t pack_words) {
  DeviceState* d = h->dev;
  if (d->cap >= want && d->pk_cur >= pack_words) return HSC_OK;
  want = std::max(want, d->cap);
  pack_words = std::max(pack_words, d->pk_cur);
  if (d->arena) { cudaFree(d->arena); d->arena = nullptr; d->arena_bytes = 0; }
  d->cap = 0;
  d->pk_cur = 0;
  d->PK = nullptr;
  size_t bytes = (size_t)bytes_per_energy(d, pack_words) * want + 64 * 256;
  char* p;
  if (d->borrow) {
    if (bytes > d->borrow_bytes)
      return hsc_fail(h, HSC_ERR_OOM, "borrowed workspace too small (" + std::to_string(bytes >> 20) + " MiB)");
    p = (char*)d->borrow;
  } else {
    cudaError_t e = cudaMalloc(&d->arena, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc workspace (" + std::to_string(bytes >> 20) + " MiB)");
    }
    d->arena_bytes = bytes;
    p = (char*)d->arena;
  }
  auto take = [&](int64_t elems, size_t esz) {
    char* r = p;
    p += ((size_t)elems * want * esz + 255) / 256 * 256;
    return r;
  };
  d->F = (c64*)take(d->aug_es, 16);
  d->L = (c64*)take(d->aug_es, 16);
  d->G = (c64*)take(d->aug_es, 16);
  d->P = (c64*)take(d->aug_es, 16);
  d->S = (c64*)take(d->sq_es, 16);
  d->LS = (c64*)take(d->sq_es, 16);
  d->X = (c64*)take(d->x_es, 16);
  d->T = (c64*)take(d->tt_es, 16);
  d->Z = (c64*)take(d->tz_es, 16);
  d->GUU = (c64*)take(d->tz_es, 16);
  d->PUU = (c64*)take(d->tz_es, 16);
  d->N = (c64*)take(d->tn_es, 16);
  d->GJT = (c64*)take(d->gjt_es, 16);
  d->piv = (int32_t*)take(d->piv_es, 4);
  d->PK = pack_words > 0 ? (uint32_t*)take(pack_words, 4) : nullptr;
  d->pk_cur = pack_words;
  d->cap = want;
  return HSC_OK;
}

GemmArgs bind(GemmArgs g, const c64* A, int64_t aes, const c64* B, int64_t bes, c64* C, int64_t ces,
              const c64* D, int64_t des) {
  g.A = A; g.a_es = aes; g.B = B; g.b_es = bes; g.C = C; g.c_es = ces; g.D = D; g.d_es = des;
  return g;
}

cudaError_t prof_start(DeviceState* d, cudaStream_t s) {
  Prof& p = d->prof;
  if (!p.on) return cudaSuccess;
  if (2 * (p.used + 1) > p.pool.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      p.pool.push_back(e);
    }
  }
  return cudaEventRecord(p.pool[2 * p.used], s);
}

cudaError_t prof_stop(DeviceState* d, cudaStream_t s, int cls, int nk, double flops, double bytes) {
  Prof& p = d->prof;
  p.launches[cls] += nk;
  if (!p.on) return cudaSuccess;
  cudaError_t err = cudaEventRecord(p.pool[2 * p.used + 1], s);
  p.cls.push_back(cls);
  p.flops.push_back(flops);
  p.bytes.push_back(bytes);
  ++p.used;
  return err;
}

#define LAUNCH(cls, nk, fl, by, call)                 \
  do {                                                \
    CK(prof_start(d, s));                             \
    CK(call);                                         \
    CK(prof_stop(d, s, cls, nk, fl, by));             \
  } while (0)

// One wave of `ne` energies with inputs already on the device.
int run_wave(hsc_ctx* h, int ne, const double* E, double eta, const c64* sr, const c64* sl,
             int64_t npair, const int64_t* poff, c64* ogr, c64* ogl, c64* pgr, c64* pgl,
             int precision, cudaStream_t s) {
  DeviceState* d = h->dev;
  const bool les = sl != nullptr;
  const int64_t ncs = h->n_contact_unknowns;
  // ---- upward (Algorithm 1 first loop, Algorithm 2 fold) ----
  bool tc = false;   // current level's GEMMs on the tensor cores (mixed mode, below the top levels)
  bool schur = false;   // the launch is Algorithm 1's Schur update (profiled separately)
  bool gjup = false;    // the launch is a Gauss-Jordan trailing update (profiled separately)
  auto gemm = [&](const GemmPair& pr, const GemmArgs& gz, const GemmArgs& gt, const GemmArgs& go) -> int {
    if (gz.total_tiles <= 0) return HSC_OK;
    if (tc && d->PK && d->use_pack)
      LAUNCH(gjup ? K_GJU_TC : schur ? K_SCHUR_TC : K_GEMM_TC, 2, gt.flops * ne, 0.0,
             gemm_tc_packed(gt, ne, d->PK, d->pk_cur, d->flag + 2, s));
    else if (tc) LAUNCH(gjup ? K_GJU_TC : schur ? K_SCHUR_TC : K_GEMM_TC, 1, gt.flops * ne, 0.0, gemm_tc(gt, ne, d->flag + 2, s));
    else if (pr.oz_faster && d->PK && oz_words(go) <= d->pk_cur)
      LAUNCH(gjup ? K_GJU_OZ : schur ? K_SCHUR_OZ : K_GEMM_OZ, 2, go.flops * ne, 0.0,
             gemm_oz(go, ne, reinterpret_cast<uint16_t*>(d->PK), 2 * d->pk_cur,
                     reinterpret_cast<double*>(d->PK + oz_scale_word(go)), d->pk_cur / 2, d->flag + 2, s));
    else LAUNCH(gjup ? K_GJU : schur ? K_SCHUR : K_GEMM, 1, gz.flops * ne, 0.0, gemm_z(gz, ne, s, d->four_products));
    return HSC_OK;
  };
#define GEMM(pair, ...)                                                                          \
  do {                                                                                           \
    int _r = gemm((pair), bind((pair).z, __VA_ARGS__), bind((pair).tc, __VA_ARGS__),             \
                  bind((pair).oz, __VA_ARGS__));                                                 \
    if (_r != HSC_OK) return _r;                                                                 \
  } while (0)
  const int nup = (int)d->up.size();
  for (int hl = 0; hl < nup; ++hl) {
    auto& U = d->up[hl];
    tc = precision == HSC_MIXED && hl < nup - d->fp64_levels;
    const LevelCluster* lc = d->lcs + U.lc;
    LAUNCH(K_ASSEMBLE, 1, 0.0, U.asm_bytes * ne,
           launch_assemble(lc, U.nl, U.total, d->cg, d->maps, d->F, d->S, d->L, d->LS, d->aug_es,
                           d->sq_es, ne, les ? 1 : 0, s));
    LAUNCH(K_ADD_A, 2, 0.0, 0.0,
           launch_add_a(lc, U.nl, U.max_h, U.max_n, d->h_rq, d->h_vi, d->hval, d->own_contact, E,
                        eta, sr, sl, ncs, d->F, d->L, d->aug_es, ne, s));
    if (d->dense_r && U.dense_n > 0)
      LAUNCH(K_ADD_A, 1, 0.0, 0.0,
             launch_add_dense(d->dense_dev + U.dense0, U.dense_n, U.dense_max, d->dense_loc,
                              d->dense_r + d->dense_e0 * d->dense_es,
                              (les && d->dense_l) ? d->dense_l + d->dense_e0 * d->dense_es : nullptr,
                              d->dense_es, d->F, d->L, d->aug_es, ne, s));
    // Gauss-Jordan inversion of A_ii in place (D_i^{-1}), panel by panel
    const GJProb* gp = d->gjp + U.gj;
    const GJProb* gpi = d->gjpi ? d->gjpi + U.gji : nullptr;
    for (size_t st = 0; st < U.steps.size(); ++st) {
      const GjStep& sd = U.sdesc[st];
      const int k0 = sd.k0;
      if (sd.kind == 2) {   // the wide panel, reduced by its nested steps: move, swap, product
        LAUNCH(K_GJ_SWAP, 1, 0.0, 0.0,
               launch_gj_move(gp, U.nmat, U.max_n, d->F, d->aug_es, d->GJT, d->GJT, d->gjt_es, k0, d->nbo,
                              ne, s));
        LAUNCH(K_GJ_SWAP, 1, 0.0, 0.0,
               launch_gj_swap(gp, U.nmat, U.max_n, d->F, d->aug_es, d->piv, d->piv_es, d->GJT,
                              d->gjt_es, k0, d->nbo, ne, s));
      } else {
        const GJProb* g = sd.kind == 1 ? gpi : gp;
        LAUNCH(K_GJ_PANEL, 1, 0.0, 0.0,
               launch_gj_panel(g, U.nmat, d->F, d->aug_es, d->piv, d->piv_es, d->GJT, d->GJT,
                               d->gjt_es, k0, d->nb, ne, d->flag, s, d->gj_cluster));
        LAUNCH(K_GJ_SWAP, 1, 0.0, 0.0,
               launch_gj_swap(g, U.nmat, U.max_n, d->F, d->aug_es, d->piv, d->piv_es, d->GJT,
                              d->gjt_es, k0, d->nb, ne, s, sd.kind == 1 ? sd.k1 : 0,
                              sd.kind == 1 ? sd.k1 + d->nbo : 1 << 30));
      }
      const bool keep = tc;
      tc = tc && !d->gj_fp64;
      gjup = true;
      if (sd.kind == 2)   // T R before the trailing product reads it
        GEMM(U.vsteps[st], d->GJT, d->gjt_es, d->GJT, d->gjt_es, d->GJT, d->gjt_es, nullptr, 0);
      GEMM(U.steps[st], d->GJT, d->gjt_es, d->GJT, d->gjt_es, d->F, d->aug_es, d->F, d->aug_es);
      gjup = false;
      tc = keep;
    }
    LAUNCH(K_GJ_PERM, 1, 0.0, 0.0,
           launch_gj_colperm(gp, U.nmat, U.max_n, d->F, d->aug_es, d->piv, d->piv_es, ne, s,
                             d->growth_wave, d->cond_wave ? d->cond_wave + U.gj : nullptr, d->ncl));
    GEMM(U.u1, d->F, d->aug_es, d->F, d->aug_es, d->X, d->x_es, nullptr, 0);
    if (U.sp_count > 0)
      LAUNCH(K_LEAF, 1, 0.0, 0.0,
             launch_leaf_x(lc, U.nl, U.max_n, d->sp_colptr, d->sp_rows, d->F, d->aug_es, d->X, d->x_es, ne, s));
    schur = true;
    GEMM(U.u2, d->F, d->aug_es, d->X, d->x_es, d->S, d->sq_es, d->S, d->sq_es);
    schur = false;
    if (U.sp_count > 0)
      LAUNCH(K_LEAF, 1, 0.0, 0.0,
             launch_leaf_schur(lc, U.nl, U.sp_max_m, d->sp_colptr, d->sp_rows, d->F, d->aug_es, d->X, d->x_es,
                               d->S, d->sq_es, ne, s));
    if (les && U.any_lesser) {
      GEMM(U.u3, d->L, d->aug_es, d->X, d->x_es, d->T, d->tt_es, d->L, d->aug_es);
      GEMM(U.u4, d->X, d->x_es, d->T, d->tt_es, d->Z, d->tz_es, nullptr, 0);
      LAUNCH(K_FOLD, 1, 0.0, 0.0, launch_fold(lc, U.nl, U.max_sq, d->LS, d->sq_es, d->Z, d->tz_es, ne, s));
    }
  }
  // ---- downward (Algorithm 1 second loop, Algorithm 2 second loop) ----
  const int ndown = (int)d->down.size();
  for (int dl = 0; dl < ndown; ++dl) {
    auto& D = d->down[dl];
    tc = precision == HSC_MIXED && dl >= d->fp64_levels;
    const LevelCluster* lc = d->lcs + D.lc;
    if (D.max_sq > 0)
      LAUNCH(K_GATHER, 1, 0.0, D.gather_bytes * ne * (les ? 1.0 : 0.5),
             launch_gather(lc, D.nl, D.max_sq, d->cg, d->u_owner, d->u_local, d->u_seg, d->posmap,
                           d->G, d->P, d->aug_es, d->GUU, les ? d->PUU : nullptr, d->tz_es, ne,
                           d->flag + 1, s));
    GEMM(D.d[0], d->X, d->x_es, d->GUU, d->tz_es, d->G, d->aug_es, nullptr, 0);
    GEMM(D.d[1], d->X, d->x_es, d->G, d->aug_es, d->G, d->aug_es, d->F, d->aug_es);
    if (!les) continue;
    if (D.any_lesser) {
      GEMM(D.d[2], d->L, d->aug_es, d->G, d->aug_es, d->N, d->tn_es, nullptr, 0);
      GEMM(D.d[3], d->L, d->aug_es, d->GUU, d->tz_es, d->N, d->tn_es, d->N, d->tn_es);
      GEMM(D.d[4], d->L, d->aug_es, d->G, d->aug_es, d->N, d->tn_es, nullptr, 0);
      GEMM(D.d[5], d->L, d->aug_es, d->G, d->aug_es, d->N, d->tn_es, d->N, d->tn_es);
      GEMM(D.d[6], d->F, d->aug_es, d->N, d->tn_es, d->P, d->aug_es, nullptr, 0);
    }
    GEMM(D.d[7], d->X, d->x_es, d->PUU, d->tz_es, d->P, d->aug_es, d->P, d->aug_es);
    GEMM(D.d[8], d->X, d->x_es, d->P, d->aug_es, d->P, d->aug_es, d->P, d->aug_es);
  }
#undef GEMM
  if (d->resid_wave && !d->dense_r)   // the residual kernel knows diagonal self-energies only
    LAUNCH(K_RESID, 1, 0.0, 0.0,
           launch_residual(h->n, d->res_rowptr, d->hval, d->res_loc, d->doff, d->unk_slot, E, eta, sr,
                           ncs, d->G, d->aug_es, d->resid_wave, ne, s));
  LAUNCH(K_OUT, npair > 0 ? 2 : 1, 0.0, 32.0 * (double)(h->n + npair) * ne * (les ? 2 : 1),
         launch_out(d->doff, h->n, poff, npair, d->G, d->P, d->aug_es, ogr, les ? ogl : nullptr, pgr,
                    les ? pgl : nullptr, ne, s));
  return HSC_OK;
}

// locate a requested pair in the stored G blocks; negative = transposed source (-off-1)
int locate_pair(const Plan& P, int64_t a, int64_t b, int64_t* out) {
  int ca = P.unk_cluster[a], cb = P.unk_cluster[b];
  int64_t la = P.unk_local[a], lb = P.unk_local[b];
  auto anc = [&](int x, int i) { return P.cl[x].first_desc <= i && i < x; };
  auto upos = [&](int i, int64_t u) -> int64_t {
    // position of unknown u in U_i (unknown granularity)
    int64_t base = P.u_off[i], m = P.cl[i].m;
    int c = P.unk_cluster[u];
    int64_t l = P.unk_local[u];
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      int oc = P.u_owner[base + mid];
      int64_t ol = P.u_local[base + mid];
      if (oc < c || (oc == c && ol < l)) lo = mid + 1;
      else hi = mid;
    }
    if (lo < m && P.u_owner[base + lo] == c && P.u_local[base + lo] == l) return lo;
    return -1;
  };
  if (ca == cb) { *out = P.off[ca].aug + la * (P.cl[ca].n + P.cl[ca].m) + lb; return 1; }
  if (anc(cb, ca)) {
    int64_t k = upos(ca, b);
    if (k < 0) return 0;
    *out = P.off[ca].aug + la * (P.cl[ca].n + P.cl[ca].m) + P.cl[ca].n + k;
    return 1;
  }
  if (anc(ca, cb)) {
    int64_t k = upos(cb, a);
    if (k < 0) return 0;
    *out = -(P.off[cb].aug + lb * (P.cl[cb].n + P.cl[cb].m) + P.cl[cb].n + k) - 1;
    return 1;
  }
  return 0;
}

int64_t budget_bytes() {
  const char* env = getenv("HSC_WORKSPACE_GB");
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  int64_t avail = (int64_t)(fr * 0.85) - ((int64_t)2 << 30);
  if (env) {
    int64_t want = (int64_t)(atof(env) * (double)(1 << 30));
    return std::min(want, avail);
  }
  return avail;
}

}  // namespace
}  // namespace hsc

using namespace hsc;

namespace hsc {
namespace {

// Creates the handle's device state on the current device with the handle's options (no schedule).
int new_state(hsc_ctx* h) {
  h->dev = new DeviceState();
  CK(cudaGetDevice(&h->dev->device));
  h->dev->nb = h->opt_nb;
  h->dev->nbo = (h->opt_nbo / h->opt_nb) * h->opt_nb;   // a multiple of the panel width
  if (h->dev->nbo <= h->opt_nb) h->dev->nbo = 0;
  h->dev->fp64_levels = h->opt_fp64_levels;
  h->dev->gj_fp64 = h->opt_gj_fp64 != 0;
  h->dev->four_products = h->opt_4m != 0;
  h->dev->fp64_engine = h->opt_fp64_engine;
  if (const char* v = getenv("HSC_FP64_ENGINE")) h->dev->fp64_engine = atoi(v);
  if (const char* v = getenv("HSC_GJ_CLUSTER")) h->dev->gj_cluster = atoi(v);
  if (h->dev->gj_cluster != 1 && h->dev->gj_cluster != 2 && h->dev->gj_cluster != 4) h->dev->gj_cluster = 0;
  if (const char* v = getenv("HSC_FP64_LEVELS")) h->dev->fp64_levels = atoi(v);
  if (const char* v = getenv("HSC_MIXED_GJ_FP64")) h->dev->gj_fp64 = atoi(v) != 0;
  if (const char* v = getenv("HSC_TC_PACK")) h->dev->use_pack = atoi(v) != 0;
  return HSC_OK;
}

// Creates the device state (applying the handle's options) and the device schedule.
int get_state(hsc_ctx* h) {
  if (!h->dev) {
    int rc = new_state(h);
    if (rc != HSC_OK) return rc;
  }
  DeviceState* d = h->dev;
  int cur = 0;
  CK(cudaGetDevice(&cur));
  if (cur != d->device) return hsc_fail(h, HSC_ERR_ARG, "current device differs from the handle's device");
  if (!d->planned) {
    int rc;
    try {
      rc = build_schedule(h);
    } catch (const std::exception& ex) {
      return hsc_fail(h, HSC_ERR_ARG, std::string("schedule: ") + ex.what());
    }
    if (rc != HSC_OK) return rc;
  }
  return HSC_OK;
}

int check_common(hsc_ctx* h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                 const hsc_c128* sigma_less, int32_t precision, int32_t n_req,
                 const int32_t* req_pairs, const hsc_c128* diag_gr, const hsc_c128* diag_gl,
                 const hsc_c128* req_gr, const hsc_c128* req_gl) {
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  if (n_E < 0 || (!E && n_E > 0)) return hsc_fail(h, HSC_ERR_ARG, "bad energy array");
  if (n_E > 0 && !diag_gr) return hsc_fail(h, HSC_ERR_ARG, "diag_gr is NULL");
  if (sigma_less && !diag_gl) return hsc_fail(h, HSC_ERR_ARG, "diag_gl is NULL");
  if (h->n_contact_unknowns > 0 && !sigma_r) return hsc_fail(h, HSC_ERR_ARG, "sigma_r is NULL");
  if (n_req < 0 || (n_req > 0 && (!req_pairs || !req_gr || (sigma_less && !req_gl))))
    return hsc_fail(h, HSC_ERR_ARG, "bad requested-pair arrays");
  if (precision != HSC_FP64 && precision != HSC_MIXED)
    return hsc_fail(h, HSC_ERR_ARG, "precision must be HSC_FP64 or HSC_MIXED");
  if (!(eta >= 0.0)) return hsc_fail(h, HSC_ERR_ARG, "eta must be >= 0");
  return HSC_OK;
}

// Locates the requested pairs and copies their source offsets into a persistent device buffer.
int upload_pairs(hsc_ctx* h, int32_t n_req, const int32_t* req_pairs) {
  std::vector<int64_t> poff(n_req);
  std::vector<int64_t> in_leaf;   // positions of the pairs inside a leaf's diagonal block
  for (int k = 0; k < n_req; ++k) {
    int64_t a = req_pairs[2 * k], b = req_pairs[2 * k + 1];
    if (a < 0 || a >= h->n || b < 0 || b >= h->n) return hsc_fail(h, HSC_ERR_ARG, "pair index out of range");
    if (!locate_pair(h->plan, a, b, &poff[k]))
      return hsc_fail(h, HSC_ERR_NOT_SELECTED, "pair (" + std::to_string(a) + "," + std::to_string(b) +
                                                   ") is outside the filled pattern");
    const int ca = h->plan.unk_cluster[a];
    if (ca == h->plan.unk_cluster[b] && h->plan.cl[ca].nchild == 0)
      in_leaf.push_back(poff[k] >= 0 ? poff[k] : -poff[k] - 1);
  }
  std::sort(in_leaf.begin(), in_leaf.end());
  in_leaf.erase(std::unique(in_leaf.begin(), in_leaf.end()), in_leaf.end());
  if (h->opt_leaf_band && in_leaf != h->band_pairs) {
    // the leaves' column bands must cover these entries: rebuild the schedule with them
    h->band_pairs = in_leaf;
    device_state_free(h->dev);
    h->dev = nullptr;
    int rc = get_state(h);
    if (rc != HSC_OK) return rc;
  }
  DeviceState* d = h->dev;
  if (n_req > d->pair_cap) {
    if (d->poff) cudaFree(d->poff);
    d->poff = nullptr;
    d->pair_cap = 0;
    if (cudaMalloc((void**)&d->poff, (size_t)n_req * sizeof(int64_t)) != cudaSuccess) {
      cudaGetLastError();
      return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc pair offsets");
    }
    d->pair_cap = n_req;
  }
  if (n_req > 0) CK(cudaMemcpy(d->poff, poff.data(), n_req * sizeof(int64_t), cudaMemcpyHostToDevice));
  return HSC_OK;
}

// Uploads, once per device state, the unknown and the contact id of every contact slot.
int ensure_slots(hsc_ctx* h) {
  DeviceState* d = h->dev;
  if (d->slot_unknown || h->n_contact_unknowns == 0) return HSC_OK;
  std::vector<int64_t> su;
  std::vector<int32_t> sc;
  for (int c = 0; c < h->n_contacts; ++c)
    for (int64_t k = h->contact_ptr[c]; k < h->contact_ptr[c + 1]; ++k)
      for (int o = 0; o < h->orb; ++o) {
        su.push_back((int64_t)h->contact_sites[k] * h->orb + o);
        sc.push_back(c);
      }
  cudaError_t e = upload(d, &d->slot_unknown, su);
  if (e == cudaSuccess) e = upload(d, &d->slot_contact, sc);
  // upload() also lists them in `fixed`; device_state_free frees them by name
  while (!d->fixed.empty() && (d->fixed.back() == d->slot_unknown || d->fixed.back() == d->slot_contact))
    d->fixed.pop_back();
  if (e != cudaSuccess) {
    if (d->slot_unknown) cudaFree(d->slot_unknown);
    if (d->slot_contact) cudaFree(d->slot_contact);
    d->slot_unknown = nullptr;
    d->slot_contact = nullptr;
    cudaGetLastError();
    return hsc_fail(h, HSC_ERR_CUDA, "upload contact slots");
  }
  return HSC_OK;
}

// Sizes (and allocates) the workspace for waves of at most `wave` energies.
int prepare_arena(hsc_ctx* h, int64_t n_E, int64_t byte_cap, int64_t* wave_out, int precision) {
  DeviceState* d = h->dev;
  const int64_t pack = pack_words_needed(d, precision);
  const int64_t per = bytes_per_energy(d, pack);
  if (d->borrow) byte_cap = std::min<int64_t>(byte_cap, (int64_t)d->borrow_bytes - 64 * 256);
  int64_t wave = std::min<int64_t>(n_E, std::max<int64_t>(byte_cap / per, 0));
  if (d->cap > 0) wave = std::max<int64_t>(std::min<int64_t>(n_E, d->cap), wave);
  if (wave <= 0) return hsc_fail(h, HSC_ERR_OOM, "one energy needs " + std::to_string(per >> 20) + " MiB of workspace");
  wave = std::min<int64_t>(wave, 65535);
  int rc = ensure_arena(h, wave, pack);
  if (rc != HSC_OK) return rc;
  *wave_out = wave;
  return HSC_OK;
}

// Sizes the per-energy growth record for a solve of n_E energies (before any capture).
int ensure_growth(hsc_ctx* h, int64_t n_E) {
  DeviceState* d = h->dev;
  if (d->growth_cap < n_E) {
    if (d->growth) cudaFree(d->growth);
    d->growth = nullptr;
    d->growth_cap = 0;
    cudaError_t e = cudaMalloc((void**)&d->growth,
                               (2 + (int64_t)d->ncl) * std::max<int64_t>(n_E, 1) * sizeof(float));
    if (e != cudaSuccess) { cudaGetLastError(); return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc growth"); }
    d->growth_cap = std::max<int64_t>(n_E, 1);
  }
  d->resid = d->growth + d->growth_cap;
  d->cond = d->resid + d->growth_cap;
  d->growth_n = n_E;
  return HSC_OK;
}

// Enqueues all waves of a device-resident solve on stream s (no host synchronisation).
int enqueue_device(hsc_ctx* h, int64_t n_E, int64_t wave, const double* E, double eta,
                   const hsc_c128* sigma_r, const hsc_c128* sigma_less, int32_t precision,
                   int32_t n_req, hsc_c128* diag_gr, hsc_c128* diag_gl, hsc_c128* req_gr,
                   hsc_c128* req_gl, cudaStream_t s) {
  DeviceState* d = h->dev;
  const int64_t n = h->n, ncs = h->n_contact_unknowns;
  CK(cudaMemsetAsync(d->flag, 0, 4 * sizeof(int), s));
  CK(cudaMemsetAsync(d->growth, 0, n_E * sizeof(float), s));
  CK(cudaMemsetAsync(d->resid, 0, n_E * sizeof(float), s));
  for (int64_t e0 = 0; e0 < n_E; e0 += wave) {
    const int ne = (int)std::min<int64_t>(wave, n_E - e0);
    d->growth_wave = d->growth + e0;
    d->resid_wave = d->resid + e0;
    d->cond_wave = d->cond + e0 * d->ncl;
    d->dense_e0 = e0;
    const c64* dsr = sigma_r ? reinterpret_cast<const c64*>(sigma_r) + e0 * ncs : nullptr;
    const c64* dsl = sigma_less ? reinterpret_cast<const c64*>(sigma_less) + e0 * ncs : nullptr;
    c64* ogr = reinterpret_cast<c64*>(diag_gr) + e0 * n;
    c64* ogl = diag_gl ? reinterpret_cast<c64*>(diag_gl) + e0 * n : nullptr;
    c64* pgr = req_gr ? reinterpret_cast<c64*>(req_gr) + e0 * n_req : nullptr;
    c64* pgl = req_gl ? reinterpret_cast<c64*>(req_gl) + e0 * n_req : nullptr;
    int rc = run_wave(h, ne, E + e0, eta, dsr, dsl, n_req, d->poff, ogr, ogl, pgr, pgl, precision, s);
    if (rc != HSC_OK) return rc;
  }
  return HSC_OK;
}

int read_flags(hsc_ctx* h, cudaStream_t s) {
  int flags[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(flags, h->dev->flag, sizeof(flags), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags[1]) return hsc_fail(h, HSC_ERR_ARG, "internal gather map error");
  if (flags[2]) return hsc_fail(h, HSC_ERR_TIMEOUT, "a tensor-core GEMM wait expired");
  if (flags[0]) return hsc_fail(h, HSC_ERR_SINGULAR, "zero pivot in a cluster block");
  return HSC_OK;
}

}  // namespace
}  // namespace hsc

namespace hsc {
namespace {

// Energies whose residual |(A G^r - I)_uu| exceeds the handle's threshold are solved again on the
// alternate separator tree v; per energy, the result of the tree with the smaller residual is kept
// (outputs and both records overwritten in place). Inputs and outputs are where the caller's
// hsc_solve had them.
int resolve_grown(int v, hsc_ctx* h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                  const hsc_c128* sigma_less, int32_t precision, int32_t n_req, const int32_t* req_pairs,
                  hsc_c128* diag_gr, hsc_c128* diag_gl, hsc_c128* req_gr, hsc_c128* req_gl,
                  cudaStream_t s, bool dev_io) {
  DeviceState* d = h->dev;
  std::vector<float> r(n_E);
  CK(cudaMemcpyAsync(r.data(), d->resid, n_E * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const float thr = (float)std::pow(10.0, -h->opt_resolve);
  std::vector<int64_t> J;
  for (int64_t k = 0; k < n_E; ++k)
    if (!(r[k] <= thr)) J.push_back(k);
  if (J.empty()) return HSC_OK;
  hsc_ctx* a = hsc_alt(h, v);
  if (!a || get_state(a) != HSC_OK) return HSC_OK;   // no alternate tree: the results so far stand
  {
    // the main solve is complete on this stream, so its workspace holds nothing live: the alternate
    // tree works in it (several alternates could not each own a workspace of that size)
    DeviceState* ad = a->dev;
    if (hsc_profile(a, d->prof.on ? 1 : 0) != HSC_OK) return HSC_OK;   // profile with the main handle
    if (ad->arena) { cudaFree(ad->arena); ad->arena = nullptr; ad->arena_bytes = 0; }
    ad->borrow = d->arena;
    ad->borrow_bytes = d->arena_bytes;
    ad->cap = 0;
    ad->pk_cur = 0;
    ad->PK = nullptr;
  }
  const int64_t nj = (int64_t)J.size(), n = h->n, ncs = h->n_contact_unknowns;
  const bool les = sigma_less != nullptr;
  const int64_t nq = n_req;
  // staging: E, Sigma^r, Sigma^< in; diag G^r, diag G^<, pairs out (host or device, as the caller's)
  const size_t bytes = nj * (8 + 16 * (ncs * (les ? 2 : 1) + (n + nq) * (les ? 2 : 1))) + 8 * 256;
  std::vector<char> hbuf;
  char* base;
  if (dev_io) {
    if (d->rs_cap < bytes) {
      if (d->rs_buf) cudaFree(d->rs_buf);
      d->rs_buf = nullptr;
      d->rs_cap = 0;
      cudaError_t e = cudaMalloc(&d->rs_buf, bytes);
      if (e != cudaSuccess) { cudaGetLastError(); return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc re-solve staging"); }
      d->rs_cap = bytes;
    }
    base = (char*)d->rs_buf;
  } else {
    hbuf.resize(bytes);
    base = hbuf.data();
  }
  char* p = base;
  auto take = [&](int64_t b) { char* r = p; p += (b + 255) / 256 * 256; return r; };
  double* sE = (double*)take(nj * 8);
  hsc_c128* ssr = (hsc_c128*)take(nj * ncs * 16);
  hsc_c128* ssl = les ? (hsc_c128*)take(nj * ncs * 16) : nullptr;
  hsc_c128* sgr = (hsc_c128*)take(nj * n * 16);
  hsc_c128* sgl = les ? (hsc_c128*)take(nj * n * 16) : nullptr;
  hsc_c128* spr = nq ? (hsc_c128*)take(nj * nq * 16) : nullptr;
  hsc_c128* spl = (nq && les) ? (hsc_c128*)take(nj * nq * 16) : nullptr;
  const cudaMemcpyKind kind = dev_io ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToHost;
  int rc = HSC_OK;
  auto copy = [&](void* dst, const void* src, size_t b) -> bool {
    if (b == 0) return true;
    if (!dev_io) { std::memcpy(dst, src, b); return true; }
    return cudaMemcpyAsync(dst, src, b, kind, s) == cudaSuccess;
  };
  for (int64_t j = 0; j < nj && rc == HSC_OK; ++j) {
    const int64_t k = J[j];
    bool ok = copy(sE + j, E + k, 8) && copy(ssr + j * ncs, sigma_r + k * ncs, ncs * 16);
    if (les) ok = ok && copy(ssl + j * ncs, sigma_less + k * ncs, ncs * 16);
    if (!ok) rc = hsc_fail(h, HSC_ERR_CUDA, "re-solve gather");
  }
  const int src = rc == HSC_OK ? hsc_solve(a, nj, sE, eta, ncs ? ssr : nullptr, ssl, precision, n_req, req_pairs,
                                           sgr, sgl, spr, spl, s, dev_io ? 1 : 0) : -1;
  if (rc == HSC_OK && src == HSC_OK) {
    {   // the alternate's kernels count in the main handle's profile
      int32_t nc = 0;
      hsc_kernel_stat st[K_NCLASS];
      if (hsc_profile_read(a, st, K_NCLASS, &nc) == HSC_OK)
        for (int c = 0; c < nc && c < K_NCLASS; ++c) {
          hsc_kernel_stat& x = d->prof.extra[c];
          x.launches += st[c].launches;
          x.timed += st[c].timed;
          x.ms += st[c].ms;
          x.flops += st[c].flops;
          x.bytes += st[c].bytes;
        }
    }
    std::vector<double> ra(nj), ga(nj);
    if (hsc_residual(a, nj, ra.data()) == HSC_OK && hsc_growth(a, nj, ga.data()) == HSC_OK) {
      for (int64_t j = 0; j < nj && rc == HSC_OK; ++j) {
        const int64_t k = J[j];
        if (!((float)ra[j] < r[k])) continue;
        bool ok = copy(diag_gr + k * n, sgr + j * n, n * 16);
        if (les) ok = ok && copy(diag_gl + k * n, sgl + j * n, n * 16);
        if (nq) ok = ok && copy(req_gr + k * nq, spr + j * nq, nq * 16);
        if (nq && les) ok = ok && copy(req_gl + k * nq, spl + j * nq, nq * 16);
        r[k] = (float)ra[j];
        const float gk = (float)ga[j];
        ok = ok && cudaMemcpyAsync(d->resid + k, &r[k], sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess &&
             cudaMemcpy(d->growth + k, &gk, sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) rc = hsc_fail(h, HSC_ERR_CUDA, "re-solve scatter");
      }
    }
  }
  // an alternate solve that failed (e.g. a requested pair outside its pattern) leaves the first
  // results in place
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == HSC_OK && e != cudaSuccess) rc = hsc_fail(h, HSC_ERR_CUDA, cudaGetErrorString(e));
  return rc;
}

}  // namespace
}  // namespace hsc

extern "C" int hsc_solve(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                         const hsc_c128* sigma_less, int32_t precision, int32_t n_req,
                         const int32_t* req_pairs, hsc_c128* diag_gr, hsc_c128* diag_gl,
                         hsc_c128* req_gr, hsc_c128* req_gl, void* cuda_stream, int32_t io_on_device) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  int rc = check_common(h, n_E, E, eta, sigma_r, sigma_less, precision, n_req, req_pairs, diag_gr,
                        diag_gl, req_gr, req_gl);
  if (rc != HSC_OK || n_E == 0) return rc;
  if ((rc = get_state(h)) != HSC_OK) return rc;
  if ((rc = upload_pairs(h, n_req, req_pairs)) != HSC_OK) return rc;
  DeviceState* d = h->dev;
  int64_t wave = 0;
  if ((rc = prepare_arena(h, n_E, budget_bytes(), &wave, precision)) != HSC_OK) return rc;
  if ((rc = ensure_growth(h, n_E)) != HSC_OK) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (io_on_device) {
    rc = enqueue_device(h, n_E, wave, E, eta, sigma_r, sigma_less, precision, n_req, diag_gr, diag_gl,
                        req_gr, req_gl, s);
    if (rc != HSC_OK) return rc;
  } else {
    const int64_t n = h->n, ncs = h->n_contact_unknowns;
    int64_t need = wave * (int64_t)(8 + 16 * (2 * ncs + 2 * n + 2 * (int64_t)n_req)) + 8 * 256;
    if (d->io_cap < need) {
      if (d->io) cudaFree(d->io);
      d->io = nullptr;
      d->io_cap = 0;
      cudaError_t e = cudaMalloc(&d->io, need);
      if (e != cudaSuccess) { cudaGetLastError(); return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc io staging"); }
      d->io_cap = need;
    }
    char* p = (char*)d->io;
    auto take = [&](int64_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return r; };
    double* sE = (double*)take(wave * 8);
    c64* ssr = (c64*)take(wave * ncs * 16);
    c64* ssl = (c64*)take(wave * ncs * 16);
    c64* sgr = (c64*)take(wave * n * 16);
    c64* sgl = (c64*)take(wave * n * 16);
    c64* spr = (c64*)take(wave * (int64_t)n_req * 16);
    c64* spl = (c64*)take(wave * (int64_t)n_req * 16);
    CK(cudaMemsetAsync(d->flag, 0, 4 * sizeof(int), s));
    CK(cudaMemsetAsync(d->growth, 0, n_E * sizeof(float), s));
    CK(cudaMemsetAsync(d->resid, 0, n_E * sizeof(float), s));
    for (int64_t e0 = 0; e0 < n_E; e0 += wave) {
      const int ne = (int)std::min<int64_t>(wave, n_E - e0);
      d->growth_wave = d->growth + e0;
      d->resid_wave = d->resid + e0;
      d->cond_wave = d->cond + e0 * d->ncl;
      d->dense_e0 = e0;
      CK(cudaMemcpyAsync(sE, E + e0, ne * 8, cudaMemcpyHostToDevice, s));
      if (ncs > 0) {
        CK(cudaMemcpyAsync(ssr, sigma_r + e0 * ncs, ne * ncs * 16, cudaMemcpyHostToDevice, s));
        if (sigma_less) CK(cudaMemcpyAsync(ssl, sigma_less + e0 * ncs, ne * ncs * 16, cudaMemcpyHostToDevice, s));
      }
      rc = run_wave(h, ne, sE, eta, ssr, sigma_less ? ssl : nullptr, n_req, d->poff, sgr, sgl, spr,
                    spl, precision, s);
      if (rc != HSC_OK) return rc;
      CK(cudaMemcpyAsync(diag_gr + e0 * n, sgr, ne * n * 16, cudaMemcpyDeviceToHost, s));
      if (sigma_less) CK(cudaMemcpyAsync(diag_gl + e0 * n, sgl, ne * n * 16, cudaMemcpyDeviceToHost, s));
      if (n_req > 0) {
        CK(cudaMemcpyAsync(req_gr + e0 * n_req, spr, ne * (int64_t)n_req * 16, cudaMemcpyDeviceToHost, s));
        if (sigma_less) CK(cudaMemcpyAsync(req_gl + e0 * n_req, spl, ne * (int64_t)n_req * 16, cudaMemcpyDeviceToHost, s));
      }
    }
  }
  if ((rc = read_flags(h, s)) != HSC_OK) return rc;
  if (h->opt_resolve > 0 && !h->is_alt && precision == HSC_FP64 && !d->dense_r)
    for (int v = 1; v <= 4; ++v)
      if (v != h->nd_variant &&
          (rc = hsc::resolve_grown(v, h, n_E, E, eta, sigma_r, sigma_less, precision, n_req, req_pairs,
                                   diag_gr, diag_gl, req_gr, req_gl, s, io_on_device != 0)) != HSC_OK)
        return rc;
  h->err.clear();
  return HSC_OK;
}

extern "C" int hsc_solve_dense(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                               const hsc_c128* sigma_less, const hsc_c128* dense_r,
                               const hsc_c128* dense_less, int32_t precision, int32_t n_req,
                               const int32_t* req_pairs, hsc_c128* diag_gr, hsc_c128* diag_gl,
                               hsc_c128* req_gr, hsc_c128* req_gl, void* cuda_stream,
                               int32_t io_on_device) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  const hsc::Plan& P = h->plan;
  if (P.dense.empty())
    return hsc_fail(h, HSC_ERR_ARG, "no contact is dense (hsc_set_contact_dense, then hsc_analyze)");
  if (n_E < 0 || (n_E > 0 && !dense_r) || (sigma_less != nullptr) != (dense_less != nullptr))
    return hsc_fail(h, HSC_ERR_ARG, "dense_r is required; dense_less goes with sigma_less");
  if (n_E == 0)
    return hsc_solve(h, n_E, E, eta, sigma_r, sigma_less, precision, n_req, req_pairs, diag_gr, diag_gl,
                     req_gr, req_gl, cuda_stream, io_on_device);
  int rc = get_state(h);
  if (rc != HSC_OK) return rc;
  hsc::DeviceState* d = h->dev;
  const int64_t des = P.dense_elems;
  struct Tmp {
    void* p = nullptr;
    ~Tmp() { if (p) cudaFree(p); }
  } tmp;
  const hsc::c64* dr = reinterpret_cast<const hsc::c64*>(dense_r);
  const hsc::c64* dl = reinterpret_cast<const hsc::c64*>(dense_less);
  if (!io_on_device) {   // the blocks go to the device whole; the rest follows hsc_solve's staging
    const size_t one = (size_t)n_E * des * 16;
    if (cudaMalloc(&tmp.p, dense_less ? 2 * one : one) != cudaSuccess) {
      tmp.p = nullptr;
      cudaGetLastError();
      return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc dense self-energy staging");
    }
    if (cudaMemcpy(tmp.p, dense_r, one, cudaMemcpyHostToDevice) != cudaSuccess ||
        (dense_less && cudaMemcpy((char*)tmp.p + one, dense_less, one, cudaMemcpyHostToDevice) != cudaSuccess))
      return hsc_fail(h, HSC_ERR_CUDA, "copy dense self-energies");
    dr = reinterpret_cast<const hsc::c64*>(tmp.p);
    dl = dense_less ? reinterpret_cast<const hsc::c64*>((char*)tmp.p + one) : nullptr;
  }
  d->dense_r = dr;
  d->dense_l = dl;
  d->dense_es = des;
  d->dense_e0 = 0;
  rc = hsc_solve(h, n_E, E, eta, sigma_r, sigma_less, precision, n_req, req_pairs, diag_gr, diag_gl, req_gr,
                 req_gl, cuda_stream, io_on_device);
  d->dense_r = nullptr;
  d->dense_l = nullptr;
  return rc;
}

extern "C" int hsc_debug_offset(hsc_t h, int32_t i, int64_t* aug, int64_t* sq, int64_t* x) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  const Plan& P = h->plan;
  if (i < 0 || i >= (int32_t)P.cl.size()) return hsc_fail(h, HSC_ERR_ARG, "cluster out of range");
  int64_t xs = 0;
  for (int k = 0; k < i; ++k) xs += P.cl[k].n * P.cl[k].m;
  if (aug) *aug = P.off[i].aug;
  if (sq) *sq = P.off[i].sq;
  if (x) *x = xs;
  return HSC_OK;
}

extern "C" int hsc_debug_blocks(hsc_t h, int32_t which, int32_t energy, hsc_c128* out, int64_t* count) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  DeviceState* d = h->dev;
  if (!d || !d->arena) return hsc_fail(h, HSC_ERR_STATE, "no solve has run");
  if (energy < 0 || energy >= d->cap || !count) return hsc_fail(h, HSC_ERR_ARG, "bad energy/count");
  const c64* base = nullptr;
  int64_t es = 0;
  switch (which) {
    case 0: base = d->F; es = d->aug_es; break;
    case 1: base = d->L; es = d->aug_es; break;
    case 2: base = d->G; es = d->aug_es; break;
    case 3: base = d->P; es = d->aug_es; break;
    case 4: base = d->S; es = d->sq_es; break;
    case 5: base = d->LS; es = d->sq_es; break;
    case 6: base = d->X; es = d->x_es; break;
    default: return hsc_fail(h, HSC_ERR_ARG, "bad block array id");
  }
  *count = es;
  if (!out) return HSC_OK;
  CK(cudaMemcpy(out, base + (int64_t)energy * es, es * sizeof(c64), cudaMemcpyDeviceToHost));
  return HSC_OK;
}

extern "C" int hsc_profile(hsc_t h, int32_t enable) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!h->dev) {   // the options set on the handle must reach the state a later solve uses
    int rc = new_state(h);
    if (rc != HSC_OK) return rc;
  }
  Prof& p = h->dev->prof;
  p.on = enable != 0;
  p.used = 0;
  p.cls.clear();
  p.flops.clear();
  p.bytes.clear();
  for (auto& l : p.launches) l = 0;
  for (auto& x : p.extra) x = hsc_kernel_stat{};
  return HSC_OK;
}

extern "C" int hsc_profile_read(hsc_t h, hsc_kernel_stat* out, int32_t cap, int32_t* n_out) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!n_out) return hsc_fail(h, HSC_ERR_ARG, "n_out is NULL");
  *n_out = K_NCLASS;
  if (!out) return HSC_OK;
  if (cap < K_NCLASS) return hsc_fail(h, HSC_ERR_ARG, "cap too small");
  for (int c = 0; c < K_NCLASS; ++c) {
    std::memset(&out[c], 0, sizeof(hsc_kernel_stat));
    std::strncpy(out[c].name, kClassName[c], sizeof(out[c].name) - 1);
  }
  DeviceState* d = h->dev;
  if (!d) return HSC_OK;
  Prof& p = d->prof;
  for (size_t k = 0; k < p.used; ++k) {
    CK(cudaEventSynchronize(p.pool[2 * k + 1]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, p.pool[2 * k], p.pool[2 * k + 1]));
    out[p.cls[k]].ms += ms;
    out[p.cls[k]].timed += 1;
    out[p.cls[k]].flops += p.flops[k];
    out[p.cls[k]].bytes += p.bytes[k];
  }
  for (int c = 0; c < K_NCLASS; ++c) {
    out[c].launches = p.launches[c] + p.extra[c].launches;
    out[c].timed += p.extra[c].timed;
    out[c].ms += p.extra[c].ms;
    out[c].flops += p.extra[c].flops;
    out[c].bytes += p.extra[c].bytes;
  }
  return HSC_OK;
}

extern "C" int hsc_debug_gemm(int32_t engine, int32_t opa, int32_t opb, int32_t M, int32_t N, int32_t K,
                              const hsc_c128* A, int32_t lda, const hsc_c128* B, int32_t ldb,
                              hsc_c128* C, int32_t ldc, const hsc_c128* D, int32_t ldd,
                              double ar, double ai, double br, double bi, void* stream) {
  if (M < 0 || N < 0 || K < 0 || opa < 0 || opa > 3 || opb < 0 || opb > 3 || engine < 0 || engine > 4)
    return hsc_fail(nullptr, HSC_ERR_ARG, "bad GEMM arguments");
  GemmProb p{};
  p.M = M; p.N = N; p.K = K;
  p.lda = lda; p.ldb = ldb; p.ldc = ldc; p.ldd = ldd;
  p.use_d = D ? 1 : 0;
  const int tile = (engine == 1 || engine == 2) ? 128 : TILE;
  p.tiles_n = (N + tile - 1) / tile;
  p.tile_start = 0;
  p.tiles_m = (M + 127) / 128;
  p.ksteps = (K + 15) / 16;
  p.pack_start = 0;
  p.pa = 0;
  p.pb = (int64_t)p.tiles_m * p.ksteps * 8192;
  int64_t pack_words = (int64_t)(p.tiles_m + p.tiles_n) * p.ksteps * 8192;
  GemmProb* dp = nullptr;
  int* flag = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMalloc(&dp, sizeof(GemmProb)) != cudaSuccess || cudaMalloc(&flag, sizeof(int)) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_OOM, "cudaMalloc");
  cudaMemcpy(dp, &p, sizeof(p), cudaMemcpyHostToDevice);
  cudaMemset(flag, 0, sizeof(int));
  GemmArgs g{};
  g.probs = dp; g.nprob = 1; g.total_tiles = ((M + tile - 1) / tile) * p.tiles_n;
  g.A = A; g.B = B; g.C = C; g.D = D;
  g.ar = ar; g.ai = ai; g.br = br; g.bi = bi; g.opa = opa; g.opb = opb;
  g.pack_blocks = (p.tiles_m + p.tiles_n) * p.ksteps;
  g.pack_words = pack_words;
  uint32_t* pk = nullptr;
  int64_t oz_slices = 0, oz_scales = 0;
  if (engine == 4) {   // FP64 emulation on the BF16 tensor cores: its own tiling and pack layout
    int blocks = 0, tiles = 0;
    oz_layout(p, blocks, tiles, oz_slices, oz_scales);
    cudaMemcpy(dp, &p, sizeof(p), cudaMemcpyHostToDevice);
    g.total_tiles = tiles;
    g.pack_blocks = blocks;
    g.pack_words = oz_slices;
    g.scale_vals = oz_scales;
    pack_words = (oz_slices + 1) / 2 + 2 * oz_scales + 4;
  }
  if ((engine == 2 || engine == 4) && cudaMalloc(&pk, std::max<int64_t>(pack_words, 1) * 4) != cudaSuccess) {
    cudaFree(dp);
    cudaFree(flag);
    return hsc_fail(nullptr, HSC_ERR_OOM, "cudaMalloc pack");
  }
  // engine 4: slices first, then the scales at the next 16-byte boundary
  const int64_t oz_sc_words = ((oz_slices + 1) / 2 + 3) / 4 * 4;
  cudaError_t e = engine == 4 ? gemm_oz(g, 1, reinterpret_cast<uint16_t*>(pk), oz_slices,
                                        reinterpret_cast<double*>(pk + oz_sc_words), oz_scales, flag, s)
                  : engine == 2 ? gemm_tc_packed(g, 1, pk, pack_words, flag, s)
                  : engine == 1 ? gemm_tc(g, 1, flag, s) : gemm_z(g, 1, s, engine == 3);
  int hf = 0;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dp);
  cudaFree(flag);
  if (pk) cudaFree(pk);
  if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
  if (hf) return hsc_fail(nullptr, HSC_ERR_TIMEOUT, "tensor-core GEMM wait expired");
  return HSC_OK;
}

namespace hsc {
namespace {
int read_record(hsc_ctx* h, int64_t n_E, double* out, bool residual) {
  if (!h || (!out && n_E > 0) || n_E < 0) return hsc_fail(h, HSC_ERR_ARG, "bad arguments");
  DeviceState* d = h->dev;
  if (!d || !d->growth || n_E > d->growth_n)
    return hsc_fail(h, HSC_ERR_STATE, "no solve of that many energies has run on this handle");
  std::vector<float> g(n_E);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(g.data(), residual ? d->resid : d->growth, n_E * sizeof(float), cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < n_E; ++k) out[k] = g[k];
  return HSC_OK;
}
}  // namespace
}  // namespace hsc

extern "C" int hsc_growth(hsc_t h, int64_t n_E, double* out) { return hsc::read_record(h, n_E, out, false); }

extern "C" int hsc_cluster_growth(hsc_t h, int64_t n_E, double* out) {
  using namespace hsc;
  if (!h || (!out && n_E > 0) || n_E < 0) return hsc_fail(h, HSC_ERR_ARG, "bad arguments");
  DeviceState* d = h->dev;
  if (!d || !d->growth || n_E > d->growth_n)
    return hsc_fail(h, HSC_ERR_STATE, "no solve of that many energies has run on this handle");
  const int nc = d->ncl;
  std::vector<float> g((size_t)n_E * nc);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(g.data(), d->cond, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < n_E; ++k)
    for (int j = 0; j < nc; ++j) out[k * nc + d->gj_owner[j]] = g[k * nc + j];
  return HSC_OK;
}
extern "C" int hsc_residual(hsc_t h, int64_t n_E, double* out) { return hsc::read_record(h, n_E, out, true); }

// ---- batched solve in one CUDA graph -----------------------------------------------------------

namespace hsc {
namespace {

struct GraphCache {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;     // capture stream (the legacy default stream cannot be captured)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
};
GraphCache g_graph;

uint64_t u64(const void* p) { return (uint64_t)(uintptr_t)p; }

}  // namespace
}  // namespace hsc

extern "C" int hsc_solve_batch(int32_t n_items, const hsc_batch_item* items, double eta,
                               int32_t precision, void* cuda_stream, int32_t use_graph) {
  if (n_items <= 0 || !items) return hsc_fail(nullptr, HSC_ERR_ARG, "no batch items");
  auto item_fail = [&](int i, hsc_ctx* h, int rc) {
    return hsc_fail(nullptr, rc, "batch item " + std::to_string(i) + ": " + (h ? h->err : std::string("")));
  };
  double need_total = 0;
  std::vector<double> need(n_items, 0.0);
  for (int i = 0; i < n_items; ++i) {
    const hsc_batch_item& it = items[i];
    hsc_ctx* h = it.h;
    if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "batch item " + std::to_string(i) + ": NULL handle");
    for (int j = 0; j < i; ++j)
      if (items[j].h == h) return hsc_fail(nullptr, HSC_ERR_ARG, "a handle appears twice in the batch");
    int rc = check_common(h, it.n_E, it.E, eta, it.sigma_r, it.sigma_less, precision, it.n_req,
                          it.req_pairs, it.diag_gr, it.diag_gl, it.req_gr, it.req_gl);
    if (rc == HSC_OK) rc = get_state(h);
    if (rc == HSC_OK) rc = upload_pairs(h, it.n_req, it.req_pairs);
    if (rc != HSC_OK) return item_fail(i, h, rc);
    need[i] = (double)bytes_per_energy(h->dev, pack_words_needed(h->dev, precision)) *
              (double)std::max<int64_t>(it.n_E, 1);
    need_total += need[i];
  }
  const double budget = (double)budget_bytes();
  std::vector<int64_t> wave(n_items, 0);
  for (int i = 0; i < n_items; ++i) {
    hsc_ctx* h = items[i].h;
    int64_t cap = (int64_t)(budget * need[i] / need_total);
    int rc = prepare_arena(h, std::max<int64_t>(items[i].n_E, 1), cap, &wave[i], precision);
    if (rc == HSC_OK) rc = ensure_growth(h, std::max<int64_t>(items[i].n_E, 1));
    if (rc != HSC_OK) return item_fail(i, h, rc);
    if (!h->dev->branch) {
      cudaError_t e = cudaStreamCreateWithFlags(&h->dev->branch, cudaStreamNonBlocking);
      if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, "cudaStreamCreate");
    }
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<uint64_t> key = {(uint64_t)n_items, (uint64_t)precision};
  {
    uint64_t eb;
    std::memcpy(&eb, &eta, sizeof(eb));
    key.push_back(eb);
    key.push_back(u64(s));
  }
  for (int i = 0; i < n_items; ++i) {
    const hsc_batch_item& it = items[i];
    DeviceState* d = it.h->dev;
    for (uint64_t v : {u64(it.h), d->gen, u64(d->arena), (uint64_t)d->cap, u64(d->growth), (uint64_t)it.n_E, u64(it.E),
                       u64(it.sigma_r), u64(it.sigma_less), (uint64_t)it.n_req, u64(d->poff),
                       u64(it.diag_gr), u64(it.diag_gl), u64(it.req_gr), u64(it.req_gl),
                       (uint64_t)wave[i]})
      key.push_back(v);
  }
  auto enqueue_all = [&](cudaStream_t s) -> int {
    for (int i = 0; i < n_items; ++i) {
      const hsc_batch_item& it = items[i];
      hsc_ctx* h = it.h;
      cudaStream_t b = h->dev->branch;
      if (cudaStreamWaitEvent(b, g_graph.fork, 0) != cudaSuccess)
        return hsc_fail(nullptr, HSC_ERR_CUDA, "cudaStreamWaitEvent");
      if (it.n_E > 0) {
        const bool prof = h->dev->prof.on;
        if (use_graph) h->dev->prof.on = false;   // no event bookkeeping inside a captured graph
        int rc = enqueue_device(h, it.n_E, wave[i], it.E, eta, it.sigma_r, it.sigma_less, precision,
                                it.n_req, it.diag_gr, it.diag_gl, it.req_gr, it.req_gl, b);
        h->dev->prof.on = prof;
        if (rc != HSC_OK) return item_fail(i, h, rc);
      }
      if (cudaEventRecord(g_graph.join[i], b) != cudaSuccess ||
          cudaStreamWaitEvent(s, g_graph.join[i], 0) != cudaSuccess)
        return hsc_fail(nullptr, HSC_ERR_CUDA, "join events");
    }
    return HSC_OK;
  };
  if (!g_graph.fork && cudaEventCreateWithFlags(&g_graph.fork, cudaEventDisableTiming) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_CUDA, "cudaEventCreate");
  while ((int)g_graph.join.size() < n_items) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return hsc_fail(nullptr, HSC_ERR_CUDA, "cudaEventCreate");
    g_graph.join.push_back(e);
  }
  if (use_graph) {
    if (!(g_graph.exec && g_graph.key == key)) {
      if (g_graph.exec) cudaGraphExecDestroy(g_graph.exec);
      g_graph.exec = nullptr;
      g_graph.key.clear();
      if (!g_graph.cap && cudaStreamCreateWithFlags(&g_graph.cap, cudaStreamNonBlocking) != cudaSuccess)
        return hsc_fail(nullptr, HSC_ERR_CUDA, "cudaStreamCreate");
      cudaStream_t cs = g_graph.cap;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      int rc = HSC_OK;
      if (cudaEventRecord(g_graph.fork, cs) != cudaSuccess) rc = hsc_fail(nullptr, HSC_ERR_CUDA, "fork event");
      if (rc == HSC_OK) rc = enqueue_all(cs);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      if (rc != HSC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&g_graph.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g_graph.exec = nullptr;
        return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      g_graph.key = key;
    }
    cudaError_t e = cudaGraphLaunch(g_graph.exec, s);
    if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  } else {
    if (cudaEventRecord(g_graph.fork, s) != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, "fork event");
    int rc = enqueue_all(s);
    if (rc != HSC_OK) return rc;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  for (int i = 0; i < n_items; ++i) {
    int rc = read_flags(items[i].h, s);
    if (rc != HSC_OK) return item_fail(i, items[i].h, rc);
  }
  return HSC_OK;
}

// ---- autotuner -----------------------------------------------------------------------------------

extern "C" int hsc_tune(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                        const hsc_c128* sigma_less, int32_t precision, const char* cache_path,
                        hsc_tune_result* out) {
  if (!h || !out || n_E <= 0 || !E) return hsc_fail(h, HSC_ERR_ARG, "bad tune arguments");
  cudaDeviceProp prop;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return hsc_fail(h, HSC_ERR_CUDA, "no CUDA device");
  char keybuf[512];
  std::snprintf(keybuf, sizeof(keybuf), "\"gpu\": \"%s\", \"dims\": [%d, %d, %d], \"orb\": %d, \"n\": %lld, \"precision\": %d",
                prop.name, h->dims[0], h->dims[1], h->dims[2], h->orb, (long long)h->n, precision);
  const std::string key(keybuf);
  std::memset(out, 0, sizeof(*out));
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[1024];
      int leaf = -1, nb = -1;
      double ms = 0;
      while (std::fgets(line, sizeof(line), f)) {
        if (!std::strstr(line, key.c_str())) continue;
        const char* a = std::strstr(line, "\"leaf_max\": ");
        const char* b = std::strstr(line, "\"gj_panel\": ");
        const char* c = std::strstr(line, "\"ms_per_energy\": ");
        if (a && b) {
          leaf = std::atoi(a + 12);
          nb = std::atoi(b + 12);
          ms = c ? std::atof(c + 17) : 0;
        }
      }
      std::fclose(f);
      if (leaf > 0 && nb > 0) {
        int rc = hsc_analyze(h, leaf, nullptr);
        if (rc == HSC_OK) rc = hsc_set_option(h, HSC_OPT_GJ_PANEL, nb);
        if (rc != HSC_OK) return rc;
        out->leaf_max = leaf;
        out->gj_panel = nb;
        out->ms_per_energy = ms;
        out->from_cache = 1;
        return HSC_OK;
      }
    }
  }
  const int64_t n = h->n;
  const int64_t ncs = h->n_contact_unknowns;
  std::vector<hsc_c128> gr(n_E * n), gl(sigma_less ? n_E * n : 0);
  int maxdim = std::max(h->dims[0], std::max(h->dims[1], h->dims[2]));
  if (maxdim <= 0) maxdim = 1 << 30;
  std::vector<int> leaves;
  for (int l : {4, 6, 8})
    if (l < maxdim) leaves.push_back(l);
  if (leaves.empty()) leaves.push_back(h->leaf_max > 0 ? h->leaf_max : 4);
  // a candidate is admissible when every probe's residual (after the solve's own re-solves) stays
  // within the handle's threshold 10^-d (HSC_OPT_RESOLVE_DIGITS, or 1e-10 when re-solves are off):
  // a cheaper tree that loses digits is not a faster solve of the same problem. The fastest
  // admissible candidate wins; if none is admissible, the one with the smallest worst residual.
  const double thr = std::pow(10.0, -(h->opt_resolve > 0 ? h->opt_resolve : 10));
  double best = 1e300, best_res = 1e300;
  bool best_ok = false;
  int best_leaf = leaves[0], best_nb = 32, tried = 0;
  std::vector<double> res(n_E);
  (void)ncs;
  for (int leaf : leaves)
    for (int nb : {16, 32, 64}) {
      int rc = hsc_analyze(h, leaf, nullptr);
      if (rc == HSC_OK) rc = hsc_set_option(h, HSC_OPT_GJ_PANEL, nb);
      if (rc == HSC_OK)
        rc = hsc_solve(h, n_E, E, eta, sigma_r, sigma_less, precision, 0, nullptr, gr.data(),
                       sigma_less ? gl.data() : nullptr, nullptr, nullptr, nullptr, 0);
      if (rc != HSC_OK) return rc;
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, 0);
      rc = hsc_solve(h, n_E, E, eta, sigma_r, sigma_less, precision, 0, nullptr, gr.data(),
                     sigma_less ? gl.data() : nullptr, nullptr, nullptr, nullptr, 0);
      cudaEventRecord(b, 0);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      if (rc != HSC_OK) return rc;
      ++tried;
      double rmax = 0.0;
      if (precision == HSC_FP64 && hsc_residual(h, n_E, res.data()) == HSC_OK)
        for (double r : res) rmax = std::max(rmax, r);
      const bool ok = rmax <= thr;
      if ((ok && (!best_ok || ms < best)) || (!ok && !best_ok && rmax < best_res)) {
        best = ms;
        best_res = rmax;
        best_ok = ok;
        best_leaf = leaf;
        best_nb = nb;
      }
    }
  int rc = hsc_analyze(h, best_leaf, nullptr);
  if (rc == HSC_OK) rc = hsc_set_option(h, HSC_OPT_GJ_PANEL, best_nb);
  if (rc != HSC_OK) return rc;
  out->leaf_max = best_leaf;
  out->gj_panel = best_nb;
  out->ms_per_energy = best / (double)n_E;
  out->n_tried = tried;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "{%s, \"leaf_max\": %d, \"gj_panel\": %d, \"ms_per_energy\": %.6f}\n", key.c_str(),
                   best_leaf, best_nb, out->ms_per_energy);
      std::fclose(f);
    }
  }
  return HSC_OK;
}

extern "C" int hsc_observables(hsc_t h, int64_t n_E, const hsc_c128* diag_gr, const hsc_c128* diag_gl,
                               const hsc_c128* sigma_r, int32_t contact, double* out, void* cuda_stream) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (n_E < 0 || (n_E > 0 && (!diag_gr || !out))) return hsc_fail(h, HSC_ERR_ARG, "bad observables arguments");
  if (contact < 0 || contact >= std::max(h->n_contacts, 1)) return hsc_fail(h, HSC_ERR_ARG, "contact out of range");
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  int rc = get_state(h);
  if (rc != HSC_OK) return rc;
  if ((rc = hsc::ensure_slots(h)) != HSC_OK) return rc;
  DeviceState* d = h->dev;
  const int64_t ncs = h->n_contact_unknowns;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(launch_observables(n_E, h->n, reinterpret_cast<const c64*>(diag_gr),
                        reinterpret_cast<const c64*>(diag_gl), reinterpret_cast<const c64*>(sigma_r), ncs,
                        d->slot_unknown, d->slot_contact, contact, out, s));
  return HSC_OK;
}

extern "C" int hsc_scba(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                        const hsc_c128* sigma_less, double d0, double mix, double tol, int32_t max_iter,
                        int32_t precision, hsc_c128* diag_gr, hsc_c128* diag_gl, int32_t* iters,
                        double* delta, void* cuda_stream, int32_t io_on_device) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!iters || !delta || n_E < 0 ||
      (n_E > 0 && (!E || !sigma_r || !sigma_less || !diag_gr || !diag_gl)))
    return hsc_fail(h, HSC_ERR_ARG, "bad SCBA arguments");
  if (!(d0 >= 0.0) || !(mix > 0.0 && mix <= 1.0) || !(tol >= 0.0) || max_iter < 1)
    return hsc_fail(h, HSC_ERR_ARG, "need d0 >= 0, 0 < mix <= 1, tol >= 0 and max_iter >= 1");
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  if (h->n_contact_unknowns != h->n)
    return hsc_fail(h, HSC_ERR_ARG,
                    "dephasing acts on every unknown: the contacts must cover every site (declare the "
                    "scattering region as a contact whose contact self-energy is zero)");
  *iters = 0;
  *delta = 0.0;
  if (n_E == 0) return HSC_OK;
  int rc = get_state(h);
  if (rc != HSC_OK) return rc;
  if ((rc = hsc::ensure_slots(h)) != HSC_OK) return rc;
  const int64_t n = h->n, ncs = h->n_contact_unknowns, slots = n_E * ncs;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // device work: S_r, S_l, Sigma_r, Sigma_l per slot, the two maxima; with host I/O also E, the
  // contact parts and the diagonals
  struct Work {
    void* p = nullptr;
    ~Work() { if (p) cudaFree(p); }
  } work;
  auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
  int64_t bytes = 4 * up(slots * 16) + 256;
  if (!io_on_device) bytes += up(n_E * 8) + 2 * up(slots * 16) + 2 * up(n_E * n * 16);
  if (cudaMalloc(&work.p, bytes) != cudaSuccess) {
    work.p = nullptr;
    cudaGetLastError();
    return hsc_fail(h, HSC_ERR_OOM, "cudaMalloc SCBA work");
  }
  char* q = (char*)work.p;
  auto take = [&](int64_t b) { char* r = q; q += up(b); return r; };
  c64* s_r = (c64*)take(slots * 16);
  c64* s_l = (c64*)take(slots * 16);
  c64* sig_r = (c64*)take(slots * 16);
  c64* sig_l = (c64*)take(slots * 16);
  unsigned long long* dmax = (unsigned long long*)take(256);
  const double* dE = E;
  const c64* cr = reinterpret_cast<const c64*>(sigma_r);
  const c64* cl = reinterpret_cast<const c64*>(sigma_less);
  c64* gr = reinterpret_cast<c64*>(diag_gr);
  c64* gl = reinterpret_cast<c64*>(diag_gl);
  if (!io_on_device) {
    double* hE = (double*)take(n_E * 8);
    c64* hcr = (c64*)take(slots * 16);
    c64* hcl = (c64*)take(slots * 16);
    gr = (c64*)take(n_E * n * 16);
    gl = (c64*)take(n_E * n * 16);
    CK(cudaMemcpyAsync(hE, E, n_E * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(hcr, sigma_r, slots * 16, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(hcl, sigma_less, slots * 16, cudaMemcpyHostToDevice, s));
    dE = hE;
    cr = hcr;
    cl = hcl;
  }
  CK(cudaMemsetAsync(s_r, 0, 2 * up(slots * 16), s));   // S_r and S_l: S_0 = 0
  CK(cudaMemcpyAsync(sig_r, cr, slots * 16, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sig_l, cl, slots * 16, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < max_iter; ++k) {
    rc = hsc_solve(h, n_E, dE, eta, reinterpret_cast<const hsc_c128*>(sig_r),
                   reinterpret_cast<const hsc_c128*>(sig_l), precision, 0, nullptr,
                   reinterpret_cast<hsc_c128*>(gr), reinterpret_cast<hsc_c128*>(gl), nullptr, nullptr, s, 1);
    if (rc != HSC_OK) return rc;
    CK(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), s));
    CK(launch_scba_mix(n_E, n, ncs, h->dev->slot_unknown, gr, gl, cr, cl, d0, mix, s_r, s_l, sig_r, sig_l,
                       dmax, s));
    unsigned long long m[2] = {0, 0};
    CK(cudaMemcpyAsync(m, dmax, sizeof(m), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double diff, scale;
    std::memcpy(&diff, &m[0], 8);
    std::memcpy(&scale, &m[1], 8);
    *iters = k + 1;
    *delta = scale > 0.0 ? diff / scale : 0.0;
    if (*delta <= tol) break;
  }
  if (!io_on_device) {
    CK(cudaMemcpyAsync(diag_gr, gr, n_E * n * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(diag_gl, gl, n_E * n * 16, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  h->err.clear();
  return HSC_OK;
}

extern "C" int hsc_debug_wait_timeout(double seconds) {
  if (!(seconds > 0.0) || seconds > 2.0) return hsc_fail(nullptr, HSC_ERR_ARG, "seconds must be in (0, 2]");
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_OOM, "cudaMalloc");
  cudaMemset(flag, 0, sizeof(int));
  cudaError_t e = launch_wait_probe(seconds, flag, 0);
  int hf = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
  if (hf) return hsc_fail(nullptr, HSC_ERR_TIMEOUT, "bounded device wait expired (as intended)");
  return HSC_OK;
}
