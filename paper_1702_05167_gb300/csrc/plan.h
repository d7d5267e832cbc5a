// Host-side analysis of the HSC-extension: nested-dissection cluster tree, update sets, index maps
// and the flop/byte model. Energy independent; built once per geometry (Section 2.2, the cluster
// tree of Algorithms 1-2; Section 2.2's multilevel nested dissection).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hsc {

struct Cluster {
  int parent = -1;
  int child[2] = {-1, -1};
  int nchild = 0;
  int height = 0;       // 0 for leaves, 1 + max(child heights) otherwise (upward schedule)
  int depth = 0;        // 0 for the root (downward schedule)
  int first_desc = 0;   // smallest postorder id in the subtree: subtree = [first_desc, id]
  bool lesser = false;  // subtree holds a contact unknown (non-zero lesser front)
  std::vector<int> sites;    // own sites, increasing site index
  std::vector<int> usites;   // update-set sites U_i, increasing permuted position
  int64_t n = 0, m = 0;      // own / update-set unknowns
};

// One contiguous region per cluster inside a per-energy array.
struct Offsets {
  int64_t aug = 0;   // n x (n+m) row-major: [X_ii | X_iU]
  int64_t sq = 0;    // m x m row-major
};

struct Plan {
  int64_t n_sites = 0, n = 0;
  int orb = 1;
  int leaf_max = 0;
  std::vector<Cluster> cl;         // postorder: children before parents, root last
  std::vector<int> site_cluster;   // owner cluster of each site
  std::vector<int> site_local;     // index of the site inside its owner's site list
  std::vector<std::vector<int>> by_height;  // clusters grouped by height (upward order)
  std::vector<std::vector<int>> by_depth;   // clusters grouped by depth (downward order)
  std::vector<Offsets> off;
  int64_t tot_aug = 0, tot_sq = 0;           // per-energy element counts
  int64_t max_level_sq = 0, max_level_aug_u = 0;  // per-level temporaries

  // ---- index maps (flattened, device-uploadable) ----
  // front assembly: for cluster i and child slot c, map_child[map_off[i][c] + q] = index of front
  // position q (0..n+m-1) inside U_child (unknown granularity), or -1.
  std::vector<int32_t> map_child;
  std::vector<int64_t> map_off;   // [2*nc]
  // original H entries of each front: row r < n, column q < n+m, value index into H's CSR
  std::vector<int32_t> h_rq;      // packed (r, q) pairs
  std::vector<int64_t> h_vi;      // CSR value index
  std::vector<int64_t> h_off;     // [nc+1]
  // diagonal of each front: contact slot of own unknown r (or -1)
  std::vector<int32_t> own_contact;   // [sum n], offset own_off[i]
  std::vector<int64_t> own_off;       // [nc+1]
  // downward gather of G_UU / P_UU: per update-set unknown k of cluster i (offset u_off[i]):
  std::vector<int32_t> u_owner;   // owner cluster
  std::vector<int32_t> u_local;   // unknown index inside owner
  std::vector<int32_t> u_seg;     // segment (owner) index within U_i, segments in ascending order
  std::vector<int64_t> u_off;     // [nc+1]
  // posmap[pm_off[i] + k*nseg[i] + s] = position of U_i[k] inside U_{seg s owner}, or -1
  std::vector<int32_t> posmap;
  std::vector<int64_t> pm_off;    // [nc+1]
  std::vector<int32_t> nseg;      // [nc]
  // permutation: position of each unknown in the cluster-ordered numbering
  std::vector<int64_t> iperm;     // [n]  unknown -> (cluster, local) via cluster_of_unknown/local
  std::vector<int32_t> unk_cluster, unk_local;   // [n]

  // DENSE contacts (Section 3.1.2), in contact order: the cluster that owns all of the contact's
  // unknowns, their number, the block's offset in a per-energy dense self-energy array (blocks
  // nu x nu row-major in the contact's slot order, contact after contact) and, from `loc`, the
  // local row inside that cluster of each slot's unknown (dense_local)
  struct Dense {
    int contact = -1, cluster = -1;
    int64_t nu = 0, blk = 0, loc = 0;
  };
  std::vector<Dense> dense;
  std::vector<int32_t> dense_local;
  int64_t dense_elems = 0;

  // ---- model ----
  double flops_gr = 0, flops_gl = 0;   // real flops per energy (complex MAC = 8)
};

struct Input {
  int64_t n = 0;      // unknowns
  int orb = 1;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  int n_contacts = 0;
  const int64_t* contact_ptr = nullptr;
  const int32_t* contact_sites = nullptr;
  int dims[3] = {0, 0, 0};   // all zero: general graph bisection
  int variant = 0;           // 1..4: alternate separator trees (cuts below the root moved +1, -1, +2, -2)
  // geometric dissection only: 1 = contact-connected (the transport axis x is cut once, at the root;
  // every deeper cut is a y or z plane, so each box below the root keeps its share of the x = 0 or
  // x = Nx-1 end plane); 0 = the longest extent is cut at every level
  int contact_connected = 0;
  const char* contact_dense = nullptr;   // per contact (nullable): 1 = one cluster on top of the tree
  // clusters (ids of the tree built without merges) whose own unknowns join their parent's
  const int32_t* merge = nullptr;
  int n_merge = 0;
  // > 0: a cluster of more sites is split into a chain of pieces of at most this many sites (the
  // degenerate sub-trees of Section 3.4); dense contacts stay whole
  int max_cluster = 0;
};

// Builds the plan. Returns an empty string on success, else an error message.
std::string analyze(const Input& in, int leaf_max, Plan& plan);

}  // namespace hsc
