// Host analysis for the HSC-extension (Section 2.2): nested dissection into a binary cluster tree,
// ancestor update sets, front assembly maps, downward gather maps and the operation-count model.
#include "plan.h"

#include <algorithm>
#include <cstdio>
#include <functional>
#include <numeric>

namespace hsc {
namespace {

struct Builder {
  const Input& in;
  int64_t n_sites;
  int leaf;
  std::vector<std::vector<int>> adj;   // site graph (no self loops)
  std::vector<Cluster>& cl;

  Builder(const Input& i, int64_t ns, int lf, std::vector<Cluster>& c)
      : in(i), n_sites(ns), leaf(lf), cl(c) {}

  int make(std::vector<int>&& sites, int c0, int c1) {
    Cluster c;
    std::sort(sites.begin(), sites.end());
    c.sites = std::move(sites);
    if (c0 >= 0) c.child[c.nchild++] = c0;
    if (c1 >= 0) c.child[c.nchild++] = c1;
    cl.push_back(std::move(c));
    int id = (int)cl.size() - 1;
    for (int k = 0; k < cl[id].nchild; ++k) cl[cl[id].child[k]].parent = id;
    return id;
  }

  // Geometric nested dissection of the box [lo, hi] (inclusive): cut the longest extent (ties in
  // x, y, z order) by the plane at floor((lo+hi)/2); stop when every extent is <= leaf. The
  // alternate trees keep the root plane and move every deeper cut by +1, -1, +2 or -2 planes
  // (in.variant = 1..4) where both halves stay non-empty, so their boxes (and isolated spectra)
  // differ.
  // Contact-connected form (in.contact_connected, for contacts on the end planes x = 0 and
  // x = Nx-1): the root cuts x; below it only the longer of y and z is cut, and a box is a leaf once
  // its y and z extents are <= leaf. Every cluster below the root then holds contact sites or has
  // children that do, so no cluster block of Algorithm 1 lacks the contacts' broadening; a box far
  // from both contacts would carry only eta, and a level of it within delta of E costs the
  // downward step of Eq. 4 a factor ~1/delta^2 of the rounding error.
  int box(int lo[3], int hi[3], int depth = 0) {
    int ext[3];
    for (int d = 0; d < 3; ++d) {
      ext[d] = hi[d] - lo[d] + 1;
      if (ext[d] <= 0) return -1;
    }
    const int Ny = in.dims[1], Nz = in.dims[2];
    auto sites_in = [&](int a[3], int b[3]) {
      std::vector<int> s;
      for (int x = a[0]; x <= b[0]; ++x)
        for (int y = a[1]; y <= b[1]; ++y)
          for (int z = a[2]; z <= b[2]; ++z) s.push_back((x * Ny + y) * Nz + z);
      return s;
    };
    const bool cc = in.contact_connected != 0;
    const bool xcut = cc && depth == 0 && ext[0] >= 3;   // the one cut across the transport axis
    if (!xcut && (cc || ext[0] <= leaf) && ext[1] <= leaf && ext[2] <= leaf)
      return make(sites_in(lo, hi), -1, -1);
    int d = 0;
    if (xcut) {
      d = 0;
    } else if (cc) {
      d = ext[2] > ext[1] ? 2 : 1;
    } else {
      for (int k = 1; k < 3; ++k)
        if (ext[k] > ext[d]) d = k;
    }
    int mid = (lo[d] + hi[d]) / 2;
    if (depth > 0 && in.variant > 0) {
      static const int kShift[5] = {0, 1, -1, 2, -2};
      const int m2 = mid + kShift[in.variant];
      if (m2 > lo[d] && m2 < hi[d]) mid = m2;
    }
    int llo[3] = {lo[0], lo[1], lo[2]}, lhi[3] = {hi[0], hi[1], hi[2]};
    int rlo[3] = {lo[0], lo[1], lo[2]}, rhi[3] = {hi[0], hi[1], hi[2]};
    lhi[d] = mid - 1;
    rlo[d] = mid + 1;
    int c0 = box(llo, lhi, depth + 1);
    int c1 = box(rlo, rhi, depth + 1);
    int slo[3] = {lo[0], lo[1], lo[2]}, shi[3] = {hi[0], hi[1], hi[2]};
    slo[d] = shi[d] = mid;
    return make(sites_in(slo, shi), c0, c1);
  }

  // General-graph bisection: breadth-first level sets from a pseudo-peripheral site; the level
  // where the running count crosses half the set is the separator (below the root, the alternate
  // trees move it by +1, -1, +2 or -2 levels (variant 1..4) where both sides stay non-empty).
  int graph(std::vector<int> S, std::vector<int>& mark, int tag) {
    if (S.empty()) return -1;
    const int64_t lim = (int64_t)leaf * leaf * leaf;
    if ((int64_t)S.size() <= lim) return make(std::move(S), -1, -1);
    for (int s : S) mark[s] = tag;
    auto bfs = [&](int root, std::vector<int>& lev, std::vector<int>& order) {
      order.clear();
      order.push_back(root);
      lev[root] = 0;
      for (size_t h = 0; h < order.size(); ++h) {
        int u = order[h];
        for (int v : adj[u])
          if (mark[v] == tag && lev[v] < 0) {
            lev[v] = lev[u] + 1;
            order.push_back(v);
          }
      }
    };
    std::vector<int> lev(n_sites, -1), order;
    bfs(S[0], lev, order);
    int far = order.back();
    for (int v : order) lev[v] = -1;
    bfs(far, lev, order);
    int maxl = lev[order.back()];
    std::vector<int> sep, left, right;
    if (maxl < 2 && order.size() == S.size()) {
      for (int v : order) lev[v] = -1;
      for (int s : S) mark[s] = -1;
      return make(std::move(S), -1, -1);
    }
    std::vector<int64_t> cnt(maxl + 1, 0);
    for (int v : order) cnt[lev[v]]++;
    int64_t run = 0;
    int cut = 0;
    for (int l = 0; l <= maxl; ++l) {
      run += cnt[l];
      if (2 * run >= (int64_t)S.size()) { cut = l; break; }
    }
    if (cut == 0) cut = std::min(1, maxl);
    if (tag > 0 && in.variant > 0) {
      static const int kShift[5] = {0, 1, -1, 2, -2};
      const int c2 = cut + kShift[in.variant];
      if (c2 >= 1 && c2 < maxl) cut = c2;
    }
    for (int s : S) {
      if (lev[s] < 0) right.push_back(s);
      else if (lev[s] < cut) left.push_back(s);
      else if (lev[s] == cut) sep.push_back(s);
      else right.push_back(s);
    }
    for (int v : order) lev[v] = -1;
    for (int s : S) mark[s] = -1;
    int c0 = graph(std::move(left), mark, tag + 1);
    int c1 = graph(std::move(right), mark, tag + 1);
    return make(std::move(sep), c0, c1);
  }
};

}  // namespace

std::string analyze(const Input& in, int leaf_max, Plan& P) {
  if (in.n <= 0 || in.orb <= 0 || in.n % in.orb) return "n must be a positive multiple of orb";
  if (leaf_max < 1) return "leaf_max must be >= 1";
  P = Plan();
  P.n = in.n;
  P.orb = in.orb;
  P.leaf_max = leaf_max;
  const int orb = in.orb;
  const int64_t ns = in.n / orb;
  P.n_sites = ns;

  std::vector<Cluster> first;   // the tree before merges (when a merge list is given)
  const bool rebuild = in.n_merge > 0 || in.max_cluster > 0;
  Builder B(in, ns, leaf_max, rebuild ? first : P.cl);
  // site graph from the unknown-level CSR
  B.adj.assign(ns, {});
  for (int64_t u = 0; u < in.n; ++u) {
    int s = (int)(u / orb);
    for (int64_t e = in.rowptr[u]; e < in.rowptr[u + 1]; ++e) {
      int64_t v = in.col[e];
      if (v < 0 || v >= in.n) return "column index out of range";
      int t = (int)(v / orb);
      if (t != s) B.adj[s].push_back(t);
    }
  }
  for (auto& a : B.adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }

  // DENSE contacts (Section 3.1.2): a dense self-energy block couples every pair of the contact's
  // unknowns, so each such contact becomes one cluster, chained on top of the nested dissection of
  // the remaining sites (an ancestor of every other cluster, so the update sets stay exact).
  std::vector<int> dense_c;
  std::vector<char> in_dense(ns, 0);
  int64_t n_dense = 0;
  for (int c = 0; c < in.n_contacts; ++c) {
    if (!in.contact_dense || !in.contact_dense[c]) continue;
    dense_c.push_back(c);
    for (int64_t k = in.contact_ptr[c]; k < in.contact_ptr[c + 1]; ++k) {
      const int s = in.contact_sites[k];
      if (s < 0 || s >= ns) return "contact site out of range";
      if (in_dense[s]) return "site appears in two contacts";
      in_dense[s] = 1;
      ++n_dense;
    }
  }
  bool geo = in.dims[0] > 0 && in.dims[1] > 0 && in.dims[2] > 0;
  if (geo && (int64_t)in.dims[0] * in.dims[1] * in.dims[2] != ns) return "grid_dims do not match n/orb";
  int x0 = 0, x1 = geo ? in.dims[0] - 1 : 0;
  if (geo && n_dense > 0) {
    // geometric dissection of the interior box when the dense contacts are whole end planes x = 0
    // and x = Nx-1; any other dense contact shape falls back to graph bisection of the rest
    const int64_t plane = (int64_t)in.dims[1] * in.dims[2];
    int64_t faces = 0;
    for (int c : dense_c) {
      const int64_t cnt = in.contact_ptr[c + 1] - in.contact_ptr[c];
      const int s0 = in.contact_sites[in.contact_ptr[c]];
      const int x = (int)(s0 / plane);
      bool face = cnt == plane && (x == 0 || x == in.dims[0] - 1) && !(x == 0 && x0 > 0) &&
                  !(x == in.dims[0] - 1 && x1 < in.dims[0] - 1);
      for (int64_t k = in.contact_ptr[c]; face && k < in.contact_ptr[c + 1]; ++k)
        face = in.contact_sites[k] / plane == x;
      if (!face) { geo = false; break; }
      if (x == 0) x0 = 1;
      else x1 = in.dims[0] - 2;
      faces += cnt;
    }
    if (geo && faces != n_dense) geo = false;
  }
  int top = -1;
  if (geo) {
    int lo[3] = {x0, 0, 0}, hi[3] = {x1, in.dims[1] - 1, in.dims[2] - 1};
    top = x0 <= x1 ? B.box(lo, hi) : -1;
  } else {
    std::vector<int> rest;
    rest.reserve(ns - n_dense);
    for (int64_t s = 0; s < ns; ++s)
      if (!in_dense[s]) rest.push_back((int)s);
    std::vector<int> mark(ns, -1);
    top = B.graph(std::move(rest), mark, 0);
  }
  for (int c : dense_c) {
    std::vector<int> sites(in.contact_sites + in.contact_ptr[c], in.contact_sites + in.contact_ptr[c + 1]);
    top = B.make(std::move(sites), top, -1);
  }
  if (rebuild) {
    // Merge the listed clusters' own sites into their parents (children of a merged cluster become
    // its parent's). A cluster left with more than two children gets pass-through clusters of no
    // own unknowns: each takes two subtrees and hands their updates on unchanged. Then a cluster of
    // more than max_cluster sites becomes a chain of pieces (each parent of the previous one).
    const int n0 = (int)first.size();
    if (n0 == 0) return "empty tree";
    std::vector<char> merged(n0, 0);
    for (int k = 0; k < in.n_merge; ++k) {
      const int c = in.merge[k];
      if (c < 0 || c >= n0) return "merge list: cluster id out of range";
      if (first[c].parent < 0) return "merge list: the root has no parent";
      merged[c] = 1;
    }
    std::vector<Cluster> out;
    Builder M(in, ns, leaf_max, out);
    auto make_split = [&](std::vector<int>&& sites, int c0, int c1) {
      const size_t K = (size_t)in.max_cluster;
      if (K == 0 || sites.size() <= K || (!sites.empty() && in_dense[sites[0]])) return M.make(std::move(sites), c0, c1);
      std::sort(sites.begin(), sites.end());
      int cur = -1;
      for (size_t a = 0; a < sites.size(); a += K) {
        std::vector<int> piece(sites.begin() + a, sites.begin() + std::min(sites.size(), a + K));
        cur = a == 0 ? M.make(std::move(piece), c0, c1) : M.make(std::move(piece), cur, -1);
      }
      return cur;
    };
    auto pair_up = [&](std::vector<int>& kids) {
      while (kids.size() > 2) {
        const int a = kids.back(); kids.pop_back();
        const int b = kids.back(); kids.pop_back();
        kids.push_back(M.make(std::vector<int>(), b, a));
      }
    };
    // own sites and new child ids of cluster i with its merged children folded in
    std::function<void(int, std::vector<int>&, std::vector<int>&)> gather =
        [&](int i, std::vector<int>& sites, std::vector<int>& kids) {
          sites.insert(sites.end(), first[i].sites.begin(), first[i].sites.end());
          for (int k = 0; k < first[i].nchild; ++k) {
            const int c = first[i].child[k];
            if (merged[c]) {
              gather(c, sites, kids);
            } else {
              std::vector<int> cs, ck;
              gather(c, cs, ck);
              pair_up(ck);
              kids.push_back(make_split(std::move(cs), ck.size() > 0 ? ck[0] : -1, ck.size() > 1 ? ck[1] : -1));
            }
          }
        };
    std::vector<int> rs, rk;
    gather(n0 - 1, rs, rk);
    pair_up(rk);
    make_split(std::move(rs), rk.size() > 0 ? rk[0] : -1, rk.size() > 1 ? rk[1] : -1);
    P.cl = std::move(out);
  }
  auto& cl = P.cl;
  const int nc = (int)cl.size();
  if (nc == 0) return "empty tree";
  int roots = 0;
  for (auto& c : cl) roots += (c.parent < 0);
  if (roots != 1 || cl.back().parent != -1) return "cluster tree is not a single rooted tree";

  // owners, heights, subtree ranges
  P.site_cluster.assign(ns, -1);
  P.site_local.assign(ns, -1);
  for (int i = 0; i < nc; ++i)
    for (size_t k = 0; k < cl[i].sites.size(); ++k) {
      int s = cl[i].sites[k];
      if (P.site_cluster[s] >= 0) return "site assigned twice";
      P.site_cluster[s] = i;
      P.site_local[s] = (int)k;
    }
  for (int64_t s = 0; s < ns; ++s)
    if (P.site_cluster[s] < 0) return "site not assigned";
  for (int c : dense_c) {
    Plan::Dense D;
    D.contact = c;
    D.cluster = P.site_cluster[in.contact_sites[in.contact_ptr[c]]];
    D.nu = (in.contact_ptr[c + 1] - in.contact_ptr[c]) * orb;
    D.blk = P.dense_elems;
    D.loc = (int64_t)P.dense_local.size();
    for (int64_t k = in.contact_ptr[c]; k < in.contact_ptr[c + 1]; ++k) {
      const int s = in.contact_sites[k];
      if (P.site_cluster[s] != D.cluster) return "a dense contact is split over clusters";
      for (int o = 0; o < orb; ++o) P.dense_local.push_back(P.site_local[s] * orb + o);
    }
    if ((int64_t)cl[D.cluster].sites.size() * orb != D.nu) return "a dense contact shares its cluster";
    P.dense_elems += D.nu * D.nu;
    P.dense.push_back(D);
  }
  for (int i = 0; i < nc; ++i) {
    cl[i].first_desc = i;
    cl[i].height = 0;
    for (int k = 0; k < cl[i].nchild; ++k) {
      const Cluster& c = cl[cl[i].child[k]];
      cl[i].first_desc = std::min(cl[i].first_desc, c.first_desc);
      cl[i].height = std::max(cl[i].height, c.height + 1);
    }
  }
  for (int i = nc - 1; i >= 0; --i) cl[i].depth = cl[i].parent < 0 ? 0 : cl[cl[i].parent].depth + 1;

  // contacts -> lesser flag and contact slot per unknown
  std::vector<int32_t> slot_of_unknown(in.n, -1);
  {
    int32_t slot = 0;
    for (int c = 0; c < in.n_contacts; ++c)
      for (int64_t k = in.contact_ptr[c]; k < in.contact_ptr[c + 1]; ++k) {
        int s = in.contact_sites[k];
        if (s < 0 || s >= ns) return "contact site out of range";
        for (int o = 0; o < orb; ++o) {
          if (slot_of_unknown[(int64_t)s * orb + o] >= 0) return "site appears in two contacts";
          slot_of_unknown[(int64_t)s * orb + o] = slot++;
        }
        cl[P.site_cluster[s]].lesser = true;
      }
  }
  for (int i = 0; i < nc; ++i)
    for (int k = 0; k < cl[i].nchild; ++k)
      if (cl[cl[i].child[k]].lesser) cl[i].lesser = true;

  // update sets U_i (sites), sorted by (owner, local) = permuted position
  auto key = [&](int s) { return ((int64_t)P.site_cluster[s] << 32) | (int64_t)P.site_local[s]; };
  auto is_anc = [&](int a, int i) { return cl[a].first_desc <= i && i < a; };   // a proper ancestor of i
  for (int i = 0; i < nc; ++i) {
    std::vector<int> cand;
    for (int s : cl[i].sites)
      for (int t : B.adj[s]) {
        int c = P.site_cluster[t];
        if (cl[i].first_desc <= c && c <= i) continue;
        if (!is_anc(c, i)) return "nested dissection separation violated";
        cand.push_back(t);
      }
    for (int k = 0; k < cl[i].nchild; ++k)
      for (int t : cl[cl[i].child[k]].usites)
        if (P.site_cluster[t] != i) cand.push_back(t);
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return key(a) < key(b); });
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cl[i].usites = std::move(cand);
    cl[i].n = (int64_t)cl[i].sites.size() * orb;
    cl[i].m = (int64_t)cl[i].usites.size() * orb;
  }

  // schedules
  int H = 0, D = 0;
  for (auto& c : cl) { H = std::max(H, c.height); D = std::max(D, c.depth); }
  P.by_height.assign(H + 1, {});
  P.by_depth.assign(D + 1, {});
  for (int i = 0; i < nc; ++i) {
    P.by_height[cl[i].height].push_back(i);
    P.by_depth[cl[i].depth].push_back(i);
  }

  // per-energy offsets
  P.off.resize(nc);
  for (int i = 0; i < nc; ++i) {
    P.off[i].aug = P.tot_aug;
    P.off[i].sq = P.tot_sq;
    P.tot_aug += cl[i].n * (cl[i].n + cl[i].m);
    P.tot_sq += cl[i].m * cl[i].m;
  }
  for (auto& lv : P.by_height) {
    int64_t sq = 0, au = 0;
    for (int i : lv) { sq += cl[i].m * cl[i].m; au += cl[i].n * cl[i].m; }
    P.max_level_sq = std::max(P.max_level_sq, sq);
    P.max_level_aug_u = std::max(P.max_level_aug_u, au);
  }
  for (auto& lv : P.by_depth) {
    int64_t sq = 0, au = 0;
    for (int i : lv) { sq += cl[i].m * cl[i].m; au += cl[i].n * cl[i].m; }
    P.max_level_sq = std::max(P.max_level_sq, sq);
    P.max_level_aug_u = std::max(P.max_level_aug_u, au);
  }

  // position of site t in U_i (site granularity), -1 if absent
  auto upos = [&](int i, int t) -> int64_t {
    const auto& U = cl[i].usites;
    int64_t kt = key(t);
    auto it = std::lower_bound(U.begin(), U.end(), kt, [&](int a, int64_t k) { return key(a) < k; });
    if (it == U.end() || *it != t) return -1;
    return it - U.begin();
  };
  // front position (site granularity, times orb) of site t in the front of cluster i
  auto fpos = [&](int i, int t) -> int64_t {
    if (P.site_cluster[t] == i) return (int64_t)P.site_local[t] * orb;
    int64_t k = upos(i, t);
    return k < 0 ? -1 : cl[i].n + k * orb;
  };

  // front assembly maps (children's update sets into the parent front)
  P.map_off.assign(2 * nc, -1);
  for (int i = 0; i < nc; ++i)
    for (int k = 0; k < cl[i].nchild; ++k) {
      int c = cl[i].child[k];
      P.map_off[2 * i + k] = (int64_t)P.map_child.size();
      P.map_child.resize(P.map_child.size() + cl[i].n + cl[i].m, -1);
      int32_t* mp = P.map_child.data() + P.map_off[2 * i + k];
      for (size_t a = 0; a < cl[c].usites.size(); ++a) {
        int64_t q = fpos(i, cl[c].usites[a]);
        if (q < 0) return "child update set not inside parent front";
        for (int o = 0; o < orb; ++o) mp[q + o] = (int32_t)(a * orb + o);
      }
    }

  // original H entries of each front, and contact slots of own unknowns
  P.h_off.assign(nc + 1, 0);
  P.own_off.assign(nc + 1, 0);
  for (int i = 0; i < nc; ++i) {
    P.h_off[i] = (int64_t)P.h_vi.size();
    P.own_off[i] = (int64_t)P.own_contact.size();
    for (size_t l = 0; l < cl[i].sites.size(); ++l) {
      int s = cl[i].sites[l];
      for (int o = 0; o < orb; ++o) {
        int64_t u = (int64_t)s * orb + o;
        int64_t r = (int64_t)l * orb + o;
        P.own_contact.push_back(slot_of_unknown[u]);
        for (int64_t e = in.rowptr[u]; e < in.rowptr[u + 1]; ++e) {
          int64_t v = in.col[e];
          int t = (int)(v / orb), ov = (int)(v % orb);
          int c = P.site_cluster[t];
          int64_t q;
          if (c == i) q = (int64_t)P.site_local[t] * orb + ov;
          else if (is_anc(c, i)) {
            int64_t k = upos(i, t);
            if (k < 0) return "ancestor neighbour missing from update set";
            q = cl[i].n + k * orb + ov;
          } else continue;   // entry lives in a descendant's front (by symmetry)
          P.h_rq.push_back((int32_t)r);
          P.h_rq.push_back((int32_t)q);
          P.h_vi.push_back(e);
        }
      }
    }
  }
  P.h_off[nc] = (int64_t)P.h_vi.size();
  P.own_off[nc] = (int64_t)P.own_contact.size();

  // downward gather maps
  P.u_off.assign(nc + 1, 0);
  P.pm_off.assign(nc + 1, 0);
  P.nseg.assign(nc, 0);
  for (int i = 0; i < nc; ++i) {
    P.u_off[i] = (int64_t)P.u_owner.size();
    P.pm_off[i] = (int64_t)P.posmap.size();
    std::vector<int> segs;
    for (int t : cl[i].usites) {
      int c = P.site_cluster[t];
      if (segs.empty() || segs.back() != c) segs.push_back(c);
    }
    P.nseg[i] = (int32_t)segs.size();
    int sidx = -1, prev = -1;
    for (int t : cl[i].usites) {
      int c = P.site_cluster[t];
      if (c != prev) { ++sidx; prev = c; }
      for (int o = 0; o < orb; ++o) {
        P.u_owner.push_back(c);
        P.u_local.push_back(P.site_local[t] * orb + o);
        P.u_seg.push_back(sidx);
      }
    }
    for (int t : cl[i].usites)
      for (int o = 0; o < orb; ++o)
        for (int s = 0; s < (int)segs.size(); ++s) {
          int p = segs[s];
          int32_t v = -1;
          if (P.site_cluster[t] != p && is_anc(P.site_cluster[t], p)) {
            int64_t k = upos(p, t);
            if (k < 0) return "update-set closure violated";
            v = (int32_t)(k * orb + o);
          }
          P.posmap.push_back(v);
        }
  }
  P.u_off[nc] = (int64_t)P.u_owner.size();
  P.pm_off[nc] = (int64_t)P.posmap.size();

  // unknown -> (cluster, local)
  P.unk_cluster.resize(in.n);
  P.unk_local.resize(in.n);
  P.iperm.resize(in.n);
  {
    std::vector<int64_t> start(nc + 1, 0);
    for (int i = 0; i < nc; ++i) start[i + 1] = start[i] + cl[i].n;
    for (int64_t u = 0; u < in.n; ++u) {
      int s = (int)(u / orb);
      P.unk_cluster[u] = P.site_cluster[s];
      P.unk_local[u] = P.site_local[s] * orb + (int)(u % orb);
      P.iperm[u] = start[P.site_cluster[s]] + P.unk_local[u];
    }
  }

  // operation-count model (complex multiply-adds, 8 real flops each) of the implemented path
  double gr = 0, gl = 0;
  for (int i = 0; i < nc; ++i) {
    double n = (double)cl[i].n, m = (double)cl[i].m;
    gr += n * n * (n + m);        // in-place Gauss-Jordan on [A_ii | A_iU]
    gr += n * m * m;              // Schur update S = S - A_Ui X
    gr += n * m * m + n * n * m;  // G_iU, G_ii
    if (cl[i].lesser) {
      double w = n;   // rows of the lesser front that can be non-zero
      bool leaf = cl[i].nchild == 0;
      if (leaf) {     // leaves: diag(Sigma^<) on the hull of the own contact rows, L_iU = 0
        int64_t lo = cl[i].n, hi = -1;
        for (int64_t r = 0; r < cl[i].n; ++r)
          if (P.own_contact[P.own_off[i] + r] >= 0) { lo = std::min(lo, r); hi = r; }
        w = hi >= lo ? (double)(hi - lo + 1) : 0.0;
        gl += w * w * m + w * m * m;                          // fold T, Z
        gl += w * w * m + w * w * n + n * w * (n + m);        // N_iU, N_ii rows, W
      } else {
        gl += n * n * m + n * m * m;                  // lesser fold T, Z
        gl += (n * n * m + n * m * m) + (n * n * n + n * n * m) + n * n * (n + m);   // N, W
      }
    }
    gl += n * m * m + n * n * m;  // P_iU, P_ii
  }
  P.flops_gr = 8.0 * gr;
  P.flops_gl = 8.0 * gl;
  return "";
}

}  // namespace hsc
