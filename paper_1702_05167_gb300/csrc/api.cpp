// Host half of the C ABI: handle creation, validation, analysis and tree queries (no GPU work).
#include <algorithm>
#include <cstring>
#include <vector>
#include <new>
#include <string>

#include "ctx.h"

static thread_local std::string g_err;

int hsc_fail(hsc_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

extern "C" int hsc_create(hsc_t* out, int64_t n, int32_t orb, const int64_t* rowptr,
                          const int32_t* col, const hsc_c128* val, int32_t n_contacts,
                          const int64_t* contact_ptr, const int32_t* contact_sites,
                          const int32_t* grid_dims) {
  if (!out) return hsc_fail(nullptr, HSC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || orb <= 0 || n % orb) return hsc_fail(nullptr, HSC_ERR_ARG, "n must be a positive multiple of orb");
  if (!rowptr || !col || !val) return hsc_fail(nullptr, HSC_ERR_ARG, "CSR pointer is NULL");
  if (n_contacts < 0 || (n_contacts > 0 && (!contact_ptr || !contact_sites)))
    return hsc_fail(nullptr, HSC_ERR_ARG, "bad contact arrays");
  if (rowptr[0] != 0) return hsc_fail(nullptr, HSC_ERR_ARG, "rowptr[0] != 0");
  for (int64_t u = 0; u < n; ++u)
    if (rowptr[u + 1] < rowptr[u]) return hsc_fail(nullptr, HSC_ERR_ARG, "rowptr not monotone");
  const int64_t nnz = rowptr[n];
  for (int64_t e = 0; e < nnz; ++e)
    if (col[e] < 0 || col[e] >= n) return hsc_fail(nullptr, HSC_ERR_ARG, "column index out of range");
  // complex symmetry H = H^T (Eq. 3: the block LDL^T form needs A = A^T): the sorted entry list
  // (row, col, value) must equal the sorted list of (col, row, value)
  {
    struct Ent { int64_t r, c; double re, im; };
    std::vector<Ent> a, b;
    try {
      a.reserve(nnz);
      b.reserve(nnz);
    } catch (...) {
      return hsc_fail(nullptr, HSC_ERR_OOM, "out of host memory");
    }
    for (int64_t u = 0; u < n; ++u)
      for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
        a.push_back({u, col[e], val[e].re, val[e].im});
        b.push_back({col[e], u, val[e].re, val[e].im});
      }
    auto lt = [](const Ent& x, const Ent& y) {
      if (x.r != y.r) return x.r < y.r;
      if (x.c != y.c) return x.c < y.c;
      if (x.re != y.re) return x.re < y.re;
      return x.im < y.im;
    };
    std::sort(a.begin(), a.end(), lt);
    std::sort(b.begin(), b.end(), lt);
    for (int64_t k = 0; k < nnz; ++k)
      if (a[k].r != b[k].r || a[k].c != b[k].c || a[k].re != b[k].re || a[k].im != b[k].im)
        return hsc_fail(nullptr, HSC_ERR_NOT_SYMMETRIC, "H is not complex symmetric (H != H^T)");
  }
  int64_t n_sites = n / orb, ncu = 0;
  if (n_contacts > 0) {
    if (contact_ptr[0] != 0) return hsc_fail(nullptr, HSC_ERR_ARG, "contact_ptr[0] != 0");
    for (int c = 0; c < n_contacts; ++c) {
      if (contact_ptr[c + 1] < contact_ptr[c]) return hsc_fail(nullptr, HSC_ERR_ARG, "contact_ptr not monotone");
      for (int64_t k = contact_ptr[c]; k < contact_ptr[c + 1]; ++k)
        if (contact_sites[k] < 0 || contact_sites[k] >= n_sites)
          return hsc_fail(nullptr, HSC_ERR_ARG, "contact site out of range");
    }
    ncu = contact_ptr[n_contacts] * orb;
  }
  if (grid_dims) {
    if (grid_dims[0] <= 0 || grid_dims[1] <= 0 || grid_dims[2] <= 0 ||
        (int64_t)grid_dims[0] * grid_dims[1] * grid_dims[2] != n_sites)
      return hsc_fail(nullptr, HSC_ERR_ARG, "grid_dims do not match n/orb");
  }
  hsc_ctx* h = new (std::nothrow) hsc_ctx();
  if (!h) return hsc_fail(nullptr, HSC_ERR_OOM, "out of host memory");
  try {
    h->n = n;
    h->orb = orb;
    h->rowptr.assign(rowptr, rowptr + n + 1);
    h->col.assign(col, col + nnz);
    h->val.assign(val, val + nnz);
    h->n_contacts = n_contacts;
    if (n_contacts > 0) {
      h->contact_ptr.assign(contact_ptr, contact_ptr + n_contacts + 1);
      h->contact_sites.assign(contact_sites, contact_sites + contact_ptr[n_contacts]);
    } else {
      h->contact_ptr.assign(1, 0);
    }
    h->n_contact_unknowns = ncu;
    if (grid_dims) std::memcpy(h->dims, grid_dims, sizeof(h->dims));
  } catch (...) {
    delete h;
    return hsc_fail(nullptr, HSC_ERR_OOM, "out of host memory");
  }
  *out = h;
  g_err.clear();
  return HSC_OK;
}

extern "C" int hsc_analyze(hsc_t h, int32_t leaf_max, hsc_tree_stats* stats) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  h->analyzed = false;
  hsc::device_state_free(h->dev);   // the device schedule belongs to the previous tree
  h->dev = nullptr;
  h->band_pairs.clear();
  hsc::Input in;
  in.n = h->n;
  in.orb = h->orb;
  in.rowptr = h->rowptr.data();
  in.col = h->col.data();
  in.n_contacts = h->n_contacts;
  in.contact_ptr = h->contact_ptr.data();
  in.contact_sites = h->contact_sites.data();
  std::memcpy(in.dims, h->dims, sizeof(in.dims));
  if (h->opt_ordering == 1) in.dims[0] = in.dims[1] = in.dims[2] = 0;   // graph bisection
  if (h->opt_ordering == 0 && in.dims[0] > 0) {
    // contact-connected dissection when every contact site lies on x = 0 or x = Nx-1 and both end
    // planes hold some (a two-terminal device along x); otherwise the plain geometric form
    const int64_t plane = (int64_t)in.dims[1] * in.dims[2];
    bool lo = false, hi = false, ends = plane > 0;
    for (int64_t k = 0; ends && k < (int64_t)h->contact_sites.size(); ++k) {
      const int64_t x = h->contact_sites[k] / plane;
      lo |= x == 0;
      hi |= x == in.dims[0] - 1;
      ends = x == 0 || x == in.dims[0] - 1;
    }
    in.contact_connected = ends && lo && hi && in.dims[0] >= 3 ? 1 : 0;
  }
  in.variant = h->nd_variant;
  in.contact_dense = h->contact_dense.empty() ? nullptr : h->contact_dense.data();
  in.merge = h->merge.empty() ? nullptr : h->merge.data();
  in.max_cluster = h->opt_max_cluster;
  in.n_merge = (int)h->merge.size();
  hsc_drop_alt(h);   // the twin follows the leaf size of this analysis
  std::string e;
  try {
    e = hsc::analyze(in, leaf_max, h->plan);
    if (e.empty() && in.contact_connected) {
      // an elongated device makes the half-device boxes costly: keep the contact-connected tree
      // only while its model cost stays within 3x the plain geometric tree's (or below 1 GFLOP per
      // energy, where the cost does not matter)
      hsc::Input plain = in;
      plain.contact_connected = 0;
      hsc::Plan alt;
      e = hsc::analyze(plain, leaf_max, alt);
      const double fc = h->plan.flops_gr + h->plan.flops_gl, fp = alt.flops_gr + alt.flops_gl;
      if (e.empty() && fc > 3.0 * fp && fc > 1e9) {
        h->plan = std::move(alt);
        in.contact_connected = 0;
      }
    }
  } catch (const std::bad_alloc&) {
    return hsc_fail(h, HSC_ERR_OOM, "out of host memory in analyze");
  }
  if (!e.empty()) return hsc_fail(h, HSC_ERR_ARG, e);
  h->tree_form = in.dims[0] <= 0 ? 2 : (in.contact_connected ? 1 : 0);
  const hsc::Plan& P = h->plan;
  hsc_tree_stats s{};
  s.n_clusters = (int32_t)P.cl.size();
  s.n_heights = (int32_t)P.by_height.size();
  s.n_depths = (int32_t)P.by_depth.size();
  for (const auto& c : P.cl) {
    s.max_n = std::max<int32_t>(s.max_n, (int32_t)c.n);
    s.max_m = std::max<int32_t>(s.max_m, (int32_t)c.m);
    s.n_lesser += c.lesser ? 1 : 0;
  }
  s.n_unknowns = h->n;
  s.flops_gr = P.flops_gr;
  s.flops_gl = P.flops_gl;
  // per energy: F, G, P, L (aug) and S, LS (square) in complex128
  s.bytes_per_energy = (4 * P.tot_aug + 2 * P.tot_sq) * 16;
  h->stats = s;
  if (stats) *stats = s;
  h->leaf_max = leaf_max;
  h->analyzed = true;
  h->err.clear();
  return HSC_OK;
}

extern "C" int hsc_cluster(hsc_t h, int32_t i, hsc_cluster_info* info, int32_t* own, int32_t* upd) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (!h->analyzed) return hsc_fail(h, HSC_ERR_STATE, "hsc_analyze has not run");
  const hsc::Plan& P = h->plan;
  if (i < 0 || i >= (int32_t)P.cl.size()) return hsc_fail(h, HSC_ERR_ARG, "cluster index out of range");
  const hsc::Cluster& c = P.cl[i];
  if (info) {
    info->n = (int32_t)c.n;
    info->m = (int32_t)c.m;
    info->parent = c.parent;
    info->child[0] = c.child[0];
    info->child[1] = c.child[1];
    info->height = c.height;
    info->depth = c.depth;
    info->lesser = c.lesser ? 1 : 0;
  }
  const int orb = h->orb;
  if (own)
    for (size_t k = 0; k < c.sites.size(); ++k)
      for (int o = 0; o < orb; ++o) own[k * orb + o] = c.sites[k] * orb + o;
  if (upd)
    for (size_t k = 0; k < c.usites.size(); ++k)
      for (int o = 0; o < orb; ++o) upd[k * orb + o] = c.usites[k] * orb + o;
  return HSC_OK;
}

extern "C" int hsc_set_option(hsc_t h, int32_t option, int32_t value) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  switch (option) {
    case HSC_OPT_GJ_PANEL:
      if (value < 1 || value > 64) return hsc_fail(h, HSC_ERR_ARG, "panel width must be in [1, 64]");
      h->opt_nb = value;
      break;
    case HSC_OPT_GJ_WIDE:
      if (value < 0 || value > 512) return hsc_fail(h, HSC_ERR_ARG, "wide panel width must be in [0, 512]");
      h->opt_nbo = value;
      break;
    case HSC_OPT_FP64_LEVELS:
      if (value < 0) return hsc_fail(h, HSC_ERR_ARG, "levels must be >= 0");
      h->opt_fp64_levels = value;
      break;
    case HSC_OPT_MIXED_GJ_FP64:
      h->opt_gj_fp64 = value != 0;
      break;
    case HSC_OPT_COMPLEX_4M:
      h->opt_4m = value != 0;
      break;
    case HSC_OPT_FP64_ENGINE:
      if (value < 0 || value > 2) return hsc_fail(h, HSC_ERR_ARG, "engine must be 0, 1 or 2");
      h->opt_fp64_engine = value;
      break;
    case HSC_OPT_RESOLVE_DIGITS:
      if (value < 0 || value > 15) return hsc_fail(h, HSC_ERR_ARG, "residual digits must be in [0, 15]");
      h->opt_resolve = value;
      break;
    case HSC_OPT_TREE_VARIANT:
      if (value < 0 || value > 4 || h->is_alt) return hsc_fail(h, HSC_ERR_ARG, "tree variant must be in [0, 4]");
      h->nd_variant = value;
      break;
    case HSC_OPT_ORDERING:
      if (value < 0 || value > 2) return hsc_fail(h, HSC_ERR_ARG, "ordering must be 0, 1 or 2");
      h->opt_ordering = value;
      break;
    case HSC_OPT_MAX_CLUSTER:
      if (value < 0) return hsc_fail(h, HSC_ERR_ARG, "max cluster size must be >= 0");
      h->opt_max_cluster = value;
      break;
    case HSC_OPT_LEAF_BAND:
      if (value < 0 || value > 1) return hsc_fail(h, HSC_ERR_ARG, "leaf band must be 0 or 1");
      h->opt_leaf_band = value;
      break;
    case HSC_OPT_LEAF_SPARSE:
      if (value < 0 || value > 1) return hsc_fail(h, HSC_ERR_ARG, "leaf sparse must be 0 or 1");
      h->opt_leaf_sparse = value;
      break;
    default:
      return hsc_fail(h, HSC_ERR_ARG, "unknown option");
  }
  hsc::device_state_free(h->dev);   // schedules depend on the options
  h->dev = nullptr;
  hsc_drop_alt(h);
  return HSC_OK;
}

extern "C" int hsc_get_option(hsc_t h, int32_t option, int32_t* value) {
  if (!h || !value) return hsc_fail(h, HSC_ERR_ARG, "NULL argument");
  switch (option) {
    case HSC_OPT_GJ_PANEL: *value = h->opt_nb; break;
    case HSC_OPT_GJ_WIDE: *value = h->opt_nbo; break;
    case HSC_OPT_LEAF_BAND: *value = h->opt_leaf_band; break;
    case HSC_OPT_LEAF_SPARSE: *value = h->opt_leaf_sparse; break;
    case HSC_OPT_FP64_LEVELS: *value = h->opt_fp64_levels; break;
    case HSC_OPT_MIXED_GJ_FP64: *value = h->opt_gj_fp64; break;
    case HSC_OPT_LEAF: *value = h->leaf_max; break;
    case HSC_OPT_COMPLEX_4M: *value = h->opt_4m; break;
    case HSC_OPT_FP64_ENGINE: *value = h->opt_fp64_engine; break;
    case HSC_OPT_RESOLVE_DIGITS: *value = h->opt_resolve; break;
    case HSC_OPT_TREE_VARIANT: *value = h->nd_variant; break;
    case HSC_OPT_ORDERING: *value = h->opt_ordering; break;
    case HSC_OPT_TREE_FORM: *value = h->analyzed ? h->tree_form : -1; break;
    case HSC_OPT_MAX_CLUSTER: *value = h->opt_max_cluster; break;
    default: return hsc_fail(h, HSC_ERR_ARG, "unknown option");
  }
  return HSC_OK;
}

extern "C" int hsc_set_merge(hsc_t h, int32_t n, const int32_t* clusters) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (h->is_alt || n < 0 || (n > 0 && !clusters)) return hsc_fail(h, HSC_ERR_ARG, "bad merge list");
  for (int32_t k = 0; k < n; ++k)
    if (clusters[k] < 0) return hsc_fail(h, HSC_ERR_ARG, "negative cluster id in the merge list");
  h->merge.assign(clusters, clusters + n);
  h->analyzed = false;   // the tree changes: analyse again
  hsc::device_state_free(h->dev);
  h->dev = nullptr;
  hsc_drop_alt(h);
  h->err.clear();
  return HSC_OK;
}

extern "C" int hsc_set_contact_dense(hsc_t h, int32_t contact, int32_t dense) {
  if (!h) return hsc_fail(nullptr, HSC_ERR_ARG, "handle is NULL");
  if (h->is_alt || contact < 0 || contact >= h->n_contacts || (dense != 0 && dense != 1))
    return hsc_fail(h, HSC_ERR_ARG, "contact out of range or dense not 0/1");
  h->contact_dense.resize(h->n_contacts, 0);
  h->contact_dense[contact] = (char)dense;
  // the cluster tree depends on it: the handle must be analysed again
  h->analyzed = false;
  hsc::device_state_free(h->dev);
  h->dev = nullptr;
  hsc_drop_alt(h);
  h->err.clear();
  return HSC_OK;
}

extern "C" const char* hsc_last_error(hsc_t h) { return h ? h->err.c_str() : g_err.c_str(); }

void hsc_drop_alt(hsc_ctx* h) {
  for (hsc_ctx*& a : h->alt) {
    if (!a) continue;
    hsc::device_state_free(a->dev);
    delete a;
    a = nullptr;
  }
}

hsc_ctx* hsc_alt(hsc_ctx* h, int v) {
  if (v < 1 || v > 4) return nullptr;
  if (h->alt[v - 1]) return h->alt[v - 1];
  if (!h->analyzed || h->is_alt || v == h->nd_variant) return nullptr;
  hsc_ctx* a = new (std::nothrow) hsc_ctx();
  if (!a) return nullptr;
  a->n = h->n;
  a->orb = h->orb;
  a->rowptr = h->rowptr;
  a->col = h->col;
  a->val = h->val;
  a->n_contacts = h->n_contacts;
  a->contact_ptr = h->contact_ptr;
  a->contact_sites = h->contact_sites;
  a->n_contact_unknowns = h->n_contact_unknowns;
  a->contact_dense = h->contact_dense;
  std::memcpy(a->dims, h->dims, sizeof(a->dims));
  a->opt_nb = h->opt_nb;
  a->opt_nbo = h->opt_nbo;
  a->opt_leaf_band = h->opt_leaf_band;
  a->opt_leaf_sparse = h->opt_leaf_sparse;
  a->opt_fp64_levels = h->opt_fp64_levels;
  a->opt_gj_fp64 = h->opt_gj_fp64;
  a->opt_4m = h->opt_4m;
  a->opt_fp64_engine = h->opt_fp64_engine;
  a->opt_ordering = h->opt_ordering;
  a->opt_max_cluster = h->opt_max_cluster;
  a->nd_variant = v;
  a->is_alt = true;
  if (hsc_analyze(a, h->leaf_max, nullptr) != HSC_OK) {
    delete a;
    return nullptr;
  }
  h->alt[v - 1] = a;
  return a;
}

extern "C" int hsc_destroy(hsc_t h) {
  if (!h) return HSC_OK;
  hsc::device_state_free(h->dev);
  hsc_drop_alt(h);
  delete h;
  return HSC_OK;
}
