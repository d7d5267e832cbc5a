// Handle state shared by the host API (api.cpp) and the device driver (solve.cu).
#pragma once
#include <string>
#include <vector>

#include "../../include/hsc.h"
#include "plan.h"

namespace hsc {
struct DeviceState;                 // defined in solve.cu
void device_state_free(DeviceState*);
}  // namespace hsc

struct hsc_ctx {
  int64_t n = 0;
  int orb = 1;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<hsc_c128> val;
  int n_contacts = 0;
  std::vector<int64_t> contact_ptr;
  std::vector<int32_t> contact_sites;
  int64_t n_contact_unknowns = 0;
  std::vector<char> contact_dense;   // per contact: 1 = DENSE self-energy block (hsc_set_contact_dense)
  int dims[3] = {0, 0, 0};
  bool analyzed = false;
  hsc::Plan plan;
  hsc_tree_stats stats{};
  std::string err;
  hsc::DeviceState* dev = nullptr;
  // options (hsc_set_option); they survive re-analysis
  int opt_nb = 16;            // Gauss-Jordan panel width (its trailing updates are GEMMs with K = width)
  int opt_nbo = 128;          // wide panel of the nested blocking (trailing products with K = this)
  int opt_fp64_levels = 2;    // HSC_MIXED: top tree levels kept on the FP64 pipe
  int opt_gj_fp64 = 0;        // HSC_MIXED: Gauss-Jordan trailing updates on the FP64 pipe
  int opt_4m = 0;             // FP64 engine: 4 real products per complex product (default 3)
  int opt_fp64_engine = 0;    // FP64-accurate products: 0 cost model, 1 FP64 pipe, 2 emulation
  int opt_resolve = 10;       // d: re-solve energies whose residual exceeds 10^-d (0: off)
  int opt_leaf_band = 1;      // leaves' G_ii, G^<_ii: only the column bands their readers need
  int opt_leaf_sparse = 1;    // leaves' X and Schur products from the sparse coupling block
  std::vector<int64_t> band_pairs;   // requested pairs inside leaf blocks (positions) the current
                                     // schedule's bands cover; cleared by re-analysis
  int opt_ordering = 0;       // 0: geometric (contact-connected for end-plane contacts), 1: graph
                              // bisection, 2: plain geometric (longest extent at every level)
  int tree_form = -1;         // tree of the last analyze: 0 plain geometric, 1 contact-connected,
                              // 2 graph bisection
  std::vector<int32_t> merge; // clusters merged into their parents by the next analyze
  int opt_max_cluster = 0;    // > 0: split larger clusters into chains (next analyze)
  int leaf_max = 0;           // last hsc_analyze leaf size
  // alternate separator trees 1..4 (cuts below the root shifted), built on first need by hsc_solve
  int nd_variant = 0;
  bool is_alt = false;
  hsc_ctx* alt[4] = {nullptr, nullptr, nullptr, nullptr};
};

int hsc_fail(hsc_ctx* h, int code, const std::string& msg);
// The alternate-tree twin of h for variant v (1..4): same matrix, contacts and options, analysed
// at h's leaf size; created on first call; nullptr if it cannot be built.
hsc_ctx* hsc_alt(hsc_ctx* h, int v);
void hsc_drop_alt(hsc_ctx* h);
