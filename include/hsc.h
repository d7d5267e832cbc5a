/* hsc.h -- C ABI of the GB300 HSC-extension selected-inversion library (libhsc.so).
 *
 * Computes, for many energies E in one call, selected entries of
 *     G^r(E) = A(E)^{-1},   A(E) = (E + i*eta) I - H - Sigma^r(E)          (Eq. 1)
 *     G^<(E) = G^r(E) Sigma^<(E) G^r(E)^dagger                             (Eq. 2)
 * by nested-dissection selected inversion: Algorithm 1 (HSC, G^r) and Algorithm 2 (HSC-extension,
 * G^<) over the binary cluster tree of Section 2.2. Selected entries are the diagonal and any
 * (a, b) inside the filled pattern of the ordered factorisation; every pair with H_ab != 0 is in it.
 *
 * Conventions
 *   - H is complex symmetric (H = H^T), given in CSR over n unknowns; the algorithms use transposes,
 *     not adjoints (Eq. 3 and Algorithm 1 rely on A = A^T).
 *   - Unknown u of site s and orbital o is u = s*orb + o. Contacts are sets of sites; the contact
 *     unknowns are listed contact after contact, site after site, orbital after orbital, and the
 *     self-energy arrays are indexed in that order ("contact slots").
 *   - Sigma^r and Sigma^< are diagonal on the contact unknowns (Section 3.1.1, SPARSE self-energy).
 *   - Complex numbers are interleaved (re, im) doubles. All outputs are in user (CSR) order.
 *   - Every call returns an hsc_status; no exception crosses the ABI; hsc_last_error() gives text.
 *   - A handle is not thread safe; distinct handles are independent.
 */
#ifndef HSC_H
#define HSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsc_ctx* hsc_t;
typedef struct { double re, im; } hsc_c128;

typedef enum {
  HSC_OK = 0,
  HSC_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, index out of range)  */
  HSC_ERR_NOT_SYMMETRIC = 2,  /* H != H^T                                                       */
  HSC_ERR_STATE = 3,          /* call out of order (solve before analyze)                        */
  HSC_ERR_SINGULAR = 4,       /* zero pivot in a cluster block (only possible with eta = 0)      */
  HSC_ERR_NOT_SELECTED = 5,   /* requested pair outside the filled pattern                       */
  HSC_ERR_OOM = 6,            /* device or host allocation failed                                */
  HSC_ERR_CUDA = 7,           /* CUDA runtime error (message in hsc_last_error)                  */
  HSC_ERR_TIMEOUT = 8         /* a bounded device-side wait expired                             */
} hsc_status;

typedef enum { HSC_FP64 = 0, HSC_MIXED = 1 } hsc_precision;

typedef struct {
  int32_t n_clusters;       /* clusters in the tree                                         */
  int32_t n_heights;        /* upward stages (leaves are height 0)                          */
  int32_t n_depths;         /* downward stages (root is depth 0)                            */
  int32_t max_n;            /* largest cluster (unknowns)                                   */
  int32_t max_m;            /* largest update set |U_i| (unknowns)                          */
  int32_t n_lesser;         /* clusters whose subtree touches a contact                     */
  int64_t n_unknowns;
  double flops_gr;          /* model: real flops per energy for G^r (complex MAC = 8)        */
  double flops_gl;          /* model: real flops per energy for G^<                          */
  int64_t bytes_per_energy; /* device workspace per energy of a solve                       */
} hsc_tree_stats;

typedef struct {
  int32_t n, m;             /* own unknowns, update-set unknowns                            */
  int32_t parent;           /* -1 for the root                                              */
  int32_t child[2];         /* -1 where absent                                              */
  int32_t height, depth;
  int32_t lesser;           /* 1 if the subtree holds a contact unknown                     */
} hsc_cluster_info;

/* hsc_create -- copy the device description into a new handle (no GPU work).
 *   n            number of unknowns (multiple of orb)
 *   orb          orbitals per site
 *   rowptr,col,val  H in CSR over unknowns: rowptr[n+1] (int64), col[nnz] (int32), val[nnz];
 *                 host memory, read only during the call (the handle keeps its own copy)
 *   n_contacts, contact_ptr[n_contacts+1], contact_sites[...]  site sets of the contacts (host)
 *   grid_dims    optional {Nx, Ny, Nz} (site = (x*Ny + y)*Nz + z): geometric nested dissection;
 *                NULL selects breadth-first level-set bisection of the site graph.
 * Errors: HSC_ERR_ARG (sizes, indices), HSC_ERR_NOT_SYMMETRIC (H != H^T), HSC_ERR_OOM.
 * On error *out is set to NULL. Cite: Eq. 1 (H, Sigma^r), Section 3.1 (cuboid grids). */
int hsc_create(hsc_t* out, int64_t n, int32_t orb,
               const int64_t* rowptr, const int32_t* col, const hsc_c128* val,
               int32_t n_contacts, const int64_t* contact_ptr, const int32_t* contact_sites,
               const int32_t* grid_dims);

/* hsc_analyze -- build the cluster tree (Section 2.2, multilevel nested dissection), the update
 *   sets, the assembly/gather maps and the operation-count model. Host only; no GPU work.
 *   leaf_max: geometric ND stops when every extent of a box is <= leaf_max sites; graph ND stops
 *   at leaf_max^3 sites. stats may be NULL. Errors: HSC_ERR_ARG, HSC_ERR_OOM. */
int hsc_analyze(hsc_t h, int32_t leaf_max, hsc_tree_stats* stats);

/* hsc_set_merge -- merge clusters into their parents at the next hsc_analyze.
 *   clusters[n]: ids of the tree that hsc_analyze builds without a merge list (n = 0 clears it). Each
 *   listed cluster's own unknowns join its parent's and its children become the parent's; where a
 *   cluster would get more than two children, pass-through clusters with no own unknowns pair them
 *   up (their fronts carry the children's updates on unchanged). Delayed pivoting at cluster
 *   granularity: a cluster whose block has a level close to E is eliminated together with its
 *   separator. The call discards the tree and device state: hsc_analyze must run again.
 *   The analysis is tested on the CPU; solves on merged trees have not been run on a GB300 yet.
 *   Errors: HSC_ERR_ARG (negative id; at hsc_analyze: id out of range or the root). */
int hsc_set_merge(hsc_t h, int32_t n, const int32_t* clusters);

/* hsc_set_contact_dense -- mark contact `contact` as DENSE (dense = 1) or diagonal (0, the default).
 *   Section 3.1.2 models open boundaries with a dense self-energy block on the contact layer, which
 *   couples every pair of the contact's unknowns. The next hsc_analyze then keeps each dense
 *   contact's unknowns in one cluster, chained on top of the nested dissection of the remaining
 *   sites (geometric dissection of the interior box when the dense contacts are whole end planes
 *   x = 0 / x = Nx-1, else graph bisection of the rest), so that block stays inside one front.
 *   The call discards the handle's tree and device state: hsc_analyze must run again.
 *   Solves on such a tree take the diagonal self-energies of hsc_solve; the dense block itself is
 *   not an input of hsc_solve yet.
 *   Errors: HSC_ERR_ARG (contact out of range, dense not 0 or 1). */
int hsc_set_contact_dense(hsc_t h, int32_t contact, int32_t dense);

/* hsc_cluster -- describe cluster i (postorder id, root = n_clusters-1) after hsc_analyze.
 *   own/upd: optional host arrays of at least n / m int32 entries receiving the user-order unknowns
 *   of the cluster and of its update set U_i (ascending in the cluster ordering).
 * Errors: HSC_ERR_STATE, HSC_ERR_ARG. */
int hsc_cluster(hsc_t h, int32_t i, hsc_cluster_info* info, int32_t* own, int32_t* upd);

/* hsc_solve -- selected G^r and G^< at n_E energies (Algorithms 1 and 2).
 *   E[n_E]                energies (eV); eta (eV) > 0 recommended (eta = 0 may be singular)
 *   sigma_r[n_E][n_cs]    diagonal Sigma^r on the n_cs contact slots, per energy
 *   sigma_less[n_E][n_cs] diagonal Sigma^< per energy, or NULL: G^< work and outputs are skipped.
 *                         Sigma^< must be anti-Hermitian (purely imaginary diagonal, i f Gamma for a
 *                         contact): Algorithm 2 builds G^< from that symmetry, and a real part is
 *                         not carried consistently
 *   precision             HSC_FP64: complex128 storage, every block product on the FP64 pipe.
 *                         HSC_MIXED: complex128 storage; block products below the top tree levels
 *                         (HSC_FP64_LEVELS, default 2: the root and its children stay FP64) run on
 *                         the tensor cores as 3xTF32 split products with FP32 accumulation
 *                         (~1e-6 relative per product). Cluster inverses keep FP64 panels
 *                         (HSC_MIXED_GJ_FP64=1 also keeps their trailing updates on the FP64 pipe).
 *                         Accuracy degrades with the elimination's growth (~||H||/eta).
 *   n_req, req_pairs[n_req][2]  user-order unknown pairs (a, b) whose G^r_ab (and G^<_ab) are
 *                         returned; every pair must be in the filled pattern
 *   diag_gr[n_E][n]       out: G^r_uu;            diag_gl[n_E][n] out: G^<_uu (ignored if
 *                         sigma_less is NULL);    req_gr[n_E][n_req], req_gl[n_E][n_req] out (may be
 *                         NULL when n_req = 0)
 *   cuda_stream           cudaStream_t to run on (NULL: the legacy default stream)
 *   io_on_device          0: E, sigma_*, req_pairs and all outputs are host memory (the call copies
 *                         them in and out through device staging buffers);
 *                         1: E, sigma_* and outputs are device memory (req_pairs stays on the host).
 *                         In both modes the call synchronises cuda_stream before returning, to
 *                         read the device error flags (singular pivot, internal map error).
 * The handle owns its device workspace (allocated on the first solve, grown as needed, freed by
 * hsc_destroy). Energies are processed in waves that fit the workspace budget
 * (HSC_WORKSPACE_GB caps it; default 85% of the free device memory).
 * Errors: HSC_ERR_STATE (no analyze), HSC_ERR_ARG, HSC_ERR_NOT_SELECTED, HSC_ERR_OOM,
 *   HSC_ERR_CUDA, HSC_ERR_SINGULAR (reported after the fact from a device flag). */
int hsc_solve(hsc_t h, int64_t n_E, const double* E, double eta,
              const hsc_c128* sigma_r, const hsc_c128* sigma_less, int32_t precision,
              int32_t n_req, const int32_t* req_pairs,
              hsc_c128* diag_gr, hsc_c128* diag_gl, hsc_c128* req_gr, hsc_c128* req_gl,
              void* cuda_stream, int32_t io_on_device);

/* hsc_solve_dense -- hsc_solve with DENSE contact self-energy blocks (Section 3.1.2) added.
 *   Needs at least one contact marked with hsc_set_contact_dense before hsc_analyze.
 *   dense_r[n_E][n_dense]   per energy, the blocks of the dense contacts in contact order, each
 *                           nu x nu row-major over the contact's unknowns in slot order (nu = its
 *                           sites x orb; n_dense = sum of nu^2). Sigma^r = diag(sigma_r) + blocks.
 *   dense_less[n_E][n_dense] the same for Sigma^< (anti-Hermitian, as i f Gamma); required exactly
 *                           when sigma_less is given
 *   Everything else as hsc_solve (dense_* on the device when io_on_device = 1; with host I/O they
 *   are staged on the device whole). The blocks are complex symmetric for a lead Hamiltonian that
 *   is (Sigma^r = tau g_s tau^T). No residual record and no re-solve: the residual kernel handles
 *   diagonal self-energies only, so hsc_residual is not defined after this call.
 *   Not yet run on a GB300 (the kernel adding the blocks, k_add_dense, is compiled and reviewed).
 *   Errors: as hsc_solve; HSC_ERR_ARG when no contact is dense or the block arrays are missing. */
int hsc_solve_dense(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
                    const hsc_c128* sigma_less, const hsc_c128* dense_r, const hsc_c128* dense_less,
                    int32_t precision, int32_t n_req, const int32_t* req_pairs, hsc_c128* diag_gr,
                    hsc_c128* diag_gl, hsc_c128* req_gr, hsc_c128* req_gl, void* cuda_stream,
                    int32_t io_on_device);

/* Options of a handle (hsc_set_option / hsc_get_option). Setting one discards the handle's device
 * schedule and workspace (rebuilt by the next solve). HSC_OPT_LEAF is read-only (the leaf_max of
 * the last hsc_analyze). */
typedef enum {
  HSC_OPT_GJ_PANEL = 1,       /* Gauss-Jordan panel width, 1..64 (default 16)                   */
  HSC_OPT_FP64_LEVELS = 2,    /* HSC_MIXED: tree levels from the top kept on the FP64 pipe (2)  */
  HSC_OPT_MIXED_GJ_FP64 = 3,  /* HSC_MIXED: 1 keeps cluster-inverse updates on the FP64 pipe (0) */
  HSC_OPT_LEAF = 4,           /* read only                                                      */
  HSC_OPT_COMPLEX_4M = 5,     /* FP64 block products with 4 real products per complex product   */
                              /* (default 0: 3 products, Im = (Ar+Ai)(Br+Bi) - ArBr - AiBi, 25 % */
                              /* less FP64-pipe work, slightly larger rounding constant)        */
  HSC_OPT_FP64_ENGINE = 6,    /* engine of the FP64-accurate block products: 0 (default) picks  */
                              /* per product list by a cost model, 1 = FP64 pipe only, 2 = FP64 */
                              /* emulation on the BF16 tensor cores wherever K > 0. The         */
                              /* emulation writes each real operand in eight balanced base-128  */
                              /* digits (one power-of-two scale per row of A and column of B for*/
                              /* the real, imaginary and summed parts), accumulates the digit   */
                              /* products exactly and combines the complex result exactly before*/
                              /* one rounding per part; its error per K value and real product  */
                              /* is below 2^-54.5 times the two scales, FP64 rounding level.    */
  HSC_OPT_RESOLVE_DIGITS = 7, /* d > 0: hsc_solve solves every energy whose residual (see      */
                              /* hsc_residual; default d = 10: on the 32^3 cube at eta = 1e-6   */
                              /* the default tree leaves 3 of 64 energies above 1e-10, the      */
                              /* median is 1e-11) exceeds 10^-d again on the alternate separator*/
                              /* trees in turn (the root plane kept, every deeper cut moved by  */
                              /* +1, -1, +2, -2 planes; an energy goes to the next tree while   */
                              /* still above the threshold) and keeps, per energy, the result   */
                              /* with the smallest residual; 0 = off. HSC_FP64 solves          */
                              /* only (a mixed-precision residual reflects its FP32 rounding).  */
                              /* Each alternate tree is analysed on first need and works in the */
                              /* handle's own workspace after the first pass.                   */
                              /* hsc_solve_batch does not re-solve.                             */
  HSC_OPT_TREE_VARIANT = 8,   /* 1..4: the next hsc_analyze builds that alternate separator     */
                              /* tree itself (0, default: the plain tree)                       */
  HSC_OPT_ORDERING = 9,       /* tree of the next hsc_analyze when grid_dims were given:        */
                              /* 0 (default): geometric dissection; when every contact site    */
                              /* lies on the end planes x = 0 and x = Nx-1 (both used), in its  */
                              /* contact-connected form: x is cut once, at the root, and every  */
                              /* deeper cut is a y or z plane (leaves: leaf_max x leaf_max      */
                              /* cross-sections spanning half the device), so every cluster     */
                              /* below the root keeps a share of a contact face. Clusters far   */
                              /* from both contacts carry only eta in their blocks, and at small*/
                              /* eta one with a level within delta of E costs the downward pass */
                              /* ~1/delta^2 in rounding (on the 32^3 cube at eta = 1e-6 the    */
                              /* plain tree loses 2 to 17 digits, this one 0 to 2; it costs     */
                              /* 855 instead of 369 model GFLOP per energy with leaf_max 8).    */
                              /* 1: breadth-first level-set bisection of the site graph (level  */
                              /* sets from a corner are diagonal planes: 260 GFLOP on 32^3; they*/
                              /* lose more digits at small eta than axis planes)                */
                              /* 2: plain geometric dissection (the longest extent is cut at    */
                              /* every level: 8^3 leaves and 369 GFLOP on 32^3 with leaf_max 8) */
  HSC_OPT_MAX_CLUSTER = 10,   /* > 0: the next hsc_analyze splits every cluster of more sites   */
                              /* into a chain of pieces of at most that many sites, each the    */
                              /* parent of the previous (Section 3.4's degenerate sub-trees for */
                              /* dense molecular blocks); dense contacts stay whole; 0 = off    */
  HSC_OPT_GJ_WIDE = 12,       /* nested blocking of the Gauss-Jordan inversion: the panels of    */
                              /* HSC_OPT_GJ_PANEL width are reduced inside a wide panel of this  */
                              /* width (rounded down to a multiple of the panel width), whose    */
                              /* columns alone their products update; one trailing product with */
                              /* K = this width then updates the rest of the block (default 128; */
                              /* 0 or <= the panel width: every panel updates the whole block)   */
  HSC_OPT_LEAF_BAND = 13,     /* 1 (default): the downward products of a leaf cluster (no       */
                              /* children) form G_ii and G^<_ii only on the column band of each */
                              /* block of <= 128 rows that spans the entries read afterwards:   */
                              /* the diagonal, the H neighbours the residual check reads (G^r), */
                              /* requested pairs inside the block, and (lesser leaves) every    */
                              /* column of G_ii's contact rows; other entries of those blocks   */
                              /* are left undefined. A solve whose requested pairs fall in a    */
                              /* leaf block outside the current bands rebuilds the schedule     */
                              /* first. 0: the whole blocks (identical computed entries)        */
  HSC_OPT_LEAF_SPARSE = 14,   /* 1 (default): a leaf cluster's front holds no children's Schur   */
                              /* complements, so its coupling block A_iU is the H entries alone:*/
                              /* X = D^{-1} A_iU and the Schur update A_iU^T X are formed as     */
                              /* gathers over that pattern in FP64 (the dense products' other   */
                              /* terms are exact zeros); and its diagonal block is banded in the */
                              /* local order (bandwidth b, no DENSE contact block on it), so the */
                              /* nested Gauss-Jordan steps skip the rows at positions >= k + b   */
                              /* (untouched until pivot k) and the columns beyond the pivot     */
                              /* rows' reach k + 2b. 0: dense block products and inversion      */
  HSC_OPT_TREE_FORM = 11      /* read only: the tree of the last hsc_analyze: 0 plain geometric,*/
                              /* 1 contact-connected geometric, 2 graph bisection (-1 before    */
                              /* any analysis). With HSC_OPT_ORDERING = 0 the contact-connected */
                              /* form is taken only while its model cost stays within 3x the    */
                              /* plain geometric tree's or below 1 GFLOP per energy (an         */
                              /* elongated device, e.g. a 64 x 12 x 12 wire, keeps the plain    */
                              /* form)                                                          */
} hsc_option;

int hsc_set_option(hsc_t h, int32_t option, int32_t value);
int hsc_get_option(hsc_t h, int32_t option, int32_t* value);

/* One device of a batched solve (hsc_solve_batch). E, sigma_r, sigma_less and all outputs are device
 * memory laid out as in hsc_solve; req_pairs is host memory. */
typedef struct {
  hsc_t h;
  int64_t n_E;
  const double* E;
  const hsc_c128* sigma_r;
  const hsc_c128* sigma_less;   /* may be NULL (no G^<)                                          */
  int32_t n_req;
  const int32_t* req_pairs;
  hsc_c128* diag_gr;
  hsc_c128* diag_gl;
  hsc_c128* req_gr;
  hsc_c128* req_gl;
} hsc_batch_item;

/* hsc_solve_batch -- solve several devices (handles, e.g. cuboids with uneven separators) and their
 *   energies in one CUDA-graph launch. Each item's level schedule is captured on its own stream,
 *   forked from and joined back into cuda_stream, so the items' kernels run concurrently and the
 *   GPU balances the uneven trees (the capture runs on an internal stream; the graph is launched
 *   into cuda_stream, which may be the legacy default stream). The instantiated graph is cached
 *   and replayed while the items
 *   (handles, pointers, sizes), eta and precision are unchanged. use_graph = 0 enqueues the same
 *   work directly on the item streams (no graph). Workspaces are sized so that all items fit the
 *   device budget together (energies of an item run in several waves if needed). The call
 *   synchronises cuda_stream and checks every item's device error flags.
 *   Errors: as hsc_solve; on error the item index is named in hsc_last_error(NULL). */
int hsc_solve_batch(int32_t n_items, const hsc_batch_item* items, double eta, int32_t precision,
                    void* cuda_stream, int32_t use_graph);

/* Result of hsc_tune. */
typedef struct {
  int32_t leaf_max;        /* chosen nested-dissection leaf size                          */
  int32_t gj_panel;        /* chosen Gauss-Jordan panel width                             */
  double ms_per_energy;    /* measured time of the chosen configuration                   */
  int32_t from_cache;      /* 1 if read from the cache file, 0 if measured now             */
  int32_t n_tried;         /* configurations timed                                        */
} hsc_tune_result;

/* hsc_tune -- autotune a handle for its geometry on this GPU: for each candidate leaf_max (4, 6, 8,
 *   when smaller than the grid) and Gauss-Jordan panel width (16, 32, 64) re-analyse, solve the given
 *   probe energies twice (host buffers, as hsc_solve, residual re-solve included) and time the
 *   second solve with CUDA events (give it probes spread over the energy window: whether a probe
 *   needs a re-solve on a given tree weighs in its time). A candidate whose worst probe residual
 *   (HSC_FP64) exceeds the handle's re-solve threshold 10^-d is not admissible (a smaller leaf
 *   loses digits at small eta); keep the fastest admissible candidate (if none is, the one with the
 *   smallest worst residual), leave the handle analysed with it, and append one JSON line (GPU name, grid,
 *   orbitals, precision, choice, time) to cache_path (may be NULL: no cache). A matching cache line
 *   is applied without timing. Errors: as hsc_analyze / hsc_solve. */
int hsc_tune(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
             const hsc_c128* sigma_less, int32_t precision, const char* cache_path,
             hsc_tune_result* out);

/* Kernel-class statistics of the launches hsc_solve made since the last hsc_profile call.
 *   launches  kernel launches of the class (counted whether or not timing is enabled)
 *   timed     launches bracketed by CUDA events (only while timing is enabled)
 *   ms        sum of the event-measured device durations of those launches (milliseconds)
 *   flops     algorithmic real flops of those launches (complex multiply-add = 8)
 *   bytes     algorithmic bytes moved by those launches (memory-bound classes only) */
typedef struct {
  char name[24];
  int64_t launches;
  int64_t timed;
  double ms;
  double flops;
  double bytes;
} hsc_kernel_stat;

/* hsc_residual -- a-posteriori check of the last solve on this handle: out[k] = max over unknowns u
 *   of |Re r_u| + |Im r_u|, r_u = (A G^r - I)_uu at energy k, evaluated from the computed blocks
 *   (every non-zero A_uv joins unknowns whose G^r entry is stored, G^r = (G^r)^T). A relative error
 *   x in the diagonal and pattern entries of G^r shows up as about |A| |G| x. Host array of
 *   n_E <= the last solve's n_E; synchronises the device. Errors: HSC_ERR_ARG, HSC_ERR_STATE,
 *   HSC_ERR_CUDA. */
int hsc_residual(hsc_t h, int64_t n_E, double* out);

/* hsc_growth -- element growth of the last solve on this handle: out[k] = max over the cluster
 *   blocks of Algorithm 1 of the largest |Re| + |Im| entry of D_i^{-1} at energy k (in 1/eV). The
 *   elimination order is fixed by the separator tree and pivots only inside a cluster block, so a
 *   cluster whose isolated levels lie within ~eta of E makes this large, and the downward pass
 *   (Eq. 4) then subtracts terms of that size from each other: the results lose digits in
 *   proportion. out: host array of n_E <= the last solve's n_E. Synchronises the device.
 *   Errors: HSC_ERR_ARG, HSC_ERR_STATE (no such solve), HSC_ERR_CUDA. */
int hsc_growth(hsc_t h, int64_t n_E, double* out);

/* hsc_cluster_growth -- per-cluster conditioning record of the last solve on this handle:
 *   out[k][c] = ||D_c^{-1}||_F (Frobenius norm, 1/eV) of cluster c's block of Algorithm 1 (Eq. 3) at
 *   energy k, for the clusters of this handle's own tree (postorder ids as hsc_cluster; 0 for a
 *   cluster with no own unknowns). It lies between 1/sigma_min(D_c) and sqrt(n_c)/sigma_min(D_c),
 *   so a level of the block within delta of E reads as ~1/delta. At small eta an interior block with
 *   such a level makes the downward step G_cc = D_c^{-1} + X_c G_UU X_c^T cancel terms of size
 *   ~1/delta^2, amplifying the rounding error its ancestors' blocks carry by about that factor.
 *   Energies that a re-solve moved to another tree keep the record of this tree.
 *   out: host array of n_E x n_clusters doubles, n_E <= the last solve's n_E. Synchronises the
 *   device. Errors: HSC_ERR_ARG, HSC_ERR_STATE (no such solve), HSC_ERR_CUDA. */
int hsc_cluster_growth(hsc_t h, int64_t n_E, double* out);

/* hsc_profile -- reset the kernel statistics; enable = 1 additionally brackets every kernel launch
 *   of subsequent hsc_solve calls with CUDA events on the solve's stream (device-side timing;
 *   a small host overhead per launch), enable = 0 stops the timing. No GPU work. */
int hsc_profile(hsc_t h, int32_t enable);

/* hsc_profile_read -- per-class statistics (host array of cap >= *n_out entries; call with
 *   out = NULL to query *n_out). Waits for the recorded events. Errors: HSC_ERR_ARG, HSC_ERR_CUDA. */
int hsc_profile_read(hsc_t h, hsc_kernel_stat* out, int32_t cap, int32_t* n_out);

/* hsc_observables -- per-energy observables from hsc_solve outputs (Section 1: the quantities the
 *   Green's functions are evaluated for), all arrays on the device:
 *   out[n_E][3] = { DOS(E) = -(1/pi) sum_u Im G^r_uu,
 *                   T(E) = sum over the slots of `contact` of Gamma_slot Im G^<_uu with
 *                          Gamma_slot = -2 Im Sigma^r_slot (the transmission into that contact when
 *                          only the other contact is filled, f = 1),
 *                   sum_u Im G^<_uu (2 pi times the electron count per unit energy) }.
 *   diag_gl and sigma_r may be NULL (then the last two entries are 0). Asynchronous on cuda_stream.
 *   Errors: HSC_ERR_ARG, HSC_ERR_STATE, HSC_ERR_CUDA. */
int hsc_observables(hsc_t h, int64_t n_E, const hsc_c128* diag_gr, const hsc_c128* diag_gl,
                    const hsc_c128* sigma_r, int32_t contact, double* out, void* cuda_stream);

/* hsc_scba -- self-consistent loop with the solve as its inner kernel: local elastic dephasing as
 *   the scattering part of Sigma^r (Section 1 splits Sigma^r of Eq. 1 into a contact part and a
 *   scattering part; the paper fixes no scattering model, this is the local one of the
 *   self-consistent Born approximation with a delta-correlated potential of strength d0, eV^2):
 *     Sigma^r_scatt,uu = d0 G^r_uu,  Sigma^<_scatt,uu = d0 G^<_uu = i d0 Im G^<_uu  on every
 *   unknown u (G^< is anti-Hermitian, so the real part of its diagonal is rounding error and is
 *   not fed back: see the Sigma^< convention of hsc_solve).
 *   Iteration, all energies together: S_0 = 0; hsc_solve with Sigma_contact + S_k gives G_k;
 *   F_k = (d0 diag G^r_k, i d0 Im diag G^<_k); delta_k = max|F_k - S_k| / max|F_k| over energies,
 *   unknowns, retarded and lesser (0 when F_k = 0); stop when delta_k <= tol or after max_iter
 *   solves; else S_{k+1} = S_k + mix (F_k - S_k). The mixing and both maxima run in one kernel; the
 *   host reads two doubles per iteration.
 *   The handle's contacts must cover every site: declare the scattering region (for instance every
 *   site outside the leads) as one more contact whose contact self-energy is zero.
 *   E, sigma_r, sigma_less, precision, cuda_stream, io_on_device: as hsc_solve; sigma_r and
 *     sigma_less[n_E][n_cs] are the contact parts (sigma_less is required)
 *   d0 >= 0, 0 < mix <= 1, tol >= 0, max_iter >= 1
 *   diag_gr, diag_gl[n_E][n]  out: the diagonals of the last solve (the one delta_k was measured on)
 *   iters, delta  out (host): solves made and the last delta_k. Reaching max_iter is not an error:
 *     compare *delta with tol.
 *   Device work memory for the self-energies (4 n_E n_cs complex) is allocated per call.
 *   Errors: as hsc_solve; HSC_ERR_ARG also when the contacts leave a site out. */
int hsc_scba(hsc_t h, int64_t n_E, const double* E, double eta, const hsc_c128* sigma_r,
             const hsc_c128* sigma_less, double d0, double mix, double tol, int32_t max_iter,
             int32_t precision, hsc_c128* diag_gr, hsc_c128* diag_gl, int32_t* iters, double* delta,
             void* cuda_stream, int32_t io_on_device);

/* hsc_device_fp64_peaks -- measure, on the current device, the throughput of the FP64 tensor pipe
 *   (mma.sync m8n8k4 f64, which the complex128 GEMMs use) and of scalar FP64 FMA, in GFLOP/s
 *   (best of three ~10 ms launches). These are the roofline denominators of the complex128 path.
 *   Errors: HSC_ERR_ARG, HSC_ERR_CUDA, HSC_ERR_OOM. */
int hsc_device_fp64_peaks(double* dmma_gflops, double* dfma_gflops);

/* hsc_block_inverse_noalloc -- invert `batch` dense n x n complex128 blocks without allocating.
 *   The paper has no counterpart: this is a deployment variant of the Gauss-Jordan block inversion
 *   (partial pivoting inside each block) that hsc_solve uses for the cluster blocks, for callers
 *   that cannot allocate device memory while they run (their memory pool already holds the free
 *   device memory, or cudaMalloc/cudaFree's implicit synchronisation is not acceptable).
 *   A     device, batch blocks of n x n, row-major, contiguous (read only unless A == Ainv)
 *   Ainv  device, same layout, receives the inverses (may equal A: in place)
 *   cuda_stream  stream to run on (NULL: legacy default stream); the call synchronises it.
 *   Limits: n <= 1024, batch <= 256, n * batch <= 8192. Scratch lives in one fixed 4.3 MiB device
 *   array per device (held until process exit); no cudaMalloc/cudaFree is called. The array exists
 *   on a device from the first call there (the library's CUDA modules load lazily): that call loads
 *   the module and looks up the array's address (cudaGetSymbolAddress). A call with batch = 0 (A and
 *   Ainv may be NULL) does only this set-up; make it on each device before the memory pool reserves
 *   the free device memory and before any stream capture. The cached address does not survive
 *   cudaDeviceReset. Calls whose work overlaps on the GPU race on the shared array: serialise them.
 *   Errors: HSC_ERR_ARG (sizes beyond the limits, NULL pointers), HSC_ERR_SINGULAR (zero pivot;
 *   the outputs are then undefined), HSC_ERR_CUDA. */
int hsc_block_inverse_noalloc(int32_t n, int32_t batch, const hsc_c128* A, hsc_c128* Ainv,
                              void* cuda_stream);

/* hsc_last_error -- text of the last failure on this handle ("" if none); valid until the next
 * call on the handle. Accepts NULL (returns the last global error, e.g. from hsc_create). */
const char* hsc_last_error(hsc_t h);

/* hsc_destroy -- free the handle and its device workspace. NULL is accepted. */
int hsc_destroy(hsc_t h);

#ifdef __cplusplus
}
#endif
#endif /* HSC_H */
