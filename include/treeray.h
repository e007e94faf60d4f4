/* treeray.h - C ABI of the GB300 (sm_103a) TreeRay/OnTheSpot hot path.
 *
 * The method is TreeRay/OnTheSpot (Wuensch et al., arXiv 2105.09644):
 * for every target cell the octree is walked with the opening criteria of
 * Sec. 2.4, accepted nodes are mapped onto N_PIX HEALPix rays x N_R radial
 * evaluation points (Sec. 2.2-2.3, App. A), each ray is swept from far to
 * near with the On-the-Spot recombination loss (Sec. 2.5, Eq. 12-17) and the
 * rays are summed into the cell's EUV photon flux and energy density
 * (Eq. 18).  Sec. 2.6 (Eq. 19-21) iterates this until the energy density
 * converges.
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers on the current CUDA device,
 *    owned by the caller, unless a comment says otherwise.  Cell arrays hold
 *    N^3 values of a uniform cubic grid in C order [iz][iy][ix] (x fastest).
 *  - Units are CGS: cm, cm^-3, photons s^-1, erg.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default).
 *    Calls that report device-side status synchronise that stream before
 *    returning, as noted.
 *  - No call aborts or throws.  A call returns TR_OK or an error code and
 *    leaves a thread-local message for tr_last_error().
 *  - Opaque handles (tr_tree, tr_rays) are owned by the library and released
 *    with their *_free function.
 */
#ifndef TREERAY_H
#define TREERAY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tr_stream;   /* same type as cudaStream_t */

typedef enum {
    TR_OK = 0,
    TR_EINVAL = 1,          /* bad argument (null pointer, size, parameter range) */
    TR_ENOMEM = 2,          /* device allocation failed */
    TR_ECUDA = 3,           /* a CUDA call failed (message has the CUDA error) */
    TR_ETIMEOUT = 4,        /* a bounded device-side wait ran out */
    TR_EUNSUPPORTED = 5,    /* valid request outside what this build implements */
    TR_EOVERFLOW = 6        /* a per-target walk stack overflowed; raise theta or report */
} tr_status;

/* Arithmetic of the three forms.  In both FP32 forms the node moments are
 * FP32 with compensated (Kahan-Neumaier) sums over the children, the centre
 * of mass stored as its offset from the node's geometric centre; the ray
 * deposits are FP32 addends summed exactly in 64-bit fixed point (order
 * independent, so the FP32 forms are bit-reproducible); and every opening
 * decision (Sec. 2.4) and every discontinuous choice of the radial
 * spreading that FP32 cannot settle within its certified error bound is
 * re-taken in FP64 against an FP64 copy of the tree, so that the accepted
 * node lists are those of the FP64 form, bit for bit.  The two FP32 forms
 * differ only in the far-to-near sweep (Sec. 2.5, Eq. 12-17):
 *  TR_FP32_SWEEP64: every segment's loss R_ij, the photon rates Phi_j and
 *    their clipping at zero in FP64 (the FP32 coefficients widened), as in
 *    the FP64 form;
 *  TR_FP32_SWEEPDF: R_ij formed in FP32 and the budgets Phi_j carried as
 *    unevaluated sums of two FP32 numbers (about 48 bits), with the final
 *    Phi_j, the flux and the classification in FP64. */
typedef enum {
    TR_FP64 = 0,            /* node moments, deposits and sweep all in FP64 */
    TR_FP32_SWEEP64 = 1,    /* FP32 moments and deposits, FP64 sweep */
    TR_FP32_SWEEPDF = 2     /* FP32 moments and deposits, double-FP32 sweep */
} tr_precision;

/* Radial kernels (App. A) that spread a node along a ray.  alpha and e use
 * W_p (default) or the truncated Gaussian W_g, normalised over the
 * evaluation points.  eps uses one of the flux-conserving kernels (W_f,3 by
 * default, two points with the sum and the flux at the target exact; W_f,1
 * and W_f,2 with the paper's other second conditions; the generalised
 * W_f,3 over every point in the node's support, Eq. A8-A10) or, for
 * comparison, W_p or W_g.  Where a flux kernel's prescription does not
 * apply (W_f,2 next to the target, a generalised W_f,3 with fewer than three
 * points or a negative weight) the two-point W_f,3 is used. */
typedef enum { TR_KERNEL_WP = 0, TR_KERNEL_WG = 1 } tr_kernel;
typedef enum {
    TR_EPS_WF3 = 0, TR_EPS_WF1 = 1, TR_EPS_WF2 = 2, TR_EPS_WF3N = 3, TR_EPS_WP = 4, TR_EPS_WG = 5
} tr_eps_kernel;

/* Boundary conditions of the walk (Sec. 2.8).  Isolated: nothing outside
 * the box.  Periodic: every node that does not contain the target is taken
 * at its copy nearest to the target (geometric centres, per axis).  Corner
 * of symmetry: the grid is one octant of a problem symmetric about its low
 * corner; the walk maps the grid and its 7 mirror images through that
 * corner onto the rays, and L_ray defaults to the diagonal of the mirrored
 * domain (2 N sqrt3 cells). */
typedef enum { TR_BC_ISOLATED = 0, TR_BC_PERIODIC = 1, TR_BC_CORNER = 2 } tr_bc;

/* Solver parameters (Sec. 2.2-2.6).  tr_params_default() fills the paper's
 * defaults: theta_lim 0.5, theta_if = theta_src = INFINITY, N_side 2,
 * eta_R 2, L_ray = domain diagonal, alpha_B 2.7e-13, h nu = 13.6 eV,
 * eps_lim 1e-2, delta per cell, one pass, FP64, zeta_g on, W_p for alpha
 * and e, W_f,3 for eps, isolated boundaries. */
typedef struct {
    double theta_lim;       /* BH opening angle: accept when h/d < theta_lim (Sec. 2.4) */
    double theta_if;        /* IF MAC angle, INFINITY disables (Sec. 2.4) */
    double theta_src;       /* Src MAC angle, INFINITY disables (Sec. 2.4) */
    int32_t nside;          /* HEALPix N_side in {1, 2, 4, 8}; N_PIX = 12 N_side^2 (Sec. 2.2) */
    int32_t eta_r;          /* radial resolution eta_R in {1, 2, 4, 8} (Eq. 4) */
    double L_ray_cm;        /* maximum ray length; <= 0 selects the domain diagonal (Eq. 5) */
    double alpha_B;         /* case-B recombination coefficient, cm^3 s^-1 */
    double hnu;             /* mean EUV photon energy, erg */
    double eps_lim;         /* iteration stops when delta < eps_lim (Sec. 2.6) */
    int32_t delta_mode;     /* 0: delta_cell (Eq. 21), 1: delta_tot (Eq. 20) */
    int32_t max_iter;       /* >= 1 passes of build + walk + sweep */
    int32_t precision;      /* tr_precision */
    int32_t zeta_g;         /* 1: apply the geometric factor zeta_g (Eq. 16) */
    int32_t kernel_alpha;   /* tr_kernel for alpha and e */
    int32_t kernel_eps;     /* tr_eps_kernel for eps */
    int32_t bc;             /* tr_bc: boundary condition of the walk */
} tr_params;

/* Uniform cubic grid.  N is a power of two with 8 <= N <= 512.
 * n_H: hydrogen number density (cm^-3), required, finite and >= 0.
 * ndot: extra per-cell EUV emission (photons s^-1), may be NULL.
 * e_prev: per-cell EUV energy density (erg cm^-3) from a previous pass, may
 *         be NULL; it enters the IF MAC (ionised mass, Sec. 2.4) and zeta_d
 *         (Eq. 17), and seeds the iteration of tr_solve (Sec. 2.6). */
typedef struct {
    int32_t N;
    double box_lo[3];       /* low corner of the box, cm */
    double dx;              /* cell edge, cm */
    const double* n_H;
    const double* ndot;
    const double* e_prev;
} tr_grid;

/* Point sources (Sec. 2.7), mapped to the cell containing them. */
typedef struct {
    int32_t n;              /* number of sources, >= 0 */
    const double* xyz;      /* device, n x 3 positions, cm */
    const double* Q;        /* device, n EUV photon rates, s^-1 */
} tr_sources;

/* AMR grid of blocks of 8^3 cells (Sec. 2.1: every block is a subtree of
 * the octree whose leaves are the cells).  Block b has refinement level
 * blk_level[b] in [0, max_level] (its cells have edge
 * 2^(max_level - blk_level[b]) finest cells) and corner
 * (blk_pos[3b], blk_pos[3b+1], blk_pos[3b+2]) = (x, y, z) in units of its
 * own edge (8 of its cells).  The blocks must tile the box exactly once.
 * N_base (base-level cells per axis) is a power of two >= 8 and
 * N_base << max_level <= 512.  blk_level and blk_pos are HOST arrays (the
 * library copies them); cell arrays are DEVICE arrays of n_blocks x 512
 * values, [b][iz][iy][ix] within each block, and a cell's index (target,
 * output position) is b * 512 + (iz * 8 + iy) * 8 + ix.  n_H, ndot and
 * e_prev mean what they mean in tr_grid. */
typedef struct {
    int32_t N_base;
    int32_t max_level;
    int32_t n_blocks;
    const int32_t* blk_level;   /* host, n_blocks */
    const int32_t* blk_pos;     /* host, 3 x n_blocks */
    double box_lo[3];           /* low corner of the box, cm */
    double dx_fine;             /* edge of a cell of level max_level, cm */
    const double* n_H;
    const double* ndot;
    const double* e_prev;
} tr_amr_grid;

typedef struct tr_tree tr_tree;
typedef struct tr_rays tr_rays;

/* Fill *p with the defaults listed above. */
void tr_params_default(tr_params* p);

/* Build the octree (Sec. 2.1, Eq. 1-3): sources are mapped to cells
 * (Sec. 2.7), emission and recombination are netted per cell, and node
 * moments (mass, centre of mass, alpha_n, eps_n, e_n, ionised mass) are
 * reduced bottom-up in Morton order.  *out may hold a tree from an earlier
 * call: it is rebuilt in place when its grid size and precision match,
 * otherwise it is freed and replaced.  The node->ray table for N_side is
 * built on the device on first use and cached for the process.
 * Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_EUNSUPPORTED.  Asynchronous. */
tr_status tr_build_tree(const tr_grid* g, const tr_sources* s, const tr_params* p,
                        tr_tree** out, tr_stream stream);

/* Build the octree of an AMR grid (Sec. 2.1, Eq. 1-3).  The tree spans the
 * finest lattice (N_base << max_level cells per axis) in the same
 * level-order Morton numbering as a uniform tree; a node is a cell (leaf,
 * never opened), a parent of eight existing nodes, or absent (inside a
 * cell).  Lengths inside are in finest cells: a cell of edge s has volume
 * s^3, mass n_H s^3, and its own emission reaches it through a sphere of
 * radius s/2 (Sec. 2.5).  Point sources go to the cell that contains them.
 * The walk calls (tr_walk_map, tr_walk_sweep, tr_walk_sweep_batch) then
 * take cell indices b * 512 + c as targets and write outputs indexed the
 * same way; targets of tr_walk_sweep_batch ranges are in walk order
 * (blocks sorted along the Morton curve of the finest lattice, cells in
 * Morton order inside a block).  *out may hold an earlier tree: it is
 * freed and replaced.  The block layout is checked on the host: levels and
 * positions in range, no block inside another, total volume = box.
 * Synchronises `stream` (the block tables are copied from the host).
 * Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_EUNSUPPORTED. */
tr_status tr_build_tree_amr(const tr_amr_grid* g, const tr_sources* s, const tr_params* p,
                            tr_tree** out, tr_stream stream);

/* Walk the tree for n_targets target cells (C-order cell indices, or
 * b * 512 + c on an AMR tree; device int64 array; NULL with n_targets = the
 * number of cells means every cell) and map the
 * accepted nodes onto each target's rays (Sec. 2.3-2.4).  The result keeps,
 * per target, the ray bins alpha/eps/e ([N_PIX][N_R] each) and the list of
 * accepted node ids (level-order Morton numbering: (8^l - 1)/7 + Morton
 * index within level l).  Meant for parity checks and the unfused path;
 * device memory grows with n_targets x N_PIX x N_R.  Synchronises `stream`.
 * Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_EOVERFLOW. */
tr_status tr_walk_map(const tr_tree* t, const int64_t* targets, int64_t n_targets,
                      tr_rays** out, tr_stream stream);

/* Sweep every ray of a tr_rays far to near (Sec. 2.5, Eq. 12-17) in FP64 and
 * sum the directions (Eq. 18).  Outputs (device, n_targets each, may be NULL):
 * F_out photon flux (photons s^-1 cm^-2), e_out energy density (erg cm^-3),
 * ion_out 1 where F > 0.  Asynchronous. */
tr_status tr_ray_sweep(const tr_rays* r, double* F_out, double* e_out, uint8_t* ion_out,
                       tr_stream stream);

/* Walk + map + sweep for every cell of a built tree in one fused kernel
 * (Sec. 2.3-2.5, Eq. 18): the ray bins of each target stay in shared memory.
 * Outputs as in tr_ray_sweep, one value per cell (N^3 in C order, or
 * n_blocks x 512 on an AMR tree; NULL allowed).  Synchronises `stream`.
 * Errors: TR_EINVAL, TR_ECUDA, TR_EOVERFLOW, TR_EUNSUPPORTED (ray bins
 * larger than a CTA's shared memory). */
tr_status tr_walk_sweep(const tr_tree* t, double* F_out, double* e_out, uint8_t* ion_out,
                        tr_stream stream);

/* Continuous batching of independent problems: ONE persistent launch walks,
 * maps and sweeps the targets of several built trees (different grid sizes,
 * sources and N_PIX allowed; one precision per batch).  For tree i it does
 * the cells whose Morton index (x bit 0, y bit 1, z bit 2 of each triple)
 * lies in [first[i], first[i] + count[i]), writing F_out[i], e_out[i] and
 * ion_out[i] at the cells' C-order indices (device arrays of that tree's
 * N^3; the pointer arrays themselves are HOST arrays and may be NULL); on
 * an AMR tree the range is in its walk order and outputs are indexed
 * b * 512 + c (see tr_build_tree_amr).  A
 * serving loop admits requests between launches and splits large ones into
 * Morton ranges, so that small requests are not held up by large ones.
 * trees, first, count: HOST arrays of n >= 1 entries.  Synchronises
 * `stream`.  Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_EOVERFLOW. */
tr_status tr_walk_sweep_batch(const tr_tree* const* trees, const int64_t* first, const int64_t* count,
                              int32_t n, double* const* F_out, double* const* e_out,
                              uint8_t* const* ion_out, tr_stream stream);

/* The fused fast path: build + walk + map + sweep for every cell, repeated
 * (Sec. 2.6) until delta < eps_lim or max_iter passes.  Outputs are N^3
 * device arrays (NULL allowed): F_out, e_out, ion_out as in tr_ray_sweep.
 * iters_out and delta_out are HOST pointers (may be NULL).  Device memory
 * is cached per device between calls and grows on demand.  Synchronises
 * `stream`.  Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_EOVERFLOW. */
tr_status tr_solve(const tr_grid* g, const tr_sources* s, const tr_params* p,
                   double* F_out, double* e_out, uint8_t* ion_out,
                   int32_t* iters_out, double* delta_out, tr_stream stream);

/* Fractional change of the energy density between two passes (Sec. 2.6):
 * delta_mode 0: delta_cell = max_c |e_new - e_old| / max(e_old, e_med)
 * (Eq. 21, e_med the lower median of e_old, absolute difference); 1:
 * delta_tot = 2 |sum e_new - sum e_old| / (sum e_new + sum e_old) (Eq. 20).
 * e_new, e_old: device arrays of n >= 1 values (erg cm^-3, >= 0).
 * *delta_out (HOST) receives delta; a zero norm with a change gives
 * INFINITY.  Synchronises `stream`.  Errors: TR_EINVAL, TR_ENOMEM, TR_ECUDA. */
tr_status tr_delta(const double* e_new, const double* e_old, int64_t n, int32_t delta_mode,
                   double* delta_out, tr_stream stream);

/* One pass of tr_solve (build + walk + map + sweep, max_iter = 1) that
 * allocates no device memory.  The paper has no counterpart: this is a
 * service to callers that cannot call cudaMalloc, such as applications whose
 * device memory is owned by a pool or arena that forbids allocations from
 * outside it, and real-time or embedded hosts that must not allocate once
 * running (cudaMalloc may block and synchronise the device).  The caller
 * still supplies inputs and outputs (as for tr_solve: N^3 device arrays,
 * NULL allowed) and gets the same results as tr_solve with the same
 * parameters.  Working memory is one fixed device array (about 18 MB)
 * inside the library, held by every GPU that loads it until the process
 * exits.  Limits: N <= 32, N_side 1 or 2, N_R <= 128, max_iter = 1; larger
 * requests return TR_EUNSUPPORTED with a message and touch nothing; other
 * arguments are checked as tr_solve checks them.
 * The first call on a device looks up that array's device address (with
 * that device current) and builds the node->ray table into it; a call with
 * a new N_side rebuilds the table.  Make the first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents;
 * every value a pass needs is rewritten or cleared by that pass.  Calls
 * whose GPU work overlaps (e.g. two streams driven from two host threads
 * that bypass its host lock) race on the array.  Every call synchronises
 * `stream` before it returns.  Errors: TR_EINVAL, TR_EUNSUPPORTED, TR_ECUDA,
 * TR_EOVERFLOW. */
tr_status tr_solve_noalloc(const tr_grid* g, const tr_sources* s, const tr_params* p,
                           double* F_out, double* e_out, uint8_t* ion_out, tr_stream stream);

/* Column-density maps (cdMaps, the TreeRay/OpticalDepth quantity that the
 * paper's ray-arrays include, Sec. 2.2): the same walk and MACs as
 * tr_walk_sweep over a built tree, but each accepted node adds to direction
 * k of the target its mass times its volume fraction in ray k over the
 * ray's cross-section at the node, w_k m / (Omega d^2), Omega = 4 pi /
 * N_PIX; no radial points, no sweep, no maximum ray length, and the target
 * cell itself left out.  out: device [n_targets][N_PIX] hydrogen column
 * densities, cm^-2 (targets as for tr_walk_map; NULL with n_targets = the
 * cell count gives row c for cell c).  Synchronises `stream`.
 * Errors: TR_EINVAL, TR_ECUDA, TR_EOVERFLOW. */
tr_status tr_column_density(const tr_tree* t, const int64_t* targets, int64_t n_targets, double* out,
                            tr_stream stream);

/* ---- inspection (parity tests) -------------------------------------- */

/* Sizes of a tree: node count, levels (log2 N + 1), N_R, N_PIX. Host outputs. */
tr_status tr_tree_info(const tr_tree* t, int64_t* n_nodes, int32_t* levels,
                       int32_t* nr, int32_t* npix);

/* Number of cells (targets) of a tree: N^3, or n_blocks x 512 for an AMR
 * tree.  Host output. */
tr_status tr_tree_cells(const tr_tree* t, int64_t* n_cells);

/* Topology of a tree, one byte per node in level-order Morton numbering
 * (device array of n_nodes): 0 absent, 1 leaf (a cell), 2 parent. */
tr_status tr_tree_flags(const tr_tree* t, uint8_t* out, tr_stream stream);

/* Counters of the last walk over this tree (host output, 6 values):
 * nodes visited, nodes accepted, table entries read, deepest stack, and,
 * in the FP32 forms, the opening decisions and the radial set-ups that were
 * re-taken in FP64 because FP32 could not settle them (0 in the FP64 form). */
tr_status tr_tree_stats(const tr_tree* t, int64_t* out6);

/* Node records as FP64 in level-order Morton numbering, 8 values per node:
 * {m, cm_x, cm_y, cm_z, alpha_n, eps_n, e_n, m_ion}; m in n_H x cells,
 * positions in cells from the box corner, alpha/eps in photons s^-1,
 * e_n in erg cm^-3 x cells.  out8 is a device array of n_nodes x 8. */
tr_status tr_tree_nodes(const tr_tree* t, double* out8, tr_stream stream);

/* Sizes of a tr_rays: targets, N_PIX, N_R, accepted-id capacity per target. */
tr_status tr_rays_info(const tr_rays* r, int64_t* n_targets, int32_t* npix, int32_t* nr,
                       int32_t* acc_cap);

/* Ray bins as FP64 [n_targets][N_PIX][N_R] (device; NULL skips): alpha and
 * eps in photons s^-1, e in erg cm^-3 x cells.  ids: [n_targets][acc_cap]
 * accepted node ids (int64, unordered), counts: [n_targets] (int32). */
tr_status tr_rays_export(const tr_rays* r, double* alpha, double* eps, double* e,
                         int64_t* ids, int32_t* counts, tr_stream stream);

/* Node->ray table for N_side (Sec. 2.3, built on the device): key count and
 * total entries (host outputs).  tr_table_export writes offsets (nkeys+1,
 * int32) and entries (pixel, count) as two int32 arrays (device). */
tr_status tr_table_info(int32_t nside, int32_t* nkeys, int32_t* n_entries);
tr_status tr_table_export(int32_t nside, int32_t* offsets, int32_t* pix, int32_t* cnt,
                          tr_stream stream);

void tr_tree_free(tr_tree* t);
void tr_rays_free(tr_rays* r);

/* Message of the last failed call on this host thread ("" if none). */
const char* tr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TREERAY_H */
