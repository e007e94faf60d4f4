/* Plain FP64 CPU oracle for the TreeRay/OnTheSpot hot path.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * Units: lengths in cells of the (uniform) grid, photon rates in s^-1,
 * energies in erg.  Positions run from 0 to N along each axis; cell (ix,iy,iz)
 * has its centre at (ix+0.5, iy+0.5, iz+0.5).  Cell arrays are N^3 float64 in
 * C order [iz][iy][ix] (x fastest).
 */
#ifndef TREERAY_ORACLE_H
#define TREERAY_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Node->ray table resolution (the paper's table is defined in Paper I, not
 * reproduced; this oracle samples each node cube with ORC_TM^3 points).
 * Keys: a face key when one axis dominates the node offset, an edge key
 * when two axes tie for the largest |offset|, a corner key when all three
 * do; an edge or corner key's representative direction lies exactly on the
 * edge or corner.  A key's weights are counts out of ORC_TW: each sample
 * point counts 2, or, for the keys whose direction lies on a plane x = +-y
 * (a symmetry plane of HEALPix), 1 in its pixel and 1 in that pixel's
 * mirror image, so that the table keeps the mirror symmetries that the
 * HEALPix pixels have. */
#define ORC_TQH 16  /* face bins on either side of the face centre */
#define ORC_TQ 33   /* (u,v) bins per cube-map face axis: 2*ORC_TQH + centre bin */
#define ORC_TB 40   /* psi = h/d bins of width 1/32 */
#define ORC_TM 8    /* sample points per axis */
#define ORC_TW (2 * ORC_TM * ORC_TM * ORC_TM)   /* weight denominator */
#define ORC_NFACEKEYS (6 * ORC_TQ * ORC_TQ * ORC_TB)
#define ORC_NEDGEKEYS (12 * ORC_TQ * ORC_TB)
#define ORC_NCORNERKEYS (8 * ORC_TB)
#define ORC_NKEYS (ORC_NFACEKEYS + ORC_NEDGEKEYS + ORC_NCORNERKEYS)

typedef struct {
    int32_t N;            /* cells per axis, power of two >= 2 */
    double dx_cm;         /* cell edge, cm */
    int32_t nside;        /* HEALPix N_side */
    int32_t eta_r;        /* radial resolution eta_R (Eq. 4) */
    double theta_lim, theta_if, theta_src;   /* opening angles; INFINITY disables */
    double lray_cells;    /* maximum ray length in cells; <= 0 means domain diagonal */
    double alpha_B;       /* case-B recombination coefficient, cm^3 s^-1 */
    double hnu;           /* mean EUV photon energy, erg */
    int32_t zeta_g;       /* 1: apply the geometric correction (Eq. 16) */
    int32_t kernel_alpha; /* radial kernel for alpha and e: ORC_K_WP or ORC_K_WG */
    int32_t kernel_eps;   /* radial kernel for eps: ORC_KE_* */
    int32_t bc;           /* boundary: ORC_BC_ISOLATED, ORC_BC_PERIODIC, ORC_BC_CORNER */
} orc_params;

/* boundary conditions of the walk (Sec. 2.8) */
enum { ORC_BC_ISOLATED = 0, ORC_BC_PERIODIC = 1, ORC_BC_CORNER = 2 };

/* kernel choices (App. A) */
enum { ORC_K_WP = 0, ORC_K_WG = 1 };
enum { ORC_KE_WF3 = 0, ORC_KE_WF1 = 1, ORC_KE_WF2 = 2, ORC_KE_WF3N = 3, ORC_KE_WP = 4, ORC_KE_WG = 5 };

typedef struct orc_tree orc_tree;

/* HEALPix ring scheme (Gorski et al. 2005) */
int64_t orc_ang2pix(int32_t nside, double x, double y, double z);
void orc_pix2vec(int32_t nside, int64_t pix, double* v3);

/* radial evaluation points (Eq. 4, Eq. 5) */
int32_t orc_num_points(int32_t eta_r, double lray_cells);
double orc_radius(int32_t i, int32_t eta_r);

/* kernels (App. A) */
double orc_wp(double x);
void orc_wf3_split(double d, int32_t nr, int32_t eta_r, double* w_out);
void orc_wp_weights(double d, double h, int32_t nr, int32_t eta_r, double* w_out);
double orc_wg(double x);
void orc_wg_weights(double d, double h, int32_t nr, int32_t eta_r, double* w_out);
void orc_wf1_split(double d, int32_t nr, int32_t eta_r, double* w_out);
void orc_wf2_split(double d, int32_t nr, int32_t eta_r, double* w_out);
void orc_wf3n_weights(double d, double h, int32_t nr, int32_t eta_r, double* w_out);
/* weights of eps for a kernel choice ORC_KE_* */
void orc_eps_weights(int32_t kind, double d, double h, int32_t nr, int32_t eta_r, double* w_out);

/* node->ray table */
int32_t orc_table_key(int64_t ox, int64_t oy, int64_t oz, int64_t s);
int32_t orc_table_entry(int32_t nside, int32_t key, int32_t* pix, int32_t* cnt, int32_t cap);

/* one ray's far-to-near sweep (Sec. 2.5); returns F_0 in rate per cell^2 */
double orc_sweep_ray(int32_t nr, int32_t eta_r, int32_t nside, int32_t zeta_g,
                     const double* alpha_vol, const double* eps, const double* e_vol,
                     double kd, double* phi0_out, double* loss_out);

/* tree */
orc_tree* orc_tree_build(int32_t N, double dx_cm, double alpha_B, const double* box_lo_cm,
                         const double* n_H, const double* ndot_cell,
                         int32_t nsrc, const double* src_xyz_cm, const double* src_Q,
                         const double* e_prev);
/* AMR grid: n_blocks blocks of 8^3 cells; block b has refinement level
 * blk_level[b] (cell edge = (N_base << max_level) >> (log2 N_base + level)
 * finest cells) and corner blk_pos[3b..3b+2] in units of its own edge;
 * cell arrays are [b][iz][iy][ix]; targets are cell indices b*512 + c. */
orc_tree* orc_tree_build_amr(int32_t N_base, int32_t max_level, double dx_fine_cm, double alpha_B,
                             const double* box_lo_cm, int32_t n_blocks, const int32_t* blk_level,
                             const int32_t* blk_pos, const double* n_H, const double* ndot_cell,
                             int32_t nsrc, const double* src_xyz_cm, const double* src_Q, const double* e_prev);
int64_t orc_tree_n_leaves(const orc_tree* t);
int32_t orc_tree_flag(const orc_tree* t, int32_t level, int64_t ix, int64_t iy, int64_t iz);
void orc_tree_free(orc_tree* t);
int32_t orc_tree_levels(const orc_tree* t);
/* out8 = {m, cm_x, cm_y, cm_z, alpha, eps, e, m_ion} */
void orc_tree_node(const orc_tree* t, int32_t level, int64_t ix, int64_t iy, int64_t iz, double* out8);
void orc_cell_quantities(const orc_tree* t, double* ndot_out, double* alpha_out, double* eps_out);

/* walk + map for one target; bins are [npix][nr]; returns visited node count */
int64_t orc_walk_target(const orc_tree* t, const orc_params* p, int64_t target,
                        double* bins_alpha, double* bins_eps, double* bins_e,
                        int64_t* accepted_ids, int64_t cap, int64_t* n_accepted);

/* one pass (walk, map, sweep) over a list of targets (NULL = all cells).
 * F in photons s^-1 cm^-2, e in erg cm^-3, ion = 1 where F > 0. */
/* column-density map of one target (cdMaps): N_PIX values, cm^-2 */
void orc_column_density(const orc_tree* t, const orc_params* p, int64_t target, double* out);

int32_t orc_solve_pass(const orc_tree* t, const orc_params* p, const int64_t* targets,
                       int64_t n_targets, double* F_out, double* e_out, uint8_t* ion_out);

/* unattenuated flux of each target (no recombination losses), cm^-2 s^-1 */
int32_t orc_free_flux(const orc_tree* t, const orc_params* p, const int64_t* targets,
                      int64_t n_targets, double* F_free_out);

/* full iteration (Sec. 2.6): passes until delta < eps_lim or max_iter.
 * delta_mode 0 = per cell (Eq. 21), 1 = total (Eq. 20). */
int32_t orc_solve(const orc_params* p, const double* box_lo_cm, const double* n_H,
                  const double* ndot_cell, int32_t nsrc, const double* src_xyz_cm,
                  const double* src_Q, const double* e_init, int32_t max_iter,
                  double eps_lim, int32_t delta_mode, double* F_out, double* e_out,
                  uint8_t* ion_out, int32_t* iters_out, double* delta_out);

double orc_delta(int64_t n, const double* e_new, const double* e_old, int32_t delta_mode);

#ifdef __cplusplus
}
#endif
#endif
