// Internal declarations of the sm_103a TreeRay/OnTheSpot library.
//
// Units inside the library (chosen so that FP32 storage neither overflows
// nor underflows): lengths in cells of the grid, photon rates in units of
// U = alpha_B dx^3 (so a cell's recombination rate is n_H^2 cells^-3 x U),
// masses in n_H x cells, energy densities in units of
// E_u = alpha_B dx h nu / c (so that a beam of flux F carries e = F).
// Conversions to CGS happen only at the boundary.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/treeray.h"

namespace tr {

// ---- node->ray table definition (Sec. 2.3; the paper's table comes from
// Paper I and is not reproduced: a node is an axis-aligned cube sampled with
// TM^3 points, keyed by the integer offset of its geometric centre; ties
// between axes have keys of their own so that the table keeps the mirror
// symmetries of the HEALPix pixels) -----------------------------------------
constexpr int TQH = 16;                     // face bins on either side of the face centre
constexpr int TQ = 2 * TQH + 1;             // face bins per axis, centre bin included
constexpr int TB = 40;                      // psi = h/d bins of width 1/32
constexpr int TM = 8;                       // sample points per cube axis
constexpr int TW = 2 * TM * TM * TM;        // weight denominator of an entry's count
// keys: face keys (one axis dominates the node offset), edge keys (two axes
// tie for the largest |offset|), corner keys (all three tie)
constexpr int NFACEKEYS = 6 * TQ * TQ * TB;
constexpr int NEDGEKEYS = 12 * TQ * TB;
constexpr int NCORNERKEYS = 8 * TB;
constexpr int NKEYS = NFACEKEYS + NEDGEKEYS + NCORNERKEYS;
constexpr int MAX_LEVELS = 10;              // N <= 512
constexpr int MAX_NR = 128;
constexpr double PI_D = 3.14159265358979323846;
constexpr double DELTA_IF = 1e-8;           // Sec. 2.4
constexpr int N_STATS = 8;                  // walk counters per tree (see tr_tree::stats)

// node topology of an AMR tree (one byte per node; uniform trees need none:
// a node is a leaf exactly when it is on the finest level)
constexpr uint8_t NODE_ABSENT = 0, NODE_LEAF = 1, NODE_PARENT = 2;

struct NodeF64 { double cmx, cmy, cmz, m, alpha, eps, e, mion; };   // 64 B
// FP32 record: the centre of mass is kept as its offset (ox, oy, oz) from the
// node's geometric centre, so that its rounding error scales with the node,
// not with the box; the sign bit of mion marks a node that holds an
// ionisation front (decided in FP64 when the tree is built).
struct NodeF32 { float ox, oy, oz, m, alpha, eps, e, mion; };       // 32 B

struct Table {                              // CSR: entries of key k are ent[off[k] .. off[k+1])
    int nside = 0;
    int n_entries = 0;
    uint32_t* off = nullptr;                // NKEYS + 1
    uint32_t* ent = nullptr;                // (pixel << 16) | count
    uint2* hdr = nullptr;                   // NKEYS x {off[k], number of entries}: one load per key
};

__host__ __device__ inline int64_t level_offset(int l) {
    return ((int64_t(1) << (3 * l)) - 1) / 7;
}

__host__ __device__ inline uint32_t spread3(uint32_t v) {   // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ inline uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}
__host__ __device__ inline uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---- host-side handles ---------------------------------------------------
struct SweepTables {                        // depend on (N_R, eta_R, N_side, N_PIX, zeta_g)
    int nr = 0, eta = 0, nside = 0, zeta_g = -1;
    double* r = nullptr;                    // r_i (cells), FP64
    float* rf = nullptr;                    // r_i, FP32
    double* inv_r2 = nullptr;               // 1/r_j^2 (0 for j = 0)
    double* inv_vol = nullptr;              // 1 / ray-cell volume (cells^-3), 4pi/N_PIX shells
    float* inv_volf = nullptr;              // the same in FP32
    double* G = nullptr;                    // [i][j] (1/2) dV_ij zeta_g,ij (Eq. 14-16)
    double* ID2 = nullptr;                  // [i][j] 1/(r_j - r_mid,i)^2
    double* GI = nullptr;                   // [i][j] G_ij ID2_ij
    float* Gf = nullptr;                    // FP32 copies of G, ID2, GI
    float* ID2f = nullptr;
    float* GIf = nullptr;
    double* HT = nullptr;                   // [j][i] (G_{i-1,j} + G_{i,j}) / V_i: lone-source loss per raw deposit
};

}  // namespace tr

struct tr_tree {
    int device = 0;
    int N = 0, L = 0, mode = 0, use_e = 0;
    int nr = 0, npix = 0;
    double box_lo[3] = {0, 0, 0}, dx = 0, U = 0, Eu = 0, lray = 0;
    tr_params p{};
    int64_t n_nodes = 0;
    void* nodes = nullptr;                  // NodeF64[n_nodes] (mode 0) or NodeF32[n_nodes]
    void* sums = nullptr;                   // build scratch: FP64 {smx,smy,smz} or FP32 offsets x mass
    // FP32 forms: the same tree in FP64 (the walk re-decides in FP64 the few
    // comparisons that FP32 cannot settle) and the bound kappa on the FP32
    // centre-of-mass error, |cm32 - cm64| <= kappa x node edge; mode 0:
    // nodes64 = nodes and kappa unused
    void* nodes64 = nullptr;
    void* sums64 = nullptr;
    float* kappa = nullptr;
    double* ndot = nullptr;                 // N^3 mapped emission (photons s^-1)
    int32_t* status = nullptr;              // device status words: [0] overflowed targets, [1] deepest stack
    unsigned long long* stats = nullptr;    // device counters of the last walk: visited, accepted, entries,
                                            // MAC decisions and deposit set-ups redone in FP64
    unsigned int* counter = nullptr;        // persistent-kernel work counter
    const tr::Table* table = nullptr;
    tr::SweepTables sw;
    size_t nodes_bytes = 0;
    void* jobbuf = nullptr;                 // device copy of the walk's job record
    double* e_work = nullptr;               // tr_solve iteration: 2 x N^3 energy densities
    void* dscratch = nullptr;               // tr_solve iteration: delta reduction state
    int64_t n_cells = 0;                    // targets: N^3, or n_blocks x 512 (AMR)
    // AMR trees only (NULL / 0 for a uniform grid)
    int32_t n_blocks = 0;
    uint8_t* flags = nullptr;               // n_nodes: NODE_ABSENT / NODE_LEAF / NODE_PARENT
    int4* blk = nullptr;                    // n_blocks: {tree level of its cells, x, y, z position in blocks}
    uint32_t* blk_order = nullptr;          // n_blocks: blocks along the Morton curve of the finest lattice
    int32_t* blkmap = nullptr;              // nodes of levels 0 .. L-3: block index, or -1
};

struct tr_rays {
    int device = 0;
    int64_t n_targets = 0;
    int npix = 0, nr = 0, acc_cap = 0, use_e = 0, mode = 0;
    float* scales = nullptr;                // FP32 form: fixed-point units of the raw bins
    double U = 0, Eu = 0, dx = 0;
    tr::SweepTables sw;                     // borrowed copy of the tree's tables (owned here)
    double* bins = nullptr;                 // [n_targets][3][npix][nr] raw bins (FP64, or FP32-form fixed point)
    int32_t* ids = nullptr;                 // [n_targets][acc_cap]
    int32_t* counts = nullptr;              // [n_targets]
    int64_t* target_idx = nullptr;          // [n_targets] C-order cell indices
    double* eps_self = nullptr;             // [n_targets] own emission (scaled)
};

namespace tr {

// error reporting and argument checks (tr_api.cu)
tr_status set_error(tr_status st, const char* fmt, ...);
void clear_error();
tr_status cuda_check(cudaError_t e, const char* what);
tr_status check_params(const tr_params* p);
tr_status check_grid(const tr_grid* g, const tr_sources* s);
double default_lray(int N, const tr_params* p);   // cells

// table (tr_table.cu)
tr_status table_get(int nside, const Table** out, cudaStream_t st);
// build the table into caller-provided device memory (t->off, t->ent, t->hdr
// set; counts: NKEYS words of scratch); TR_EUNSUPPORTED if it needs more
// than ent_capacity entries.  Synchronises st.
tr_status table_build_into(int nside, Table* t, uint32_t* counts, uint32_t ent_capacity, cudaStream_t st);

// tree (tr_tree.cu)
tr_status tree_build(tr_tree* t, const tr_grid* g, const tr_sources* s, cudaStream_t st);
// AMR: t->flags, blk, blk_order, blkmap are set up (device) and t->n_cells
// = n_blocks x 512; n_H, ndot, e_prev are cell arrays in block order
tr_status tree_build_amr(tr_tree* t, const double* n_H, const double* ndot, const double* e_prev,
                         const tr_sources* s, cudaStream_t st);
// AMR: flags and block map from t->blk (once per block layout)
tr_status amr_topology(tr_tree* t, cudaStream_t st);
tr_status tree_export(const tr_tree* t, double* out8, cudaStream_t st);
// FP32 forms: IF flags and the centre-of-mass error bound from the FP64 tree
tr_status finalize_f32(tr_tree* t, cudaStream_t st);
tr_status flags_export(const tr_tree* t, uint8_t* out, cudaStream_t st);
tr_status sweep_tables_make(SweepTables* sw, int nr, int eta, int nside, int npix, int zeta_g,
                            cudaStream_t st);
void sweep_tables_free(SweepTables* sw);
// fill tables whose device pointers are already set (no allocation)
tr_status sweep_tables_fill(SweepTables* sw, int nr, int eta, int nside, int npix, int zeta_g, cudaStream_t st);

// walk (tr_walk.cu)
struct WalkOut {
    double* F = nullptr;                    // CGS outputs, indexed like the targets
    double* e = nullptr;
    uint8_t* ion = nullptr;
    double* bins = nullptr;                 // dump mode: [target][3][npix][nr]
    int32_t* ids = nullptr;                 // dump mode: [target][acc_cap]
    int32_t* counts = nullptr;
    double* eps_self = nullptr;
    float* scales = nullptr;
    int acc_cap = 0;
};
tr_status walk_run(const tr_tree* t, const int64_t* targets, int64_t n_targets, bool dump,
                   const WalkOut& out, cudaStream_t st);
tr_status sweep_run(const tr_rays* r, double* F, double* e, uint8_t* ion, cudaStream_t st);
// column-density maps of targets (NULL: cells 0 .. n_targets-1), out [target][N_PIX]
tr_status cd_run(const tr_tree* t, const int64_t* targets, int64_t n_targets, double* out, cudaStream_t st);
size_t walk_job_bytes(int n_jobs);
tr_status walk_batch_run(const tr_tree* const* trees, const int64_t* first, const int64_t* count, int n,
                         double* const* F, double* const* e, uint8_t* const* ion, void* jobbuf, unsigned int* counter,
                         cudaStream_t st);
tr_status read_status(const tr_tree* t, cudaStream_t st);

// iteration error control (tr_iter.cu)
size_t delta_scratch_bytes();
tr_status delta_compute(const double* e_new, const double* e_old, int64_t n, int mode, void* scratch, double* out,
                        cudaStream_t st);

}  // namespace tr
