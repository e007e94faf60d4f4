// C ABI of the library: argument checks, handle management, and the order
// of the kernels for each entry point.  See include/treeray.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <unordered_set>
#include <utility>
#include <vector>

#include "tr_internal.cuh"

namespace tr {

static thread_local char g_err[512] = "";

tr_status set_error(tr_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_err[0] = '\0'; }

tr_status cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TR_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(TR_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(TR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
constexpr double C_LIGHT = 2.99792458e10;   // cm s^-1
bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
}  // namespace

tr_status check_params(const tr_params* p) {
    if (!p) return set_error(TR_EINVAL, "params is NULL");
    if (!(p->theta_lim > 0.0) || !(p->theta_if > 0.0) || !(p->theta_src > 0.0))
        return set_error(TR_EINVAL, "opening angles must be > 0 (INFINITY disables IF/Src MACs)");
    if (p->nside != 1 && p->nside != 2 && p->nside != 4 && p->nside != 8)
        return set_error(TR_EINVAL, "nside must be 1, 2, 4 or 8 (got %d)", p->nside);
    if (!is_pow2(p->eta_r) || p->eta_r > 8)
        return set_error(TR_EINVAL, "eta_r must be 1, 2, 4 or 8 (got %d)", p->eta_r);
    if (!(p->alpha_B > 0.0) || !std::isfinite(p->alpha_B)) return set_error(TR_EINVAL, "alpha_B must be finite and > 0");
    if (!(p->hnu > 0.0) || !std::isfinite(p->hnu)) return set_error(TR_EINVAL, "hnu must be finite and > 0");
    if (p->precision != TR_FP64 && p->precision != TR_FP32_SWEEP64 && p->precision != TR_FP32_SWEEPDF)
        return set_error(TR_EINVAL, "precision must be TR_FP64, TR_FP32_SWEEP64 or TR_FP32_SWEEPDF");
    if (p->max_iter < 1) return set_error(TR_EINVAL, "max_iter must be >= 1");
    if (p->delta_mode != 0 && p->delta_mode != 1) return set_error(TR_EINVAL, "delta_mode must be 0 or 1");
    if (p->kernel_alpha != TR_KERNEL_WP && p->kernel_alpha != TR_KERNEL_WG)
        return set_error(TR_EINVAL, "kernel_alpha must be TR_KERNEL_WP or TR_KERNEL_WG (got %d)", p->kernel_alpha);
    if (p->kernel_eps < TR_EPS_WF3 || p->kernel_eps > TR_EPS_WG)
        return set_error(TR_EINVAL, "kernel_eps must be one of tr_eps_kernel (got %d)", p->kernel_eps);
    if (p->bc < TR_BC_ISOLATED || p->bc > TR_BC_CORNER)
        return set_error(TR_EINVAL, "bc must be one of tr_bc (got %d)", p->bc);
    return TR_OK;
}

// default maximum ray length in cells: the domain diagonal (of the mirrored
// domain under the corner-of-symmetry boundary)
double default_lray(int N, const tr_params* p) {
    return (p->bc == TR_BC_CORNER ? 2.0 : 1.0) * (double)N * std::sqrt(3.0);
}

tr_status check_grid(const tr_grid* g, const tr_sources* s) {
    if (!g) return set_error(TR_EINVAL, "grid is NULL");
    if (!is_pow2(g->N) || g->N < 8 || g->N > 512)
        return set_error(TR_EINVAL, "N must be a power of two in [8, 512] (got %d)", g->N);
    if (!(g->dx > 0.0) || !std::isfinite(g->dx)) return set_error(TR_EINVAL, "dx must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->box_lo[a])) return set_error(TR_EINVAL, "box_lo must be finite");
    if (!g->n_H) return set_error(TR_EINVAL, "n_H is NULL");
    if (s && s->n < 0) return set_error(TR_EINVAL, "negative source count");
    if (s && s->n > 0 && (!s->xyz || !s->Q)) return set_error(TR_EINVAL, "source arrays are NULL");
    return TR_OK;
}

namespace {

template <typename T>
tr_status dev_alloc(T** p, size_t bytes, const char* what) {
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(TR_ENOMEM, "cannot allocate %zu bytes for %s", bytes, what);
    }
    return TR_OK;
}

void tree_release(tr_tree* t) {
    if (!t) return;
    if (t->nodes64 != t->nodes) cudaFree(t->nodes64);
    if (t->sums64 != t->sums) cudaFree(t->sums64);
    cudaFree(t->kappa);
    cudaFree(t->nodes);
    cudaFree(t->sums);
    cudaFree(t->ndot);
    cudaFree(t->status);
    cudaFree(t->stats);
    cudaFree(t->counter);
    cudaFree(t->jobbuf);
    cudaFree(t->e_work);
    cudaFree(t->dscratch);
    cudaFree(t->flags);
    cudaFree(t->blk);
    cudaFree(t->blk_order);
    cudaFree(t->blkmap);
    sweep_tables_free(&t->sw);
    delete t;
}

// The FP64 tree beside the FP32 record of the FP32 forms (mode 0: the tree
// itself), and the device word of the centre-of-mass error bound.
tr_status alloc_sidecar(tr_tree* t) {
    if (t->mode == 0) {
        t->nodes64 = t->nodes;
        t->sums64 = t->sums;
        return TR_OK;
    }
    tr_status rc = dev_alloc(&t->nodes64, sizeof(NodeF64) * (size_t)t->n_nodes, "FP64 tree nodes");
    if (rc == TR_OK) rc = dev_alloc(&t->sums64, 3 * sizeof(double) * (size_t)t->n_nodes, "FP64 tree build sums");
    if (rc == TR_OK) rc = dev_alloc(&t->kappa, sizeof(float), "centre-of-mass error bound");
    return rc;
}

// Allocate (or reuse) a tree for this grid and parameters, then build it.
tr_status build(const tr_grid* g, const tr_sources* s, const tr_params* p, tr_tree** inout, cudaStream_t st) {
    tr_status rc = check_params(p);
    if (rc == TR_OK) rc = check_grid(g, s);
    if (rc != TR_OK) return rc;
    int dev = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) != TR_OK) return rc;
    const int N = g->N;
    int L = 0;
    while ((1 << L) < N) ++L;
    const double lray = p->L_ray_cm > 0.0 ? p->L_ray_cm / g->dx : default_lray(N, p);
    const int nr = p->eta_r * (int)std::floor(std::sqrt(2.0 * lray)) + 1;      // Eq. 5
    if (nr > MAX_NR) return set_error(TR_EUNSUPPORTED, "N_R = %d exceeds %d evaluation points", nr, MAX_NR);
    if (nr < 3) return set_error(TR_EINVAL, "L_ray too short: N_R = %d", nr);
    const int mode = p->precision;
    const int64_t n_nodes = level_offset(L + 1);
    const size_t rec = mode == 0 ? sizeof(NodeF64) : sizeof(NodeF32);
    const size_t sum_bytes = (size_t)n_nodes * 3 * (mode == 0 ? sizeof(double) : sizeof(float));
    tr_tree* t = *inout;
    if (t && (t->N != N || t->mode != mode || t->device != dev || t->flags)) {
        // the iteration buffers belong to the tree and go with it
        tree_release(t);
        t = nullptr;
        *inout = nullptr;
    }
    if (!t) {
        t = new tr_tree();
        t->device = dev;
        t->N = N; t->L = L; t->mode = mode;
        t->n_nodes = n_nodes;
        t->n_cells = (int64_t)N * N * N;
        t->nodes_bytes = (size_t)n_nodes * rec;
        if ((rc = dev_alloc(&t->nodes, t->nodes_bytes, "tree nodes")) != TR_OK ||
            (rc = dev_alloc(&t->sums, sum_bytes, "tree build sums")) != TR_OK ||
            (rc = alloc_sidecar(t)) != TR_OK ||
            (rc = dev_alloc(&t->ndot, sizeof(double) * (size_t)N * N * N, "cell emission")) != TR_OK ||
            (rc = dev_alloc(&t->status, 4 * sizeof(int32_t), "status words")) != TR_OK ||
            (rc = dev_alloc(&t->stats, N_STATS * sizeof(unsigned long long), "walk counters")) != TR_OK ||
            (rc = dev_alloc(&t->counter, sizeof(unsigned int), "work counter")) != TR_OK ||
            (rc = dev_alloc((unsigned char**)&t->jobbuf, walk_job_bytes(1), "walk job record")) != TR_OK) {
            tree_release(t);
            return rc;
        }
    }
    t->p = *p;
    t->use_e = g->e_prev != nullptr;
    t->nr = nr;
    t->npix = 12 * p->nside * p->nside;
    for (int a = 0; a < 3; ++a) t->box_lo[a] = g->box_lo[a];
    t->dx = g->dx;
    t->U = p->alpha_B * g->dx * g->dx * g->dx;
    t->Eu = p->alpha_B * g->dx * p->hnu / C_LIGHT;
    t->lray = lray;
    *inout = t;
    if ((rc = table_get(p->nside, &t->table, st)) != TR_OK) return rc;
    if ((rc = sweep_tables_make(&t->sw, nr, p->eta_r, p->nside, t->npix, p->zeta_g ? 1 : 0, st)) != TR_OK) return rc;
    return tree_build(t, g, s, st);
}

// AMR block layout checks (host): levels and positions in range, no block
// inside another, and the blocks' volume equal to the box's.
tr_status check_amr(const tr_amr_grid* g, const tr_sources* s, int* L_out, int* Lb_out) {
    if (!g) return set_error(TR_EINVAL, "grid is NULL");
    if (!is_pow2(g->N_base) || g->N_base < 8) return set_error(TR_EINVAL, "N_base must be a power of two >= 8 (got %d)", g->N_base);
    if (g->max_level < 0 || g->max_level > 6) return set_error(TR_EINVAL, "max_level out of range (got %d)", g->max_level);
    const int64_t Nf = (int64_t)g->N_base << g->max_level;
    if (Nf > 512) return set_error(TR_EUNSUPPORTED, "finest lattice N_base << max_level = %lld exceeds 512", (long long)Nf);
    if (g->n_blocks < 1 || !g->blk_level || !g->blk_pos) return set_error(TR_EINVAL, "no blocks");
    if (!g->n_H) return set_error(TR_EINVAL, "n_H is NULL");
    if (!(g->dx_fine > 0.0) || !std::isfinite(g->dx_fine)) return set_error(TR_EINVAL, "dx_fine must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->box_lo[a])) return set_error(TR_EINVAL, "box_lo must be finite");
    if (s && s->n < 0) return set_error(TR_EINVAL, "negative source count");
    if (s && s->n > 0 && (!s->xyz || !s->Q)) return set_error(TR_EINVAL, "source arrays are NULL");
    int L = 0, Lb = 0;
    while ((1 << L) < Nf) ++L;
    while ((1 << Lb) < g->N_base) ++Lb;
    // blocks as nodes of the octree: level Lb - 3 + level, position in blocks
    std::unordered_set<uint64_t> keys;
    keys.reserve((size_t)g->n_blocks * 2);
    auto key = [](int l, int64_t x, int64_t y, int64_t z) {
        return ((uint64_t)l << 60) | ((uint64_t)z << 40) | ((uint64_t)y << 20) | (uint64_t)x;
    };
    unsigned __int128 vol = 0;
    for (int b = 0; b < g->n_blocks; ++b) {
        const int lev = g->blk_level[b];
        if (lev < 0 || lev > g->max_level) return set_error(TR_EINVAL, "block %d: level %d out of range", b, lev);
        const int64_t nb = (int64_t)(g->N_base >> 3) << lev;
        for (int a = 0; a < 3; ++a)
            if (g->blk_pos[3 * b + a] < 0 || g->blk_pos[3 * b + a] >= nb)
                return set_error(TR_EINVAL, "block %d: position out of range", b);
        if (!keys.insert(key(lev, g->blk_pos[3 * b], g->blk_pos[3 * b + 1], g->blk_pos[3 * b + 2])).second)
            return set_error(TR_EINVAL, "block %d repeats another block", b);
        const int64_t e = (int64_t)1 << (g->max_level - lev);
        vol += (unsigned __int128)(e * e * e);
    }
    for (int b = 0; b < g->n_blocks; ++b) {
        const int lev = g->blk_level[b];
        for (int l = lev - 1; l >= 0; --l) {
            const int sh = lev - l;
            if (keys.count(key(l, g->blk_pos[3 * b] >> sh, g->blk_pos[3 * b + 1] >> sh, g->blk_pos[3 * b + 2] >> sh)))
                return set_error(TR_EINVAL, "block %d lies inside a coarser block", b);
        }
    }
    const int64_t nb0 = g->N_base >> 3;
    const unsigned __int128 e0 = (unsigned __int128)1 << g->max_level;
    if (vol != (unsigned __int128)(nb0 * nb0 * nb0) * e0 * e0 * e0)
        return set_error(TR_EINVAL, "the blocks do not fill the box");
    *L_out = L;
    *Lb_out = Lb;
    return TR_OK;
}

tr_status build_amr(const tr_amr_grid* g, const tr_sources* s, const tr_params* p, tr_tree** inout, cudaStream_t st) {
    tr_status rc = check_params(p);
    int L = 0, Lb = 0;
    if (rc == TR_OK) rc = check_amr(g, s, &L, &Lb);
    if (rc != TR_OK) return rc;
    int dev = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) != TR_OK) return rc;
    const int N = g->N_base << g->max_level;
    const double lray = p->L_ray_cm > 0.0 ? p->L_ray_cm / g->dx_fine : default_lray(N, p);
    const int nr = p->eta_r * (int)std::floor(std::sqrt(2.0 * lray)) + 1;      // Eq. 5
    if (nr > MAX_NR) return set_error(TR_EUNSUPPORTED, "N_R = %d exceeds %d evaluation points", nr, MAX_NR);
    if (nr < 3) return set_error(TR_EINVAL, "L_ray too short: N_R = %d", nr);
    // host tables: {cell level, x, y, z} per block, and the walk order (the
    // Morton code of each block's corner on the finest lattice; aligned
    // cubes are contiguous along the Morton curve)
    const int nb = g->n_blocks;
    std::vector<int4> hblk(nb);
    std::vector<std::pair<uint32_t, uint32_t>> order(nb);
    for (int b = 0; b < nb; ++b) {
        const int lev = g->blk_level[b];
        hblk[b] = make_int4(Lb + lev, g->blk_pos[3 * b], g->blk_pos[3 * b + 1], g->blk_pos[3 * b + 2]);
        const uint32_t e = 8u << (g->max_level - lev);
        order[b] = {morton3(g->blk_pos[3 * b] * e, g->blk_pos[3 * b + 1] * e, g->blk_pos[3 * b + 2] * e), (uint32_t)b};
    }
    std::sort(order.begin(), order.end());
    std::vector<uint32_t> horder(nb);
    for (int b = 0; b < nb; ++b) horder[b] = order[b].second;

    if (*inout) { tree_release(*inout); *inout = nullptr; }
    const int mode = p->precision;
    tr_tree* t = new tr_tree();
    t->device = dev;
    t->N = N; t->L = L; t->mode = mode;
    t->n_nodes = level_offset(L + 1);
    t->n_cells = (int64_t)nb * 512;
    t->n_blocks = nb;
    t->nodes_bytes = (size_t)t->n_nodes * (mode == 0 ? sizeof(NodeF64) : sizeof(NodeF32));
    const size_t sum_bytes = (size_t)t->n_nodes * 3 * (mode == 0 ? sizeof(double) : sizeof(float));
    if ((rc = dev_alloc(&t->nodes, t->nodes_bytes, "tree nodes")) != TR_OK ||
        (rc = dev_alloc(&t->sums, sum_bytes, "tree build sums")) != TR_OK ||
        (rc = alloc_sidecar(t)) != TR_OK ||
        (rc = dev_alloc(&t->ndot, sizeof(double) * (size_t)t->n_cells, "cell emission")) != TR_OK ||
        (rc = dev_alloc(&t->status, 4 * sizeof(int32_t), "status words")) != TR_OK ||
        (rc = dev_alloc(&t->stats, N_STATS * sizeof(unsigned long long), "walk counters")) != TR_OK ||
        (rc = dev_alloc(&t->counter, sizeof(unsigned int), "work counter")) != TR_OK ||
        (rc = dev_alloc((unsigned char**)&t->jobbuf, walk_job_bytes(1), "walk job record")) != TR_OK ||
        (rc = dev_alloc(&t->flags, (size_t)t->n_nodes, "node flags")) != TR_OK ||
        (rc = dev_alloc(&t->blk, sizeof(int4) * (size_t)nb, "block table")) != TR_OK ||
        (rc = dev_alloc(&t->blk_order, sizeof(uint32_t) * (size_t)nb, "block order")) != TR_OK ||
        (rc = dev_alloc(&t->blkmap, sizeof(int32_t) * (size_t)level_offset(L - 2), "block map")) != TR_OK) {
        tree_release(t);
        return rc;
    }
    t->p = *p;
    t->use_e = g->e_prev != nullptr;
    t->nr = nr;
    t->npix = 12 * p->nside * p->nside;
    for (int a = 0; a < 3; ++a) t->box_lo[a] = g->box_lo[a];
    t->dx = g->dx_fine;
    t->U = p->alpha_B * g->dx_fine * g->dx_fine * g->dx_fine;
    t->Eu = p->alpha_B * g->dx_fine * p->hnu / C_LIGHT;
    t->lray = lray;
    *inout = t;
    rc = cuda_check(cudaMemcpyAsync(t->blk, hblk.data(), sizeof(int4) * nb, cudaMemcpyHostToDevice, st), "block table copy");
    if (rc == TR_OK)
        rc = cuda_check(cudaMemcpyAsync(t->blk_order, horder.data(), sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st),
                        "block order copy");
    if (rc == TR_OK) rc = amr_topology(t, st);
    // the host tables go out of scope on return
    if (rc == TR_OK) rc = cuda_check(cudaStreamSynchronize(st), "block tables");
    if (rc != TR_OK) return rc;
    if ((rc = table_get(p->nside, &t->table, st)) != TR_OK) return rc;
    if ((rc = sweep_tables_make(&t->sw, nr, p->eta_r, p->nside, t->npix, p->zeta_g ? 1 : 0, st)) != TR_OK) return rc;
    return tree_build_amr(t, g->n_H, g->ndot, g->e_prev, s, st);
}

std::mutex g_solve_mu;
std::map<int, tr_tree*> g_solve_trees;   // per device, reused by tr_solve

__global__ void k_iota(int64_t* v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

__device__ double raw_bin(const double* slot, int mode, float scale) {
    if (mode == 0) return *slot;
    const uint2 v = *reinterpret_cast<const uint2*>(slot);
    return ((double)v.y * 4294967296.0 + (double)v.x) / (double)scale;
}

__global__ void k_export_bins(const double* bins, int64_t n, int nbins, int mode, const float* sc, double U, double Eu,
                              double* a, double* e, double* ee) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nbins) return;
    const int64_t q = i / nbins, b = i % nbins;
    const double* in = bins + q * 3 * nbins;
    if (a) a[i] = raw_bin(in + b, mode, sc[0]) * U;
    if (e) e[i] = raw_bin(in + nbins + b, mode, sc[1]) * U;
    if (ee) ee[i] = raw_bin(in + 2 * nbins + b, mode, sc[2]) * Eu;
}

__global__ void k_export_ids(const int32_t* ids, const int32_t* counts, int64_t n, int cap, int64_t* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * cap) return;
    const int64_t q = i / cap;
    const int k = (int)(i % cap);
    out[i] = (k < counts[q]) ? (int64_t)ids[i] : -1;
}

__global__ void k_table_split(const uint32_t* off, const uint32_t* ent, int nkeys, int32_t* o, int32_t* pix,
                              int32_t* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nkeys && o) o[i] = (int32_t)off[i];
    if (i < (int)off[nkeys]) {
        if (pix) pix[i] = (int32_t)(ent[i] >> 16);
        if (cnt) cnt[i] = (int32_t)(ent[i] & 0xffffu);
    }
}

}  // namespace
}  // namespace tr

using namespace tr;

extern "C" {

void tr_params_default(tr_params* p) {
    if (!p) return;
    p->theta_lim = 0.5;
    p->theta_if = INFINITY;
    p->theta_src = INFINITY;
    p->nside = 2;
    p->eta_r = 2;
    p->L_ray_cm = 0.0;
    p->alpha_B = 2.7e-13;
    p->hnu = 13.6 * 1.602176634e-12;
    p->eps_lim = 1e-2;
    p->delta_mode = 0;
    p->max_iter = 1;
    p->precision = TR_FP64;
    p->zeta_g = 1;
    p->kernel_alpha = TR_KERNEL_WP;
    p->kernel_eps = TR_EPS_WF3;
    p->bc = TR_BC_ISOLATED;
}

const char* tr_last_error(void) { return g_err; }

tr_status tr_build_tree_amr(const tr_amr_grid* g, const tr_sources* s, const tr_params* p, tr_tree** out,
                            tr_stream stream) {
    g_err[0] = '\0';
    if (!out) return set_error(TR_EINVAL, "out is NULL");
    return build_amr(g, s, p, out, (cudaStream_t)stream);
}

tr_status tr_tree_cells(const tr_tree* t, int64_t* n_cells) {
    g_err[0] = '\0';
    if (!t || !n_cells) return set_error(TR_EINVAL, "tree or output is NULL");
    *n_cells = t->n_cells;
    return TR_OK;
}

tr_status tr_build_tree(const tr_grid* g, const tr_sources* s, const tr_params* p, tr_tree** out, tr_stream stream) {
    g_err[0] = '\0';
    if (!out) return set_error(TR_EINVAL, "out is NULL");
    return build(g, s, p, out, (cudaStream_t)stream);
}

tr_status tr_walk_map(const tr_tree* t, const int64_t* targets, int64_t n_targets, tr_rays** out, tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    if (!t || !out) return set_error(TR_EINVAL, "tree or out is NULL");
    const int64_t ncell = t->n_cells;
    if (n_targets < 0 || n_targets > ncell) return set_error(TR_EINVAL, "n_targets out of range");
    if (!targets && n_targets != ncell) return set_error(TR_EINVAL, "targets NULL requires n_targets = the cell count");
    tr_rays* r = new tr_rays();
    r->device = t->device;
    r->n_targets = n_targets;
    r->npix = t->npix; r->nr = t->nr; r->use_e = t->use_e; r->mode = t->mode;
    r->U = t->U; r->Eu = t->Eu; r->dx = t->dx;
    r->acc_cap = 4096;
    const int nbins = t->npix * t->nr;
    const int64_t nt = n_targets > 0 ? n_targets : 1;
    tr_status rc;
    if ((rc = dev_alloc(&r->bins, sizeof(double) * 3 * nbins * (size_t)nt, "ray bins")) != TR_OK ||
        (rc = dev_alloc(&r->ids, sizeof(int32_t) * (size_t)r->acc_cap * nt, "accepted ids")) != TR_OK ||
        (rc = dev_alloc(&r->counts, sizeof(int32_t) * (size_t)nt, "accepted counts")) != TR_OK ||
        (rc = dev_alloc(&r->eps_self, sizeof(double) * (size_t)nt, "own emission")) != TR_OK ||
        (rc = dev_alloc(&r->target_idx, sizeof(int64_t) * (size_t)nt, "targets")) != TR_OK ||
        (rc = dev_alloc(&r->scales, 4 * sizeof(float), "bin scales")) != TR_OK) {
        tr_rays_free(r);
        return rc;
    }
    if (targets) rc = cuda_check(cudaMemcpyAsync(r->target_idx, targets, sizeof(int64_t) * n_targets,
                                                 cudaMemcpyDeviceToDevice, st), "copy targets");
    else { k_iota<<<(unsigned)((n_targets + 255) / 256), 256, 0, st>>>(r->target_idx, n_targets); rc = cuda_check(cudaGetLastError(), "iota"); }
    if (rc == TR_OK) rc = sweep_tables_make(&r->sw, t->nr, t->p.eta_r, t->p.nside, t->npix, t->p.zeta_g ? 1 : 0, st);
    if (rc == TR_OK && n_targets > 0) {
        WalkOut o;
        o.bins = r->bins; o.ids = r->ids; o.counts = r->counts; o.eps_self = r->eps_self; o.acc_cap = r->acc_cap;
        o.scales = r->scales;
        rc = walk_run(t, r->target_idx, n_targets, true, o, st);
        if (rc == TR_OK) rc = read_status(t, st);
    }
    if (rc != TR_OK) { tr_rays_free(r); return rc; }
    *out = r;
    return TR_OK;
}

tr_status tr_ray_sweep(const tr_rays* r, double* F_out, double* e_out, uint8_t* ion_out, tr_stream stream) {
    g_err[0] = '\0';
    if (!r) return set_error(TR_EINVAL, "rays is NULL");
    if (r->n_targets == 0) return TR_OK;
    return sweep_run(r, F_out, e_out, ion_out, (cudaStream_t)stream);
}

tr_status tr_walk_sweep(const tr_tree* t, double* F_out, double* e_out, uint8_t* ion_out, tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    if (!t) return set_error(TR_EINVAL, "tree is NULL");
    WalkOut o;
    o.F = F_out; o.e = e_out; o.ion = ion_out;
    tr_status rc = walk_run(t, nullptr, t->n_cells, false, o, st);
    if (rc == TR_OK) rc = read_status(t, st);
    return rc;
}

namespace {
struct BatchSpace {                          // per device: job records and work counter of batched walks
    void* jobbuf = nullptr;
    size_t bytes = 0;
    unsigned int* counter = nullptr;
};
std::mutex g_batch_mu;
std::map<int, BatchSpace> g_batch;
}  // namespace

tr_status tr_walk_sweep_batch(const tr_tree* const* trees, const int64_t* first, const int64_t* count, int32_t n,
                              double* const* F_out, double* const* e_out, uint8_t* const* ion_out, tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    if (!trees || !first || !count || n < 1) return set_error(TR_EINVAL, "bad batch arguments");
    int dev = 0;
    tr_status rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc != TR_OK) return rc;
    for (int i = 0; i < n; ++i) {
        const tr_tree* t = trees[i];
        if (!t) return set_error(TR_EINVAL, "tree %d is NULL", i);
        if (t->device != dev) return set_error(TR_EINVAL, "tree %d lives on device %d, current is %d", i, t->device, dev);
        if (t->mode != trees[0]->mode) return set_error(TR_EINVAL, "trees of one batch share a precision");
        if (first[i] < 0 || count[i] < 0 || first[i] + count[i] > t->n_cells)
            return set_error(TR_EINVAL, "target range %d out of [0, cells)", i);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchSpace& b = g_batch[dev];
    const size_t need = walk_job_bytes(n);
    if (b.bytes < need) {
        cudaFree(b.jobbuf);
        b.jobbuf = nullptr;
        b.bytes = 0;
        if ((rc = dev_alloc((unsigned char**)&b.jobbuf, need, "batch job records")) != TR_OK) return rc;
        b.bytes = need;
    }
    if (!b.counter && (rc = dev_alloc(&b.counter, sizeof(unsigned int), "batch work counter")) != TR_OK) return rc;
    if ((rc = walk_batch_run(trees, first, count, n, F_out, e_out, ion_out, b.jobbuf, b.counter, st)) != TR_OK)
        return rc;
    for (int i = 0; i < n; ++i)
        if ((rc = read_status(trees[i], st)) != TR_OK) return rc;
    return TR_OK;
}

tr_status tr_column_density(const tr_tree* t, const int64_t* targets, int64_t n_targets, double* out,
                            tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    if (!t || !out) return set_error(TR_EINVAL, "tree or output is NULL");
    if (n_targets < 0 || n_targets > t->n_cells) return set_error(TR_EINVAL, "n_targets out of range");
    if (!targets && n_targets != t->n_cells) return set_error(TR_EINVAL, "targets NULL requires n_targets = the cell count");
    tr_status rc = cd_run(t, targets, n_targets, out, st);
    if (rc == TR_OK) rc = read_status(t, st);
    return rc;
}

tr_status tr_tree_stats(const tr_tree* t, int64_t* out6) {
    g_err[0] = '\0';
    if (!t || !out6) return set_error(TR_EINVAL, "tree or output is NULL");
    unsigned long long h[N_STATS] = {};
    int32_t st[4] = {0, 0, 0, 0};
    tr_status rc = cuda_check(cudaMemcpy(h, t->stats, sizeof h, cudaMemcpyDeviceToHost), "stats copy");
    if (rc == TR_OK) rc = cuda_check(cudaMemcpy(st, t->status, sizeof st, cudaMemcpyDeviceToHost), "status copy");
    if (rc != TR_OK) return rc;
    out6[0] = (int64_t)h[0]; out6[1] = (int64_t)h[1]; out6[2] = (int64_t)h[2]; out6[3] = st[1];
    out6[4] = (int64_t)h[3]; out6[5] = (int64_t)h[4];
    return TR_OK;
}

tr_status tr_solve(const tr_grid* g, const tr_sources* s, const tr_params* p, double* F_out, double* e_out,
                   uint8_t* ion_out, int32_t* iters_out, double* delta_out, tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    tr_status rc = check_params(p);
    if (rc == TR_OK) rc = check_grid(g, s);
    if (rc != TR_OK) return rc;
    if (!(p->eps_lim >= 0.0)) return set_error(TR_EINVAL, "eps_lim must be >= 0");
    int dev = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) != TR_OK) return rc;
    std::lock_guard<std::mutex> lock(g_solve_mu);
    tr_tree*& t = g_solve_trees[dev];
    const int64_t ncell = (int64_t)g->N * g->N * g->N;
    const bool need_delta = p->max_iter > 1 || (delta_out && g->e_prev);
    if (!need_delta) {
        // one pass (Sec. 2.3-2.5)
        if ((rc = build(g, s, p, &t, st)) != TR_OK) return rc;
        WalkOut o;
        o.F = F_out; o.e = e_out; o.ion = ion_out;
        if ((rc = walk_run(t, nullptr, ncell, false, o, st)) != TR_OK) return rc;
        if ((rc = read_status(t, st)) != TR_OK) return rc;
        if (iters_out) *iters_out = 1;
        if (delta_out) *delta_out = INFINITY;
        return TR_OK;
    }
    // outer iteration (Sec. 2.6): each pass builds the tree with the energy
    // density of the previous pass (IF MAC, zeta_d) until delta < eps_lim
    if ((rc = build(g, s, p, &t, st)) != TR_OK) return rc;     // allocates / sizes the tree
    if (!t->e_work && (rc = dev_alloc(&t->e_work, 2 * sizeof(double) * (size_t)ncell, "iteration buffers")) != TR_OK)
        return rc;
    if (!t->dscratch && (rc = dev_alloc((unsigned char**)&t->dscratch, delta_scratch_bytes(), "delta state")) != TR_OK)
        return rc;
    double* e_old = t->e_work;
    double* e_new = t->e_work + ncell;
    if (g->e_prev) rc = cuda_check(cudaMemcpyAsync(e_old, g->e_prev, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, st), "copy e_prev");
    else rc = cuda_check(cudaMemsetAsync(e_old, 0, sizeof(double) * ncell, st), "clear e");
    if (rc != TR_OK) return rc;
    int it = 0;
    double delta = INFINITY;
    while (it < p->max_iter) {
        tr_grid gi = *g;
        gi.e_prev = (it == 0 && !g->e_prev) ? nullptr : e_old;   // all-zero e is the same as none
        if ((rc = build(&gi, s, p, &t, st)) != TR_OK) return rc;
        WalkOut o;
        o.F = F_out; o.e = e_new; o.ion = ion_out;
        if ((rc = walk_run(t, nullptr, ncell, false, o, st)) != TR_OK) return rc;
        if ((rc = read_status(t, st)) != TR_OK) return rc;
        ++it;
        if ((rc = delta_compute(e_new, e_old, ncell, p->delta_mode, t->dscratch, &delta, st)) != TR_OK) return rc;
        double* tmp = e_old; e_old = e_new; e_new = tmp;
        if (delta < p->eps_lim) break;
    }
    if (e_out && (rc = cuda_check(cudaMemcpyAsync(e_out, e_old, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, st),
                                  "copy e")) != TR_OK)
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(st), "final copy")) != TR_OK) return rc;
    if (iters_out) *iters_out = it;
    if (delta_out) *delta_out = delta;
    return TR_OK;
}

tr_status tr_delta(const double* e_new, const double* e_old, int64_t n, int32_t delta_mode, double* delta_out,
                   tr_stream stream) {
    g_err[0] = '\0';
    if (!e_new || !e_old || !delta_out || n < 1) return set_error(TR_EINVAL, "bad arguments to tr_delta");
    if (delta_mode != 0 && delta_mode != 1) return set_error(TR_EINVAL, "delta_mode must be 0 or 1");
    void* scratch = nullptr;
    tr_status rc = dev_alloc((unsigned char**)&scratch, delta_scratch_bytes(), "delta state");
    if (rc != TR_OK) return rc;
    rc = delta_compute(e_new, e_old, n, delta_mode, scratch, delta_out, (cudaStream_t)stream);
    cudaFree(scratch);
    return rc;
}

tr_status tr_tree_info(const tr_tree* t, int64_t* n_nodes, int32_t* levels, int32_t* nr, int32_t* npix) {
    g_err[0] = '\0';
    if (!t) return set_error(TR_EINVAL, "tree is NULL");
    if (n_nodes) *n_nodes = t->n_nodes;
    if (levels) *levels = t->L + 1;
    if (nr) *nr = t->nr;
    if (npix) *npix = t->npix;
    return TR_OK;
}

tr_status tr_tree_flags(const tr_tree* t, uint8_t* out, tr_stream stream) {
    g_err[0] = '\0';
    if (!t || !out) return set_error(TR_EINVAL, "tree or output is NULL");
    return flags_export(t, out, (cudaStream_t)stream);
}

tr_status tr_tree_nodes(const tr_tree* t, double* out8, tr_stream stream) {
    g_err[0] = '\0';
    if (!t || !out8) return set_error(TR_EINVAL, "tree or output is NULL");
    return tree_export(t, out8, (cudaStream_t)stream);
}

tr_status tr_rays_info(const tr_rays* r, int64_t* n_targets, int32_t* npix, int32_t* nr, int32_t* acc_cap) {
    g_err[0] = '\0';
    if (!r) return set_error(TR_EINVAL, "rays is NULL");
    if (n_targets) *n_targets = r->n_targets;
    if (npix) *npix = r->npix;
    if (nr) *nr = r->nr;
    if (acc_cap) *acc_cap = r->acc_cap;
    return TR_OK;
}

tr_status tr_rays_export(const tr_rays* r, double* alpha, double* eps, double* e, int64_t* ids, int32_t* counts,
                         tr_stream stream) {
    g_err[0] = '\0';
    cudaStream_t st = (cudaStream_t)stream;
    if (!r) return set_error(TR_EINVAL, "rays is NULL");
    if (r->n_targets == 0) return TR_OK;
    const int nbins = r->npix * r->nr;
    const int64_t n = r->n_targets * nbins;
    if (alpha || eps || e)
        k_export_bins<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r->bins, r->n_targets, nbins, r->mode, r->scales,
                                                                   r->U, r->Eu, alpha, eps, e);
    if (ids) {
        const int64_t m = r->n_targets * r->acc_cap;
        k_export_ids<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(r->ids, r->counts, r->n_targets, r->acc_cap, ids);
    }
    tr_status rc = cuda_check(cudaGetLastError(), "export kernels");
    if (rc == TR_OK && counts)
        rc = cuda_check(cudaMemcpyAsync(counts, r->counts, sizeof(int32_t) * r->n_targets, cudaMemcpyDeviceToDevice, st),
                        "copy counts");
    return rc;
}

tr_status tr_table_info(int32_t nside, int32_t* nkeys, int32_t* n_entries) {
    g_err[0] = '\0';
    if (nside != 1 && nside != 2 && nside != 4 && nside != 8) return set_error(TR_EINVAL, "bad nside %d", nside);
    const Table* t = nullptr;
    tr_status rc = table_get(nside, &t, 0);
    if (rc != TR_OK) return rc;
    if (nkeys) *nkeys = NKEYS;
    if (n_entries) *n_entries = t->n_entries;
    return TR_OK;
}

tr_status tr_table_export(int32_t nside, int32_t* offsets, int32_t* pix, int32_t* cnt, tr_stream stream) {
    g_err[0] = '\0';
    if (nside != 1 && nside != 2 && nside != 4 && nside != 8) return set_error(TR_EINVAL, "bad nside %d", nside);
    cudaStream_t st = (cudaStream_t)stream;
    const Table* t = nullptr;
    tr_status rc = table_get(nside, &t, st);
    if (rc != TR_OK) return rc;
    const int n = (t->n_entries > NKEYS + 1) ? t->n_entries : NKEYS + 1;
    k_table_split<<<(n + 255) / 256, 256, 0, st>>>(t->off, t->ent, NKEYS, offsets, pix, cnt);
    return cuda_check(cudaGetLastError(), "table export kernel");
}

void tr_tree_free(tr_tree* t) { tree_release(t); }

void tr_rays_free(tr_rays* r) {
    if (!r) return;
    cudaFree(r->bins);
    cudaFree(r->ids);
    cudaFree(r->counts);
    cudaFree(r->eps_self);
    cudaFree(r->target_idx);
    cudaFree(r->scales);
    sweep_tables_free(&r->sw);
    delete r;
}

}  // extern "C"
