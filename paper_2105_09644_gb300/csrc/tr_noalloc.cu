// tr_solve_noalloc: one build + walk + sweep pass that allocates no device
// memory.  Its working memory (mapped emission, the FP64 tree and, for the
// FP32 forms, the FP32 tree beside it, build sums, status words, ray tables
// and the node->ray table) lives in one file-scope device array of fixed
// size, held by every GPU that loads the library until the process exits.
// See include/treeray.h for who needs it and its limits.
#include <cmath>
#include <mutex>

#include "tr_internal.cuh"

namespace tr {
namespace {

constexpr int NA_MAX_N = 32;                     // grids up to 32^3 cells
constexpr int NA_MAX_NSIDE = 2;                  // up to N_PIX = 48 rays
constexpr int64_t NA_NCELL = (int64_t)NA_MAX_N * NA_MAX_N * NA_MAX_N;
constexpr int64_t NA_NNODES = 37449;             // (8^6 - 1) / 7 nodes of a 32^3 octree
constexpr uint32_t NA_ENT_CAP = 1800000;         // node->ray table entries (N_side 2 needs 1,748,216)
constexpr size_t NR2 = (size_t)MAX_NR * MAX_NR;

constexpr size_t up(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_NDOT = 0;
constexpr size_t OFF_NODES = up(OFF_NDOT + sizeof(double) * NA_NCELL);          // FP64 tree
constexpr size_t OFF_SUMS = up(OFF_NODES + sizeof(NodeF64) * NA_NNODES);
constexpr size_t OFF_NODES32 = up(OFF_SUMS + 3 * sizeof(double) * NA_NNODES);   // FP32 tree (FP32 forms)
constexpr size_t OFF_SUMS32 = up(OFF_NODES32 + sizeof(NodeF32) * NA_NNODES);
constexpr size_t OFF_KAPPA = up(OFF_SUMS32 + 3 * sizeof(float) * NA_NNODES);
constexpr size_t OFF_STATUS = up(OFF_KAPPA + sizeof(float));
constexpr size_t OFF_STATS = up(OFF_STATUS + 4 * sizeof(int32_t));
constexpr size_t OFF_COUNTER = up(OFF_STATS + N_STATS * sizeof(unsigned long long));
constexpr size_t OFF_JOB = up(OFF_COUNTER + sizeof(unsigned int));
constexpr size_t JOB_BYTES = 1024;                // one walk job record (checked at run time)
constexpr size_t OFF_R = up(OFF_JOB + JOB_BYTES);
constexpr size_t OFF_RF = up(OFF_R + sizeof(double) * MAX_NR);
constexpr size_t OFF_INVR2 = up(OFF_RF + sizeof(float) * MAX_NR);
constexpr size_t OFF_INVVOL = up(OFF_INVR2 + sizeof(double) * MAX_NR);
constexpr size_t OFF_INVVOLF = up(OFF_INVVOL + sizeof(double) * MAX_NR);
constexpr size_t OFF_G = up(OFF_INVVOLF + sizeof(float) * MAX_NR);
constexpr size_t OFF_ID2 = up(OFF_G + sizeof(double) * NR2);
constexpr size_t OFF_GI = up(OFF_ID2 + sizeof(double) * NR2);
constexpr size_t OFF_GF = up(OFF_GI + sizeof(double) * NR2);
constexpr size_t OFF_ID2F = up(OFF_GF + sizeof(float) * NR2);
constexpr size_t OFF_GIF = up(OFF_ID2F + sizeof(float) * NR2);
constexpr size_t OFF_HT = up(OFF_GIF + sizeof(float) * NR2);
constexpr size_t OFF_TCOUNTS = up(OFF_HT + sizeof(double) * NR2);
constexpr size_t OFF_TOFF = up(OFF_TCOUNTS + sizeof(uint32_t) * NKEYS);
constexpr size_t OFF_THDR = up(OFF_TOFF + sizeof(uint32_t) * (NKEYS + 1));
constexpr size_t OFF_TENT = up(OFF_THDR + sizeof(uint2) * NKEYS);
constexpr size_t NA_BYTES = up(OFF_TENT + sizeof(uint32_t) * NA_ENT_CAP);   // about 18 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr double C_LIGHT = 2.99792458e10;
constexpr int NA_MAX_DEVICES = 64;
static_assert(NA_BYTES < (24u << 20), "the fixed working memory stays modest");

struct DeviceState {
    bool ready = false;                          // symbol address resolved on this device
    unsigned char* base = nullptr;               // device address of g_noalloc_scratch
    Table table;                                 // node->ray table inside the array
    bool table_ok = false;
    SweepTables sw;                              // ray tables inside the array
    bool sw_ok = false;
};

std::mutex g_mu;
DeviceState g_state[NA_MAX_DEVICES];

template <typename T>
T* at(unsigned char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

}  // namespace
}  // namespace tr

using namespace tr;

extern "C" tr_status tr_solve_noalloc(const tr_grid* g, const tr_sources* s, const tr_params* p, double* F_out,
                                      double* e_out, uint8_t* ion_out, tr_stream stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    // the checks of tr_solve, then the limits of the fixed working memory
    tr_status rc0 = check_params(p);
    if (rc0 == TR_OK) rc0 = check_grid(g, s);
    if (rc0 != TR_OK) return rc0;
    if (g->N > NA_MAX_N)
        return set_error(TR_EUNSUPPORTED, "tr_solve_noalloc holds grids up to %d^3 cells in its fixed scratch (got %d^3)",
                         NA_MAX_N, g->N);
    if (p->nside > NA_MAX_NSIDE)
        return set_error(TR_EUNSUPPORTED, "tr_solve_noalloc supports N_side 1 or 2 (got %d)", p->nside);
    if (p->max_iter != 1) return set_error(TR_EUNSUPPORTED, "tr_solve_noalloc runs one pass (max_iter = 1)");
    const int N = g->N;
    int L = 0;
    while ((1 << L) < N) ++L;
    const double lray = p->L_ray_cm > 0.0 ? p->L_ray_cm / g->dx : default_lray(N, p);
    const int nr = p->eta_r * (int)std::floor(std::sqrt(2.0 * lray)) + 1;     // Eq. 5
    if (nr > MAX_NR || nr < 3) return set_error(TR_EUNSUPPORTED, "N_R = %d outside [3, %d]", nr, MAX_NR);

    int dev = 0;
    tr_status rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc != TR_OK) return rc;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(TR_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState& ds = g_state[dev];
    if (!ds.ready) {
        // first call on this device: the host-side name of the array is not a
        // device address, so ask the runtime for it (this device is current)
        void* ptr = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)");
        if (rc != TR_OK) return rc;
        ds.base = static_cast<unsigned char*>(ptr);
        ds.table.off = at<uint32_t>(ds.base, OFF_TOFF);
        ds.table.ent = at<uint32_t>(ds.base, OFF_TENT);
        ds.table.hdr = at<uint2>(ds.base, OFF_THDR);
        ds.sw.r = at<double>(ds.base, OFF_R);
        ds.sw.rf = at<float>(ds.base, OFF_RF);
        ds.sw.inv_r2 = at<double>(ds.base, OFF_INVR2);
        ds.sw.inv_vol = at<double>(ds.base, OFF_INVVOL);
        ds.sw.inv_volf = at<float>(ds.base, OFF_INVVOLF);
        ds.sw.G = at<double>(ds.base, OFF_G);
        ds.sw.ID2 = at<double>(ds.base, OFF_ID2);
        ds.sw.GI = at<double>(ds.base, OFF_GI);
        ds.sw.Gf = at<float>(ds.base, OFF_GF);
        ds.sw.ID2f = at<float>(ds.base, OFF_ID2F);
        ds.sw.GIf = at<float>(ds.base, OFF_GIF);
        ds.sw.HT = at<double>(ds.base, OFF_HT);
        ds.ready = true;
    }
    if (!ds.table_ok || ds.table.nside != p->nside) {
        ds.table_ok = false;
        rc = table_build_into(p->nside, &ds.table, at<uint32_t>(ds.base, OFF_TCOUNTS), NA_ENT_CAP, st);
        if (rc != TR_OK) return rc;
        ds.table_ok = true;
    }
    const int npix = 12 * p->nside * p->nside;
    const int zg = p->zeta_g ? 1 : 0;
    if (!ds.sw_ok || ds.sw.nr != nr || ds.sw.eta != p->eta_r || ds.sw.nside != p->nside || ds.sw.zeta_g != zg) {
        ds.sw_ok = false;
        rc = sweep_tables_fill(&ds.sw, nr, p->eta_r, p->nside, npix, zg, st);
        if (rc != TR_OK) return rc;
        ds.sw_ok = true;
    }
    // a tree whose storage is the fixed array; nothing here is allocated or freed
    tr_tree t;
    t.device = dev;
    t.N = N; t.L = L; t.mode = p->precision;
    t.n_nodes = level_offset(L + 1);
    t.n_cells = NA_NCELL < (int64_t)N * N * N ? NA_NCELL : (int64_t)N * N * N;
    t.nodes64 = ds.base + OFF_NODES;
    t.sums64 = ds.base + OFF_SUMS;
    if (t.mode == 0) {
        t.nodes = t.nodes64;
        t.sums = t.sums64;
    } else {
        t.nodes = ds.base + OFF_NODES32;
        t.sums = ds.base + OFF_SUMS32;
        t.kappa = at<float>(ds.base, OFF_KAPPA);
    }
    t.ndot = at<double>(ds.base, OFF_NDOT);
    t.status = at<int32_t>(ds.base, OFF_STATUS);
    t.stats = at<unsigned long long>(ds.base, OFF_STATS);
    t.counter = at<unsigned int>(ds.base, OFF_COUNTER);
    if (walk_job_bytes(1) > JOB_BYTES) return set_error(TR_EUNSUPPORTED, "walk job record larger than its slot");
    t.jobbuf = ds.base + OFF_JOB;
    t.table = &ds.table;
    t.sw = ds.sw;
    t.p = *p;
    t.use_e = g->e_prev != nullptr;
    t.nr = nr;
    t.npix = npix;
    for (int a = 0; a < 3; ++a) t.box_lo[a] = g->box_lo[a];
    t.dx = g->dx;
    t.U = p->alpha_B * g->dx * g->dx * g->dx;
    t.Eu = p->alpha_B * g->dx * p->hnu / C_LIGHT;
    t.lray = lray;
    if ((rc = tree_build(&t, g, s, st)) != TR_OK) return rc;
    WalkOut o;
    o.F = F_out; o.e = e_out; o.ion = ion_out;
    if ((rc = walk_run(&t, nullptr, (int64_t)N * N * N, false, o, st)) != TR_OK) return rc;
    return read_status(&t, st);
}
