// Octree build (Sec. 2.1, Eq. 1-3) with source mapping (Sec. 2.7), and the
// per-ray constant tables of the sweep (Eq. 4, 15, 16).
//
// Layout: nodes of all levels in one array, level-order, Morton order inside
// a level: node (l, m) has id (8^l - 1)/7 + m and children 8m + c at l + 1
// (c = x | y << 1 | z << 2), so the eight children of a node are contiguous.
// Leaves are the cells (level L = log2 N).  Parents are reduced from their
// children in child order c = 0..7: plain FP64 sums, or FP32
// Kahan-Neumaier (compensated) sums.  The FP32 record keeps the centre of
// mass as its offset from the node's geometric centre (first moments are
// summed about each parent's centre), and the FP32 forms build the FP64 tree
// beside it: the walk settles in FP64 the rare comparisons that FP32 cannot
// (a bound kappa on the FP32 centre-of-mass error, per unit of node edge, is
// measured here against the FP64 tree), and the IF flag of each node is
// decided on the FP64 masses.
#include "tr_internal.cuh"

namespace tr {
namespace {

__global__ void k_ndot_init(double* ndot, const double* ndot_in, int64_t n) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < n) ndot[c] = ndot_in ? ndot_in[c] : 0.0;
}

// Point sources go to the cell that contains them (radius 0), clamped to the box.
__global__ void k_map_sources(double* ndot, int N, double lo0, double lo1, double lo2, double dx,
                              const double* xyz, const double* Q, int n) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double lo[3] = {lo0, lo1, lo2};
    int64_t ic[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(__ddiv_rn(__dsub_rn(xyz[3 * s + a], lo[a]), dx));
        f = fmin(fmax(f, 0.0), (double)(N - 1));
        ic[a] = (int64_t)f;
    }
    atomicAdd(&ndot[(ic[2] * N + ic[1]) * N + ic[0]], Q[s]);
}

struct F32Sum {                              // Kahan-Neumaier accumulator
    float s = 0.f, c = 0.f;
    __device__ void add(float x) {
        float t = s + x;
        if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ float value() const { return s + c; }
};

// Leaves (cells): netting of Eq. 1-2 per cell, e of Eq. 3, ionised mass.
template <int MODE>
__global__ void k_leaves(void* nodes_v, void* sums_v, int N, int L, const double* n_H,
                         const double* ndot, const double* e_prev, double invU, double invEu) {
    const int64_t nleaf = (int64_t)N * N * N;
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= nleaf) return;
    const uint32_t ix = compact3((uint32_t)m), iy = compact3((uint32_t)m >> 1), iz = compact3((uint32_t)m >> 2);
    const int64_t c = ((int64_t)iz * N + iy) * N + ix;
    const int64_t id = level_offset(L) + m;
    const double n = n_H[c];
    const double rec = n * n;                       // alpha_B n^2 dV in units of U
    const double src = ndot[c] * invU;
    const double ep = e_prev ? e_prev[c] : 0.0;
    if (MODE == 0) {
        NodeF64 nd;
        nd.m = n;
        double sx = __dmul_rn(n, (double)ix + 0.5), sy = __dmul_rn(n, (double)iy + 0.5),
               sz = __dmul_rn(n, (double)iz + 0.5);
        if (n > 0.0) { nd.cmx = __ddiv_rn(sx, n); nd.cmy = __ddiv_rn(sy, n); nd.cmz = __ddiv_rn(sz, n); }
        else { nd.cmx = (double)ix + 0.5; nd.cmy = (double)iy + 0.5; nd.cmz = (double)iz + 0.5; }
        nd.alpha = fmax(rec - src, 0.0);
        nd.eps = fmax(src - rec, 0.0);
        nd.e = ep * invEu;
        nd.mion = (ep > 0.0) ? n : 0.0;
        ((NodeF64*)nodes_v)[id] = nd;
        double* sm = (double*)sums_v + 3 * id;
        sm[0] = sx; sm[1] = sy; sm[2] = sz;
    } else {
        NodeF32 nd;                                 // a cell's mass sits at its centre: offset 0
        const float nf = (float)n;
        nd.m = nf;
        nd.ox = 0.f; nd.oy = 0.f; nd.oz = 0.f;
        nd.alpha = (float)fmax(rec - src, 0.0);
        nd.eps = (float)fmax(src - rec, 0.0);
        nd.e = (float)(ep * invEu);
        nd.mion = (ep > 0.0) ? nf : 0.f;
        ((NodeF32*)nodes_v)[id] = nd;
        float* sm = (float*)sums_v + 3 * id;
        sm[0] = 0.f; sm[1] = 0.f; sm[2] = 0.f;
    }
}

// ---- AMR grids: blocks of 8^3 cells, cells of edge N >> level ------------

// Topology: every cell of a block is a leaf; the 64 + 8 + 1 nodes above the
// cells inside the block and every ancestor of the block are parents (many
// blocks store the same byte into a shared ancestor).  The block's own node
// also records the block index, so a cell can be found from its position.
__global__ void k_amr_topology(uint8_t* flags, int32_t* blkmap, const int4* blk, int n_blocks) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_blocks * 512) return;
    const int b = (int)(i >> 9), c = (int)(i & 511);
    const int4 bm = blk[b];
    const int tl = bm.x;
    const uint32_t bx = (uint32_t)bm.y, by = (uint32_t)bm.z, bz = (uint32_t)bm.w;
    flags[level_offset(tl) + morton3(8 * bx + (c & 7), 8 * by + ((c >> 3) & 7), 8 * bz + (c >> 6))] = NODE_LEAF;
    if (c < 64) {
        flags[level_offset(tl - 1) + morton3(4 * bx + (c & 3), 4 * by + ((c >> 2) & 3), 4 * bz + (c >> 4))] = NODE_PARENT;
    } else if (c < 72) {
        const int k = c - 64;
        flags[level_offset(tl - 2) + morton3(2 * bx + (k & 1), 2 * by + ((k >> 1) & 1), 2 * bz + (k >> 2))] = NODE_PARENT;
    } else if (c == 72) {
        const int64_t id = level_offset(tl - 3) + morton3(bx, by, bz);
        flags[id] = NODE_PARENT;
        blkmap[id] = b;
    } else if (c - 73 < tl - 3) {
        const int l = tl - 4 - (c - 73), sh = tl - 3 - l;
        flags[level_offset(l) + morton3(bx >> sh, by >> sh, bz >> sh)] = NODE_PARENT;
    }
}

// Point sources go to the cell containing their finest-lattice cell: the
// first leaf on the way down from the root.
__global__ void k_amr_map_sources(double* ndot, const uint8_t* flags, const int32_t* blkmap, int N, int L,
                                  double lo0, double lo1, double lo2, double dx, const double* xyz, const double* Q,
                                  int n) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double lo[3] = {lo0, lo1, lo2};
    uint32_t f[3];
    for (int a = 0; a < 3; ++a) {
        double v = floor(__ddiv_rn(__dsub_rn(xyz[3 * s + a], lo[a]), dx));
        v = fmin(fmax(v, 0.0), (double)(N - 1));
        f[a] = (uint32_t)v;
    }
    for (int l = 3; l <= L; ++l) {                   // a cell lies at level >= 3 (N_base >= 8)
        const int sh = L - l;
        const uint32_t x = f[0] >> sh, y = f[1] >> sh, z = f[2] >> sh;
        if (flags[level_offset(l) + morton3(x, y, z)] == NODE_LEAF) {
            const int b = blkmap[level_offset(l - 3) + morton3(x >> 3, y >> 3, z >> 3)];
            const int64_t cell = ((int64_t)b << 9) + (int64_t)(((z & 7) * 8 + (y & 7)) * 8 + (x & 7));
            atomicAdd(&ndot[cell], Q[s]);
            return;
        }
    }
}

// AMR cells: Eq. 1-3 for a cell of edge s (volume s^3 finest cells), stored
// at its own level of the finest-lattice octree.
template <int MODE>
__global__ void k_amr_leaves(void* nodes_v, void* sums_v, int N, const int4* blk, int n_blocks, const double* n_H,
                             const double* ndot, const double* e_prev, double invU, double invEu) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_blocks * 512) return;
    const int b = (int)(i >> 9), c = (int)(i & 511);
    const int4 bm = blk[b];
    const int tl = bm.x;
    const uint32_t ix = 8 * (uint32_t)bm.y + (c & 7), iy = 8 * (uint32_t)bm.z + ((c >> 3) & 7),
                   iz = 8 * (uint32_t)bm.w + (c >> 6);
    const int64_t id = level_offset(tl) + morton3(ix, iy, iz);
    const double s = (double)(N >> tl), vol = s * s * s;
    const double n = n_H[i];
    const double rec = n * n * vol;                  // alpha_B n^2 dV in units of U
    const double src = ndot[i] * invU;
    const double ep = e_prev ? e_prev[i] : 0.0;
    const double px = ((double)ix + 0.5) * s, py = ((double)iy + 0.5) * s, pz = ((double)iz + 0.5) * s;
    if (MODE == 0) {
        NodeF64 nd;
        nd.m = __dmul_rn(n, vol);
        const double sx = __dmul_rn(nd.m, px), sy = __dmul_rn(nd.m, py), sz = __dmul_rn(nd.m, pz);
        if (nd.m > 0.0) { nd.cmx = __ddiv_rn(sx, nd.m); nd.cmy = __ddiv_rn(sy, nd.m); nd.cmz = __ddiv_rn(sz, nd.m); }
        else { nd.cmx = px; nd.cmy = py; nd.cmz = pz; }
        nd.alpha = fmax(rec - src, 0.0);
        nd.eps = fmax(src - rec, 0.0);
        nd.e = ep * invEu * vol;
        nd.mion = (ep > 0.0) ? nd.m : 0.0;
        ((NodeF64*)nodes_v)[id] = nd;
        double* sm = (double*)sums_v + 3 * id;
        sm[0] = sx; sm[1] = sy; sm[2] = sz;
    } else {
        NodeF32 nd;                                 // offset 0 from the cell's centre
        const float mf = (float)(n * vol);
        nd.m = mf;
        nd.ox = 0.f; nd.oy = 0.f; nd.oz = 0.f;
        nd.alpha = (float)fmax(rec - src, 0.0);
        nd.eps = (float)fmax(src - rec, 0.0);
        nd.e = (float)(ep * invEu * vol);
        nd.mion = (ep > 0.0) ? mf : 0.f;
        ((NodeF32*)nodes_v)[id] = nd;
        float* sm = (float*)sums_v + 3 * id;
        sm[0] = 0.f; sm[1] = 0.f; sm[2] = 0.f;
    }
}

// One level of parents from their eight contiguous children (on an AMR
// tree only the nodes flagged as parents).
template <int MODE>
__global__ void k_parents(void* nodes_v, void* sums_v, int l, int N, const uint8_t* flags) {
    const int64_t nl = int64_t(1) << (3 * l);
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= nl) return;
    const int64_t id = level_offset(l) + m;
    if (flags && flags[id] != NODE_PARENT) return;
    const int64_t ch = level_offset(l + 1) + 8 * m;
    const uint32_t ix = compact3((uint32_t)m), iy = compact3((uint32_t)m >> 1), iz = compact3((uint32_t)m >> 2);
    const double s = (double)(N >> l);
    if (MODE == 0) {
        const NodeF64* c = (const NodeF64*)nodes_v + ch;
        const double* cs = (const double*)sums_v + 3 * ch;
        NodeF64 p = c[0];
        double sx = cs[0], sy = cs[1], sz = cs[2];
        for (int k = 1; k < 8; ++k) {
            const NodeF64 q = c[k];
            p.m = __dadd_rn(p.m, q.m);
            sx = __dadd_rn(sx, cs[3 * k + 0]);
            sy = __dadd_rn(sy, cs[3 * k + 1]);
            sz = __dadd_rn(sz, cs[3 * k + 2]);
            p.alpha = __dadd_rn(p.alpha, q.alpha);
            p.eps = __dadd_rn(p.eps, q.eps);
            p.e = __dadd_rn(p.e, q.e);
            p.mion = __dadd_rn(p.mion, q.mion);
        }
        if (p.m > 0.0) { p.cmx = __ddiv_rn(sx, p.m); p.cmy = __ddiv_rn(sy, p.m); p.cmz = __ddiv_rn(sz, p.m); }
        else { p.cmx = ((double)ix + 0.5) * s; p.cmy = ((double)iy + 0.5) * s; p.cmz = ((double)iz + 0.5) * s; }
        ((NodeF64*)nodes_v)[id] = p;
        double* ps = (double*)sums_v + 3 * id;
        ps[0] = sx; ps[1] = sy; ps[2] = sz;
    } else {
        // first moments about this node's centre: each child's own, plus its
        // mass times the offset of its centre, +-s/4 per axis (a power of
        // two, so the product is exact)
        const NodeF32* c = (const NodeF32*)nodes_v + ch;
        const float* cs = (const float*)sums_v + 3 * ch;
        const float q4 = 0.25f * (float)s;
        F32Sum m_, sx, sy, sz, al, ep, ee, mi;
        for (int k = 0; k < 8; ++k) {
            const NodeF32 q = c[k];
            const float mq = q.m * q4;
            m_.add(q.m); al.add(q.alpha); ep.add(q.eps); ee.add(q.e); mi.add(q.mion);
            sx.add(cs[3 * k + 0]); sx.add((k & 1) ? mq : -mq);
            sy.add(cs[3 * k + 1]); sy.add((k & 2) ? mq : -mq);
            sz.add(cs[3 * k + 2]); sz.add((k & 4) ? mq : -mq);
        }
        NodeF32 p;
        p.m = m_.value(); p.alpha = al.value(); p.eps = ep.value(); p.e = ee.value(); p.mion = mi.value();
        const float fx = sx.value(), fy = sy.value(), fz = sz.value();
        if (p.m > 0.f) { p.ox = fx / p.m; p.oy = fy / p.m; p.oz = fz / p.m; }
        else { p.ox = 0.f; p.oy = 0.f; p.oz = 0.f; }           // no mass: the geometric centre
        ((NodeF32*)nodes_v)[id] = p;
        float* ps = (float*)sums_v + 3 * id;
        ps[0] = fx; ps[1] = fy; ps[2] = fz;
    }
}

// Level of node `id` in the level-order numbering.
__device__ __forceinline__ int node_level(int64_t id) {
    int l = 0;
    while (level_offset(l + 1) <= id) ++l;
    return l;
}

// FP32 forms, after both builds: the IF flag of every node (Sec. 2.4,
// delta_IF m < m_ion < (1 - delta_IF) m on the FP64 masses, as the FP64 walk
// decides it) goes into the sign bit of the FP32 m_ion, and kappa =
// max |cm32 - cm64| / edge over the nodes that exist (rounded up).
__global__ void k_finalize(NodeF32* nodes, const NodeF64* nodes64, const uint8_t* flags, int64_t n, int N,
                           float* kappa) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float kap = 0.f;
    if (i < n && !(flags && flags[i] == NODE_ABSENT)) {
        const NodeF64 q = nodes64[i];
        NodeF32& f = nodes[i];
        const int l = node_level(i);
        const uint32_t m = (uint32_t)(i - level_offset(l));
        const double s = (double)(N >> l);
        const double gx = ((double)compact3(m) + 0.5) * s, gy = ((double)compact3(m >> 1) + 0.5) * s,
                     gz = ((double)compact3(m >> 2) + 0.5) * s;
        const double ex = fabs(gx + (double)f.ox - q.cmx), ey = fabs(gy + (double)f.oy - q.cmy),
                     ez = fabs(gz + (double)f.oz - q.cmz);
        kap = __double2float_ru(fmax(ex, fmax(ey, ez)) / s);
        const bool is_if = (__dmul_rn(DELTA_IF, q.m) < q.mion) && (q.mion < __dmul_rn(1.0 - DELTA_IF, q.m));
        f.mion = is_if ? -fabsf(f.mion) : fabsf(f.mion);
    }
    for (int o = 16; o > 0; o >>= 1) kap = fmaxf(kap, __shfl_xor_sync(0xffffffffu, kap, o));
    if ((threadIdx.x & 31) == 0 && kap > 0.f) atomicMax(reinterpret_cast<unsigned int*>(kappa), __float_as_uint(kap));
}

template <int MODE>
__global__ void k_export(const void* nodes_v, int64_t n, double* out, double U, double Eu, int N, const uint8_t* flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[8];
    if (MODE == 0) {
        NodeF64 q = ((const NodeF64*)nodes_v)[i];
        v[0] = q.m; v[1] = q.cmx; v[2] = q.cmy; v[3] = q.cmz;
        v[4] = q.alpha; v[5] = q.eps; v[6] = q.e; v[7] = q.mion;
    } else {                                       // centre of mass = geometric centre + offset
        NodeF32 q = ((const NodeF32*)nodes_v)[i];
        const bool absent = flags && flags[i] == NODE_ABSENT;
        const int l = node_level(i);
        const uint32_t m = (uint32_t)(i - level_offset(l));
        const double s = (double)(N >> l);
        v[0] = q.m;
        v[1] = absent ? 0.0 : ((double)compact3(m) + 0.5) * s + (double)q.ox;
        v[2] = absent ? 0.0 : ((double)compact3(m >> 1) + 0.5) * s + (double)q.oy;
        v[3] = absent ? 0.0 : ((double)compact3(m >> 2) + 0.5) * s + (double)q.oz;
        v[4] = q.alpha; v[5] = q.eps; v[6] = q.e; v[7] = fabsf(q.mion);
    }
    v[4] *= U; v[5] *= U; v[6] *= Eu;
    for (int k = 0; k < 8; ++k) out[8 * i + k] = v[k];
}

// Ray constants: r_i (Eq. 4), ray-cell volumes, and for each segment i and
// source point j > i the loss geometry (1/2) dV_ij zeta_g,ij (Eq. 14-16: the
// 1/2 of the segment's mean coefficient, so that a sweep multiplies it by
// alpha_i + alpha_{i+1}) and the inverse square distance from j to the
// segment midpoint.  HT[j][i] = (G_{i-1,j} + G_{i,j}) / V_i: the weight of
// point i's raw recombination deposit in the total loss of a lone source at
// j (Eq. 13-14 with zeta_s = zeta_d = 1, the volume V_i of the ray cell
// folded in), so that the total is sum_i bin_i HT[j][i].
__device__ __forceinline__ double seg_geom(int i, int j, int nr, int eta, int nside, int zeta_g) {
    if (!(j > i && i + 1 < nr && i >= 0)) return 0.0;
    auto rad = [eta](int k) { return (double)((int64_t)k * k) / (2.0 * (double)eta * (double)eta); };
    const double ri = rad(i), ri1 = rad(i + 1), rj = rad(j);
    const double a = rj - ri, b = rj - ri1;
    const double dV = (a * a * a - b * b * b) / 3.0;
    const double zg = zeta_g ? fmin(1.0, (double)nside * (rj - ri) / (2.0 * rj)) : 1.0;
    return 0.5 * dV * zg;
}

__global__ void k_sweep_tables(int nr, int eta, int nside, int npix, int zeta_g, double* r, float* rf,
                               double* inv_r2, double* inv_vol, float* inv_volf, double* G, double* ID2, double* GI,
                               float* Gf, float* ID2f, float* GIf, double* HT) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    auto rad = [eta](int i) { return (double)((int64_t)i * i) / (2.0 * (double)eta * (double)eta); };
    if (t < nr) {
        const int i = t;
        const double ri = rad(i);
        r[i] = ri;
        rf[i] = (float)ri;
        inv_r2[i] = (i > 0) ? 1.0 / (ri * ri) : 0.0;
        const double lo = (i == 0) ? 0.0 : 0.5 * (rad(i - 1) + ri);
        const double hi = (i == nr - 1) ? ri : 0.5 * (ri + rad(i + 1));
        inv_vol[i] = 1.0 / ((4.0 * PI_D / (double)npix) * (hi * hi * hi - lo * lo * lo) / 3.0);
        inv_volf[i] = (float)inv_vol[i];
    }
    if (t < nr * nr) {
        const int i = t / nr, j = t % nr;
        const double g = seg_geom(i, j, nr, eta, nside, zeta_g);
        double id2 = 0.0;
        if (j > i && i + 1 < nr) {
            const double rm = 0.5 * (rad(i) + rad(i + 1)), rj = rad(j);
            id2 = 1.0 / ((rj - rm) * (rj - rm));
        }
        G[t] = g;
        ID2[t] = id2;
        GI[t] = g * id2;
        Gf[t] = (float)g;
        ID2f[t] = (float)id2;
        GIf[t] = (float)(g * id2);
        const int jj = t / nr, ii = t % nr;                 // HT is indexed [j][i]
        const double lo = (ii == 0) ? 0.0 : 0.5 * (rad(ii - 1) + rad(ii));
        const double hi = (ii == nr - 1) ? rad(ii) : 0.5 * (rad(ii) + rad(ii + 1));
        const double vol = (4.0 * PI_D / (double)npix) * (hi * hi * hi - lo * lo * lo) / 3.0;
        HT[t] = (seg_geom(ii - 1, jj, nr, eta, nside, zeta_g) + seg_geom(ii, jj, nr, eta, nside, zeta_g)) / vol;
    }
}

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_uniform_flags(uint8_t* out, int64_t n, int64_t first_leaf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = i >= first_leaf ? NODE_LEAF : NODE_PARENT;
}

}  // namespace

tr_status sweep_tables_make(SweepTables* sw, int nr, int eta, int nside, int npix, int zeta_g,
                            cudaStream_t st) {
    if (sw->r && sw->nr == nr && sw->eta == eta && sw->nside == nside && sw->zeta_g == zeta_g) return TR_OK;
    sweep_tables_free(sw);
    const size_t n2 = (size_t)nr * nr;
    tr_status s = TR_OK;
    if (cudaMalloc(&sw->r, sizeof(double) * nr) != cudaSuccess ||
        cudaMalloc(&sw->rf, sizeof(float) * nr) != cudaSuccess ||
        cudaMalloc(&sw->inv_r2, sizeof(double) * nr) != cudaSuccess ||
        cudaMalloc(&sw->inv_vol, sizeof(double) * nr) != cudaSuccess ||
        cudaMalloc(&sw->inv_volf, sizeof(float) * nr) != cudaSuccess ||
        cudaMalloc(&sw->G, sizeof(double) * n2) != cudaSuccess ||
        cudaMalloc(&sw->ID2, sizeof(double) * n2) != cudaSuccess ||
        cudaMalloc(&sw->GI, sizeof(double) * n2) != cudaSuccess ||
        cudaMalloc(&sw->Gf, sizeof(float) * n2) != cudaSuccess ||
        cudaMalloc(&sw->ID2f, sizeof(float) * n2) != cudaSuccess ||
        cudaMalloc(&sw->GIf, sizeof(float) * n2) != cudaSuccess ||
        cudaMalloc(&sw->HT, sizeof(double) * n2) != cudaSuccess) {
        cudaGetLastError();
        sweep_tables_free(sw);
        return set_error(TR_ENOMEM, "cannot allocate the ray tables (N_R = %d)", nr);
    }
    k_sweep_tables<<<grid_for((int64_t)n2, 128), 128, 0, st>>>(nr, eta, nside, npix, zeta_g, sw->r, sw->rf,
                                                                sw->inv_r2, sw->inv_vol, sw->inv_volf, sw->G, sw->ID2, sw->GI,
                                                                sw->Gf, sw->ID2f, sw->GIf, sw->HT);
    s = cuda_check(cudaGetLastError(), "ray table kernel");
    if (s != TR_OK) return s;
    sw->nr = nr; sw->eta = eta; sw->nside = nside; sw->zeta_g = zeta_g;
    return TR_OK;
}

tr_status sweep_tables_fill(SweepTables* sw, int nr, int eta, int nside, int npix, int zeta_g, cudaStream_t st) {
    const size_t n2 = (size_t)nr * nr;
    k_sweep_tables<<<grid_for((int64_t)n2, 128), 128, 0, st>>>(nr, eta, nside, npix, zeta_g, sw->r, sw->rf,
                                                                sw->inv_r2, sw->inv_vol, sw->inv_volf, sw->G, sw->ID2,
                                                                sw->GI, sw->Gf, sw->ID2f, sw->GIf, sw->HT);
    tr_status s = cuda_check(cudaGetLastError(), "ray table kernel");
    if (s != TR_OK) return s;
    sw->nr = nr; sw->eta = eta; sw->nside = nside; sw->zeta_g = zeta_g;
    return TR_OK;
}

void sweep_tables_free(SweepTables* sw) {
    cudaFree(sw->r); cudaFree(sw->rf); cudaFree(sw->inv_r2); cudaFree(sw->inv_vol); cudaFree(sw->inv_volf);
    cudaFree(sw->G); cudaFree(sw->ID2); cudaFree(sw->GI); cudaFree(sw->Gf); cudaFree(sw->ID2f); cudaFree(sw->GIf);
    cudaFree(sw->HT);
    *sw = SweepTables();
}

tr_status finalize_f32(tr_tree* t, cudaStream_t st) {
    tr_status rc = cuda_check(cudaMemsetAsync(t->kappa, 0, sizeof(float), st), "clear kappa");
    if (rc != TR_OK) return rc;
    k_finalize<<<grid_for(t->n_nodes, 256), 256, 0, st>>>((NodeF32*)t->nodes, (const NodeF64*)t->nodes64, t->flags,
                                                          t->n_nodes, t->N, t->kappa);
    return cuda_check(cudaGetLastError(), "FP32 tree finalize kernel");
}

tr_status tree_build(tr_tree* t, const tr_grid* g, const tr_sources* s, cudaStream_t st) {
    const int64_t ncell = (int64_t)t->N * t->N * t->N;
    const double invU = 1.0 / t->U, invEu = 1.0 / t->Eu;
    k_ndot_init<<<grid_for(ncell, 256), 256, 0, st>>>(t->ndot, g->ndot, ncell);
    if (s && s->n > 0)
        k_map_sources<<<grid_for(s->n, 128), 128, 0, st>>>(t->ndot, t->N, g->box_lo[0], g->box_lo[1],
                                                           g->box_lo[2], g->dx, s->xyz, s->Q, s->n);
    // the FP64 tree (the whole tree in mode 0, the sidecar of the FP32 forms)
    k_leaves<0><<<grid_for(ncell, 256), 256, 0, st>>>(t->nodes64, t->sums64, t->N, t->L, g->n_H, t->ndot,
                                                     g->e_prev, invU, invEu);
    for (int l = t->L - 1; l >= 0; --l) {
        const int64_t nl = int64_t(1) << (3 * l);
        k_parents<0><<<grid_for(nl, 128), 128, 0, st>>>(t->nodes64, t->sums64, l, t->N, nullptr);
    }
    if (t->mode != 0) {
        k_leaves<1><<<grid_for(ncell, 256), 256, 0, st>>>(t->nodes, t->sums, t->N, t->L, g->n_H, t->ndot,
                                                         g->e_prev, invU, invEu);
        for (int l = t->L - 1; l >= 0; --l) {
            const int64_t nl = int64_t(1) << (3 * l);
            k_parents<1><<<grid_for(nl, 128), 128, 0, st>>>(t->nodes, t->sums, l, t->N, nullptr);
        }
        tr_status rc = finalize_f32(t, st);
        if (rc != TR_OK) return rc;
    }
    return cuda_check(cudaGetLastError(), "tree build kernels");
}

tr_status amr_topology(tr_tree* t, cudaStream_t st) {
    tr_status rc = cuda_check(cudaMemsetAsync(t->flags, 0, (size_t)t->n_nodes, st), "clear flags");
    if (rc == TR_OK)
        rc = cuda_check(cudaMemsetAsync(t->blkmap, 0xff, sizeof(int32_t) * (size_t)level_offset(t->L - 2), st),
                        "clear block map");
    if (rc != TR_OK) return rc;
    k_amr_topology<<<grid_for(t->n_cells, 256), 256, 0, st>>>(t->flags, t->blkmap, t->blk, t->n_blocks);
    return cuda_check(cudaGetLastError(), "topology kernel");
}

tr_status tree_build_amr(tr_tree* t, const double* n_H, const double* ndot, const double* e_prev,
                         const tr_sources* s, cudaStream_t st) {
    const int64_t ncell = t->n_cells;
    const double invU = 1.0 / t->U, invEu = 1.0 / t->Eu;
    // nodes inside a cell are never written by the build: keep them zero
    tr_status rc = cuda_check(cudaMemsetAsync(t->nodes, 0, t->nodes_bytes, st), "clear nodes");
    if (rc == TR_OK && t->nodes64 != t->nodes)
        rc = cuda_check(cudaMemsetAsync(t->nodes64, 0, sizeof(NodeF64) * (size_t)t->n_nodes, st), "clear FP64 nodes");
    if (rc != TR_OK) return rc;
    k_ndot_init<<<grid_for(ncell, 256), 256, 0, st>>>(t->ndot, ndot, ncell);
    if (s && s->n > 0)
        k_amr_map_sources<<<grid_for(s->n, 128), 128, 0, st>>>(t->ndot, t->flags, t->blkmap, t->N, t->L, t->box_lo[0],
                                                               t->box_lo[1], t->box_lo[2], t->dx, s->xyz, s->Q, s->n);
    k_amr_leaves<0><<<grid_for(ncell, 256), 256, 0, st>>>(t->nodes64, t->sums64, t->N, t->blk, t->n_blocks, n_H,
                                                         t->ndot, e_prev, invU, invEu);
    for (int l = t->L - 1; l >= 0; --l) {
        const int64_t nl = int64_t(1) << (3 * l);
        k_parents<0><<<grid_for(nl, 128), 128, 0, st>>>(t->nodes64, t->sums64, l, t->N, t->flags);
    }
    if (t->mode != 0) {
        k_amr_leaves<1><<<grid_for(ncell, 256), 256, 0, st>>>(t->nodes, t->sums, t->N, t->blk, t->n_blocks, n_H,
                                                             t->ndot, e_prev, invU, invEu);
        for (int l = t->L - 1; l >= 0; --l) {
            const int64_t nl = int64_t(1) << (3 * l);
            k_parents<1><<<grid_for(nl, 128), 128, 0, st>>>(t->nodes, t->sums, l, t->N, t->flags);
        }
        tr_status rc2 = finalize_f32(t, st);
        if (rc2 != TR_OK) return rc2;
    }
    return cuda_check(cudaGetLastError(), "AMR tree build kernels");
}

tr_status flags_export(const tr_tree* t, uint8_t* out, cudaStream_t st) {
    if (t->flags)
        return cuda_check(cudaMemcpyAsync(out, t->flags, (size_t)t->n_nodes, cudaMemcpyDeviceToDevice, st), "flags copy");
    k_uniform_flags<<<grid_for(t->n_nodes, 256), 256, 0, st>>>(out, t->n_nodes, level_offset(t->L));
    return cuda_check(cudaGetLastError(), "flags kernel");
}

tr_status tree_export(const tr_tree* t, double* out8, cudaStream_t st) {
    if (t->mode == 0)
        k_export<0><<<grid_for(t->n_nodes, 256), 256, 0, st>>>(t->nodes, t->n_nodes, out8, t->U, t->Eu, t->N, t->flags);
    else
        k_export<1><<<grid_for(t->n_nodes, 256), 256, 0, st>>>(t->nodes, t->n_nodes, out8, t->U, t->Eu, t->N, t->flags);
    return cuda_check(cudaGetLastError(), "node export kernel");
}

}  // namespace tr
