// Node->ray table (Sec. 2.3, first mapping step), built on the device.
//
// The paper divides each node between rays in proportion to the volume of
// the node-ray intersection, read from a table over the node's angular
// position and angular size (defined in Paper I, not reproduced here).  This
// table: a node is an axis-aligned cube; its weight in ray k is the fraction
// of TM^3 sample points of the cube whose direction from the target falls in
// HEALPix pixel k.  The key is computed from the integer offset between the
// node's geometric centre and the target centre (in half cells): cube-map
// face of the dominant axis, a mirror-symmetric bin of each of the other two
// face coordinates, and the bin floor(32 psi) of psi = node size / centre
// distance.  Offsets whose largest component is shared by two axes (three
// axes) have edge (corner) keys whose representative direction lies on that
// cube edge (corner).  Each key's weights are those of a representative cube
// at distance 1 in the key's direction with psi at the bin centre.  Every
// sample counts 2 out of TW = 2 TM^3; for keys whose direction lies on a
// plane x = +-y (a mirror plane of the HEALPix pixels) a sample counts 1 in
// its pixel and 1 in the mirror pixel, so the table has those symmetries.
//
// Storage is CSR: ent[off[k] .. off[k+1]) holds (pixel << 16) | count,
// sorted by pixel; the weight is count / TW.
#include <map>
#include <mutex>
#include <utility>

#include "tr_internal.cuh"

namespace tr {
namespace {

// HEALPix ring-scheme pixel of a direction (Gorski et al. 2005).  Products
// and sums are rounded one by one (no contraction) so that the sample
// coordinates and the ring arithmetic are reproducible.
__device__ int ang2pix_ring(int nside, double x, double y, double z) {
    const double ns = (double)nside;
    const int nl4 = 4 * nside, ncap = 2 * nside * (nside - 1), npix = 12 * nside * nside;
    double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    double zc = __ddiv_rn(z, r);
    double za = fabs(zc);
    double phi = atan2(y, x);
    if (phi < 0.0) phi = __dadd_rn(phi, 2.0 * PI_D);
    double tt = __ddiv_rn(phi, 0.5 * PI_D);                 // [0, 4]
    if (tt >= 4.0) tt = __dsub_rn(tt, 4.0);
    if (za <= 2.0 / 3.0) {
        double t1 = __dmul_rn(ns, __dadd_rn(0.5, tt));
        double t2 = __dmul_rn(__dmul_rn(ns, zc), 0.75);
        long jp = (long)floor(__dsub_rn(t1, t2));            // ascending edge line
        long jm = (long)floor(__dadd_rn(t1, t2));            // descending edge line
        long ir = nside + 1 + jp - jm;                       // ring in the belt, 1..2N+1
        long kshift = 1 - (ir & 1);
        long num = jp + jm - nside + kshift + 1;
        long ip = (num >= 0) ? num / 2 : -((-num + 1) / 2);
        ip %= nl4;
        if (ip < 0) ip += nl4;
        return (int)(ncap + (ir - 1) * nl4 + ip);
    }
    double tp = __dsub_rn(tt, floor(tt));
    double tmp = __dmul_rn(ns, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
    long jp = (long)floor(__dmul_rn(tp, tmp));
    long jm = (long)floor(__dmul_rn(__dsub_rn(1.0, tp), tmp));
    long ir = jp + jm + 1;                                   // ring from the nearer pole
    long ip = (long)floor(__dmul_rn(tt, (double)ir));
    ip %= 4 * ir;
    if (ip < 0) ip += 4 * ir;
    if (zc > 0.0) return (int)(2 * ir * (ir - 1) + ip);
    return (int)(npix - 2 * ir * (ir + 1) + ip);
}

__device__ double face_coord(int u) {
    if (u == TQH) return 0.0;
    if (u > TQH) return (2.0 * (double)(u - TQH - 1) + 1.0) / (2.0 * TQH);
    return -(2.0 * (double)(TQH - 1 - u) + 1.0) / (2.0 * TQH);
}

// Centre of ring-scheme pixel k as (z, phi) (Gorski et al. 2005): rings are
// numbered from the north pole; a polar-cap ring i holds 4i pixels, an
// equatorial ring 4 N_side, every other one of them shifted by half a pixel.
__device__ void pix_centre(int nside, int k, double& z, double& phi) {
    const int npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
    const double ns = (double)nside;
    if (k < ncap) {                                          // north cap
        int i = (int)floor(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)k)));
        while (2 * i * (i - 1) > k) --i;
        while (2 * (i + 1) * i <= k) ++i;
        const int j = k - 2 * i * (i - 1);                   // 0-based in the ring
        z = 1.0 - (double)(i * i) / (3.0 * ns * ns);
        phi = ((double)j + 0.5) * 0.5 * PI_D / (double)i;
    } else if (k < npix - ncap) {                            // equatorial belt
        const int q = k - ncap;
        const int i = q / (4 * nside) + nside;               // ring N .. 3N
        const int j = q % (4 * nside);
        const double shift = ((i - nside) & 1) ? 0.0 : 0.5;
        z = (2.0 * ns - (double)i) * 2.0 / (3.0 * ns);
        phi = ((double)j + shift) * 0.5 * PI_D / ns;
    } else {                                                 // south cap, mirror of the north
        const int q = npix - 1 - k;
        int i = (int)floor(0.5 * (1.0 + sqrt(1.0 + 2.0 * (double)q)));
        while (2 * i * (i - 1) > q) --i;
        while (2 * (i + 1) * i <= q) ++i;
        const int jr = q - 2 * i * (i - 1);                  // 0-based from the ring's end
        z = -(1.0 - (double)(i * i) / (3.0 * ns * ns));
        phi = ((double)(4 * i - 1 - jr) + 0.5) * 0.5 * PI_D / (double)i;
    }
}

// The pixel that the reflection through the plane x = t y (t = +-1) maps
// pixel k to: the pixel of the mirrored centre (HEALPix has the symmetry).
__device__ int mirror_pixel(int nside, int k, double t) {
    double z, phi;
    pix_centre(nside, k, z, phi);
    const double st = sqrt((1.0 - z) * (1.0 + z));
    const double x = st * cos(phi), y = st * sin(phi);
    return ang2pix_ring(nside, t * y, t * x, z);
}

// Representative direction of a key (not normalised) and whether it lies on
// a plane x = +-y (mirror = +-1) or not (0).
__device__ void key_direction(int key, double* p, int& mirror) {
    mirror = 0;
    if (key < NFACEKEYS) {
        int rest = key / TB;
        const int v = rest % TQ;
        rest /= TQ;
        const int u = rest % TQ;
        const int face = rest / TQ;
        const int a = face / 2, b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
        p[a] = (face & 1) ? -1.0 : 1.0;
        p[b] = face_coord(u);
        p[c] = face_coord(v);
    } else if (key < NFACEKEYS + NEDGEKEYS) {
        const int rest = (key - NFACEKEYS) / TB;
        const int v = rest % TQ, edge = rest / TQ, pair = edge / 4;
        const int a = (pair == 2) ? 1 : 0, b = (pair == 0) ? 1 : 2, c = 3 - a - b;
        const double sa = (edge & 2) ? -1.0 : 1.0, sb = (edge & 1) ? -1.0 : 1.0;
        p[a] = sa; p[b] = sb; p[c] = face_coord(v);
        if (pair == 0) mirror = sa == sb ? 1 : -1;
    } else {
        const int corner = (key - NFACEKEYS - NEDGEKEYS) / TB;
        p[0] = (corner & 1) ? -1.0 : 1.0;
        p[1] = (corner & 2) ? -1.0 : 1.0;
        p[2] = (corner & 4) ? -1.0 : 1.0;
        mirror = p[0] == p[1] ? 1 : -1;
    }
}

// Histogram of the key's representative cube over the pixels (block-wide),
// in counts out of TW.
__device__ void key_histogram(int nside, int key, int* hist) {
    const int npix = 12 * nside * nside;
    for (int k = threadIdx.x; k < npix; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    const int pb = key % TB;
    double p[3];
    int mirror;
    key_direction(key, p, mirror);
    double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(p[0], p[0]), __dmul_rn(p[1], p[1])),
                                    __dmul_rn(p[2], p[2])));
    double C0 = __ddiv_rn(p[0], n), C1 = __ddiv_rn(p[1], n), C2 = __ddiv_rn(p[2], n);
    double psi = ((double)pb + 0.5) / 32.0;
    for (int s = threadIdx.x; s < TM * TM * TM; s += blockDim.x) {
        int ix = s % TM, iy = (s / TM) % TM, iz = s / (TM * TM);
        double fx = ((double)ix + 0.5) / TM - 0.5;
        double fy = ((double)iy + 0.5) / TM - 0.5;
        double fz = ((double)iz + 0.5) / TM - 0.5;
        double qx = __dadd_rn(C0, __dmul_rn(psi, fx));
        double qy = __dadd_rn(C1, __dmul_rn(psi, fy));
        double qz = __dadd_rn(C2, __dmul_rn(psi, fz));
        const int k = ang2pix_ring(nside, qx, qy, qz);
        if (mirror) {
            atomicAdd(&hist[k], 1);
            atomicAdd(&hist[mirror_pixel(nside, k, (double)mirror)], 1);
        } else {
            atomicAdd(&hist[k], 2);
        }
    }
    __syncthreads();
}

__global__ void k_table_count(int nside, uint32_t* counts) {
    extern __shared__ int hist[];
    const int key = blockIdx.x;
    key_histogram(nside, key, hist);
    const int npix = 12 * nside * nside;
    int local = 0;
    for (int k = threadIdx.x; k < npix; k += blockDim.x) local += hist[k] > 0;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    __shared__ int warp_sum[32];
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sum[w];
        counts[key] = (uint32_t)tot;
    }
}

// Exclusive scan of n counts into off[0..n] by one block of 1024 threads.
__global__ void k_scan(const uint32_t* counts, uint32_t* off, int n) {
    __shared__ uint32_t part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < (int)blockDim.x; ++w) { uint32_t t = part[w]; part[w] = run; run += t; }
        off[n] = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int i = lo; i < hi; ++i) { off[i] = run; run += counts[i]; }
}

__global__ void k_table_fill(int nside, const uint32_t* off, uint32_t* ent) {
    extern __shared__ int hist[];
    const int key = blockIdx.x;
    key_histogram(nside, key, hist);
    if (threadIdx.x == 0) {
        const int npix = 12 * nside * nside;
        uint32_t w = off[key];
        for (int k = 0; k < npix; ++k)
            if (hist[k] > 0) ent[w++] = ((uint32_t)k << 16) | (uint32_t)hist[k];
    }
}

__global__ void k_table_hdr(const uint32_t* off, uint2* hdr, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) hdr[k] = make_uint2(off[k], off[k + 1] - off[k]);
}

std::mutex g_mu;
std::map<std::pair<int, int>, Table*> g_tables;

}  // namespace

tr_status table_get(int nside, const Table** out, cudaStream_t st) {
    int dev = 0;
    tr_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != TR_OK) return s;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tables.find({dev, nside});
    if (it != g_tables.end()) { *out = it->second; return TR_OK; }
    Table* t = new Table();
    t->nside = nside;
    uint32_t* counts = nullptr;
    const int npix = 12 * nside * nside;
    const size_t shm = sizeof(int) * (size_t)npix;
    if ((s = cuda_check(cudaMalloc(&counts, sizeof(uint32_t) * NKEYS), "cudaMalloc(table counts)")) != TR_OK ||
        (s = cuda_check(cudaMalloc(&t->off, sizeof(uint32_t) * (NKEYS + 1)), "cudaMalloc(table offsets)")) != TR_OK) {
        cudaFree(counts);
        delete t;
        return s == TR_ECUDA ? TR_ENOMEM : s;
    }
    k_table_count<<<NKEYS, 256, shm, st>>>(nside, counts);
    k_scan<<<1, 1024, 0, st>>>(counts, t->off, NKEYS);
    uint32_t total = 0;
    s = cuda_check(cudaMemcpyAsync(&total, t->off + NKEYS, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                   "table size copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "table count kernels");
    if (s == TR_OK) s = cuda_check(cudaMalloc(&t->ent, sizeof(uint32_t) * (size_t)(total + 1)), "cudaMalloc(table)");
    if (s == TR_OK) {
        k_table_fill<<<NKEYS, 256, shm, st>>>(nside, t->off, t->ent);
        s = cuda_check(cudaMalloc(&t->hdr, sizeof(uint2) * NKEYS), "cudaMalloc(table headers)");
    }
    if (s == TR_OK) {
        k_table_hdr<<<(NKEYS + 255) / 256, 256, 0, st>>>(t->off, t->hdr, NKEYS);
        s = cuda_check(cudaStreamSynchronize(st), "table fill kernels");
    }
    cudaFree(counts);
    if (s != TR_OK) {
        cudaFree(t->off);
        cudaFree(t->ent);
        cudaFree(t->hdr);
        delete t;
        return s;
    }
    t->n_entries = (int)total;
    g_tables[{dev, nside}] = t;
    *out = t;
    return TR_OK;
}

tr_status table_build_into(int nside, Table* t, uint32_t* counts, uint32_t ent_capacity, cudaStream_t st) {
    const int npix = 12 * nside * nside;
    const size_t shm = sizeof(int) * (size_t)npix;
    k_table_count<<<NKEYS, 256, shm, st>>>(nside, counts);
    k_scan<<<1, 1024, 0, st>>>(counts, t->off, NKEYS);
    uint32_t total = 0;
    tr_status s = cuda_check(cudaMemcpyAsync(&total, t->off + NKEYS, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                             "table size copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "table count kernels");
    if (s != TR_OK) return s;
    if (total > ent_capacity)
        return set_error(TR_EUNSUPPORTED, "node->ray table for N_side %d needs %u entries, room for %u", nside, total,
                         ent_capacity);
    k_table_fill<<<NKEYS, 256, shm, st>>>(nside, t->off, t->ent);
    k_table_hdr<<<(NKEYS + 255) / 256, 256, 0, st>>>(t->off, t->hdr, NKEYS);
    s = cuda_check(cudaStreamSynchronize(st), "table fill kernels");
    if (s != TR_OK) return s;
    t->nside = nside;
    t->n_entries = (int)total;
    return TR_OK;
}

}  // namespace tr
