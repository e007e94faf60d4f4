// Tree walk + node->ray mapping + far-to-near sweep, one warp per target.
//
// Walk (Sec. 2.3-2.4): a warp keeps a stack of opened nodes in shared
// memory.  Each step pops up to four opened nodes and evaluates their 32
// children at once, one child per lane: a child that contains the target, or
// fails the BH MAC (h/d < theta_lim), the IF MAC (nodes holding an
// ionisation front: h/d < theta_IF) or the Src MAC (emitting nodes:
// h/d < theta_src), is pushed as opened; the others are accepted.
// Map (Sec. 2.3, App. A): every accepted node is spread by the warp over
// the rays its table entry lists (angular weights) and over the evaluation
// points its radial kernel reaches: W_p for the recombination rate alpha and
// the energy e, W_f,3 for the emission eps.  The ray bins live in shared
// memory; each node's (ray, point) cells are distinct, so the lanes write
// without atomics, and in FP32 mode every bin is a compensated
// (Kahan-Neumaier) pair.
// Sweep (Sec. 2.5, Eq. 12-17): the bins become per-volume coefficients and
// photon rates in FP64; each lane sweeps whole rays far to near and the warp
// sums the rays (Eq. 18).
#include "tr_internal.cuh"

namespace tr {
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int MODE> struct Prec;
template <> struct Prec<0> { using real = double; using Node = NodeF64; };
template <> struct Prec<1> { using real = float; using Node = NodeF32; };

struct WalkArgs {
    const void* nodes;
    int N, L, nr, npix, eta, nside, use_e, stack_cap;
    double th_lim2, th_if2, th_src2, lray;
    float th_lim2f, th_if2f, th_src2f, lrayf;
    const uint32_t* toff;
    const uint32_t* tent;
    const double* r;
    const float* rf;
    const double* inv_r2;
    const double* vol;
    const double* G;
    const double* ID2;
    const int64_t* targets;                 // NULL: all cells, visited in Morton order
    int64_t n_targets;
    double Fconv, Econv;                    // scaled flux -> CGS flux / energy density
    double* F;
    double* E;
    uint8_t* ion;
    double* bins_out;
    int32_t* ids_out;
    int32_t* counts_out;
    double* eps_self_out;
    int acc_cap;
    int32_t* status;
    unsigned int* counter;
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// W_p of App. A (Eq. A2), outer branch rebuilt from the constraints printed
// with it: W_p2(x) = (x - sqrt3/2)^2 (a2 x + 2A(2 + sqrt3) - a2/2).
template <typename T>
__device__ __forceinline__ T wp_kernel(T x) {
    const T a1 = T(1.21), a2 = T(-6.35), A = T(4.08), M = T(1.184);
    const T s3h = T(0.86602540378443864676);
    const T c2 = T(2.0) * A * (T(2.0) + T(1.73205080756887729353)) - T(0.5) * a2;
    if (x < T(0.5)) return M + x * x * (a1 * x - (T(0.5) * a1 + T(4.0) * (M - A)));
    if (x < s3h) { T t = x - s3h; return t * t * (a2 * x + c2); }
    return T(0);
}

__device__ __forceinline__ int face_bin(int x, int A) {
    if (x == 0) return TQH;
    int q = (TQH * abs(x)) / A;
    q = min(q, TQH - 1);
    return x > 0 ? TQH + 1 + q : TQH - 1 - q;
}

// Table key of a node from the integer offset o = 2 (node centre - target
// centre) in half cells and the node edge s in cells.
__device__ __forceinline__ int table_key(int ox, int oy, int oz, int s) {
    const int ax = abs(ox), ay = abs(oy), az = abs(oz);
    int a = 0, A = ax;
    if (ay > A) { a = 1; A = ay; }
    if (az > A) { a = 2; A = az; }
    const int ob = (a == 0) ? oy : ox;
    const int oc = (a == 2) ? oy : oz;
    const int oa = (a == 0) ? ox : (a == 1 ? oy : oz);
    const int face = 2 * a + (oa < 0 ? 1 : 0);
    const int u = face_bin(ob, A), v = face_bin(oc, A);
    const long long o2 = (long long)ox * ox + (long long)oy * oy + (long long)oz * oz;
    const long long lim = 64LL * s, lim2 = lim * lim;
    long long pb = (long long)((float)lim * rsqrtf((float)o2));
    while (pb > 0 && pb * pb * o2 > lim2) --pb;
    while ((pb + 1) * (pb + 1) * o2 <= lim2) ++pb;
    if (pb > TB - 1) pb = TB - 1;
    return ((face * TQ + u) * TQ + v) * TB + (int)pb;
}

template <int MODE>
__device__ __forceinline__ void bin_add(double* slot, typename Prec<MODE>::real x) {
    if (MODE == 0) {
        *slot += (double)x;
    } else {
        float2* p = reinterpret_cast<float2*>(slot);
        float2 v = *p;
        const float xf = (float)x;
        const float t = v.x + xf;
        if (fabsf(v.x) >= fabsf(xf)) v.y += (v.x - t) + xf;
        else v.y += (xf - t) + v.x;
        v.x = t;
        *p = v;
    }
}

template <int MODE>
__device__ __forceinline__ double bin_value(const double* slot) {
    if (MODE == 0) return *slot;
    const float2 v = *reinterpret_cast<const float2*>(slot);
    return (double)v.x + (double)v.y;
}

template <int MODE>
__device__ __forceinline__ void load_node(const void* nodes, int64_t id, typename Prec<MODE>::real* cm,
                                          typename Prec<MODE>::real& m, typename Prec<MODE>::real* q,
                                          typename Prec<MODE>::real& mion) {
    if (MODE == 0) {
        const double2* p = reinterpret_cast<const double2*>((const NodeF64*)nodes + id);
        const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
        cm[0] = a.x; cm[1] = a.y; cm[2] = b.x; m = b.y;
        q[0] = c.x; q[1] = c.y; q[2] = d.x; mion = d.y;
    } else {
        const float4* p = reinterpret_cast<const float4*>((const NodeF32*)nodes + id);
        const float4 a = __ldg(p), b = __ldg(p + 1);
        cm[0] = a.x; cm[1] = a.y; cm[2] = a.z; m = a.w;
        q[0] = b.x; q[1] = b.y; q[2] = b.z; mion = b.w;
    }
}

// Opening decision of a non-leaf node that does not contain the target.
__device__ __forceinline__ bool must_open(double h2, double d2, double m, double mion, double eps,
                                          const WalkArgs& a) {
    const bool acc_lim = h2 < __dmul_rn(a.th_lim2, d2);
    const bool is_if = (__dmul_rn(DELTA_IF, m) < mion) && (mion < __dmul_rn(1.0 - DELTA_IF, m));
    const bool acc_if = !is_if || (h2 < __dmul_rn(a.th_if2, d2));
    const bool acc_src = !(eps > 0.0) || (h2 < __dmul_rn(a.th_src2, d2));
    return !(acc_lim && acc_if && acc_src);
}
__device__ __forceinline__ bool must_open(float h2, float d2, float m, float mion, float eps, const WalkArgs& a) {
    const bool acc_lim = h2 < a.th_lim2f * d2;
    const bool is_if = (1e-8f * m < mion) && (mion < (1.0f - 1e-8f) * m);
    const bool acc_if = !is_if || (h2 < a.th_if2f * d2);
    const bool acc_src = !(eps > 0.f) || (h2 < a.th_src2f * d2);
    return !(acc_lim && acc_if && acc_src);
}

__device__ __forceinline__ double dist2(double tx, double ty, double tz, const double* cm) {
    const double dx = __dsub_rn(tx, cm[0]), dy = __dsub_rn(ty, cm[1]), dz = __dsub_rn(tz, cm[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ float dist2(float tx, float ty, float tz, const float* cm) {
    const float dx = tx - cm[0], dy = ty - cm[1], dz = tz - cm[2];
    return dx * dx + dy * dy + dz * dz;
}

// Map one accepted node onto the warp's ray bins (all lanes call this with
// the same, broadcast, arguments).
template <int MODE>
__device__ void map_node(const WalkArgs& a, double* bins_a, double* bins_eps, double* bins_e,
                         typename Prec<MODE>::real* wrad, int key, typename Prec<MODE>::real d, int s,
                         typename Prec<MODE>::real alpha, typename Prec<MODE>::real eps,
                         typename Prec<MODE>::real e, int lane) {
    using real = typename Prec<MODE>::real;
    const int nr = a.nr;
    const real* r = nullptr;
    if (MODE == 0) r = reinterpret_cast<const real*>(a.r);
    else r = reinterpret_cast<const real*>(a.rf);
    const real rlast = r[nr - 1];
    const uint32_t eo = __ldg(a.toff + key), en = __ldg(a.toff + key + 1) - eo;
    const real inv_m3 = real(1.0) / real(TM * TM * TM);
    const bool do_e = a.use_e && e != real(0);
    if (alpha != real(0) || do_e) {
        // radial weights W_p(|r_i - d| / h), normalised over the points (App. A)
        int i0, ni;
        const real h = (real)s;
        if (d >= rlast) {
            i0 = nr - 1; ni = 1;
            if (lane == 0) wrad[0] = real(1);
        } else {
            const real reach = real(0.8661) * h;
            const real dlo = d > reach ? d - reach : real(0);
            int lo = (int)floor((real)a.eta * sqrt(real(2) * dlo)) - 1;
            int hi = (int)ceil((real)a.eta * sqrt(real(2) * (d + reach))) + 1;
            lo = max(lo, 0);
            hi = min(hi, nr - 1);
            i0 = lo; ni = hi - lo + 1;
            real S = real(0);
            for (int j = lane; j < ni; j += 32) {
                const real w = wp_kernel<real>(fabs(r[i0 + j] - d) / h);
                wrad[j] = w;
                S += w;
            }
            S = warp_sum(S);
            __syncwarp();
            if (S > real(0)) {
                for (int j = lane; j < ni; j += 32) wrad[j] = wrad[j] / S;
            } else {
                int i = (int)floor((real)a.eta * sqrt(real(2) * d));
                i = min(max(i, 0), nr - 2);
                while (i + 1 < nr - 1 && r[i + 1] <= d) ++i;
                while (i > 0 && r[i] > d) --i;
                i0 = i; ni = 2;
                if (lane == 0) {
                    const real ra = r[i], rb = r[i + 1];
                    wrad[0] = (rb - d) / (rb - ra);
                    wrad[1] = (d - ra) / (rb - ra);
                }
            }
        }
        __syncwarp();
        const int total = (int)en * ni;
        for (int p = lane; p < total; p += 32) {
            const int ei = p / ni, j = p - ei * ni;
            const uint32_t ent = __ldg(a.tent + eo + ei);
            const int b = (int)(ent >> 16) * nr + i0 + j;
            const real wk = (real)(ent & 0xffffu) * inv_m3 * wrad[j];
            if (alpha != real(0)) bin_add<MODE>(bins_a + b, wk * alpha);
            if (do_e) bin_add<MODE>(bins_e + b, wk * e);
        }
        __syncwarp();
    }
    if (eps != real(0)) {
        // W_f,3 (App. A.3): two points r_i <= d < r_{i+1} keeping the sum and
        // the flux at the target exact
        int i;
        real w0, w1;
        if (d >= rlast) {
            i = nr - 2; w0 = real(0); w1 = real(1);
        } else {
            i = (int)floor((real)a.eta * sqrt(real(2) * d));
            i = min(max(i, 0), nr - 2);
            while (i + 1 < nr - 1 && r[i + 1] <= d) ++i;
            while (i > 0 && r[i] > d) --i;
            if (i == 0) {
                w0 = real(0); w1 = real(1);
            } else {
                const real ri = r[i], rj = r[i + 1];
                const real ia = real(1) / (ri * ri), ib = real(1) / (rj * rj), it = real(1) / (d * d);
                w1 = (ia - it) / (ia - ib);
                w0 = real(1) - w1;
            }
        }
        for (int p = lane; p < 2 * (int)en; p += 32) {
            const int ei = p >> 1, k = p & 1;
            const uint32_t ent = __ldg(a.tent + eo + ei);
            const real wk = (real)(ent & 0xffffu) * inv_m3 * (k ? w1 : w0);
            if (wk != real(0)) bin_add<MODE>(bins_eps + (int)(ent >> 16) * nr + i + k, wk * eps);
        }
        __syncwarp();
    }
}

// Far-to-near sweep of one ray (Sec. 2.5): al = alpha per volume, ph = photon
// rates per steradian (Phi_j, updated in place), ev = energy density or NULL.
__device__ double sweep_ray(const WalkArgs& a, const double* al, double* ph, const double* ev) {
    const int nr = a.nr;
    uint64_t m0 = 0, m1 = 0;
    for (int j = 1; j < nr; ++j)
        if (ph[j] > 0.0) { if (j < 64) m0 |= 1ull << j; else m1 |= 1ull << (j - 64); }
    if (!(m0 | m1)) return 0.0;
    const int jtop = m1 ? 64 + 63 - __clzll((long long)m1) : 63 - __clzll((long long)m0);
    for (int i = jtop - 1; i >= 0; --i) {
        // sources strictly beyond r_i
        const int b = i + 1;
        uint64_t a0 = (b < 64) ? (m0 & (~0ull << b)) : 0ull;
        uint64_t a1 = (b <= 64) ? m1 : (m1 & (~0ull << (b - 64)));
        if (!(a0 | a1)) continue;
        const double* id2 = a.ID2 + (size_t)i * nr;
        const double* g = a.G + (size_t)i * nr;
        double Ftot = 0.0;
        for (uint64_t w = a0; w; w &= w - 1) { const int j = __ffsll((long long)w) - 1; Ftot += ph[j] * __ldg(id2 + j); }
        for (uint64_t w = a1; w; w &= w - 1) { const int j = 64 + __ffsll((long long)w) - 1; Ftot += ph[j] * __ldg(id2 + j); }
        if (!(Ftot > 0.0)) continue;
        double zd = 1.0;                                       // Eq. 17
        if (ev && ev[i + 1] > 0.0) zd = fmin(2.0, Ftot / ev[i + 1]);
        const double A = 0.5 * (al[i] + al[i + 1]);
        const double cf = A * zd / Ftot;                       // zeta_s = F_j / Ftot (Eq. 16)
        for (uint64_t w = a0; w; w &= w - 1) {
            const int j = __ffsll((long long)w) - 1;
            const double R = cf * __ldg(g + j) * (ph[j] * __ldg(id2 + j));     // Eq. 14
            const double np = ph[j] - R;                                      // Eq. 13
            if (np > 0.0) ph[j] = np; else { ph[j] = 0.0; m0 &= ~(1ull << j); }
        }
        for (uint64_t w = a1; w; w &= w - 1) {
            const int j = 64 + __ffsll((long long)w) - 1;
            const double R = cf * __ldg(g + j) * (ph[j] * __ldg(id2 + j));
            const double np = ph[j] - R;
            if (np > 0.0) ph[j] = np; else { ph[j] = 0.0; m1 &= ~(1ull << (j - 64)); }
        }
    }
    double F0 = 0.0;                                            // Eq. 10-11 at r = 0
    for (uint64_t w = m0; w; w &= w - 1) { const int j = __ffsll((long long)w) - 1; F0 += ph[j] * __ldg(a.inv_r2 + j); }
    for (uint64_t w = m1; w; w &= w - 1) { const int j = 64 + __ffsll((long long)w) - 1; F0 += ph[j] * __ldg(a.inv_r2 + j); }
    return F0;
}

// Convert the bins in place into FP64 per-volume coefficients and photon
// rates, sweep all rays and return the warp's total flux (scaled units).
template <int MODE>
__device__ double sweep_bins(const WalkArgs& a, double* bins_a, double* bins_eps, double* bins_e, int lane) {
    const int nr = a.nr, nbins = a.npix * nr;
    for (int b = lane; b < nbins; b += 32) {
        const int i = b % nr;
        const double vol = __ldg(a.vol + i);
        const double va = bin_value<MODE>(bins_a + b);
        const double ve = bin_value<MODE>(bins_eps + b);
        bins_a[b] = va / vol;
        bins_eps[b] = ve / (4.0 * PI_D);                        // Eq. 12
        if (a.use_e) bins_e[b] = bin_value<MODE>(bins_e + b) / vol;
    }
    __syncwarp();
    double F = 0.0;
    for (int k = lane; k < a.npix; k += 32)
        F += sweep_ray(a, bins_a + k * nr, bins_eps + k * nr, a.use_e ? bins_e + k * nr : nullptr);
    return warp_sum(F);
}

template <int MODE, bool DUMP>
__global__ void __launch_bounds__(32) k_walk(WalkArgs a) {
    using real = typename Prec<MODE>::real;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x;
    const int nr = a.nr, nbins = a.npix * nr;
    const int nq = a.use_e ? 3 : 2;
    double* bins_a = reinterpret_cast<double*>(smem);
    double* bins_eps = bins_a + nbins;
    double* bins_e = a.use_e ? bins_eps + nbins : nullptr;
    uint32_t* stack = reinterpret_cast<uint32_t*>(bins_a + (size_t)nq * nbins);
    real* wrad = reinterpret_cast<real*>(stack + a.stack_cap);
    const int N = a.N, L = a.L;
    const unsigned lanemask_lt = (1u << lane) - 1u;

    for (;;) {
        unsigned int qq = 0;
        if (lane == 0) qq = atomicAdd(a.counter, 1u);
        const int64_t q = (int64_t)__shfl_sync(FULL, qq, 0);
        if (q >= a.n_targets) break;
        int tx, ty, tz;
        int64_t cell;
        if (a.targets) {
            cell = a.targets[q];
            tx = (int)(cell % N); ty = (int)((cell / N) % N); tz = (int)(cell / ((int64_t)N * N));
        } else {
            tx = (int)compact3((uint32_t)q); ty = (int)compact3((uint32_t)q >> 1); tz = (int)compact3((uint32_t)q >> 2);
            cell = ((int64_t)tz * N + ty) * N + tx;
        }
        const real px = (real)tx + real(0.5), py = (real)ty + real(0.5), pz = (real)tz + real(0.5);
        for (int b = lane; b < nq * nbins; b += 32) bins_a[b] = 0.0;
        if (lane == 0) stack[0] = 0u;                           // the root, opened
        int top = 1, nacc = 0;
        bool overflow = false;
        __syncwarp();
        while (top > 0) {
            const int np = min(4, top);
            const int pi = lane >> 3, c = lane & 7;
            const uint32_t pe = (pi < np) ? stack[top - np + pi] : 0u;
            __syncwarp();
            top -= np;
            int action = 0;                                     // 1 open, 2 accept
            int lev = 0, s = 0, key = 0;
            uint32_t mort = 0;
            real d = real(0), alpha = real(0), eps = real(0), e = real(0);
            if (pi < np) {
                lev = (int)(pe >> 27) + 1;
                mort = ((pe & 0x7ffffffu) << 3) | (uint32_t)c;
                s = N >> lev;
                const int cx = (int)compact3(mort) * s, cy = (int)compact3(mort >> 1) * s,
                          cz = (int)compact3(mort >> 2) * s;
                const bool contains = (tx >= cx && tx < cx + s) && (ty >= cy && ty < cy + s) &&
                                      (tz >= cz && tz < cz + s);
                if (contains) {
                    action = (lev == L) ? 0 : 1;
                } else {
                    real cm[3], m, qv[3], mion;
                    load_node<MODE>(a.nodes, level_offset(lev) + mort, cm, m, qv, mion);
                    const real d2 = dist2(px, py, pz, cm);
                    const real h2 = (real)s * (real)s;
                    if (lev < L && must_open(h2, d2, m, mion, qv[1], a)) {
                        action = 1;
                    } else {
                        action = 2;
                        d = sqrt(d2);
                        alpha = qv[0]; eps = qv[1]; e = qv[2];
                        key = table_key(2 * cx + s - 2 * tx - 1, 2 * cy + s - 2 * ty - 1, 2 * cz + s - 2 * tz - 1, s);
                    }
                }
            }
            const unsigned open_mask = __ballot_sync(FULL, action == 1);
            const int nopen = __popc(open_mask);
            if (top + nopen > a.stack_cap) { overflow = true; break; }
            if (action == 1) stack[top + __popc(open_mask & lanemask_lt)] = ((uint32_t)lev << 27) | mort;
            top += nopen;
            unsigned acc_mask = __ballot_sync(FULL, action == 2);
            if (DUMP) {
                if (action == 2) {
                    const int slot = nacc + __popc(acc_mask & lanemask_lt);
                    if (slot < a.acc_cap) a.ids_out[q * a.acc_cap + slot] = (int32_t)(level_offset(lev) + mort);
                }
                nacc += __popc(acc_mask);
            }
            while (acc_mask) {
                const int src = __ffs(acc_mask) - 1;
                acc_mask &= acc_mask - 1;
                const real al_b = __shfl_sync(FULL, alpha, src), ep_b = __shfl_sync(FULL, eps, src);
                const real e_b = __shfl_sync(FULL, e, src);
                const real d_b = __shfl_sync(FULL, d, src);
                const int s_b = __shfl_sync(FULL, s, src), key_b = __shfl_sync(FULL, key, src);
                const bool in_reach = (MODE == 0) ? ((double)d_b <= a.lray) : ((float)d_b <= a.lrayf);
                if (in_reach && (al_b != real(0) || ep_b != real(0) || (a.use_e && e_b != real(0))))
                    map_node<MODE>(a, bins_a, bins_eps, bins_e, wrad, key_b, d_b, s_b, al_b, ep_b, e_b, lane);
            }
            __syncwarp();
        }
        // own emission of the target (Sec. 2.5 footnote: target sphere r_tp = dx/2)
        real cmt[3], mt, qt[3], miont;
        load_node<MODE>(a.nodes, level_offset(L) + morton3(tx, ty, tz), cmt, mt, qt, miont);
        const double eps_self = (double)qt[1];
        if (overflow) {
            if (lane == 0) {
                atomicAdd(a.status, 1);
                if (a.F) a.F[a.targets ? q : cell] = __longlong_as_double(0x7ff8000000000000LL);
            }
            continue;
        }
        if (DUMP) {
            double* out = a.bins_out + (size_t)q * 3 * nbins;
            for (int b = lane; b < nbins; b += 32) {
                out[b] = bin_value<MODE>(bins_a + b);
                out[nbins + b] = bin_value<MODE>(bins_eps + b);
                out[2 * nbins + b] = a.use_e ? bin_value<MODE>(bins_e + b) : 0.0;
            }
            if (lane == 0) { a.counts_out[q] = nacc; a.eps_self_out[q] = eps_self; }
            __syncwarp();
            continue;
        }
        const double F = sweep_bins<MODE>(a, bins_a, bins_eps, bins_e, lane) + eps_self / (4.0 * PI_D * 0.25);
        if (lane == 0) {
            const int64_t o = a.targets ? q : cell;
            if (a.F) a.F[o] = F * a.Fconv;
            if (a.E) a.E[o] = F * a.Econv;
            if (a.ion) a.ion[o] = (uint8_t)(F > 0.0);
        }
        __syncwarp();
    }
}

// Unfused sweep over bins stored by the dump walk: one warp per target.
__global__ void __launch_bounds__(32) k_sweep_stored(WalkArgs a, const double* bins_in, const double* eps_self) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x;
    const int nbins = a.npix * a.nr;
    double* bins_a = reinterpret_cast<double*>(smem);
    double* bins_eps = bins_a + nbins;
    double* bins_e = a.use_e ? bins_eps + nbins : nullptr;
    for (int64_t q = blockIdx.x; q < a.n_targets; q += gridDim.x) {
        const double* in = bins_in + (size_t)q * 3 * nbins;
        for (int b = lane; b < nbins; b += 32) {
            bins_a[b] = in[b];
            bins_eps[b] = in[nbins + b];
            if (a.use_e) bins_e[b] = in[2 * nbins + b];
        }
        __syncwarp();
        const double F = sweep_bins<0>(a, bins_a, bins_eps, bins_e, lane) + eps_self[q] / (4.0 * PI_D * 0.25);
        if (lane == 0) {
            if (a.F) a.F[q] = F * a.Fconv;
            if (a.E) a.E[q] = F * a.Econv;
            if (a.ion) a.ion[q] = (uint8_t)(F > 0.0);
        }
        __syncwarp();
    }
}

WalkArgs make_args(const tr_tree* t) {
    WalkArgs a{};
    a.nodes = t->nodes;
    a.N = t->N; a.L = t->L; a.nr = t->nr; a.npix = t->npix; a.eta = t->p.eta_r; a.nside = t->p.nside;
    a.use_e = t->use_e;
    a.th_lim2 = t->p.theta_lim * t->p.theta_lim;
    a.th_if2 = t->p.theta_if * t->p.theta_if;
    a.th_src2 = t->p.theta_src * t->p.theta_src;
    a.lray = t->lray;
    a.th_lim2f = (float)a.th_lim2; a.th_if2f = (float)a.th_if2; a.th_src2f = (float)a.th_src2;
    a.lrayf = (float)t->lray;
    a.toff = t->table->off; a.tent = t->table->ent;
    a.r = t->sw.r; a.rf = t->sw.rf; a.inv_r2 = t->sw.inv_r2; a.vol = t->sw.vol; a.G = t->sw.G; a.ID2 = t->sw.ID2;
    a.Fconv = t->U / (t->dx * t->dx);
    a.Econv = t->Eu;
    a.status = t->status;
    a.counter = t->counter;
    return a;
}

int stack_cap_for(const tr_tree* t) {
    // opened nodes pending on the stack stay well below this for theta >= 0.25
    (void)t;
    return 2048;
}

size_t walk_smem(const tr_tree* t, int stack_cap) {
    const int nq = t->use_e ? 3 : 2;
    return (size_t)nq * t->npix * t->nr * 8 + (size_t)stack_cap * 4 + MAX_NR * 8;
}

template <typename K>
tr_status launch_persistent(K kernel, size_t smem, const WalkArgs& a, cudaStream_t st) {
    tr_status s = cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "cudaFuncSetAttribute(smem)");
    if (s != TR_OK) return s;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, smem), "occupancy query");
    if (s != TR_OK) return s;
    if (per_sm < 1) return set_error(TR_EUNSUPPORTED, "ray bins need %zu bytes of shared memory per warp", smem);
    s = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st), "counter reset");
    if (s != TR_OK) return s;
    kernel<<<sms * per_sm, 32, smem, st>>>(a);
    return cuda_check(cudaGetLastError(), "walk kernel launch");
}

}  // namespace

tr_status walk_run(const tr_tree* t, const int64_t* targets, int64_t n_targets, bool dump, const WalkOut& out,
                   cudaStream_t st) {
    WalkArgs a = make_args(t);
    a.targets = targets;
    a.n_targets = n_targets;
    a.F = out.F; a.E = out.e; a.ion = out.ion;
    a.bins_out = out.bins; a.ids_out = out.ids; a.counts_out = out.counts; a.eps_self_out = out.eps_self;
    a.acc_cap = out.acc_cap;
    a.stack_cap = stack_cap_for(t);
    const size_t smem = walk_smem(t, a.stack_cap);
    tr_status s = cuda_check(cudaMemsetAsync(t->status, 0, 4 * sizeof(int32_t), st), "status reset");
    if (s != TR_OK) return s;
    if (t->mode == 0) s = dump ? launch_persistent(k_walk<0, true>, smem, a, st) : launch_persistent(k_walk<0, false>, smem, a, st);
    else s = dump ? launch_persistent(k_walk<1, true>, smem, a, st) : launch_persistent(k_walk<1, false>, smem, a, st);
    return s;
}

tr_status sweep_run(const tr_rays* r, double* F, double* e, uint8_t* ion, cudaStream_t st) {
    WalkArgs a{};
    a.nr = r->nr; a.npix = r->npix; a.use_e = r->use_e;
    a.r = r->sw.r; a.inv_r2 = r->sw.inv_r2; a.vol = r->sw.vol; a.G = r->sw.G; a.ID2 = r->sw.ID2;
    a.n_targets = r->n_targets;
    a.Fconv = r->U / (r->dx * r->dx);
    a.Econv = r->Eu;
    a.F = F; a.E = e; a.ion = ion;
    const size_t smem = (size_t)(r->use_e ? 3 : 2) * r->npix * r->nr * 8;
    tr_status s = cuda_check(cudaFuncSetAttribute(k_sweep_stored, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "cudaFuncSetAttribute(sweep smem)");
    if (s != TR_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = r->n_targets < (int64_t)sms * 8 ? r->n_targets : (int64_t)sms * 8;
    if (blocks > 0) k_sweep_stored<<<(unsigned)blocks, 32, smem, st>>>(a, r->bins, r->eps_self);
    return cuda_check(cudaGetLastError(), "sweep kernel launch");
}

tr_status read_status(const tr_tree* t, cudaStream_t st) {
    int32_t h[4] = {0, 0, 0, 0};
    tr_status s = cuda_check(cudaMemcpyAsync(h, t->status, sizeof h, cudaMemcpyDeviceToHost, st), "status copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "walk kernels");
    if (s != TR_OK) return s;
    if (h[0] > 0)
        return set_error(TR_EOVERFLOW, "the walk stack overflowed for %d target(s); their outputs are NaN", h[0]);
    return TR_OK;
}

}  // namespace tr
