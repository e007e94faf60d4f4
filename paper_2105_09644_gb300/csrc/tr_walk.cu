// Tree walk + node->ray mapping + far-to-near sweep, one CTA per target.
//
// A persistent grid takes targets (cells) from a job list: a job is one
// built tree and a range or list of its cells, so one launch can serve
// several independent problems.
// Walk (Sec. 2.3-2.4): the CTA keeps a stack of opened nodes in shared
// memory.  Each step pops up to NT/8 opened nodes and evaluates their NT
// children at once, one child per thread: a child that contains the target,
// or fails the BH MAC (h/d < theta_lim), the IF MAC (nodes holding an
// ionisation front: h/d < theta_IF) or the Src MAC (emitting nodes:
// h/d < theta_src), is pushed as opened; the others are accepted.  On an
// AMR tree a node flagged as a cell is never opened.
// In the FP32 forms the distances come from FP32 records, and every opening
// decision and every discontinuous choice of the radial spreading (beyond
// L_ray or not, beyond the last point or not, a kernel support that is empty
// or holds one point) that FP32 cannot settle within a certified bound on
// its distance error is re-taken in FP64 from an FP64 copy of the tree: the
// accepted nodes are those of the FP64 form, bit for bit.
// Map (Sec. 2.3, App. A): the nodes accepted in a step are spread by the
// whole CTA over the rays their table entry lists (angular weights) and the
// evaluation points their radial kernel reaches (W_p or W_g for the
// recombination rate alpha and the energy e; W_f,3 or another flux kernel
// for the emission eps), with shared-memory atomics into the ray bins: FP64
// adds in the FP64 form, exact 64-bit fixed point in the FP32 forms.
// Sweep (Sec. 2.5, Eq. 12-17): each ray is swept far to near (FP64 and
// FP32 + FP64-sweep forms: a thread per ray, FP64 arithmetic; FP32 +
// double-FP32-sweep form: two lanes per ray, FP32 losses, double-FP32
// budgets) and the CTA sums the rays (Eq. 18).
// Variants: wide CTAs (512 / 256 threads) when the bins fill an SM, a
// register-capped walk when six CTAs fit, a dump mode keeping the raw bins
// and accepted ids, a column-density mode without radial points, and a
// separate instantiation for non-default kernels and boundaries.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tr_internal.cuh"

namespace tr {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// MODE 0: FP64 form; 1: FP32 walk + FP64 sweep; 2: FP32 walk + double-FP32 sweep
template <int MODE> struct Prec;
template <> struct Prec<0> { using real = double; using Node = NodeF64; };
template <> struct Prec<1> { using real = float; using Node = NodeF32; };
template <> struct Prec<2> { using real = float; using Node = NodeF32; };

constexpr float U32 = 5.9604645e-8f;        // 2^-24, the unit roundoff of FP32

struct WalkArgs {
    const void* nodes;
    const NodeF64* nodes64;                 // FP32 forms: the FP64 tree (exact re-decisions)
    const float* kappa;                     // FP32 forms: |cm32 - cm64| <= kappa x edge
    int N, L, nr, npix, eta, nside, use_e, stack_cap;
    double th_lim2, th_if2, th_src2, lray;
    double r_coef;                          // r_i = i^2 r_coef cells, r_coef = 1 / (2 eta^2) (Eq. 4)
    float r_coeff;                          // the same (a power of two: exact in FP32)
    float th_lim2f, th_if2f, th_src2f, lrayf;
    const uint32_t* toff;
    const uint32_t* tent;
    const uint2* hdr;
    const double* r;
    const float* rf;
    const double* inv_r2;
    const double* inv_vol;
    const float* inv_volf;
    const double* G;
    const double* ID2;
    const double* GI;
    const float* Gf;
    const float* ID2f;
    const float* GIf;
    const double* HT;                       // [j][i] lone-source loss per raw recombination deposit
    const int64_t* targets;                 // NULL: cells first .. first+n_targets-1 in walk order
    int64_t first;
    const uint8_t* flags;                   // AMR tree: node topology (NULL: uniform grid)
    const int4* blk;                        // AMR tree: per block {cell level, x, y, z}
    const uint32_t* blk_order;              // AMR tree: blocks in walk order
    int64_t n_cells;                        // valid target indices are [0, n_cells)
    int kern_a, kern_e;                     // tr_kernel (alpha, e) and tr_eps_kernel (eps)
    int bc;                                 // tr_bc of the walk
    double* cd_out;                         // column-density maps: [target][N_PIX], cm^-2
    double cd_conv;                         // n_H cells -> cm^-2 (the cell edge dx)
    double cd_omega;                        // 4 pi / N_PIX
    int64_t n_targets;
    double Fconv, Econv;                    // scaled flux -> CGS flux / energy density
    double* F;
    double* E;
    uint8_t* ion;
    double* bins_out;
    int32_t* ids_out;
    int32_t* counts_out;
    double* eps_self_out;
    float* scales_out;                      // dump: the fixed-point units of the FP32 form
    const float* scales_in;                 // stored sweep: the same, read back
    int acc_cap;
    int32_t* status;
    unsigned long long* stats;
};

__device__ __forceinline__ double warp_sum(double v) {
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
    if constexpr (sizeof(T) == 8) {          // FP64: evaluate only the branch needed
        if (x < T(0.5)) return M + x * x * (a1 * x - (T(0.5) * a1 + T(4.0) * (M - A)));
        if (x < s3h) { T t = x - s3h; return t * t * (a2 * x + c2); }
        return T(0);
    } else {                                 // FP32: both branches and a select (lanes of a warp
        const T inner = M + x * x * (a1 * x - (T(0.5) * a1 + T(4.0) * (M - A)));   // sit on either side)
        const T t = x - s3h;
        const T outer = t * t * (a2 * x + c2);
        return x < T(0.5) ? inner : (x < s3h ? outer : T(0));
    }
}

// W_g of App. A (Eq. A1): exp(-x^2), truncated at sqrt3/2.
constexpr double S3H_D = 0.86602540378443864676;

template <typename T>
__device__ __forceinline__ T wg_kernel(T x) {
    return x < T(S3H_D) ? exp(-x * x) : T(0);
}

// The smoothing kernel of alpha and e at distance `dist` from the node:
// W_p(dist / h) with hpar = 1/h, or W_g(dist / h) with hpar = h (a true
// division, since W_g jumps at its truncation and the argument must round
// as the definition's quotient does).
template <typename T>
__device__ __forceinline__ T radial_w(T dist, T hpar, int gauss) {
    return gauss ? wg_kernel<T>(dist / hpar) : wp_kernel<T>(dist * hpar);
}

// Stack entry standing for "evaluate the root node" (real entries hold a
// level <= 9 in their top 5 bits, so this value never occurs as one).
constexpr uint32_t ROOT_EVAL = 0xffffffffu;

// One axis of the node copy the boundary condition puts next to the target
// (Sec. 2.8): g2, t2 = twice the node's and the target's centre (finest
// cells).  Corner of symmetry, axis mirrored: the node seen from the
// mirrored target.  Periodic: the nearest copy, offset wrapped into [-N, N)
// half cells.
template <typename T>
__device__ __forceinline__ void bc_frame(int bc, int mirrored, int N, int g2, int t2, T p, int& o, T& q) {
    if (bc == TR_BC_CORNER && mirrored) { o = -(g2 + t2); q = -p; return; }
    o = g2 - t2;
    q = p;
    if (bc == TR_BC_PERIODIC) {
        if (o >= N) { o -= 2 * N; q += (T)N; }
        else if (o < -N) { o += 2 * N; q -= (T)N; }
    }
}

__device__ __forceinline__ int face_bin(int x, int A) {
    if (x == 0) return TQH;
    int q = (TQH * abs(x)) / A;
    q = min(q, TQH - 1);
    return x > 0 ? TQH + 1 + q : TQH - 1 - q;
}

// Table key of a node from the integer offset o = 2 (node centre - target
// centre) in half cells and the node edge s in cells: a face key when one
// axis has the largest |o|, an edge key when two tie for it, a corner key
// when all three do.
__device__ __forceinline__ int table_key(int ox, int oy, int oz, int s) {
    const int ax = abs(ox), ay = abs(oy), az = abs(oz);
    const int A = max(ax, max(ay, az));
    const long long o2 = (long long)ox * ox + (long long)oy * oy + (long long)oz * oz;
    const long long lim = 64LL * s, lim2 = lim * lim;
    long long pb = (long long)((float)lim * rsqrtf((float)o2));
    while (pb > 0 && pb * pb * o2 > lim2) --pb;
    while ((pb + 1) * (pb + 1) * o2 <= lim2) ++pb;
    if (pb > TB - 1) pb = TB - 1;
    const int tx = ax == A, ty = ay == A, tz = az == A;
    const int ntie = tx + ty + tz;
    if (ntie == 1) {
        const int a = tx ? 0 : (ty ? 1 : 2);
        const int ob = (a == 0) ? oy : ox;
        const int oc = (a == 2) ? oy : oz;
        const int oa = (a == 0) ? ox : (a == 1 ? oy : oz);
        const int face = 2 * a + (oa < 0 ? 1 : 0);
        const int u = face_bin(ob, A), v = face_bin(oc, A);
        return ((face * TQ + u) * TQ + v) * TB + (int)pb;
    }
    if (ntie == 2) {                         // edge of the tied axes a < b, the third axis c binned
        const int c = !tx ? 0 : (!ty ? 1 : 2);
        const int pair = c == 2 ? 0 : (c == 1 ? 1 : 2);
        const int oa = c == 0 ? oy : ox, ob = c == 2 ? oy : oz, oc = c == 0 ? ox : (c == 1 ? oy : oz);
        const int edge = 4 * pair + 2 * (oa < 0) + (ob < 0);
        return NFACEKEYS + (edge * TQ + face_bin(oc, A)) * TB + (int)pb;
    }
    const int corner = (ox < 0) + 2 * (oy < 0) + 4 * (oz < 0);
    return NFACEKEYS + NEDGEKEYS + corner * TB + (int)pb;
}

// Ray bins.  FP64 form: one double per bin, atomic FP64 adds.  FP32 form: the
// FP32 addends are accumulated exactly in 64-bit fixed point, kept as two
// 32-bit words (low word, high word) updated by two integer atomics with the
// carry of the low word propagated: an order-independent sum whose only
// rounding is that of each FP32 addend.  The fixed-point unit is a power of
// two chosen from the root node's total, so that no bin can exceed 2^62.
struct Scales { float a, eps, e; };          // fixed-point units per quantity (FP32 form)

__device__ __forceinline__ float fixed_scale(float total) {
    int ex = 0;
    frexpf(total > 0.f ? total : 1.f, &ex);   // total < 2^ex
    return ldexpf(1.0f, min(62 - ex, 126));
}

template <int MODE>
__device__ __forceinline__ double bin_value(const double* slot, float scale) {
    if (MODE == 0) return *slot;
    const uint2 v = *reinterpret_cast<const uint2*>(slot);
    return ((double)v.y * 4294967296.0 + (double)v.x) / (double)scale;
}

template <int MODE>
__device__ __forceinline__ float bin_value_f(const double* slot, float inv_scale) {
    const uint2 v = *reinterpret_cast<const uint2*>(slot);
    return ((float)v.y * 4294967296.0f + (float)v.x) * inv_scale;
}

template <int MODE>
__device__ __forceinline__ bool bin_nonzero(const double* slot) {
    if (MODE == 0) return *slot > 0.0;
    const uint2 v = *reinterpret_cast<const uint2*>(slot);
    return (v.x | v.y) != 0u;
}

template <int MODE>
__device__ __forceinline__ void bin_atomic_add(double* slot, typename Prec<MODE>::real x, float scale) {
    if (MODE == 0) {
        atomicAdd(slot, (double)x);
    } else {
        const float v = (float)x * scale;                     // exact: scale is a power of two
        if (!(v > 0.f)) return;
        const float hf = floorf(v * 2.3283064365386963e-10f);  // v / 2^32, exact
        const float lf = v - hf * 4294967296.0f;              // exact, < 2^32
        const unsigned lo = (unsigned)lf, hi = (unsigned)hf;
        unsigned* w = reinterpret_cast<unsigned*>(slot);
        const unsigned old = atomicAdd(w, lo);
        const unsigned carry = (old + lo < old) ? 1u : 0u;
        if (hi + carry) atomicAdd(w + 1, hi + carry);
    }
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
// The same decision taken in FP64 with the node's IF flag given (FP32 forms,
// when FP32 cannot settle it).
__device__ __forceinline__ bool must_open_exact(double h2, double d2, bool is_if, bool has_eps, const WalkArgs& a) {
    const bool acc_lim = h2 < __dmul_rn(a.th_lim2, d2);
    const bool acc_if = !is_if || (h2 < __dmul_rn(a.th_if2, d2));
    const bool acc_src = !has_eps || (h2 < __dmul_rn(a.th_src2, d2));
    return !(acc_lim && acc_if && acc_src);
}

// Bound on |d2 - d2_64| for an FP32 squared distance d2 whose per-axis
// displacement carries an error of at most E from the stored centre of mass
// (plus the rounding of the displacement, the squares and the sums): with
// e_a <= E + u d per axis, |sum dx^2 - sum dx64^2| <= 2 sqrt3 d e + 3 e^2,
// plus 3.1 u d2 of rounding; a factor 2 of margin on top.
__device__ __forceinline__ float d2_err_bound(float d2, float E) {
    const float d = d2 * rsqrtf(d2) * 1.000001f;
    const float e = E + 1.01f * U32 * d;
    return 2.f * (3.4641017f * d * e + 3.f * e * e + 3.1f * U32 * d2);
}

// One criterion h2 < t2 d2_64 with d2_64 in [lo, hi]: 1 surely true, 0 surely
// false, -1 undecided (lo and hi carry the roundings of t2 and the product).
__device__ __forceinline__ int mac_tri(float h2, float t2, float lo, float hi) {
    if (h2 < t2 * lo) return 1;
    if (h2 >= t2 * hi) return 0;
    return -1;
}

// Opening decision of the FP32 forms: 1 open, 0 accept, -1 undecided within
// the error bound B of d2 (then taken by must_open_exact on FP64 data).
__device__ __forceinline__ int mac_f32(float h2, float d2, float B, bool is_if, bool has_eps, const WalkArgs& a) {
    const float lo = fmaxf(d2 - B, 0.f) * (1.f - 8.f * U32);
    const float hi = (d2 + B) * (1.f + 8.f * U32);
    int r = mac_tri(h2, a.th_lim2f, lo, hi);
    if (r == 0) return 1;
    bool und = r < 0;
    if (is_if) { r = mac_tri(h2, a.th_if2f, lo, hi); if (r == 0) return 1; und |= r < 0; }
    if (has_eps) { r = mac_tri(h2, a.th_src2f, lo, hi); if (r == 0) return 1; und |= r < 0; }
    return und ? -1 : 0;
}

__device__ __forceinline__ double dist2(double tx, double ty, double tz, const double* cm) {
    const double dx = __dsub_rn(tx, cm[0]), dy = __dsub_rn(ty, cm[1]), dz = __dsub_rn(tz, cm[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
// FP32 forms: the squared distance of node nid from the target centre (tx,
// ty, tz) in FP64 from the FP64 tree, exactly as the FP64 form computes it.
__device__ __forceinline__ double exact_d2(const WalkArgs& a, int64_t nid, float tx, float ty, float tz) {
    const double2 c01 = __ldg(reinterpret_cast<const double2*>(a.nodes64 + nid));
    const double cm[3] = {c01.x, c01.y, __ldg(&a.nodes64[nid].cmz)};
    return dist2((double)tx, (double)ty, (double)tz, cm);
}

// Radial spread of one accepted node (App. A), prepared by the thread that
// accepted it and applied by the whole CTA, one (node, ray) pair per thread.
// kind 0: W_p(|r_i - d| / h) / S over points lo .. lo+npts-1 (S = sum over
// all points); kind 1: everything on one point (node beyond the last point);
// kind 2: linear split w0, w1 between the two points bracketing d (no point
// inside the W_p support).
template <int MODE>
struct RadialSpread {
    typename Prec<MODE>::real d, a, b;      // kind 0/3: d, 1/h, 1/S; kind 2: -, w0, w1
    typename Prec<MODE>::real alpha, e;
    uint32_t off;                           // first table entry of the node's key
    int16_t lo, npts;
    uint8_t kind, woff;                     // kind 3: raw W_p values kept in the setup thread's row
    uint16_t src;                           //   of the weight scratch, from column woff
};

constexpr int MAXW = 12;                    // W_p values kept per node (longer supports recompute)

// r_i of Eq. 4: in FP32 from its index, i^2 times a power of two (exact, no
// load); in FP64 from the table (an FP64 multiply costs more than the load)
template <typename T>
__device__ __forceinline__ T radius_at(int i, T coef, const double* tab) {
    if constexpr (sizeof(T) == 8) return __ldg(tab + i);
    else return (T)(i * i) * coef;
}

template <int MODE>
__device__ __forceinline__ typename Prec<MODE>::real spread_weight(const RadialSpread<MODE>& n, int j,
                                                                 typename Prec<MODE>::real rcoef, const double* rtab,
                                                                 const typename Prec<MODE>::real* wts, int gauss) {
    using real = typename Prec<MODE>::real;
    if (n.kind == 3) return wts[n.src * MAXW + n.woff + j] * n.b;
    if (n.kind == 0) return radial_w<real>(fabs(radius_at<real>(n.lo + j, rcoef, rtab) - n.d), n.a, gauss) * n.b;
    if (n.kind == 1) return real(1);
    return j == 0 ? n.a : n.b;
}

// W_p normalisation of an accepted node: the support of the kernel on the
// evaluation points and 1/S.  FP32 forms (dtol = bound on the error of d):
// returns true when a discontinuous choice -- d beyond the last point or
// not, or a support that is empty or holds only points within rounding of
// its edge (the normalisation then jumps between one point and the linear
// split) -- is not settled in FP32; radial_setup_exact then takes it in FP64.
template <int MODE>
__device__ __forceinline__ bool radial_setup(const WalkArgs& a, RadialSpread<MODE>& n, typename Prec<MODE>::real d,
                                             int s, typename Prec<MODE>::real* wrow, int gauss, float dtol) {
    using real = typename Prec<MODE>::real;
    const int nr = a.nr;
    const real rc = (MODE == 0) ? (real)a.r_coef : (real)a.r_coeff;
    n.d = d;
    const real rlast = radius_at<real>(nr - 1, rc, a.r);
    if (d >= rlast) {
        n.kind = 1; n.lo = (int16_t)(nr - 1); n.npts = 1; n.a = real(1); n.b = real(1);
        return MODE != 0 && (float)d - dtol < (float)rlast;
    }
    if (MODE != 0 && (float)d + dtol >= (float)rlast) return true;
    const real h = (real)s, inv_h = real(1) / h;
    const real hpar = gauss ? h : inv_h;
    const real reach = real(0.8661) * h + (real)dtol;
    // a point whose kernel argument lies within xtol of sqrt3/2 may fall on
    // the other side of the support's edge in FP64
    const float xtol = MODE != 0 ? 2.f * (dtol + U32 * (2.f * (float)d + (float)reach)) * (float)inv_h + 4.f * U32
                                 : 0.f;
    int n_sure = 0;
    bool near_edge = false;
    const real dlo = d > reach ? d - reach : real(0);
    // floor / ceil of the support's index bounds (i = eta sqrt(2 r), Eq. 4),
    // in FP32 in both forms: an error below one index only widens the range
    // by a point, and the weights themselves are computed in the form's
    // precision (an FP64 square root costs a dozen FP64-pipe instructions)
    const int lo = max((int)floorf((float)a.eta * sqrtf(2.f * (float)dlo)), 0);
    const int hi = min((int)ceilf((float)a.eta * sqrtf(2.f * (float)(d + reach))), nr - 1);
    real S = real(0);
    int first = hi + 1, last = lo - 1;
    const bool keep = MODE == 0 && hi - lo + 1 <= MAXW;
    for (int i = lo; i <= hi; ++i) {
        const real dist = fabs(radius_at<real>(i, rc, a.r) - d);
        const real w = radial_w<real>(dist, hpar, gauss);
        if (keep) wrow[i - lo] = w;
        if (w > real(0)) { S += w; first = min(first, i); last = i; }
        if (MODE != 0) {
            const bool ne = fabsf((float)(dist * inv_h) - (float)S3H_D) <= xtol;
            near_edge |= ne;
            n_sure += (w > real(0) && !ne) ? 1 : 0;
        }
    }
    if (MODE != 0 && near_edge && n_sure == 0) return true;
    if (S > real(0)) {
        n.kind = keep ? 3 : 0; n.woff = (uint8_t)(first - lo);
        n.lo = (int16_t)first; n.npts = (int16_t)(last - first + 1); n.a = hpar; n.b = real(1) / S;
        return false;
    }
    int i = min(max((int)floorf((float)a.eta * sqrtf(2.f * (float)d)), 0), nr - 2);   // a guess, corrected below
    while (i + 1 < nr - 1 && radius_at<real>(i + 1, rc, a.r) <= d) ++i;
    while (i > 0 && radius_at<real>(i, rc, a.r) > d) --i;
    const real ra = radius_at<real>(i, rc, a.r), rb = radius_at<real>(i + 1, rc, a.r);
    n.kind = 2; n.lo = (int16_t)i; n.npts = 2;
    n.a = (rb - d) / (rb - ra);
    n.b = (d - ra) / (rb - ra);
    return false;
}

// The other eps kernels (App. A.3), in FP64 whatever the form: emitting
// nodes are few.  The weights of points lo .. lo+n-1 are p0, p1 (two
// points), a + b k (generalised W_f,3, p0 = a, p1 = b) or a smoothing
// kernel over 1/S (p0).
struct EpsSpread {
    int lo, n, kind;                        // kind 0 two points, 1 linear, 2 W_p, 3 W_g
    double p0, p1, d, h;
};

__device__ __forceinline__ int bracket_d(const double* r, int nr, int eta, double d) {
    int i = min(max((int)floor((double)eta * sqrt(2.0 * d)), 0), nr - 2);
    while (i + 1 < nr - 1 && r[i + 1] <= d) ++i;
    while (i > 0 && r[i] > d) --i;
    return i;
}

// FP32 forms: the radial set-up of an accepted node taken on its FP64
// distance d, when radial_setup could not settle it.  Only the supports
// that FP32 left open reach here (at most two points, both at the edge, or
// none), so the weights are stored explicitly: one point (weight 1), two
// consecutive points, or the linear split between the points bracketing d.
template <int MODE>
__device__ void radial_setup_exact(const WalkArgs& a, RadialSpread<MODE>& n, double d, int s, int gauss) {
    const int nr = a.nr;
    n.d = (float)d;
    if (d >= __ldg(a.r + nr - 1)) {
        n.kind = 1; n.lo = (int16_t)(nr - 1); n.npts = 1; n.a = 1.f; n.b = 1.f;
        return;
    }
    const double h = (double)s, inv_h = 1.0 / h, hpar = gauss ? h : inv_h;
    const double reach = 0.8661 * h;
    const int lo = max((int)floor((double)a.eta * sqrt(2.0 * fmax(d - reach, 0.0))) - 1, 0);
    const int hi = min((int)ceil((double)a.eta * sqrt(2.0 * (d + reach))) + 1, nr - 1);
    int first = -1, cnt = 0;
    double w0 = 0.0, w1 = 0.0, S = 0.0;
    for (int i = lo; i <= hi; ++i) {
        const double w = radial_w<double>(fabs(__ldg(a.r + i) - d), hpar, gauss);
        if (w > 0.0) {
            if (cnt == 0) { first = i; w0 = w; } else if (cnt == 1) { w1 = w; }
            S += w;
            ++cnt;
        }
    }
    if (cnt == 1) { n.kind = 1; n.lo = (int16_t)first; n.npts = 1; n.a = 1.f; n.b = 1.f; return; }
    if (cnt == 2) { n.kind = 2; n.lo = (int16_t)first; n.npts = 2; n.a = (float)(w0 / S); n.b = (float)(w1 / S); return; }
    if (cnt > 2) {                          // not reached (FP32 saw no point well inside); FP32 weights
        n.kind = 0; n.lo = (int16_t)first; n.npts = (int16_t)cnt; n.a = (float)hpar; n.b = (float)(1.0 / S);
        return;
    }
    const int i = bracket_d(a.r, nr, a.eta, d);
    const double ra = __ldg(a.r + i), rb = __ldg(a.r + i + 1);
    n.kind = 2; n.lo = (int16_t)i; n.npts = 2;
    n.a = (float)((rb - d) / (rb - ra));
    n.b = (float)((d - ra) / (rb - ra));
}

// two-point W_f,3: the sum and the flux at r = 0 exact
__device__ void eps_wf3(const double* r, int nr, int eta, double d, EpsSpread& s) {
    s.kind = 0;
    if (d >= r[nr - 1]) { s.lo = nr - 1; s.n = 1; s.p0 = 1.0; return; }
    const int i = bracket_d(r, nr, eta, d);
    if (i == 0) { s.lo = 1; s.n = 1; s.p0 = 1.0; return; }
    const double ri = r[i], rj = r[i + 1];
    const double ia = 1.0 / (ri * ri), ib = 1.0 / (rj * rj), it = 1.0 / (d * d);
    const double w1 = (ia - it) / (ia - ib);
    s.lo = i; s.n = 2; s.p0 = 1.0 - w1; s.p1 = w1;
}

__device__ void eps_setup(const WalkArgs& a, double d, double h, EpsSpread& s) {
    const double* r = a.r;
    const int nr = a.nr, eta = a.eta;
    s.d = d; s.h = h;
    if (a.kern_e == TR_EPS_WF1 || a.kern_e == TR_EPS_WF2) {
        // W_f,1: w_{i+1} / w_i = (d - r_i) / (r_{i+1} - d); W_f,2: the flux also
        // exact at r_{i-1}; both with the flux at r = 0 exact
        const int i = d >= r[nr - 1] ? nr - 1 : bracket_d(r, nr, eta, d);
        if (d >= r[nr - 1] || i == 0 || (a.kern_e == TR_EPS_WF2 && i < 2)) { eps_wf3(r, nr, eta, d, s); return; }
        const double ri = r[i], rj = r[i + 1];
        double w0, w1;
        if (a.kern_e == TR_EPS_WF1) {
            const double ratio = (d - ri) / (rj - d);
            w0 = 1.0 / ((d * d) * (1.0 / (ri * ri) + ratio / (rj * rj)));
            w1 = ratio * w0;
        } else {
            const double rm = r[i - 1];
            const double a11 = 1.0 / (ri * ri), a12 = 1.0 / (rj * rj), b1 = 1.0 / (d * d);
            const double a21 = 1.0 / ((ri - rm) * (ri - rm)), a22 = 1.0 / ((rj - rm) * (rj - rm));
            const double b2 = 1.0 / ((d - rm) * (d - rm));
            const double det = a11 * a22 - a12 * a21;
            w0 = (b1 * a22 - a12 * b2) / det;
            w1 = (a11 * b2 - a21 * b1) / det;
            if (!(w0 >= 0.0 && w1 >= 0.0)) { eps_wf3(r, nr, eta, d, s); return; }
        }
        s.kind = 0; s.lo = i; s.n = 2; s.p0 = w0; s.p1 = w1;
        return;
    }
    if (a.kern_e == TR_EPS_WF3N) {
        // Eq. A8-A10 over the points i >= 1 inside the support
        if (d >= r[nr - 1]) { eps_wf3(r, nr, eta, d, s); return; }
        int lo = -1, n = 0;
        for (int i = 1; i < nr; ++i)
            if (fabs(r[i] - d) < S3H_D * h) { if (lo < 0) lo = i; ++n; }
        if (n <= 2) { eps_wf3(r, nr, eta, d, s); return; }
        double A1 = 0.0, A2 = 0.0;
        for (int k = 0; k < n; ++k) {
            const double rk = r[lo + k];
            A1 += 1.0 / (rk * rk);
            A2 += (double)k / (rk * rk);
        }
        const double b = (1.0 / (d * d) - A1 / (double)n) / (A2 - (double)(n - 1) * A1 / 2.0);
        const double c = 1.0 / (double)n - b * (double)(n - 1) / 2.0;
        if (c < 0.0 || c + b * (double)(n - 1) < 0.0) { eps_wf3(r, nr, eta, d, s); return; }   // linear: ends suffice
        s.kind = 1; s.lo = lo; s.n = n; s.p0 = c; s.p1 = b;
        return;
    }
    // W_p or W_g normalised over the points, as for alpha
    const int gauss = a.kern_e == TR_EPS_WG;
    if (d >= r[nr - 1]) { s.kind = 0; s.lo = nr - 1; s.n = 1; s.p0 = 1.0; return; }
    double S = 0.0;
    int first = nr, last = -1;
    for (int i = 0; i < nr; ++i) {
        const double x = fabs(r[i] - d) / h;
        const double w = gauss ? wg_kernel<double>(x) : wp_kernel<double>(x);
        if (w > 0.0) { S += w; first = min(first, i); last = i; }
    }
    if (S > 0.0) { s.kind = gauss ? 3 : 2; s.lo = first; s.n = last - first + 1; s.p0 = 1.0 / S; return; }
    const int i = bracket_d(r, nr, eta, d);
    s.kind = 0; s.lo = i; s.n = 2;
    s.p0 = (r[i + 1] - d) / (r[i + 1] - r[i]);
    s.p1 = (d - r[i]) / (r[i + 1] - r[i]);
}

__device__ __forceinline__ double eps_weight(const EpsSpread& s, const double* r, int j) {
    if (s.kind == 0) return j == 0 ? s.p0 : s.p1;
    if (s.kind == 1) return s.p0 + s.p1 * (double)j;
    const double x = fabs(r[s.lo + j] - s.d) / s.h;
    return (s.kind == 3 ? wg_kernel<double>(x) : wp_kernel<double>(x)) * s.p0;
}

// eps deposit with a kernel other than the default.
template <int MODE>
__device__ __forceinline__ void deposit_eps_variant(const WalkArgs& a, double* bins_eps, uint32_t off, int ne, double d,
                                                 typename Prec<MODE>::real eps, float scale, int s_edge) {
    using real = typename Prec<MODE>::real;
    const int nr = a.nr;
    EpsSpread sp;
    eps_setup(a, d, (double)s_edge, sp);
    const real inv_m3v = real(1.0) / real(TW);
    for (int k = 0; k < ne; ++k) {
        const uint32_t en = __ldg(a.tent + off + k);
        const int b = (int)(en >> 16) * nr + sp.lo;
        const real wk = (real)(en & 0xffffu) * inv_m3v;
        for (int j = 0; j < sp.n; ++j) {
            const real w = (real)eps_weight(sp, a.r, j);
            if (w != real(0)) bin_atomic_add<MODE>(bins_eps + b + j, wk * w * eps, scale);
        }
    }
}

// Deposit of an emitting node's eps (App. A.3).  Default W_f,3: two points
// r_i <= d < r_{i+1} keeping the sum and the flux at the target exact (a
// continuous function of d).  The other kernels take their FP64 distance
// dvar (in the FP32 forms, from the FP64 tree: their choices jump).
// Emitting nodes are few (they contain a source), so the accepting thread
// does it alone.
template <int MODE, bool VAR>
__device__ void deposit_eps(const WalkArgs& a, double* bins_eps, uint32_t off, int ne,
                            typename Prec<MODE>::real d, typename Prec<MODE>::real eps, float scale, int s_edge,
                            double dvar) {
    using real = typename Prec<MODE>::real;
    const int nr = a.nr;
    if (VAR && a.kern_e != TR_EPS_WF3) {
        deposit_eps_variant<MODE>(a, bins_eps, off, ne, dvar, eps, scale, s_edge);
        return;
    }
    const real* r = (MODE == 0) ? reinterpret_cast<const real*>(a.r) : reinterpret_cast<const real*>(a.rf);
    int i;
    real w0, w1;
    if (d >= r[nr - 1]) {
        i = nr - 2; w0 = real(0); w1 = real(1);
    } else {
        i = min(max((int)floorf((float)a.eta * sqrtf(2.f * (float)d)), 0), nr - 2);   // a guess, corrected below
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
    const real inv_m3 = real(1.0) / real(TW);
    for (int k = 0; k < ne; ++k) {
        const uint32_t en = __ldg(a.tent + off + k);
        const int b = (int)(en >> 16) * nr + i;
        const real wk = (real)(en & 0xffffu) * inv_m3;
        if (w0 != real(0)) bin_atomic_add<MODE>(bins_eps + b, wk * w0 * eps, scale);
        if (w1 != real(0)) bin_atomic_add<MODE>(bins_eps + b + 1, wk * w1 * eps, scale);
    }
}

// 1/a in FP64 by the Newton-Raphson iteration y <- y + y (1 - a y), seeded with
// the correctly rounded FP32 reciprocal: the relative error squares at each
// step (2^-23 -> 2^-46 -> below FP64 rounding), two steps suffice.
__device__ __forceinline__ double recip_nr(double a) {
    const float af = (float)a;
    if (!(fabsf(af) > 1e-30f && fabsf(af) < 1e30f)) return 1.0 / a;
    double y = (double)__frcp_rn(af);
    double e = fma(-a, y, 1.0);
    y = fma(y, e, y);
    e = fma(-a, y, 1.0);
    return fma(y, e, y);
}

// The same after one step: relative error about 2^-46, far below the
// rounding that the inputs of the loss coefficient A zeta_d / F_tot already
// carry, and two FP64 instructions fewer per segment of the sweep.
__device__ __forceinline__ double recip1(double a) {
    const float af = (float)a;
    if (!(fabsf(af) > 1e-30f && fabsf(af) < 1e30f)) return 1.0 / a;
    const double y = (double)__frcp_rn(af);
    return fma(y, fma(-a, y, 1.0), y);
}

// Recombination coefficient per unit volume at point i of a ray.  In the
// FP32 + FP64-sweep form the deposits are FP32, so the coefficient is formed
// in FP32 and widened; the photon budget (Phi_j, its losses and their
// clipping) is FP64.
template <int MODE>
__device__ __forceinline__ double alpha_at(const WalkArgs& a, const double* ba, int i, float inv_scale) {
    if (MODE == 0) return ba[i] * __ldg(a.inv_vol + i);
    return (double)(bin_value_f<MODE>(ba + i, inv_scale) * __ldg(a.inv_volf + i));
}

// Far-to-near sweep of one ray (Sec. 2.5) straight from its bins, by a pair
// of lanes of one warp (gl = 0, 1; gmask = the pair): ba, be, bee are the
// ray's N_R slots of alpha, eps and e (raw deposits).  Lane gl owns the
// ray's source points j with j % 2 == gl and keeps their photon rates Phi_j
// (FP64, in place of their eps slots); the total flux of a segment (zeta_s,
// zeta_d) is summed over the pair with one shuffle.  All of it is FP64
// arithmetic (the FP32 forms' coefficients widened).  The loss of source j
// over segment i is R_ij = (alpha_i + alpha_{i+1}) G_ij zeta_d zeta_s with
// G_ij = (1/2) dV_ij zeta_g,ij (Eq. 14-16), and Phi_j <- max(Phi_j - R_ij,
// 0) (Eq. 13) is one FMA and a test of the sign bit.  GB300 issues FP64 at
// 1/64 of the FP32 rate and a deep chain of dependent FP64 operations per
// segment sets the sweep's time, so the pair halves that chain.  Rays
// without emission cost only the scan for it.  Both lanes return F_0.
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }

constexpr uint64_t EVEN_BITS = 0x5555555555555555ull;   // bits j with j % 2 == 0

template <int MODE>
__device__ double sweep_ray(const WalkArgs& a, const double* ba, double* be, const double* bee, const Scales& sc,
                            int gl, unsigned gmask) {
    const int nr = a.nr;
    uint64_t m0 = 0, m1 = 0;
    for (int j = 2 - gl; j < nr; j += 2) {                    // lane gl scans its parity (j >= 1)
        if (bin_nonzero<MODE>(be + j)) { if (j < 64) m0 |= 1ull << j; else m1 |= 1ull << (j - 64); }
    }
    m0 |= __shfl_xor_sync(gmask, m0, 1);
    m1 |= __shfl_xor_sync(gmask, m1, 1);
    if (!(m0 | m1)) return 0.0;
    const uint64_t sel = EVEN_BITS << gl;                     // the lane's parity (64 is even)
    uint64_t o0 = m0 & sel, o1 = m1 & sel;                    // own live sources
    const double inv4pi = 1.0 / (4.0 * PI_D);
    for (uint64_t w = o0; w; w &= w - 1) { const int j = __ffsll((long long)w) - 1; be[j] = bin_value<MODE>(be + j, sc.eps) * inv4pi; }
    for (uint64_t w = o1; w; w &= w - 1) { const int j = 64 + __ffsll((long long)w) - 1; be[j] = bin_value<MODE>(be + j, sc.eps) * inv4pi; }
    double* ph = be;                                              // Eq. 12
    __syncwarp(gmask);
    const float ia = 1.0f / sc.a, ie = 1.0f / sc.e;
    const int jtop = m1 ? 64 + 63 - __clzll((long long)m1) : 63 - __clzll((long long)m0);
    if (!bee && __popcll((long long)m0) + __popcll((long long)m1) == 1) {
        // a lone source and no e: zeta_s = zeta_d = 1 on every segment, every
        // R_ij >= 0, so clipping once at the end equals clipping per segment
        // (Eq. 13): Phi_0 = max(Phi_j - sum_i bin_i HT[j][i], 0), an FP64 dot
        // product split over the pair
        const double* h = a.HT + (size_t)jtop * nr;
        double s0 = 0.0;
        for (int i = gl; i <= jtop; i += 2)
            s0 = fma((double)(MODE == 0 ? ba[i] : (double)bin_value_f<MODE>(ba + i, ia)), __ldg(h + i), s0);
        s0 += __shfl_xor_sync(gmask, s0, 1);
        const double phi = ph[jtop] - s0;
        return positive(phi) ? phi * __ldg(a.inv_r2 + jtop) : 0.0;
    }
    double a_hi = alpha_at<MODE>(a, ba, jtop, ia);
    for (int i = jtop - 1; i >= 0; --i) {
        const int b = i + 1;                                      // sources strictly beyond r_i
        const uint64_t a0 = (b < 64) ? (o0 & (~0ull << b)) : 0ull;
        const uint64_t a1 = (b <= 64) ? o1 : (o1 & (~0ull << (b - 64)));
        const int own = __popcll((long long)a0) + __popcll((long long)a1);
        const int cnt = own + __shfl_xor_sync(gmask, own, 1);
        if (cnt == 0) {                                           // nothing left beyond r_i on the ray
            if (!__any_sync(gmask, (o0 | o1) != 0ull)) break;
            a_hi = alpha_at<MODE>(a, ba, i, ia);
            continue;
        }
        const double a_lo = alpha_at<MODE>(a, ba, i, ia);
        const double A = a_lo + a_hi;                             // twice the mean coefficient
        if (!bee && cnt == 1) {
            // one source on the segment: zeta_s = 1, and zeta_d = 1 without e
            if (own) {
                const int j = a0 ? __ffsll((long long)a0) - 1 : 64 + __ffsll((long long)a1) - 1;
                const double np = fma(-A, __ldg(a.G + (size_t)i * nr + j), ph[j]);   // Eq. 13-14
                if (positive(np)) ph[j] = np;
                else { ph[j] = 0.0; if (j < 64) o0 &= ~(1ull << j); else o1 &= ~(1ull << (j - 64)); }
            }
        } else {
            const double* id2 = a.ID2 + (size_t)i * nr;
            const double* gi = a.GI + (size_t)i * nr;
            double Fl = 0.0;                                      // Eq. 11 at the segment midpoint
            for (uint64_t w = a0; w; w &= w - 1) { const int j = __ffsll((long long)w) - 1; Fl = fma(ph[j], __ldg(id2 + j), Fl); }
            for (uint64_t w = a1; w; w &= w - 1) { const int j = 64 + __ffsll((long long)w) - 1; Fl = fma(ph[j], __ldg(id2 + j), Fl); }
            const double Ftot = Fl + __shfl_xor_sync(gmask, Fl, 1);
            if (positive(Ftot)) {
                const double inv_F = recip1(Ftot);
                double zd = 1.0;                                  // Eq. 17
                if (bee) {
                    const double ev = alpha_at<MODE>(a, bee, i + 1, ie);
                    if (positive(ev)) zd = fmin(2.0, Ftot * recip_nr(ev));
                }
                const double cf = bee ? A * zd * inv_F : A * inv_F;   // zeta_s = F_j / Ftot (Eq. 16)
                for (uint64_t w = a0; w; w &= w - 1) {
                    const int j = __ffsll((long long)w) - 1;
                    const double np = fma(-cf * __ldg(gi + j), ph[j], ph[j]);   // Eq. 13-14
                    if (positive(np)) ph[j] = np; else { ph[j] = 0.0; o0 &= ~(1ull << j); }
                }
                for (uint64_t w = a1; w; w &= w - 1) {
                    const int j = 64 + __ffsll((long long)w) - 1;
                    const double np = fma(-cf * __ldg(gi + j), ph[j], ph[j]);
                    if (positive(np)) ph[j] = np; else { ph[j] = 0.0; o1 &= ~(1ull << (j - 64)); }
                }
            }
        }
        a_hi = a_lo;
    }
    double F0 = 0.0;                                              // Eq. 10-11 at r = 0
    for (uint64_t w = o0; w; w &= w - 1) { const int j = __ffsll((long long)w) - 1; F0 = fma(ph[j], __ldg(a.inv_r2 + j), F0); }
    for (uint64_t w = o1; w; w &= w - 1) { const int j = 64 + __ffsll((long long)w) - 1; F0 = fma(ph[j], __ldg(a.inv_r2 + j), F0); }
    return F0 + __shfl_xor_sync(gmask, F0, 1);
}

// The sweep of the FP32 form.  The deposits (alpha, e) and the geometric
// factors are FP32 quantities, so each segment's loss R_ij (Eq. 14) is formed
// in FP32.  The emitted budget E_j = eps_j / 4pi (Eq. 12) and the running loss
// L_j = sum of R_ij are carried as unevaluated sums of two FP32 numbers
// (hi + lo, about 48 significant bits; L by compensated addition), so that
// the per-segment work needs no FP64 instruction -- on GB300 FP64 runs at
// 1/64 of the FP32 rate and would make the sweep cost grow with the number
// of sources on a ray.  A source is spent when L_j reaches E_j
// (Phi = max(E - L, 0), Eq. 13).  The cancellation Phi_j = E_j - L_j that
// decides the flux near the ionisation front, the flux F_0 (Eq. 10-11) and
// hence the ionised/neutral classification are done in FP64 at the end of
// the ray.
__device__ __forceinline__ float2 two_sum(float a, float b) {    // Knuth: a + b = s + e exactly
    const float s = a + b;
    const float bp = s - a;
    const float e = (a - (s - bp)) + (b - bp);
    return make_float2(s, e);
}

__device__ __forceinline__ float phi_f(const float2 E, const float2 Lr) {  // E - L to FP32 precision
    return (E.x - Lr.x) + (E.y - Lr.y);
}

// FP32-form sweep of one ray by a group of SG lanes of one warp (gmask):
// lane gl owns the ray's source points j with j % SG == gl and keeps their
// budgets and losses; the total flux of each segment (for zeta_s, zeta_d) is
// summed over the group with shuffles.  All lanes of the group return F_0.
constexpr int SG = 2;
constexpr uint64_t SG_PATTERN = 0x5555555555555555ull;   // bits j with j % 2 == 0

__device__ double sweep_ray_group(const WalkArgs& a, const double* ba, double* be, const double* bee,
                                  const Scales& sc, int gl, unsigned gmask) {
    const int nr = a.nr;
    uint64_t m0 = 0, m1 = 0;
    for (int j = 1 + ((gl + SG - 1) % SG); j < nr; j += SG) {   // lane gl scans j == gl (mod SG)
        if (bin_nonzero<1>(be + j)) { if (j < 64) m0 |= 1ull << j; else m1 |= 1ull << (j - 64); }
    }
    for (int o = 1; o < SG; o <<= 1) {
        m0 |= __shfl_xor_sync(gmask, m0, o);
        m1 |= __shfl_xor_sync(gmask, m1, o);
    }
    if (!(m0 | m1)) return 0.0;
    const uint64_t sel = SG_PATTERN << gl;                    // 64 % SG == 0: same pattern for m1
    const uint64_t o0 = m0 & sel, o1 = m1 & sel;
    const double inv4pi = 1.0 / (4.0 * PI_D);
    float2* E = reinterpret_cast<float2*>(be);
    float2* Ls = reinterpret_cast<float2*>(const_cast<double*>(ba));
    for (int half = 0; half < 2; ++half)
        for (uint64_t w = half ? o1 : o0; w; w &= w - 1) {
            const int j = (half ? 64 : 0) + __ffsll((long long)w) - 1;
            const double v = bin_value<1>(be + j, sc.eps) * inv4pi;   // Eq. 12
            const float hi = (float)v;
            E[j] = make_float2(hi, (float)(v - (double)hi));
        }
    const float ia = 1.0f / sc.a, ie = 1.0f / sc.e;
    const int jtop = m1 ? 64 + 63 - __clzll((long long)m1) : 63 - __clzll((long long)m0);
    float a_hi = bin_value_f<1>(ba + jtop, ia) * __ldg(a.inv_volf + jtop);
    __syncwarp(gmask);                                        // alpha at jtop read before any overwrite
    uint64_t d0 = 0, d1 = 0;                                  // own spent sources
    for (int i = jtop - 1; i >= 0; --i) {
        if (!__any_sync(gmask, ((o0 & ~d0) | (o1 & ~d1)) != 0ull)) break;
        const float a_lo = bin_value_f<1>(ba + i, ia) * __ldg(a.inv_volf + i);
        __syncwarp(gmask);                                    // everyone has read alpha_i
        const int b = i + 1;                                  // source b starts: its loss slot was alpha_b
        if (((b < 64 ? (o0 >> b) : (o1 >> (b - 64))) & 1ull)) Ls[b] = make_float2(0.f, 0.f);
        const uint64_t a0 = (b < 64) ? (o0 & ~d0 & (~0ull << b)) : 0ull;
        const uint64_t a1 = (b <= 64) ? (o1 & ~d1) : (o1 & ~d1 & (~0ull << (b - 64)));
        const float* id2 = a.ID2f + (size_t)i * nr;
        float Fl = 0.f;
        for (int half = 0; half < 2; ++half)
            for (uint64_t w = half ? a1 : a0; w; w &= w - 1) {
                const int j = (half ? 64 : 0) + __ffsll((long long)w) - 1;
                Fl = fmaf(phi_f(E[j], Ls[j]), __ldg(id2 + j), Fl);
            }
        int cnt = __popcll((long long)a0) + __popcll((long long)a1);
        for (int o = 1; o < SG; o <<= 1) {
            Fl += __shfl_xor_sync(gmask, Fl, o);
            cnt += __shfl_xor_sync(gmask, cnt, o);
        }
        if (cnt > 0) {
            const float A = a_lo + a_hi;                      // G carries the 1/2 of the mean
            const bool single = !bee && cnt == 1;             // zeta_s = 1, zeta_d = 1
            float cf = 0.f;
            bool go = true;
            if (!single) {
                if (Fl > 0.f) {
                    float zd = 1.f;                           // Eq. 17
                    if (bee) {
                        const float ev = bin_value_f<1>(bee + i + 1, ie) * __ldg(a.inv_volf + i + 1);
                        if (ev > 0.f) zd = fminf(2.f, __fdividef(Fl, ev));
                    }
                    cf = __fdividef(A * zd, Fl);              // zeta_s = F_j / Ftot (Eq. 16)
                } else {
                    go = false;
                }
            }
            if (go) {
                const float* gi = a.GIf + (size_t)i * nr;
                const float* g = a.Gf + (size_t)i * nr;
                for (int half = 0; half < 2; ++half)
                    for (uint64_t w = half ? a1 : a0; w; w &= w - 1) {
                        const int j = (half ? 64 : 0) + __ffsll((long long)w) - 1;
                        const float2 e = E[j];
                        const float2 L = Ls[j];
                        const float R = single ? A * __ldg(g + j) : cf * (__ldg(gi + j) * phi_f(e, L));   // Eq. 14
                        const float2 t = two_sum(L.x, R);     // compensated L += R
                        const float2 Ln = two_sum(t.x, t.y + L.y);
                        if (phi_f(e, Ln) > 0.f) Ls[j] = Ln;
                        else if (half) d1 |= 1ull << (j - 64); else d0 |= 1ull << j;   // spent: Phi = 0
                    }
            }
        }
        a_hi = a_lo;
    }
    double F0 = 0.0;                                          // Eq. 10-11 at r = 0, in FP64
    for (int half = 0; half < 2; ++half)
        for (uint64_t w = half ? (o1 & ~d1) : (o0 & ~d0); w; w &= w - 1) {
            const int j = (half ? 64 : 0) + __ffsll((long long)w) - 1;
            const float2 e = E[j];
            const float2 L = Ls[j];
            const double phi = ((double)e.x + (double)e.y) - ((double)L.x + (double)L.y);
            if (phi > 0.0) F0 = fma(phi, __ldg(a.inv_r2 + j), F0);
        }
    for (int o = 1; o < SG; o <<= 1) F0 += __shfl_xor_sync(gmask, F0, o);
    return F0;
}

// Per-target ray tables for the double-FP32 sweep, in shared scratch:
// order[npix] (u16, the ray of each rank), off[npix] (u16, first lane of each
// lane group), cnt[npix] (u8, emitting points of each ray), then four ints:
// the rays with sources, the lanes of the groups, the rays swept by pairs,
// the emitting points of all rays.
constexpr int MAX_NPIX = 12 * 8 * 8;                  // N_side <= 8
constexpr int GROUP_MAX = 32;                         // rays with more points go to lane pairs
constexpr int GROUP_MEAN_MAX = 14;                    // lane groups while a lit ray has at most this many points on average
__host__ __device__ constexpr size_t sweep_hdr_offset(int npix) { return ((size_t)npix * 5 + 3) & ~(size_t)3; }
__host__ __device__ constexpr size_t sweep_scratch_bytes(int npix) { return sweep_hdr_offset(npix) + 16; }

// Lanes given to a ray with c emitting points in a lane group: the next
// power of two.
__device__ __forceinline__ int group_width(int c) { return c <= 1 ? c : 1 << (32 - __clz(c - 1)); }

// Ranks the rays of a target for the double-FP32 sweep, ties by ray index:
// first the rays with more than GROUP_MAX emitting points (swept by lane
// pairs), then the others by decreasing lane-group width, each group's first
// lane recorded (groups sorted by decreasing power-of-two width never
// straddle a warp), rays without sources last.  Deterministic: the ranks
// depend only on the bins.
template <int NT>
__device__ __forceinline__ void rank_rays(const WalkArgs& a, const double* bins_eps, unsigned char* scratch) {
    const int npix = a.npix, nr = a.nr, tid = threadIdx.x;
    uint16_t* order = reinterpret_cast<uint16_t*>(scratch);
    uint16_t* off = order + npix;
    uint8_t* cnt = reinterpret_cast<uint8_t*>(off + npix);
    int* hdr = reinterpret_cast<int*>(scratch + sweep_hdr_offset(npix));
    for (int k = tid; k < npix; k += NT) {
        const double* be = bins_eps + (size_t)k * nr;
        int c = 0;
        for (int j = 1; j < nr; ++j) c += bin_nonzero<1>(be + j) ? 1 : 0;
        cnt[k] = (uint8_t)c;
    }
    __syncthreads();                                          // counts visible
    auto key = [](int c) { return c > GROUP_MAX ? 2 * GROUP_MAX : group_width(c); };
    for (int k = tid; k < npix; k += NT) {
        const int ck = key(cnt[k]);
        int rank = 0, lanes = 0, nz = 0, total = 0, nbig = 0, npts = 0;
        for (int k2 = 0; k2 < npix; ++k2) {
            const int c2 = cnt[k2], key2 = key(c2);
            const bool before = key2 > ck || (key2 == ck && k2 < k);
            const int w2 = c2 > GROUP_MAX ? 0 : key2;
            rank += before ? 1 : 0;
            lanes += before ? w2 : 0;
            total += w2;
            nz += c2 > 0 ? 1 : 0;
            nbig += c2 > GROUP_MAX ? 1 : 0;
            npts += c2;
        }
        order[rank] = (uint16_t)k;
        off[rank] = (uint16_t)lanes;
        if (k == 0) { hdr[0] = nz; hdr[1] = total; hdr[2] = nbig; hdr[3] = npts; }
    }
    __syncthreads();                                          // ranks visible
}

// Double-FP32 sweep of the rays of a target with 1..GROUP_MAX emitting
// points, a lane per point (a lane per point spends less on bookkeeping than
// a lane pair looping over a ray's points, but idles on the points not yet
// reached; it wins while rays carry few points): the rays' lane groups (rank order, group_width
// lanes each) are laid end to end over the CTA's warps, and lane `slot` of a
// ray's group keeps the ray's slot-th emitting point in registers: its
// budget E_j = eps_j / 4pi and running loss L_j as unevaluated FP32 pairs
// (Eq. 12-14, as in sweep_ray_group), with the segments swept far to near in
// lockstep over the warp.  A segment's total flux (zeta_s, zeta_d; Eq.
// 16-17) is a butterfly sum over the group, the same in every lane of it.  A
// ray with one point and no e has zeta_s = zeta_d = 1, R_ij = A_i G_ij.
// Each group's first lane returns its ray's F_0 (FP64) in the sum.
template <int NT>
__device__ double sweep_groups(const WalkArgs& a, const double* bins_a, const double* bins_eps, const double* bins_e,
                               const Scales& sc, const unsigned char* scratch) {
    const int npix = a.npix, nr = a.nr, lane = threadIdx.x & 31;
    const uint16_t* order = reinterpret_cast<const uint16_t*>(scratch);
    const uint16_t* off = order + npix;
    const uint8_t* cnt = reinterpret_cast<const uint8_t*>(off + npix);
    const int* hdr = reinterpret_cast<const int*>(scratch + sweep_hdr_offset(npix));
    const int nz = hdr[0], T = hdr[1], nbig = hdr[2];
    const double inv4pi = 1.0 / (4.0 * PI_D);
    const float ia = 1.0f / sc.a, ie = 1.0f / sc.e;
    double Fk = 0.0;
    for (int base = threadIdx.x & ~31; base < T; base += NT) {  // warp-uniform
        const int p = base + lane;
        const bool in = p < T;
        int g = nbig;                                         // the last rank whose group starts at or before p
        if (in) {
            int hi = nz - 1;
            while (g < hi) {
                const int mid = (g + hi + 1) >> 1;
                if ((int)off[mid] <= p) g = mid; else hi = mid - 1;
            }
        }
        const int k = in ? order[g] : 0;
        const int c = in ? cnt[k] : 0;
        const int w = group_width(c);
        const int slot = in ? p - (int)off[g] : 0;
        const double* ba = bins_a + (size_t)k * nr;
        const double* be = bins_eps + (size_t)k * nr;
        const double* bee = bins_e ? bins_e + (size_t)k * nr : nullptr;
        int jA = 0, jtop = 0;                                 // own point, the ray's farthest
        if (in) {
            int n = 0;
            for (int j = 1; j < nr; ++j)
                if (bin_nonzero<1>(be + j)) {
                    if (n == slot) jA = j;
                    jtop = j;
                    ++n;
                }
        }
        const bool vA = slot < c;
        float2 EA = make_float2(0.f, 0.f), LA = EA;
        if (vA) { const double v = bin_value<1>(be + jA, sc.eps) * inv4pi; EA.x = (float)v; EA.y = (float)(v - (double)EA.x); }
        bool sA = !vA;                                        // spent, or no point
        const bool single = c == 1 && !bee;                   // zeta_s = zeta_d = 1 throughout
        const int wmax = __reduce_max_sync(FULL, (unsigned)w);
        const int itop = __reduce_max_sync(FULL, (unsigned)jtop);
        float a_hi = in ? bin_value_f<1>(ba + itop, ia) * __ldg(a.inv_volf + itop) : 0.f;
        for (int i = itop - 1; i >= 0; --i) {
            if (!__any_sync(FULL, !sA)) break;                // every point of the warp spent
            const float a_lo = in ? bin_value_f<1>(ba + i, ia) * __ldg(a.inv_volf + i) : 0.f;
            const bool live = !sA && jA > i;
            const float ph = live ? phi_f(EA, LA) : 0.f;
            float Fl = live ? ph * __ldg(a.ID2f + (size_t)i * nr + jA) : 0.f;   // Eq. 11 at the segment midpoint
            for (int o = 1; o < wmax; o <<= 1) {
                const float t = __shfl_xor_sync(FULL, Fl, o);
                if (o < w) Fl += t;
            }
            if (live) {                                       // then Fl > 0
                const float A = a_lo + a_hi;                  // G carries the 1/2 of the mean
                float R;
                if (single) {
                    R = A * __ldg(a.Gf + (size_t)i * nr + jA);                       // Eq. 14
                } else {
                    float zd = 1.f;                           // Eq. 17
                    if (bee) {
                        const float ev = bin_value_f<1>(bee + i + 1, ie) * __ldg(a.inv_volf + i + 1);
                        if (ev > 0.f) zd = fminf(2.f, __fdividef(Fl, ev));
                    }
                    R = __fdividef(A * zd, Fl) * (__ldg(a.GIf + (size_t)i * nr + jA) * ph);   // zeta_s = F_j / Ftot
                }
                const float2 t = two_sum(LA.x, R);            // compensated L += R
                const float2 Ln = two_sum(t.x, t.y + LA.y);
                if (phi_f(EA, Ln) > 0.f) LA = Ln; else sA = true;   // spent: Phi = 0 (Eq. 13)
            }
            a_hi = a_lo;
        }
        double F0 = 0.0;                                      // Eq. 10-11 at r = 0, in FP64
        if (!sA) {
            const double phi = ((double)EA.x + (double)EA.y) - ((double)LA.x + (double)LA.y);
            if (phi > 0.0) F0 = fma(phi, __ldg(a.inv_r2 + jA), F0);
        }
        for (int o = 1; o < wmax; o <<= 1) {
            const double t = __shfl_xor_sync(FULL, F0, o);
            if (o < w) F0 += t;
        }
        if (in && slot == 0) Fk += F0;
    }
    return Fk;
}

// Sum over the rays of one target (Eq. 18).  FP64 sweeps (FP64 form and
// FP32 + FP64-sweep form): a pair of consecutive lanes per ray -- GB300
// charges an FP64 warp instruction in full however few lanes it has, so the
// FP64 work is packed onto consecutive lanes.  Double-FP32 sweep, ranked by
// rank_rays: a target whose lit rays carry more than GROUP_MEAN_MAX emitting
// points on average is swept by lane pairs (sweep_ray_group); otherwise its
// rays with more than GROUP_MAX points by lane pairs and the others a lane per
// point (sweep_groups).  The choice depends only on the bins.  `scratch` holds
// sweep_scratch_bytes(npix) bytes of shared memory; all threads call.
template <int MODE, int NT>
__device__ __forceinline__ double sweep_rays(const WalkArgs& a, double* bins_a, double* bins_eps, double* bins_e,
                                             const Scales& sc, unsigned char* scratch) {
    const int nr = a.nr, tid = threadIdx.x, lane = tid & 31;
    double Fk = 0.0;
    if constexpr (MODE != 2) {
        const int gl = tid & 1;
        const unsigned gmask = 3u << (lane & ~1);
        for (int k = tid >> 1; k < a.npix; k += NT / 2) {
            const double f = sweep_ray<MODE>(a, bins_a + k * nr, bins_eps + k * nr, a.use_e ? bins_e + k * nr : nullptr,
                                             sc, gl, gmask);
            if (gl == 0) Fk += f;
        }
        return Fk;
    } else {
    rank_rays<NT>(a, bins_eps, scratch);
    const uint16_t* order = reinterpret_cast<const uint16_t*>(scratch);
    const int* hdr = reinterpret_cast<const int*>(scratch + sweep_hdr_offset(a.npix));
    const int gl = tid % SG;
    const unsigned gmask = ((1u << SG) - 1u) << (lane & ~(SG - 1));
    if (hdr[3] > GROUP_MEAN_MAX * hdr[0]) {
        // many points per ray: every ray by lane pairs, in ray order (ranked
        // order would put the heaviest rays in one warp, which then holds
        // the CTA's barrier)
        for (int k = tid / SG; k < a.npix; k += NT / SG) {
            const double f = sweep_ray_group(a, bins_a + k * nr, bins_eps + k * nr,
                                             a.use_e ? bins_e + k * nr : nullptr, sc, gl, gmask);
            if (gl == 0) Fk += f;
        }
        return Fk;
    }
    // the pair-swept rays round-robin over the warps, so that no warp holds
    // the CTA's barrier with all of them
    constexpr int NW = NT / 32;
    const int nbig = hdr[2];
    for (int r = (tid >> 5) + NW * (lane / SG); r < nbig; r += NT / SG) {
        const int k = order[r];
        const double f = sweep_ray_group(a, bins_a + k * nr, bins_eps + k * nr,
                                         a.use_e ? bins_e + k * nr : nullptr, sc, gl, gmask);
        if (gl == 0) Fk += f;
    }
    return Fk + sweep_groups<NT>(a, bins_a, bins_eps, a.use_e ? bins_e : nullptr, sc, scratch);
    }
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;                                                      // valid in thread 0
}

// One CTA of NT threads per target (persistent over targets).  Each step
// pops NT/8 opened nodes and evaluates their NT children, one per thread.
// Per-thread walk counters go to the job's counters (one atomic per warp).
struct WalkCounters {
    unsigned long long vis = 0, acc = 0, ent = 0;
    unsigned fb_mac = 0, fb_dep = 0;        // FP32 forms: decisions re-taken in FP64
};

__device__ __forceinline__ void flush_counters(const WalkArgs& a, WalkCounters& c) {
    unsigned long long fm = c.fb_mac, fd = c.fb_dep;
    for (int o = 16; o > 0; o >>= 1) {
        c.vis += __shfl_xor_sync(FULL, c.vis, o);
        c.acc += __shfl_xor_sync(FULL, c.acc, o);
        c.ent += __shfl_xor_sync(FULL, c.ent, o);
        fm += __shfl_xor_sync(FULL, fm, o);
        fd += __shfl_xor_sync(FULL, fd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.stats + 0, c.vis);
        atomicAdd(a.stats + 1, c.acc);
        atomicAdd(a.stats + 2, c.ent);
        if (fm) atomicAdd(a.stats + 3, fm);
        if (fd) atomicAdd(a.stats + 4, fd);
    }
    c = WalkCounters();
}

// One CTA of NT threads per target, persistent over the targets of a list of
// jobs (a job = one tree and a range or list of its cells).  Several trees in
// one launch is how independent requests are batched together.  Each step
// pops NT/8 opened nodes and evaluates their NT children, one per thread.
// VAR: the kernel choices other than W_p / W_f,3 and the periodic and
// corner-of-symmetry boundaries are compiled in (a separate instantiation,
// so that the default walk keeps its registers).
// OUT: OUT_FUSED walk + map + sweep; OUT_DUMP keeps the raw bins and
// accepted ids; OUT_CD column-density maps (no radial points, no sweep).
constexpr int OUT_FUSED = 0, OUT_DUMP = 1, OUT_CD = 2;

// Column-density map deposit of an accepted node (cdMaps): each table entry
// (ray k, volume fraction w_k) adds w_k m / (Omega d^2).
template <int MODE>
__device__ __forceinline__ void deposit_cd(const WalkArgs& a, double* bins, uint32_t off, int ne,
                                           typename Prec<MODE>::real m, typename Prec<MODE>::real d) {
    const double md = (double)m / (a.cd_omega * ((double)d * (double)d));
    const double inv_m3 = 1.0 / (double)TW;
    for (int k = 0; k < ne; ++k) {
        const uint32_t en = __ldg(a.tent + off + k);
        atomicAdd(bins + (en >> 16), ((double)(en & 0xffffu) * inv_m3) * md);
    }
}

template <int MODE, int OUT, int NT, bool VAR>
__device__ __forceinline__ void walk_body(const WalkArgs* __restrict__ jobs, const int64_t* __restrict__ job_end,
                                          int n_jobs, unsigned int* counter) {
    using real = typename Prec<MODE>::real;
    constexpr int NW = NT / 32, P = NT / 8;
    constexpr bool DUMP = OUT == OUT_DUMP, CD = OUT == OUT_CD;
    extern __shared__ __align__(16) unsigned char smem[];
    // per step: stack pushes, and spread nodes (high word) with their
    // (node, ray) pairs (low word), reserved by one atomic per warp; two
    // sets, by step parity, so that a set is cleared a step after its use
    __shared__ int s_push[2];
    __shared__ unsigned long long s_spread[2];
    __shared__ int s_over;
    __shared__ double s_red[NW];
    __shared__ unsigned int s_q;
    __shared__ int s_j;
    __shared__ int s_nacc;
    __shared__ __align__(16) WalkArgs s_a;                       // the current job
    __shared__ RadialSpread<MODE> s_node[NT];                    // the step's nodes to spread
    static_assert(sizeof(RadialSpread<MODE>) * NT >= sweep_scratch_bytes(MAX_NPIX), "sweep scratch in s_node");
    __shared__ int s_pair0[NT + 1];                              // their first (node, ray) pair
    // W_p values kept by the setup threads: the FP64 form saves recomputing
    // them in FP64; in the FP32 form recomputing is cheaper than the shared
    // memory (occupancy) they would take
    __shared__ real s_w[MODE == 0 ? NT * MAXW : 1];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const WalkArgs& a = s_a;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const real inv_m3 = real(1.0) / real(TW);
    const int64_t total = job_end[n_jobs - 1];
    WalkCounters cnt;                                        // per-thread counters
    float kap = 0.f;                                         // FP32 forms: the tree's kappa
    int cur = -1;
    int nr = 0, nbins = 0, nq = 2, N = 0, L = 0;
    double *bins_a = nullptr, *bins_eps = nullptr, *bins_e = nullptr;
    uint32_t* stack = nullptr;
    real rcoef = real(0);
    Scales sc{1.f, 1.f, 1.f};

    for (;;) {
        if (tid == 0) {
            const unsigned int qq = atomicAdd(counter, 1u);
            int j = -1;
            if ((int64_t)qq < total) { j = 0; while (job_end[j] <= (int64_t)qq) ++j; }
            s_q = qq;
            s_j = j;
        }
        __syncthreads();
        const int j = s_j;
        const int64_t qg = (int64_t)s_q;
        if (j < 0) break;
        if (j != cur) {                                          // load the job (uniform over the CTA)
            if (cur >= 0) flush_counters(a, cnt);
            __syncthreads();
            const int* src = reinterpret_cast<const int*>(jobs + j);
            int* dst = reinterpret_cast<int*>(&s_a);
            for (int k = tid; k < (int)(sizeof(WalkArgs) / sizeof(int)); k += NT) dst[k] = src[k];
            __syncthreads();
            cur = j;
            nr = a.nr; nbins = CD ? a.npix : a.npix * nr; nq = CD ? 1 : (a.use_e ? 3 : 2); N = a.N; L = a.L;
            bins_a = reinterpret_cast<double*>(smem);
            bins_eps = bins_a + nbins;
            bins_e = a.use_e ? bins_eps + nbins : nullptr;
            stack = reinterpret_cast<uint32_t*>(bins_a + (size_t)nq * nbins);
            rcoef = (MODE == 0) ? (real)a.r_coef : (real)a.r_coeff;
            if (MODE != 0) {                                     // fixed-point units from the root totals
                real cm0[3], m0, q0[3], mi0;
                load_node<MODE>(a.nodes, 0, cm0, m0, q0, mi0);
                sc.a = fixed_scale((float)q0[0]);
                sc.eps = fixed_scale((float)q0[1]);
                sc.e = fixed_scale((float)q0[2]);
                kap = __ldg(a.kappa) * 1.000001f;
            }
        }
        const int64_t q = qg - (j > 0 ? job_end[j - 1] : 0);    // index within the job
        if (a.targets) {                                         // caller's list: reject bad indices
            const int64_t c = a.targets[q];
            if (c < 0 || c >= a.n_cells) {                       // (uniform over the CTA)
                if (tid == 0) atomicAdd(a.status + 2, 1);
                __syncthreads();                                 // s_q, s_j read before thread 0 rewrites them
                continue;
            }
        }
        int tx, ty, tz;                                          // target corner (finest cells)
        int ts = 1, tl = L;                                      // its edge and level
        int64_t cell;
        if (a.blk) {                                             // AMR: cell c of block b
            int b, lx, ly, lz;
            if (a.targets) {
                cell = a.targets[q];
                b = (int)(cell >> 9);
                const int c = (int)(cell & 511);
                lx = c & 7; ly = (c >> 3) & 7; lz = c >> 6;
            } else {
                const int64_t k = a.first + q;
                b = (int)__ldg(a.blk_order + (k >> 9));
                const uint32_t lm = (uint32_t)(k & 511);
                lx = (int)compact3(lm); ly = (int)compact3(lm >> 1); lz = (int)compact3(lm >> 2);
                cell = ((int64_t)b << 9) + (lz * 8 + ly) * 8 + lx;
            }
            const int4 bm = __ldg(a.blk + b);
            tl = bm.x;
            ts = N >> tl;
            tx = (8 * bm.y + lx) * ts; ty = (8 * bm.z + ly) * ts; tz = (8 * bm.w + lz) * ts;
        } else if (a.targets) {
            cell = a.targets[q];
            tx = (int)(cell % N); ty = (int)((cell / N) % N); tz = (int)(cell / ((int64_t)N * N));
        } else {
            const uint32_t m = (uint32_t)(a.first + q);
            tx = (int)compact3(m); ty = (int)compact3(m >> 1); tz = (int)compact3(m >> 2);
            cell = ((int64_t)tz * N + ty) * N + tx;
        }
        const real hts = real(0.5) * (real)ts;
        const real px = (real)tx + hts, py = (real)ty + hts, pz = (real)tz + hts;
        for (int b = tid; b < nq * nbins; b += NT) bins_a[b] = 0.0;
        if (tid == 0) {                                          // the root, opened
            stack[0] = 0u; s_nacc = 0;
            s_push[0] = s_push[1] = 0; s_spread[0] = s_spread[1] = 0ull; s_over = 0;
        }
        int top = 1, max_top = 1, par = 0;
        bool overflow = false;
        __syncthreads();
        // corner of symmetry: the original and its 7 mirror images (bit k of
        // img mirrors axis k through the low corner), all onto the same rays
        const int n_img = (VAR && a.bc == TR_BC_CORNER) ? 8 : 1;
        for (int img = 0; img < n_img && !overflow; ++img) {
        if (img > 0) {
            if (tid == 0) stack[0] = ROOT_EVAL;
            top = 1;
            __syncthreads();                                     // the image's root visible
        }
        while (top > 0) {
            const int np = min(P, top);
            const int pi = tid >> 3, c = tid & 7;
            const uint32_t pe = (pi < np) ? stack[top - np + pi] : 0u;
            __syncthreads();                                     // parents read before the pushes
            top -= np;
            int action = 0;                                      // 1 open, 2 accept
            int lev = 0, ne = 0;
            uint32_t mort = 0;
            RadialSpread<MODE> node;
            bool spread = false;
            // ROOT_EVAL: the root itself is evaluated (a mirror image does not
            // contain the target, so its root is subject to the MACs)
            if (pi < np && (!VAR || pe != ROOT_EVAL || c == 0)) {
                ++cnt.vis;
                lev = (VAR && pe == ROOT_EVAL) ? 0 : (int)(pe >> 27) + 1;
                mort = (VAR && pe == ROOT_EVAL) ? 0u : (((pe & 0x7ffffffu) << 3) | (uint32_t)c);
                const int s = N >> lev;
                const int cx = (int)compact3(mort) * s, cy = (int)compact3(mort >> 1) * s,
                          cz = (int)compact3(mort >> 2) * s;
                const bool contains = img == 0 && (tx >= cx && tx < cx + s) && (ty >= cy && ty < cy + s) &&
                                      (tz >= cz && tz < cz + s);
                const int64_t nid = level_offset(lev) + mort;
                const bool leaf = a.flags ? (__ldg(a.flags + nid) == NODE_LEAF) : (lev == L);
                if (contains) {
                    action = leaf ? 0 : 1;                       // a leaf holding the target is the target
                } else {
                    real cm[3], m, qv[3], mion;
                    load_node<MODE>(a.nodes, nid, cm, m, qv, mion);
                    // offset o = 2 (node centre - target centre) in half cells of the node
                    // copy that the boundary puts next to the target, and the target
                    // centre to measure that copy's distance from in the node's frame
                    int ox = 2 * cx + s - 2 * tx - ts, oy = 2 * cy + s - 2 * ty - ts, oz = 2 * cz + s - 2 * tz - ts;
                    real qx = px, qy = py, qz = pz;
                    if (VAR && a.bc != TR_BC_ISOLATED) {
                        bc_frame<real>(a.bc, img & 1, N, 2 * cx + s, 2 * tx + ts, px, ox, qx);
                        bc_frame<real>(a.bc, (img >> 1) & 1, N, 2 * cy + s, 2 * ty + ts, py, oy, qy);
                        bc_frame<real>(a.bc, (img >> 2) & 1, N, 2 * cz + s, 2 * tz + ts, pz, oz, qz);
                    }
                    real d2;
                    float B = 0.f;                       // FP32 forms: bound on |d2 - d2 in FP64|
                    if constexpr (MODE == 0) {
                        d2 = dist2(qx, qy, qz, cm);
                    } else {
                        // centre of mass - target = o/2 + offset (a mirror image
                        // of the corner of symmetry mirrors the offset too)
                        const bool mir = VAR && a.bc == TR_BC_CORNER;
                        const float ex = fmaf(0.5f, (float)ox, (mir && (img & 1)) ? -cm[0] : cm[0]);
                        const float ey = fmaf(0.5f, (float)oy, (mir && (img & 2)) ? -cm[1] : cm[1]);
                        const float ez = fmaf(0.5f, (float)oz, (mir && (img & 4)) ? -cm[2] : cm[2]);
                        d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        B = d2_err_bound(d2, kap * (float)s);
                    }
                    const real h2 = (real)s * (real)s;
                    bool open = false;
                    if (!leaf) {
                        if constexpr (MODE == 0) {
                            open = must_open(h2, d2, m, mion, qv[1], a);
                        } else {
                            const int r = mac_f32(h2, d2, B, signbit(mion), qv[1] > 0.f, a);
                            if (r < 0) {
                                ++cnt.fb_mac;
                                open = must_open_exact((double)h2, exact_d2(a, nid, qx, qy, qz), signbit(mion),
                                                       qv[1] > 0.f, a);
                            } else {
                                open = r == 1;
                            }
                        }
                    }
                    if (open) {
                        action = 1;
                    } else if (CD) {
                        action = 2;
                        if (m > real(0)) {
                            const uint2 hd = __ldg(a.hdr + table_key(ox, oy, oz, s));
                            cnt.ent += hd.y;
                            deposit_cd<MODE>(a, bins_a, hd.x, (int)hd.y, m, sqrt(d2));
                        }
                    } else {
                        action = 2;
                        const real d = sqrt(d2);
                        // FP32 forms: |d - d64| <= dtol; the choices that jump
                        // with d and lie closer than that are taken on d64
                        const float dtol = MODE != 0 ? B / (float)d + 4.f * U32 * (float)d : 0.f;
                        double d64 = -1.0;
                        auto exact_d = [&]() -> double {
                            if (d64 < 0.0) { d64 = sqrt(exact_d2(a, nid, qx, qy, qz)); ++cnt.fb_dep; }
                            return d64;
                        };
                        bool in_reach;
                        if constexpr (MODE == 0) {
                            in_reach = d <= a.lray;
                        } else {
                            if ((float)d + dtol < a.lrayf * (1.f - 2.f * U32)) in_reach = true;
                            else if ((float)d - dtol > a.lrayf * (1.f + 2.f * U32)) in_reach = false;
                            else in_reach = exact_d() <= a.lray;
                        }
                        const bool has_ae = qv[0] != real(0) || (a.use_e && qv[2] != real(0));
                        if (in_reach && (has_ae || qv[1] != real(0))) {
                            const int key = table_key(ox, oy, oz, s);
                            const uint2 hd = __ldg(a.hdr + key);
                            ne = (int)hd.y;
                            cnt.ent += ne;
                            if (qv[1] != real(0)) {
                                const double dvar = (MODE != 0 && VAR && a.kern_e != TR_EPS_WF3) ? exact_d() : (double)d;
                                deposit_eps<MODE, VAR>(a, bins_eps, hd.x, ne, d, qv[1], sc.eps, s, dvar);
                            }
                            if (has_ae && ne > 0) {
                                const int gauss = VAR ? a.kern_a : 0;
                                if (radial_setup<MODE>(a, node, d, s, s_w + tid * MAXW, gauss, dtol)) {
                                    if constexpr (MODE != 0) radial_setup_exact<MODE>(a, node, exact_d(), s, gauss);
                                }
                                node.src = (uint16_t)tid;
                                node.alpha = qv[0];
                                node.e = a.use_e ? qv[2] : real(0);
                                node.off = hd.x;
                                spread = true;
                            }
                        }
                    }
                }
            }
            // stack slots of the pushes and spread-list slots of the nodes to
            // spread: one shared atomic per warp reserves them (the order of
            // the warps' blocks is immaterial: fixed-point or FP64 atomic
            // deposits, accepted nodes a set)
            const unsigned om = __ballot_sync(FULL, action == 1);
            const unsigned bm = __ballot_sync(FULL, spread);
            // work items of this thread's node: (ray, point) triples (FP64) or rays (FP32)
            int pc = spread ? (MODE == 0 ? ne * node.npts : ne) : 0;
            int incl = pc;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int wpairs = __shfl_sync(FULL, incl, 31);      // the warp's pairs
            int obase = 0;
            unsigned long long nbp = 0ull;
            if (lane == 0) {
                if (om) obase = atomicAdd(&s_push[par], __popc(om));
                if (bm) nbp = atomicAdd(&s_spread[par], ((unsigned long long)__popc(bm) << 32) |
                                                          (unsigned long long)(unsigned)wpairs);
            }
            obase = __shfl_sync(FULL, obase, 0);
            nbp = __shfl_sync(FULL, nbp, 0);
            if (action == 1) {
                const int slot = top + obase + __popc(om & lanemask_lt);
                if (slot < a.stack_cap) stack[slot] = ((uint32_t)lev << 27) | mort;
                else s_over = 1;                                 // never written past
            }
            if (spread) {
                const int k = (int)(nbp >> 32) + __popc(bm & lanemask_lt);
                s_node[k] = node;
                s_pair0[k] = (int)(nbp & 0xffffffffull) + incl - pc;
            }
            if (action == 2) {
                ++cnt.acc;
                if (DUMP) {
                    const int slot = atomicAdd(&s_nacc, 1);
                    if (slot < a.acc_cap) a.ids_out[q * a.acc_cap + slot] = (int32_t)(level_offset(lev) + mort);
                }
            }
            __syncthreads();                                     // pushes and spread list visible
            const int ototal = s_push[par];
            const unsigned long long sp = s_spread[par];
            const int ntotal = (int)(sp >> 32), ptotal = (int)(sp & 0xffffffffull);
            overflow = s_over != 0;                              // same value in every thread
            if (tid == 0) { s_push[par ^ 1] = 0; s_spread[par ^ 1] = 0ull; }   // read by all a step ago
            par ^= 1;
            if (overflow) break;
            // spread the step's nodes.  FP64 form: each thread takes a contiguous
            // run of (node, table entry, radial point) triples, so that every
            // thread makes about the same number of deposits.  FP32 form: runs of
            // (node, table entry) pairs with the points in an inner loop (the
            // bookkeeping of the triples costs more than the balance gains there).
            if constexpr (MODE == 0) {
                if (ptotal > 0) {
                    const int chunk = (ptotal + NT - 1) / NT;
                    const int p0 = tid * chunk, p1 = min(p0 + chunk, ptotal);
                    if (p0 < p1) {
                        int k = 0, hi = ntotal - 1;
                        while (k < hi) {
                            const int mid = (k + hi + 1) >> 1;
                            if (s_pair0[mid] <= p0) k = mid; else hi = mid - 1;
                        }
                        RadialSpread<MODE> n = s_node[k];
                        const int li = p0 - s_pair0[k];
                        int e = li / n.npts, j = li - e * n.npts;
                        int ne_k = ((k + 1 < ntotal ? s_pair0[k + 1] : ptotal) - s_pair0[k]) / n.npts;
                        uint32_t en = __ldg(a.tent + n.off + e);
                        int b0 = (int)(en >> 16) * nr + n.lo;
                        real wk = (real)(en & 0xffffu) * inv_m3;
                        for (int p = p0; p < p1; ++p) {
                            const real w = spread_weight<MODE>(n, j, rcoef, a.r, s_w, VAR ? a.kern_a : 0) * wk;
                            if (w != real(0)) {
                                if (n.alpha != real(0)) bin_atomic_add<MODE>(bins_a + b0 + j, w * n.alpha, sc.a);
                                if (a.use_e && n.e != real(0)) bin_atomic_add<MODE>(bins_e + b0 + j, w * n.e, sc.e);
                            }
                            if (++j == n.npts) {                     // next table entry, or next node
                                j = 0;
                                if (++e == ne_k) {
                                    if (p + 1 >= p1) break;
                                    ++k;
                                    n = s_node[k];
                                    e = 0;
                                    ne_k = ((k + 1 < ntotal ? s_pair0[k + 1] : ptotal) - s_pair0[k]) / n.npts;
                                }
                                en = __ldg(a.tent + n.off + e);
                                b0 = (int)(en >> 16) * nr + n.lo;
                                wk = (real)(en & 0xffffu) * inv_m3;
                            }
                        }
                    }
                }
            } else {
                if (ptotal > 0) {
                    const int chunk = (ptotal + NT - 1) / NT;
                    const int p0 = tid * chunk, p1 = min(p0 + chunk, ptotal);
                    if (p0 < p1) {
                        int k = 0, hi = ntotal - 1;
                        while (k < hi) {
                            const int mid = (k + hi + 1) >> 1;
                            if (s_pair0[mid] <= p0) k = mid; else hi = mid - 1;
                        }
                        RadialSpread<MODE> n = s_node[k];
                        int kend = k + 1 < ntotal ? s_pair0[k + 1] : ptotal;
                        for (int p = p0; p < p1; ++p) {
                            if (p >= kend) { ++k; n = s_node[k]; kend = k + 1 < ntotal ? s_pair0[k + 1] : ptotal; }
                            const uint32_t en = __ldg(a.tent + n.off + (p - s_pair0[k]));
                            const int b0 = (int)(en >> 16) * nr + n.lo;
                            const real wk = (real)(en & 0xffffu) * inv_m3;
                            for (int j = 0; j < n.npts; ++j) {
                                const real w = spread_weight<MODE>(n, j, rcoef, a.r, s_w, VAR ? a.kern_a : 0) * wk;
                                if (w == real(0)) continue;
                                if (n.alpha != real(0)) bin_atomic_add<MODE>(bins_a + b0 + j, w * n.alpha, sc.a);
                                if (a.use_e && n.e != real(0)) bin_atomic_add<MODE>(bins_e + b0 + j, w * n.e, sc.e);
                            }
                        }
                    }
                }
            }
            top += ototal;
            max_top = max(max_top, top);
        }
        }                                                        // images
        __syncthreads();                                         // all spreads done
        if (CD) {
            if (tid == 0) atomicMax(a.status + 1, max_top);
            if (overflow) {
                if (tid == 0) atomicAdd(a.status, 1);
                continue;
            }
            double* out = a.cd_out + (size_t)(a.targets ? q : cell) * a.npix;
            for (int k = tid; k < a.npix; k += NT) out[k] = bins_a[k] * a.cd_conv;
            continue;
        }
        // own emission of the target (Sec. 2.5 footnote: target sphere of
        // radius r_tp = half the cell edge)
        real cmt[3], mt, qt[3], miont;
        load_node<MODE>(a.nodes, level_offset(tl) + morton3(tx / ts, ty / ts, tz / ts), cmt, mt, qt, miont);
        const double r_tp2 = 0.25 * (double)ts * (double)ts;
        const double eps_self = (double)qt[1];
        if (tid == 0) atomicMax(a.status + 1, max_top);
        if (overflow) {
            if (tid == 0) {
                atomicAdd(a.status, 1);
                if (a.F) a.F[a.targets ? q : cell] = __longlong_as_double(0x7ff8000000000000LL);
            }
            continue;
        }
        if (DUMP) {                                              // raw bins, as the sweep reads them
            double* out = a.bins_out + (size_t)q * 3 * nbins;
            for (int b = tid; b < nbins; b += NT) {
                out[b] = bins_a[b];
                out[nbins + b] = bins_eps[b];
                out[2 * nbins + b] = a.use_e ? bins_e[b] : 0.0;
            }
            if (tid == 0) {
                a.counts_out[q] = s_nacc;
                a.eps_self_out[q] = eps_self / ((double)ts * (double)ts);   // reaches the centre as for ts = 1
                if (q == 0) { a.scales_out[0] = sc.a; a.scales_out[1] = sc.eps; a.scales_out[2] = sc.e; }
            }
            continue;
        }
        const double Fk = sweep_rays<MODE, NT>(a, bins_a, bins_eps, bins_e, sc,
                                                 reinterpret_cast<unsigned char*>(s_node));
        const double F = block_sum<NT>(Fk, s_red) + eps_self / (4.0 * PI_D * r_tp2);
        if (tid == 0) {
            const int64_t o = a.targets ? q : cell;
            if (a.F) a.F[o] = F * a.Fconv;
            if (a.E) a.E[o] = F * a.Econv;
            if (a.ion) a.ion[o] = (uint8_t)(F > 0.0);
        }
    }
    if (cur >= 0) flush_counters(a, cnt);
}

template <int MODE, int OUT, int NT, bool VAR>
__global__ void __launch_bounds__(NT) k_walk(const WalkArgs* __restrict__ jobs, const int64_t* __restrict__ job_end,
                                            int n_jobs, unsigned int* counter) {
    walk_body<MODE, OUT, NT, VAR>(jobs, job_end, n_jobs, counter);
}

// The double-FP32 form's walk with its CTAs per SM stated: five 128-thread
// CTAs (its lane-group sweep would otherwise take enough registers to drop
// it to four), or one wide CTA (left to the default, the compiler aims at two
// and spills).
template <int MODE, int OUT, int NT, bool VAR>
__global__ void __launch_bounds__(NT, NT == 128 ? 5 : 1) k_walk5(const WalkArgs* __restrict__ jobs, const int64_t* __restrict__ job_end,
                                                 int n_jobs, unsigned int* counter) {
    walk_body<MODE, OUT, NT, VAR>(jobs, job_end, n_jobs, counter);
}

template <int MODE, int OUT, int NT, bool VAR>
constexpr auto walk_kernel() {
    if constexpr (MODE == 2 && !VAR) return &k_walk5<MODE, OUT, NT, VAR>;
    else return &k_walk<MODE, OUT, NT, VAR>;
}

// The same walk with registers capped so that six 128-thread CTAs fit an SM:
// chosen when the ray bins are small enough for six (N_R <= ~30 at N_PIX 48)
// and registers would otherwise hold the SM to five.
template <int MODE, int OUT, int NT, bool VAR>
__global__ void __launch_bounds__(NT, 6) k_walk_cap6(const WalkArgs* __restrict__ jobs,
                                                     const int64_t* __restrict__ job_end, int n_jobs,
                                                     unsigned int* counter) {
    walk_body<MODE, OUT, NT, VAR>(jobs, job_end, n_jobs, counter);
}

// Unfused sweep over bins stored by the dump walk: one CTA per target.
template <int MODE, int NT>
__global__ void __launch_bounds__(NT) k_sweep_stored(WalkArgs a, const double* bins_in, const double* eps_self) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[NT / 32];
    const int tid = threadIdx.x;
    const int nbins = a.npix * a.nr;
    double* bins_a = reinterpret_cast<double*>(smem);
    double* bins_eps = bins_a + nbins;
    double* bins_e = a.use_e ? bins_eps + nbins : nullptr;
    for (int64_t q = blockIdx.x; q < a.n_targets; q += gridDim.x) {
        const double* in = bins_in + (size_t)q * 3 * nbins;
        __syncthreads();
        for (int b = tid; b < nbins; b += NT) {
            bins_a[b] = in[b];
            bins_eps[b] = in[nbins + b];
            if (a.use_e) bins_e[b] = in[2 * nbins + b];
        }
        __syncthreads();
        const double Fk = sweep_rays<MODE, NT>(a, bins_a, bins_eps, bins_e,
                                               Scales{a.scales_in[0], a.scales_in[1], a.scales_in[2]},
                                               smem + (size_t)(a.use_e ? 3 : 2) * nbins * sizeof(double));
        const double F = block_sum<NT>(Fk, s_red) + eps_self[q] / (4.0 * PI_D * 0.25);
        if (tid == 0) {
            if (a.F) a.F[q] = F * a.Fconv;
            if (a.E) a.E[q] = F * a.Econv;
            if (a.ion) a.ion[q] = (uint8_t)(F > 0.0);
        }
    }
}

constexpr int WALK_NT = 128;                // threads per target (one CTA)
// Wide CTAs for targets whose ray bins leave room for fewer than three
// 128-thread CTAs on an SM (N_PIX = 192 with N_R ~ 60 fills most of it):
// one CTA per SM then brings 16 (FP32 form) or 8 (FP64) warps instead of 4.
// The FP64 form keeps NT * 12 W_p values in shared memory, hence 256.
constexpr int WALK_NT_WIDE_F32 = 512;
constexpr int WALK_NT_WIDE_F64 = 256;

// Opened nodes waiting on a target's stack.  The stack never holds more
// than the target's opened nodes (a few hundred at theta = 0.5); overflow
// is detected and reported, never written past.
constexpr int STACK_CAP = 512;

size_t walk_smem(const tr_tree* t) {
    const int nq = t->use_e ? 3 : 2;
    return (size_t)nq * t->npix * t->nr * 8 + (size_t)STACK_CAP * 4;
}

WalkArgs make_args(const tr_tree* t) {
    WalkArgs a{};
    a.nodes = t->nodes;
    a.nodes64 = (const NodeF64*)t->nodes64;
    a.kappa = t->kappa;
    a.N = t->N; a.L = t->L; a.nr = t->nr; a.npix = t->npix; a.eta = t->p.eta_r; a.nside = t->p.nside;
    a.use_e = t->use_e;
    a.stack_cap = STACK_CAP;
    a.th_lim2 = t->p.theta_lim * t->p.theta_lim;
    a.th_if2 = t->p.theta_if * t->p.theta_if;
    a.th_src2 = t->p.theta_src * t->p.theta_src;
    a.lray = t->lray;
    a.r_coef = 1.0 / (2.0 * (double)t->p.eta_r * (double)t->p.eta_r);
    a.r_coeff = (float)a.r_coef;
    a.th_lim2f = (float)a.th_lim2; a.th_if2f = (float)a.th_if2; a.th_src2f = (float)a.th_src2;
    a.lrayf = (float)t->lray;
    a.toff = t->table->off; a.tent = t->table->ent; a.hdr = t->table->hdr;
    a.r = t->sw.r; a.rf = t->sw.rf; a.inv_r2 = t->sw.inv_r2; a.inv_vol = t->sw.inv_vol; a.inv_volf = t->sw.inv_volf;
    a.G = t->sw.G; a.ID2 = t->sw.ID2; a.GI = t->sw.GI; a.Gf = t->sw.Gf; a.ID2f = t->sw.ID2f; a.GIf = t->sw.GIf;
    a.HT = t->sw.HT;
    a.Fconv = t->U / (t->dx * t->dx);
    a.Econv = t->Eu;
    a.status = t->status;
    a.stats = t->stats;
    a.n_cells = t->n_cells;
    a.kern_a = t->p.kernel_alpha;
    a.kern_e = t->p.kernel_eps;
    a.bc = t->p.bc;
    a.flags = t->flags;
    a.blk = t->blk;
    a.blk_order = t->blk_order;
    return a;
}

template <int NT, typename K>
tr_status launch_persistent(K kernel, size_t smem, const WalkArgs* jobs, const int64_t* job_end, int n_jobs,
                            int64_t total, unsigned int* counter, cudaStream_t st) {
    {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa{};
        cudaGetDevice(&dev);
        tr_status c = cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                                 "shared memory limit");
        if (c == TR_OK) c = cuda_check(cudaFuncGetAttributes(&fa, kernel), "kernel attributes");
        if (c != TR_OK) return c;
        if (smem + fa.sharedSizeBytes > (size_t)optin)
            return set_error(TR_EUNSUPPORTED,
                             "ray bins need %zu + %zu bytes of shared memory per target, more than the %d a CTA can have"
                             " (fewer rays, a shorter L_ray or no e_prev)", smem, (size_t)fa.sharedSizeBytes, optin);
    }
    tr_status s = cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "cudaFuncSetAttribute(smem)");
    if (s != TR_OK) return s;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem), "occupancy query");
    if (s != TR_OK) return s;
    if (per_sm < 1) return set_error(TR_EUNSUPPORTED, "ray bins need %zu bytes of shared memory per target", smem);
    s = cuda_check(cudaMemsetAsync(counter, 0, sizeof(unsigned int), st), "counter reset");
    if (s != TR_OK) return s;
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > total) blocks = total > 0 ? total : 1;
    kernel<<<(unsigned)blocks, NT, smem, st>>>(jobs, job_end, n_jobs, counter);
    return cuda_check(cudaGetLastError(), "walk kernel launch");
}

template <int MODE>
bool wide_ctas_m(size_t smem) {
    int per_sm = 0;
    const void* k = (const void*)walk_kernel<MODE, OUT_FUSED, WALK_NT, false>();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WALK_NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return true;                                             // too large for 128 threads: try wide
    }
    return per_sm < 3;
}

bool wide_ctas(int mode, size_t smem) {
    return mode == 0 ? wide_ctas_m<0>(smem) : (mode == 1 ? wide_ctas_m<1>(smem) : wide_ctas_m<2>(smem));
}

// whether the register-capped walk fits more CTAs per SM than the plain one
bool more_ctas_capped(const void* plain, const void* capped, size_t smem) {
    int a = 0, b = 0;
    if (cudaFuncSetAttribute(plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(capped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, plain, WALK_NT, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, capped, WALK_NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return b > a;
}

// The walk kernel of one form and output.  MODE 2 (double-FP32 sweep) only
// differs from MODE 1 in the sweep, so its dump and column-density walks are
// those of MODE 1 (chosen by launch_jobs).
template <int MODE, bool VAR>
tr_status launch_mode(int out, bool wide, size_t smem, const WalkArgs* jobs, const int64_t* job_end, int n_jobs,
                      int64_t total, unsigned int* counter, cudaStream_t st) {
    constexpr int W = MODE == 0 ? WALK_NT_WIDE_F64 : WALK_NT_WIDE_F32, T = WALK_NT;
    constexpr int F = OUT_FUSED;
    if constexpr (MODE != 2) {
        constexpr int D = OUT_DUMP, C = OUT_CD;
        if (out == C) return launch_persistent<T>(walk_kernel<MODE, C, T, VAR>(), smem, jobs, job_end, n_jobs, total, counter, st);
        if (out == D)
            return wide ? launch_persistent<W>(walk_kernel<MODE, D, W, VAR>(), smem, jobs, job_end, n_jobs, total, counter, st)
                        : launch_persistent<T>(walk_kernel<MODE, D, T, VAR>(), smem, jobs, job_end, n_jobs, total, counter, st);
    }
    if (wide) return launch_persistent<W>(walk_kernel<MODE, F, W, VAR>(), smem, jobs, job_end, n_jobs, total, counter, st);
    if constexpr (MODE != 0) {
        if (more_ctas_capped((const void*)walk_kernel<MODE, F, T, VAR>(), (const void*)k_walk_cap6<MODE, F, T, VAR>, smem))
            return launch_persistent<T>(k_walk_cap6<MODE, F, T, VAR>, smem, jobs, job_end, n_jobs, total, counter, st);
    }
    return launch_persistent<T>(walk_kernel<MODE, F, T, VAR>(), smem, jobs, job_end, n_jobs, total, counter, st);
}

template <bool VAR>
tr_status launch_jobs_v(int mode, int out, bool wide, size_t smem, const WalkArgs* jobs, const int64_t* job_end,
                        int n_jobs, int64_t total, unsigned int* counter, cudaStream_t st) {
    if (mode == 0) return launch_mode<0, VAR>(out, wide, smem, jobs, job_end, n_jobs, total, counter, st);
    if (mode == 1 || out != OUT_FUSED)
        return launch_mode<1, VAR>(out, wide, smem, jobs, job_end, n_jobs, total, counter, st);
    return launch_mode<2, VAR>(out, wide, smem, jobs, job_end, n_jobs, total, counter, st);
}

// var: some job uses a kernel choice other than W_p / W_f,3 or a boundary
// other than isolated
tr_status launch_jobs(int mode, int out, bool var, size_t smem, const WalkArgs* jobs, const int64_t* job_end,
                      int n_jobs, int64_t total, unsigned int* counter, cudaStream_t st) {
    const bool wide = out != OUT_CD && wide_ctas(out == OUT_FUSED ? mode : (mode != 0 ? 1 : 0), smem);
    return var ? launch_jobs_v<true>(mode, out, wide, smem, jobs, job_end, n_jobs, total, counter, st)
               : launch_jobs_v<false>(mode, out, wide, smem, jobs, job_end, n_jobs, total, counter, st);
}

bool uses_variants(const tr_tree* t) {
    return t->p.kernel_alpha != TR_KERNEL_WP || t->p.kernel_eps != TR_EPS_WF3 || t->p.bc != TR_BC_ISOLATED;
}

}  // namespace

size_t walk_job_bytes(int n_jobs) { return (size_t)n_jobs * (sizeof(WalkArgs) + sizeof(int64_t)); }

tr_status walk_run(const tr_tree* t, const int64_t* targets, int64_t n_targets, bool dump, const WalkOut& out,
                   cudaStream_t st) {
    WalkArgs a = make_args(t);
    a.targets = targets;
    a.first = 0;
    a.n_targets = n_targets;
    a.F = out.F; a.E = out.e; a.ion = out.ion;
    a.bins_out = out.bins; a.ids_out = out.ids; a.counts_out = out.counts; a.eps_self_out = out.eps_self;
    a.scales_out = out.scales;
    a.acc_cap = out.acc_cap;
    // the job record goes to the tree's job buffer; the copy completes before
    // return (host staging), so the stack record may go away afterwards
    unsigned char host[sizeof(WalkArgs) + sizeof(int64_t)];
    memcpy(host, &a, sizeof(WalkArgs));
    memcpy(host + sizeof(WalkArgs), &n_targets, sizeof(int64_t));
    tr_status s = cuda_check(cudaMemsetAsync(t->status, 0, 4 * sizeof(int32_t), st), "status reset");
    if (s == TR_OK) s = cuda_check(cudaMemsetAsync(t->stats, 0, N_STATS * sizeof(unsigned long long), st), "stats reset");
    if (s == TR_OK) s = cuda_check(cudaMemcpyAsync(t->jobbuf, host, sizeof host, cudaMemcpyHostToDevice, st), "job copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "job copy");
    if (s != TR_OK || n_targets <= 0) return s;
    const WalkArgs* jobs = reinterpret_cast<const WalkArgs*>(t->jobbuf);
    const int64_t* job_end = reinterpret_cast<const int64_t*>(reinterpret_cast<const unsigned char*>(t->jobbuf) + sizeof(WalkArgs));
    return launch_jobs(t->mode, dump ? OUT_DUMP : OUT_FUSED, uses_variants(t), walk_smem(t), jobs, job_end, 1, n_targets,
                       t->counter, st);
}

tr_status cd_run(const tr_tree* t, const int64_t* targets, int64_t n_targets, double* out, cudaStream_t st) {
    WalkArgs a = make_args(t);
    a.targets = targets;
    a.first = 0;
    a.n_targets = n_targets;
    a.cd_out = out;
    a.cd_conv = t->dx;
    a.cd_omega = 4.0 * PI_D / (double)t->npix;
    unsigned char host[sizeof(WalkArgs) + sizeof(int64_t)];
    memcpy(host, &a, sizeof(WalkArgs));
    memcpy(host + sizeof(WalkArgs), &n_targets, sizeof(int64_t));
    tr_status s = cuda_check(cudaMemsetAsync(t->status, 0, 4 * sizeof(int32_t), st), "status reset");
    if (s == TR_OK) s = cuda_check(cudaMemsetAsync(t->stats, 0, N_STATS * sizeof(unsigned long long), st), "stats reset");
    if (s == TR_OK) s = cuda_check(cudaMemcpyAsync(t->jobbuf, host, sizeof host, cudaMemcpyHostToDevice, st), "job copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "job copy");
    if (s != TR_OK || n_targets <= 0) return s;
    const WalkArgs* jobs = reinterpret_cast<const WalkArgs*>(t->jobbuf);
    const int64_t* job_end = reinterpret_cast<const int64_t*>(reinterpret_cast<const unsigned char*>(t->jobbuf) + sizeof(WalkArgs));
    const size_t smem = (size_t)t->npix * 8 + (size_t)STACK_CAP * 4;
    return launch_jobs(t->mode, OUT_CD, uses_variants(t), smem, jobs, job_end, 1, n_targets, t->counter, st);
}

tr_status walk_batch_run(const tr_tree* const* trees, const int64_t* first, const int64_t* count, int n,
                         double* const* F, double* const* e, uint8_t* const* ion, void* jobbuf, unsigned int* counter,
                         cudaStream_t st) {
    std::vector<unsigned char> host(walk_job_bytes(n));
    WalkArgs* hj = reinterpret_cast<WalkArgs*>(host.data());
    int64_t* he = reinterpret_cast<int64_t*>(host.data() + (size_t)n * sizeof(WalkArgs));
    size_t smem = 0;
    int64_t total = 0;
    bool var = false;
    tr_status s = TR_OK;
    for (int i = 0; i < n; ++i) {
        var = var || uses_variants(trees[i]);
        WalkArgs a = make_args(trees[i]);
        a.targets = nullptr;
        a.first = first[i];
        a.n_targets = count[i];
        a.F = F ? F[i] : nullptr; a.E = e ? e[i] : nullptr; a.ion = ion ? ion[i] : nullptr;
        hj[i] = a;
        total += count[i];
        he[i] = total;
        smem = std::max(smem, walk_smem(trees[i]));
        if (s == TR_OK) s = cuda_check(cudaMemsetAsync(trees[i]->status, 0, 4 * sizeof(int32_t), st), "status reset");
        if (s == TR_OK) s = cuda_check(cudaMemsetAsync(trees[i]->stats, 0, N_STATS * sizeof(unsigned long long), st), "stats reset");
    }
    if (s == TR_OK) s = cuda_check(cudaMemcpyAsync(jobbuf, host.data(), host.size(), cudaMemcpyHostToDevice, st), "job copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "job copy");
    if (s != TR_OK || total == 0) return s;
    const WalkArgs* jobs = reinterpret_cast<const WalkArgs*>(jobbuf);
    const int64_t* job_end = reinterpret_cast<const int64_t*>(reinterpret_cast<unsigned char*>(jobbuf) + (size_t)n * sizeof(WalkArgs));
    return launch_jobs(trees[0]->mode, OUT_FUSED, var, smem, jobs, job_end, n, total, counter, st);
}

tr_status sweep_run(const tr_rays* r, double* F, double* e, uint8_t* ion, cudaStream_t st) {
    WalkArgs a{};
    a.nr = r->nr; a.npix = r->npix; a.use_e = r->use_e;
    a.r = r->sw.r; a.inv_r2 = r->sw.inv_r2; a.inv_vol = r->sw.inv_vol; a.inv_volf = r->sw.inv_volf; a.G = r->sw.G; a.ID2 = r->sw.ID2; a.GI = r->sw.GI; a.Gf = r->sw.Gf; a.ID2f = r->sw.ID2f; a.GIf = r->sw.GIf;
    a.HT = r->sw.HT;
    a.n_targets = r->n_targets;
    a.Fconv = r->U / (r->dx * r->dx);
    a.Econv = r->Eu;
    a.F = F; a.E = e; a.ion = ion;
    a.scales_in = r->scales;
    const size_t smem = (size_t)(r->use_e ? 3 : 2) * r->npix * r->nr * 8 + sweep_scratch_bytes(r->npix);
    auto kern = r->mode == 0 ? k_sweep_stored<0, WALK_NT>
                             : (r->mode == 1 ? k_sweep_stored<1, WALK_NT> : k_sweep_stored<2, WALK_NT>);
    tr_status s = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "cudaFuncSetAttribute(sweep smem)");
    if (s != TR_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = r->n_targets < (int64_t)sms * 4 ? r->n_targets : (int64_t)sms * 4;
    if (blocks > 0) kern<<<(unsigned)blocks, WALK_NT, smem, st>>>(a, r->bins, r->eps_self);
    return cuda_check(cudaGetLastError(), "sweep kernel launch");
}

tr_status read_status(const tr_tree* t, cudaStream_t st) {
    int32_t h[4] = {0, 0, 0, 0};
    tr_status s = cuda_check(cudaMemcpyAsync(h, t->status, sizeof h, cudaMemcpyDeviceToHost, st), "status copy");
    if (s == TR_OK) s = cuda_check(cudaStreamSynchronize(st), "walk kernels");
    if (s != TR_OK) return s;
    if (h[2] > 0) return set_error(TR_EINVAL, "%d target index(es) outside [0, %lld)", h[2], (long long)t->n_cells);
    if (h[0] > 0)
        return set_error(TR_EOVERFLOW, "the walk stack overflowed for %d target(s); their outputs are NaN", h[0]);
    return TR_OK;
}

}  // namespace tr
