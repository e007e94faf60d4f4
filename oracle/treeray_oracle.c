/* Plain FP64 CPU oracle for the TreeRay/OnTheSpot hot path
 * (Wuensch et al., "Tree-based solvers for adaptive mesh refinement code
 * FLASH - II: radiation transport module TreeRay", arXiv 2105.09644).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg call this file.  It is slow on purpose: every
 * step is the paper's definition written out, in the paper's order, with no
 * blocking or fusion, so that it can be checked against the paper by eye.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared treeray_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum separately rounded.)
 *
 * Readings of the paper used here (the paper is silent, garbled or
 * inconsistent at these places):
 *  R1 Eq. 1-2: the emission and recombination of a cell are netted and
 *     clipped per cell; node values are plain sums of the clipped cell values.
 *  R2 point sources (radius 0) go to the cell containing them,
 *     floor((x-lo)/dx) clamped to [0, N-1].
 *  R3 d = distance from the target centre to the node mass centre (geometric
 *     centre if the node has no mass); h = node edge; a node that contains
 *     the target is always opened; the target cell itself is never mapped and
 *     contributes its own emission as eps_c / (4 pi r_tp^2), r_tp = dx/2.
 *     Children are visited in Morton order (x fastest).
 *  R4 node->ray weights: the node is an axis-aligned cube; weight of ray k =
 *     fraction of ORC_TM^3 sample points of the cube that fall in HEALPix
 *     pixel k, for a representative cube chosen by an integer key of the
 *     node's geometric-centre offset (cube-map face, (u,v) bin, psi = h/d bin).
 *     A node whose offset ties between two (three) axes for the largest
 *     component gets an edge (corner) key with its representative direction
 *     on that edge (corner); where that direction lies on a plane x = +-y,
 *     each sample counts half in its pixel and half in the mirror pixel, so
 *     that the table -- and the radiation field of a mirror-symmetric scene
 *     (Sec. 3.4: symmetric about x = y) -- keeps the mirror symmetries of
 *     the HEALPix pixels.
 *  R5 W_p (Eq. A2): the printed outer branch violates its own constraints;
 *     it is rebuilt from them: W_p2(x) = (x - sqrt3/2)^2 (a2 x + 2A(2+sqrt3) - a2/2)
 *     with the printed a1, a2, A, M.  W_p is used in |x| and normalised over
 *     the evaluation points; with no point inside the support the node is
 *     split linearly between the two bracketing points.
 *  R6 units on rays: eps_i is a photon rate (the node's share), alpha_i and
 *     e_i are per unit volume, the deposited amount divided by the ray-cell
 *     volume (4pi/N_PIX)(r_{i+1/2}^3 - r_{i-1/2}^3)/3 with shell edges at
 *     midpoints clamped to [0, r_{N-1}].  A node at d >= r_{N-1} goes to the
 *     last point; a node beyond the maximum ray length is not mapped.
 *  R7 the loss over segment [r_i, r_{i+1}] is
 *     1/2 (alpha_i + alpha_{i+1}) dV_{i,j} zeta_d zeta_s zeta_g, with all
 *     sources of the ray processed together per segment, far to near; the
 *     fluxes in zeta_s and zeta_d are taken at the segment midpoint
 *     (F_j = Phi_j / (r_j - r_m)^2) to avoid the singular j = i+1 term;
 *     zeta_s = 0 when the total flux is 0; zeta_d = 1 when e is absent or 0;
 *     the [0,2] truncation applies to zeta_d (Eq. 17).
 *  R8 zeta_g is applied literally (Eq. 16) behind a switch.
 *  R9 delta_cell (Eq. 21) and delta_tot (Eq. 20) use absolute differences;
 *     the median is the lower median.
 *  R10 AMR grids: lengths are in cells of the finest level; a cell of edge
 *     s (finest cells) has volume s^3 and mass n_H s^3; the target sphere of
 *     such a cell has r_tp = s/2; a parent sums its eight children, and a
 *     leaf (an AMR cell) is never opened.
 *  R11 kernel variants (App. A): W_g is normalised over the evaluation points
 *     like W_p, with the same linear split when no point is inside its
 *     support.  The two-point flux kernels W_f,1 / W_f,2 / W_f,3 use the
 *     bracket r_i <= d < r_{i+1}; with d < r_1 everything goes to r_1.
 *     W_f,2 needs r_{i-1} > 0: at i = 1 its two conditions coincide, and
 *     there W_f,3 is used.  The generalised W_f,3 spans the points i >= 1
 *     with |r_i - d| < (sqrt3/2) h; the printed A_2 sums (i - 1)/r_i^2, read
 *     as (offset from the lowest index)/r_i^2, which is what the two
 *     conditions give; with N <= 2 points, or when the linear prescription
 *     makes a weight negative, the two-point W_f,3 is used (emission stays
 *     non-negative and both conditions still hold).
 *  R12 boundaries (Sec. 2.8): periodic takes, for every node that does not
 *     contain the target, the copy whose geometric centre is nearest to the
 *     target centre, per axis, with the offset o in half cells wrapped into
 *     [-N, N) (N finest cells per axis); the distance uses that copy's
 *     centre of mass.  Corner of symmetry puts the corner at the grid's low
 *     corner: the walk runs over the original and its 7 mirror images
 *     (every subset of the axes mirrored through the corner planes), all
 *     deposited onto the same rays; only the original can contain the
 *     target, and the default maximum ray length becomes the diagonal of
 *     the mirrored domain, 2 N sqrt3.
 *  R13 column-density maps (cdMaps, Sec. 2.2; defined in Paper I, which is
 *     not given): the same walk, and each accepted node adds to direction k
 *     its mass times its volume fraction in cone k over the cone's
 *     cross-section at the node, w_k m / (Omega d^2) with Omega = 4 pi /
 *     N_PIX, so that sum_k Omega N_k = sum_n m_n / d_n^2.  All accepted
 *     nodes count (a map has no radial points, so no maximum ray length);
 *     the target cell itself is left out.
 */
#include "treeray_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double ORC_PI = 3.14159265358979323846;
static const double C_LIGHT = 2.99792458e10;   /* cm s^-1 */
static const double DELTA_IF = 1e-8;           /* Sec. 2.4 */

/* ------------------------------------------------------------------------ */
/* HEALPix ring scheme (Gorski et al. 2005), used for the ray directions     */
/* (Sec. 2.2: N_PIX = 12 N_side^2 equal-area pixels).                        */
/* ------------------------------------------------------------------------ */

static int64_t floor_div2(int64_t a) { return (a >= 0) ? a / 2 : -((-a + 1) / 2); }
static int64_t pos_mod(int64_t a, int64_t m) { int64_t r = a % m; return r < 0 ? r + m : r; }

int64_t orc_ang2pix(int32_t nside, double x, double y, double z)
{
    const int64_t ns = nside, nl4 = 4 * ns, ncap = 2 * ns * (ns - 1), npix = 12 * ns * ns;
    double r = sqrt((x * x + y * y) + z * z);
    double zc = z / r;
    double za = fabs(zc);
    double phi = atan2(y, x);
    if (phi < 0.0) phi += 2.0 * ORC_PI;
    double tt = phi / (0.5 * ORC_PI);           /* in [0, 4] */
    if (tt >= 4.0) tt -= 4.0;
    if (za <= 2.0 / 3.0) {                      /* equatorial belt */
        double t1 = (double)ns * (0.5 + tt);
        double t2 = (double)ns * zc * 0.75;
        int64_t jp = (int64_t)floor(t1 - t2);   /* ascending edge line index */
        int64_t jm = (int64_t)floor(t1 + t2);   /* descending edge line index */
        int64_t ir = ns + 1 + jp - jm;          /* ring within the belt, 1..2ns+1 */
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = pos_mod(floor_div2(jp + jm - ns + kshift + 1), nl4);
        return ncap + (ir - 1) * nl4 + ip;
    }
    double tp = tt - floor(tt);                 /* polar caps */
    double tmp = (double)ns * sqrt(3.0 * (1.0 - za));
    int64_t jp = (int64_t)floor(tp * tmp);
    int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
    int64_t ir = jp + jm + 1;                   /* ring counted from the nearer pole */
    int64_t ip = pos_mod((int64_t)floor(tt * (double)ir), 4 * ir);
    if (zc > 0.0) return 2 * ir * (ir - 1) + ip;
    return npix - 2 * ir * (ir + 1) + ip;
}

static int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

void orc_pix2vec(int32_t nside, int64_t pix, double* v3)
{
    const int64_t ns = nside, ncap = 2 * ns * (ns - 1), npix = 12 * ns * ns;
    double z, phi;
    if (pix < ncap) {
        int64_t ir = (1 + isqrt64(1 + 2 * pix)) / 2;
        int64_t iphi = pix + 1 - 2 * ir * (ir - 1);
        z = 1.0 - (double)(ir * ir) / (3.0 * (double)(ns * ns));
        phi = ((double)iphi - 0.5) * ORC_PI / (2.0 * (double)ir);
    } else if (pix < npix - ncap) {
        int64_t ip = pix - ncap;
        int64_t ir = ip / (4 * ns) + ns;
        int64_t iphi = ip % (4 * ns) + 1;
        double fodd = ((ir + ns) & 1) ? 1.0 : 0.5;
        z = (double)(2 * ns - ir) * 2.0 / (3.0 * (double)ns);
        phi = ((double)iphi - fodd) * ORC_PI / (2.0 * (double)ns);
    } else {
        int64_t ip = npix - pix;
        int64_t ir = (1 + isqrt64(2 * ip - 1)) / 2;
        int64_t iphi = 4 * ir + 1 - (ip - 2 * ir * (ir - 1));
        z = -1.0 + (double)(ir * ir) / (3.0 * (double)(ns * ns));
        phi = ((double)iphi - 0.5) * ORC_PI / (2.0 * (double)ir);
    }
    double st = sqrt((1.0 - z) * (1.0 + z));
    v3[0] = st * cos(phi);
    v3[1] = st * sin(phi);
    v3[2] = z;
}

/* ------------------------------------------------------------------------ */
/* Evaluation points on rays (Sec. 2.2, Eq. 4 and Eq. 5).                    */
/* ------------------------------------------------------------------------ */

double orc_radius(int32_t i, int32_t eta_r)
{   /* Eq. 4: r_i = dx i^2 / (2 eta_R^2), dx = 1 cell */
    return (double)((int64_t)i * i) / (2.0 * (double)eta_r * (double)eta_r);
}

int32_t orc_num_points(int32_t eta_r, double lray_cells)
{   /* Eq. 5: N_R = eta_R floor(sqrt(2 L_ray / dx)) + 1 */
    return eta_r * (int32_t)floor(sqrt(2.0 * lray_cells)) + 1;
}

/* ------------------------------------------------------------------------ */
/* Radial kernels (App. A).                                                  */
/* ------------------------------------------------------------------------ */

double orc_wp(double x)
{   /* Eq. A2 with a1 = 1.21, a2 = -6.35, A = 4.08, M = 1.184 (reading R5) */
    const double a1 = 1.21, a2 = -6.35, A = 4.08, M = 1.184;
    const double s3h = 0.5 * sqrt(3.0);
    x = fabs(x);
    if (x < 0.5)
        return a1 * x * x * x - (0.5 * a1 + 4.0 * (M - A)) * x * x + M;
    if (x < s3h) {
        double t = x - s3h;
        return t * t * (a2 * x + 2.0 * A * (2.0 + sqrt(3.0)) - 0.5 * a2);
    }
    return 0.0;
}

double orc_wg(double x)
{   /* Eq. A1: Gaussian truncated at sqrt3/2 */
    x = fabs(x);
    return x < 0.5 * sqrt(3.0) ? exp(-x * x) : 0.0;
}

/* index i with r_i <= d < r_{i+1}, for r_0 <= d < r_{nr-1} */
static int32_t bracket(double d, int32_t nr, int32_t eta_r)
{
    int32_t i = 0;
    while (i + 1 < nr - 1 && orc_radius(i + 1, eta_r) <= d) i++;
    return i;
}

static void smooth_weights(int32_t gauss, double d, double h, int32_t nr, int32_t eta_r, double* w)
{   /* W_p or W_g normalised so that the weights over all evaluation points
     * sum to one (App. A, kernel tabulation paragraph); readings R5, R6, R11 */
    for (int32_t i = 0; i < nr; ++i) w[i] = 0.0;
    double rlast = orc_radius(nr - 1, eta_r);
    if (d >= rlast) { w[nr - 1] = 1.0; return; }
    double S = 0.0;
    for (int32_t i = 0; i < nr; ++i) {
        double x = (orc_radius(i, eta_r) - d) / h;
        double W = gauss ? orc_wg(x) : orc_wp(x);
        w[i] = W;
        S += W;
    }
    if (S > 0.0) {
        for (int32_t i = 0; i < nr; ++i) w[i] = w[i] / S;
        return;
    }
    int32_t i = bracket(d, nr, eta_r);
    double ri = orc_radius(i, eta_r), rj = orc_radius(i + 1, eta_r);
    w[i] = (rj - d) / (rj - ri);
    w[i + 1] = (d - ri) / (rj - ri);
}

void orc_wp_weights(double d, double h, int32_t nr, int32_t eta_r, double* w)
{
    smooth_weights(0, d, h, nr, eta_r, w);
}

void orc_wg_weights(double d, double h, int32_t nr, int32_t eta_r, double* w)
{
    smooth_weights(1, d, h, nr, eta_r, w);
}

void orc_wf3_split(double d, int32_t nr, int32_t eta_r, double* w)
{   /* W_f,3 (App. A.3): two points r_i <= d < r_{i+1} with
     * w_i + w_{i+1} = 1 and w_i / r_i^2 + w_{i+1} / r_{i+1}^2 = 1 / d^2 */
    for (int32_t i = 0; i < nr; ++i) w[i] = 0.0;
    double rlast = orc_radius(nr - 1, eta_r);
    if (d >= rlast) { w[nr - 1] = 1.0; return; }
    int32_t i = bracket(d, nr, eta_r);
    if (i == 0) { w[1] = 1.0; return; }   /* d < r_1: cannot occur for a non-target node */
    double ri = orc_radius(i, eta_r), rj = orc_radius(i + 1, eta_r);
    double a = 1.0 / (ri * ri), b = 1.0 / (rj * rj), t = 1.0 / (d * d);
    double wj = (a - t) / (a - b);
    w[i + 1] = wj;
    w[i] = 1.0 - wj;
}

void orc_wf1_split(double d, int32_t nr, int32_t eta_r, double* w)
{   /* W_f,1 (App. A.3): w_{i+1} / w_i = (d - r_i) / (r_{i+1} - d) and the
     * flux at r = 0 exact, w_i / r_i^2 + w_{i+1} / r_{i+1}^2 = 1 / d^2 */
    for (int32_t i = 0; i < nr; ++i) w[i] = 0.0;
    double rlast = orc_radius(nr - 1, eta_r);
    if (d >= rlast) { w[nr - 1] = 1.0; return; }
    int32_t i = bracket(d, nr, eta_r);
    if (i == 0) { w[1] = 1.0; return; }
    double ri = orc_radius(i, eta_r), rj = orc_radius(i + 1, eta_r);
    double ratio = (d - ri) / (rj - d);
    double wi = 1.0 / ((d * d) * (1.0 / (ri * ri) + ratio / (rj * rj)));
    w[i] = wi;
    w[i + 1] = ratio * wi;
}

void orc_wf2_split(double d, int32_t nr, int32_t eta_r, double* w)
{   /* W_f,2 (App. A.3): the flux exact at r = 0 and at r_{i-1}:
     * w_i / r_i^2 + w_{i+1} / r_{i+1}^2 = 1 / d^2 and
     * w_i / (r_i - r_{i-1})^2 + w_{i+1} / (r_{i+1} - r_{i-1})^2 = 1 / (d - r_{i-1})^2,
     * solved by Cramer's rule; reading R11 where it does not apply */
    double rlast = orc_radius(nr - 1, eta_r);
    int32_t i = d >= rlast ? nr - 1 : bracket(d, nr, eta_r);
    if (d >= rlast || i < 2) { orc_wf3_split(d, nr, eta_r, w); return; }
    for (int32_t k = 0; k < nr; ++k) w[k] = 0.0;
    double rm = orc_radius(i - 1, eta_r), ri = orc_radius(i, eta_r), rj = orc_radius(i + 1, eta_r);
    double a11 = 1.0 / (ri * ri), a12 = 1.0 / (rj * rj), b1 = 1.0 / (d * d);
    double a21 = 1.0 / ((ri - rm) * (ri - rm)), a22 = 1.0 / ((rj - rm) * (rj - rm)), b2 = 1.0 / ((d - rm) * (d - rm));
    double det = a11 * a22 - a12 * a21;
    double wi = (b1 * a22 - a12 * b2) / det;
    double wj = (a11 * b2 - a21 * b1) / det;
    if (!(wi >= 0.0 && wj >= 0.0)) { orc_wf3_split(d, nr, eta_r, w); return; }
    w[i] = wi;
    w[i + 1] = wj;
}

void orc_wf3n_weights(double d, double h, int32_t nr, int32_t eta_r, double* w)
{   /* generalised W_f,3 (Eq. A8-A10): the N points in the support carry
     * eps (a + b k), k = offset from the lowest index, with the sum and the
     * flux at r = 0 exact; reading R11 for A_2 and the fallback */
    double rlast = orc_radius(nr - 1, eta_r);
    if (d >= rlast) { orc_wf3_split(d, nr, eta_r, w); return; }
    int32_t lo = -1, n = 0;
    for (int32_t i = 1; i < nr; ++i)
        if (fabs(orc_radius(i, eta_r) - d) < 0.5 * sqrt(3.0) * h) { if (lo < 0) lo = i; n++; }
    if (n <= 2) { orc_wf3_split(d, nr, eta_r, w); return; }
    double A1 = 0.0, A2 = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        double r = orc_radius(lo + k, eta_r);
        A1 += 1.0 / (r * r);
        A2 += (double)k / (r * r);
    }
    double b = (1.0 / (d * d) - A1 / (double)n) / (A2 - (double)(n - 1) * A1 / 2.0);
    double a = 1.0 / (double)n - b * (double)(n - 1) / 2.0;
    for (int32_t k = 0; k < n; ++k)
        if (a + b * (double)k < 0.0) { orc_wf3_split(d, nr, eta_r, w); return; }
    for (int32_t i = 0; i < nr; ++i) w[i] = 0.0;
    for (int32_t k = 0; k < n; ++k) w[lo + k] = a + b * (double)k;
}

void orc_eps_weights(int32_t kind, double d, double h, int32_t nr, int32_t eta_r, double* w)
{
    switch (kind) {
    case ORC_KE_WF1: orc_wf1_split(d, nr, eta_r, w); break;
    case ORC_KE_WF2: orc_wf2_split(d, nr, eta_r, w); break;
    case ORC_KE_WF3N: orc_wf3n_weights(d, h, nr, eta_r, w); break;
    case ORC_KE_WP: orc_wp_weights(d, h, nr, eta_r, w); break;
    case ORC_KE_WG: orc_wg_weights(d, h, nr, eta_r, w); break;
    default: orc_wf3_split(d, nr, eta_r, w); break;
    }
}

/* ------------------------------------------------------------------------ */
/* Node -> ray table (Sec. 2.3 first mapping step; reading R4).             */
/* ------------------------------------------------------------------------ */

/* (u,v) bin of a face coordinate x in [-A, A]: a centre bin for x = 0 and
 * ORC_TQH bins of width A/ORC_TQH on either side, so that the binning is
 * exactly mirror-symmetric (bin u <-> ORC_TQ - 1 - u under x -> -x) */
static int64_t face_bin(int64_t x, int64_t A)
{
    if (x == 0) return ORC_TQH;
    int64_t q = ((int64_t)ORC_TQH * (x > 0 ? x : -x)) / A;
    if (q > ORC_TQH - 1) q = ORC_TQH - 1;
    return x > 0 ? ORC_TQH + 1 + q : ORC_TQH - 1 - q;
}

/* representative face coordinate of bin u */
static double face_coord(int64_t u)
{
    if (u == ORC_TQH) return 0.0;
    if (u > ORC_TQH) return (2.0 * (double)(u - ORC_TQH - 1) + 1.0) / (2.0 * ORC_TQH);
    return -(2.0 * (double)(ORC_TQH - 1 - u) + 1.0) / (2.0 * ORC_TQH);
}

int32_t orc_table_key(int64_t ox, int64_t oy, int64_t oz, int64_t s)
{
    int64_t o[3] = {ox, oy, oz};
    int64_t ab[3] = {llabs(ox), llabs(oy), llabs(oz)};
    int64_t A = ab[0];
    if (ab[1] > A) A = ab[1];
    if (ab[2] > A) A = ab[2];
    int ntie = (ab[0] == A) + (ab[1] == A) + (ab[2] == A);
    /* psi = h / |centre offset| = 2s / |o|; bin = floor(32 psi) */
    int64_t o2 = ox * ox + oy * oy + oz * oz;
    int64_t lim = 64 * s, lim2 = lim * lim;
    int64_t pb = (int64_t)floor((double)lim / sqrt((double)o2));
    while (pb > 0 && pb * pb * o2 > lim2) pb--;
    while ((pb + 1) * (pb + 1) * o2 <= lim2) pb++;
    if (pb > ORC_TB - 1) pb = ORC_TB - 1;
    if (ntie == 1) {                            /* face of the dominant axis */
        int a = (ab[0] == A) ? 0 : ((ab[1] == A) ? 1 : 2);
        int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
        int face = 2 * a + (o[a] < 0 ? 1 : 0);
        int64_t u = face_bin(o[b], A);
        int64_t v = face_bin(o[c], A);
        return (int32_t)(((face * ORC_TQ + u) * ORC_TQ + v) * ORC_TB + pb);
    }
    if (ntie == 2) {                            /* edge between the two tied faces */
        int c = (ab[0] != A) ? 0 : ((ab[1] != A) ? 1 : 2);
        int a = (c == 0) ? 1 : 0, b = (c == 2) ? 1 : 2;
        int pair = (c == 2) ? 0 : ((c == 1) ? 1 : 2);           /* (0,1), (0,2), (1,2) */
        int edge = 4 * pair + 2 * (o[a] < 0) + (o[b] < 0);
        int64_t v = face_bin(o[c], A);
        return (int32_t)(ORC_NFACEKEYS + (edge * ORC_TQ + v) * ORC_TB + pb);
    }
    int corner = (ox < 0) + 2 * (oy < 0) + 4 * (oz < 0);
    return (int32_t)(ORC_NFACEKEYS + ORC_NEDGEKEYS + corner * ORC_TB + pb);
}

typedef struct { int32_t n; int32_t* pix; int32_t* cnt; } orc_entry;
typedef struct { int32_t nside; orc_entry* e; } orc_table;
static orc_table g_tables[16];   /* one lazily filled table per N_side */

/* The representative direction of a key (not normalised) and its psi bin.
 * *mirror = +1 or -1 for the keys whose direction lies on the plane x = y
 * (resp. x = -y) -- edge keys of the x-y edges and corner keys -- and 0
 * otherwise. */
static void key_geometry(int32_t key, double p[3], int32_t* pb, int* mirror)
{
    *pb = key % ORC_TB;
    *mirror = 0;
    if (key < ORC_NFACEKEYS) {
        int32_t rest = key / ORC_TB;
        int32_t v = rest % ORC_TQ; rest /= ORC_TQ;
        int32_t u = rest % ORC_TQ;
        int32_t face = rest / ORC_TQ;
        int a = face / 2;
        int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
        p[a] = (face & 1) ? -1.0 : 1.0;
        p[b] = face_coord(u);
        p[c] = face_coord(v);
        return;
    }
    if (key < ORC_NFACEKEYS + ORC_NEDGEKEYS) {
        int32_t rest = (key - ORC_NFACEKEYS) / ORC_TB;
        int32_t v = rest % ORC_TQ;
        int32_t edge = rest / ORC_TQ;
        int pair = edge / 4;
        int a = (pair == 2) ? 1 : 0, b = (pair == 0) ? 1 : 2, c = 3 - a - b;
        double sa = (edge & 2) ? -1.0 : 1.0, sb = (edge & 1) ? -1.0 : 1.0;
        p[a] = sa; p[b] = sb; p[c] = face_coord(v);
        if (pair == 0) *mirror = (sa == sb) ? 1 : -1;
        return;
    }
    int32_t corner = (key - ORC_NFACEKEYS - ORC_NEDGEKEYS) / ORC_TB;
    p[0] = (corner & 1) ? -1.0 : 1.0;
    p[1] = (corner & 2) ? -1.0 : 1.0;
    p[2] = (corner & 4) ? -1.0 : 1.0;
    *mirror = (p[0] == p[1]) ? 1 : -1;
}

/* The pixel that the reflection through the plane x = t y (t = +-1) maps
 * pixel k to: HEALPix has that symmetry, so the image of the pixel's centre
 * is the centre of its mirror pixel. */
static int64_t mirror_pixel(int32_t nside, int64_t k, int t)
{
    double v[3];
    orc_pix2vec(nside, k, v);
    return orc_ang2pix(nside, t * v[1], t * v[0], v[2]);
}

static void compute_entry(int32_t nside, int32_t key, orc_entry* out)
{
    double p[3];
    int32_t pb;
    int mirror;
    key_geometry(key, p, &pb, &mirror);
    double n = sqrt((p[0] * p[0] + p[1] * p[1]) + p[2] * p[2]);
    double C[3] = {p[0] / n, p[1] / n, p[2] / n};
    double psi = ((double)pb + 0.5) / 32.0;
    int64_t npix = 12 * (int64_t)nside * nside;
    int32_t* hist = (int32_t*)calloc((size_t)npix, sizeof(int32_t));
    for (int iz = 0; iz < ORC_TM; ++iz)
        for (int iy = 0; iy < ORC_TM; ++iy)
            for (int ix = 0; ix < ORC_TM; ++ix) {
                double fx = (ix + 0.5) / ORC_TM - 0.5;
                double fy = (iy + 0.5) / ORC_TM - 0.5;
                double fz = (iz + 0.5) / ORC_TM - 0.5;
                int64_t k = orc_ang2pix(nside, C[0] + psi * fx, C[1] + psi * fy, C[2] + psi * fz);
                if (mirror) {                   /* half to the pixel, half to its mirror */
                    hist[k] += 1;
                    hist[mirror_pixel(nside, k, mirror)] += 1;
                } else {
                    hist[k] += 2;
                }
            }
    int32_t n_nz = 0;
    for (int64_t k = 0; k < npix; ++k) n_nz += hist[k] > 0;
    out->n = n_nz;
    out->pix = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_nz);
    out->cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_nz);
    int32_t j = 0;
    for (int64_t k = 0; k < npix; ++k)
        if (hist[k] > 0) { out->pix[j] = (int32_t)k; out->cnt[j] = hist[k]; ++j; }
    free(hist);
}

static const orc_entry* table_entry(int32_t nside, int32_t key)
{
    int slot = 0;
    while (nside > (1 << slot)) slot++;
    orc_table* t = &g_tables[slot];
    if (!t->e) {
        t->nside = nside;
        t->e = (orc_entry*)calloc(ORC_NKEYS, sizeof(orc_entry));
        for (int64_t k = 0; k < ORC_NKEYS; ++k) t->e[k].n = -1;
    }
    orc_entry* e = &t->e[key];
    if (e->n < 0) compute_entry(nside, key, e);
    return e;
}

int32_t orc_table_entry(int32_t nside, int32_t key, int32_t* pix, int32_t* cnt, int32_t cap)
{
    const orc_entry* e = table_entry(nside, key);
    for (int32_t j = 0; j < e->n && j < cap; ++j) { pix[j] = e->pix[j]; cnt[j] = e->cnt[j]; }
    return e->n;
}

/* ------------------------------------------------------------------------ */
/* Tree build (Sec. 2.1, Eq. 1-3; source mapping Sec. 2.7).                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    double m, smx, smy, smz;   /* mass and mass-weighted position sums */
    double cm[3];              /* centre of mass */
    double alpha, eps, e, mion;
} orc_node;

enum { ORC_UNUSED = 0, ORC_LEAF = 1, ORC_INTERNAL = 2 };

struct orc_tree {
    int32_t N, L;           /* N = cells per axis of the finest level */
    double dx_cm;           /* finest cell edge */
    int use_e;
    orc_node** lv;          /* lv[l] has (2^l)^3 nodes, index (iz*n + iy)*n + ix */
    uint8_t** flag;         /* AMR: per node ORC_LEAF / ORC_INTERNAL / ORC_UNUSED; NULL: uniform */
    int64_t n_leaf;         /* cells (targets): N^3 uniform, blocks x 512 AMR */
    int8_t* leaf_lev;       /* AMR: tree level of each cell */
    int32_t* leaf_pos;      /* AMR: 3 per cell, position at that level */
    double* ndot;           /* per-cell emission rate after source mapping */
    double* alpha_c;        /* per-cell clipped recombination rate (Eq. 2) */
    double* eps_c;          /* per-cell clipped emission rate (Eq. 1) */
};

static int node_flag(const orc_tree* t, int32_t level, int64_t idx)
{
    if (!t->flag) return level == t->L ? ORC_LEAF : ORC_INTERNAL;
    return t->flag[level][idx];
}

/* level, position (at that level) and edge (finest cells) of target cell q */
static void target_geom(const orc_tree* t, int64_t q, int32_t* lev, int64_t* p3, int64_t* edge)
{
    if (!t->flag) {
        int64_t N = t->N;
        *lev = t->L;
        p3[0] = q % N; p3[1] = (q / N) % N; p3[2] = q / (N * N);
        *edge = 1;
        return;
    }
    *lev = t->leaf_lev[q];
    for (int a = 0; a < 3; ++a) p3[a] = t->leaf_pos[3 * q + a];
    *edge = (int64_t)(t->N >> *lev);
}

static int64_t lidx(int64_t n, int64_t ix, int64_t iy, int64_t iz) { return (iz * n + iy) * n + ix; }

orc_tree* orc_tree_build(int32_t N, double dx_cm, double alpha_B, const double* box_lo_cm,
                         const double* n_H, const double* ndot_cell,
                         int32_t nsrc, const double* src_xyz_cm, const double* src_Q,
                         const double* e_prev)
{
    if (N < 2 || (N & (N - 1)) != 0) return NULL;   /* the octree needs a power-of-two grid */
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    int32_t L = 0;
    while ((1 << L) < N) L++;
    t->N = N; t->L = L; t->dx_cm = dx_cm; t->use_e = (e_prev != NULL);
    int64_t nc = (int64_t)N * N * N;
    t->n_leaf = nc;
    t->ndot = (double*)calloc((size_t)nc, sizeof(double));
    t->alpha_c = (double*)calloc((size_t)nc, sizeof(double));
    t->eps_c = (double*)calloc((size_t)nc, sizeof(double));
    /* source mapping onto the grid, point sources (reading R2) */
    if (ndot_cell)
        for (int64_t c = 0; c < nc; ++c) t->ndot[c] = ndot_cell[c];
    for (int32_t s = 0; s < nsrc; ++s) {
        int64_t ic[3];
        for (int a = 0; a < 3; ++a) {
            double f = floor((src_xyz_cm[3 * s + a] - box_lo_cm[a]) / dx_cm);
            if (f < 0.0) f = 0.0;
            if (f > N - 1) f = N - 1;
            ic[a] = (int64_t)f;
        }
        t->ndot[lidx(N, ic[0], ic[1], ic[2])] += src_Q[s];
    }
    /* Eq. 1-2 netted per cell (reading R1) */
    double dv_cm3 = dx_cm * dx_cm * dx_cm;
    for (int64_t c = 0; c < nc; ++c) {
        double rec = alpha_B * (n_H[c] * n_H[c]) * dv_cm3;
        t->eps_c[c] = fmax(t->ndot[c] - rec, 0.0);
        t->alpha_c[c] = fmax(rec - t->ndot[c], 0.0);
    }
    t->lv = (orc_node**)calloc((size_t)L + 1, sizeof(orc_node*));
    for (int32_t l = 0; l <= L; ++l) {
        int64_t n = (int64_t)1 << l;
        t->lv[l] = (orc_node*)calloc((size_t)(n * n * n), sizeof(orc_node));
    }
    /* leaves: cells; mass in units of n_H x (cell volume = 1) */
    for (int64_t iz = 0; iz < N; ++iz)
        for (int64_t iy = 0; iy < N; ++iy)
            for (int64_t ix = 0; ix < N; ++ix) {
                int64_t c = lidx(N, ix, iy, iz);
                orc_node* nd = &t->lv[L][c];
                nd->m = n_H[c];
                nd->smx = nd->m * ((double)ix + 0.5);
                nd->smy = nd->m * ((double)iy + 0.5);
                nd->smz = nd->m * ((double)iz + 0.5);
                nd->alpha = t->alpha_c[c];
                nd->eps = t->eps_c[c];
                nd->e = e_prev ? e_prev[c] : 0.0;             /* Eq. 3, dV = 1 cell */
                nd->mion = (e_prev && e_prev[c] > 0.0) ? nd->m : 0.0;
            }
    /* parents: sum of the eight children in Morton order */
    for (int32_t l = L - 1; l >= 0; --l) {
        int64_t n = (int64_t)1 << l;
        for (int64_t iz = 0; iz < n; ++iz)
            for (int64_t iy = 0; iy < n; ++iy)
                for (int64_t ix = 0; ix < n; ++ix) {
                    orc_node* p = &t->lv[l][lidx(n, ix, iy, iz)];
                    for (int ch = 0; ch < 8; ++ch) {
                        const orc_node* q = &t->lv[l + 1][lidx(2 * n, 2 * ix + (ch & 1),
                                                               2 * iy + ((ch >> 1) & 1),
                                                               2 * iz + ((ch >> 2) & 1))];
                        if (ch == 0) {
                            p->m = q->m; p->smx = q->smx; p->smy = q->smy; p->smz = q->smz;
                            p->alpha = q->alpha; p->eps = q->eps; p->e = q->e; p->mion = q->mion;
                        } else {
                            p->m += q->m; p->smx += q->smx; p->smy += q->smy; p->smz += q->smz;
                            p->alpha += q->alpha; p->eps += q->eps; p->e += q->e; p->mion += q->mion;
                        }
                    }
                }
    }
    /* centres of mass (geometric centre for a massless node) */
    for (int32_t l = 0; l <= L; ++l) {
        int64_t n = (int64_t)1 << l;
        double s = (double)(N >> l);
        for (int64_t iz = 0; iz < n; ++iz)
            for (int64_t iy = 0; iy < n; ++iy)
                for (int64_t ix = 0; ix < n; ++ix) {
                    orc_node* p = &t->lv[l][lidx(n, ix, iy, iz)];
                    if (p->m > 0.0) {
                        p->cm[0] = p->smx / p->m; p->cm[1] = p->smy / p->m; p->cm[2] = p->smz / p->m;
                    } else {
                        p->cm[0] = ((double)ix + 0.5) * s;
                        p->cm[1] = ((double)iy + 0.5) * s;
                        p->cm[2] = ((double)iz + 0.5) * s;
                    }
                }
    }
    return t;
}

static int32_t ilog2(int64_t v) { int32_t l = 0; while (((int64_t)1 << l) < v) ++l; return l; }

orc_tree* orc_tree_build_amr(int32_t N_base, int32_t max_level, double dx_fine_cm, double alpha_B,
                             const double* box_lo_cm, int32_t n_blocks, const int32_t* blk_level,
                             const int32_t* blk_pos, const double* n_H, const double* ndot_cell,
                             int32_t nsrc, const double* src_xyz_cm, const double* src_Q, const double* e_prev)
{
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    int32_t N = N_base << max_level, L = ilog2(N), Lb = ilog2(N_base);
    t->N = N; t->L = L; t->dx_cm = dx_fine_cm; t->use_e = (e_prev != NULL);
    int64_t nl = (int64_t)n_blocks * 512;
    t->n_leaf = nl;
    t->ndot = (double*)calloc((size_t)nl, sizeof(double));
    t->alpha_c = (double*)calloc((size_t)nl, sizeof(double));
    t->eps_c = (double*)calloc((size_t)nl, sizeof(double));
    t->leaf_lev = (int8_t*)malloc((size_t)nl);
    t->leaf_pos = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nl);
    t->lv = (orc_node**)calloc((size_t)L + 1, sizeof(orc_node*));
    t->flag = (uint8_t**)calloc((size_t)L + 1, sizeof(uint8_t*));
    int32_t** leafid = (int32_t**)calloc((size_t)L + 1, sizeof(int32_t*));
    for (int32_t l = 0; l <= L; ++l) {
        int64_t n = (int64_t)1 << l;
        t->lv[l] = (orc_node*)calloc((size_t)(n * n * n), sizeof(orc_node));
        t->flag[l] = (uint8_t*)calloc((size_t)(n * n * n), 1);
        leafid[l] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * n * n));
    }
    /* the cells of every block are the leaves */
    for (int32_t b = 0; b < n_blocks; ++b) {
        int32_t lc = Lb + blk_level[b];
        int64_t n = (int64_t)1 << lc;
        for (int c = 0; c < 512; ++c) {
            int64_t q = (int64_t)b * 512 + c;
            int64_t ix = 8 * (int64_t)blk_pos[3 * b + 0] + (c & 7);
            int64_t iy = 8 * (int64_t)blk_pos[3 * b + 1] + ((c >> 3) & 7);
            int64_t iz = 8 * (int64_t)blk_pos[3 * b + 2] + (c >> 6);
            t->leaf_lev[q] = (int8_t)lc;
            t->leaf_pos[3 * q + 0] = (int32_t)ix; t->leaf_pos[3 * q + 1] = (int32_t)iy; t->leaf_pos[3 * q + 2] = (int32_t)iz;
            t->flag[lc][lidx(n, ix, iy, iz)] = ORC_LEAF;
            leafid[lc][lidx(n, ix, iy, iz)] = (int32_t)q;
            if (ndot_cell) t->ndot[q] = ndot_cell[q];
        }
    }
    /* point sources to the cell containing them (reading R2 on the finest lattice) */
    for (int32_t s = 0; s < nsrc; ++s) {
        int64_t f[3];
        for (int a = 0; a < 3; ++a) {
            double v = floor((src_xyz_cm[3 * s + a] - box_lo_cm[a]) / dx_fine_cm);
            if (v < 0.0) v = 0.0;
            if (v > N - 1) v = N - 1;
            f[a] = (int64_t)v;
        }
        for (int32_t l = 0; l <= L; ++l) {
            int64_t n = (int64_t)1 << l, sh = L - l;
            int64_t id = lidx(n, f[0] >> sh, f[1] >> sh, f[2] >> sh);
            if (t->flag[l][id] == ORC_LEAF) { t->ndot[leafid[l][id]] += src_Q[s]; break; }
        }
    }
    /* leaves: Eq. 1-3 per cell of edge s (volume s^3 finest cells) */
    double dvf = dx_fine_cm * dx_fine_cm * dx_fine_cm;
    for (int64_t q = 0; q < nl; ++q) {
        int32_t lc = t->leaf_lev[q];
        int64_t n = (int64_t)1 << lc;
        double s = (double)(N >> lc), vol = s * s * s;
        double rec = alpha_B * (n_H[q] * n_H[q]) * (dvf * vol);
        t->eps_c[q] = fmax(t->ndot[q] - rec, 0.0);
        t->alpha_c[q] = fmax(rec - t->ndot[q], 0.0);
        orc_node* nd = &t->lv[lc][lidx(n, t->leaf_pos[3 * q], t->leaf_pos[3 * q + 1], t->leaf_pos[3 * q + 2])];
        nd->m = n_H[q] * vol;
        nd->smx = nd->m * (((double)t->leaf_pos[3 * q + 0] + 0.5) * s);
        nd->smy = nd->m * (((double)t->leaf_pos[3 * q + 1] + 0.5) * s);
        nd->smz = nd->m * (((double)t->leaf_pos[3 * q + 2] + 0.5) * s);
        nd->alpha = t->alpha_c[q];
        nd->eps = t->eps_c[q];
        nd->e = e_prev ? e_prev[q] * vol : 0.0;
        nd->mion = (e_prev && e_prev[q] > 0.0) ? nd->m : 0.0;
    }
    /* parents: the sum of their eight children, in Morton order */
    for (int32_t l = L - 1; l >= 0; --l) {
        int64_t n = (int64_t)1 << l;
        for (int64_t iz = 0; iz < n; ++iz)
            for (int64_t iy = 0; iy < n; ++iy)
                for (int64_t ix = 0; ix < n; ++ix) {
                    int64_t id = lidx(n, ix, iy, iz);
                    if (t->flag[l][id] == ORC_LEAF) continue;
                    if (t->flag[l + 1][lidx(2 * n, 2 * ix, 2 * iy, 2 * iz)] == ORC_UNUSED) continue;
                    t->flag[l][id] = ORC_INTERNAL;
                    orc_node* p = &t->lv[l][id];
                    for (int ch = 0; ch < 8; ++ch) {
                        const orc_node* q = &t->lv[l + 1][lidx(2 * n, 2 * ix + (ch & 1), 2 * iy + ((ch >> 1) & 1),
                                                               2 * iz + ((ch >> 2) & 1))];
                        if (ch == 0) {
                            p->m = q->m; p->smx = q->smx; p->smy = q->smy; p->smz = q->smz;
                            p->alpha = q->alpha; p->eps = q->eps; p->e = q->e; p->mion = q->mion;
                        } else {
                            p->m += q->m; p->smx += q->smx; p->smy += q->smy; p->smz += q->smz;
                            p->alpha += q->alpha; p->eps += q->eps; p->e += q->e; p->mion += q->mion;
                        }
                    }
                }
    }
    for (int32_t l = 0; l <= L; ++l) {
        int64_t n = (int64_t)1 << l;
        double s = (double)(N >> l);
        for (int64_t iz = 0; iz < n; ++iz)
            for (int64_t iy = 0; iy < n; ++iy)
                for (int64_t ix = 0; ix < n; ++ix) {
                    orc_node* p = &t->lv[l][lidx(n, ix, iy, iz)];
                    if (p->m > 0.0) {
                        p->cm[0] = p->smx / p->m; p->cm[1] = p->smy / p->m; p->cm[2] = p->smz / p->m;
                    } else {
                        p->cm[0] = ((double)ix + 0.5) * s;
                        p->cm[1] = ((double)iy + 0.5) * s;
                        p->cm[2] = ((double)iz + 0.5) * s;
                    }
                }
    }
    for (int32_t l = 0; l <= L; ++l) free(leafid[l]);
    free(leafid);
    return t;
}

int64_t orc_tree_n_leaves(const orc_tree* t) { return t->n_leaf; }

/* 1 for a leaf (a grid cell), 2 for a parent, 0 for a position inside a cell */
int32_t orc_tree_flag(const orc_tree* t, int32_t level, int64_t ix, int64_t iy, int64_t iz)
{
    int64_t n = (int64_t)1 << level;
    return node_flag(t, level, lidx(n, ix, iy, iz));
}

void orc_tree_free(orc_tree* t)
{
    if (!t) return;
    for (int32_t l = 0; l <= t->L; ++l) free(t->lv[l]);
    if (t->flag) for (int32_t l = 0; l <= t->L; ++l) free(t->flag[l]);
    free(t->flag); free(t->leaf_lev); free(t->leaf_pos);
    free(t->lv); free(t->ndot); free(t->alpha_c); free(t->eps_c); free(t);
}

int32_t orc_tree_levels(const orc_tree* t) { return t->L + 1; }

void orc_tree_node(const orc_tree* t, int32_t level, int64_t ix, int64_t iy, int64_t iz, double* out)
{
    const orc_node* p = &t->lv[level][lidx((int64_t)1 << level, ix, iy, iz)];
    out[0] = p->m; out[1] = p->cm[0]; out[2] = p->cm[1]; out[3] = p->cm[2];
    out[4] = p->alpha; out[5] = p->eps; out[6] = p->e; out[7] = p->mion;
}

void orc_cell_quantities(const orc_tree* t, double* ndot_out, double* alpha_out, double* eps_out)
{
    int64_t nc = t->n_leaf;
    for (int64_t c = 0; c < nc; ++c) {
        if (ndot_out) ndot_out[c] = t->ndot[c];
        if (alpha_out) alpha_out[c] = t->alpha_c[c];
        if (eps_out) eps_out[c] = t->eps_c[c];
    }
}

/* ------------------------------------------------------------------------ */
/* Tree walk with MACs (Sec. 2.3-2.4) and mapping onto rays (Sec. 2.3).      */
/* ------------------------------------------------------------------------ */

static int64_t morton3(int64_t ix, int64_t iy, int64_t iz, int32_t bits)
{
    int64_t m = 0;
    for (int32_t b = 0; b < bits; ++b)
        m |= (((ix >> b) & 1) << (3 * b)) | (((iy >> b) & 1) << (3 * b + 1)) | (((iz >> b) & 1) << (3 * b + 2));
    return m;
}

static int64_t canonical_id(int32_t level, int64_t ix, int64_t iy, int64_t iz)
{   /* level-order numbering: (8^l - 1)/7 + Morton index within the level */
    int64_t off = (((int64_t)1 << (3 * level)) - 1) / 7;
    return off + morton3(ix, iy, iz, level);
}

typedef struct {
    const orc_tree* t;
    const orc_params* p;
    int64_t tx, ty, tz;       /* target corner, finest cells */
    int64_t ts;               /* target edge, finest cells */
    double cx, cy, cz;        /* target centre */
    int32_t img;              /* corner of symmetry: mirrored axes (bit a: axis a) of this image */
    int32_t nr;
    double lray;
    double th_lim2, th_if2, th_src2;
    double *ba, *be, *bee;
    double *wa, *we, *wee;
    int64_t* acc; int64_t cap; int64_t nacc;
    int64_t visited;
    double* cd;               /* column-density map of the target (R13), or NULL */
} walk_ctx;

/* Offset o = 2 (node geometric centre - target centre), in half cells, of
 * the copy of the node that the boundary condition puts next to the target
 * (R12), and the target centre to measure that copy's distance from in the
 * node's own frame. */
static void node_frame(const walk_ctx* w, int32_t level, int64_t ix, int64_t iy, int64_t iz,
                       int64_t o[3], double tc[3])
{
    int64_t N = w->t->N, s = N >> level;
    int64_t g2[3] = {2 * ix * s + s, 2 * iy * s + s, 2 * iz * s + s};
    int64_t t2[3] = {2 * w->tx + w->ts, 2 * w->ty + w->ts, 2 * w->tz + w->ts};
    double c[3] = {w->cx, w->cy, w->cz};
    for (int a = 0; a < 3; ++a) {
        if (w->p->bc == ORC_BC_CORNER && ((w->img >> a) & 1)) {
            /* image mirrored in axis a: the node sits at -g, i.e. the
             * original node seen from the mirrored target -t */
            o[a] = -(g2[a] + t2[a]);
            tc[a] = -c[a];
        } else {
            o[a] = g2[a] - t2[a];
            tc[a] = c[a];
            if (w->p->bc == ORC_BC_PERIODIC) {
                int64_t k = 0;
                if (o[a] >= N) k = -1;
                else if (o[a] < -N) k = 1;
                o[a] += 2 * N * k;             /* copy shifted by k N cells */
                tc[a] -= (double)(k * N);
            }
        }
    }
}

static void map_node(walk_ctx* w, int32_t level, int64_t ix, int64_t iy, int64_t iz,
                     const orc_node* nd, double d)
{
    const orc_params* p = w->p;
    if (w->acc) { if (w->nacc < w->cap) w->acc[w->nacc] = canonical_id(level, ix, iy, iz); }
    w->nacc++;
    if (w->cd) {                                   /* column-density map (R13) */
        if (nd->m == 0.0) return;
        int64_t o[3];
        double tc[3];
        node_frame(w, level, ix, iy, iz, o, tc);
        const orc_entry* ent = table_entry(p->nside, orc_table_key(o[0], o[1], o[2], (int64_t)(w->t->N >> level)));
        double omega = 4.0 * ORC_PI / (double)(12 * (int64_t)p->nside * p->nside);
        const double inv_m3 = 1.0 / (double)ORC_TW;
        for (int32_t j = 0; j < ent->n; ++j)
            w->cd[ent->pix[j]] += ((double)ent->cnt[j] * inv_m3) * nd->m / (omega * (d * d));
        return;
    }
    int use_e = w->t->use_e;
    if (nd->alpha == 0.0 && nd->eps == 0.0 && (!use_e || nd->e == 0.0)) return;
    if (d > w->lray) return;                       /* beyond the maximum ray length (R6) */
    int64_t s = (int64_t)(w->t->N >> level);
    int64_t o[3];
    double tc[3];
    node_frame(w, level, ix, iy, iz, o, tc);
    const orc_entry* ent = table_entry(p->nside, orc_table_key(o[0], o[1], o[2], s));
    int32_t nr = w->nr;
    double h = (double)s;
    if (nd->alpha != 0.0) smooth_weights(p->kernel_alpha == ORC_K_WG, d, h, nr, p->eta_r, w->wa);
    if (nd->eps != 0.0) orc_eps_weights(p->kernel_eps, d, h, nr, p->eta_r, w->we);
    if (use_e && nd->e != 0.0) smooth_weights(p->kernel_alpha == ORC_K_WG, d, h, nr, p->eta_r, w->wee);
    const double inv_m3 = 1.0 / (double)ORC_TW;
    for (int32_t j = 0; j < ent->n; ++j) {
        double wk = (double)ent->cnt[j] * inv_m3;     /* volume fraction in ray k */
        int64_t k = ent->pix[j];
        for (int32_t i = 0; i < nr; ++i) {
            if (nd->alpha != 0.0) w->ba[k * nr + i] += wk * w->wa[i] * nd->alpha;
            if (nd->eps != 0.0) w->be[k * nr + i] += wk * w->we[i] * nd->eps;
            if (use_e && nd->e != 0.0) w->bee[k * nr + i] += wk * w->wee[i] * nd->e;
        }
    }
}

static void walk_node(walk_ctx* w, int32_t level, int64_t ix, int64_t iy, int64_t iz)
{
    const orc_tree* t = w->t;
    int64_t n = (int64_t)1 << level;
    const orc_node* nd = &t->lv[level][lidx(n, ix, iy, iz)];
    int64_t s = (int64_t)(t->N >> level);
    int fl = node_flag(t, level, lidx(n, ix, iy, iz));
    w->visited++;
    int contains = w->img == 0 &&
                   (w->tx >= ix * s && w->tx < ix * s + s) && (w->ty >= iy * s && w->ty < iy * s + s) &&
                   (w->tz >= iz * s && w->tz < iz * s + s);
    if (contains) {
        if (fl == ORC_LEAF) return;                /* the target itself (R3) */
        for (int ch = 0; ch < 8; ++ch)
            walk_node(w, level + 1, 2 * ix + (ch & 1), 2 * iy + ((ch >> 1) & 1), 2 * iz + ((ch >> 2) & 1));
        return;
    }
    int64_t o[3];
    double tc[3];
    node_frame(w, level, ix, iy, iz, o, tc);       /* the copy of the node next to the target (R12) */
    double dx = tc[0] - nd->cm[0];
    double dy = tc[1] - nd->cm[1];
    double dz = tc[2] - nd->cm[2];
    double d2 = (dx * dx + dy * dy) + dz * dz;
    if (fl != ORC_LEAF) {
        double h2 = (double)s * (double)s;
        int acc_lim = h2 < w->th_lim2 * d2;                               /* BH MAC */
        int is_if = (DELTA_IF * nd->m < nd->mion) && (nd->mion < (1.0 - DELTA_IF) * nd->m);
        int acc_if = !is_if || (h2 < w->th_if2 * d2);                      /* IF MAC */
        int acc_src = !(nd->eps > 0.0) || (h2 < w->th_src2 * d2);          /* Src MAC */
        if (!(acc_lim && acc_if && acc_src)) {
            for (int ch = 0; ch < 8; ++ch)
                walk_node(w, level + 1, 2 * ix + (ch & 1), 2 * iy + ((ch >> 1) & 1), 2 * iz + ((ch >> 2) & 1));
            return;
        }
    }
    map_node(w, level, ix, iy, iz, nd, sqrt(d2));
}

static double lray_of(const orc_params* p)
{
    if (p->lray_cells > 0.0) return p->lray_cells;
    return (p->bc == ORC_BC_CORNER ? 2.0 : 1.0) * (double)p->N * sqrt(3.0);   /* R12 */
}

int64_t orc_walk_target(const orc_tree* t, const orc_params* p, int64_t target,
                        double* bins_alpha, double* bins_eps, double* bins_e,
                        int64_t* accepted_ids, int64_t cap, int64_t* n_accepted)
{
    walk_ctx w;
    memset(&w, 0, sizeof w);
    w.t = t; w.p = p;
    {
        int32_t tl;
        int64_t p3[3], edge;
        target_geom(t, target, &tl, p3, &edge);
        w.tx = p3[0] * edge; w.ty = p3[1] * edge; w.tz = p3[2] * edge; w.ts = edge;
        w.cx = (double)w.tx + 0.5 * (double)edge;
        w.cy = (double)w.ty + 0.5 * (double)edge;
        w.cz = (double)w.tz + 0.5 * (double)edge;
    }
    w.lray = lray_of(p);
    w.nr = orc_num_points(p->eta_r, w.lray);
    w.th_lim2 = p->theta_lim * p->theta_lim;
    w.th_if2 = p->theta_if * p->theta_if;
    w.th_src2 = p->theta_src * p->theta_src;
    int64_t nbin = 12 * (int64_t)p->nside * p->nside * w.nr;
    for (int64_t b = 0; b < nbin; ++b) { bins_alpha[b] = 0.0; bins_eps[b] = 0.0; if (bins_e) bins_e[b] = 0.0; }
    w.ba = bins_alpha; w.be = bins_eps; w.bee = bins_e;
    double* scratch = (double*)malloc(sizeof(double) * 3 * (size_t)w.nr);
    w.wa = scratch; w.we = scratch + w.nr; w.wee = scratch + 2 * w.nr;
    w.acc = accepted_ids; w.cap = cap;
    orc_tree tt = *t;
    if (!bins_e) tt.use_e = 0;
    w.t = &tt;
    int32_t n_img = p->bc == ORC_BC_CORNER ? 8 : 1;
    for (w.img = 0; w.img < n_img; ++w.img) walk_node(&w, 0, 0, 0, 0);
    free(scratch);
    if (n_accepted) *n_accepted = w.nacc;
    return w.visited;
}

void orc_column_density(const orc_tree* t, const orc_params* p, int64_t target, double* out)
{   /* cdMaps (R13): N_PIX column densities of one target, cm^-2 */
    walk_ctx w;
    memset(&w, 0, sizeof w);
    w.t = t; w.p = p;
    int32_t tl;
    int64_t p3[3], edge;
    target_geom(t, target, &tl, p3, &edge);
    w.tx = p3[0] * edge; w.ty = p3[1] * edge; w.tz = p3[2] * edge; w.ts = edge;
    w.cx = (double)w.tx + 0.5 * (double)edge;
    w.cy = (double)w.ty + 0.5 * (double)edge;
    w.cz = (double)w.tz + 0.5 * (double)edge;
    w.lray = lray_of(p);
    w.th_lim2 = p->theta_lim * p->theta_lim;
    w.th_if2 = p->theta_if * p->theta_if;
    w.th_src2 = p->theta_src * p->theta_src;
    int64_t npix = 12 * (int64_t)p->nside * p->nside;
    for (int64_t k = 0; k < npix; ++k) out[k] = 0.0;
    w.cd = out;
    int32_t n_img = p->bc == ORC_BC_CORNER ? 8 : 1;
    for (w.img = 0; w.img < n_img; ++w.img) walk_node(&w, 0, 0, 0, 0);
    /* mass n_H cells^3 over cells^2 -> n_H cells -> cm^-2 */
    for (int64_t k = 0; k < npix; ++k) out[k] *= t->dx_cm;
}

/* ------------------------------------------------------------------------ */
/* RTE along one ray in the OnTheSpot form (Sec. 2.5, Eq. 12-17).            */
/* ------------------------------------------------------------------------ */

double orc_sweep_ray(int32_t nr, int32_t eta_r, int32_t nside, int32_t zeta_g,
                     const double* alpha_vol, const double* eps, const double* e_vol,
                     double kd, double* phi0_out, double* loss_out)
{
    double* phi = (double*)malloc(sizeof(double) * (size_t)nr);
    for (int32_t j = 0; j < nr; ++j) {                 /* Eq. 12 */
        phi[j] = eps[j] / (4.0 * ORC_PI);
        if (loss_out) loss_out[j] = 0.0;
    }
    for (int32_t i = nr - 2; i >= 0; --i) {             /* far to near, segment [r_i, r_{i+1}] */
        double ri = orc_radius(i, eta_r), ri1 = orc_radius(i + 1, eta_r);
        double rm = 0.5 * (ri + ri1);
        double Ftot = 0.0;                              /* Eq. 11 at the segment midpoint (R7) */
        for (int32_t j = i + 1; j < nr; ++j) {
            double rj = orc_radius(j, eta_r);
            Ftot += phi[j] / ((rj - rm) * (rj - rm));
        }
        if (!(Ftot > 0.0)) continue;
        double zd = 1.0;                                /* Eq. 17, reading R7 */
        if (e_vol && e_vol[i + 1] > 0.0) zd = fmin(2.0, Ftot * kd / e_vol[i + 1]);
        double A = 0.5 * (alpha_vol[i] + alpha_vol[i + 1]);
        for (int32_t j = i + 1; j < nr; ++j) {
            if (!(phi[j] > 0.0)) continue;
            double rj = orc_radius(j, eta_r);
            double zs = (phi[j] / ((rj - rm) * (rj - rm))) / Ftot;        /* Eq. 16 (zeta_s) */
            double zg = 1.0;
            if (zeta_g) zg = fmin(1.0, (double)nside * (rj - ri) / (2.0 * rj));   /* Eq. 16 (zeta_g) */
            double a = rj - ri, b = rj - ri1;
            double dV = (a * a * a - b * b * b) / 3.0;                    /* Eq. 15 */
            double R = A * dV * zd * zs * zg;                             /* Eq. 14 */
            double np = phi[j] - R;                                       /* Eq. 13 */
            if (np < 0.0) np = 0.0;
            if (loss_out) loss_out[j] += phi[j] - np;
            phi[j] = np;
        }
    }
    double F0 = 0.0;                                    /* Eq. 10-11 at r_0 = 0 */
    for (int32_t j = 1; j < nr; ++j) {
        double rj = orc_radius(j, eta_r);
        F0 += phi[j] / (rj * rj);
    }
    if (phi0_out) for (int32_t j = 0; j < nr; ++j) phi0_out[j] = phi[j];
    free(phi);
    return F0;
}

/* ------------------------------------------------------------------------ */
/* One pass over the targets (Sec. 2.5 sum over directions, Eq. 18).         */
/* ------------------------------------------------------------------------ */

int32_t orc_solve_pass(const orc_tree* t, const orc_params* p, const int64_t* targets,
                       int64_t n_targets, double* F_out, double* e_out, uint8_t* ion_out)
{
    int64_t nc = t->n_leaf;
    double lray = lray_of(p);
    int32_t nr = orc_num_points(p->eta_r, lray);
    int64_t npix = 12 * (int64_t)p->nside * p->nside;
    int64_t nbin = npix * nr;
    double* ba = (double*)malloc(sizeof(double) * (size_t)nbin);
    double* be = (double*)malloc(sizeof(double) * (size_t)nbin);
    double* bee = t->use_e ? (double*)malloc(sizeof(double) * (size_t)nbin) : NULL;
    double* av = (double*)malloc(sizeof(double) * (size_t)nr);
    double* ev = (double*)malloc(sizeof(double) * (size_t)nr);
    double* vol = (double*)malloc(sizeof(double) * (size_t)nr);
    /* ray-cell volumes (R6) */
    for (int32_t i = 0; i < nr; ++i) {
        double lo = (i == 0) ? 0.0 : 0.5 * (orc_radius(i - 1, p->eta_r) + orc_radius(i, p->eta_r));
        double hi = (i == nr - 1) ? orc_radius(nr - 1, p->eta_r)
                                  : 0.5 * (orc_radius(i, p->eta_r) + orc_radius(i + 1, p->eta_r));
        vol[i] = (4.0 * ORC_PI / (double)npix) * (hi * hi * hi - lo * lo * lo) / 3.0;
    }
    double dx2 = t->dx_cm * t->dx_cm;
    double kd = p->hnu / (C_LIGHT * dx2);     /* F (per cell^2) -> F hnu / c in erg cm^-3 */
    int64_t n = targets ? n_targets : nc;
    for (int64_t q = 0; q < n; ++q) {
        int64_t tgt = targets ? targets[q] : q;
        orc_walk_target(t, p, tgt, ba, be, bee, NULL, 0, NULL);
        double F = 0.0;
        for (int64_t k = 0; k < npix; ++k) {
            for (int32_t i = 0; i < nr; ++i) {
                av[i] = ba[k * nr + i] / vol[i];
                if (bee) ev[i] = bee[k * nr + i] / vol[i];
            }
            F += orc_sweep_ray(nr, p->eta_r, p->nside, p->zeta_g, av, &be[k * nr],
                               bee ? ev : NULL, kd, NULL, NULL);
        }
        {
            int32_t tl;
            int64_t p3[3], edge;
            target_geom(t, tgt, &tl, p3, &edge);
            double rtp = 0.5 * (double)edge;
            F += t->eps_c[tgt] / (4.0 * ORC_PI * (rtp * rtp));   /* own emission, r_tp = half the cell (R3) */
        }
        double Fphys = F / dx2;
        if (F_out) F_out[q] = Fphys;
        if (e_out) e_out[q] = Fphys * p->hnu / C_LIGHT;   /* Eq. 18 */
        if (ion_out) ion_out[q] = (uint8_t)(F > 0.0);
    }
    free(ba); free(be); free(bee); free(av); free(ev); free(vol);
    return 0;
}

/* The flux each target would receive if nothing were absorbed: the photon
 * rates on its rays taken to the target unattenuated, sum_k sum_j
 * (eps_kj / 4 pi) / r_j^2, plus its own emission (R3); photons s^-1 cm^-2.
 * F_free - F is the flux the recombinations removed: a rounding error of
 * relative size u in the recombination terms moves F by about u times it,
 * which is how the tests judge reduced-precision results near a front. */
int32_t orc_free_flux(const orc_tree* t, const orc_params* p, const int64_t* targets,
                      int64_t n_targets, double* F_free_out)
{
    double lray = lray_of(p);
    int32_t nr = orc_num_points(p->eta_r, lray);
    int64_t npix = 12 * (int64_t)p->nside * p->nside;
    int64_t nbin = npix * nr;
    double* ba = (double*)malloc(sizeof(double) * (size_t)nbin);
    double* be = (double*)malloc(sizeof(double) * (size_t)nbin);
    double dx2 = t->dx_cm * t->dx_cm;
    int64_t n = targets ? n_targets : t->n_leaf;
    for (int64_t q = 0; q < n; ++q) {
        int64_t tgt = targets ? targets[q] : q;
        orc_walk_target(t, p, tgt, ba, be, NULL, NULL, 0, NULL);
        double F = 0.0;
        for (int64_t k = 0; k < npix; ++k)
            for (int32_t j = 1; j < nr; ++j) {
                double rj = orc_radius(j, p->eta_r);
                F += be[k * nr + j] / (4.0 * ORC_PI) / (rj * rj);
            }
        int32_t tl;
        int64_t p3[3], edge;
        target_geom(t, tgt, &tl, p3, &edge);
        double rtp = 0.5 * (double)edge;
        F += t->eps_c[tgt] / (4.0 * ORC_PI * (rtp * rtp));
        F_free_out[q] = F / dx2;
    }
    free(ba); free(be);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Iterations and error control (Sec. 2.6, Eq. 19-21).                       */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

double orc_delta(int64_t n, const double* e_new, const double* e_old, int32_t delta_mode)
{
    if (delta_mode == 1) {                      /* Eq. 20 (uniform cells: dV cancels) */
        double sn = 0.0, so = 0.0;
        for (int64_t c = 0; c < n; ++c) { sn += e_new[c]; so += e_old[c]; }
        if (sn + so == 0.0) return 0.0;
        return fabs(2.0 * (sn - so) / (sn + so));
    }
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);   /* Eq. 21 */
    memcpy(tmp, e_old, sizeof(double) * (size_t)n);
    qsort(tmp, (size_t)n, sizeof(double), cmp_double);
    double med = tmp[(n - 1) / 2];
    free(tmp);
    double dmax = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        double norm = fmax(e_old[c], med);
        double diff = fabs(e_new[c] - e_old[c]);
        double term = (norm > 0.0) ? diff / norm : (diff > 0.0 ? INFINITY : 0.0);
        if (term > dmax) dmax = term;
    }
    return dmax;
}

int32_t orc_solve(const orc_params* p, const double* box_lo_cm, const double* n_H,
                  const double* ndot_cell, int32_t nsrc, const double* src_xyz_cm,
                  const double* src_Q, const double* e_init, int32_t max_iter,
                  double eps_lim, int32_t delta_mode, double* F_out, double* e_out,
                  uint8_t* ion_out, int32_t* iters_out, double* delta_out)
{
    int64_t nc = (int64_t)p->N * p->N * p->N;
    double* e = (double*)calloc((size_t)nc, sizeof(double));
    double* en = (double*)calloc((size_t)nc, sizeof(double));
    if (e_init) memcpy(e, e_init, sizeof(double) * (size_t)nc);
    int32_t it = 0;
    double delta = INFINITY;
    while (it < max_iter) {
        orc_tree* t = orc_tree_build(p->N, p->dx_cm, p->alpha_B, box_lo_cm, n_H, ndot_cell,
                                     nsrc, src_xyz_cm, src_Q, e);
        orc_solve_pass(t, p, NULL, 0, F_out, en, ion_out);
        orc_tree_free(t);
        ++it;
        delta = orc_delta(nc, en, e, delta_mode);
        memcpy(e, en, sizeof(double) * (size_t)nc);
        if (delta < eps_lim) break;
    }
    if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)nc);
    if (iters_out) *iters_out = it;
    if (delta_out) *delta_out = delta;
    free(e); free(en);
    return 0;
}
