/*
 * hts_oracle.c -- plain, slow FP64 CPU oracle for the per-iteration gradient
 * of hyperbolic t-SNE ("Accelerating hyperbolic t-SNE", arXiv 2401.13708).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The CUDA
 * product path never calls it, links it or shares code with it.
 *
 * What it computes (all in double precision, C only, OpenMP over query rows):
 *   - Poincare-disk geometry: conformal factor (Eq. PoincareMetric), distance
 *     (Eq. PoincareDistance), its derivative (Eq. PoincareDistanceDerivative),
 *     Moebius addition and the exponential map (Sec. 4.2), the projection back
 *     into the disk (Eq. HyperbolicProjection), the Einstein midpoint
 *     (Eq. EinsteinMidpoint, Sec. 4.1).
 *   - The exact gradient of KL(P||Q^H) (Eq. KLGradientHyperbolic, split form
 *     Eq. KlGradientHyperbolicSplit), the normalisation Z^H (Eq.
 *     LowDimensionalProbabilityHyperbolic) and the KL cost (Eq. KLDivergence).
 *   - The modified polar quadtree (Sec. 4.1): annulus root, splits at the
 *     middle of the angular range and of the disk radius (Eq.
 *     EqualEmbeddingLengthsSplitting; Eq. EqualAreaSplitting as an option),
 *     built by literal one-point-at-a-time insertion with leaf capacity one,
 *     cell size r_cell (longest internal distance of a polar quad, Sec. 4.1),
 *     and a second, key-sorted construction used to check the first.
 *   - The Barnes-Hut repulsion: depth-first walk with the criterion
 *     r_cell / d^H(y_i, y_cell) < theta and the cell term of Eq.
 *     CellApproximation (Sec. 4.2).
 *   - The Riemannian gradient step with momentum (Sec. 5.1 protocol).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   R1  The printed Eq. KLGradientHyperbolic omits a factor d_ij: the exact
 *       derivative of KL with w = (1+d^2)^-1 is 4 sum (p-q) w d dd/dy, since
 *       dw = -2 w^2 d dd.  grad_form 0 uses the exact form (default), 1 the
 *       printed one.  The cell term gets the same factor.
 *   R2  "Product of lambda^-1 with the variation": the step rescales the
 *       Euclidean gradient by lambda^-metric_pow (default 1, the text).
 *   R3  r_cell = max of the hyperbolic lengths of the diagonal, one radial
 *       edge and the outer arc chord; the root annulus is always opened.
 *   R4  Root annulus r in [min|y|, max|y|], phi in [0, 2 pi) from atan2.
 *   R5  Equal-length splits are exact binary midpoints of the normalised
 *       coordinates rho^ = (r - r_min)/(r_max - r_min), phi^ = phi / 2 pi;
 *       a point on a split line goes to the upper child.
 *   R6  Depth cap L = 29 levels; a depth-L cell holding several points is a
 *       bucket whose points interact exactly.
 *   R7  j = i is skipped in leaves and buckets; an accepted cell that
 *       contains i keeps its full N_cell (cannot happen for theta < 1).
 *   R8  Gains (optional): +0.2 where sign(g) != sign(v), else *0.8, floor 0.01.
 *   R9  proj(y) = y (1 - eps) / |y| when |y| >= 1 - eps/2, eps = 1e-5.
 *   R13 Z^H = sum over ordered pairs k != l of (1 + d_kl^2)^-1.
 *   R14 The BH Z is the sum, over all query points, of the same walk's
 *       accepted-cell and leaf terms.
 *   R15 The Einstein midpoint is taken in Klein coordinates v = 2y/(1+|y|^2)
 *       with gamma(v) = (1+|y|^2)/(1-|y|^2), and mapped back to the disk
 *       by m / (1 + sqrt(1 - |m|^2)).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so every expression below rounds exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef _Float128 wide_t;

#define HO_LEVELS 29
#define HO_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */
/* ------------------------------------------------------------------------ */

int ho_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Geometry of the Poincare disk (Sec. 2.3)                                  */
/* ------------------------------------------------------------------------ */

static double sq2(double x, double y) { return x * x + y * y; }

/* Conformal factor lambda_y = 2 / (1 - |y|^2), Eq. PoincareMetric. */
double ho_lambda(const double *y) { return 2.0 / (1.0 - sq2(y[0], y[1])); }

/* acosh(1 + delta) written as log1p(delta + sqrt(delta (delta + 2))), the
 * identity acosh(x) = log(x + sqrt(x^2 - 1)) with x = 1 + delta, which keeps
 * full relative accuracy for small delta. */
double ho_acosh1p(double delta) { return log1p(delta + sqrt(delta * (delta + 2.0))); }

/* delta = gamma - 1 = 2 |a - b|^2 / ((1 - |a|^2)(1 - |b|^2)), Eq. PoincareDistance. */
static double pd_delta(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1];
    double al = 1.0 - sq2(a[0], a[1]);
    double be = 1.0 - sq2(b[0], b[1]);
    return 2.0 * sq2(dx, dy) / (al * be);
}

/* Hyperbolic distance d^H(a, b), Eq. PoincareDistance. */
double ho_dist(const double *a, const double *b) { return ho_acosh1p(pd_delta(a, b)); }

/* Derivative of d^H(y_i, y_j) with respect to y_i, Eq. PoincareDistanceDerivative:
 *   4 ((|y_j|^2 - 2<y_i,y_j> + 1) y_i / alpha - y_j) / (alpha beta sqrt(gamma^2 - 1)).
 * Since |y_j|^2 - 2<y_i,y_j> + 1 = |y_i - y_j|^2 + alpha = s + alpha, the
 * numerator vector equals (y_i - y_j) + (s / alpha) y_i; that form is used
 * because the printed one cancels for close pairs near the rim.
 * sqrt(gamma^2 - 1) is evaluated as sqrt(delta (delta + 2)).  Undefined at
 * y_i == y_j; returns 0 there (callers only use d * dd/dy, which tends to 0). */
void ho_dist_grad(const double *yi, const double *yj, double *out)
{
    double al = 1.0 - sq2(yi[0], yi[1]);
    double be = 1.0 - sq2(yj[0], yj[1]);
    double dx = yi[0] - yj[0], dy = yi[1] - yj[1];
    double s = sq2(dx, dy);
    if (s == 0.0) { out[0] = 0.0; out[1] = 0.0; return; }
    double delta = 2.0 * s / (al * be);
    double root = sqrt(delta * (delta + 2.0));
    double den = al * be * root;
    out[0] = 4.0 * (dx + (s / al) * yi[0]) / den;
    out[1] = 4.0 * (dy + (s / al) * yi[1]) / den;
}

/* Moebius addition a (+) b, Sec. 4.2. */
void ho_mobius_add(const double *a, const double *b, double *out)
{
    double ab = a[0] * b[0] + a[1] * b[1];
    double na = sq2(a[0], a[1]), nb = sq2(b[0], b[1]);
    double ca = 1.0 + 2.0 * ab + nb;
    double cb = 1.0 - na;
    double den = 1.0 + 2.0 * ab + na * nb;
    out[0] = (ca * a[0] + cb * b[0]) / den;
    out[1] = (ca * a[1] + cb * b[1]) / den;
}

/* Exponential map exp_y(v) = y (+) tanh(lambda_y |v| / 2) v / |v|, Sec. 4.2. */
void ho_exp_map(const double *y, const double *v, double *out)
{
    double nv = sqrt(sq2(v[0], v[1]));
    if (nv == 0.0) { out[0] = y[0]; out[1] = y[1]; return; }
    double t = tanh(ho_lambda(y) * nv / 2.0);
    double u[2] = {t * v[0] / nv, t * v[1] / nv};
    ho_mobius_add(y, u, out);
}

/* Projection into the open disk, Eq. HyperbolicProjection with reading R9. */
void ho_project(const double *y, double eps, double *out)
{
    double r = sqrt(sq2(y[0], y[1]));
    if (r >= 1.0 - eps / 2.0) {
        out[0] = y[0] * (1.0 - eps) / r;
        out[1] = y[1] * (1.0 - eps) / r;
    } else {
        out[0] = y[0];
        out[1] = y[1];
    }
}

/* Per-point Einstein terms (R15): gamma_j and gamma_j * v_j with v_j the
 * Klein coordinates of y_j.  gamma_j v_j simplifies to 2 y_j / (1 - |y_j|^2). */
static void einstein_terms(const double *y, double *g, double *ux, double *uy)
{
    double n2 = sq2(y[0], y[1]);
    double a = 1.0 - n2;
    *g = (1.0 + n2) / a;
    *ux = (2.0 * y[0]) / a;
    *uy = (2.0 * y[1]) / a;
}

/* Klein midpoint m = S_u / S_gamma mapped back to the Poincare disk. */
static void klein_to_poincare(double sg, double sux, double suy, double *out)
{
    double mx = sux / sg, my = suy / sg;
    double s = sqrt(1.0 - sq2(mx, my));
    out[0] = mx / (1.0 + s);
    out[1] = my / (1.0 + s);
}

/* Einstein midpoint of n points (Eq. EinsteinMidpoint), in disk coordinates. */
void ho_einstein_midpoint(int64_t n, const double *y, double *out)
{
    wide_t sg = 0, sx = 0, sy = 0;
    for (int64_t j = 0; j < n; ++j) {
        double g, ux, uy;
        einstein_terms(y + 2 * j, &g, &ux, &uy);
        sg += g; sx += ux; sy += uy;
    }
    klein_to_poincare((double)sg, (double)sx, (double)sy, out);
}

/* Hyperbolic distance between the polar points (ra, 0) and (rb, dphi),
 * given their exact radial gap drr = rb - ra.  The law of cosines written
 * as |p - q|^2 = drr^2 + 4 ra rb sin^2(dphi / 2) and 1 - r^2 = (1 - r)(1 + r)
 * avoid the cancellation of the Cartesian form for small cells. */
static double polar_dist(double ra, double rb, double drr, double dphi)
{
    double sh = sin(dphi / 2.0);
    double s = drr * drr + 4.0 * ra * rb * sh * sh;
    double delta = 2.0 * s / (((1.0 - ra) * (1.0 + ra)) * ((1.0 - rb) * (1.0 + rb)));
    return ho_acosh1p(delta);
}

/* Longest internal distance of the polar quad [r0, r1] x [phi, phi + dphi]
 * with radial gap dr = r1 - r0 (Sec. 4.1, reading R3): the max of the
 * diagonal, the radial edge and the outer-arc chord, each a hyperbolic
 * distance. */
static double rcell_gap(double r0, double r1, double dr, double dphi)
{
    double diag = polar_dist(r0, r1, dr, dphi);
    double radial = polar_dist(r0, r1, dr, 0.0);
    double arc = polar_dist(r1, r1, 0.0, dphi);
    double m = diag > radial ? diag : radial;
    return m > arc ? m : arc;
}

double ho_rcell(double r0, double r1, double dphi) { return rcell_gap(r0, r1, r1 - r0, dphi); }

/* ------------------------------------------------------------------------ */
/* Pair terms shared by the exact and Barnes-Hut sums                        */
/* ------------------------------------------------------------------------ */

/* For the pair (y_i, y_j): w = (1 + d^2)^-1 and the vector
 *   f = w * d * dd/dy_i (grad_form 0, reading R1)  or  w * dd/dy_i (grad_form 1).
 * Callers multiply f by p_ij (attraction) or by w (repulsion). */
static void pair_terms(const double *yi, const double *yj, int grad_form, double *w, double f[2])
{
    double d = ho_dist(yi, yj);
    double dd[2];
    ho_dist_grad(yi, yj, dd);
    *w = 1.0 / (1.0 + d * d);
    double k = grad_form == 0 ? (*w) * d : (*w);
    f[0] = k * dd[0];
    f[1] = k * dd[1];
}

static void attraction_row(int64_t i, const double *y, const int64_t *indptr, const int32_t *indices,
                           const double *vals, int grad_form, double out[2])
{
    out[0] = 0.0; out[1] = 0.0;
    for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) {
        int64_t j = indices[e];
        if (j == i) continue;
        double w, f[2];
        pair_terms(y + 2 * i, y + 2 * j, grad_form, &w, f);
        out[0] += vals[e] * f[0];
        out[1] += vals[e] * f[1];
    }
}

/* ------------------------------------------------------------------------ */
/* Exact gradient, Z and KL                                                   */
/* ------------------------------------------------------------------------ */

/* Exact sums over all ordered pairs j != i:
 *   Z = sum w_ij,  F_rep,i = sum w_ij f_ij,  F_attr,i = sum_{P row i} p_ij f_ij,
 *   g_i = 4 (exag F_attr,i - F_rep,i / Z)   (Eqs. KLGradientHyperbolic, KlGradientHyperbolicSplit).
 * Any output pointer may be NULL. */
void ho_exact_grad(int64_t n, const double *y, const int64_t *indptr, const int32_t *indices,
                   const double *vals, double exag, int grad_form,
                   double *g, double *fattr, double *frep, double *zrow, double *Z_out)
{
    double *fr = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double *fa = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double *zr = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double sx = 0, sy = 0, z = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double w, f[2];
            pair_terms(y + 2 * i, y + 2 * j, grad_form, &w, f);
            z += w;
            sx += w * f[0];
            sy += w * f[1];
        }
        fr[2 * i] = sx; fr[2 * i + 1] = sy; zr[i] = z;
        if (indptr) attraction_row(i, y, indptr, indices, vals, grad_form, fa + 2 * i);
        else { fa[2 * i] = 0; fa[2 * i + 1] = 0; }
    }
    double Z = 0;
    for (int64_t i = 0; i < n; ++i) Z += zr[i];
    for (int64_t i = 0; i < n; ++i) {
        double inv = Z > 0 ? 1.0 / Z : 0.0;
        if (g) {
            g[2 * i] = 4.0 * (exag * fa[2 * i] - fr[2 * i] * inv);
            g[2 * i + 1] = 4.0 * (exag * fa[2 * i + 1] - fr[2 * i + 1] * inv);
        }
        if (fattr) { fattr[2 * i] = fa[2 * i]; fattr[2 * i + 1] = fa[2 * i + 1]; }
        if (frep) { frep[2 * i] = fr[2 * i]; frep[2 * i + 1] = fr[2 * i + 1]; }
        if (zrow) zrow[i] = zr[i];
    }
    if (Z_out) *Z_out = Z;
    free(fr); free(fa); free(zr);
}

/* KL(P||Q^H) = sum p log p - sum p log w + (sum p) log Z over the stored
 * entries of P (Eq. KLDivergence with q = w / Z); p = 0 entries add nothing. */
double ho_kl_given_Z(int64_t n, const double *y, const int64_t *indptr, const int32_t *indices,
                     const double *vals, double Z)
{
    double s_plogp = 0, s_plogw = 0, s_p = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) {
            double p = vals[e];
            if (p <= 0.0) continue;
            double d = ho_dist(y + 2 * i, y + 2 * (int64_t)indices[e]);
            s_plogp += p * log(p);
            s_plogw += p * (-log1p(d * d));
            s_p += p;
        }
    }
    return s_plogp - s_plogw + s_p * log(Z);
}

double ho_exact_Z(int64_t n, const double *y)
{
    double Z = 0;
#pragma omp parallel for reduction(+ : Z) schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double z = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i) z += 1.0 / (1.0 + pow(ho_dist(y + 2 * i, y + 2 * j), 2));
        Z += z;
    }
    return Z;
}

/* ------------------------------------------------------------------------ */
/* Modified polar quadtree (Sec. 4.1)                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int depth;          /* 0 = root annulus */
    int is_leaf;
    int64_t ia, ib;     /* radial / angular cell index at this depth */
    int64_t child[4];   /* child c = 2 * (radial upper half) + (angular upper half); -1 = empty */
    int64_t point;      /* first point of a leaf (single point or depth-L bucket) */
    int64_t count;      /* N_cell */
    wide_t sg, sux, suy;/* Einstein sums: sum gamma_j, sum gamma_j v_j */
    double ycell[2];    /* midpoint (internal) or the point itself (leaf) */
    double rcell;       /* longest internal distance; +inf for the root */
} onode;

typedef struct {
    int64_t n, cap, size;
    onode *nodes;
    int64_t *next;      /* bucket chains: next point in the same depth-L cell */
    double *uh, *vh;    /* normalised radial / angular coordinates in [0, 1] */
    double radial_lo, radial_hi; /* root annulus in the split coordinate */
    int split_rule;     /* 0 = equal embedding length (Eq. 15), 1 = equal area (Eq. 6) */
} otree;

/* Radial split coordinate of a point: the disk radius r (equal length) or
 * cosh of the hyperbolic radius, (1 + r^2)/(1 - r^2) (equal area: Eq.
 * EqualAreaSplitting is the arithmetic midpoint of cosh). */
static double radial_coord(const double *y, int split_rule)
{
    double n2 = sq2(y[0], y[1]);
    if (split_rule == 1) return (1.0 + n2) / (1.0 - n2);
    return sqrt(n2);
}

/* Disk radius from a radial split coordinate. */
static double radius_of(double c, int split_rule)
{
    if (split_rule == 1) return sqrt((c - 1.0) / (c + 1.0));
    return c;
}

/* Size of the depth-`depth` cell with radial index ia: disk radii r0, r1 of
 * its bounds and their gap.  The gap in the split coordinate is
 * span * 2^-depth exactly; under equal-area splitting the radius gap follows
 * from r^2 = 1 - 2 / (c + 1):  r1 - r0 = 2 dc / ((c0 + 1)(c1 + 1)(r0 + r1)). */
static double cell_rcell(double lo, double hi, int64_t ia, int depth, int split_rule)
{
    double scale = ldexp(1.0, -depth);
    double span = hi - lo;
    double c0 = lo + span * ((double)ia * scale);
    double c1 = lo + span * ((double)(ia + 1) * scale);
    double dc = span * scale;
    double r0 = radius_of(c0, split_rule), r1 = radius_of(c1, split_rule);
    double dr = split_rule == 1 ? (r0 + r1 > 0.0 ? 2.0 * dc / ((c0 + 1.0) * (c1 + 1.0) * (r0 + r1)) : 0.0) : dc;
    return rcell_gap(r0, r1, dr, HO_TWO_PI * scale);
}

/* Normalised coordinates (R4, R5). */
static void normalise(int64_t n, const double *y, int split_rule, double *uh, double *vh, double *lo, double *hi)
{
    double rlo = INFINITY, rhi = -INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        double c = radial_coord(y + 2 * j, split_rule);
        if (c < rlo) rlo = c;
        if (c > rhi) rhi = c;
    }
    if (n == 0) { rlo = 0; rhi = 0; }
    for (int64_t j = 0; j < n; ++j) {
        double c = radial_coord(y + 2 * j, split_rule);
        uh[j] = rhi > rlo ? (c - rlo) / (rhi - rlo) : 0.0;
        double phi = atan2(y[2 * j + 1], y[2 * j]);
        if (phi < 0.0) phi += HO_TWO_PI;
        vh[j] = phi / HO_TWO_PI;
    }
    *lo = rlo; *hi = rhi;
}

/* Quantised, interleaved key (R5): digit l (l = 1 is the most significant)
 * is 2 * radial_bit + angular_bit of the depth-l cell.  Identical to the
 * path of the literal insertion below. */
static uint64_t quantise(double u)
{
    double s = floor(u * (double)(1u << HO_LEVELS));
    uint64_t q = (uint64_t)s;
    uint64_t top = ((uint64_t)1 << HO_LEVELS) - 1;
    return q > top ? top : q;
}

static uint64_t interleave(uint64_t qa, uint64_t qb, int levels)
{
    uint64_t k = 0;
    for (int b = 0; b < levels; ++b) {
        k |= ((qa >> b) & 1u) << (2 * b + 1);
        k |= ((qb >> b) & 1u) << (2 * b);
    }
    return k;
}

void ho_keys(int64_t n, const double *y, int split_rule, uint64_t *keys, double *bounds)
{
    double *uh = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *vh = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double lo, hi;
    normalise(n, y, split_rule, uh, vh, &lo, &hi);
    for (int64_t j = 0; j < n; ++j) keys[j] = interleave(quantise(uh[j]), quantise(vh[j]), HO_LEVELS);
    if (bounds) { bounds[0] = lo; bounds[1] = hi; }
    free(uh); free(vh);
}

static int64_t new_node(otree *t, int depth, int64_t ia, int64_t ib)
{
    if (t->size == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->nodes = (onode *)realloc(t->nodes, sizeof(onode) * (size_t)t->cap);
    }
    onode *nd = &t->nodes[t->size];
    memset(nd, 0, sizeof(onode));
    nd->depth = depth; nd->ia = ia; nd->ib = ib; nd->is_leaf = 1;
    nd->point = -1;
    for (int c = 0; c < 4; ++c) nd->child[c] = -1;
    return t->size++;
}

/* Child of `node` that holds point j: compare with the midpoints of the
 * node's normalised bounds [ia, ia+1) / 2^depth and [ib, ib+1) / 2^depth
 * (Eq. EqualEmbeddingLengthsSplitting for the radius, mid_phi = (max+min)/2). */
static int child_for(const otree *t, const onode *nd, int64_t j)
{
    double scale = ldexp(1.0, -nd->depth);
    double ulo = nd->ia * scale, uhi = (nd->ia + 1) * scale;
    double vlo = nd->ib * scale, vhi = (nd->ib + 1) * scale;
    int up_r = t->uh[j] >= (ulo + uhi) / 2.0;
    int up_a = t->vh[j] >= (vlo + vhi) / 2.0;
    return 2 * up_r + up_a;
}

static void add_terms(onode *nd, const double *yj)
{
    double g, ux, uy;
    einstein_terms(yj, &g, &ux, &uy);
    nd->sg += g; nd->sux += ux; nd->suy += uy;
}

/* Literal insertion of point j (Sec. 4.1: points are added one at a time and
 * the cell midpoints updated on the way down). */
static void insert_point(otree *t, const double *y, int64_t j)
{
    int64_t cur = 0;
    for (;;) {
        onode *nd = &t->nodes[cur];
        nd->count += 1;
        add_terms(nd, y + 2 * j);
        if (nd->is_leaf) {
            if (nd->count == 1) { nd->point = j; return; }
            if (nd->depth == HO_LEVELS) {      /* bucket (R6) */
                t->next[j] = t->next[nd->point];
                t->next[nd->point] = j;
                return;
            }
            /* split: push the resident point one level down */
            int64_t old = nd->point;
            nd->point = -1;
            nd->is_leaf = 0;
            int c = child_for(t, nd, old);
            int64_t ch = new_node(t, nd->depth + 1, 2 * t->nodes[cur].ia + (c >> 1), 2 * t->nodes[cur].ib + (c & 1));
            nd = &t->nodes[cur];
            nd->child[c] = ch;
            onode *cn = &t->nodes[ch];
            cn->count = 1; cn->point = old;
            add_terms(cn, y + 2 * old);
        }
        int c = child_for(t, nd, j);
        if (nd->child[c] < 0) {
            int64_t ch = new_node(t, nd->depth + 1, 2 * t->nodes[cur].ia + (c >> 1), 2 * t->nodes[cur].ib + (c & 1));
            t->nodes[cur].child[c] = ch;
            onode *cn = &t->nodes[ch];
            cn->count = 1; cn->point = j;
            add_terms(cn, y + 2 * j);
            return;
        }
        cur = nd->child[c];
    }
}

/* Midpoints and cell sizes once all points are in. */
static void finish_nodes(otree *t, const double *y)
{
    for (int64_t k = 0; k < t->size; ++k) {
        onode *nd = &t->nodes[k];
        if (nd->is_leaf && nd->count == 1) {
            nd->ycell[0] = y[2 * nd->point];
            nd->ycell[1] = y[2 * nd->point + 1];
        } else {
            klein_to_poincare((double)nd->sg, (double)nd->sux, (double)nd->suy, nd->ycell);
        }
        if (nd->depth == 0)
            nd->rcell = INFINITY;
        else
            nd->rcell = cell_rcell(t->radial_lo, t->radial_hi, nd->ia, nd->depth, t->split_rule);
    }
}

static otree *tree_build_insert(int64_t n, const double *y, int split_rule)
{
    otree *t = (otree *)calloc(1, sizeof(otree));
    t->n = n;
    t->split_rule = split_rule;
    t->uh = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    t->vh = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    t->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) t->next[j] = -1;
    normalise(n, y, split_rule, t->uh, t->vh, &t->radial_lo, &t->radial_hi);
    new_node(t, 0, 0, 0);
    for (int64_t j = 0; j < n; ++j) insert_point(t, y, j);
    finish_nodes(t, y);
    return t;
}

static void tree_free(otree *t)
{
    if (!t) return;
    free(t->nodes); free(t->next); free(t->uh); free(t->vh); free(t);
}

/* ------------------------------------------------------------------------ */
/* Tree export in compressed form (chains of one-child cells collapse to the  */
/* deepest cell), pre-order with children in key order.                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t cap, size;
    int32_t *depth; uint64_t *prefix; int64_t *count; int64_t *first;
    double *ycell; double *beta; double *rcell;
} export_t;

static void emit(export_t *ex, int depth, uint64_t prefix, int64_t count, int64_t first,
                 const double *yc, double rc)
{
    int64_t k = ex->size++;
    if (k >= ex->cap) return;
    if (ex->depth) ex->depth[k] = depth;
    if (ex->prefix) ex->prefix[k] = prefix;
    if (ex->count) ex->count[k] = count;
    if (ex->first) ex->first[k] = first;
    if (ex->ycell) { ex->ycell[2 * k] = yc[0]; ex->ycell[2 * k + 1] = yc[1]; }
    if (ex->beta) ex->beta[k] = 1.0 - sq2(yc[0], yc[1]);
    if (ex->rcell) ex->rcell[k] = rc;
}

static int nonempty_children(const onode *nd)
{
    int c = 0;
    for (int k = 0; k < 4; ++k) c += nd->child[k] >= 0;
    return c;
}

static void export_insert_rec(const otree *t, int64_t k, export_t *ex)
{
    const onode *nd = &t->nodes[k];
    if (!nd->is_leaf && nonempty_children(nd) == 1) {      /* chain: skip */
        for (int c = 0; c < 4; ++c)
            if (nd->child[c] >= 0) export_insert_rec(t, nd->child[c], ex);
        return;
    }
    uint64_t prefix = interleave((uint64_t)nd->ia, (uint64_t)nd->ib, nd->depth);
    int64_t first = nd->is_leaf ? nd->point : -1;
    if (nd->is_leaf && nd->count > 1) {                     /* bucket: smallest index first */
        int64_t m = nd->point;
        for (int64_t p = t->next[nd->point]; p >= 0; p = t->next[p]) if (p < m) m = p;
        first = m;
    }
    emit(ex, nd->depth, prefix, nd->count, first, nd->ycell, nd->rcell);
    if (!nd->is_leaf)
        for (int c = 0; c < 4; ++c)
            if (nd->child[c] >= 0) export_insert_rec(t, nd->child[c], ex);
}

/* Key-sorted construction: sort by key, then split each range on the next
 * key digit; sums taken directly over each range.  Used only to check that
 * the keys reproduce the inserted tree. */
static const uint64_t *g_sort_keys;
static int cmp_key(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
    if (ki != kj) return ki < kj ? -1 : 1;
    return i < j ? -1 : (i > j);
}

typedef struct {
    const double *y; const uint64_t *keys; const int64_t *order;
    double radial_lo, radial_hi; int split_rule;
} keytree_t;

static void export_key_rec(const keytree_t *kt, int depth, int64_t lo, int64_t hi, export_t *ex)
{
    uint64_t key0 = kt->keys[kt->order[lo]];
    if (hi - lo == 1) {
        int64_t j = kt->order[lo];
        uint64_t prefix = depth ? key0 >> (2 * (HO_LEVELS - depth)) : 0;
        double rc = INFINITY;
        emit(ex, depth, prefix, 1, j, kt->y + 2 * j, rc);
        return;
    }
    if (depth < HO_LEVELS) {
        int64_t cut[5]; int ne = 0;
        int shift = 2 * (HO_LEVELS - depth - 1);
        cut[0] = lo;
        for (int d = 0; d < 4; ++d) {
            int64_t e = cut[d];
            while (e < hi && (int)((kt->keys[kt->order[e]] >> shift) & 3u) == d) ++e;
            cut[d + 1] = e;
            ne += e > cut[d];
        }
        if (ne == 1) { export_key_rec(kt, depth + 1, lo, hi, ex); return; }
    }
    wide_t sg = 0, sx = 0, sy = 0;
    int64_t mfirst = kt->order[lo];
    for (int64_t e = lo; e < hi; ++e) {
        double g, ux, uy;
        int64_t j = kt->order[e];
        einstein_terms(kt->y + 2 * j, &g, &ux, &uy);
        sg += g; sx += ux; sy += uy;
        if (j < mfirst) mfirst = j;
    }
    double yc[2];
    klein_to_poincare((double)sg, (double)sx, (double)sy, yc);
    double rc = INFINITY;
    if (depth > 0) {
        uint64_t prefix = key0 >> (2 * (HO_LEVELS - depth));
        uint64_t ia = 0;
        for (int b = 0; b < depth; ++b) ia |= ((prefix >> (2 * b + 1)) & 1u) << b;
        rc = cell_rcell(kt->radial_lo, kt->radial_hi, (int64_t)ia, depth, kt->split_rule);
    }
    uint64_t prefix = depth ? key0 >> (2 * (HO_LEVELS - depth)) : 0;
    emit(ex, depth, prefix, hi - lo, depth == HO_LEVELS ? mfirst : -1, yc, rc);
    if (depth == HO_LEVELS) return;                       /* bucket */
    int shift = 2 * (HO_LEVELS - depth - 1);
    int64_t s = lo;
    while (s < hi) {
        int d = (int)((kt->keys[kt->order[s]] >> shift) & 3u);
        int64_t e = s;
        while (e < hi && (int)((kt->keys[kt->order[e]] >> shift) & 3u) == d) ++e;
        export_key_rec(kt, depth + 1, s, e, ex);
        s = e;
    }
}

/* Export the compressed tree.  which = 0: literal insertion; 1: key-sorted.
 * Returns the node count; arrays (each nullable) are filled up to `cap`.
 * For a single-point leaf `first` is the point and `rcell` is +inf; for a
 * bucket `first` is its smallest point index; internal nodes have first = -1.
 * bounds (nullable) receives the root annulus [lo, hi] of the radial
 * split coordinate. */
int64_t ho_tree_export(int64_t n, const double *y, int split_rule, int which, int64_t cap,
                       int32_t *depth, uint64_t *prefix, int64_t *count, int64_t *first,
                       double *ycell, double *beta, double *rcell, double *bounds)
{
    export_t ex = {cap, 0, depth, prefix, count, first, ycell, beta, rcell};
    if (n == 0) return 0;
    if (which == 0) {
        otree *t = tree_build_insert(n, y, split_rule);
        /* leaves report rcell = +inf and their own point as midpoint */
        for (int64_t k = 0; k < t->size; ++k)
            if (t->nodes[k].is_leaf && t->nodes[k].count == 1) t->nodes[k].rcell = INFINITY;
        export_insert_rec(t, 0, &ex);
        if (bounds) { bounds[0] = t->radial_lo; bounds[1] = t->radial_hi; }
        tree_free(t);
    } else {
        uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
        int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        double bb[2];
        ho_keys(n, y, split_rule, keys, bb);
        for (int64_t j = 0; j < n; ++j) order[j] = j;
        g_sort_keys = keys;
        qsort(order, (size_t)n, sizeof(int64_t), cmp_key);
        keytree_t kt = {y, keys, order, bb[0], bb[1], split_rule};
        export_key_rec(&kt, 0, 0, n, &ex);
        if (bounds) { bounds[0] = bb[0]; bounds[1] = bb[1]; }
        free(keys); free(order);
    }
    return ex.size;
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut repulsion (Sec. 4.2, Eq. CellApproximation)                     */
/* ------------------------------------------------------------------------ */

typedef struct { double fx, fy, z; int64_t accepted, pairs, visits; } bh_acc;

static void bh_visit(const otree *t, const double *y, int64_t k, int64_t i, double theta,
                     int grad_form, bh_acc *acc)
{
    const onode *nd = &t->nodes[k];
    const double *yi = y + 2 * i;
    acc->visits += 1;
    if (nd->is_leaf) {
        for (int64_t j = nd->point; j >= 0; j = t->next[j]) {
            if (j == i) continue;
            double w, f[2];
            pair_terms(yi, y + 2 * j, grad_form, &w, f);
            acc->z += w; acc->fx += w * f[0]; acc->fy += w * f[1];
            acc->pairs += 1;
        }
        return;
    }
    if (nd->depth >= 1) {
        double d = ho_dist(yi, nd->ycell);
        if (d > 0.0 && nd->rcell / d < theta) {
            double w, f[2];
            double m = (double)nd->count;
            pair_terms(yi, nd->ycell, grad_form, &w, f);
            acc->z += m * w; acc->fx += m * w * f[0]; acc->fy += m * w * f[1];
            acc->accepted += 1;
            return;
        }
    }
    for (int c = 0; c < 4; ++c)
        if (nd->child[c] >= 0) bh_visit(t, y, nd->child[c], i, theta, grad_form, acc);
}

/* Barnes-Hut gradient.  Z is the BH sum over all n query points (R14); the
 * per-row outputs are written for `rows` (nrows entries; rows == NULL means
 * all n rows in order).  stats (nullable): [accepted cells, leaf pairs,
 * visited nodes] summed over all n walks.  theta == 0 gives the exact sums. */
void ho_bh_grad(int64_t n, const double *y, const int64_t *indptr, const int32_t *indices,
                const double *vals, double theta, double exag, int split_rule, int grad_form,
                int64_t nrows, const int64_t *rows, double *g, double *fattr, double *frep,
                double *zall, double *Z_out, int64_t *stats)
{
    if (n == 0) { if (Z_out) *Z_out = 0; return; }
    otree *t = tree_build_insert(n, y, split_rule);
    double *zi = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t st[3] = {0, 0, 0};
    /* walk every point for Z; keep the forces of the requested rows */
    double *fr_all = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    int64_t acc_a = 0, acc_p = 0, acc_v = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : acc_a, acc_p, acc_v)
    for (int64_t i = 0; i < n; ++i) {
        bh_acc a = {0, 0, 0, 0, 0, 0};
        bh_visit(t, y, 0, i, theta, grad_form, &a);
        zi[i] = a.z; fr_all[2 * i] = a.fx; fr_all[2 * i + 1] = a.fy;
        acc_a += a.accepted; acc_p += a.pairs; acc_v += a.visits;
    }
    st[0] = acc_a; st[1] = acc_p; st[2] = acc_v;
    double Z = 0;
    for (int64_t i = 0; i < n; ++i) Z += zi[i];
    int64_t m = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < m; ++r) {
        int64_t i = rows ? rows[r] : r;
        double fa[2] = {0, 0};
        if (indptr) attraction_row(i, y, indptr, indices, vals, grad_form, fa);
        double inv = Z > 0 ? 1.0 / Z : 0.0;
        if (g) {
            g[2 * r] = 4.0 * (exag * fa[0] - fr_all[2 * i] * inv);
            g[2 * r + 1] = 4.0 * (exag * fa[1] - fr_all[2 * i + 1] * inv);
        }
        if (fattr) { fattr[2 * r] = fa[0]; fattr[2 * r + 1] = fa[1]; }
        if (frep) { frep[2 * r] = fr_all[2 * i]; frep[2 * r + 1] = fr_all[2 * i + 1]; }
    }
    if (zall) memcpy(zall, zi, sizeof(double) * (size_t)n);
    if (Z_out) *Z_out = Z;
    if (stats) { stats[0] = st[0]; stats[1] = st[1]; stats[2] = st[2]; }
    free(zi); free(fr_all);
    tree_free(t);
}

/* Barnes-Hut gradient for a subset of rows only, with Z supplied by the
 * caller (taken from a full oracle pass).  Used for sampled checks at large n. */
void ho_bh_rows(int64_t n, const double *y, const int64_t *indptr, const int32_t *indices,
                const double *vals, double theta, double exag, int split_rule, int grad_form,
                double Z, int64_t nrows, const int64_t *rows, double *g, double *frep_zi)
{
    otree *t = tree_build_insert(n, y, split_rule);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        bh_acc a = {0, 0, 0, 0, 0, 0};
        bh_visit(t, y, 0, i, theta, grad_form, &a);
        double fa[2] = {0, 0};
        if (indptr) attraction_row(i, y, indptr, indices, vals, grad_form, fa);
        if (g) {
            g[2 * r] = 4.0 * (exag * fa[0] - a.fx / Z);
            g[2 * r + 1] = 4.0 * (exag * fa[1] - a.fy / Z);
        }
        if (frep_zi) { frep_zi[3 * r] = a.fx; frep_zi[3 * r + 1] = a.fy; frep_zi[3 * r + 2] = a.z; }
    }
    tree_free(t);
}

/* A tree built once and walked for many row samples (timing of the oracle
 * on bounded samples).  Same arithmetic as ho_bh_rows. */
void *ho_bh_prepare(int64_t n, const double *y, int split_rule) { return tree_build_insert(n, y, split_rule); }

void ho_bh_release(void *t) { tree_free((otree *)t); }

void ho_bh_walk_rows(void *tp, const double *y, const int64_t *indptr, const int32_t *indices,
                     const double *vals, double theta, double exag, int grad_form, double Z, int64_t nrows,
                     const int64_t *rows, double *g)
{
    const otree *t = (const otree *)tp;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        bh_acc a = {0, 0, 0, 0, 0, 0};
        bh_visit(t, y, 0, i, theta, grad_form, &a);
        double fa[2] = {0, 0};
        if (indptr) attraction_row(i, y, indptr, indices, vals, grad_form, fa);
        if (g) {
            g[2 * r] = 4.0 * (exag * fa[0] - a.fx / Z);
            g[2 * r + 1] = 4.0 * (exag * fa[1] - a.fy / Z);
        }
    }
}

/* KL cost with the BH normalisation (theta > 0) or the exact one (theta == 0). */
double ho_kl(int64_t n, const double *y, const int64_t *indptr, const int32_t *indices,
             const double *vals, double theta, int split_rule)
{
    double Z;
    if (theta == 0.0) Z = ho_exact_Z(n, y);
    else ho_bh_grad(n, y, NULL, NULL, NULL, theta, 1.0, split_rule, 0, 0, NULL, NULL, NULL, NULL, NULL, &Z, NULL);
    return ho_kl_given_Z(n, y, indptr, indices, vals, Z);
}

/* ------------------------------------------------------------------------ */
/* Riemannian gradient step (Sec. 4.2 and Sec. 5.1)                           */
/* ------------------------------------------------------------------------ */

/* CO-SNE objective (Sec. 4.3): lambda1 KL + lambda2 H with
 *   H = (1/n) sum_i (|x_i|^2 - |y_i|^2)^2.
 * dH/dy_i = -(4/n)(|x_i|^2 - |y_i|^2) y_i, so the gradient is
 *   lambda1 g_KL,i - (4 lambda2 / n)(|x_i|^2 - |y_i|^2) y_i
 * (the variation printed in Sec. 4.3 carries the opposite sign; this is the
 * derivative of the stated cost).  xsq[i] = |x_i|^2. */
double ho_cosne_H(int64_t n, const double *y, const double *xsq)
{
    double h = 0;
    for (int64_t i = 0; i < n; ++i) {
        double t = xsq[i] - sq2(y[2 * i], y[2 * i + 1]);
        h += t * t;
    }
    return n > 0 ? h / (double)n : 0.0;
}

void ho_cosne_grad(int64_t n, const double *y, const double *xsq, double l1, double l2, const double *gkl,
                   double *g)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = xsq[i] - sq2(y[2 * i], y[2 * i + 1]);
        double c = 4.0 * l2 / (double)n * t;
        g[2 * i] = l1 * gkl[2 * i] - c * y[2 * i];
        g[2 * i + 1] = l1 * gkl[2 * i + 1] - c * y[2 * i + 1];
    }
}

/* n_iter iterations of: g = gradient (exact when theta == 0, else BH; with
 * the CO-SNE term when xsq != NULL); r = lambda^-metric_pow g (R2); optional
 * gains (R8); v = momentum v - lr gains r; y = proj(exp_y(v)) (R9).  y, v,
 * gains (nullable when use_gains == 0) are updated in place. */
static void step_impl(int64_t n, double *y, double *v, double *gains, const int64_t *indptr,
                      const int32_t *indices, const double *vals, int n_iter, double theta, double exag,
                      double lr, double momentum, int split_rule, int grad_form, int metric_pow, double eps,
                      int use_gains, const double *xsq, double l1, double l2)
{
    double *g = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    for (int it = 0; it < n_iter; ++it) {
        if (theta == 0.0)
            ho_exact_grad(n, y, indptr, indices, vals, exag, grad_form, g, NULL, NULL, NULL, NULL);
        else
            ho_bh_grad(n, y, indptr, indices, vals, theta, exag, split_rule, grad_form, 0, NULL,
                       g, NULL, NULL, NULL, NULL, NULL);
        if (xsq) ho_cosne_grad(n, y, xsq, l1, l2, g, g);
        for (int64_t i = 0; i < n; ++i) {
            double *yi = y + 2 * i, *vi = v + 2 * i;
            double lam = ho_lambda(yi);
            double scale = metric_pow == 2 ? 1.0 / (lam * lam) : 1.0 / lam;
            for (int k = 0; k < 2; ++k) {
                double r = g[2 * i + k] * scale;
                double gk = 1.0;
                if (use_gains) {
                    double *gn = gains + 2 * i + k;
                    int same = (g[2 * i + k] > 0.0) == (vi[k] > 0.0);
                    *gn = same ? (*gn) * 0.8 : (*gn) + 0.2;
                    if (*gn < 0.01) *gn = 0.01;
                    gk = *gn;
                }
                vi[k] = momentum * vi[k] - lr * gk * r;
            }
            double ye[2], yp[2];
            ho_exp_map(yi, vi, ye);
            ho_project(ye, eps, yp);
            yi[0] = yp[0]; yi[1] = yp[1];
        }
    }
    free(g);
}

void ho_step(int64_t n, double *y, double *v, double *gains, const int64_t *indptr,
             const int32_t *indices, const double *vals, int n_iter, double theta, double exag,
             double lr, double momentum, int split_rule, int grad_form, int metric_pow,
             double eps, int use_gains)
{
    step_impl(n, y, v, gains, indptr, indices, vals, n_iter, theta, exag, lr, momentum, split_rule, grad_form,
              metric_pow, eps, use_gains, NULL, 1.0, 0.0);
}

void ho_step_cosne(int64_t n, double *y, double *v, const int64_t *indptr, const int32_t *indices,
                   const double *vals, int n_iter, double theta, double exag, double lr, double momentum,
                   const double *xsq, double l1, double l2)
{
    step_impl(n, y, v, NULL, indptr, indices, vals, n_iter, theta, exag, lr, momentum, 0, 0, 1, 1e-5, 0, xsq,
              l1, l2);
}
