/*
 * paraboloid.c -- oracle for the cut-cell quantities the paper takes from the
 * fitted paraboloid itself (Sec. 3.2, the paragraph after Eq. volumefit2):
 * with z = P(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 x y + a5 y^2 in the cell
 * frame [t1 t2 n] (origin at the cell centre, lengths in cell widths, so the
 * cell is [-1/2, 1/2]^3 and V_C = 1),
 *
 *   alpha_P = V_P = |{X in cell : n.X <= P(t1.X, t2.X)}|     (alpha = V_P / V_C)
 *   A       = area of the surface S = {z = P(x, y)} inside the cell
 *   kbar    = (1/A) int_{S in cell} kappa dA,   kappa = div n (> 0 on a sphere)
 *   nbar    = int_{S in cell} n dA / |int_{S in cell} n dA|, n the upward normal
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Every quantity is its definition,
 * integrated by nested adaptive Gauss-Kronrod (7/15) quadrature:
 *  - V_P: over the cell's (X1, X2) square; along X3 the set below the
 *    paraboloid is found exactly (F(X) = P - n.X is a quadratic in X3: its
 *    roots split [-1/2, 1/2] and a midpoint test keeps the pieces with F > 0).
 *  - the surface integrals: over the (x, y) parameter plane of the graph,
 *    dA = W dx dy, W = sqrt(1 + Px^2 + Py^2); for each y the set of x whose
 *    surface point lies in the cell is found exactly (each world coordinate
 *    of the point is a quadratic in x), and the smooth integrand is integrated
 *    over its pieces.
 * Each smooth piece is integrated adaptively: a panel is accepted when its
 * 15-point Kronrod value agrees with the sum over its halves within the
 * tolerance per unit length (1e-12 for the outer integrals, a fifth and a tenth
 * of that for the inner ones, whose error is the outer integrand's noise), or
 * at a width of 1e-9; differences below 1e-12 of the panel's value count as
 * noise (the column length comes from roots of a quadratic sampled at three
 * points, relative errors of a few 1e-14, more near a double root).  The
 * results are good to about 1e-12.
 * Parity: pinned by the closed forms of planes cutting a cube, of paraboloids
 * that cross the whole cell, by the complement identity V(P) + V(-P) = 1, by
 * cube symmetries and by the divergence identity for int n dA.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* 15-point Kronrod nodes on [-1, 1] (descending, last = 0), their weights, and
 * the weights of the embedded 7-point Gauss rule (nodes 1, 3, 5 and 7). */
static const double GK_X[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
static const double GK_WK[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

#define PB_ND 5

typedef void (*pb_fn)(const void* ctx, double s, double* out);

static void pb_gk15(pb_fn f, const void* ctx, int nd, double a, double b, double* K, double* err) {
    const double c = 0.5 * (a + b), hw = 0.5 * (b - a);
    double fc[PB_ND], f1[PB_ND], f2[PB_ND], G[PB_ND];
    f(ctx, c, fc);
    for (int d = 0; d < nd; d++) {
        K[d] = GK_WK[7] * fc[d];
        G[d] = GK_WG[3] * fc[d];
    }
    for (int j = 0; j < 7; j++) {
        const double x = hw * GK_X[j];
        f(ctx, c - x, f1);
        f(ctx, c + x, f2);
        for (int d = 0; d < nd; d++) {
            K[d] += GK_WK[j] * (f1[d] + f2[d]);
            if (j & 1) G[d] += GK_WG[j >> 1] * (f1[d] + f2[d]);
        }
    }
    double e = 0.0;
    for (int d = 0; d < nd; d++) {
        K[d] *= hw;
        G[d] *= hw;
        const double dd = fabs(K[d] - G[d]);
        if (dd > e) e = dd;
    }
    *err = e;
}

/* adds the integral of f over [a, b] to out[0..nd): a panel whose 15-point
 * Kronrod value K agrees with the sum of the Kronrod values of its two halves
 * (and whose embedded Gauss value agrees with K) within tol per unit length
 * keeps the halves' sum; else each half is refined with its value reused. */
static void pb_refine(pb_fn f, const void* ctx, int nd, double a, double b, const double* K, double tol, double* out,
                      int depth) {
    const double m = 0.5 * (a + b);
    double Kl[PB_ND], Kr[PB_ND], el, er;
    pb_gk15(f, ctx, nd, a, m, Kl, &el);
    pb_gk15(f, ctx, nd, m, b, Kr, &er);
    double e = 0.0, mag = 0.0;
    for (int d = 0; d < nd; d++) {
        const double dd = fabs(K[d] - (Kl[d] + Kr[d]));
        if (dd > e) e = dd;
        if (fabs(K[d]) > mag) mag = fabs(K[d]);
    }
    /* the noise floor of the panel values (roots from sampled quadratics carry
     * relative errors of a few 1e-14; inner integrals their own tolerance):
     * below it a difference says nothing */
    const double floor = 1e-12 * mag;
    if ((e <= tol * (b - a) + floor && el <= tol * (m - a) + floor && er <= tol * (b - m) + floor) ||
        b - a <= 1e-9 || depth >= 60) {
        for (int d = 0; d < nd; d++) out[d] += Kl[d] + Kr[d];
        return;
    }
    pb_refine(f, ctx, nd, a, m, Kl, tol, out, depth + 1);
    pb_refine(f, ctx, nd, m, b, Kr, tol, out, depth + 1);
}

static void pb_adapt(pb_fn f, const void* ctx, int nd, double a, double b, double tol, double* out, int depth) {
    double K[PB_ND], e;
    pb_gk15(f, ctx, nd, a, b, K, &e);
    pb_refine(f, ctx, nd, a, b, K, tol, out, depth);
}

/* the same over `np` equal panels of [a, b] first (so that the error estimate
 * of a first, wide panel cannot pass over a narrow feature) */
static void pb_adapt_n(pb_fn f, const void* ctx, int nd, double a, double b, double tol, double* out, int np) {
    for (int i = 0; i < np; i++)
        pb_adapt(f, ctx, nd, a + (b - a) * i / np, a + (b - a) * (i + 1) / np, tol, out, 0);
}

typedef struct {
    double t1[3], t2[3], n[3], a[6];
} pb_cell;

static double pb_P(const pb_cell* q, double x, double y) {
    const double* a = q->a;
    return a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y;
}

/* F(X) = P(t1.X, t2.X) - n.X: positive below the paraboloid */
static double pb_F(const pb_cell* q, const double X[3]) {
    const double x = q->t1[0] * X[0] + q->t1[1] * X[1] + q->t1[2] * X[2];
    const double y = q->t2[0] * X[0] + q->t2[1] * X[1] + q->t2[2] * X[2];
    const double z = q->n[0] * X[0] + q->n[1] * X[1] + q->n[2] * X[2];
    return pb_P(q, x, y) - z;
}

/* real roots of c2 s^2 + c1 s + c0 strictly inside (lo, hi), appended to r */
static int pb_roots(double c2, double c1, double c0, double lo, double hi, double* r) {
    int n = 0;
    double s[2];
    int k = 0;
    if (c2 == 0.0) {
        if (c1 != 0.0) s[k++] = -c0 / c1;
    } else {
        const double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc >= 0.0) {
            const double qq = -0.5 * (c1 + copysign(sqrt(disc), c1));
            s[k++] = qq / c2;
            if (qq != 0.0) s[k++] = c0 / qq;
        }
    }
    for (int i = 0; i < k; i++)
        if (s[i] > lo && s[i] < hi) r[n++] = s[i];
    return n;
}

static void pb_sort(double* v, int n) {
    for (int i = 1; i < n; i++) {
        const double x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; j--; }
        v[j + 1] = x;
    }
}

/* ---- V_P ---- */

typedef struct {
    const pb_cell* q;
    double X1;
    double tol;
} pb_vctx;

/* length of {s in [-1/2, 1/2] : F(X1, X2, s) > 0} */
static void pb_column(const void* c, double X2, double* out) {
    const pb_vctx* v = (const pb_vctx*)c;
    double X[3] = {v->X1, X2, -0.5};
    const double fm = pb_F(v->q, X);
    X[2] = 0.0;
    const double f0 = pb_F(v->q, X);
    X[2] = 0.5;
    const double fp = pb_F(v->q, X);
    /* F along the column is quadratic in s: c0 + c1 s + c2 s^2 through the three values */
    const double c0 = f0, c1 = fp - fm, c2 = 2.0 * (fp + fm - 2.0 * f0);
    double pts[4];
    int np = 0;
    pts[np++] = -0.5;
    np += pb_roots(c2, c1, c0, -0.5, 0.5, pts + np);
    pts[np++] = 0.5;
    pb_sort(pts, np);
    double len = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        X[2] = 0.5 * (pts[i] + pts[i + 1]);
        if (pb_F(v->q, X) > 0.0) len += pts[i + 1] - pts[i];
    }
    out[0] = len;
}

/* the column lengths over X2 in [-1/2, 1/2] at this X1.  The length is smooth
 * between the X2 where a root of the column quadratic crosses s = +-1/2 or
 * the two roots meet (its discriminant vanishes); both sets are quadratics in
 * X2, found from three samples.  Each piece is integrated in the variable
 * tau with X2 = p + (q - p)(1 - cos(pi tau))/2, which turns the square-root
 * behaviour at a piece end into a smooth function of tau. */
typedef struct {
    pb_vctx v;
    double p, q;
} pb_piece;

static void pb_column_tau(const void* c, double tau, double* out) {
    const pb_piece* pc = (const pb_piece*)c;
    const double X2 = pc->p + (pc->q - pc->p) * 0.5 * (1.0 - cos(M_PI * tau));
    pb_column(&pc->v, X2, out);
    out[0] *= (pc->q - pc->p) * 0.5 * M_PI * sin(M_PI * tau);
}

static void pb_disc_at(const pb_vctx* v, double X2, double* dv, double* fm_out, double* fp_out) {
    double X[3] = {v->X1, X2, -0.5};
    const double fm = pb_F(v->q, X);
    X[2] = 0.0;
    const double f0 = pb_F(v->q, X);
    X[2] = 0.5;
    const double fp = pb_F(v->q, X);
    const double c0 = f0, c1 = fp - fm, c2 = 2.0 * (fp + fm - 2.0 * f0);
    *dv = c1 * c1 - 4.0 * c2 * c0;
    *fm_out = fm;
    *fp_out = fp;
}

static void pb_slab(const void* c, double X1, double* out) {
    pb_piece pc;
    pc.v = *(const pb_vctx*)c;
    pc.v.X1 = X1;
    double d[3], fm[3], fp[3];
    const double xs[3] = {-0.5, 0.0, 0.5};
    for (int i = 0; i < 3; i++) pb_disc_at(&pc.v, xs[i], &d[i], &fm[i], &fp[i]);
    double pts[12];
    int np = 0;
    pts[np++] = -0.5;
    /* each sampled function g is quadratic in X2: c0 + c1 X2 + c2 X2^2 */
    const double* g[3] = {d, fm, fp};
    for (int k = 0; k < 3; k++) {
        const double c0 = g[k][1], c1 = g[k][2] - g[k][0], c2 = 2.0 * (g[k][2] + g[k][0] - 2.0 * g[k][1]);
        np += pb_roots(c2, c1, c0, -0.5, 0.5, pts + np);
    }
    pts[np++] = 0.5;
    pb_sort(pts, np);
    out[0] = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        if (!(pts[i + 1] > pts[i])) continue;
        pc.p = pts[i];
        pc.q = pts[i + 1];
        pb_adapt_n(pb_column_tau, &pc, 1, 0.0, 1.0, pc.v.tol, out, 4);
    }
}

/* ---- surface integrals ---- */

typedef struct {
    const pb_cell* q;
    double y;
    double tol;
} pb_sctx;

/* W, kappa W and the world components of n W at the surface point over (x, y) */
static void pb_surface_point(const void* c, double x, double* out) {
    const pb_sctx* s = (const pb_sctx*)c;
    const double* a = s->q->a;
    const double y = s->y;
    const double px = a[1] + 2.0 * a[3] * x + a[4] * y, py = a[2] + a[4] * x + 2.0 * a[5] * y;
    const double pxx = 2.0 * a[3], pxy = a[4], pyy = 2.0 * a[5];
    const double W2 = 1.0 + px * px + py * py, W = sqrt(W2);
    /* mean curvature (sum of the principal curvatures) of the graph, > 0 where it bends down */
    const double kappa = -((1.0 + py * py) * pxx - 2.0 * px * py * pxy + (1.0 + px * px) * pyy) / (W2 * W);
    out[0] = W;
    out[1] = kappa * W;
    /* n dA = (-Px t1 - Py t2 + n) dx dy */
    for (int d = 0; d < 3; d++) out[2 + d] = -px * s->q->t1[d] - py * s->q->t2[d] + s->q->n[d];
}

static int pb_in_cell(const pb_cell* q, double x, double y) {
    const double z = pb_P(q, x, y);
    for (int d = 0; d < 3; d++) {
        const double X = x * q->t1[d] + y * q->t2[d] + z * q->n[d];
        if (!(fabs(X) <= 0.5)) return 0;
    }
    return 1;
}

static const double PB_R = 0.8660254037844387; /* |x|, |y| <= sqrt(3)/2 on the cell */

static void pb_row(const void* c, double y, double* out) {
    pb_sctx row = *(const pb_sctx*)c;
    row.y = y;
    const pb_sctx* s = &row;
    const pb_cell* q = s->q;
    const double* a = q->a;
    for (int d = 0; d < PB_ND; d++) out[d] = 0.0;
    /* world coordinate d of the surface point: X_d(x) = e2 x^2 + e1 x + e0 */
    double pts[16];
    int np = 0;
    pts[np++] = -PB_R;
    for (int d = 0; d < 3; d++) {
        const double e2 = q->n[d] * a[3];
        const double e1 = q->t1[d] + q->n[d] * (a[1] + a[4] * s->y);
        const double e0 = q->t2[d] * s->y + q->n[d] * (a[0] + a[2] * s->y + a[5] * s->y * s->y);
        np += pb_roots(e2, e1, e0 - 0.5, -PB_R, PB_R, pts + np);
        np += pb_roots(e2, e1, e0 + 0.5, -PB_R, PB_R, pts + np);
    }
    pts[np++] = PB_R;
    pb_sort(pts, np);
    for (int i = 0; i + 1 < np; i++) {
        if (!(pts[i + 1] > pts[i])) continue;
        if (!pb_in_cell(q, 0.5 * (pts[i] + pts[i + 1]), s->y)) continue;
        pb_adapt(pb_surface_point, s, PB_ND, pts[i], pts[i + 1], s->tol, out, 0);
    }
}

/* The row integral is smooth in y between the y where the set of x changes:
 * where one of the six curves X_d = +-1/2 on the surface has a double root in
 * x (its discriminant, a quadratic in y, vanishes) and where the surface
 * crosses a cube edge (a quadratic along the edge).  Pieces use the same
 * cosine substitution as the volume. */
typedef struct {
    pb_sctx s;
    double p, q;
} pb_spiece;

static void pb_row_tau(const void* c, double tau, double* out) {
    const pb_spiece* pc = (const pb_spiece*)c;
    const double y = pc->p + (pc->q - pc->p) * 0.5 * (1.0 - cos(M_PI * tau));
    pb_row(&pc->s, y, out);
    const double J = (pc->q - pc->p) * 0.5 * M_PI * sin(M_PI * tau);
    for (int d = 0; d < PB_ND; d++) out[d] *= J;
}

static void pb_surface(const pb_cell* q, double tol, double* I) {
    const double* a = q->a;
    double pts[64];
    int np = 0;
    pts[np++] = -PB_R;
    for (int d = 0; d < 3; d++) {
        /* X_d(x) = e2 x^2 + e1(y) x + e0(y): e1 linear, e0 quadratic in y */
        const double e2 = q->n[d] * a[3];
        const double e1c = q->t1[d] + q->n[d] * a[1], e1y = q->n[d] * a[4];
        const double e0c = q->n[d] * a[0], e0y = q->t2[d] + q->n[d] * a[2], e0yy = q->n[d] * a[5];
        for (int sg = -1; sg <= 1; sg += 2) {
            /* discriminant e1^2 - 4 e2 (e0 - sg/2) as a quadratic in y */
            const double c2 = e1y * e1y - 4.0 * e2 * e0yy;
            const double c1 = 2.0 * e1c * e1y - 4.0 * e2 * e0y;
            const double c0 = e1c * e1c - 4.0 * e2 * (e0c - 0.5 * sg);
            np += pb_roots(c2, c1, c0, -PB_R, PB_R, pts + np);
        }
    }
    /* a world coordinate that does not depend on x (the surface is a cylinder
     * along x in that direction, as a plane lying in a cube face is) bounds the
     * domain at the y where it equals +-1/2 */
    for (int d = 0; d < 3; d++) {
        if (q->n[d] * a[3] != 0.0 || q->t1[d] + q->n[d] * a[1] != 0.0 || q->n[d] * a[4] != 0.0) continue;
        for (int sg = -1; sg <= 1; sg += 2)
            np += pb_roots(q->n[d] * a[5], q->t2[d] + q->n[d] * a[2], q->n[d] * a[0] - 0.5 * sg, -PB_R, PB_R,
                           pts + np);
    }
    /* the twelve cube edges: X_d = +-1/2, X_e = +-1/2, the third coordinate free */
    for (int f = 0; f < 3; f++)
        for (int s1 = -1; s1 <= 1; s1 += 2)
            for (int s2 = -1; s2 <= 1; s2 += 2) {
                const int d = (f + 1) % 3, e = (f + 2) % 3;
                double X[3], fv[3];
                X[d] = 0.5 * s1;
                X[e] = 0.5 * s2;
                const double ts[3] = {-0.5, 0.0, 0.5};
                for (int i = 0; i < 3; i++) {
                    X[f] = ts[i];
                    fv[i] = pb_F(q, X);
                }
                double r[2];
                const int nr = pb_roots(2.0 * (fv[2] + fv[0] - 2.0 * fv[1]), fv[2] - fv[0], fv[1], -0.5, 0.5, r);
                for (int i = 0; i < nr; i++) {
                    X[f] = r[i];
                    pts[np++] = q->t2[0] * X[0] + q->t2[1] * X[1] + q->t2[2] * X[2];
                }
            }
    pts[np++] = PB_R;
    pb_sort(pts, np);
    pb_spiece pc;
    pc.s.q = q;
    pc.s.y = 0.0;
    pc.s.tol = 0.1 * tol;  /* inner integrals below the outer tolerance */
    for (int d = 0; d < PB_ND; d++) I[d] = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        if (!(pts[i + 1] > pts[i])) continue;
        pc.p = pts[i];
        pc.q = pts[i + 1];
        pb_adapt_n(pb_row_tau, &pc, PB_ND, 0.0, 1.0, tol, I, 4);
    }
}

/* The slab area I(X1) = int len dX2 is smooth between the X1 at which the
 * cross-section {F(X1, ., .) = 0} of the square [-1/2, 1/2]^2 changes shape:
 * it passes through a corner of the square (the surface crosses a cube edge
 * along X1), touches a side (the discriminant along that side vanishes), or
 * degenerates (the determinant of the section's 3x3 conic matrix vanishes).
 * Each is a quadratic in X1, found from three samples.  The pieces use the
 * cosine substitution. */
typedef struct {
    pb_vctx v;
    double p, q;
} pb_xpiece;

static void pb_slab_tau(const void* c, double tau, double* out) {
    const pb_xpiece* pc = (const pb_xpiece*)c;
    const double X1 = pc->p + (pc->q - pc->p) * 0.5 * (1.0 - cos(M_PI * tau));
    pb_slab(&pc->v, X1, out);
    out[0] *= (pc->q - pc->p) * 0.5 * M_PI * sin(M_PI * tau);
}

/* the section quadratic q(u, v) = F(X1, u, v) = Quu u^2 + Quv u v + Qvv v^2 + Lu u + Lv v + c */
static void pb_section(const pb_cell* q, double X1, double* Q) {
    double X[3] = {X1, 0.0, 0.0};
    const double f00 = pb_F(q, X);
    X[1] = 0.5;
    const double fp0 = pb_F(q, X);
    X[1] = -0.5;
    const double fm0 = pb_F(q, X);
    X[1] = 0.0;
    X[2] = 0.5;
    const double f0p = pb_F(q, X);
    X[2] = -0.5;
    const double f0m = pb_F(q, X);
    X[1] = 0.5;
    X[2] = 0.5;
    const double fpp = pb_F(q, X);
    const double Lu = fp0 - fm0, Quu = 2.0 * (fp0 + fm0 - 2.0 * f00);
    const double Lv = f0p - f0m, Qvv = 2.0 * (f0p + f0m - 2.0 * f00);
    const double Quv = 4.0 * (fpp - f00 - 0.5 * Lu - 0.5 * Lv - 0.25 * Quu - 0.25 * Qvv);
    Q[0] = Quu; Q[1] = Quv; Q[2] = Qvv; Q[3] = Lu; Q[4] = Lv; Q[5] = f00;
}

/* the event functions at X1: 4 corner values, 4 side discriminants, the conic determinant */
static void pb_events(const pb_cell* q, double X1, double* ev) {
    double Q[6];
    pb_section(q, X1, Q);
    const double Quu = Q[0], Quv = Q[1], Qvv = Q[2], Lu = Q[3], Lv = Q[4], c = Q[5];
    int k = 0;
    for (int su = -1; su <= 1; su += 2)
        for (int sv = -1; sv <= 1; sv += 2) {
            const double u = 0.5 * su, v = 0.5 * sv;
            ev[k++] = Quu * u * u + Quv * u * v + Qvv * v * v + Lu * u + Lv * v + c;
        }
    for (int s = -1; s <= 1; s += 2) {
        const double u = 0.5 * s;  /* side u = +-1/2: quadratic in v */
        const double b = Quv * u + Lv, cc = Quu * u * u + Lu * u + c;
        ev[k++] = b * b - 4.0 * Qvv * cc;
        const double v = 0.5 * s;  /* side v = +-1/2: quadratic in u */
        const double b2 = Quv * v + Lu, c2 = Qvv * v * v + Lv * v + c;
        ev[k++] = b2 * b2 - 4.0 * Quu * c2;
    }
    /* det [[Quu, Quv/2, Lu/2], [Quv/2, Qvv, Lv/2], [Lu/2, Lv/2, c]] */
    const double a11 = Quu, a12 = 0.5 * Quv, a13 = 0.5 * Lu, a22 = Qvv, a23 = 0.5 * Lv, a33 = c;
    ev[k++] = a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13) + a13 * (a12 * a23 - a22 * a13);
}

static double pb_volume(const pb_cell* q, double tol) {
    double e[3][9];
    const double xs[3] = {-0.5, 0.0, 0.5};
    for (int i = 0; i < 3; i++) pb_events(q, xs[i], e[i]);
    double pts[24];
    int np = 0;
    pts[np++] = -0.5;
    for (int k = 0; k < 9; k++) {
        /* every event function is a quadratic in X1 */
        const double c0 = e[1][k], c1 = e[2][k] - e[0][k], c2 = 2.0 * (e[2][k] + e[0][k] - 2.0 * e[1][k]);
        np += pb_roots(c2, c1, c0, -0.5, 0.5, pts + np);
    }
    pts[np++] = 0.5;
    pb_sort(pts, np);
    pb_xpiece pc;
    pc.v.q = q;
    pc.v.X1 = 0.0;
    pc.v.tol = 0.2 * tol;  /* inner integrals below the outer tolerance */
    double V = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        if (!(pts[i + 1] > pts[i])) continue;
        pc.p = pts[i];
        pc.q = pts[i + 1];
        pb_adapt_n(pb_slab_tau, &pc, 1, 0.0, 1.0, tol, &V, 4);
    }
    return V;
}

void og_paraboloid_cell(const double* frame, const double* coeffs, double* alpha, double* area, double* kbar,
                        double* nbar, int* status) {
    pb_cell q;
    memcpy(q.t1, frame, 3 * sizeof(double));
    memcpy(q.t2, frame + 3, 3 * sizeof(double));
    memcpy(q.n, frame + 6, 3 * sizeof(double));
    memcpy(q.a, coeffs, 6 * sizeof(double));
    const double V = pb_volume(&q, 1e-12);
    double I[PB_ND];
    pb_surface(&q, 1e-12, I);
    *alpha = V;
    *area = I[0];
    int st = 0;
    if (I[0] > 0.0) {
        *kbar = I[1] / I[0];
        const double nl = sqrt(I[2] * I[2] + I[3] * I[3] + I[4] * I[4]);
        for (int d = 0; d < 3; d++) nbar[d] = I[2 + d] / nl;
    } else {
        /* the surface misses the cell: the point values at the frame origin */
        const double* a = q.a;
        const double g2 = 1.0 + a[1] * a[1] + a[2] * a[2];
        *kbar = -(2.0 * a[3] * (1.0 + a[2] * a[2]) - 2.0 * a[1] * a[2] * a[4] + 2.0 * a[5] * (1.0 + a[1] * a[1])) /
                (g2 * sqrt(g2));
        double nv[3];
        for (int d = 0; d < 3; d++) nv[d] = q.n[d] - a[1] * q.t1[d] - a[2] * q.t2[d];
        const double nl = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        for (int d = 0; d < 3; d++) nbar[d] = nv[d] / nl;
        st = 1;
    }
    *status = st;
}

void og_paraboloid_cells(int64_t m, const double* frame, const double* coeffs, double* alpha, double* area,
                         double* kbar, double* nbar, int8_t* status) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < m; c++) {
        int st = 0;
        og_paraboloid_cell(frame + 9 * c, coeffs + 6 * c, alpha + c, area + c, kbar + c, nbar + 3 * c, &st);
        status[c] = (int8_t)st;
    }
}
