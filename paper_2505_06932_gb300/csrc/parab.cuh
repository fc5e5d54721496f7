// parab.cuh -- the cut-cell quantities of a fitted paraboloid (Sec. 3.2):
// with z = P(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 x y + a5 y^2 in the cell
// frame [t1 t2 n] (origin at the cell centre, lengths in cell widths, so the
// cell is [-1/2, 1/2]^3):
//   V  = |{X in cell : n.X <= P(t1.X, t2.X)}|      (alpha = V_P / V_C = V)
//   A  = int_{S in cell} dA,   K = int_{S in cell} kappa dA   (kappa = div n)
//   N  = int_{S in cell} n dA                      (S the surface z = P)
//
// The paper takes these from closed forms obtained by repeated use of the
// divergence theorem (Evrard et al. 2023, not reproduced); here:
//  * V: with Fv = (0, 0, z - P) (div Fv = 1, Fv = 0 on S) the divergence
//    theorem over the part of the cell below S leaves only the cell faces:
//    V = -sum_faces (nu_f . n) int_face max(F, 0) dA, F = P - z a quadratic in
//    the face's two coordinates.
//  * A, K, N: integrals over the parameter domain D = {(x, y) : the surface
//    point lies in the cell} with dA = W dx dy, W = sqrt(1 + Px^2 + Py^2) and
//    n dA = (-Px t1 - Py t2 + n) dx dy.  (N integrated over the surface keeps
//    its relative accuracy on small patches, which the equivalent face form,
//    differences of face areas of order one, would not.)
// Every 2D integral is iterated: the inner direction exactly (the set where a
// quadratic is positive, from its roots, and a polynomial antiderivative) for
// V, by Gauss-Legendre on exact intervals for A, K, N.  The outer direction is
// cut where the inner set changes (roots crossing the square's edges, the
// surface crossing cube edges) and at the branch points of the inner roots
// (zeros of their discriminants; the real parts of complex pairs); each piece
// is integrated by Gauss-Legendre under a map that is flat at ends holding a
// branch point (turning a square-root end into an analytic function) and cut
// geometrically towards nearby branch points (see graded()).
//
// Host and device code: one definition for the kernels; the host build only
// serves offline checks of the quadrature.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define PB_HD __host__ __device__ __forceinline__
#else
#define PB_HD inline
#endif
#ifdef __CUDA_ARCH__
#define PB_RSQRT(x) rsqrt(x)
#else
#define PB_RSQRT(x) (1.0 / sqrt(x))
#endif

namespace parab {

constexpr int kNS = 16;  // nodes per outer piece
constexpr int kNX = 12;  // nodes per inner interval of the surface integrals
constexpr int kN8 = 8;   // nodes of either when every singular point is >= 2 lengths away
constexpr double kR = 0.86602540378443865;  // |x|, |y| <= sqrt(3)/2 on the cell

// Gauss-Legendre rules on [0, 1] under four maps s(u) of the unit interval:
// m = 0 linear, 1 s = u^2 (flat at 0), 2 s = 1 - (1 - u)^2 (flat at 1),
// 3 s = 3u^2 - 2u^3 (flat at both ends); node s(u_k), weight w_k s'(u_k).
struct Rule {
    double os[4][kNS], ow[4][kNS];
    double ix[kNX], iw[kNX];
    double x8[kN8], w8[kN8];  // linear map
};

// squared distance from the singular points to the segment [a, b]
PB_HD double seg_dist2(double a, double b, const double* sre, const double* sim, int ns) {
    double best = 1e300;
    for (int i = 0; i < ns; i++) {
        const double dx = (sre[i] < a) ? a - sre[i] : ((sre[i] > b) ? sre[i] - b : 0.0);
        best = fmin(best, dx * dx + sim[i] * sim[i]);
    }
    return best;
}

struct Out {
    double V, A, K, N[3];
};

// A cell's quadrature can be shared by G threads (G divides kNS): every
// thread walks the same breakpoints and pieces, and of each piece's kNS outer
// nodes thread g takes nodes g, g + G, ..., so that the G threads evaluate
// different nodes at the same time; the G partial results add up to the
// cell's (G = 1: one thread does everything).
struct Split {
    int g, G;
};

// The x-interval structure of each strip of D (see row_plan) packed in 64
// bits: the interval count in bits 0-2, then per interval the tags of its two
// ends plus 2 (4 bits each).  The threads sharing a cell can share these: each
// plans the strips i = pg, pg + pG, ... into a common store, sync() makes them
// visible, and every thread reads all of them (one thread alone: pg = 0,
// pG = 1, sync() does nothing).
constexpr int kMaxStrips = 45;
struct PlanShare {
    unsigned long long* plans;  // kMaxStrips entries
    int pg, pG;
};

// real roots of c2 t^2 + c1 t + c0 strictly inside (lo, hi), appended at r[n..]
PB_HD int roots_in(double c2, double c1, double c0, double lo, double hi, double* r, int n) {
    if (c2 == 0.0) {
        if (c1 != 0.0) {
            const double t = -c0 / c1;
            if (t > lo && t < hi) r[n++] = t;
        }
        return n;
    }
    const double disc = c1 * c1 - 4.0 * c2 * c0;
    if (disc < 0.0) return n;
    const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
    const double t1 = q / c2;
    if (t1 > lo && t1 < hi) r[n++] = t1;
    if (q != 0.0) {
        const double t2 = c0 / q;
        if (t2 > lo && t2 < hi) r[n++] = t2;
    }
    return n;
}

// roots of c2 t^2 + c1 t + c0 as (re, im >= 0) pairs appended at re/im[n..]
PB_HD int croots(double c2, double c1, double c0, double* re, double* im, int n) {
    if (c2 == 0.0) {
        if (c1 != 0.0) {
            re[n] = -c0 / c1;
            im[n++] = 0.0;
        }
        return n;
    }
    const double disc = c1 * c1 - 4.0 * c2 * c0;
    if (disc >= 0.0) {
        const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
        re[n] = q / c2;
        im[n++] = 0.0;
        if (q != 0.0) {
            re[n] = c0 / q;
            im[n++] = 0.0;
        }
    } else {
        re[n] = -c1 / (2.0 * c2);
        im[n++] = sqrt(-disc) / (2.0 * fabs(c2));
    }
    return n;
}

PB_HD void sort_small(double* v, int n) {
    for (int i = 1; i < n; i++) {
        const double x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) {
            v[j + 1] = v[j];
            j--;
        }
        v[j + 1] = x;
    }
}

// Cutting [y0, y1] for a function analytic inside except for branch points at
// (sre, sim): a branch point at an end is taken by a map flat at that end;
// towards an end with other branch points at a distance d below half the
// length, the piece is cut at d, 3d, 7d, ... from that end (d (2^k - 1)), so
// that every sub-piece is at least as far from them as it is long
// (Gauss-Legendre then converges like 5.8^-2n or faster).  The sub-pieces are
// generated one by one from their index (no list), and the integrand is
// expanded at one call site.  `inner`: the x integrals, no branch points at
// the ends, the kNX-node rule.
struct Cut {
    double y0, y1, d0, d1;
    bool s0, s1, inner;
    int nl, nr;  // pieces cut from the lower / upper end
};

PB_HD Cut make_cut(double y0, double y1, const double* sre, const double* sim, int ns, bool inner) {
    Cut c;
    c.y0 = y0;
    c.y1 = y1;
    c.inner = inner;
    const double L = y1 - y0, eps2 = inner ? -1.0 : 1e-24 * L * L;
    double d0 = 4.0 * L * L, d1 = 4.0 * L * L;  // squared distances
    c.s0 = c.s1 = false;
    for (int i = 0; i < ns; i++) {
        const double u0 = sre[i] - y0, u1 = sre[i] - y1, v2 = sim[i] * sim[i];
        const double e0 = u0 * u0 + v2, e1 = u1 * u1 + v2;
        if (e0 <= eps2)
            c.s0 = true;
        else if (e0 < d0)
            d0 = e0;
        if (e1 <= eps2)
            c.s1 = true;
        else if (e1 < d1)
            d1 = e1;
    }
    c.d0 = sqrt(d0);
    c.d1 = sqrt(d1);
    c.nl = c.nr = 0;
    double a = y0;
    if (c.d0 < 0.5 * L)
        for (double st = c.d0; a + st < y0 + 0.5 * L; st *= 2.0) {
            a += st;
            c.nl++;
        }
    double b = y1;
    if (c.d1 < 0.5 * L)
        for (double st = c.d1; b - st > a && b - st > y1 - 0.5 * L; st *= 2.0) {
            b -= st;
            c.nr++;
        }
    return c;
}

// sub-piece i of nl + nr + 1 (lower-end pieces, the middle, upper-end pieces)
// and its rule: 0..3 map with kNS nodes (see Rule), 4 linear with kN8 nodes
// (every singular point at least two lengths away, where 8 nodes converge to
// rounding), 5 the inner kNX-node rule
PB_HD void cut_seg(const Cut& c, int i, const double* sre, const double* sim, int ns, double& a, double& b, int& m) {
    bool fa = false, fb = false;
    if (i < c.nl) {
        a = c.y0 + c.d0 * (ldexp(1.0, i) - 1.0);
        b = c.y0 + c.d0 * (ldexp(1.0, i + 1) - 1.0);
        fa = c.s0 && i == 0;
    } else if (i == c.nl) {
        a = c.y0 + c.d0 * (ldexp(1.0, c.nl) - 1.0);
        b = c.y1 - c.d1 * (ldexp(1.0, c.nr) - 1.0);
        fa = c.s0 && c.nl == 0;
        fb = c.s1 && c.nr == 0;
    } else {
        const int j = c.nl + c.nr - i;  // 0: the piece next to y1
        a = c.y1 - c.d1 * (ldexp(1.0, j + 1) - 1.0);
        b = c.y1 - c.d1 * (ldexp(1.0, j) - 1.0);
        fb = c.s1 && j == 0;
    }
    m = c.inner ? 5 : (fa ? 1 : 0) + (fb ? 2 : 0);
    if ((m == 0 || m == 5) && seg_dist2(a, b, sre, sim, ns) >= 4.0 * (b - a) * (b - a)) m = 4;
}

template <class Fn>
PB_HD void run_cut(const Cut& c, const double* sre, const double* sim, int ns, const Rule& R, int g, int G, Fn& f) {
    const int nseg = c.nl + c.nr + 1;
    for (int i = 0; i < nseg; i++) {
        double a, b;
        int m;
        cut_seg(c, i, sre, sim, ns, a, b, m);
        const double h = b - a;
        const double* xs = (m == 4) ? R.x8 : ((m == 5) ? R.ix : R.os[m]);
        const double* ws = (m == 4) ? R.w8 : ((m == 5) ? R.iw : R.ow[m]);
        const int nn = (m == 4) ? kN8 : ((m == 5) ? kNX : kNS);
        for (int k = g; k < nn; k += G) f(a + h * xs[k], h * ws[k]);
    }
}

// outer integral over [y0, y1]: thread sp.g of sp.G takes the nodes g, g + G, ...
// of each sub-piece.  f(y, w) accumulates w * integrand(y).
template <class Fn>
PB_HD void graded(double y0, double y1, const double* sre, const double* sim, int ns, const Rule& R, const Split& sp,
                  Fn&& f) {
    const Cut c = make_cut(y0, y1, sre, sim, ns, false);
    run_cut(c, sre, sim, ns, R, sp.g, sp.G, f);
}

// the inner x integrals: a complex singular point over the interval's
// interior within 1.25 lengths first cuts it at its real part (beyond that
// 12 nodes already converge to rounding), so that its distance is measured
// from an end
template <class Fn>
PB_HD void graded_x(double x0, double x1, const double* sre, const double* sim, int ns, const Rule& R, Fn&& f) {
    double xs = x0;
    double best = 1.25 * (x1 - x0);
    for (int i = 0; i < ns; i++)
        if (sre[i] > x0 && sre[i] < x1 && sim[i] < best) {
            best = sim[i];
            xs = sre[i];
        }
    const int nh = (xs > x0) ? 2 : 1;
    for (int hh = 0; hh < nh; hh++) {
        const double lo = (hh == 0) ? x0 : xs, hi = (nh == 1 || hh == 1) ? x1 : xs;
        const Cut c = make_cut(lo, hi, sre, sim, ns, true);
        run_cut(c, sre, sim, ns, R, 0, 1, f);
    }
}

// int_{-1/2}^{1/2} max(f, 0) du for f(u) = al u^2 + be u + ga
PB_HD double row_positive(double al, double be, double ga) {
    double p[4];
    p[0] = -0.5;
    int np = roots_in(al, be, ga, -0.5, 0.5, p, 1);
    if (np == 3 && p[1] > p[2]) {
        const double t = p[1];
        p[1] = p[2];
        p[2] = t;
    }
    p[np++] = 0.5;
    double I = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        const double u0 = p[i], u1 = p[i + 1], m = 0.5 * (u0 + u1);
        if ((al * m + be) * m + ga > 0.0) {
            // antiderivative u (ga + u (be/2 + u al/3))
            const double F1 = u1 * (ga + u1 * (0.5 * be + u1 * (al * (1.0 / 3.0))));
            const double F0 = u0 * (ga + u0 * (0.5 * be + u0 * (al * (1.0 / 3.0))));
            I += F1 - F0;
        }
    }
    return I;
}

// int over the face [-1/2, 1/2]^2 of max(F, 0), with F(u, v) = Auu u^2 +
// Auv u v + Avv v^2 + Bu u + Bv v + C.  The row integral is analytic in v
// except where a root crosses u = +-1/2 (kinks: cut there) and at the branch
// points of the roots, the zeros of the discriminant in u (cut at real ones
// and at the real part of a complex pair; the pieces are graded towards them).
PB_HD double face_positive(double Auu, double Auv, double Avv, double Bu, double Bv, double C, const Rule& R,
                           const Split& sp) {
    double sre[2], sim[2];
    const int ns = croots(Auv * Auv - 4.0 * Auu * Avv, 2.0 * Auv * Bu - 4.0 * Auu * Bv, Bu * Bu - 4.0 * Auu * C, sre,
                          sim, 0);
    double p[8];
    p[0] = -0.5;
    int np = 1;
    np = roots_in(Avv, Bv + 0.5 * Auv, C + 0.5 * Bu + 0.25 * Auu, -0.5, 0.5, p, np);
    np = roots_in(Avv, Bv - 0.5 * Auv, C - 0.5 * Bu + 0.25 * Auu, -0.5, 0.5, p, np);
    bool real_branch = false;
    for (int i = 0; i < ns; i++) real_branch |= (sim[i] == 0.0 && sre[i] > -0.5 && sre[i] < 0.5);
    if (np == 1 && !real_branch) {
        // no root crosses an edge and the number of real roots per row never
        // changes: every row has as many roots inside as the middle row; none
        // there means that F keeps one sign on the whole face
        double r[2];
        if (roots_in(Auu, Bu, C, -0.5, 0.5, r, 0) == 0)
            return (sp.g == 0 && C > 0.0) ? C + (Auu + Avv) * (1.0 / 12.0) : 0.0;
    }
    for (int i = 0; i < ns; i++)
        if (sre[i] > -0.5 && sre[i] < 0.5) p[np++] = sre[i];
    p[np++] = 0.5;
    sort_small(p, np);
    double I = 0.0;
    for (int i = 0; i + 1 < np; i++) {
        if (!(p[i + 1] > p[i])) continue;
        graded(p[i], p[i + 1], sre, sim, ns, R, sp,
               [&](double v, double w) { I += w * row_positive(Auu, Auv * v + Bu, (Avv * v + Bv) * v + C); });
    }
    return I;
}

// The surface in world (cell) coordinates: X_d(x, y) = e2 x^2 + (e1c + e1y y) x
// + (e0c + e0y y + e0yy y^2), one row per axis d.
struct Surf {
    double e2[3], e1c[3], e1y[3], e0c[3], e0y[3], e0yy[3];
};

PB_HD bool on_cell(const Surf& S, double x, double y) {
    for (int d = 0; d < 3; d++) {
        const double X = S.e2[d] * x * x + (S.e1c[d] + S.e1y[d] * y) * x + (S.e0c[d] + (S.e0y[d] + S.e0yy[d] * y) * y);
        if (!(fabs(X) <= 0.5)) return false;
    }
    return true;
}

// The roots of c2 x^2 + c1 x + c0 as an ordered pair (lo <= hi): 2 for a
// quadratic with a real pair (a negative discriminant that rounding produced
// next to a double root counts as zero), 1 for a linear equation (lo = hi), 0
// otherwise.  Tagging and evaluating the ends of D's rows both go through it,
// so a tag always names the same root whatever the rounding.
PB_HD int root_pair(double c2, double c1, double c0, bool clamp, double& lo, double& hi) {
    if (c2 == 0.0) {
        if (c1 == 0.0) return 0;
        lo = hi = -c0 / c1;
        return 1;
    }
    double disc = c1 * c1 - 4.0 * c2 * c0;
    if (disc < 0.0) {
        if (!clamp) return 0;
        disc = 0.0;
    }
    const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
    const double r1 = q / c2, r2 = (q != 0.0) ? c0 / q : r1;
    lo = fmin(r1, r2);
    hi = fmax(r1, r2);
    return 2;
}

// Inside a strip of y between breakpoints the x-intervals of D keep their
// structure: each end is the same root of the same curve.  A tag names it:
// 4 d + 2 l + b for the smaller (b = 0) or larger (b = 1) root of X_d = -1/2
// (l = 0) or +1/2 (l = 1) (the only root if the curve is linear in x), and
// -1 / -2 for the range ends -kR / kR.
PB_HD void curve_coeffs(const Surf& S, int d, int l, double y, double& c2, double& c1, double& c0) {
    c2 = S.e2[d];
    c1 = S.e1c[d] + S.e1y[d] * y;
    c0 = S.e0c[d] + (S.e0y[d] + S.e0yy[d] * y) * y - (l ? 0.5 : -0.5);
}

PB_HD double tagged_root(const Surf& S, int tag, double y) {
    if (tag == -1) return -kR;
    if (tag == -2) return kR;
    const int d = tag >> 2, l = (tag >> 1) & 1, b = tag & 1;
    double c2, c1, c0, lo = 0.0, hi = 0.0;
    curve_coeffs(S, d, l, y, c2, c1, c0);
    root_pair(c2, c1, c0, true, lo, hi);
    return b ? hi : lo;
}

// the x-intervals of D at y (at most 7) as the tags of their ends
PB_HD int row_plan(const Surf& S, double y, int* tlo, int* thi) {
    double p[14];
    int tg[14];
    p[0] = -kR;
    tg[0] = -1;
    int np = 1;
    for (int d = 0; d < 3; d++)
        for (int l = 0; l < 2; l++) {
            double c2, c1, c0, lo, hi;
            curve_coeffs(S, d, l, y, c2, c1, c0);
            const int nr = root_pair(c2, c1, c0, false, lo, hi);
            if (nr >= 1 && lo > -kR && lo < kR) {
                p[np] = lo;
                tg[np++] = 4 * d + 2 * l;
            }
            if (nr == 2 && hi > -kR && hi < kR) {
                p[np] = hi;
                tg[np++] = 4 * d + 2 * l + 1;
            }
        }
    p[np] = kR;
    tg[np++] = -2;
    for (int i = 1; i < np; i++) {  // insertion sort carrying the tags
        const double x = p[i];
        const int t = tg[i];
        int j = i - 1;
        while (j >= 0 && p[j] > x) {
            p[j + 1] = p[j];
            tg[j + 1] = tg[j];
            j--;
        }
        p[j + 1] = x;
        tg[j + 1] = t;
    }
    int ni = 0;
    for (int i = 0; i + 1 < np; i++) {
        if (!(p[i + 1] > p[i])) continue;
        if (!on_cell(S, 0.5 * (p[i] + p[i + 1]), y)) continue;
        if (ni > 0 && thi[ni - 1] == tg[i]) {
            thi[ni - 1] = tg[i + 1];  // a split by a root that does not bound D
        } else {
            tlo[ni] = tg[i];
            thi[ni] = tg[i + 1];
            ni++;
        }
    }
    return ni;
}

// this thread's share (sp) of the cell's V, A, K and N
template <class Sync>
PB_HD void parab_cell(const double t1[3], const double t2[3], const double n[3], const double a[6], const Rule& R,
                      const Split& sp, const PlanShare& ps, Sync&& sync, Out& o) {
    // F(X) = P(t1.X, t2.X) - n.X = a0 + g.X + X^T H X
    double g[3], H[3][3];
    for (int i = 0; i < 3; i++) {
        g[i] = a[1] * t1[i] + a[2] * t2[i] - n[i];
        for (int j = 0; j < 3; j++)
            H[i][j] = a[3] * t1[i] * t1[j] + 0.5 * a[4] * (t1[i] * t2[j] + t2[i] * t1[j]) + a[5] * t2[i] * t2[j];
    }
    o.V = 0.0;
    for (int d = 0; d < 3; d++) {
        const int p = (d + 1) % 3, q = (d + 2) % 3;
        for (int s = -1; s <= 1; s += 2) {
            const double I = face_positive(H[p][p], 2.0 * H[p][q], H[q][q], g[p] + s * H[p][d], g[q] + s * H[q][d],
                                           a[0] + 0.5 * s * g[d] + 0.25 * H[d][d], R, sp);
            o.V -= s * n[d] * I;
        }
    }

    // surface integrals over D
    Surf S;
    for (int d = 0; d < 3; d++) {
        S.e2[d] = n[d] * a[3];
        S.e1c[d] = t1[d] + n[d] * a[1];
        S.e1y[d] = n[d] * a[4];
        S.e0c[d] = n[d] * a[0];
        S.e0y[d] = t2[d] + n[d] * a[2];
        S.e0yy[d] = n[d] * a[5];
    }
    double yb[46], sre[12], sim[12];
    yb[0] = -kR;
    int nb = 1, ns = 0;
    // branch points of the x-roots: zeros of each curve's discriminant in x
    // (X_d = +-1/2 has a double root); real ones and the real parts of complex
    // pairs cut the y range
    for (int d = 0; d < 3; d++)
        for (int s = -1; s <= 1; s += 2) {
            const int n0 = ns;
            ns = croots(S.e1y[d] * S.e1y[d] - 4.0 * S.e2[d] * S.e0yy[d],
                        2.0 * S.e1c[d] * S.e1y[d] - 4.0 * S.e2[d] * S.e0y[d],
                        S.e1c[d] * S.e1c[d] - 4.0 * S.e2[d] * (S.e0c[d] - 0.5 * s), sre, sim, ns);
            for (int i = n0; i < ns; i++)
                if (sre[i] > -kR && sre[i] < kR) yb[nb++] = sre[i];
        }
    // a coordinate that does not depend on x (the surface is a cylinder along
    // x in that direction, e.g. a plane lying in a cube face) bounds D at the
    // y where it equals +-1/2
    for (int d = 0; d < 3; d++)
        if (S.e2[d] == 0.0 && S.e1c[d] == 0.0 && S.e1y[d] == 0.0)
            for (int s = -1; s <= 1; s += 2) nb = roots_in(S.e0yy[d], S.e0y[d], S.e0c[d] - 0.5 * s, -kR, kR, yb, nb);
    // y where the surface crosses one of the twelve cube edges
    for (int f = 0; f < 3; f++) {
        const int d = (f + 1) % 3, e = (f + 2) % 3;
        for (int s1 = -1; s1 <= 1; s1 += 2)
            for (int s2 = -1; s2 <= 1; s2 += 2) {
                const double Xd = 0.5 * s1, Xe = 0.5 * s2;
                double r[2];
                const int nr = roots_in(H[f][f], g[f] + 2.0 * (H[f][d] * Xd + H[f][e] * Xe),
                                        a[0] + g[d] * Xd + g[e] * Xe + H[d][d] * Xd * Xd + 2.0 * H[d][e] * Xd * Xe +
                                            H[e][e] * Xe * Xe,
                                        -0.5, 0.5, r, 0);
                for (int i = 0; i < nr; i++) {
                    double X[3];
                    X[f] = r[i];
                    X[d] = Xd;
                    X[e] = Xe;
                    yb[nb++] = t2[0] * X[0] + t2[1] * X[1] + t2[2] * X[2];
                }
            }
    }
    yb[nb++] = kR;
    sort_small(yb, nb);
    // plan the strips (this thread's share), then integrate every strip
    for (int i = ps.pg; i + 1 < nb; i += ps.pG) {
        unsigned long long code = 0;
        if (yb[i + 1] > yb[i]) {
            int tlo[7], thi[7];
            const int ni = row_plan(S, 0.5 * (yb[i] + yb[i + 1]), tlo, thi);
            code = (unsigned long long)ni;
            for (int j = 0; j < ni; j++)
                code |= (unsigned long long)((tlo[j] + 2) | ((thi[j] + 2) << 4)) << (3 + 8 * j);
        }
        ps.plans[i] = code;
    }
    sync();
    double A = 0.0, K = 0.0, Nx = 0.0, Ny = 0.0, Nz = 0.0;
    const double pxx = 2.0 * a[3], pxy = a[4], pyy = 2.0 * a[5];
    for (int i = 0; i + 1 < nb; i++) {
        const double y0 = yb[i], y1 = yb[i + 1];
        const unsigned long long code = ps.plans[i];
        const int ni = (int)(code & 7u);
        if (ni == 0) continue;  // D does not meet this strip (or it is empty)
        int tlo[7], thi[7];
        for (int j = 0; j < ni; j++) {
            const int b = (int)((code >> (3 + 8 * j)) & 0xffu);
            tlo[j] = (b & 15) - 2;
            thi[j] = (b >> 4) - 2;
        }
        graded(y0, y1, sre, sim, ns, R, sp, [&](double y, double wy) {
            // W^2 = 1 + px^2 + py^2 is a quadratic in x; its complex zeros are
            // the branch points (W) and poles (kappa W) of the row integrand
            const double b1 = a[1] + pxy * y, b2 = a[2] + pyy * y;
            double xre[2], xim[2];
            const int nx = croots(pxx * pxx + pxy * pxy, 2.0 * (pxx * b1 + pxy * b2), 1.0 + b1 * b1 + b2 * b2, xre,
                                  xim, 0);
            for (int j = 0; j < ni; j++) {
                const double lo = tagged_root(S, tlo[j], y), hi = tagged_root(S, thi[j], y);
                if (!(hi > lo)) continue;
                graded_x(lo, hi, xre, xim, nx, R, [&](double x, double wx) {
                    const double px = b1 + pxx * x, py = b2 + pxy * x;
                    const double W2 = 1.0 + px * px + py * py, rW = PB_RSQRT(W2);
                    const double w = wy * wx;
                    A += w * (W2 * rW);
                    // kappa W = -((1 + py^2) pxx - 2 px py pxy + (1 + px^2) pyy) / W^2
                    K -= w * ((1.0 + py * py) * pxx - 2.0 * px * py * pxy + (1.0 + px * px) * pyy) * (rW * rW);
                    Nx -= w * px;
                    Ny -= w * py;
                    Nz += w;
                });
            }
        });
    }
    o.A = A;
    o.K = K;
    for (int d = 0; d < 3; d++) o.N[d] = Nx * t1[d] + Ny * t2[d] + Nz * n[d];
}

// Gauss-Legendre rule of order n on [0, 1] by Newton's iteration on P_n
inline void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; i++) {
        double t = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; k++) {
            const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = 0.5 * (1.0 - t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
    }
}

inline Rule make_rule() {
    Rule R;
    double u[kNS], w[kNS];
    gauss_legendre01(kNS, u, w);
    for (int k = 0; k < kNS; k++) {
        const double v = 1.0 - u[k];
        R.os[0][k] = u[k];
        R.ow[0][k] = w[k];
        R.os[1][k] = u[k] * u[k];
        R.ow[1][k] = w[k] * 2.0 * u[k];
        R.os[2][k] = 1.0 - v * v;
        R.ow[2][k] = w[k] * 2.0 * v;
        R.os[3][k] = u[k] * u[k] * (3.0 - 2.0 * u[k]);
        R.ow[3][k] = w[k] * 6.0 * u[k] * v;
    }
    gauss_legendre01(kNX, R.ix, R.iw);
    gauss_legendre01(kN8, R.x8, R.w8);
    return R;
}

}  // namespace parab
