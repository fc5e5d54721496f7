/*
 * oracle.c -- plain, slow FP64 CPU oracle for the front/fluid coupling of the
 * sharp front-tracking method (Gorges et al., arXiv 2505.06932).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline / reference arm are its only users.  It shares no code with the
 * CUDA path.  Build with -std=c11 -ffp-contract=off (no fused multiply-add), so
 * that the binning predicate rounds exactly as its definition says.
 *
 * Functions follow the paper's statement step by step:
 *   og_bin      -- interfacial cells (Sec. 3.2), canonical clip predicate
 *   og_alpha    -- alpha_C = (1/V_C) int_C I dx (Sec. 3.2), column integration
 *   og_ppic     -- PPIC volume fit, Eqs. volumefit / Wendland / volumefit2
 *                  (Sec. 3.2), curvature of the paraboloid at the local origin
 *   og_csf      -- S = sigma kappa grad alpha (Eq. csf) + curvature smoothing
 *                  (Sec. 3.3)
 *   og_face_force -- balanced-force face term sigma kbar_f (alpha_Q - alpha_P)/h
 *                  (Sec. 3.3, Eq. mwi_disc)
 *   og_interp   -- divergence-preserving velocity interpolation (Sec. 3.1)
 *   og_advect_rk4 -- one fourth-order Runge-Kutta step of the front vertices
 *                  in the interpolated velocity (Sec. 3.1)
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_MAXV 32 /* Sutherland-Hodgman on a triangle and 6 planes never exceeds 28 */

typedef struct {
    int n;
    double p[OG_MAXV][3];
} og_poly;

/* ------------------------------------------------------------------------ */
/* grid and canonical clip                                                   */
/* ------------------------------------------------------------------------ */

/* plane coordinate origin + idx*h, rounded once per operation (no FMA) */
static double og_plane(const og_grid* g, int ax, int64_t idx) {
    return g->origin[ax] + (double)idx * g->h;
}

/* One Sutherland-Hodgman step against coord[ax] >= pv (ge = 1) or <= pv (ge = 0).
 * A crossing on edge prev->cur is prev + t (cur - prev), t = (pv - prev)/(cur - prev),
 * with the clipped coordinate set exactly to pv. */
static void og_clip_half(const og_poly* in, og_poly* out, int ax, double pv, int ge) {
    const int n = in->n;
    out->n = 0;
    for (int i = 0; i < n; i++) {
        const double* cur = in->p[i];
        const double* prev = in->p[(i + n - 1) % n];
        const int cin = ge ? (cur[ax] >= pv) : (cur[ax] <= pv);
        const int pin = ge ? (prev[ax] >= pv) : (prev[ax] <= pv);
        if (cin != pin) {
            const double t = (pv - prev[ax]) / (cur[ax] - prev[ax]);
            double* q = out->p[out->n++];
            for (int c = 0; c < 3; c++) q[c] = (c == ax) ? pv : prev[c] + t * (cur[c] - prev[c]);
        }
        if (cin) memcpy(out->p[out->n++], cur, sizeof(double) * 3);
    }
}

/* Canonical clip of triangle (a,b,c) against cell (i,j,k): planes in the order
 * x >= X_i, x <= X_i+1, y >= Y_j, y <= Y_j+1, z >= Z_k, z <= Z_k+1.  The cell
 * accepts the triangle iff every stage keeps >= 3 vertices, the fan area
 * vector sum_m (p_m - p_0) x (p_m+1 - p_0) is not the zero vector, and the
 * polygon does not lie entirely in one of the cell's upper faces (a fragment
 * lying in a face shared by two cells belongs to the upper cell only). */
static int og_canon(const double* a, const double* b, const double* c, const og_grid* g,
                    int64_t i, int64_t j, int64_t k, og_poly* res) {
    og_poly A, B;
    og_poly* src = &A;
    og_poly* dst = &B;
    A.n = 3;
    memcpy(A.p[0], a, sizeof(double) * 3);
    memcpy(A.p[1], b, sizeof(double) * 3);
    memcpy(A.p[2], c, sizeof(double) * 3);
    const int64_t idx[3] = {i, j, k};
    for (int ax = 0; ax < 3; ax++) {
        og_clip_half(src, dst, ax, og_plane(g, ax, idx[ax]), 1);
        if (dst->n < 3) return 0;
        og_poly* t = src; src = dst; dst = t;
        og_clip_half(src, dst, ax, og_plane(g, ax, idx[ax] + 1), 0);
        if (dst->n < 3) return 0;
        t = src; src = dst; dst = t;
    }
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const double* p0 = src->p[0];
    for (int m = 1; m + 1 < src->n; m++) {
        const double e1x = src->p[m][0] - p0[0], e1y = src->p[m][1] - p0[1], e1z = src->p[m][2] - p0[2];
        const double e2x = src->p[m + 1][0] - p0[0], e2y = src->p[m + 1][1] - p0[1],
                     e2z = src->p[m + 1][2] - p0[2];
        s0 = s0 + (e1y * e2z - e1z * e2y);
        s1 = s1 + (e1z * e2x - e1x * e2z);
        s2 = s2 + (e1x * e2y - e1y * e2x);
    }
    if (s0 == 0.0 && s1 == 0.0 && s2 == 0.0) return 0;
    for (int ax = 0; ax < 3; ax++) {
        const double up = og_plane(g, ax, idx[ax] + 1);
        int all = 1;
        for (int m = 0; m < src->n; m++)
            if (src->p[m][ax] != up) { all = 0; break; }
        if (all) return 0;
    }
    if (res) *res = *src;
    return src->n;
}

/* Candidate cells along one axis: the cells whose closed extent [X_i, X_i+1]
 * meets [lo, hi]: i0 = min{i : X_i+1 >= lo}, i1 = max{i : X_i <= hi}. */
static void og_range(const og_grid* g, int ax, double lo, double hi, int64_t* i0, int64_t* i1) {
    const int64_t n = g->n[ax];
    double f = floor((lo - g->origin[ax]) / g->h);
    int64_t e = (f >= 0.0) ? ((f <= (double)(n - 1)) ? (int64_t)f : n - 1) : 0;
    while (e > 0 && og_plane(g, ax, e) >= lo) e--;
    while (e < n - 1 && og_plane(g, ax, e + 1) < lo) e++;
    *i0 = e;
    f = floor((hi - g->origin[ax]) / g->h);
    e = (f >= 0.0) ? ((f <= (double)(n - 1)) ? (int64_t)f : n - 1) : 0;
    while (e < n - 1 && og_plane(g, ax, e + 1) <= hi) e++;
    while (e > 0 && og_plane(g, ax, e) > hi) e--;
    *i1 = e;
}

/* Triangle t's vertices and candidate box; returns 0 if valid, else a status bit. */
static uint32_t og_tri_setup(const double* verts, int64_t nv, const int32_t* tris, int64_t t,
                             const og_grid* g, int32_t margin, const double** pv, int64_t lo[3],
                             int64_t hi[3]) {
    for (int c = 0; c < 3; c++) {
        const int32_t vi = tris[3 * t + c];
        if (vi < 0 || vi >= nv) return OG_BAD_INDEX;
        pv[c] = verts + 3 * (int64_t)vi;
        for (int ax = 0; ax < 3; ax++)
            if (!isfinite(pv[c][ax])) return OG_OUTSIDE_GRID;
    }
    for (int ax = 0; ax < 3; ax++) {
        double mn = pv[0][ax], mx = pv[0][ax];
        for (int c = 1; c < 3; c++) {
            if (pv[c][ax] < mn) mn = pv[c][ax];
            if (pv[c][ax] > mx) mx = pv[c][ax];
        }
        og_range(g, ax, mn, mx, &lo[ax], &hi[ax]);
        if (lo[ax] < margin || hi[ax] > (int64_t)g->n[ax] - 1 - margin) return OG_OUTSIDE_GRID;
    }
    return 0;
}

static int og_cmp_u64(const void* a, const void* b) {
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

typedef struct {
    uint64_t* v;
    int64_t n, cap;
} og_vec;

static void og_push(og_vec* v, uint64_t x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->v = (uint64_t*)realloc(v->v, sizeof(uint64_t) * (size_t)v->cap);
    }
    v->v[v->n++] = x;
}

static uint64_t og_key(const og_grid* g, int64_t i, int64_t j, int64_t k) {
    return (uint64_t)((i * g->n[1] + j) * g->n[2] + k);
}

/* sorted (key << 32 | tri) pairs of every accepted (cell, triangle) */
static og_vec og_pairs(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                       const og_grid* g, int32_t margin, uint32_t* status) {
    og_vec out = {0, 0, 0};
    uint32_t st = 0;
    for (int64_t t = 0; t < nt; t++) {
        const double* pv[3];
        int64_t lo[3], hi[3];
        const uint32_t e = og_tri_setup(verts, nv, tris, t, g, margin, pv, lo, hi);
        if (e) { st |= e; continue; }
        for (int64_t i = lo[0]; i <= hi[0]; i++)
            for (int64_t j = lo[1]; j <= hi[1]; j++)
                for (int64_t k = lo[2]; k <= hi[2]; k++)
                    if (og_canon(pv[0], pv[1], pv[2], g, i, j, k, NULL))
                        og_push(&out, (og_key(g, i, j, k) << 32) | (uint64_t)t);
    }
    if (out.n) qsort(out.v, (size_t)out.n, sizeof(uint64_t), og_cmp_u64);
    if (status) *status |= st;
    return out;
}

int64_t og_bin(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const og_grid* g,
               int32_t margin, int64_t cap, uint32_t* keys, int32_t* tri_ids, uint32_t* status) {
    og_vec pr = og_pairs(verts, nv, tris, nt, g, margin, status);
    for (int64_t q = 0; q < pr.n && q < cap; q++) {
        keys[q] = (uint32_t)(pr.v[q] >> 32);
        tri_ids[q] = (int32_t)(pr.v[q] & 0xffffffffu);
    }
    const int64_t n = pr.n;
    free(pr.v);
    return n;
}

int64_t og_bin_bruteforce(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          const og_grid* g, int64_t cap, uint32_t* keys, int32_t* tri_ids) {
    og_vec out = {0, 0, 0};
    for (int64_t t = 0; t < nt; t++) {
        const double* pv[3];
        int bad = 0;
        for (int c = 0; c < 3; c++) {
            if (tris[3 * t + c] < 0 || tris[3 * t + c] >= nv) bad = 1;
            else pv[c] = verts + 3 * (int64_t)tris[3 * t + c];
        }
        if (bad) continue;
        for (int64_t i = 0; i < g->n[0]; i++)
            for (int64_t j = 0; j < g->n[1]; j++)
                for (int64_t k = 0; k < g->n[2]; k++)
                    if (og_canon(pv[0], pv[1], pv[2], g, i, j, k, NULL))
                        og_push(&out, (og_key(g, i, j, k) << 32) | (uint64_t)t);
    }
    if (out.n) qsort(out.v, (size_t)out.n, sizeof(uint64_t), og_cmp_u64);
    for (int64_t q = 0; q < out.n && q < cap; q++) {
        keys[q] = (uint32_t)(out.v[q] >> 32);
        tri_ids[q] = (int32_t)(out.v[q] & 0xffffffffu);
    }
    const int64_t n = out.n;
    free(out.v);
    return n;
}

int og_clip_fragment(const double* tri9, const og_grid* g, int32_t i, int32_t j, int32_t k,
                     double* poly_out) {
    og_poly r;
    const int n = og_canon(tri9, tri9 + 3, tri9 + 6, g, i, j, k, &r);
    for (int m = 0; m < n; m++) memcpy(poly_out + 3 * m, r.p[m], sizeof(double) * 3);
    return n;
}

/* ------------------------------------------------------------------------ */
/* polygon integrals                                                        */
/* ------------------------------------------------------------------------ */

/* z-component of the area vector (signed xy-projected area) and the integral
 * int_poly z n_z dA, summed over the fan triangles (p0, p_m, p_m+1). */
static void og_fan_z(const og_poly* q, double* az, double* zaz) {
    double a = 0.0, za = 0.0;
    for (int m = 1; m + 1 < q->n; m++) {
        const double* p0 = q->p[0];
        const double* p1 = q->p[m];
        const double* p2 = q->p[m + 1];
        const double cz = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]));
        a += cz;
        za += cz * (p0[2] + p1[2] + p2[2]) / 3.0;
    }
    *az = a;
    *zaz = za;
}

/* Newell's area vector 0.5 * sum_i (y_i - y_i+1)(z_i + z_i+1), ... */
static void og_newell(const double (*p)[3], int n, double* N) {
    N[0] = N[1] = N[2] = 0.0;
    for (int i = 0; i < n; i++) {
        const double* a = p[i];
        const double* b = p[(i + 1) % n];
        N[0] += (a[1] - b[1]) * (a[2] + b[2]);
        N[1] += (a[2] - b[2]) * (a[0] + b[0]);
        N[2] += (a[0] - b[0]) * (a[1] + b[1]);
    }
    N[0] *= 0.5; N[1] *= 0.5; N[2] *= 0.5;
}

/* area centroid of a planar polygon with unit normal nh (fan decomposition) */
static void og_centroid(const double (*p)[3], int n, const double* nh, double* c) {
    double w = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    for (int m = 1; m + 1 < n; m++) {
        const double* p0 = p[0];
        const double* p1 = p[m];
        const double* p2 = p[m + 1];
        const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double a = 0.5 * (cr[0] * nh[0] + cr[1] * nh[1] + cr[2] * nh[2]);
        w += a;
        cx += a * (p0[0] + p1[0] + p2[0]) / 3.0;
        cy += a * (p0[1] + p1[1] + p2[1]) / 3.0;
        cz += a * (p0[2] + p1[2] + p2[2]) / 3.0;
    }
    if (w != 0.0) { c[0] = cx / w; c[1] = cy / w; c[2] = cz / w; }
    else {
        c[0] = c[1] = c[2] = 0.0;
        for (int m = 0; m < n; m++) { c[0] += p[m][0] / n; c[1] += p[m][1] / n; c[2] += p[m][2] / n; }
    }
}

/* Signed area moments of a simple 2D polygon by Green's theorem:
 * m = [int 1, int x, int y, int x^2, int xy, int y^2] dx dy (counter-clockwise > 0). */
void og_green_moments(const double* x, const double* y, int n, double* m) {
    double a = 0, mx = 0, my = 0, mxx = 0, mxy = 0, myy = 0;
    for (int i = 0; i < n; i++) {
        const int j = (i + 1) % n;
        const double xi = x[i], yi = y[i], xj = x[j], yj = y[j];
        const double c = xi * yj - xj * yi;
        a += c;
        mx += (xi + xj) * c;
        my += (yi + yj) * c;
        mxx += (xi * xi + xi * xj + xj * xj) * c;
        myy += (yi * yi + yi * yj + yj * yj) * c;
        mxy += (xi * yj + 2.0 * xi * yi + 2.0 * xj * yj + xj * yi) * c;
    }
    m[0] = a / 2.0;
    m[1] = mx / 6.0;
    m[2] = my / 6.0;
    m[3] = mxx / 12.0;
    m[4] = mxy / 24.0;
    m[5] = myy / 12.0;
}

double og_signed_volume(const double* v, const int32_t* t, int64_t nt) {
    double s = 0.0;
    for (int64_t f = 0; f < nt; f++) {
        const double* a = v + 3 * (int64_t)t[3 * f];
        const double* b = v + 3 * (int64_t)t[3 * f + 1];
        const double* c = v + 3 * (int64_t)t[3 * f + 2];
        s += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
             a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    return s / 6.0;
}

/* ------------------------------------------------------------------------ */
/* volume fraction                                                           */
/* ------------------------------------------------------------------------ */

/* For a vertical line through the column of cell (i,j,k), the part of it inside
 * the enclosed region and inside [Z_k, Z_k+1] has length
 *   sum over crossings sign(n_z) (clamp(z, Z_k, Z_k+1) - Z_k)
 * (crossings alternate entry/exit on a closed surface).  Integrating over the
 * column cross-section turns the sum into surface integrals, so
 *   vol(Omega cap C) = sum_t [ int_{t cap slab} (z - Z_k) n_z dA
 *                              + h int_{t above slab} n_z dA ]
 * with t clipped to the column's four side planes. */
int og_alpha(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const og_grid* g,
             int32_t margin, double* alpha, uint32_t* status) {
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    const double h = g->h, h3 = h * h * h;
    uint32_t st = 0;
    /* interfacial cells, by the binning predicate */
    uint8_t* inter = (uint8_t*)calloc((size_t)(n0 * n1 * n2), 1);
    og_vec pr = og_pairs(verts, nv, tris, nt, g, margin, &st);
    for (int64_t q = 0; q < pr.n; q++) inter[pr.v[q] >> 32] = 1;
    free(pr.v);
    /* column -> triangle lists (closed xy-extent overlap) */
    int64_t* cnt = (int64_t*)calloc((size_t)(n0 * n1 + 1), sizeof(int64_t));
    int64_t* box = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)(nt ? nt : 1));
    for (int64_t t = 0; t < nt; t++) {
        const double* pv[3];
        int64_t lo[3], hi[3];
        const uint32_t e = og_tri_setup(verts, nv, tris, t, g, margin, pv, lo, hi);
        if (e) { box[4 * t] = -1; continue; }
        box[4 * t] = lo[0]; box[4 * t + 1] = hi[0]; box[4 * t + 2] = lo[1]; box[4 * t + 3] = hi[1];
        for (int64_t i = lo[0]; i <= hi[0]; i++)
            for (int64_t j = lo[1]; j <= hi[1]; j++) cnt[i * n1 + j + 1]++;
    }
    for (int64_t c = 0; c < n0 * n1; c++) cnt[c + 1] += cnt[c];
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[n0 * n1] ? cnt[n0 * n1] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n0 * n1));
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(n0 * n1));
    for (int64_t t = 0; t < nt; t++) {
        if (box[4 * t] < 0) continue;
        for (int64_t i = box[4 * t]; i <= box[4 * t + 1]; i++)
            for (int64_t j = box[4 * t + 2]; j <= box[4 * t + 3]; j++) list[fill[i * n1 + j]++] = t;
    }
    free(fill);
    free(box);

#pragma omp parallel for schedule(dynamic, 16) reduction(| : st)
    for (int64_t col = 0; col < n0 * n1; col++) {
        const int64_t i = col / n1, j = col % n1;
        double* V = alpha + col * n2;
        for (int64_t k = 0; k < n2; k++) V[k] = 0.0;
        for (int64_t e = cnt[col]; e < cnt[col + 1]; e++) {
            const int64_t t = list[e];
            og_poly A, B;
            A.n = 3;
            for (int c = 0; c < 3; c++) memcpy(A.p[c], verts + 3 * (int64_t)tris[3 * t + c], sizeof(double) * 3);
            og_clip_half(&A, &B, 0, og_plane(g, 0, i), 1);
            if (B.n < 3) continue;
            og_clip_half(&B, &A, 0, og_plane(g, 0, i + 1), 0);
            if (A.n < 3) continue;
            og_clip_half(&A, &B, 1, og_plane(g, 1, j), 1);
            if (B.n < 3) continue;
            og_clip_half(&B, &A, 1, og_plane(g, 1, j + 1), 0);
            if (A.n < 3) continue;
            double az, zaz, zmin = A.p[0][2], zmax = A.p[0][2];
            og_fan_z(&A, &az, &zaz);
            for (int m = 1; m < A.n; m++) {
                if (A.p[m][2] < zmin) zmin = A.p[m][2];
                if (A.p[m][2] > zmax) zmax = A.p[m][2];
            }
            for (int64_t k = 0; k < n2; k++) {
                const double zk = og_plane(g, 2, k), zk1 = og_plane(g, 2, k + 1);
                if (zmax <= zk) continue;             /* entirely below: clamp(z) - Z_k = 0 */
                if (zmin >= zk1) { V[k] += h * az; continue; } /* entirely above */
                og_poly S, T, U;
                og_clip_half(&A, &S, 2, zk, 1);
                if (S.n >= 3) {
                    og_clip_half(&S, &T, 2, zk1, 0);
                    if (T.n >= 3) {
                        double a2, za2;
                        og_fan_z(&T, &a2, &za2);
                        V[k] += za2 - zk * a2;
                    }
                }
                og_clip_half(&A, &U, 2, zk1, 1);
                if (U.n >= 3) {
                    double a3, za3;
                    og_fan_z(&U, &a3, &za3);
                    V[k] += h * a3;
                }
            }
        }
        for (int64_t k = 0; k < n2; k++) {
            const double a = V[k] / h3;
            if (inter[col * n2 + k]) {
                V[k] = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
            } else {
                const double r = floor(a + 0.5);
                if (fabs(a - r) > 1e-9) st |= OG_NOT_CLOSED;
                if (r != 0.0 && r != 1.0) st |= OG_ORIENTATION;
                V[k] = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
            }
        }
    }
    free(list);
    free(cnt);
    free(inter);
    if (status) *status |= st;
    return st ? -1 : 0;
}

/* vertex -> incident triangles, each list in ascending triangle order */
typedef struct {
    int64_t* off; /* nv + 1 */
    int32_t* tri; /* 3 nt   */
} og_inc;

static og_inc og_incidence(int64_t nv, const int32_t* tris, int64_t nt) {
    og_inc I;
    I.off = (int64_t*)calloc((size_t)nv + 1, sizeof(int64_t));
    I.tri = (int32_t*)malloc(sizeof(int32_t) * (size_t)(3 * nt + 1));
    for (int64_t t = 0; t < nt; t++)
        for (int c = 0; c < 3; c++) I.off[tris[3 * t + c] + 1]++;
    for (int64_t v = 0; v < nv; v++) I.off[v + 1] += I.off[v];
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    memcpy(cur, I.off, sizeof(int64_t) * (size_t)(nv + 1));
    for (int64_t t = 0; t < nt; t++) /* ascending t: lists come out sorted */
        for (int c = 0; c < 3; c++) I.tri[cur[tris[3 * t + c]]++] = (int32_t)t;
    free(cur);
    return I;
}

static void og_inc_free(og_inc* I) {
    free(I->off);
    free(I->tri);
}

static int og_cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* The k-ring of triangles around vertex v (k >= 1): the triangles incident to
 * v; then, k - 1 times, every triangle sharing a vertex with the ring so far.
 * Returns a malloc'ed ascending list and its length. */
static int32_t* og_ring_list(const og_inc* I, const int32_t* tris, int64_t v, int32_t k, int64_t* count) {
    int64_t n = I->off[v + 1] - I->off[v];
    int32_t* ring = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    memcpy(ring, I->tri + I->off[v], sizeof(int32_t) * (size_t)n);
    for (int32_t r = 2; r <= k; r++) {
        int64_t cap = 0;
        for (int64_t q = 0; q < n; q++)
            for (int c = 0; c < 3; c++) {
                const int64_t u = tris[3 * (int64_t)ring[q] + c];
                cap += I->off[u + 1] - I->off[u];
            }
        int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap + 1));
        int64_t m = 0;
        for (int64_t q = 0; q < n; q++)
            for (int c = 0; c < 3; c++) {
                const int64_t u = tris[3 * (int64_t)ring[q] + c];
                for (int64_t e = I->off[u]; e < I->off[u + 1]; e++) cand[m++] = I->tri[e];
            }
        qsort(cand, (size_t)m, sizeof(int32_t), og_cmp_i32);
        int64_t u = 0;
        for (int64_t q = 0; q < m; q++)
            if (q == 0 || cand[q] != cand[q - 1]) cand[u++] = cand[q];
        free(ring);
        ring = cand;
        n = u;
    }
    *count = n;
    return ring;
}

int64_t og_ring(int64_t nv, const int32_t* tris, int64_t nt, int64_t v, int32_t k, int32_t* out, int64_t cap) {
    og_inc I = og_incidence(nv, tris, nt);
    int64_t n = 0;
    int32_t* r = og_ring_list(&I, tris, v, k, &n);
    for (int64_t q = 0; q < n && q < cap; q++) out[q] = r[q];
    free(r);
    og_inc_free(&I);
    return n;
}

/* cell centre of (i, j, k): origin + (index + 1/2) h, each operation rounded */
static void og_cell_centre(const og_grid* g, int64_t i, int64_t j, int64_t k, double* xc) {
    xc[0] = g->origin[0] + ((double)i + 0.5) * g->h;
    xc[1] = g->origin[1] + ((double)j + 0.5) * g->h;
    xc[2] = g->origin[2] + ((double)k + 0.5) * g->h;
}

/* The front vertex closest to xc: |x - xc|^2 = (dx dx + dy dy) + dz dz with
 * every operation rounded; the lowest index among equal distances. */
static int64_t og_closest_one(const double* verts, int64_t nv, const double* xc) {
    int64_t best = -1;
    double bd = INFINITY;
    for (int64_t v = 0; v < nv; v++) {
        const double dx = verts[3 * v] - xc[0], dy = verts[3 * v + 1] - xc[1], dz = verts[3 * v + 2] - xc[2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < bd) {
            bd = d2;
            best = v;
        }
    }
    return best;
}

/* Normal of vertex v: the normalized sum of the area vectors (b - a) x (c - a)
 * of its triangles (a, b, c), in ascending triangle order; -1 if the sum is 0. */
static int og_vertex_normal(const double* verts, const int32_t* tris, const og_inc* I, int64_t v, double* n) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t q = I->off[v]; q < I->off[v + 1]; q++) {
        const int64_t t = I->tri[q];
        const double* a = verts + 3 * (int64_t)tris[3 * t];
        const double* b = verts + 3 * (int64_t)tris[3 * t + 1];
        const double* c = verts + 3 * (int64_t)tris[3 * t + 2];
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        s[0] += e1[1] * e2[2] - e1[2] * e2[1];
        s[1] += e1[2] * e2[0] - e1[0] * e2[2];
        s[2] += e1[0] * e2[1] - e1[1] * e2[0];
    }
    const double l = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (!(l > 0.0)) return -1;
    for (int d = 0; d < 3; d++) n[d] = s[d] / l;
    return 0;
}

void og_closest_vertex(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const og_grid* g,
                       int64_t ncells, const uint32_t* cells, int32_t* closest, double* vnormal) {
    og_inc I = og_incidence(nv, tris, nt);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < ncells; c++) {
        const uint64_t key = cells[c];
        const int64_t k = (int64_t)(key % (uint64_t)g->n[2]);
        const int64_t j = (int64_t)((key / (uint64_t)g->n[2]) % (uint64_t)g->n[1]);
        const int64_t i = (int64_t)(key / ((uint64_t)g->n[2] * (uint64_t)g->n[1]));
        double xc[3];
        og_cell_centre(g, i, j, k, xc);
        const int64_t v = og_closest_one(verts, nv, xc);
        closest[c] = (int32_t)v;
        if (vnormal) {
            double n[3] = {0.0, 0.0, 0.0};
            if (v >= 0) og_vertex_normal(verts, tris, &I, v, n);
            for (int d = 0; d < 3; d++) vnormal[3 * c + d] = n[d];
        }
    }
    og_inc_free(&I);
}

/* ------------------------------------------------------------------------ */
/* PPIC volume fit                                                           */
/* ------------------------------------------------------------------------ */

/* Wendland C2 function, Eq. Wendland: (1 + 4q)(1 - q)^4 for q = d/delta <= 1 */
static double og_wendland(double q) {
    if (q >= 1.0) return 0.0;
    const double s = 1.0 - q;
    return (1.0 + 4.0 * q) * s * s * s * s;
}

double og_wendland_weight(double q) { return og_wendland(q); }

/* Orthonormal basis (t1, t2) completing the unit normal n.  The paper leaves
 * the tangents open (the fit is isotropic in (t1, t2)); this reading applies
 * the branchless construction of Duff et al. 2017 ("Building an orthonormal
 * basis, revisited") to m = R n in a fixed rotated reference frame R, whose
 * third row is (sin 1 cos 1, sin 1 sin 1, cos 1), and rotates the tangents back.  Duff's
 * construction switches with sign(m_z); in the rotated frame that switch no
 * longer falls on fronts with an exactly vertical normal (n_z = 0), which
 * axis-aligned or symmetric geometry produces routinely. */
static const double OG_R[3][3] = {{0.890670841215793, -0.3614406733922875, -0.2758008198422935},
                                  {0.0, 0.6066239971779142, -0.7949888842291382},
                                  {0.4546487134128409, 0.7080734182735712, 0.5403023058681398}};

static void og_basis(const double* n, double* t1, double* t2) {
    double m[3], u1[3], u2[3];
    for (int r = 0; r < 3; r++) m[r] = OG_R[r][0] * n[0] + OG_R[r][1] * n[1] + OG_R[r][2] * n[2];
    const double sg = copysign(1.0, m[2]);
    const double a = -1.0 / (sg + m[2]);
    const double b = m[0] * m[1] * a;
    u1[0] = 1.0 + sg * m[0] * m[0] * a; u1[1] = sg * b; u1[2] = -sg * m[0];
    u2[0] = b; u2[1] = sg + m[1] * m[1] * a; u2[2] = -m[1];
    for (int c = 0; c < 3; c++) {
        t1[c] = OG_R[0][c] * u1[0] + OG_R[1][c] * u1[1] + OG_R[2][c] * u1[2];
        t2[c] = OG_R[0][c] * u2[0] + OG_R[1][c] * u2[1] + OG_R[2][c] * u2[2];
    }
}

/* Gaussian elimination with partial pivoting on an n x n system (row-major). */
static int og_solve(double* A, double* b, int n, double* x) {
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < n; k++) { double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; r++) {
            const double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

/* the pivots of elimination without pivoting (= LDL^T pivots of an SPD matrix) */
static double og_min_pivot(const double* M, int n) {
    double A[36];
    memcpy(A, M, sizeof(double) * (size_t)(n * n));
    double mn = INFINITY;
    for (int c = 0; c < n; c++) {
        const double d = A[c * n + c];
        if (d < mn) mn = d;
        if (d == 0.0) return 0.0;
        for (int r = c + 1; r < n; r++) {
            const double f = A[r * n + c] / d;
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
        }
    }
    return mn;
}

typedef struct {
    int64_t m;              /* number of interfacial cells */
    uint64_t* keys;         /* sorted cell keys */
    int64_t* off;           /* pair ranges per cell */
    int64_t* voff;          /* vertex offsets per pair */
    double* pv;             /* fragment polygon vertices */
} og_frags;

static og_frags og_build_frags(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                               const og_grid* g, int32_t margin) {
    og_frags F;
    uint32_t st = 0;
    og_vec pr = og_pairs(verts, nv, tris, nt, g, margin, &st);
    F.keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr.n + 1));
    F.off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(pr.n + 2));
    F.voff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(pr.n + 1));
    F.pv = (double*)malloc(sizeof(double) * 3 * OG_MAXV * (size_t)(pr.n + 1));
    F.m = 0;
    F.voff[0] = 0;
    for (int64_t q = 0; q < pr.n; q++) {
        const uint64_t key = pr.v[q] >> 32;
        const int64_t t = (int64_t)(pr.v[q] & 0xffffffffu);
        if (q == 0 || key != (pr.v[q - 1] >> 32)) { F.keys[F.m] = key; F.off[F.m] = q; F.m++; }
        const int64_t k = (int64_t)(key % (uint64_t)g->n[2]);
        const int64_t j = (int64_t)((key / (uint64_t)g->n[2]) % (uint64_t)g->n[1]);
        const int64_t i = (int64_t)(key / ((uint64_t)g->n[2] * (uint64_t)g->n[1]));
        og_poly r;
        const int n = og_canon(verts + 3 * (int64_t)tris[3 * t], verts + 3 * (int64_t)tris[3 * t + 1],
                               verts + 3 * (int64_t)tris[3 * t + 2], g, i, j, k, &r);
        memcpy(F.pv + 3 * F.voff[q], r.p, sizeof(double) * 3 * (size_t)n);
        F.voff[q + 1] = F.voff[q] + n;
    }
    F.off[F.m] = pr.n;
    free(pr.v);
    return F;
}

static int64_t og_find(const og_frags* F, uint64_t key) {
    int64_t lo = 0, hi = F->m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (F->keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < F->m && F->keys[lo] == key) ? lo : -1;
}

int og_ppic(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const og_grid* g,
            const og_params* p, int64_t ncells, const uint32_t* cells, double* kappa, double* normal,
            double* coeffs, int8_t* fit_status, double* frame) {
    const int32_t margin = 2 + (int32_t)ceil(p->delta_max_h);
    og_frags F = og_build_frags(verts, nv, tris, nt, g, margin);
    const double h = g->h;
    /* the paper's own neighbourhood and frame (Sec. 3.2) need the mesh incidence */
    const int variant = p->fit_ring > 0 || p->frame_vertex;
    og_inc I = {NULL, NULL};
    if (variant) I = og_incidence(nv, tris, nt);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : err)
    for (int64_t c = 0; c < ncells; c++) {
        const uint64_t key = cells[c];
        const int64_t ci = og_find(&F, key);
        int8_t stc = 0;
        double a[6] = {0, 0, 0, 0, 0, 0};
        if (ci < 0) {
            err |= 1;
            kappa[c] = 0.0;
            normal[3 * c] = normal[3 * c + 1] = normal[3 * c + 2] = 0.0;
            if (coeffs) for (int r = 0; r < 6; r++) coeffs[6 * c + r] = 0.0;
            if (frame) for (int r = 0; r < 9; r++) frame[9 * c + r] = 0.0;
            fit_status[c] = -1;
            continue;
        }
        const int64_t k0 = (int64_t)(key % (uint64_t)g->n[2]);
        const int64_t j0 = (int64_t)((key / (uint64_t)g->n[2]) % (uint64_t)g->n[1]);
        const int64_t i0 = (int64_t)(key / ((uint64_t)g->n[2] * (uint64_t)g->n[1]));
        const double xc[3] = {g->origin[0] + ((double)i0 + 0.5) * h, g->origin[1] + ((double)j0 + 0.5) * h,
                              g->origin[2] + ((double)k0 + 0.5) * h};
        double rv[OG_MAXV][3];
        /* 1. local normal: normalized sum of the fragment area vectors of this cell */
        double N[3] = {0, 0, 0}, sa = 0.0, best = -1.0, Nb[3] = {0, 0, 0};
        for (int64_t q = F.off[ci]; q < F.off[ci + 1]; q++) {
            const int nvq = (int)(F.voff[q + 1] - F.voff[q]);
            for (int m = 0; m < nvq; m++)
                for (int d = 0; d < 3; d++) rv[m][d] = (F.pv[3 * (F.voff[q] + m) + d] - xc[d]) / h;
            double Nf[3];
            og_newell((const double(*)[3])rv, nvq, Nf);
            const double af = sqrt(Nf[0] * Nf[0] + Nf[1] * Nf[1] + Nf[2] * Nf[2]);
            N[0] += Nf[0]; N[1] += Nf[1]; N[2] += Nf[2];
            sa += af;
            if (af > best) { best = af; Nb[0] = Nf[0]; Nb[1] = Nf[1]; Nb[2] = Nf[2]; }
        }
        double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        if (nn < 1e-3 * sa) {
            N[0] = Nb[0]; N[1] = Nb[1]; N[2] = Nb[2];
            nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
            stc |= 4;
        }
        double n[3] = {N[0] / nn, N[1] / nn, N[2] / nn};
        /* the paper's reading: the front vertex closest to the cell centre gives
         * the frame normal and the centre of the k-ring of fit triangles */
        int64_t vc = -1;
        if (variant) {
            vc = og_closest_one(verts, nv, xc);
            double nv_[3];
            if (p->frame_vertex) {
                if (vc >= 0 && og_vertex_normal(verts, tris, &I, vc, nv_) == 0) {
                    for (int d = 0; d < 3; d++) n[d] = nv_[d];
                    stc &= ~4;
                } else {
                    stc |= 4; /* no usable vertex normal: the fragment normal stays */
                }
            }
        }
        int64_t nring = 0;
        int32_t* ring = (p->fit_ring > 0 && vc >= 0) ? og_ring_list(&I, tris, vc, p->fit_ring, &nring) : NULL;
        double t1[3], t2[3];
        og_basis(n, t1, t2);
        if (p->frame_angle != 0.0) {
            const double cs = cos(p->frame_angle), sn = sin(p->frame_angle);
            double u1[3], u2[3];
            for (int d = 0; d < 3; d++) { u1[d] = cs * t1[d] + sn * t2[d]; u2[d] = -sn * t1[d] + cs * t2[d]; }
            memcpy(t1, u1, sizeof u1);
            memcpy(t2, u2, sizeof u2);
        }
        /* 2-4. weighted normal equations; grow the support until fit_min fragments count */
        double delta = p->delta_h;
        double M[36], b[6];
        for (;;) {
            memset(M, 0, sizeof M);
            memset(b, 0, sizeof b);
            int64_t count = 0;
            /* whole triangles of the ring: the Wendland distance from the triangle's centre */
            for (int64_t q = 0; q < nring; q++) {
                const int64_t t = ring[q];
                for (int m = 0; m < 3; m++)
                    for (int d = 0; d < 3; d++) rv[m][d] = (verts[3 * (int64_t)tris[3 * t + m] + d] - xc[d]) / h;
                double cf[3];
                for (int d = 0; d < 3; d++) cf[d] = (rv[0][d] + rv[1][d] + rv[2][d]) / 3.0;
                const double dist = sqrt(cf[0] * cf[0] + cf[1] * cf[1] + cf[2] * cf[2]);
                if (!(dist < delta)) continue;
                count++;
                const double w = og_wendland(dist / delta);
                double xs[3], ys[3], mom[6];
                for (int m = 0; m < 3; m++) {
                    xs[m] = t1[0] * rv[m][0] + t1[1] * rv[m][1] + t1[2] * rv[m][2];
                    ys[m] = t2[0] * rv[m][0] + t2[1] * rv[m][1] + t2[2] * rv[m][2];
                }
                og_green_moments(xs, ys, 3, mom);
                const double zc = n[0] * cf[0] + n[1] * cf[1] + n[2] * cf[2];
                const double G = mom[0] * zc;
                for (int r = 0; r < 6; r++) {
                    for (int s2 = 0; s2 < 6; s2++) M[r * 6 + s2] += w * mom[r] * mom[s2];
                    b[r] += w * G * mom[r];
                }
            }
            const int64_t R = (p->fit_ring > 0) ? -1 : (int64_t)ceil(delta - 0.5);
            for (int64_t di = -R; di <= R; di++)
                for (int64_t dj = -R; dj <= R; dj++)
                    for (int64_t dk = -R; dk <= R; dk++) {
                        const int64_t ii = i0 + di, jj = j0 + dj, kk = k0 + dk;
                        if (ii < 0 || jj < 0 || kk < 0 || ii >= g->n[0] || jj >= g->n[1] || kk >= g->n[2]) continue;
                        const int64_t cj = og_find(&F, og_key(g, ii, jj, kk));
                        if (cj < 0) continue;
                        for (int64_t q = F.off[cj]; q < F.off[cj + 1]; q++) {
                            const int nvq = (int)(F.voff[q + 1] - F.voff[q]);
                            for (int m = 0; m < nvq; m++)
                                for (int d = 0; d < 3; d++) rv[m][d] = (F.pv[3 * (F.voff[q] + m) + d] - xc[d]) / h;
                            double Nf[3], cf[3];
                            og_newell((const double(*)[3])rv, nvq, Nf);
                            const double af = sqrt(Nf[0] * Nf[0] + Nf[1] * Nf[1] + Nf[2] * Nf[2]);
                            const double nh[3] = {Nf[0] / af, Nf[1] / af, Nf[2] / af};
                            og_centroid((const double(*)[3])rv, nvq, nh, cf);
                            const double dist = sqrt(cf[0] * cf[0] + cf[1] * cf[1] + cf[2] * cf[2]);
                            if (!(dist < delta)) continue;
                            count++;
                            const double w = og_wendland(dist / delta);
                            /* projection onto (t1, t2): the domain Gamma_t of Eq. volumefit */
                            double xs[OG_MAXV], ys[OG_MAXV], mom[6];
                            for (int m = 0; m < nvq; m++) {
                                xs[m] = t1[0] * rv[m][0] + t1[1] * rv[m][1] + t1[2] * rv[m][2];
                                ys[m] = t2[0] * rv[m][0] + t2[1] * rv[m][1] + t2[2] * rv[m][2];
                            }
                            og_green_moments(xs, ys, nvq, mom);
                            /* int_Gamma g_t dA = (projected area) x (height of the centroid) */
                            const double zc = n[0] * cf[0] + n[1] * cf[1] + n[2] * cf[2];
                            const double G = mom[0] * zc;
                            for (int r = 0; r < 6; r++) {
                                for (int s = 0; s < 6; s++) M[r * 6 + s] += w * mom[r] * mom[s];
                                b[r] += w * G * mom[r];
                            }
                        }
                    }
            if (count >= p->fit_min || delta >= p->delta_max_h) break;
            delta = delta * p->delta_growth;
            if (delta > p->delta_max_h) delta = p->delta_max_h;
            stc |= 1;
        }
        /* 5. solve the normal equations (Eq. volumefit2) */
        double tr = 0.0;
        for (int r = 0; r < 6; r++) tr += M[r * 6 + r];
        double A6[36], b6[6];
        memcpy(A6, M, sizeof A6);
        memcpy(b6, b, sizeof b6);
        if (!(og_min_pivot(M, 6) >= 1e-12 * tr) || og_solve(A6, b6, 6, a) != 0) {
            double A3[9], b3[3], a3[3];
            for (int r = 0; r < 3; r++) {
                for (int s = 0; s < 3; s++) A3[r * 3 + s] = M[r * 6 + s];
                b3[r] = b[r];
            }
            for (int r = 0; r < 6; r++) a[r] = 0.0;
            if (og_solve(A3, b3, 3, a3) == 0) { a[0] = a3[0]; a[1] = a3[1]; a[2] = a3[2]; }
            stc |= 2;
        }
        /* 6. mean curvature of the graph z = P(x, y) at the origin, kappa = div n (> 0 on a sphere) */
        const double g2 = 1.0 + a[1] * a[1] + a[2] * a[2];
        const double kl = -(2.0 * a[3] * (1.0 + a[2] * a[2]) - 2.0 * a[1] * a[2] * a[4] +
                            2.0 * a[5] * (1.0 + a[1] * a[1])) / (g2 * sqrt(g2));
        kappa[c] = kl / h;
        double nv3[3];
        for (int d = 0; d < 3; d++) nv3[d] = n[d] - a[1] * t1[d] - a[2] * t2[d];
        const double nl = sqrt(nv3[0] * nv3[0] + nv3[1] * nv3[1] + nv3[2] * nv3[2]);
        for (int d = 0; d < 3; d++) normal[3 * c + d] = nv3[d] / nl;
        if (coeffs) for (int r = 0; r < 6; r++) coeffs[6 * c + r] = a[r];
        if (frame)
            for (int d = 0; d < 3; d++) {
                frame[9 * c + d] = t1[d];
                frame[9 * c + 3 + d] = t2[d];
                frame[9 * c + 6 + d] = n[d];
            }
        fit_status[c] = stc;
        free(ring);
    }
    if (variant) og_inc_free(&I);
    free(F.keys); free(F.off); free(F.voff); free(F.pv);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* CSF force                                                                 */
/* ------------------------------------------------------------------------ */

/* The curvature of cell (i,j,k) used by the surface-tension terms (Sec. 3.3):
 * its own kappa if it is interfacial, else the weighted mean
 * kbar = sum_Q kappa_Q w_Q / sum_Q w_Q, w_Q = |s_Q . n_Q| / |s_Q|, over the
 * interfacial cells Q among its 26 neighbours (the plain mean if every w_Q is 0,
 * 0 if there is none). */
static double og_cell_kappa(const og_grid* g, const int32_t* map, const double* kappa, const double* normal,
                            int64_t i, int64_t j, int64_t k) {
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    const int64_t key = (i * n1 + j) * n2 + k;
    if (map[key] >= 0) return kappa[map[key]];
    double num = 0.0, den = 0.0, ksum = 0.0;
    int cnt = 0;
    for (int di = -1; di <= 1; di++)
        for (int dj = -1; dj <= 1; dj++)
            for (int dk = -1; dk <= 1; dk++) {
                if (!di && !dj && !dk) continue;
                const int64_t ii = i + di, jj = j + dj, kk = k + dk;
                if (ii < 0 || jj < 0 || kk < 0 || ii >= n0 || jj >= n1 || kk >= n2) continue;
                const int32_t q = map[(ii * n1 + jj) * n2 + kk];
                if (q < 0) continue;
                const double* nq = normal + 3 * (int64_t)q;
                const double sl = sqrt((double)(di * di + dj * dj + dk * dk));
                const double w = fabs(di * nq[0] + dj * nq[1] + dk * nq[2]) / sl;
                num += kappa[q] * w;
                den += w;
                ksum += kappa[q];
                cnt++;
            }
    return den > 0.0 ? num / den : (cnt ? ksum / cnt : 0.0);
}

static int32_t* og_index_map(const og_grid* g, int64_t ncells, const uint32_t* cells) {
    const int64_t NC = (int64_t)g->n[0] * g->n[1] * g->n[2];
    int32_t* map = (int32_t*)malloc(sizeof(int32_t) * (size_t)NC);
    for (int64_t c = 0; c < NC; c++) map[c] = -1;
    for (int64_t m = 0; m < ncells; m++) map[cells[m]] = (int32_t)m;
    return map;
}

int og_csf(const og_grid* g, const double* alpha, int64_t ncells, const uint32_t* cells,
           const double* kappa, const double* normal, double sigma, double* force) {
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2], NC = n0 * n1 * n2;
    int32_t* map = og_index_map(g, ncells, cells);
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n0; i++)
        for (int64_t j = 0; j < n1; j++)
            for (int64_t k = 0; k < n2; k++) {
                const int64_t key = (i * n1 + j) * n2 + k;
                /* alpha outside the domain is 0 */
                const double axp = (i + 1 < n0) ? alpha[key + n1 * n2] : 0.0;
                const double axm = (i > 0) ? alpha[key - n1 * n2] : 0.0;
                const double ayp = (j + 1 < n1) ? alpha[key + n2] : 0.0;
                const double aym = (j > 0) ? alpha[key - n2] : 0.0;
                const double azp = (k + 1 < n2) ? alpha[key + 1] : 0.0;
                const double azm = (k > 0) ? alpha[key - 1] : 0.0;
                const double gr[3] = {(axp - axm) / (2.0 * h), (ayp - aym) / (2.0 * h), (azp - azm) / (2.0 * h)};
                if (gr[0] == 0.0 && gr[1] == 0.0 && gr[2] == 0.0) {
                    force[key] = force[NC + key] = force[2 * NC + key] = 0.0;
                    continue;
                }
                const double kp = og_cell_kappa(g, map, kappa, normal, i, j, k);
                for (int d = 0; d < 3; d++) force[d * NC + key] = sigma * kp * gr[d];
            }
    free(map);
    return 0;
}

/* Face term of the balanced-force treatment of surface tension (Sec. 3.3,
 * Eq. mwi_disc): on the face f between cells P and Q = P + e_d,
 *   S_f = sigma kbar_f (alpha_Q - alpha_P) / h,  kbar_f = (kappa_P + kappa_Q) / 2,
 * with kappa_P the cell curvature of og_cell_kappa; outside the grid alpha and
 * kappa are 0.  F[d] has the staggered layout of the face velocities:
 * (n0+1, n1, n2), (n0, n1+1, n2), (n0, n1, n2+1); face index i along d is the
 * face between cells i-1 and i. */
int og_face_force(const og_grid* g, const double* alpha, int64_t ncells, const uint32_t* cells,
                  const double* kappa, const double* normal, double sigma, double* Fx, double* Fy, double* Fz) {
    const int64_t n[3] = {g->n[0], g->n[1], g->n[2]};
    int32_t* map = og_index_map(g, ncells, cells);
    double* F[3] = {Fx, Fy, Fz};
    const double h = g->h;
    for (int d = 0; d < 3; d++) {
        int64_t e[3] = {n[0], n[1], n[2]};
        e[d] += 1;
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < e[0]; a++)
            for (int64_t b = 0; b < e[1]; b++)
                for (int64_t c = 0; c < e[2]; c++) {
                    const int64_t f = (a * e[1] + b) * e[2] + c;
                    int64_t q[3] = {a, b, c}; /* cell Q (upper side) */
                    int64_t p[3] = {a, b, c};
                    p[d] -= 1;                 /* cell P (lower side) */
                    const int pin = p[d] >= 0, qin = q[d] < n[d];
                    const double ap = pin ? alpha[(p[0] * n[1] + p[1]) * n[2] + p[2]] : 0.0;
                    const double aq = qin ? alpha[(q[0] * n[1] + q[1]) * n[2] + q[2]] : 0.0;
                    if (ap == aq) {
                        F[d][f] = 0.0;
                        continue;
                    }
                    const double kp = pin ? og_cell_kappa(g, map, kappa, normal, p[0], p[1], p[2]) : 0.0;
                    const double kq = qin ? og_cell_kappa(g, map, kappa, normal, q[0], q[1], q[2]) : 0.0;
                    F[d][f] = sigma * 0.5 * (kp + kq) * (aq - ap) / h;
                }
    }
    free(map);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* velocity interpolation                                                    */
/* ------------------------------------------------------------------------ */

/* face value of a staggered array with extents (e0, e1, e2) */
static double og_at(const double* A, int64_t e1, int64_t e2, int64_t i, int64_t j, int64_t k) {
    return A[(i * e1 + j) * e2 + k];
}

/* derivative along `dir` of the face array A at face (i,j,k): central in the
 * interior, one-sided at the first and last face rows of that direction */
static double og_tgrad(const double* A, const int64_t e[3], int dir, int64_t i, int64_t j, int64_t k, double h) {
    int64_t idx[3] = {i, j, k};
    const int64_t c = idx[dir], n = e[dir];
    int64_t lo = c - 1, hi = c + 1;
    double span = 2.0 * h;
    if (c == 0) { lo = 0; hi = 1; span = h; }
    else if (c == n - 1) { lo = n - 2; hi = n - 1; span = h; }
    idx[dir] = hi;
    const double vh = og_at(A, e[1], e[2], idx[0], idx[1], idx[2]);
    idx[dir] = lo;
    const double vl = og_at(A, e[1], e[2], idx[0], idx[1], idx[2]);
    return (vh - vl) / span;
}

/* the interpolated velocity at one point x (Sec. 3.1) */
static void og_interp_one(const og_grid* g, const double* const F[3], const int64_t* const E[3], const double* x,
                          double* vel) {
    const double h = g->h;
    int64_t c[3];
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        double f = floor((x[d] - g->origin[d]) / h);
        const int64_t nd = g->n[d];
        c[d] = (f >= 0.0) ? ((f <= (double)(nd - 1)) ? (int64_t)f : nd - 1) : 0;
        lo[d] = og_plane(g, d, c[d]);
        hi[d] = og_plane(g, d, c[d] + 1);
    }
    /* component d along its own axis: faces c[d] (minus) and c[d]+1 (plus) */
    for (int d = 0; d < 3; d++) {
        const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
        const double* A = F[d];
        const int64_t* ext = E[d];
        int64_t im[3] = {c[0], c[1], c[2]}, ip[3] = {c[0], c[1], c[2]};
        ip[d] += 1;
        const double Am = og_at(A, ext[1], ext[2], im[0], im[1], im[2]);
        const double Ap = og_at(A, ext[1], ext[2], ip[0], ip[1], ip[2]);
        const double g1m = og_tgrad(A, ext, e1, im[0], im[1], im[2], h);
        const double g2m = og_tgrad(A, ext, e2, im[0], im[1], im[2], h);
        const double g1p = og_tgrad(A, ext, e1, ip[0], ip[1], ip[2], h);
        const double g2p = og_tgrad(A, ext, e2, ip[0], ip[1], ip[2], h);
        const double y1 = x[e1] - (lo[e1] + hi[e1]) / 2.0;
        const double y2 = x[e2] - (lo[e2] + hi[e2]) / 2.0;
        /* transverse derivatives along d of the two other components on their own faces */
        double corr = 0.0;
        for (int s = 1; s <= 2; s++) {
            const int o = (d + s) % 3;
            const double* B = F[o];
            const int64_t* eb = E[o];
            int64_t bm[3] = {c[0], c[1], c[2]}, bp[3] = {c[0], c[1], c[2]};
            bp[o] += 1;
            corr += og_tgrad(B, eb, d, bp[0], bp[1], bp[2], h) - og_tgrad(B, eb, d, bm[0], bm[1], bm[2], h);
        }
        const double xi = x[d];
        vel[d] = (xi - lo[d]) / h * (Ap + y1 * g1p + y2 * g2p) + (hi[d] - xi) / h * (Am + y1 * g1m + y2 * g2m) +
                 (hi[d] - xi) * (xi - lo[d]) / (2.0 * h) * corr;
    }
}

void og_interp(const og_grid* g, const double* U, const double* V, const double* W, const double* pts,
               int64_t np, double* vel) {
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    const int64_t eU[3] = {n0 + 1, n1, n2}, eV[3] = {n0, n1 + 1, n2}, eW[3] = {n0, n1, n2 + 1};
    const double* const F[3] = {U, V, W};
    const int64_t* const E[3] = {eU, eV, eW};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) og_interp_one(g, F, E, pts + 3 * p, vel + 3 * p);
}

/* One step of the classical fourth-order Runge-Kutta scheme for dx/dt = u(x)
 * (Sec. 3.1), u the interpolated velocity of the face field, which is held
 * fixed during the step:
 *   k1 = u(x), k2 = u(x + dt/2 k1), k3 = u(x + dt/2 k2), k4 = u(x + dt k3),
 *   x_new = x + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * vel (may be NULL) receives k1, the interpolated velocity at the start. */
void og_advect_rk4(const og_grid* g, const double* U, const double* V, const double* W, const double* pts,
                   int64_t np, double dt, double* out, double* vel) {
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    const int64_t eU[3] = {n0 + 1, n1, n2}, eV[3] = {n0, n1 + 1, n2}, eW[3] = {n0, n1, n2 + 1};
    const double* const F[3] = {U, V, W};
    const int64_t* const E[3] = {eU, eV, eW};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) {
        const double* x = pts + 3 * p;
        double k1[3], k2[3], k3[3], k4[3], y[3];
        og_interp_one(g, F, E, x, k1);
        for (int d = 0; d < 3; d++) y[d] = x[d] + 0.5 * dt * k1[d];
        og_interp_one(g, F, E, y, k2);
        for (int d = 0; d < 3; d++) y[d] = x[d] + 0.5 * dt * k2[d];
        og_interp_one(g, F, E, y, k3);
        for (int d = 0; d < 3; d++) y[d] = x[d] + dt * k3[d];
        og_interp_one(g, F, E, y, k4);
        for (int d = 0; d < 3; d++) {
            out[3 * p + d] = x[d] + dt / 6.0 * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);
            if (vel) vel[3 * p + d] = k1[d];
        }
    }
}

void og_set_threads(int nthreads) {
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
    (void)nthreads;
#endif
}

int og_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* local roughness detection and smoothing (Sec. 3.4)                        */
/* ------------------------------------------------------------------------ */

/* position of vertex v in triangle t (0..2), -1 if absent */
static int og_slot(const int32_t* tris, int64_t t, int64_t v) {
    for (int c = 0; c < 3; c++)
        if (tris[3 * t + c] == v) return c;
    return -1;
}

/* the triangle (other than t) that holds the directed edge b -> a, found among
 * the triangles incident to a; -1 if the mesh is open there */
static int64_t og_twin(const og_inc* I, const int32_t* tris, int64_t a, int64_t b) {
    for (int64_t q = I->off[a]; q < I->off[a + 1]; q++) {
        const int64_t t = I->tri[q];
        const int sb = og_slot(tris, t, b);
        if (sb >= 0 && tris[3 * t + (sb + 1) % 3] == a) return t;
    }
    return -1;
}

int og_roughness(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double* gl, double* rough,
                 double* r1, double* r2, double* rt, double* G, double* V) {
    og_inc I = og_incidence(nv, tris, nt);
    double* nrm = (double*)malloc(sizeof(double) * 3 * (size_t)(nt + 1));
    double* area = (double*)malloc(sizeof(double) * (size_t)(nt + 1));
    for (int64_t t = 0; t < nt; t++) {
        const double* a = verts + 3 * (int64_t)tris[3 * t];
        const double* b = verts + 3 * (int64_t)tris[3 * t + 1];
        const double* c = verts + 3 * (int64_t)tris[3 * t + 2];
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double x[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double l = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        area[t] = 0.5 * l;
        for (int d = 0; d < 3; d++) nrm[3 * t + d] = l > 0.0 ? x[d] / l : 0.0;
    }
    for (int64_t i = 0; i < nv; i++) {
        const double* xi = verts + 3 * i;
        /* geometric Laplacian (Karni and Gotsman 2000): x_i minus the inverse-
         * distance weighted mean of the one-ring; every neighbour of a closed
         * mesh lies in exactly two incident triangles, so summing over the
         * incident triangles' other vertices weights each neighbour twice */
        double sw = 0.0, sx[3] = {0.0, 0.0, 0.0};
        /* edge roughness over the edges i -> next(i) of the incident triangles
         * (each undirected edge at i exactly once on a closed oriented mesh) */
        double sum = 0.0, sum2 = 0.0;
        int ne = 0;
        for (int64_t q = I.off[i]; q < I.off[i + 1]; q++) {
            const int64_t t = I.tri[q];
            const int s = og_slot(tris, t, i);
            for (int o = 1; o <= 2; o++) {
                const double* xj = verts + 3 * (int64_t)tris[3 * t + (s + o) % 3];
                const double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                const double w = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
                sw += w;
                for (int d = 0; d < 3; d++) sx[d] += w * xj[d];
            }
            const int64_t j = tris[3 * t + (s + 1) % 3];
            const int64_t u = og_twin(&I, tris, i, j);
            if (u < 0) continue;
            const double re = 1.0 - (nrm[3 * t] * nrm[3 * u] + nrm[3 * t + 1] * nrm[3 * u + 1] +
                                     nrm[3 * t + 2] * nrm[3 * u + 2]);
            sum += re;
            sum2 += re * re;
            ne++;
        }
        for (int d = 0; d < 3; d++) gl[3 * i + d] = sw > 0.0 ? xi[d] - sx[d] / sw : 0.0;
        G[i] = ne ? sum / ne : 0.0;
        /* variance of the edge roughness at i (population variance) */
        V[i] = ne ? sum2 / ne - G[i] * G[i] : 0.0;
        if (V[i] < 0.0) V[i] = 0.0;
    }
    for (int64_t t = 0; t < nt; t++) {
        /* R_t = sum G_i V_i / sum V_i over its vertices (Corsini et al. 2007);
         * equal weights when every V_i is zero */
        double num = 0.0, den = 0.0, gm = 0.0;
        for (int c = 0; c < 3; c++) {
            const int64_t v = tris[3 * t + c];
            num += G[v] * V[v];
            den += V[v];
            gm += G[v];
        }
        rt[t] = den > 0.0 ? num / den : gm / 3.0;
    }
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt + 1));
    for (int64_t t = 0; t < nt; t++) mark[t] = -1;
    for (int64_t i = 0; i < nv; i++) {
        /* one ring: the incident triangles; two rings: the triangles incident to
         * i or to one of its neighbours (each counted once) */
        double s1 = 0.0, s2 = 0.0;
        int64_t c1 = 0, c2 = 0;
        for (int64_t q = I.off[i]; q < I.off[i + 1]; q++) {
            const int64_t t = I.tri[q];
            s1 += area[t] * rt[t];
            c1++;
            for (int c = 0; c < 3; c++) {
                const int64_t v = tris[3 * t + c];
                for (int64_t q2 = I.off[v]; q2 < I.off[v + 1]; q2++) {
                    const int64_t t2 = I.tri[q2];
                    if (mark[t2] == (int32_t)i) continue;
                    mark[t2] = (int32_t)i;
                    s2 += area[t2] * rt[t2];
                    c2++;
                }
            }
        }
        r1[i] = c1 ? s1 / c1 : 0.0;
        r2[i] = c2 ? s2 / c2 : 0.0;
        rough[i] = r1[i] > r2[i] ? r1[i] : r2[i];
    }
    free(mark);
    free(nrm);
    free(area);
    og_inc_free(&I);
    return 0;
}

/* Edge priority of the parallel smoothing schedule: the 64-bit finalizer of
 * SplitMix64 (Steele, Lea and Flood 2014) applied to the edge id. */
uint64_t og_edge_priority(uint64_t e) {
    uint64_t z = e + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* The volume-conserving move of edge (a, b) (Kuprat et al. 2001, Algorithm 4,
 * as stated in Sec. 3.4): simultaneous Laplacian smoothing of both vertices,
 * then a common shift h n along the direction that keeps the enclosed volume,
 * with |h n| minimal.  Moving a by da and b by db changes six times the
 * enclosed volume by da.A_a + db.A_b + da.(db x y), A_i = sum over the
 * triangles (i, j, k) at i of x_j x x_k, y = x_p - x_q for the triangles
 * (a, b, p) and (b, a, q) holding the edge; with da = d_a + h n, db = d_b + h n
 * this is linear in h. */
static void og_kuprat_move(const double* verts, const og_inc* I, const int32_t* tris, int64_t a, int64_t b,
                           int64_t p, int64_t q, double* xa_new, double* xb_new) {
    const double* xa = verts + 3 * a;
    const double* xb = verts + 3 * b;
    double Sa[3] = {0, 0, 0}, Sb[3] = {0, 0, 0}, Aa[3] = {0, 0, 0}, Ab[3] = {0, 0, 0};
    int64_t na = 0, nb = 0;
    for (int side = 0; side < 2; side++) {
        const int64_t v = side ? b : a;
        const int64_t other = side ? a : b;
        double* S = side ? Sb : Sa;
        double* A = side ? Ab : Aa;
        int64_t cnt = 0;
        for (int64_t r = I->off[v]; r < I->off[v + 1]; r++) {
            const int64_t t = I->tri[r];
            const int s = og_slot(tris, t, v);
            const double* xj = verts + 3 * (int64_t)tris[3 * t + (s + 1) % 3];
            const double* xk = verts + 3 * (int64_t)tris[3 * t + (s + 2) % 3];
            A[0] += xj[1] * xk[2] - xj[2] * xk[1];
            A[1] += xj[2] * xk[0] - xj[0] * xk[2];
            A[2] += xj[0] * xk[1] - xj[1] * xk[0];
            /* neighbours other than the edge partner: next(v) of every triangle */
            const int64_t jn = tris[3 * t + (s + 1) % 3];
            cnt++;
            if (jn != other)
                for (int d = 0; d < 3; d++) S[d] += verts[3 * jn + d];
        }
        if (side)
            nb = cnt;
        else
            na = cnt;
    }
    /* x_a^s = (x_b^s + S_a)/n_a, x_b^s = (x_a^s + S_b)/n_b solved together */
    double xsa[3], xsb[3], da[3], db[3], y[3], m[3];
    const double den = (double)na * (double)nb - 1.0;
    for (int d = 0; d < 3; d++) {
        xsa[d] = (Sb[d] + (double)nb * Sa[d]) / den;
        xsb[d] = (xsa[d] + Sb[d]) / (double)nb;
        da[d] = xsa[d] - xa[d];
        db[d] = xsb[d] - xb[d];
        y[d] = verts[3 * p + d] - verts[3 * q + d];
    }
    const double ydd[3] = {y[1] * (da[2] - db[2]) - y[2] * (da[1] - db[1]), y[2] * (da[0] - db[0]) - y[0] * (da[2] - db[2]),
                           y[0] * (da[1] - db[1]) - y[1] * (da[0] - db[0])};
    for (int d = 0; d < 3; d++) m[d] = Aa[d] + Ab[d] + ydd[d];
    const double ml = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    const double dbxy[3] = {db[1] * y[2] - db[2] * y[1], db[2] * y[0] - db[0] * y[2], db[0] * y[1] - db[1] * y[0]};
    const double c0 = da[0] * Aa[0] + da[1] * Aa[1] + da[2] * Aa[2] + db[0] * Ab[0] + db[1] * Ab[1] + db[2] * Ab[2] +
                      da[0] * dbxy[0] + da[1] * dbxy[1] + da[2] * dbxy[2];
    double h = 0.0, n[3] = {0.0, 0.0, 0.0};
    if (ml > 0.0) {
        for (int d = 0; d < 3; d++) n[d] = m[d] / ml;
        h = -c0 / ml; /* n . m = |m| */
    }
    for (int d = 0; d < 3; d++) {
        xa_new[d] = xsa[d] + h * n[d];
        xb_new[d] = xsb[d] + h * n[d];
    }
}

/* Local roughness smoothing (Sec. 3.4): a vertex is rough when |GL| > gl_thr
 * and its roughness R > r_thr; every edge with a rough endpoint is smoothed by
 * og_kuprat_move.  Edges are taken in rounds: an edge moves in a round when its
 * priority (og_edge_priority of its id 3t + s, the triangle t and slot s where
 * it runs a -> b with a < b) is the smallest among the pending edges that touch
 * the closed one-rings of a and b; the moves of a round read the positions at
 * its start and touch disjoint vertex stars.  verts is updated in place;
 * returns the number of rounds (at most max_rounds), *moved the edges moved. */
int og_roughness_smooth(double* verts, int64_t nv, const int32_t* tris, int64_t nt, double gl_thr, double r_thr,
                        int max_rounds, int64_t* moved) {
    double* gl = (double*)malloc(sizeof(double) * 3 * (size_t)(nv + 1));
    double* rough = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    double* r1 = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    double* r2 = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    double* rtt = (double*)malloc(sizeof(double) * (size_t)(nt + 1));
    double* G = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    double* V = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    og_roughness(verts, nv, tris, nt, gl, rough, r1, r2, rtt, G, V);
    og_inc I = og_incidence(nv, tris, nt);
    uint8_t* pend = (uint8_t*)calloc((size_t)(3 * nt + 1), 1);
    int64_t npend = 0;
    for (int64_t t = 0; t < nt; t++)
        for (int s = 0; s < 3; s++) {
            const int64_t a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
            if (a >= b) continue;
            const int ra = sqrt(gl[3 * a] * gl[3 * a] + gl[3 * a + 1] * gl[3 * a + 1] + gl[3 * a + 2] * gl[3 * a + 2]) > gl_thr &&
                           rough[a] > r_thr;
            const int rb = sqrt(gl[3 * b] * gl[3 * b] + gl[3 * b + 1] * gl[3 * b + 1] + gl[3 * b + 2] * gl[3 * b + 2]) > gl_thr &&
                           rough[b] > r_thr;
            if (ra || rb) {
                pend[3 * t + s] = 1;
                npend++;
            }
        }
    int64_t total = 0;
    int rounds = 0;
    double* newpos = (double*)malloc(sizeof(double) * 6 * (size_t)(3 * nt + 1));
    uint8_t* sel = (uint8_t*)calloc((size_t)(3 * nt + 1), 1);
    while (npend > 0 && rounds < max_rounds) {
        /* selection against the pending set at the start of the round */
        for (int64_t e = 0; e < 3 * nt; e++) {
            sel[e] = 0;
            if (!pend[e]) continue;
            const int64_t t = e / 3;
            const int s = (int)(e % 3);
            const int64_t a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
            const uint64_t pe = og_edge_priority((uint64_t)e);
            int best = 1;
            /* pending edges with an endpoint in the closed one-ring of a or b:
             * every such edge has an endpoint w in a triangle incident to a or b,
             * and is listed in a triangle incident to w */
            for (int side = 0; side < 2 && best; side++) {
                const int64_t v = side ? b : a;
                for (int64_t r = I.off[v]; r < I.off[v + 1] && best; r++) {
                    const int64_t t1 = I.tri[r];
                    for (int c = 0; c < 3 && best; c++) {
                        const int64_t w = tris[3 * t1 + c];
                        for (int64_t r2 = I.off[w]; r2 < I.off[w + 1] && best; r2++) {
                            const int64_t t2 = I.tri[r2];
                            for (int s2 = 0; s2 < 3; s2++) {
                                const int64_t f = 3 * t2 + s2;
                                if (f == e || !pend[f]) continue;
                                const uint64_t pf = og_edge_priority((uint64_t)f);
                                if (pf < pe || (pf == pe && f < e)) {
                                    best = 0;
                                    break;
                                }
                            }
                        }
                    }
                }
            }
            sel[e] = (uint8_t)best;
        }
        for (int64_t e = 0; e < 3 * nt; e++) {
            if (!sel[e]) continue;
            const int64_t t = e / 3;
            const int s = (int)(e % 3);
            const int64_t a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
            const int64_t p = tris[3 * t + (s + 2) % 3];
            const int64_t u = og_twin(&I, tris, a, b);
            const int64_t q = u >= 0 ? tris[3 * u + (og_slot(tris, u, b) + 2) % 3] : p;
            og_kuprat_move(verts, &I, tris, a, b, p, q, newpos + 6 * e, newpos + 6 * e + 3);
        }
        for (int64_t e = 0; e < 3 * nt; e++) {
            if (!sel[e]) continue;
            const int64_t t = e / 3;
            const int s = (int)(e % 3);
            const int64_t a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
            for (int d = 0; d < 3; d++) {
                verts[3 * a + d] = newpos[6 * e + d];
                verts[3 * b + d] = newpos[6 * e + 3 + d];
            }
            pend[e] = 0;
            npend--;
            total++;
        }
        rounds++;
    }
    free(sel);
    free(newpos);
    free(pend);
    og_inc_free(&I);
    free(gl);
    free(rough);
    free(r1);
    free(r2);
    free(rtt);
    free(G);
    free(V);
    if (moved) *moved = total;
    return rounds;
}
