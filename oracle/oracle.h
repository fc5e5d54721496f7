/*
 * oracle.h -- plain, slow FP64 CPU oracle for the front/fluid coupling of the
 * sharp front-tracking method (Gorges et al., arXiv 2505.06932).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The product
 * path (the CUDA library and its Python binding) never calls it, and it shares
 * no code, header or table with that path.
 *
 * Every array is a host array owned by the caller.  Grids are uniform and
 * cubic: cell (i,j,k) spans origin + h*[i,i+1] x h*[j,j+1] x h*[k,k+1] and has
 * key (i*n1 + j)*n2 + k.  Fronts are closed triangle meshes, counter-clockwise
 * seen from outside the enclosed (indicator = 1) region.
 *
 * Parity status of each function (what pins it) is listed in its comment.
 */
#ifndef FT_ORACLE_H
#define FT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n[3];
    int32_t pad;
    double origin[3];
    double h;
} og_grid;

typedef struct {
    double delta_h;      /* initial Wendland support / h            (Sec. 3.2: 2.5) */
    double delta_growth; /* support growth factor when too few fragments       */
    double delta_max_h;  /* largest support / h                                 */
    double sigma;        /* surface tension coefficient (Eq. csf)               */
    int32_t fit_min;     /* minimum number of non-zero weights (Sec. 3.2: 24)   */
    int32_t fit_ring;    /* 0: clipped fragments within delta (default);
                            k = 1..3: whole triangles of the k-ring of the
                            front vertex closest to the cell centre (Sec. 3.2) */
    double frame_angle;  /* test hook: rotate (t1,t2) about n by this angle     */
    int32_t frame_vertex;/* 0: n from the cell's fragment area vectors (default);
                            1: the normal of the closest front vertex (Sec. 3.2) */
    int32_t pad;
} og_params;

/* status bits */
#define OG_OUTSIDE_GRID 1u
#define OG_NOT_CLOSED 2u
#define OG_ORIENTATION 4u
#define OG_BAD_INDEX 8u

/* Bins (Sec. 3.2: "interfacial cells").  All (cell key, triangle) pairs whose
 * canonical clip is accepted, sorted by key then triangle.  Returns the pair
 * count P; writes at most `cap` pairs.  `margin` cells must separate every
 * candidate cell from the grid boundary, else the triangle is skipped and
 * OG_OUTSIDE_GRID is set.  Pinned by brute force, an independent separating-
 * axis overlap test and the area-partition identities. */
int64_t og_bin(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
               const og_grid* g, int32_t margin, int64_t cap, uint32_t* keys,
               int32_t* tri_ids, uint32_t* status);

/* Same predicate evaluated on every (triangle, cell) pair of the grid
 * (no candidate restriction).  Tiny inputs only. */
int64_t og_bin_bruteforce(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                          const og_grid* g, int64_t cap, uint32_t* keys, int32_t* tri_ids);

/* Canonical clip of one triangle against one cell: writes the fragment polygon
 * (up to 32 vertices, xyz) and returns its vertex count if accepted, else 0. */
int og_clip_fragment(const double* tri9, const og_grid* g, int32_t i, int32_t j, int32_t k,
                     double* poly_out);

/* Volume fraction alpha_C = (1/V_C) int_C I dx (Sec. 3.2), for every cell, by
 * integrating the front column by column (divergence theorem along z).  Cells
 * without front get the exact 0/1 value.  Pinned by the mesh volume, a plane
 * cut of one cube, convex clipping, winding numbers and translation. */
int og_alpha(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
             const og_grid* g, int32_t margin, double* alpha, uint32_t* status);

/* PPIC volume fit (Sec. 3.2, Eqs. volumefit, Wendland, volumefit2) in the
 * listed interfacial cells: curvature kappa (= div n, 2/R on a sphere), the
 * paraboloid normal at the cell's local origin, the coefficients a1..a6 (local
 * frame, lengths in units of h; may be NULL) and a status per cell
 * (bit0 support grown, bit1 singular -> plane fit, bit2 normal fallback),
 * and the frame (t1, t2, n) of each cell as 9 doubles (may be NULL).
 * Pinned by sphere convergence, planes, ellipsoids, frame invariance. */
int og_ppic(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
            const og_grid* g, const og_params* p, int64_t ncells, const uint32_t* cells,
            double* kappa, double* normal, double* coeffs, int8_t* fit_status, double* frame);

/* The front vertex closest to each cell centre (brute force over every vertex;
 * distance^2 rounded operation by operation, ties to the lowest index) and its
 * normal, the normalized sum of the area vectors (b - a) x (c - a) of its
 * triangles in ascending triangle order.  closest (ncells) and vnormal
 * (ncells x 3, may be NULL). */
void og_closest_vertex(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const og_grid* g,
                       int64_t ncells, const uint32_t* cells, int32_t* closest, double* vnormal);

/* The k-ring of triangles around vertex v (k >= 1): the triangles incident to
 * v, then repeatedly every triangle sharing a vertex with the previous ring;
 * ascending triangle ids into out (capacity cap).  Returns the count (which
 * may exceed cap; only cap are written). */
int64_t og_ring(int64_t nv, const int32_t* tris, int64_t nt, int64_t v, int32_t k, int32_t* out, int64_t cap);

/* CSF source S = sigma kappa grad(alpha) (Eq. csf) with the weighted curvature
 * smoothing of Sec. 3.3 in non-interfacial cells.  force is (3, n0*n1*n2). */
int og_csf(const og_grid* g, const double* alpha, int64_t ncells, const uint32_t* cells,
           const double* kappa, const double* normal, double sigma, double* force);

/* Balanced-force face term (Sec. 3.3, Eq. mwi_disc): F_d on the faces normal to
 * axis d (staggered layout of U, V, W), sigma kbar_f (alpha_Q - alpha_P)/h with
 * kbar_f the mean of the two cells' curvatures (own kappa in interfacial cells,
 * the smoothed kbar elsewhere; 0 outside the grid). */
int og_face_force(const og_grid* g, const double* alpha, int64_t ncells, const uint32_t* cells,
                  const double* kappa, const double* normal, double sigma, double* Fx, double* Fy, double* Fz);

/* Divergence-preserving interpolation of staggered face velocities to points
 * (Sec. 3.1).  U (n0+1,n1,n2), V (n0,n1+1,n2), W (n0,n1,n2+1); vel (np,3). */
void og_interp(const og_grid* g, const double* U, const double* V, const double* W,
               const double* pts, int64_t np, double* vel);

/* One classical RK4 step of dx/dt = u(x) (Sec. 3.1) in the interpolated velocity
 * of the fixed face field: out (np, 3) = new positions; vel (np, 3, may be NULL)
 * = k1, the velocity at the start. */
void og_advect_rk4(const og_grid* g, const double* U, const double* V, const double* W,
                   const double* pts, int64_t np, double dt, double* out, double* vel);

/* Local roughness (Sec. 3.4): per vertex the geometric Laplacian gl (nv, 3),
 * R^1, R^2, R = max(R^1, R^2) and the mean G and variance V of the edge
 * roughness 1 - n1.n2 of its edges; per triangle R_t (nt). */
int og_roughness(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double* gl, double* rough,
                 double* r1, double* r2, double* rt, double* G, double* V);

/* Local roughness smoothing (Sec. 3.4; Kuprat et al. 2001, Algorithm 4) in
 * rounds of independent edges; verts updated in place; returns the rounds. */
int og_roughness_smooth(double* verts, int64_t nv, const int32_t* tris, int64_t nt, double gl_thr, double r_thr,
                        int max_rounds, int64_t* moved);
uint64_t og_edge_priority(uint64_t e);

/* Helpers exposed for pin tests. */
/* The paper's own cut-cell quantities from a fitted paraboloid (Sec. 3.2):
 * frame = (t1, t2, n) as 9 doubles (rows, orthonormal), coeffs = a0..a5 of
 * z = P(x, y) in that frame, cell units (the cell is [-1/2, 1/2]^3).  Writes
 * alpha = V_P (volume below the paraboloid), area = surface area inside the
 * cell, kbar = area-averaged mean curvature, nbar = normalised
 * area-integrated normal; status 1 when the surface misses the cell (then kbar
 * and nbar are the point values at the frame origin).  Nested adaptive
 * quadrature of the definitions (paraboloid.c); pinned by plane and
 * whole-cell closed forms, the complement identity, cube symmetries and the
 * divergence identity. */
void og_paraboloid_cell(const double* frame, const double* coeffs, double* alpha, double* area, double* kbar,
                        double* nbar, int* status);
/* the same for m cells (frame m x 9, coeffs m x 6), threads over cells */
void og_paraboloid_cells(int64_t m, const double* frame, const double* coeffs, double* alpha, double* area,
                         double* kbar, double* nbar, int8_t* status);

void og_green_moments(const double* x, const double* y, int n, double* m6);
double og_signed_volume(const double* verts, const int32_t* tris, int64_t nt);
double og_wendland_weight(double q); /* Eq. Wendland with q = d/delta */
void og_set_threads(int nthreads);
int og_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
