/*
 * front.h -- C ABI of libfront.so, the GB300 (sm_103a) implementation of the
 * front/fluid coupling of sharp front tracking (Gorges, Evrard, Chiodi,
 * van Wachem, Denner; arXiv 2505.06932).
 *
 * Every time step a closed triangulated front is coupled to a uniform Cartesian
 * fluid mesh only in the interfacial cells, in five steps:
 *   front_bin              cells touched by each triangle           (Sec. 3.2)
 *   front_volume_fraction  alpha_C = (1/V_C) int_C I dx              (Sec. 3.2)
 *   front_curvature_ppic   PPIC volume fit -> curvature, normal      (Sec. 3.2,
 *                          Eqs. volumefit, Wendland, volumefit2)
 *   front_csf_force        S = sigma kappa grad alpha + smoothing    (Sec. 3.3,
 *                          Eq. csf)
 *   front_interp_velocity  divergence-preserving face -> vertex      (Sec. 3.1)
 *
 * Conventions (all calls):
 *   - Array arguments are CUDA device pointers owned by the caller; the library
 *     never frees or retains them beyond the call.  Host pointers are allowed
 *     only where a parameter says "host".
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  They return FT_OK or a negative FT_ERR_* code
 *     for errors detected on the host (bad arguments, allocation, launch).
 *   - Errors found on the device (capacity, front outside the grid margin, open
 *     or inverted front, bad vertex index, timeout) are OR-ed into the
 *     workspace's status word as FT_ST_* bits; ft_status() synchronizes the
 *     stream, returns them and clears the word.  Kernels never trap.
 *   - Cell (i,j,k) of grid g spans origin + h*[i,i+1] x h*[j,j+1] x h*[k,k+1];
 *     its key is (i*n1 + j)*n2 + k (k fastest).  Dense cell arrays are indexed
 *     by key.  Fronts are closed 2-manifold triangle meshes whose triangles are
 *     counter-clockwise seen from outside the region with indicator 1.
 *   - A workspace is tied to one grid shape and one device, and is not safe to
 *     use from two streams at once, with one exception: once front_bin (or
 *     front_bin_batch) has completed, front_volume_fraction(_batch) and
 *     front_curvature_ppic may run on two streams at the same time (they read
 *     the binned fragments and write disjoint state; the calls themselves come
 *     from one host thread); front_csf_force(_batch) must then wait for both.
 *     front_interp_velocity takes no workspace.
 */
#ifndef FRONT_H
#define FRONT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Uniform grid of n[0] x n[1] x n[2] cubic cells of edge h starting at origin. */
typedef struct {
    int32_t n[3];
    int32_t pad;
    double origin[3];
    double h;
} ft_grid;

/* Closed front: verts (nv, 3) float64 xyz, tris (nt, 3) int32 vertex indices. */
typedef struct {
    const double* verts;
    int64_t nv;
    const int32_t* tris;
    int64_t nt;
} ft_front;

/* Method parameters (Sec. 3.2 and 3.3). */
typedef struct {
    double delta_h;      /* initial Wendland support radius / h (paper: 2.5)     */
    double delta_growth; /* support growth factor while too few fragments (1.25) */
    double delta_max_h;  /* largest support radius / h (4.0; at most 7.0)        */
    double sigma;        /* surface tension coefficient of Eq. csf (1.0)         */
    int32_t fit_min;     /* minimum fragments with non-zero weight (paper: 24)   */
    int32_t precision;   /* FT_FP64 (plain) or FT_FP32C (FP32 + compensation)    */
    int32_t fit_ring;    /* PPIC fit elements: 0 (default) the clipped fragments
                            within delta of the cell centre; k = 1..3 the whole
                            triangles of the k-ring around the front vertex
                            closest to the cell centre (Sec. 3.2: k = 3)       */
    int32_t frame;       /* PPIC frame normal: FT_FRAME_FRAGMENTS (default) or
                            FT_FRAME_VERTEX, the normal of the closest front
                            vertex (Sec. 3.2)                                  */
} ft_params;

enum {
    FT_FRAME_FRAGMENTS = 0, /* normalized sum of the cell's fragment area vectors */
    FT_FRAME_VERTEX = 1     /* normalized sum of the area vectors of the triangles
                               at the front vertex closest to the cell centre */
};

/* Workspace capacities; 0 selects a default derived from max_nt. */
typedef struct {
    int64_t max_nt;    /* most triangles of one front                          */
    int64_t max_cand;  /* most (triangle, candidate cell) pairs (default 16*nt) */
    int64_t max_cells; /* most interfacial cells (default max_cand)            */
} ft_capacity;

typedef struct ft_workspace ft_workspace; /* opaque; owns library device memory */

enum {
    FT_FP64 = 0,
    FT_FP32C = 1
};

enum {
    FT_OK = 0,
    FT_ERR_ARG = -1,          /* null pointer, bad size, grid mismatch          */
    FT_ERR_ALLOC = -2,        /* cudaMalloc failed                               */
    FT_ERR_CAPACITY = -3,     /* a capacity was exceeded (see ft_counts)         */
    FT_ERR_OUTSIDE_GRID = -4, /* front not inside the grid margin                */
    FT_ERR_NOT_CLOSED = -5,   /* column parity residue > 1e-9: front not closed  */
    FT_ERR_ORIENTATION = -6,  /* inverted front (negative enclosed volume)       */
    FT_ERR_TIMEOUT = -7,      /* a bounded device wait gave up                   */
    FT_ERR_CUDA = -8,         /* CUDA runtime error                              */
    FT_ERR_STATE = -9         /* call order violated (e.g. no front_bin yet)     */
};

/* device status bits (ft_status) */
#define FT_ST_CAPACITY 0x01u
#define FT_ST_OUTSIDE_GRID 0x02u
#define FT_ST_NOT_CLOSED 0x04u
#define FT_ST_ORIENTATION 0x08u
#define FT_ST_BAD_INDEX 0x10u
#define FT_ST_TIMEOUT 0x20u

/* per-cell fit_status bits of front_curvature_ppic */
#define FT_FIT_GROWN 0x1     /* support radius was grown beyond delta_h          */
#define FT_FIT_SINGULAR 0x2  /* normal equations singular: plane fit, kappa = 0  */

/* per-cell status of the paraboloid cut-cell calls */
#define FT_PARAB_MISS 0x1    /* the surface misses the cell: kappa and normal are
                                the point values at the frame origin, area 0    */
#define FT_FIT_NORMAL 0x4    /* opposing sheets: normal of the largest fragment  */

/* Create a workspace for grid *g on CUDA device `device`; *bytes (host, may be
 * NULL) receives the device memory it holds.  The front must keep
 * 2 + ceil(delta_max_h) cells from every grid face. */
int ft_workspace_create(ft_workspace** ws, const ft_grid* g, const ft_capacity* cap, int device,
                        size_t* bytes);
int ft_workspace_destroy(ft_workspace* ws);

/* Synchronize `stream`, write the accumulated FT_ST_* bits to *bits (host) and
 * clear them. */
int ft_status(ft_workspace* ws, void* stream, uint32_t* bits);

/* Synchronize `stream` and write 5 host int64: interfacial cells M, binned
 * (cell, triangle) pairs P, candidate pairs used, candidate pairs needed, and
 * the (cell, fragment) pairs inside the support of the last PPIC call. */
int ft_counts(ft_workspace* ws, void* stream, int64_t* out5);

/* Synchronize `stream` and write the first n (at most FT_WORK_COUNTS) of:
 * triangles T of the last binning, interfacial cells M, binned pairs P,
 * candidate pairs used and needed, (cell, fragment) pairs in the support of
 * the last PPIC call, pairs of the last FP32-form binning that the binary64
 * canonical clip decided (near-degenerate pairs; 0 in the FP64 path), and the
 * non-interfacial cells of the last CSF call's ring (host int64).  The work
 * counts behind the per-kernel roofline figures. */
#define FT_WORK_COUNTS 8
int ft_work_counts(ft_workspace* ws, void* stream, int64_t* out, int32_t n);

const char* ft_status_string(int code);

/* Copy the sorted (cell key, triangle) pairs of the last front_bin into
 * keys (uint32) and tris (int32), both of length >= cap (device pointers);
 * pairs beyond cap are dropped (FT_ST_CAPACITY).  For inspection and tests. */
int ft_bin_pairs(ft_workspace* ws, int64_t cap, uint32_t* keys, int32_t* tris, void* stream);

/* (a1) Bin the front (Sec. 3.2, interfacial cells).  For every triangle, every
 * cell whose closed box meets the triangle's bounding box is clipped against
 * the triangle (Sutherland-Hodgman, planes x>=X_i, x<=X_i+1, y.., z..; crossing
 * points prev + t (cur - prev) with t = (X - prev)/(cur - prev), all in IEEE
 * binary64 without contraction); the cell keeps the triangle iff every stage
 * leaves >= 3 vertices, the fan area vector is not zero, and the fragment does
 * not lie entirely in one of the cell's upper faces.  The kept (cell, triangle)
 * pairs are put in cell-key order (triangles ascending within a cell); their
 * fragment moments are kept in the workspace for the next steps.  Requires
 * f->nt <= capacity.max_nt.  p->delta_max_h sets the grid margin. */
int front_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, void* stream);

/* (a2) Volume fraction (Sec. 3.2) of every cell into alpha (n0*n1*n2 float64,
 * by key).  Interfacial cells: (1/h^3)[ int_{front in C} (z - Z_k) n_z dA
 * + h int_{front above C in its column} n_z dA ]; other cells: the rounded
 * column parity, exactly 0 or 1 (FT_ST_NOT_CLOSED if the residue > 1e-9).
 * Results are clamped to [0,1].  Needs front_bin on this workspace. */
int front_volume_fraction(ft_workspace* ws, double* alpha, void* stream);

/* (a3) PPIC curvature (Sec. 3.2) in every interfacial cell, in ascending key
 * order: cell_keys (M uint32), kappa (M float64, kappa = div n > 0 on a sphere,
 * 2/R), normal (M x 3 float64, paraboloid normal at the local origin), coeffs
 * (M x 6 float64, a1..a6 in the local frame with lengths in units of h; may be
 * NULL) and fit_status (M int8, FT_FIT_* bits).  Local frame: n = normalized
 * sum of the cell's fragment area vectors, (t1,t2) completing it (Duff et al.
 * 2017); fit data: fragments of cells within ceil(delta - 1/2) cells whose area
 * centroid lies closer than delta to the cell centre, Wendland weights, volume
 * fit normal equations solved in float64.  `cap` is the length of the output
 * arrays; M > cap sets FT_ST_CAPACITY and writes nothing.  Needs front_bin.
 * The paper's own neighbourhood and frame (p->fit_ring > 0 and/or p->frame =
 * FT_FRAME_VERTEX; one-front workspaces only, else FT_ERR_ARG): the closest
 * front vertex to a cell centre is the argmin of |x - x_c|^2 (each operation
 * rounded, ties to the lowest vertex index) over the vertices of the front's
 * triangles, x_c =
 * origin + (i + 1/2) h per axis; its normal is the normalized sum of the area
 * vectors (b - a) x (c - a) of its triangles; the k-ring is its triangles, then
 * k - 1 times every triangle sharing a vertex with the ring; each ring
 * triangle enters the fit whole, its Wendland distance taken from its centre
 * (vertex mean), the support growing while fewer than fit_min triangles lie
 * inside it.  The ring fit runs in float64 in both precisions (at most 512
 * ring triangles per cell, else FT_ST_CAPACITY).  These variants read the
 * vertices and triangles passed to the last front_bin (keep them alive and
 * unchanged), and the first such call on a workspace, or one with a larger
 * front, allocates device memory for the mesh incidence: make it before any
 * stream capture. */
int front_curvature_ppic(ft_workspace* ws, const ft_params* p, int64_t cap, uint32_t* cell_keys,
                         double* kappa, double* normal, double* coeffs, int8_t* fit_status,
                         void* stream);

/* (a4) CSF source (Eq. csf, Sec. 3.3) into force (3 x n0*n1*n2 float64, SoA):
 * S_P = sigma kappa_P grad alpha_P, grad by central differences with alpha = 0
 * outside the grid; kappa_P is the cell's own curvature in interfacial cells
 * and, elsewhere, sum_Q kappa_Q w_Q / sum_Q w_Q over interfacial Q among the 26
 * neighbours with w_Q = |s_Q . n_Q| / |s_Q|.  kappa and normal are the M-long
 * outputs of front_curvature_ppic for the same bins. */
int front_csf_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                    const double* normal, double* force, void* stream);

/* (a4, split) front_csf_force as three calls, so that its parts that need
 * neither kappa nor alpha can run earlier in the step, off the chain of calls
 * that the force waits for.  The force of Eq. csf is non-zero only in the
 * interfacial cells and their face neighbours (Sec. 3.3: the gradient of alpha
 * vanishes between full or empty cells); the non-interfacial ones among those
 * neighbours are the "ring" cells, whose curvature is the smoothed one.
 *   front_force_clear sets force (3 x n0*n1*n2 float64, device, caller-owned)
 *     to zero; it needs no binning (so it can run beside front_bin).
 *   front_csf_prepare lists the ring cells of the last front_bin (or
 *     front_bin_batch) in the workspace; it needs only the binning (so it can
 *     run beside front_curvature_ppic).  One-front and batch workspaces.
 *   front_csf_force_cells writes S_P of front_csf_force in the interfacial and
 *     ring cells and leaves every other cell of force as it is; it reads the
 *     list of the last front_csf_prepare, which must have been issued after the
 *     last front_bin (else FT_ERR_STATE).
 * After front_force_clear and front_csf_prepare (ordered before the cells call
 * on one stream or by events), force holds exactly what front_csf_force
 * writes.  Arguments and errors as for front_csf_force; front_force_clear and
 * front_csf_force_cells give FT_ERR_ARG on a batch workspace. */
int front_force_clear(ft_workspace* ws, double* force, void* stream);
int front_csf_prepare(ft_workspace* ws, void* stream);
int front_csf_force_cells(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                          const double* normal, double* force, void* stream);

/* (a4, compact) The CSF source of front_csf_force written only where it can be
 * non-zero (the interfacial cells and their face neighbours, Sec. 3.3): per
 * slot a cell key (keys, uint32) and its force (force, 3 float64: x, y, z).
 * Slots [0, M) are the interfacial cells in the order of front_curvature_ppic;
 * slots [M, *count) the other cells with a non-zero gradient, in unspecified
 * order.  *count (device int64) receives the slot count; slots at or beyond
 * `cap` are not written and set FT_ST_CAPACITY.  Every cell not listed has a
 * zero force.  One-front workspaces only.  No dense array is written (or
 * cleared): the form for callers that move the force off the device. */
int front_csf_force_compact(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                            const double* normal, int64_t cap, uint32_t* keys, double* force, int64_t* count,
                            void* stream);

/* (a2, compact) The volume fraction of front_volume_fraction in two parts:
 * full_bits (device, ceil(n0*n1*n2 / 32) uint32) with bit q % 32 of word q / 32
 * set iff alpha[q] > 1/2 (the exact value of every non-interfacial cell, which
 * is 0 or 1), and alpha_cells (device, M float64) the values at the interfacial
 * cells in the order of front_curvature_ppic (M > cap sets FT_ST_CAPACITY and
 * writes no values).  alpha is the array front_volume_fraction wrote. */
int front_alpha_pack(ft_workspace* ws, const double* alpha, int64_t cap, uint32_t* full_bits, double* alpha_cells,
                     void* stream);

/* Balanced-force face term of the surface tension (Sec. 3.3, Eq. mwi_disc: the
 * term that enters the face fluxes of the pressure-velocity coupling): on the
 * face between cells P and Q = P + e_d, sigma kbar_f (alpha_Q - alpha_P) / h with
 * kbar_f = (kappa_P + kappa_Q) / 2, each cell's curvature being its own kappa if
 * it is interfacial and otherwise the smoothed kbar of front_csf_force (0 if it
 * has no interfacial neighbour); alpha and kappa are 0 outside the grid.  Output
 * fx (n0+1,n1,n2), fy (n0,n1+1,n2), fz (n0,n1,n2+1) float64, face index i along d
 * being the face between cells i-1 and i.  kappa and normal as for
 * front_csf_force. */
int front_face_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                     const double* normal, double* fx, double* fy, double* fz, void* stream);

/* The paper's own indicator and interface properties from the fitted
 * paraboloids (Sec. 3.2, the paragraph after Eq. volumefit2), for m cells
 * given directly.  frame: m x 9 float64, the rows t1, t2, n of an orthonormal
 * frame whose origin is the cell centre; coeffs: m x 6 float64, a1..a6 of
 * z = P(x, y) = a1 + a2 x + a3 y + a4 x^2 + a5 x y + a6 y^2 in that frame,
 * lengths in cell widths (the cell is [-1/2, 1/2]^3).  Outputs per cell:
 * alpha (m float64) = V_P / V_C, the fraction of the cell below the surface
 * (z < P, the side n points away from), clamped to [0, 1]; area (m float64,
 * cell widths squared) of the surface inside the cell; kappa (m float64, per
 * cell width) = the mean curvature (div n, > 0 on a sphere) averaged over that
 * surface; normal (m x 3 float64) = the normalised integral of the upward
 * surface normal over it; status (m int8, FT_PARAB_* bits).  area, kappa,
 * normal and status may be NULL.  The integrals are evaluated to float64
 * rounding by graded Gauss-Legendre quadrature (the paper uses the closed
 * forms of Evrard et al. 2023). */
int front_paraboloid_cells(const double* frame, const double* coeffs, int64_t m, double* alpha, double* area,
                           double* kappa, double* normal, int8_t* status, void* stream);

/* The frames (t1, t2, n) of the interfacial cells of the last
 * front_curvature_ppic call on ws, as m x 9 float64 in its cell order (the
 * frame in which its coeffs are given).  `cap` as for that call. */
int front_ppic_frame(ft_workspace* ws, int64_t cap, double* frame, void* stream);

/* The paper's indicator in the cut cells (Sec. 3.2): after front_volume_fraction
 * and front_curvature_ppic (with coeffs) on ws, replaces alpha at every
 * interfacial cell by V_P / V_C of that cell's fitted paraboloid (full and
 * empty cells keep their column-parity value, the paper's flood fill), and
 * writes per interfacial cell, in the order of front_curvature_ppic, the
 * surface-averaged kappa (1/length), normal and area (length^2) and the status
 * as for front_paraboloid_cells (each may be NULL).  coeffs is the array that
 * front_curvature_ppic wrote; `cap` is the length of the per-cell arrays
 * (M > cap sets FT_ST_CAPACITY and writes nothing).  FT_ERR_STATE unless a
 * fit ran since the last front_bin. */
int front_volume_fraction_ppic(ft_workspace* ws, const double* coeffs, int64_t cap, double* alpha, double* kappa,
                               double* normal, double* area, int8_t* status, void* stream);

/* (a5) Divergence-preserving velocity interpolation (Sec. 3.1) of the staggered
 * face velocities U (n0+1,n1,n2), V (n0,n1+1,n2), W (n0,n1,n2+1) to the nv
 * points verts (nv x 3) into vel (nv x 3).  The cell is floor((x - origin)/h)
 * clamped to the grid; transverse face gradients are central differences,
 * one-sided on the first and last face rows.  Needs no workspace.
 * U, V and W may be device arrays or page-locked host memory mapped into the
 * device's address space (cudaHostAlloc or cudaHostRegister; with unified
 * addressing the host pointer is the device pointer): the kernel then reads
 * in place only the face values around the points (at most 54 per point; on
 * GB300 over NVLink-C2C), so a caller whose face field lives on the host need
 * not copy the whole field.  The result is the same bit for bit.  verts and vel
 * are device arrays. */
int front_interp_velocity(const ft_grid* g, const double* U, const double* V, const double* W,
                          const double* verts, int64_t nv, double* vel, void* stream);

/* Front advection (Sec. 3.1): one classical fourth-order Runge-Kutta step of
 * dx/dt = u(x) for the nv points verts, u the interpolated velocity of
 * front_interp_velocity with the face field U, V, W held fixed during the step:
 * k1 = u(x), k2 = u(x + dt/2 k1), k3 = u(x + dt/2 k2), k4 = u(x + dt k3),
 * verts_out = x + dt/6 (k1 + 2 k2 + 2 k3 + k4).  verts_out (nv x 3) may be verts
 * itself (each point's stages read only that point); vel (nv x 3, may be NULL)
 * receives k1.  Points must stay inside the grid. */
int front_advect_rk4(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                     int64_t nv, double dt, double* verts_out, double* vel, void* stream);

/* Allocation-free volume fraction (no counterpart in the paper).
 *
 * Some callers cannot allocate device memory while they run: a flow solver
 * that owns all GPU memory through its own pool and fixes its budget before
 * time stepping, a process under a hard per-process memory limit, or a time
 * loop that cannot afford cudaMalloc's implicit device-wide synchronization.
 * For them this call bins the front and writes its volume fraction (the same
 * result as front_bin followed by front_volume_fraction) using only scratch
 * that the library holds in one static device array of
 * FT_NOALLOC_SCRATCH_BYTES, reserved on every device that loads the library
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Arguments: grid g and front f as for front_bin (device verts/tris), method
 * parameters p (delta_max_h sets the grid margin; p->precision is ignored: the
 * scratch holds float64 fragment records only, so this call always computes
 * the plain float64 path), alpha (device, n0*n1*n2 float64, by key) and status
 * (device, one uint32 that receives the FT_ST_* bits of this call).  Runs on the current device and `stream`.
 * Limits: n0*n1*n2 <= FT_NOALLOC_MAX_GRID_CELLS and nt <= FT_NOALLOC_MAX_TRIANGLES,
 * else FT_ERR_CAPACITY is returned before any work; more than
 * FT_NOALLOC_MAX_CANDIDATES (triangle, candidate cell) pairs or interfacial
 * cells sets FT_ST_CAPACITY in *status and alpha is not valid.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  Every call shares
 * the one array and resets the parts that must start cleared, so calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller. */
#define FT_NOALLOC_SCRATCH_BYTES 8388608
#define FT_NOALLOC_MAX_GRID_CELLS 262144
#define FT_NOALLOC_MAX_TRIANGLES 16384
#define FT_NOALLOC_MAX_CANDIDATES 32768
int ft_volume_fraction_noalloc(const ft_grid* g, const ft_front* f, const ft_params* p, double* alpha,
                               uint32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * Batched form (no counterpart in the paper, which couples one front per
 * simulation).  Many independent fronts, each with its own grid, run through
 * one launch sequence: their cells share one batch-global key space (front b's
 * cell with local key q has key key_base[b] + q, key_base[b] = sum of the
 * earlier fronts' n0*n1*n2), one pair placement and one interfacial-cell worklist,
 * so small fronts do not each pay a launch sequence.  Every front's results are
 * bit for bit those of the one-front calls on that front alone (each cell's
 * sums run over the same fragments in the same order).  Errors of one front (outside
 * the grid, bad index, not closed, inverted) skip or flag that front only and
 * are reported per front by ft_batch_status; capacity errors concern the batch.
 * --------------------------------------------------------------------------- */

/* One front of a batch: its grid and its device arrays, owned by the caller and
 * kept alive while the table is in use.  alpha (n0*n1*n2 float64) is written by
 * front_volume_fraction_batch and read by front_csf_force_batch; force
 * (3 x n0*n1*n2 SoA) is written by front_csf_force_batch; U, V, W (faces as in
 * front_interp_velocity) are read and vel (nv x 3) written by
 * front_interp_velocity_batch and front_advect_rk4_batch, which writes the
 * advected positions to verts_next.  Pointers of steps that are not called may
 * be NULL. */
typedef struct {
    ft_grid grid;
    const double* verts;
    int64_t nv;
    const int32_t* tris; /* indices into this front's verts */
    int64_t nt;
    double* alpha;
    double* force;
    const double* U;
    const double* V;
    const double* W;
    double* vel;
    double* verts_next; /* front_advect_rk4_batch output positions (may equal verts) */
    double dt;          /* front_advect_rk4_batch time step of this front            */
    double* face_force[3]; /* front_face_force_batch output, staggered like U, V, W  */
} ft_batch_front;

/* Capacities of a batch workspace; 0 selects the default of ft_capacity. */
typedef struct {
    int32_t max_fronts;     /* fronts in one table                                 */
    int32_t pad;
    int64_t max_grid_cells; /* sum of n0*n1*n2 over the table (< 2^32 - 1)          */
    int64_t max_nt;         /* sum of triangles over the table                      */
    int64_t max_cand;       /* (triangle, candidate cell) pairs (default 16*max_nt) */
    int64_t max_cells;      /* interfacial cells (default max_cand)                 */
} ft_batch_capacity;

/* Create a batch workspace on `device`; *bytes (host, may be NULL) receives the
 * device memory it holds (the index map takes 4 B per grid cell). */
int ft_batch_workspace_create(ft_workspace** ws, const ft_batch_capacity* cap, int device, size_t* bytes);

/* Install the table of nf fronts (host array) on the workspace: copies the
 * descriptors to the device on `stream` and synchronizes it.  Returns
 * FT_ERR_CAPACITY if the table exceeds the workspace.  Not capturable in a CUDA
 * graph; graphs captured earlier keep the previous table's launch sizes and
 * must be captured again. */
int ft_batch_set(ft_workspace* ws, int32_t nf, const ft_batch_front* fronts, void* stream);

/* (a1) front_bin over every front of the table; cell keys are batch-global. */
int front_bin_batch(ft_workspace* ws, const ft_params* p, void* stream);

/* (a2) front_volume_fraction of every front into its own alpha array. */
int front_volume_fraction_batch(ft_workspace* ws, void* stream);

/* (a3) is front_curvature_ppic itself: on a batch workspace its M outputs cover
 * every front in ascending batch-global key order, so front b's cells are the
 * rows [off[b], off[b+1]) given by ft_batch_cell_ranges. */

/* (a4) front_csf_force of every front from its alpha into its force. */
int front_csf_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                          void* stream);

/* (a4, split) front_force_clear and front_csf_force_cells of every front of
 * the table (the table's force arrays; FT_ERR_STATE before ft_batch_set, and
 * for the cells call without a front_csf_prepare after the last
 * front_bin_batch). */
int front_force_clear_batch(ft_workspace* ws, void* stream);
int front_csf_force_cells_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                                void* stream);

/* front_face_force of every front, from its alpha into its face_force arrays. */
int front_face_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                           void* stream);

/* front_volume_fraction_ppic of every front: alpha_P into each front's alpha
 * at its interfacial cells; per-cell outputs in the batch's cell order. */
int front_volume_fraction_ppic_batch(ft_workspace* ws, const double* coeffs, int64_t cap, double* kappa,
                                     double* normal, double* area, int8_t* status, void* stream);

/* (a5) front_interp_velocity of every front (its U, V, W, verts -> vel). */
int front_interp_velocity_batch(ft_workspace* ws, void* stream);

/* Front advection of every front of the table: front_advect_rk4 with its
 * verts, U, V, W and dt into verts_next (vel, if not NULL, receives k1). */
int front_advect_rk4_batch(ft_workspace* ws, void* stream);

/* off (device, nf + 1 int64): first row of each front in the outputs of
 * front_curvature_ppic; off[nf] = M.  Needs front_bin_batch. */
int ft_batch_cell_ranges(ft_workspace* ws, int64_t* off, void* stream);

/* Synchronize `stream`, write the FT_ST_* bits of each front (host, nf
 * uint32) and clear them (the workspace-wide word of ft_status is separate). */
int ft_batch_status(ft_workspace* ws, void* stream, uint32_t* bits);

/* ---------------------------------------------------------------------------
 * Launch tuning (no counterpart in the paper).  The grid sizes of the kernels
 * whose work is distributed over a grid-stride or work-counter loop (any value
 * from 1 to 32), the register/occupancy variant and the cell schedule of the
 * PPIC accumulation; every choice gives the same results.  ft_autotune picks
 * them by timing.
 * --------------------------------------------------------------------------- */
typedef struct {
    int32_t clip_blocks_per_sm; /* canonical clip (front_bin), default 3            */
    int32_t ppic_blocks_per_sm; /* PPIC accumulation, default 4                      */
    int32_t csf_blocks_per_sm;  /* force clear (batch) and face force, default 16     */
    int32_t fill_blocks_per_sm; /* column parity fill, default 8                     */
    int32_t ppic_min_blocks;    /* FP32 PPIC accumulation compiled for 4 (default) or
                                   6 resident blocks per SM (fewer registers each)   */
    int32_t ppic_dynamic;       /* PPIC cells from a global work counter (1) or
                                   interleaved over the warps (0, default)           */
    int32_t sort_blocks;        /* segments of the binning's scans: the triangle counts
                                   (one block each) and the key range (four blocks
                                   each); 1 to the SM count, 0: the SM count
                                   (default)                                         */
    int32_t pad;
    /* outputs of ft_autotune: what the tuned workload needed, for sizing a
     * workspace (ft_capacity / ft_batch_capacity) to it */
    int64_t cand_need;
    int64_t cells_need;
    int64_t fit_pairs;
    double step_ms;             /* bin + alpha + PPIC + CSF time with the result  */
} ft_tuning;

int ft_set_tuning(ft_workspace* ws, const ft_tuning* t);
int ft_get_tuning(ft_workspace* ws, ft_tuning* t);

/* Time bin + volume fraction + PPIC + CSF on this workspace for a set of launch
 * shapes (coordinate by coordinate, `reps` timed runs each after one warm-up,
 * median time) and install the fastest; *best (host) receives it.  f is the
 * front for a one-front workspace and NULL for a batch workspace (the table's
 * alpha and force arrays are overwritten).  Allocates and frees temporary
 * device memory for the outputs and synchronizes `stream`: call it at set-up,
 * not inside a capture. */
int ft_autotune(ft_workspace* ws, const ft_front* f, const ft_params* p, int32_t reps, ft_tuning* best,
                void* stream);

/* ---------------------------------------------------------------------------
 * Local roughness detection and smoothing of the front mesh (Sec. 3.4).  The
 * front is a closed, consistently oriented triangle mesh (as everywhere here).
 * A roughness workspace holds the mesh adjacency built on the device.
 * --------------------------------------------------------------------------- */
typedef struct ft_rough ft_rough;

int ft_rough_create(ft_rough** r, int64_t max_nv, int64_t max_nt, int device, size_t* bytes);
int ft_rough_destroy(ft_rough* r);

/* Synchronize `stream`, return the FT_ST_* bits of the last call (capacity:
 * a two-ring neighbourhood of more than 512 triangles) and clear them. */
int ft_rough_status(ft_rough* r, void* stream, uint32_t* bits);

/* Roughness metrics of the front verts (nv x 3) / tris (nt x 3), device arrays:
 * gl (nv x 3) the geometric Laplacian x_i - sum_j w_ij x_j / sum_j w_ij over the
 * one-ring, w_ij = 1/|x_i - x_j| (Karni and Gotsman 2000); for every edge the
 * roughness R_e = 1 - n_1 . n_2 of its two triangles; G, V (nv; may be NULL) the
 * mean and variance of R_e over the edges of each vertex; rt (nt; may be NULL)
 * the triangle roughness sum G_i V_i / sum V_i over its vertices (the mean G_i
 * when every V_i is 0) (Corsini et al. 2007); r1, r2 (nv; may be NULL) the
 * vertex roughness (1/|N|) sum A_t R_t over the triangles of its one- and
 * two-ring neighbourhood; rough (nv) = max(r1, r2).  Synchronizes `stream` once
 * (index check); FT_ERR_ARG for a vertex index out of range. */
int front_roughness(ft_rough* r, const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double* gl,
                    double* rough, double* r1, double* r2, double* rt, double* G, double* V, void* stream);

/* Local roughness smoothing (Sec. 3.4): a vertex is rough when |gl| > gl_thr and
 * rough > r_thr (the paper sets both at 1.2 to 1.5 times their maximum on the
 * initial front); every edge with a rough endpoint gets the volume-conserving
 * move of Kuprat et al. (2001, Algorithm 4): simultaneous Laplacian smoothing of
 * both endpoints, then a common shift h n with 6 dV = d_a.A_a + d_b.A_b +
 * d_a.(d_b x y) = 0 (A_i = sum of x_j x x_k over the triangles (i, j, k) at i,
 * y = x_p - x_q for the triangles (a, b, p) and (b, a, q) of the edge), n along
 * the gradient of that volume change so that |h n| is minimal.  Edges move in
 * rounds; in a round, an edge moves when its priority (the SplitMix64 finalizer
 * of its id 3 t + s, the triangle t and slot s where it runs a -> b with a < b)
 * is the smallest among the pending edges touching the closed one-rings of its
 * endpoints, so the moves of a round touch disjoint stars and each keeps the
 * enclosed volume.  verts is updated in place; *rounds, *moved and *status
 * (host; may be NULL) receive the rounds run (at most max_rounds), the edges
 * moved and the FT_ST_* bits.  Synchronizes `stream` once per round. */
int front_roughness_smooth(ft_rough* r, double* verts, int64_t nv, const int32_t* tris, int64_t nt, double gl_thr,
                           double r_thr, int32_t max_rounds, int32_t* rounds, int64_t* moved, uint32_t* status,
                           void* stream);

/* Number of kernels this library has launched since it was loaded (all
 * devices, all workspaces). */
int64_t ft_launch_count(void);

/* Per-kernel timing (no counterpart in the paper).  ft_trace_start creates
 * `capacity` pairs of CUDA events on the current device and opens a trace:
 * from then on every launch of the five steps' kernels that is not made during
 * stream capture is bracketed by an event pair recorded on its own stream
 * (launches beyond `capacity` are counted as dropped).  ft_trace_stop waits
 * for the recorded events, closes the trace, frees the events and writes, per
 * distinct kernel in order of first launch, its name (host, max_kernels rows
 * of FT_TRACE_NAME chars, NUL-terminated), its launch count (host int64) and
 * its summed device time in milliseconds (host double); *n_kernels (host)
 * receives the number of rows and *dropped (host, may be NULL) the launches
 * not traced.  FT_ERR_STATE if no trace is open (or one is already open for
 * start); FT_ERR_CAPACITY if more than max_kernels distinct kernels ran (the
 * first max_kernels are written).  The events add a few microseconds between
 * launches: trace eager steps, never the timed graph replays. */
#define FT_TRACE_NAME 48
int ft_trace_start(int64_t capacity);
int ft_trace_stop(int32_t max_kernels, char* names, int64_t* launches, double* total_ms, int32_t* n_kernels,
                  int64_t* dropped);

/* Throughput probe (no counterpart in the paper): runs dependent FMA chains on
 * every SM (kind 0: float64, 1: float32) and writes the achieved FLOP/s
 * (host *flops); used to state the ALU roofline of the kernels above. */
int ft_probe_fma_rate(int kind, int device, double* flops);

#ifdef __cplusplus
}
#endif
#endif
