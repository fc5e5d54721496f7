// ft_internal.cuh -- internal declarations of libfront.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "front.h"

#define FT_WARP 32
#define FT_SENTINEL 0xffffffffu

// Device-side counters of one workspace.
struct ft_counters {
    unsigned int status;   // FT_ST_* bits
    unsigned int pad;
    long long T;           // triangles of the last front_bin
    long long C_need;      // candidate pairs needed
    long long C;           // candidate pairs used (0 if C_need > capacity)
    long long P;           // binned pairs
    long long M;           // interfacial cells (also: entries set in the index map)
    long long fit_pairs;   // (cell, fragment) pairs inside the support, last PPIC
    long long work;        // next cell of the dynamically scheduled PPIC accumulation
    long long big;         // cells with more than 32 pairs (worklist of the per-cell ordering)
    long long clip_f64;    // FP32 clip: pairs listed for the binary64 clip (k_clip_list), last front_bin
    unsigned long long lmax2_bits;  // longest triangle edge squared (float64 bits), paper-neighbourhood fit
};

// Fragment record (cell-local, lengths in units of h, relative to the centre of
// the fragment's own cell): area vector AN = A n_f, area centroid c and central
// second moment per unit area K = (1/A) int (x-c)(x-c)^T dA (xx,yy,zz,xy,xz,yz).
struct __align__(16) ft_frag {
    double an[3];
    double c[3];
    double k[6];
};

// The same record in float32 (the FP32-compensated form), 48 B.
struct __align__(16) ft_frag32 {
    float an[3];
    float c[3];
    float k[6];
};

// Per interfacial cell, the volume-fit normal equations left by the
// accumulation kernel for the solve kernel: packed upper triangle of the 6x6
// matrix (21), right-hand side (6), frame normal (3) and the height shift z0 of
// the fitted heights -- as doubles (FP64) or as hi/lo float pairs (FP32 form).
struct __align__(16) ft_cellsys {
    double v[32];
};

// One front of a batch as the kernels see it: its grid and its caller-owned
// device arrays (see ft_batch_front in front.h).  128 B.
struct __align__(16) ft_fdesc {
    ft_grid g;
    const double* verts;
    const int* tris;
    double* alpha;
    double* force;
    const double* U;
    const double* V;
    const double* W;
    double* vel;
    double* verts_next;  // RK4 output positions (may equal verts)
    double* fface[3];    // balanced-force face term, staggered like U, V, W
    double dt;           // RK4 time step
    long long nv;
    long long nt;
    // grid plane coordinates X_i = origin + i h (i = 0..n0, then Y, then Z),
    // computed once with the canonical operations; NULL: computed on the fly
    const double* planes;
    double inv_h;  // 1 / h (moments and interpolation weights; never in the predicate)
};

// Launch-shape parameters (see ft_tuning in front.h).
struct ft_tune {
    int clip_bps;   // k_clip blocks per SM
    int ppic_bps;   // k_ppic_acc blocks per SM
    int csf_bps;    // k_zero_force / k_face_force blocks per SM
    int fill_bps;   // k_alpha_fill blocks per SM
    int ppic_min_blocks;  // FP32 k_ppic_acc compiled for 4 (more registers) or 6 resident blocks per SM
    int ppic_dynamic;     // k_ppic_acc cells from a global work counter (1) or interleaved (0)
    int seg_blocks;       // segments of the binning's scans (key range: four blocks each), <= grid_blocks
};

struct ft_workspace {
    int device;
    int sm_count;
    int grid_blocks;       // blocks of the segmented scan/sort kernels
    ft_grid g;
    long long ncells;
    long long max_nt, max_cand, max_cells;
    size_t bytes;
    bool binned;
    bool fitted;           // front_curvature_ppic ran since the last bin
    int last_precision;
    bool sys_fp32;         // the last PPIC call left its normal equations as float pairs
    bool clip32_ok;        // every grid keeps |coordinate| / h within the float32 clip's bounds
    // binnings issued on this workspace, and the binning the ring list of
    // front_csf_prepare belongs to (host-side order of the calls)
    unsigned long long bin_epoch, ring_epoch;

    ft_counters* ctr;
    int* idx_map;          // ncells: interfacial index or -1
    int* tri_cnt;          // max_nt
    int* tri_off;          // max_nt
    int* tri_box;          // max_nt * 8: lo[3], ext[3], front, 0
    double* tri_nrm;       // max_nt * 4: normal direction of each triangle (x, y, z, 0)
    float* tri32;          // max_nt * 32 (or null): the FP32 clip's triangle record (k_bin.cu, Tri32)
    double* planes;        // grid plane coordinates of every front (see ft_fdesc)
    long long planes_cap;  // entries allocated in planes
    int* cand_tri;         // max_cand
    unsigned* keys[2];     // max_cand
    unsigned* vals[2];     // max_cand
    ft_frag* rec;          // max_cand (FP64 records)
    ft_frag32* rec32;      // max_cand (FP32 records)
    float4* cen32;         // max_cand: float copy of the FP64 centroids (support filter)
    ft_frag* srec;         // max_cand: FP64 records in sorted pair order
    ft_frag32* srec32;     // max_cand: FP32 records in sorted pair order
    float4* scen;          // max_cand: float centroids in sorted pair order (support filter)
    ft_cellsys* sys;       // max_cells: normal equations per cell
    int* fit_info;         // max_cells x 2: fragments in support, status bits
    unsigned* cells;       // max_cells + 1
    int* cell_off;         // max_cells + 1
    int* cell_cnt;         // index-map entries: kept pairs per cell key while binning, else all zero
    double* cell_L;        // max_cells
    double* cell_P;        // max_cells
    int* partials;         // 2 (4 grid_blocks + 1): per-block sums (int64) of the segmented scans
    int sorted_buf;        // which keys/vals buffer holds the pairs in cell order
    ft_tune tune;

    // the front of the last front_bin (the paper-neighbourhood fit reads it)
    const double* f_verts;
    const int* f_tris;
    long long f_nv, f_nt;
    // paper-neighbourhood fit (allocated on first use, grown with the front):
    // vertex -> triangles incidence and per-cell closest vertex and its normal
    long long inc_nv_cap, inc_nt_cap;
    int* inc_cnt;          // inc_nv_cap + 1
    int* inc_off;          // inc_nv_cap + 1
    int* inc_cur;          // inc_nv_cap + 1
    int* inc_part;         // inc_nv_cap / 1024 + 2
    int* inc;              // 3 inc_nt_cap
    int* cv;               // max_cells
    double* vn;            // 3 max_cells

    // batched form (nf > 0 after ft_batch_set; 0 for a one-front workspace)
    bool batch;
    int nf, max_fronts;
    long long max_grid_cells;   // index-map entries (sum of the fronts' cells)
    long long ncols;            // sum of the fronts' (i, j) columns
    long long nt_total, nv_total;
    ft_fdesc* fdesc;            // max_fronts descriptors (device)
    long long* fbase;           // 4 x (max_fronts + 1): key, column, triangle, vertex bases (device)
    unsigned* fstatus;          // max_fronts per-front status words (device)
    ft_fdesc* h_fdesc;          // host copies of the table (pinned staging)
    long long* h_fbase;
};

// kernels / launchers (one translation unit each)
namespace ft {
cudaError_t launch_parab_cells(const double* frame, const double* coeffs, long long m, double* alpha, double* area,
                               double* kappa, double* normal, int8_t* status, int sm_count, cudaStream_t s);
cudaError_t launch_parab_ppic(ft_workspace* ws, const double* coeffs, long long cap, double* alpha, double* area,
                              double* kappa, double* normal, int8_t* status, cudaStream_t s);
cudaError_t launch_parab_ppic_batch(ft_workspace* ws, const double* coeffs, long long cap, double* area,
                                    double* kappa, double* normal, int8_t* status, cudaStream_t s);
cudaError_t launch_ppic_frame(ft_workspace* ws, long long cap, double* frame, cudaStream_t s);


void count_launches(int n);  // kernels launched by this library (ft_launch_count)

// While a trace is open (ft_trace_start), brackets the launches made in its
// scope on stream s with two CUDA events attributed to `name` (a string
// literal); a no-op otherwise and during stream capture.
class Trace {
  public:
    Trace(cudaStream_t s, const char* name);
    ~Trace();
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;

  private:
    long long slot_;
    cudaStream_t s_;
};

cudaError_t launch_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, cudaStream_t s);
// vertex -> incident triangles (CSR, ascending lists), no host synchronization
cudaError_t launch_incidence(const int* tris, long long nt, long long nv, int* cnt, int* off, int* cur, int* inc,
                             int* part, unsigned* status, cudaStream_t s);
// candidate offsets of the triangles (a scan of their counts, in triangle order)
// and the triangle index of every candidate slot; sets C_need and C
cudaError_t launch_candidates(ft_workspace* ws, cudaStream_t s);
// the kept pairs into cell order: interfacial cell list, offsets, index map
// (the counts k_clip left in cell_cnt over keys [0, nkeys)); resets cell_cnt
cudaError_t launch_place_pairs(ft_workspace* ws, long long nkeys, cudaStream_t s);
cudaError_t launch_export_pairs(ft_workspace* ws, long long cap, unsigned* keys, int* tris, cudaStream_t s);
cudaError_t launch_alpha(ft_workspace* ws, double* alpha, cudaStream_t s);
cudaError_t launch_ppic(ft_workspace* ws, const ft_params* p, long long cap, unsigned* cell_keys,
                        double* kappa, double* normal, double* coeffs, int8_t* fit_status,
                        cudaStream_t s);
// the CSF force; clear: zero the dense arrays first (else the caller has);
// list: list the ring cells first (else launch_csf_prepare has, for this binning)
cudaError_t launch_csf(ft_workspace* ws, const ft_params* p, const double* alpha,
                       const double* kappa, const double* normal, double* force, cudaStream_t s, bool clear,
                       bool list);
cudaError_t launch_csf_prepare(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_force_clear(ft_workspace* ws, double* force, cudaStream_t s);
// compact outputs (one front): force at the interfacial and ring cells with their
// keys; alpha as a bit per cell (alpha > 1/2) and the interfacial cells' values
cudaError_t launch_csf_compact(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                               const double* normal, long long cap, unsigned* keys, double* force, long long* count,
                               cudaStream_t s);
cudaError_t launch_alpha_pack(ft_workspace* ws, const double* alpha, long long cap, unsigned* bits, double* acells,
                              cudaStream_t s);
cudaError_t launch_interp(const ft_grid* g, const double* U, const double* V, const double* W,
                          const double* verts, long long nv, double* vel, cudaStream_t s);
// batched form: the fronts of the workspace's table
cudaError_t launch_bin_batch(ft_workspace* ws, const ft_params* p, cudaStream_t s);
cudaError_t launch_alpha_batch(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_csf_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                             cudaStream_t s, bool clear, bool list);
cudaError_t launch_force_clear_batch(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_interp_batch(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_advect(const ft_grid* g, const double* U, const double* V, const double* W,
                          const double* verts, long long nv, double dt, double* verts_out, double* vel,
                          cudaStream_t s);
cudaError_t launch_advect_batch(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_cell_ranges(ft_workspace* ws, long long* off, cudaStream_t s);
cudaError_t launch_face_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                              const double* normal, double* fx, double* fy, double* fz, cudaStream_t s);
cudaError_t launch_face_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                                    cudaStream_t s);
// plane tables: of the workspace's grid (one front), or of every front of the table
cudaError_t launch_planes_one(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_planes_batch(ft_workspace* ws, int max_planes, cudaStream_t s);
cudaError_t probe_fma(int kind, double* flops);

}  // namespace ft

// small device helpers shared by the kernels
__device__ __forceinline__ void ft_flag(ft_counters* c, unsigned bits) {
    atomicOr(&c->status, bits);
}

__device__ __forceinline__ double ft_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long ft_warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int ft_warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// float -> double (exact) with integer operations: on this GPU the conversion
// instruction runs on the float64 pipe at the float64 rate.  Zero and normal
// floats are widened here; anything else takes the hardware conversion.
__device__ __forceinline__ double ft_f2d(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if ((b << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)b << 32));
    if (e == 0u || e == 0xffu) return (double)x;
    const unsigned hi = (b & 0x80000000u) | ((e - 127u + 1023u) << 20) | ((b & 0x7fffffu) >> 3);
    const unsigned lo = (b & 7u) << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// plane coordinate origin + idx*h, rounded once per operation (never fused)
__device__ __forceinline__ double ft_plane(double o, double h, long long idx) {
    return __dadd_rn(o, __dmul_rn((double)idx, h));
}

// entries of a front's plane table: (n0 + 1) + (n1 + 1) + (n2 + 1)
inline long long ft_plane_count(const ft_grid& g) { return (long long)g.n[0] + g.n[1] + g.n[2] + 3; }

// The float32 clip's error bounds hold while binary64 rounding of a coordinate,
// in cell units, stays far below float32 rounding: |coordinate| / h <= 2^24 on
// the whole grid (unit-cube grids: n <= 2^24), so that binary64 plane
// coordinates X_i = origin + i h (two roundings) are spaced h apart to within
// 2^-51 * 2^24 h < 1e-8 h.
inline bool ft_clip32_grid_ok(const ft_grid& g) {
    for (int d = 0; d < 3; d++) {
        const double ext = (g.origin[d] < 0 ? -g.origin[d] : g.origin[d]) + (double)g.n[d] * g.h;
        if (!(ext / g.h <= 16777216.0)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Front lookups.  Kernels are instantiated for one of two policies:
//  * FrontsOne  -- a single front; its descriptor is a kernel argument and every
//                  lookup is a constant (the one-front entry points);
//  * FrontsMany -- a batch: the front owning a batch-global cell key, (i, j)
//                  column, triangle or vertex is found by binary search of the
//                  prefix bases (the batched entry points).
// Batch-global numbering: front b's cells are keys key_base[b] + local key, its
// columns col_base[b] + i n1 + j, its triangles tri_base[b] + t, its vertices
// vert_base[b] + v; each base array ends with the total.
// ---------------------------------------------------------------------------
struct FrontsOne {
    ft_fdesc d0;
    long long ncells, ncols;
    __device__ __forceinline__ int by_key(long long) const { return 0; }
    __device__ __forceinline__ int by_col(long long) const { return 0; }
    __device__ __forceinline__ int by_tri(long long) const { return 0; }
    __device__ __forceinline__ int by_vert(long long) const { return 0; }
    __device__ __forceinline__ const ft_fdesc& desc(int) const { return d0; }
    __device__ __forceinline__ long long key_base(int) const { return 0; }
    __device__ __forceinline__ long long col_base(int) const { return 0; }
    __device__ __forceinline__ long long tri_base(int) const { return 0; }
    __device__ __forceinline__ long long vert_base(int) const { return 0; }
    __device__ __forceinline__ void flag(int, unsigned) const {}
};

struct FrontsMany {
    const ft_fdesc* d;
    const long long* base;  // key, column, triangle, vertex bases, (nf + 1) each
    unsigned* fstatus;
    int nf;
    long long ncells, ncols;
    // largest b with b-th base <= x (empty fronts share their successor's base)
    __device__ __forceinline__ int search(int which, long long x) const {
        const long long* b = base + (long long)which * (nf + 1);
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(b + mid) <= x)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ int by_key(long long x) const { return search(0, x); }
    __device__ __forceinline__ int by_col(long long x) const { return search(1, x); }
    __device__ __forceinline__ int by_tri(long long x) const { return search(2, x); }
    __device__ __forceinline__ int by_vert(long long x) const { return search(3, x); }
    __device__ __forceinline__ const ft_fdesc& desc(int b) const { return d[b]; }
    __device__ __forceinline__ long long key_base(int b) const { return __ldg(base + b); }
    __device__ __forceinline__ long long col_base(int b) const { return __ldg(base + (nf + 1) + b); }
    __device__ __forceinline__ long long tri_base(int b) const { return __ldg(base + 2 * (nf + 1) + b); }
    __device__ __forceinline__ long long vert_base(int b) const { return __ldg(base + 3 * (nf + 1) + b); }
    __device__ __forceinline__ void flag(int b, unsigned bits) const { atomicOr(fstatus + b, bits); }
};

// host-side construction of the policies
inline FrontsOne ft_one(const ft_workspace* ws, const double* verts, const int* tris, long long nv, long long nt) {
    FrontsOne f;
    f.d0 = ft_fdesc{};
    f.d0.g = ws->g;
    f.d0.planes = ws->planes;
    f.d0.inv_h = 1.0 / ws->g.h;
    f.d0.verts = verts;
    f.d0.tris = tris;
    f.d0.nv = nv;
    f.d0.nt = nt;
    f.ncells = ws->ncells;
    f.ncols = (long long)ws->g.n[0] * ws->g.n[1];
    return f;
}

inline FrontsMany ft_many(const ft_workspace* ws) {
    FrontsMany f;
    f.d = ws->fdesc;
    f.base = ws->fbase;
    f.fstatus = ws->fstatus;
    f.nf = ws->nf;
    f.ncells = ws->ncells;
    f.ncols = ws->ncols;
    return f;
}
