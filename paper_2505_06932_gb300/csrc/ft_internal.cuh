// ft_internal.cuh -- internal declarations of libfront.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "front.h"

#define FT_WARP 32
#define FT_SENTINEL 0xffffffffu

// Device-side counters of one workspace (one cache line).
struct ft_counters {
    unsigned int status;   // FT_ST_* bits
    unsigned int pad;
    long long T;           // triangles of the last front_bin
    long long C_need;      // candidate pairs needed
    long long C;           // candidate pairs used (0 if C_need > capacity)
    long long P;           // binned pairs
    long long M;           // interfacial cells (also: entries set in the index map)
    long long fit_pairs;   // (cell, fragment) pairs inside the support, last PPIC
    long long pad2;
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

struct ft_workspace {
    int device;
    int sm_count;
    int grid_blocks;       // blocks of the segmented scan/sort kernels
    int key_bits;          // bits of the largest cell key
    ft_grid g;
    long long ncells;
    long long max_nt, max_cand, max_cells;
    size_t bytes;
    bool binned;
    int last_precision;

    ft_counters* ctr;
    int* idx_map;          // ncells: interfacial index or -1
    int* tri_cnt;          // max_nt
    int* tri_off;          // max_nt
    int* tri_box;          // max_nt * 6: lo[3], ext[3]
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
    int* heads;            // max_cand: cell index of each sorted pair (scan output)
    double* cell_L;        // max_cells
    double* cell_P;        // max_cells
    int* partials;         // grid_blocks + 1
    int* hist;             // 256 * grid_blocks
    int sorted_buf;        // which keys/vals buffer holds the sorted pairs
};

// kernels / launchers (one translation unit each)
namespace ft {

void count_launches(int n);  // kernels launched by this library (ft_launch_count)

cudaError_t launch_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, cudaStream_t s);
cudaError_t launch_scan_counts(ft_workspace* ws, const int* in, int* out, const long long* n,
                               long long* total, cudaStream_t s);
cudaError_t launch_scan_heads(ft_workspace* ws, const unsigned* keys, int* out, const long long* n,
                              long long* total, cudaStream_t s);
cudaError_t launch_sort(ft_workspace* ws, cudaStream_t s);
cudaError_t prepare_sort(int grid_blocks);
cudaError_t launch_rle(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_gather(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_clear_map(ft_workspace* ws, cudaStream_t s);
cudaError_t launch_export_pairs(ft_workspace* ws, long long cap, unsigned* keys, int* tris, cudaStream_t s);
cudaError_t launch_alpha(ft_workspace* ws, double* alpha, cudaStream_t s);
cudaError_t launch_ppic(ft_workspace* ws, const ft_params* p, long long cap, unsigned* cell_keys,
                        double* kappa, double* normal, double* coeffs, int8_t* fit_status,
                        cudaStream_t s);
cudaError_t launch_csf(ft_workspace* ws, const ft_params* p, const double* alpha,
                       const double* kappa, const double* normal, double* force, cudaStream_t s);
cudaError_t launch_interp(const ft_grid* g, const double* U, const double* V, const double* W,
                          const double* verts, long long nv, double* vel, cudaStream_t s);
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

// plane coordinate origin + idx*h, rounded once per operation (never fused)
__device__ __forceinline__ double ft_plane(double o, double h, long long idx) {
    return __dadd_rn(o, __dmul_rn((double)idx, h));
}
