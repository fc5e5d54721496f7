// ft_api.cu -- the extern "C" entry points of libfront.so (declared and
// documented in include/front.h): argument checks, workspace memory and the
// launch sequence of each step.  All compute runs in the kernels of k_*.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ft_internal.cuh"

namespace {
unsigned long long g_launches = 0;
}

namespace ft {
void count_launches(int n) { __atomic_add_fetch(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
}  // namespace ft

namespace {

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int cuda_err(cudaError_t e) { return e == cudaSuccess ? FT_OK : FT_ERR_CUDA; }

bool grid_ok(const ft_grid* g) {
    if (!g) return false;
    for (int d = 0; d < 3; d++)
        if (g->n[d] < 1 || !isfinite(g->origin[d])) return false;
    const double nc = (double)g->n[0] * g->n[1] * g->n[2];
    return g->h > 0.0 && isfinite(g->h) && nc < 4294967295.0;
}

bool params_ok(const ft_params* p) {
    return p && p->delta_h > 0.0 && p->delta_max_h >= p->delta_h && p->delta_max_h <= 7.0 &&
           p->delta_growth > 1.0 && p->fit_min >= 0 && (p->precision == FT_FP64 || p->precision == FT_FP32C) &&
           isfinite(p->sigma);
}

template <class T>
cudaError_t alloc(T** p, size_t n, size_t* total) {
    *p = nullptr;
    if (n == 0) n = 1;
    *total += n * sizeof(T);
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

void release(ft_workspace* ws) {
    void* ptrs[] = {ws->ctr,     ws->idx_map, ws->tri_cnt,  ws->tri_off,  ws->tri_box, ws->cand_tri,
                    ws->keys[0], ws->keys[1], ws->vals[0],  ws->vals[1],  ws->rec,     ws->cells,
                    ws->cell_off, ws->heads,  ws->cell_L,   ws->cell_P,   ws->partials, ws->hist,
                    ws->rec32,   ws->cen32,   ws->sys,      ws->fit_info, ws->srec, ws->srec32, ws->scen};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

extern "C" {

const char* ft_status_string(int code) {
    switch (code) {
        case FT_OK: return "ok";
        case FT_ERR_ARG: return "invalid argument";
        case FT_ERR_ALLOC: return "device allocation failed";
        case FT_ERR_CAPACITY: return "workspace capacity exceeded";
        case FT_ERR_OUTSIDE_GRID: return "front outside the grid margin";
        case FT_ERR_NOT_CLOSED: return "front is not closed";
        case FT_ERR_ORIENTATION: return "front is inverted";
        case FT_ERR_TIMEOUT: return "device wait timed out";
        case FT_ERR_CUDA: return "CUDA error";
        case FT_ERR_STATE: return "call order violated";
        default: return "unknown status";
    }
}

int ft_workspace_create(ft_workspace** out, const ft_grid* g, const ft_capacity* cap, int device, size_t* bytes) {
    if (!out || !grid_ok(g) || !cap || cap->max_nt < 0) return FT_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return FT_ERR_CUDA;
    ft_workspace* ws = (ft_workspace*)calloc(1, sizeof(ft_workspace));
    if (!ws) return FT_ERR_ALLOC;
    ws->device = device;
    ws->g = *g;
    ws->ncells = (long long)g->n[0] * g->n[1] * g->n[2];
    ws->max_nt = cap->max_nt > 0 ? cap->max_nt : 1;
    ws->max_cand = cap->max_cand > 0 ? cap->max_cand : 16 * ws->max_nt + 1024;
    ws->max_cells = cap->max_cells > 0 ? cap->max_cells : ws->max_cand;
    if (ws->max_cand > 0x7fffffffLL - 1 || ws->max_cells > ws->max_cand) {
        free(ws);
        return FT_ERR_ARG;
    }
    cudaDeviceGetAttribute(&ws->sm_count, cudaDevAttrMultiProcessorCount, device);
    // segments of the scan / sort kernels; the sort stages 256 x grid_blocks counts in shared memory
    ws->grid_blocks = ws->sm_count > 192 ? 192 : ws->sm_count;
    int bits = 1;
    while (bits < 32 && ((ws->ncells - 1) >> bits) > 0) bits++;
    ws->key_bits = bits < 8 ? 8 : bits;
    size_t tot = 0;
    cudaError_t e = cudaSuccess;
    const size_t C = (size_t)ws->max_cand, Mx = (size_t)ws->max_cells, T = (size_t)ws->max_nt;
    e = e ? e : alloc(&ws->ctr, 1, &tot);
    e = e ? e : alloc(&ws->idx_map, (size_t)ws->ncells, &tot);
    e = e ? e : alloc(&ws->tri_cnt, T, &tot);
    e = e ? e : alloc(&ws->tri_off, T, &tot);
    e = e ? e : alloc(&ws->tri_box, 6 * T, &tot);
    e = e ? e : alloc(&ws->cand_tri, C, &tot);
    e = e ? e : alloc(&ws->keys[0], C, &tot);
    e = e ? e : alloc(&ws->keys[1], C, &tot);
    e = e ? e : alloc(&ws->vals[0], C, &tot);
    e = e ? e : alloc(&ws->vals[1], C, &tot);
    e = e ? e : alloc(&ws->rec, C, &tot);
    e = e ? e : alloc(&ws->rec32, C, &tot);
    e = e ? e : alloc(&ws->cen32, C, &tot);
    e = e ? e : alloc(&ws->srec, C, &tot);
    e = e ? e : alloc(&ws->srec32, C, &tot);
    e = e ? e : alloc(&ws->scen, C, &tot);
    e = e ? e : alloc(&ws->sys, Mx, &tot);
    e = e ? e : alloc(&ws->fit_info, 2 * Mx, &tot);
    e = e ? e : alloc(&ws->cells, Mx + 1, &tot);
    e = e ? e : alloc(&ws->cell_off, Mx + 1, &tot);
    e = e ? e : alloc(&ws->heads, C, &tot);
    e = e ? e : alloc(&ws->cell_L, Mx, &tot);
    e = e ? e : alloc(&ws->cell_P, Mx, &tot);
    e = e ? e : alloc(&ws->partials, 2 * (size_t)(ws->grid_blocks + 1), &tot);
    e = e ? e : alloc(&ws->hist, 256 * (size_t)ws->grid_blocks, &tot);
    if (e == cudaSuccess) e = ft::prepare_sort(ws->grid_blocks);
    if (e == cudaSuccess) e = cudaMemset(ws->ctr, 0, sizeof(ft_counters));
    if (e == cudaSuccess) e = cudaMemset(ws->idx_map, 0xff, sizeof(int) * (size_t)ws->ncells);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        release(ws);
        free(ws);
        cudaGetLastError();
        return FT_ERR_ALLOC;
    }
    ws->bytes = tot;
    if (bytes) *bytes = tot;
    *out = ws;
    return FT_OK;
}

int ft_workspace_destroy(ft_workspace* ws) {
    if (!ws) return FT_ERR_ARG;
    cudaSetDevice(ws->device);
    cudaDeviceSynchronize();
    release(ws);
    free(ws);
    return FT_OK;
}

int ft_status(ft_workspace* ws, void* stream, uint32_t* bits) {
    if (!ws || !bits) return FT_ERR_ARG;
    cudaSetDevice(ws->device);
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, &ws->ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, as_stream(stream));
    if (e == cudaSuccess) e = cudaMemsetAsync(&ws->ctr->status, 0, sizeof(unsigned), as_stream(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    *bits = v;
    return cuda_err(e);
}

int ft_counts(ft_workspace* ws, void* stream, int64_t* out5) {
    if (!ws || !out5) return FT_ERR_ARG;
    cudaSetDevice(ws->device);
    ft_counters c;
    cudaError_t e = cudaMemcpyAsync(&c, ws->ctr, sizeof(c), cudaMemcpyDeviceToHost, as_stream(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    out5[0] = c.M;
    out5[1] = c.P;
    out5[2] = c.C;
    out5[3] = c.C_need;
    out5[4] = c.fit_pairs;
    return cuda_err(e);
}

int ft_bin_pairs(ft_workspace* ws, int64_t cap, uint32_t* keys, int32_t* tris, void* stream) {
    if (!ws || cap < 0 || !keys || !tris) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_export_pairs(ws, cap, keys, tris, as_stream(stream)));
}

int front_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, void* stream) {
    if (!ws || !f || !params_ok(p) || f->nt < 0 || f->nv < 0 || f->nt > ws->max_nt) return FT_ERR_ARG;
    if (f->nt > 0 && (!f->verts || !f->tris)) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = ft::launch_clear_map(ws, s);
    if (e == cudaSuccess) e = ft::launch_bin(ws, f, p, s);
    if (e == cudaSuccess) e = ft::launch_sort(ws, s);
    if (e == cudaSuccess) e = ft::launch_rle(ws, s);
    if (e == cudaSuccess) e = ft::launch_gather(ws, s);
    ws->binned = (e == cudaSuccess);
    return cuda_err(e);
}

int front_volume_fraction(ft_workspace* ws, double* alpha, void* stream) {
    if (!ws || !alpha) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_alpha(ws, alpha, as_stream(stream)));
}

int front_curvature_ppic(ft_workspace* ws, const ft_params* p, int64_t cap, uint32_t* cell_keys, double* kappa,
                         double* normal, double* coeffs, int8_t* fit_status, void* stream) {
    if (!ws || !params_ok(p) || cap < 0 || !cell_keys || !kappa || !normal || !fit_status) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_ppic(ws, p, cap, cell_keys, kappa, normal, coeffs, fit_status, as_stream(stream)));
}

int front_csf_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                    const double* normal, double* force, void* stream) {
    if (!ws || !params_ok(p) || !alpha || !kappa || !normal || !force) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf(ws, p, alpha, kappa, normal, force, as_stream(stream)));
}

int front_interp_velocity(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                          int64_t nv, double* vel, void* stream) {
    if (!grid_ok(g) || nv < 0 || (nv > 0 && (!U || !V || !W || !verts || !vel))) return FT_ERR_ARG;
    for (int d = 0; d < 3; d++)
        if (g->n[d] < 2) return FT_ERR_ARG;
    if (nv > 0) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, verts) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return FT_ERR_ARG;
        }
        if (cudaSetDevice(at.device) != cudaSuccess) return FT_ERR_CUDA;
    }
    return cuda_err(ft::launch_interp(g, U, V, W, verts, nv, vel, as_stream(stream)));
}

int64_t ft_launch_count(void) { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int ft_probe_fma_rate(int kind, int device, double* flops) {
    if (!flops || (kind != 0 && kind != 1)) return FT_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::probe_fma(kind, flops));
}

}  // extern "C"
