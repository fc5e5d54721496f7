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
           isfinite(p->sigma) && p->fit_ring >= 0 && p->fit_ring <= 3 && (p->frame == FT_FRAME_FRAGMENTS ||
                                                                        p->frame == FT_FRAME_VERTEX);
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
                    ws->cell_off, ws->cell_cnt, ws->cell_L,   ws->cell_P,   ws->partials,
                    ws->rec32,   ws->cen32,   ws->sys,      ws->fit_info, ws->srec, ws->srec32, ws->scen,
                    ws->fdesc,   ws->fbase,   ws->fstatus, ws->tri_nrm, ws->tri32, ws->planes,
                    ws->inc_cnt, ws->inc_off, ws->inc_cur, ws->inc_part, ws->inc, ws->cv, ws->vn};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ws->h_fdesc) cudaFreeHost(ws->h_fdesc);
    if (ws->h_fbase) cudaFreeHost(ws->h_fbase);
}

// Device memory of a workspace for `map_cells` index-map entries, once the
// capacities are set; frees everything and returns FT_ERR_ALLOC on failure.
int allocate(ft_workspace* ws, long long map_cells) {
    cudaDeviceGetAttribute(&ws->sm_count, cudaDevAttrMultiProcessorCount, ws->device);
    // segments (blocks) of the scan kernels; the down-sweeps take one partial per thread
    ws->grid_blocks = ws->sm_count > 192 ? 192 : ws->sm_count;
    ws->tune = ft_tune{3, 4, 16, 8, 4, 0, ws->grid_blocks};
    size_t tot = 0;
    cudaError_t e = cudaSuccess;
    const size_t C = (size_t)ws->max_cand, Mx = (size_t)ws->max_cells, T = (size_t)ws->max_nt;
    e = e ? e : alloc(&ws->ctr, 1, &tot);
    e = e ? e : alloc(&ws->idx_map, (size_t)map_cells, &tot);
    e = e ? e : alloc(&ws->tri_cnt, T, &tot);
    e = e ? e : alloc(&ws->tri_off, T, &tot);
    e = e ? e : alloc(&ws->tri_box, 8 * T, &tot);
    e = e ? e : alloc(&ws->tri_nrm, 4 * T, &tot);
    e = e ? e : alloc(&ws->tri32, 32 * T, &tot);
    if (!ws->batch) {
        ws->planes_cap = ft_plane_count(ws->g);
        e = e ? e : alloc(&ws->planes, (size_t)ws->planes_cap, &tot);
        if (e == cudaSuccess) e = ft::launch_planes_one(ws, 0);
    }
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
    e = e ? e : alloc(&ws->cell_cnt, (size_t)map_cells, &tot);
    e = e ? e : alloc(&ws->cell_L, Mx, &tot);
    e = e ? e : alloc(&ws->cell_P, Mx, &tot);
    e = e ? e : alloc(&ws->partials, 2 * (size_t)(4 * ws->grid_blocks + 1), &tot);
    if (ws->batch) {
        const size_t F = (size_t)ws->max_fronts;
        e = e ? e : alloc(&ws->fdesc, F, &tot);
        e = e ? e : alloc(&ws->fbase, 4 * (F + 1), &tot);
        e = e ? e : alloc(&ws->fstatus, F, &tot);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&ws->h_fdesc), F * sizeof(ft_fdesc));
        if (e == cudaSuccess)
            e = cudaMallocHost(reinterpret_cast<void**>(&ws->h_fbase), 4 * (F + 1) * sizeof(long long));
        if (e == cudaSuccess) e = cudaMemset(ws->fstatus, 0, F * sizeof(unsigned));
    }
    if (e == cudaSuccess) e = cudaMemset(ws->ctr, 0, sizeof(ft_counters));
    if (e == cudaSuccess) e = cudaMemset(ws->idx_map, 0xff, sizeof(int) * (size_t)map_cells);
    if (e == cudaSuccess) e = cudaMemset(ws->cell_cnt, 0, sizeof(int) * (size_t)map_cells);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        release(ws);
        cudaGetLastError();
        return FT_ERR_ALLOC;
    }
    ws->bytes = tot;
    return FT_OK;
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
    ws->clip32_ok = ft_clip32_grid_ok(*g);
    ws->ncells = (long long)g->n[0] * g->n[1] * g->n[2];
    ws->max_nt = cap->max_nt > 0 ? cap->max_nt : 1;
    ws->max_cand = cap->max_cand > 0 ? cap->max_cand : 16 * ws->max_nt + 1024;
    ws->max_cells = cap->max_cells > 0 ? cap->max_cells : ws->max_cand;
    if (ws->max_cand > 0x7fffffffLL - 1 || ws->max_cells > ws->max_cand) {
        free(ws);
        return FT_ERR_ARG;
    }
    const int r = allocate(ws, ws->ncells);
    if (r != FT_OK) {
        free(ws);
        return r;
    }
    if (bytes) *bytes = ws->bytes;
    *out = ws;
    return FT_OK;
}

int ft_batch_workspace_create(ft_workspace** out, const ft_batch_capacity* cap, int device, size_t* bytes) {
    if (!out || !cap || cap->max_fronts < 1 || cap->max_grid_cells < 1 || cap->max_grid_cells >= 0xffffffffLL ||
        cap->max_nt < 0 || cap->max_cand < 0 || cap->max_cells < 0)
        return FT_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return FT_ERR_CUDA;
    ft_workspace* ws = (ft_workspace*)calloc(1, sizeof(ft_workspace));
    if (!ws) return FT_ERR_ALLOC;
    ws->device = device;
    ws->batch = true;
    ws->max_fronts = cap->max_fronts;
    ws->max_grid_cells = cap->max_grid_cells;
    ws->max_nt = cap->max_nt > 0 ? cap->max_nt : 1;
    ws->max_cand = cap->max_cand > 0 ? cap->max_cand : 16 * ws->max_nt + 1024;
    ws->max_cells = cap->max_cells > 0 ? cap->max_cells : ws->max_cand;
    if (ws->max_cand > 0x7fffffffLL - 1 || ws->max_cells > ws->max_cand) {
        free(ws);
        return FT_ERR_ARG;
    }
    const int r = allocate(ws, ws->max_grid_cells);
    if (r != FT_OK) {
        free(ws);
        return r;
    }
    if (bytes) *bytes = ws->bytes;
    *out = ws;
    return FT_OK;
}

int ft_batch_set(ft_workspace* ws, int32_t nf, const ft_batch_front* fr, void* stream) {
    if (!ws || !ws->batch || nf < 1 || !fr) return FT_ERR_ARG;
    if (nf > ws->max_fronts) return FT_ERR_CAPACITY;
    long long cells = 0, cols = 0, nt = 0, nv = 0;
    for (int b = 0; b < nf; b++) {
        const ft_batch_front& f = fr[b];
        if (!grid_ok(&f.grid) || f.nt < 0 || f.nv < 0 || f.nt > 0x7fffffffLL || f.nv > 0x7fffffffLL) return FT_ERR_ARG;
        if (f.nt > 0 && (!f.verts || !f.tris)) return FT_ERR_ARG;
        cells += (long long)f.grid.n[0] * f.grid.n[1] * f.grid.n[2];
        cols += (long long)f.grid.n[0] * f.grid.n[1];
        nt += f.nt;
        nv += f.nv;
    }
    if (cells > ws->max_grid_cells || nt > ws->max_nt) return FT_ERR_CAPACITY;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    // the staging buffers may still feed the previous table's copy
    if (cudaStreamSynchronize(s) != cudaSuccess) return FT_ERR_CUDA;
    // plane tables of every front (grown here when the table needs more)
    long long nplanes = 0, max_planes = 0;
    for (int b = 0; b < nf; b++) {
        const long long q = ft_plane_count(fr[b].grid);
        nplanes += q;
        if (q > max_planes) max_planes = q;
    }
    if (nplanes > ws->planes_cap) {
        if (cudaDeviceSynchronize() != cudaSuccess) return FT_ERR_CUDA;
        if (ws->planes) cudaFree(ws->planes);
        ws->planes = nullptr;
        ws->planes_cap = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&ws->planes), sizeof(double) * (size_t)nplanes) != cudaSuccess) {
            cudaGetLastError();
            return FT_ERR_ALLOC;
        }
        ws->planes_cap = nplanes;
        ws->bytes += sizeof(double) * (size_t)nplanes;
    }
    long long* kb = ws->h_fbase;
    long long* cb = kb + (nf + 1);
    long long* tb = cb + (nf + 1);
    long long* vb = tb + (nf + 1);
    kb[0] = cb[0] = tb[0] = vb[0] = 0;
    long long pofs = 0;
    ws->clip32_ok = true;
    for (int b = 0; b < nf; b++) {
        const ft_batch_front& f = fr[b];
        ws->clip32_ok = ws->clip32_ok && ft_clip32_grid_ok(f.grid);
        ft_fdesc& d = ws->h_fdesc[b];
        d = ft_fdesc{};
        d.g = f.grid;
        d.verts = f.verts;
        d.tris = f.tris;
        d.alpha = f.alpha;
        d.force = f.force;
        d.U = f.U;
        d.V = f.V;
        d.W = f.W;
        d.vel = f.vel;
        d.verts_next = f.verts_next;
        d.dt = f.dt;
        for (int k = 0; k < 3; k++) d.fface[k] = f.face_force[k];
        d.nv = f.nv;
        d.nt = f.nt;
        d.planes = ws->planes + pofs;
        d.inv_h = 1.0 / f.grid.h;
        pofs += ft_plane_count(f.grid);
        kb[b + 1] = kb[b] + (long long)f.grid.n[0] * f.grid.n[1] * f.grid.n[2];
        cb[b + 1] = cb[b] + (long long)f.grid.n[0] * f.grid.n[1];
        tb[b + 1] = tb[b] + f.nt;
        vb[b + 1] = vb[b] + f.nv;
    }
    cudaError_t e = cudaMemcpyAsync(ws->fdesc, ws->h_fdesc, sizeof(ft_fdesc) * nf, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws->fbase, ws->h_fbase, sizeof(long long) * 4 * (nf + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->fstatus, 0, sizeof(unsigned) * nf, s);
    ws->nf = nf;
    if (e == cudaSuccess) e = ft::launch_planes_batch(ws, (int)max_planes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ws->nf = 0;
        return FT_ERR_CUDA;
    }
    ws->ncells = cells;
    ws->ncols = cols;
    ws->fitted = false;
    ws->nt_total = nt;
    ws->nv_total = nv;
    ws->binned = false;
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

int ft_work_counts(ft_workspace* ws, void* stream, int64_t* out, int32_t n) {
    if (!ws || !out || n < 0) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    ft_counters c;
    cudaError_t e = cudaMemcpyAsync(&c, ws->ctr, sizeof(c), cudaMemcpyDeviceToHost, as_stream(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    const int64_t v[FT_WORK_COUNTS] = {c.T, c.M, c.P, c.C, c.C_need, c.fit_pairs, c.clip_f64, (int64_t)c.pad};
    for (int i = 0; i < n && i < FT_WORK_COUNTS; i++) out[i] = v[i];
    return cuda_err(e);
}

int ft_bin_pairs(ft_workspace* ws, int64_t cap, uint32_t* keys, int32_t* tris, void* stream) {
    if (!ws || cap < 0 || !keys || !tris) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_export_pairs(ws, cap, keys, tris, as_stream(stream)));
}

int front_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, void* stream) {
    if (!ws || ws->batch || !f || !params_ok(p) || f->nt < 0 || f->nv < 0 || f->nt > ws->max_nt) return FT_ERR_ARG;
    if (f->nt > 0 && (!f->verts || !f->tris)) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    ws->f_verts = f->verts;
    ws->f_tris = f->tris;
    ws->f_nv = f->nv;
    ws->f_nt = f->nt;
    ws->bin_epoch++;
    cudaError_t e = ft::launch_bin(ws, f, p, s);
    if (e == cudaSuccess) e = ft::launch_place_pairs(ws, ws->ncells, s);
    ws->binned = (e == cudaSuccess);
    ws->fitted = false;
    return cuda_err(e);
}

int front_volume_fraction(ft_workspace* ws, double* alpha, void* stream) {
    if (!ws || ws->batch || !alpha) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_alpha(ws, alpha, as_stream(stream)));
}

int front_curvature_ppic(ft_workspace* ws, const ft_params* p, int64_t cap, uint32_t* cell_keys, double* kappa,
                         double* normal, double* coeffs, int8_t* fit_status, void* stream) {
    if (!ws || !params_ok(p) || cap < 0 || !cell_keys || !kappa || !normal || !fit_status) return FT_ERR_ARG;
    if ((p->fit_ring > 0 || p->frame != FT_FRAME_FRAGMENTS) && ws->batch) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    const cudaError_t e = ft::launch_ppic(ws, p, cap, cell_keys, kappa, normal, coeffs, fit_status, as_stream(stream));
    ws->fitted = (e == cudaSuccess);
    return cuda_err(e);
}

int front_paraboloid_cells(const double* frame, const double* coeffs, int64_t m, double* alpha, double* area,
                           double* kappa, double* normal, int8_t* status, void* stream) {
    if (m < 0 || (m > 0 && (!frame || !coeffs || !alpha))) return FT_ERR_ARG;
    if (m == 0) return FT_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, frame) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return FT_ERR_ARG;
    }
    if (cudaSetDevice(at.device) != cudaSuccess) return FT_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, at.device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_parab_cells(frame, coeffs, m, alpha, area, kappa, normal, status, sms,
                                           as_stream(stream)));
}

int front_ppic_frame(ft_workspace* ws, int64_t cap, double* frame, void* stream) {
    if (!ws || cap < 0 || !frame) return FT_ERR_ARG;
    if (!ws->binned || !ws->fitted) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_ppic_frame(ws, cap, frame, as_stream(stream)));
}

int front_volume_fraction_ppic(ft_workspace* ws, const double* coeffs, int64_t cap, double* alpha, double* kappa,
                               double* normal, double* area, int8_t* status, void* stream) {
    if (!ws || ws->batch || cap < 0 || !coeffs || !alpha) return FT_ERR_ARG;
    if (!ws->binned || !ws->fitted) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_parab_ppic(ws, coeffs, cap, alpha, area, kappa, normal, status, as_stream(stream)));
}

int front_volume_fraction_ppic_batch(ft_workspace* ws, const double* coeffs, int64_t cap, double* kappa,
                                     double* normal, double* area, int8_t* status, void* stream) {
    if (!ws || !ws->batch || cap < 0 || !coeffs) return FT_ERR_ARG;
    if (!ws->binned || !ws->fitted) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++)
        if (!ws->h_fdesc[b].alpha) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_parab_ppic_batch(ws, coeffs, cap, area, kappa, normal, status, as_stream(stream)));
}

int front_csf_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                    const double* normal, double* force, void* stream) {
    if (!ws || ws->batch || !params_ok(p) || !alpha || !kappa || !normal || !force) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf(ws, p, alpha, kappa, normal, force, as_stream(stream), true, true));
}

int front_csf_prepare(ft_workspace* ws, void* stream) {
    if (!ws) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    const cudaError_t e = ft::launch_csf_prepare(ws, as_stream(stream));
    if (e == cudaSuccess) ws->ring_epoch = ws->bin_epoch;
    return cuda_err(e);
}

int front_force_clear(ft_workspace* ws, double* force, void* stream) {
    if (!ws || ws->batch || !force) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_force_clear(ws, force, as_stream(stream)));
}

int front_csf_force_cells(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                          const double* normal, double* force, void* stream) {
    if (!ws || ws->batch || !params_ok(p) || !alpha || !kappa || !normal || !force) return FT_ERR_ARG;
    if (!ws->binned || ws->ring_epoch != ws->bin_epoch) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf(ws, p, alpha, kappa, normal, force, as_stream(stream), false, false));
}

int front_csf_force_compact(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                            const double* normal, int64_t cap, uint32_t* keys, double* force, int64_t* count,
                            void* stream) {
    if (!ws || ws->batch || !params_ok(p) || !alpha || !kappa || !normal || cap < 0 || !keys || !force || !count)
        return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf_compact(ws, p, alpha, kappa, normal, cap, keys, force,
                                           reinterpret_cast<long long*>(count), as_stream(stream)));
}

int front_alpha_pack(ft_workspace* ws, const double* alpha, int64_t cap, uint32_t* full_bits, double* alpha_cells,
                     void* stream) {
    if (!ws || ws->batch || !alpha || cap < 0 || !full_bits || !alpha_cells) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_alpha_pack(ws, alpha, cap, full_bits, alpha_cells, as_stream(stream)));
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

int front_bin_batch(ft_workspace* ws, const ft_params* p, void* stream) {
    if (!ws || !ws->batch || !params_ok(p)) return FT_ERR_ARG;
    if (ws->nf < 1) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    ws->bin_epoch++;
    cudaError_t e = ft::launch_bin_batch(ws, p, s);
    if (e == cudaSuccess) e = ft::launch_place_pairs(ws, ws->ncells, s);
    ws->binned = (e == cudaSuccess);
    ws->fitted = false;
    return cuda_err(e);
}

int front_volume_fraction_batch(ft_workspace* ws, void* stream) {
    if (!ws || !ws->batch) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++)
        if (!ws->h_fdesc[b].alpha) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_alpha_batch(ws, as_stream(stream)));
}

int front_csf_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                          void* stream) {
    if (!ws || !ws->batch || !params_ok(p) || !kappa || !normal) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++)
        if (!ws->h_fdesc[b].alpha || !ws->h_fdesc[b].force) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf_batch(ws, p, kappa, normal, as_stream(stream), true, true));
}

int front_force_clear_batch(ft_workspace* ws, void* stream) {
    if (!ws || !ws->batch) return FT_ERR_ARG;
    if (ws->nf < 1) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++)
        if (!ws->h_fdesc[b].force) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_force_clear_batch(ws, as_stream(stream)));
}

int front_csf_force_cells_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                                void* stream) {
    if (!ws || !ws->batch || !params_ok(p) || !kappa || !normal) return FT_ERR_ARG;
    if (!ws->binned || ws->ring_epoch != ws->bin_epoch) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++)
        if (!ws->h_fdesc[b].alpha || !ws->h_fdesc[b].force) return FT_ERR_ARG;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_csf_batch(ws, p, kappa, normal, as_stream(stream), false, false));
}

int front_face_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                     const double* normal, double* fx, double* fy, double* fz, void* stream) {
    if (!ws || ws->batch || !params_ok(p) || !alpha || !kappa || !normal || !fx || !fy || !fz) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_face_force(ws, p, alpha, kappa, normal, fx, fy, fz, as_stream(stream)));
}

int front_face_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                           void* stream) {
    if (!ws || !ws->batch || !params_ok(p) || !kappa || !normal) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++) {
        const ft_fdesc& d = ws->h_fdesc[b];
        if (!d.alpha || !d.fface[0] || !d.fface[1] || !d.fface[2]) return FT_ERR_ARG;
    }
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_face_force_batch(ws, p, kappa, normal, as_stream(stream)));
}

int front_interp_velocity_batch(ft_workspace* ws, void* stream) {
    if (!ws || !ws->batch) return FT_ERR_ARG;
    if (ws->nf < 1) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++) {
        const ft_fdesc& d = ws->h_fdesc[b];
        if (d.nv == 0) continue;
        if (!d.U || !d.V || !d.W || !d.verts || !d.vel) return FT_ERR_ARG;
        for (int k = 0; k < 3; k++)
            if (d.g.n[k] < 2) return FT_ERR_ARG;
    }
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_interp_batch(ws, as_stream(stream)));
}

int front_advect_rk4_batch(ft_workspace* ws, void* stream) {
    if (!ws || !ws->batch) return FT_ERR_ARG;
    if (ws->nf < 1) return FT_ERR_STATE;
    for (int b = 0; b < ws->nf; b++) {
        const ft_fdesc& d = ws->h_fdesc[b];
        if (d.nv == 0) continue;
        if (!d.U || !d.V || !d.W || !d.verts || !d.verts_next || !isfinite(d.dt)) return FT_ERR_ARG;
        for (int k = 0; k < 3; k++)
            if (d.g.n[k] < 2) return FT_ERR_ARG;
    }
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_advect_batch(ws, as_stream(stream)));
}

int ft_batch_cell_ranges(ft_workspace* ws, int64_t* off, void* stream) {
    if (!ws || !ws->batch || !off) return FT_ERR_ARG;
    if (!ws->binned) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::launch_cell_ranges(ws, reinterpret_cast<long long*>(off), as_stream(stream)));
}

int ft_batch_status(ft_workspace* ws, void* stream, uint32_t* bits) {
    if (!ws || !ws->batch || !bits) return FT_ERR_ARG;
    if (ws->nf < 1) return FT_ERR_STATE;
    if (cudaSetDevice(ws->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(bits, ws->fstatus, sizeof(unsigned) * ws->nf, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->fstatus, 0, sizeof(unsigned) * ws->nf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(e);
}

int ft_set_tuning(ft_workspace* ws, const ft_tuning* t) {
    if (!ws || !t) return FT_ERR_ARG;
    const int v[4] = {t->clip_blocks_per_sm, t->ppic_blocks_per_sm, t->csf_blocks_per_sm, t->fill_blocks_per_sm};
    for (int x : v)
        if (x < 1 || x > 32) return FT_ERR_ARG;
    if (t->ppic_min_blocks != 4 && t->ppic_min_blocks != 6) return FT_ERR_ARG;
    if (t->ppic_dynamic != 0 && t->ppic_dynamic != 1) return FT_ERR_ARG;
    const int seg = t->sort_blocks == 0 ? ws->grid_blocks : t->sort_blocks;
    if (seg < 1 || seg > ws->grid_blocks) return FT_ERR_ARG;
    ws->tune = ft_tune{v[0], v[1], v[2], v[3], t->ppic_min_blocks, t->ppic_dynamic, seg};
    return FT_OK;
}

int ft_get_tuning(ft_workspace* ws, ft_tuning* t) {
    if (!ws || !t) return FT_ERR_ARG;
    memset(t, 0, sizeof(*t));
    t->clip_blocks_per_sm = ws->tune.clip_bps;
    t->ppic_blocks_per_sm = ws->tune.ppic_bps;
    t->csf_blocks_per_sm = ws->tune.csf_bps;
    t->fill_blocks_per_sm = ws->tune.fill_bps;
    t->ppic_min_blocks = ws->tune.ppic_min_blocks;
    t->ppic_dynamic = ws->tune.ppic_dynamic;
    t->sort_blocks = ws->tune.seg_blocks;
    return FT_OK;
}

int front_advect_rk4(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                     int64_t nv, double dt, double* verts_out, double* vel, void* stream) {
    if (!grid_ok(g) || nv < 0 || !isfinite(dt) || (nv > 0 && (!U || !V || !W || !verts || !verts_out)))
        return FT_ERR_ARG;
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
    return cuda_err(ft::launch_advect(g, U, V, W, verts, nv, dt, verts_out, vel, as_stream(stream)));
}

int64_t ft_launch_count(void) { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int ft_probe_fma_rate(int kind, int device, double* flops) {
    if (!flops || (kind != 0 && kind != 1)) return FT_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FT_ERR_CUDA;
    return cuda_err(ft::probe_fma(kind, flops));
}

}  // extern "C"
