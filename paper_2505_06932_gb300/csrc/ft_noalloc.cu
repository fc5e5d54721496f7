// ft_noalloc.cu -- ft_volume_fraction_noalloc: the volume fraction of one front
// (binning + alpha) without any device allocation.  All scratch lives in one
// file-scope static device array of FT_NOALLOC_SCRATCH_BYTES; the caller passes
// only the front, the grid and the output.  The existing binning and alpha
// kernels run unchanged on a workspace view carved out of that array.
#include <math.h>
#include <mutex>

#include "ft_internal.cuh"

namespace {

constexpr long long kMaxCells = FT_NOALLOC_MAX_GRID_CELLS;
constexpr long long kMaxNt = FT_NOALLOC_MAX_TRIANGLES;
constexpr long long kMaxCand = FT_NOALLOC_MAX_CANDIDATES;
constexpr long long kMaxIcells = FT_NOALLOC_MAX_CANDIDATES;
constexpr int kBlocks = 32;  // segments (blocks) of the scan kernels

constexpr size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// byte offsets of each buffer inside the scratch array
constexpr size_t kOffCtr = 0;
constexpr size_t kOffMap = kOffCtr + up256(sizeof(ft_counters));
constexpr size_t kOffTriCnt = kOffMap + up256(sizeof(int) * kMaxCells);
constexpr size_t kOffTriOff = kOffTriCnt + up256(sizeof(int) * kMaxNt);
constexpr size_t kOffTriBox = kOffTriOff + up256(sizeof(int) * kMaxNt);
constexpr size_t kOffTriNrm = kOffTriBox + up256(sizeof(int) * 8 * kMaxNt);
constexpr size_t kOffCandTri = kOffTriNrm + up256(sizeof(double) * 4 * kMaxNt);
constexpr size_t kOffKeys0 = kOffCandTri + up256(sizeof(int) * kMaxCand);
constexpr size_t kOffKeys1 = kOffKeys0 + up256(sizeof(unsigned) * kMaxCand);
constexpr size_t kOffVals0 = kOffKeys1 + up256(sizeof(unsigned) * kMaxCand);
constexpr size_t kOffVals1 = kOffVals0 + up256(sizeof(unsigned) * kMaxCand);
constexpr size_t kOffRec = kOffVals1 + up256(sizeof(unsigned) * kMaxCand);
constexpr size_t kOffCells = kOffRec + up256(sizeof(ft_frag) * kMaxCand);
constexpr size_t kOffCellOff = kOffCells + up256(sizeof(unsigned) * (kMaxIcells + 1));
constexpr size_t kOffCnt = kOffCellOff + up256(sizeof(int) * (kMaxIcells + 1));
constexpr size_t kOffCellL = kOffCnt + up256(sizeof(int) * kMaxCells);
constexpr size_t kOffCellP = kOffCellL + up256(sizeof(double) * kMaxIcells);
constexpr size_t kOffPartials = kOffCellP + up256(sizeof(double) * kMaxIcells);
constexpr size_t kEnd = kOffPartials + up256(sizeof(long long) * (4 * kBlocks + 1));
static_assert(kEnd <= FT_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the static array");

// The scratch itself.  Every device that loads the library holds one copy
// until the process exits.  In host code this name is only a host-side handle:
// its device address comes from cudaGetSymbolAddress (see scratch_on).
static __device__ __align__(256) unsigned char g_scratch[FT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device; it must not run during stream capture).
cudaError_t scratch_on(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

__global__ void k_copy_status(const ft_counters* ctr, unsigned* out) { *out = ctr->status; }

}  // namespace

extern "C" int ft_volume_fraction_noalloc(const ft_grid* g, const ft_front* f, const ft_params* p, double* alpha,
                                          uint32_t* status, void* stream) {
    if (!g || !f || !p || !alpha || !status) return FT_ERR_ARG;
    for (int d = 0; d < 3; d++)
        if (g->n[d] < 1 || !isfinite(g->origin[d])) return FT_ERR_ARG;
    if (!(g->h > 0.0) || !isfinite(g->h) || f->nt < 0 || f->nv < 0) return FT_ERR_ARG;
    if (f->nt > 0 && (!f->verts || !f->tris)) return FT_ERR_ARG;
    if (!(p->delta_max_h >= 0.0) || p->delta_max_h > 7.0) return FT_ERR_ARG;
    const long long ncells = (long long)g->n[0] * g->n[1] * g->n[2];
    if (ncells > kMaxCells || f->nt > kMaxNt) return FT_ERR_CAPACITY;  // beyond the static scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FT_ERR_CUDA;
    unsigned char* base = nullptr;
    if (scratch_on(dev, &base) != cudaSuccess) return FT_ERR_CUDA;

    ft_workspace ws = {};
    ws.device = dev;
    if (cudaDeviceGetAttribute(&ws.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        ws.sm_count < 1)
        return FT_ERR_CUDA;
    ws.grid_blocks = kBlocks;
    ws.tune = ft_tune{4, 4, 16, 8, 4, 0, kBlocks};
    ws.g = *g;
    ws.ncells = ncells;
    ws.max_nt = kMaxNt;
    ws.max_cand = kMaxCand;
    ws.max_cells = kMaxIcells;
    ws.ctr = reinterpret_cast<ft_counters*>(base + kOffCtr);
    ws.idx_map = reinterpret_cast<int*>(base + kOffMap);
    ws.tri_cnt = reinterpret_cast<int*>(base + kOffTriCnt);
    ws.tri_off = reinterpret_cast<int*>(base + kOffTriOff);
    ws.tri_box = reinterpret_cast<int*>(base + kOffTriBox);
    ws.tri_nrm = reinterpret_cast<double*>(base + kOffTriNrm);
    ws.planes = nullptr;  // plane coordinates are computed on the fly here
    ws.cand_tri = reinterpret_cast<int*>(base + kOffCandTri);
    ws.keys[0] = reinterpret_cast<unsigned*>(base + kOffKeys0);
    ws.keys[1] = reinterpret_cast<unsigned*>(base + kOffKeys1);
    ws.vals[0] = reinterpret_cast<unsigned*>(base + kOffVals0);
    ws.vals[1] = reinterpret_cast<unsigned*>(base + kOffVals1);
    ws.rec = reinterpret_cast<ft_frag*>(base + kOffRec);
    ws.cells = reinterpret_cast<unsigned*>(base + kOffCells);
    ws.cell_off = reinterpret_cast<int*>(base + kOffCellOff);
    ws.cell_cnt = reinterpret_cast<int*>(base + kOffCnt);
    ws.cell_L = reinterpret_cast<double*>(base + kOffCellL);
    ws.cell_P = reinterpret_cast<double*>(base + kOffCellP);
    ws.partials = reinterpret_cast<int*>(base + kOffPartials);

    // the scratch holds float64 fragment records only: this call always computes
    // in float64, whatever p->precision asks for
    ft_params p64 = *p;
    p64.precision = FT_FP64;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: reset counters, index map and cell counts
    cudaError_t e = cudaMemsetAsync(ws.ctr, 0, sizeof(ft_counters), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.idx_map, 0xff, sizeof(int) * (size_t)ncells, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.cell_cnt, 0, sizeof(int) * (size_t)ncells, s);
    if (e == cudaSuccess) e = ft::launch_bin(&ws, f, &p64, s);
    if (e == cudaSuccess) e = ft::launch_place_pairs(&ws, ncells, s);
    if (e == cudaSuccess) e = ft::launch_alpha(&ws, alpha, s);
    if (e == cudaSuccess) {
        ft::count_launches(1);
        k_copy_status<<<1, 1, 0, s>>>(ws.ctr, status);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}
