// k_sort.cu -- front_bin, part 2: the (cell key, candidate slot) pairs put
// into cell order by counting, with the interfacial-cell list, its pair
// offsets and the index map; the record gather and the per-front cell ranges.
//
// Pair and cell counts live in device memory (no host round trip).  No kernel
// waits on another block: the key-range scan is a reduce launch and a
// down-sweep launch (the down-sweep combines the per-block partials itself).
#include "ft_internal.cuh"

namespace {

constexpr int kB = 256;             // threads per block

// exclusive block scan of one value per thread; returns the block total
__device__ __forceinline__ long long block_excl_scan(long long v, long long& excl, long long* sm_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = (lane < kB / 32) ? sm_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kB / 32) sm_warp[lane] = t;
    }
    __syncthreads();
    const long long before = (w > 0) ? sm_warp[w - 1] : 0;
    const long long total = sm_warp[kB / 32 - 1];
    excl = before + x - v;
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// Pairs into cell order by counting.  k_clip counted every kept pair into
// cell_cnt[key]; the atomic's return value, the pair's rank among its cell's
// pairs in arrival order, sits in ranks[slot].  Then:
//  k_cnt_reduce, k_cnt_down -- one exclusive scan over the whole key range of
//    the packed counts (pairs << 32 | has pairs): a key with pairs becomes
//    interfacial cell m with pair offset cell_off[m] (cells, cell_off,
//    idx_map), and its count goes back to zero, so that cell_cnt is all zero
//    again for the next binning;
//  k_place -- every kept pair to cell_off[m] + rank;
//  k_cell_order -- each cell's pairs into ascending triangle order (the
//    candidate ranges of the triangles are laid out in any order).
// ---------------------------------------------------------------------------

__device__ __forceinline__ long long pack_cnt(int c) { return ((long long)c << 32) | (c > 0 ? 1 : 0); }

constexpr int kKeysPT = 16;  // keys per thread and tile of the key-range scan (four 16-byte loads in flight)

// segment of the key range per block: whole tiles of kKeysPT keys per thread
__device__ __forceinline__ long long key_seg(long long n, int G) {
    const long long s = (n + G - 1) / G;
    return (s + kKeysPT * kB - 1) / (kKeysPT * kB) * (kKeysPT * kB);
}

// this thread's counts of a tile: keys i .. i + kKeysPT - 1 (i a multiple of 4;
// the array is 16-byte aligned), zeros past b1
__device__ __forceinline__ void load_cnt_tile(const int* __restrict__ cnt, long long i, long long b1,
                                              int (&c)[kKeysPT]) {
#pragma unroll
    for (int u = 0; u < kKeysPT / 4; u++) {
        const long long k = i + 4 * u;
        int4 v = make_int4(0, 0, 0, 0);
        if (k + 3 < b1) {
            v = *reinterpret_cast<const int4*>(cnt + k);
        } else {
            if (k < b1) v.x = cnt[k];
            if (k + 1 < b1) v.y = cnt[k + 1];
            if (k + 2 < b1) v.z = cnt[k + 2];
        }
        c[4 * u] = v.x;
        c[4 * u + 1] = v.y;
        c[4 * u + 2] = v.z;
        c[4 * u + 3] = v.w;
    }
}

__global__ void __launch_bounds__(kB) k_cnt_reduce(const int* __restrict__ cnt, long long nkeys,
                                                   long long* __restrict__ partials) {
    __shared__ long long sm[kB / 32];
    const long long s = key_seg(nkeys, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(nkeys, b0 + s);
    long long acc = 0;
    for (long long i = b0 + kKeysPT * threadIdx.x; i < b1; i += kKeysPT * kB) {
        int c[kKeysPT];
        load_cnt_tile(cnt, i, b1, c);
#pragma unroll
        for (int u = 0; u < kKeysPT; u++) acc += pack_cnt(c[u]);
    }
    long long excl;
    const long long tot = block_excl_scan(acc, excl, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Writes nothing but the totals and the count reset when M exceeds the
// capacity (k_cap_cells then flags it and resets M and P).
__global__ void __launch_bounds__(kB) k_cnt_down(int* __restrict__ cnt, long long nkeys,
                                                 const long long* __restrict__ partials, unsigned* __restrict__ cells,
                                                 int* __restrict__ cell_off, int* __restrict__ idx_map,
                                                 long long max_cells, ft_counters* ctr) {
    __shared__ long long sm[kB / 32];
    const long long s = key_seg(nkeys, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(nkeys, b0 + s);
    long long carry, all;
    {
        // the partials of the blocks before this one (gridDim.x may exceed kB)
        long long pc = 0, pa = 0;
        for (int t = threadIdx.x; t < (int)gridDim.x; t += kB) {
            const long long p = partials[t];
            pa += p;
            if (t < (int)blockIdx.x) pc += p;
        }
        long long excl;
        carry = block_excl_scan(pc, excl, sm);
        all = block_excl_scan(pa, excl, sm);
    }
    const long long P = all >> 32, M = all & 0xffffffffLL;
    const bool fits = M <= max_cells;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->P = P;
        ctr->M = M;
        if (fits) cell_off[M] = (int)P;
    }
    for (long long base = b0; base < b1; base += kKeysPT * kB) {
        const long long i = base + kKeysPT * threadIdx.x;
        int c[kKeysPT];
        load_cnt_tile(cnt, i, b1, c);
        long long mine = 0;
#pragma unroll
        for (int u = 0; u < kKeysPT; u++) mine += pack_cnt(c[u]);
        long long excl;
        const long long tot = block_excl_scan(mine, excl, sm);
        if (mine != 0) {  // keys with pairs are rare: most threads skip the walk
            long long run = carry + excl;
#pragma unroll
            for (int u = 0; u < kKeysPT; u++) {
                if (c[u] > 0) {
                    const long long key = i + u;
                    if (fits) {
                        const int m = (int)(run & 0xffffffffLL);
                        cells[m] = (unsigned)key;
                        cell_off[m] = (int)(run >> 32);
                        idx_map[key] = m;
                    }
                    cnt[key] = 0;
                }
                run += pack_cnt(c[u]);
            }
        }
        carry += tot;
    }
}

__global__ void __launch_bounds__(kB) k_place(const unsigned* __restrict__ keys, const unsigned* __restrict__ ranks,
                                              const int* __restrict__ idx_map, const int* __restrict__ cell_off,
                                              unsigned* __restrict__ skeys, unsigned* __restrict__ svals,
                                              long long max_cells, const ft_counters* ctr) {
    const long long C = ctr->C;
    if (ctr->M > max_cells) return;
    for (long long c = (long long)blockIdx.x * kB + threadIdx.x; c < C; c += (long long)gridDim.x * kB) {
        const unsigned k = keys[c];
        if (k == FT_SENTINEL) continue;
        const long long dst = (long long)cell_off[idx_map[k]] + ranks[c];
        skeys[dst] = k;
        svals[dst] = (unsigned)c;
    }
}

// One warp per cell puts the cell's pairs in triangle order (a triangle meets
// a cell at most once, so the triangles of a cell are distinct): a pair's
// place is the number of pairs of the cell with a smaller triangle.  Up to 32
// pairs the lanes hold them and count by shuffles, then write in place; a
// larger cell is ranked from memory into tmp and copied back.
__global__ void __launch_bounds__(kB) k_cell_order(const int* __restrict__ cell_off, unsigned* __restrict__ svals,
                                                   const int* __restrict__ cand_tri, unsigned* __restrict__ tmp,
                                                   long long max_cells, const ft_counters* ctr) {
    const long long M = ctr->M;
    if (M > max_cells) return;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (kB / 32);
    for (long long m = ((long long)blockIdx.x * kB + threadIdx.x) >> 5; m < M; m += nw) {
        const int q0 = cell_off[m], n = cell_off[m + 1] - q0;
        if (n <= 1) continue;
        unsigned* v = svals + q0;
        if (n <= 32) {
            const unsigned x = (lane < n) ? v[lane] : 0u;
            const int tr = (lane < n) ? cand_tri[x] : 0x7fffffff;
            int r = 0;
            for (int o = 0; o < n; o++) r += (__shfl_sync(0xffffffffu, tr, o) < tr) ? 1 : 0;
            __syncwarp();
            if (lane < n) v[r] = x;
        } else {
            unsigned* t = tmp + q0;
            for (int a = lane; a < n; a += 32) {
                const unsigned x = v[a];
                const int tr = cand_tri[x];
                int r = 0;
                for (int b = 0; b < n; b++) r += (cand_tri[v[b]] < tr) ? 1 : 0;
                t[r] = x;
            }
            __syncwarp();
            for (int a = lane; a < n; a += 32) v[a] = t[a];
        }
        __syncwarp();
    }
}

__global__ void k_cap_cells(long long max_cells, ft_counters* ctr) {
    if (ctr->M > max_cells) {
        ft_flag(ctr, FT_ST_CAPACITY);
        ctr->M = 0;
        ctr->P = 0;
    }
}

__global__ void __launch_bounds__(kB) k_export_pairs(const unsigned* __restrict__ skeys, const unsigned* __restrict__ svals,
                                                     const int* __restrict__ cand_tri, long long cap,
                                                     unsigned* __restrict__ keys, int* __restrict__ tris,
                                                     ft_counters* ctr) {
    const long long P = ctr->P;
    if (P > cap && blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
    const long long n = P < cap ? P : cap;
    for (long long q = (long long)blockIdx.x * kB + threadIdx.x; q < n; q += (long long)gridDim.x * kB) {
        keys[q] = skeys[q];
        tris[q] = cand_tri[svals[q]];
    }
}

// fragment records in sorted pair order, so later kernels read a cell's
// fragments as one contiguous range (no indirection through the slot)
__global__ void __launch_bounds__(kB) k_gather(const unsigned* __restrict__ svals, const ft_frag* __restrict__ rec,
                                               const ft_frag32* __restrict__ rec32, ft_frag* __restrict__ srec,
                                               ft_frag32* __restrict__ srec32, float4* __restrict__ scen, int fp32,
                                               const ft_counters* ctr) {
    const long long P = ctr->P;
    for (long long q = (long long)blockIdx.x * kB + threadIdx.x; q < P; q += (long long)gridDim.x * kB) {
        const unsigned c = svals[q];
        if (fp32) {
            const ft_frag32 f = rec32[c];
            srec32[q] = f;
            scen[q] = make_float4(f.c[0], f.c[1], f.c[2], 0.f);
        } else {
            const ft_frag f = rec[c];
            srec[q] = f;
            scen[q] = make_float4((float)f.c[0], (float)f.c[1], (float)f.c[2], 0.f);
        }
    }
}

// Batched form: off[f] = first interfacial cell of front f in the sorted cell
// list (the cells of front f are the keys in [key_base[f], key_base[f+1])),
// off[nf] = M.
__global__ void __launch_bounds__(kB) k_cell_ranges(const unsigned* __restrict__ cells,
                                                    const long long* __restrict__ key_base, int nf,
                                                    long long* __restrict__ off, const ft_counters* ctr) {
    const int f = blockIdx.x * kB + threadIdx.x;
    if (f > nf) return;
    const long long M = ctr->M;
    const long long kf = key_base[f];
    long long lo = 0, hi = M;  // first index with cells[i] >= kf
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)cells[mid] < kf)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[f] = lo;
}

}  // namespace

namespace ft {

cudaError_t launch_gather(ft_workspace* ws, cudaStream_t s) {
    if (!ws->srec || !ws->srec32 || !ws->scen) return cudaSuccess;  // a workspace without sorted copies
    count_launches(1);
    k_gather<<<ws->sm_count * 4, kB, 0, s>>>(ws->vals[ws->sorted_buf], ws->rec, ws->rec32, ws->srec, ws->srec32,
                                             ws->scen, ws->last_precision == FT_FP32C ? 1 : 0, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_export_pairs(ft_workspace* ws, long long cap, unsigned* keys, int* tris, cudaStream_t s) {
    count_launches(1);
    k_export_pairs<<<ws->sm_count * 2, kB, 0, s>>>(ws->keys[ws->sorted_buf], ws->vals[ws->sorted_buf], ws->cand_tri,
                                                   cap, keys, tris, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_place_pairs(ft_workspace* ws, long long nkeys, cudaStream_t s) {
    // the key range is read once per scan kernel: four blocks per segment of
    // the tuning (up to 4 grid_blocks partials) keep enough loads in flight
    const int G = 4 * ws->tune.seg_blocks;
    long long* part = reinterpret_cast<long long*>(ws->partials);
    count_launches(5);
    k_cnt_reduce<<<G, kB, 0, s>>>(ws->cell_cnt, nkeys, part);
    k_cnt_down<<<G, kB, 0, s>>>(ws->cell_cnt, nkeys, part, ws->cells, ws->cell_off, ws->idx_map, ws->max_cells,
                                ws->ctr);
    k_place<<<ws->sm_count * 4, kB, 0, s>>>(ws->keys[0], ws->vals[0], ws->idx_map, ws->cell_off, ws->keys[1],
                                            ws->vals[1], ws->max_cells, ws->ctr);
    // the ranks in vals[0] are spent once placed: that buffer is the scratch of large cells
    k_cell_order<<<ws->sm_count * 8, kB, 0, s>>>(ws->cell_off, ws->vals[1], ws->cand_tri, ws->vals[0], ws->max_cells,
                                                 ws->ctr);
    k_cap_cells<<<1, 1, 0, s>>>(ws->max_cells, ws->ctr);
    ws->sorted_buf = 1;
    return cudaGetLastError();
}

cudaError_t launch_cell_ranges(ft_workspace* ws, long long* off, cudaStream_t s) {
    count_launches(1);
    k_cell_ranges<<<(ws->nf + 1 + kB - 1) / kB, kB, 0, s>>>(ws->cells, ws->fbase, ws->nf, off, ws->ctr);
    return cudaGetLastError();
}

}  // namespace ft
