// k_sort.cu -- front_bin, part 2: the (cell key, candidate slot) pairs put
// into cell order by counting, with the interfacial-cell list, its pair
// offsets and the index map (the fragment records follow their slots into
// cell order as each cell is ordered); the per-front cell ranges.
//
// Pair and cell counts live in device memory (no host round trip).  No kernel
// waits on another block: the key-range scan is a reduce launch and a
// down-sweep launch (the down-sweep combines the per-block partials itself).
#include "ft_internal.cuh"

namespace {

constexpr int kB = 256;             // threads per block

__device__ __forceinline__ long long seg_len(long long n, int G) {
    long long s = (n + G - 1) / G;
    return (s + kB - 1) / kB * kB;  // whole tiles per segment
}

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

struct LoadCounts {
    const int* in;
    __device__ long long operator()(long long i) const { return in[i]; }
};

template <class L>
__global__ void __launch_bounds__(kB) k_scan_reduce(L ld, const long long* n_ptr, long long* partials) {
    __shared__ long long sm[kB / 32];
    const long long n = *n_ptr;
    const long long s = seg_len(n, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(n, b0 + s);
    long long acc = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += kB) acc += ld(i);
    long long excl;
    const long long tot = block_excl_scan(acc, excl, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// The down-sweep of the triangle counts: each block sums the reduce partials
// of the blocks before it (gridDim <= kB, one per thread) for its carry; then
// its segment is scanned tile by tile into the candidate offsets, and every
// triangle's candidate slots are filled with its index (when the total fits
// max_cand; block 0 sets the candidate count C, 0 and the capacity flag if not).
__global__ void __launch_bounds__(kB) k_scan_expand(const int* __restrict__ cnt, const long long* n_ptr,
                                                    const long long* __restrict__ partials, int* __restrict__ off,
                                                    long long max_cand, int* __restrict__ cand_tri, ft_counters* ctr) {
    __shared__ long long sm[kB / 32];
    const long long n = *n_ptr;
    const long long s = seg_len(n, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(n, b0 + s);
    long long carry, all;
    {
        const long long p = (threadIdx.x < gridDim.x) ? partials[threadIdx.x] : 0;
        long long excl;
        carry = block_excl_scan((threadIdx.x < blockIdx.x) ? p : 0, excl, sm);
        all = block_excl_scan(p, excl, sm);
    }
    const bool ok = all <= max_cand;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->C_need = all;
        ctr->C = ok ? all : 0;
        if (!ok) ft_flag(ctr, FT_ST_CAPACITY);
    }
    for (long long base = b0; base < b1; base += kB) {
        const long long i = base + threadIdx.x;
        const int v = (i < b1) ? cnt[i] : 0;
        long long excl;
        const long long tot = block_excl_scan(v, excl, sm);
        if (i < b1) {
            const long long o = carry + excl;
            off[i] = (int)o;
            if (ok)
                for (int l = 0; l < v; l++) cand_tri[o + l] = (int)i;
        }
        carry += tot;
    }
}

// ---------------------------------------------------------------------------
// Pairs into cell order by counting.  k_clip counted every kept pair into
// cell_cnt[key]; the atomic's return value, the pair's rank among its cell's
// pairs in arrival order, sits in ranks[slot].  Then:
//  k_cnt_reduce, k_cnt_down -- one exclusive scan over the whole key range of
//    the packed counts (pairs << 32 | has pairs): a key with pairs becomes
//    interfacial cell m with pair offset cell_off[m] (cells, cell_off,
//    idx_map), and its count is replaced by that offset;
//  k_place -- every kept pair to its cell's offset + rank;
//  k_cell_order, k_cell_order_big -- each cell's pairs into ascending slot
//    order, the order of a stable sort by key (pairs are generated in slot
//    order, and slot order is triangle order), each pair's fragment record
//    copied to its place in cell order as soon as it is known; k_cell_order
//    also sets each cell's counter back to zero, so that cell_cnt is all zero
//    again for the next binning.
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
// capacity (k_cell_order_big then flags it and resets M and P).
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
        ctr->big = 0;
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
                    // the count becomes the cell's pair offset, read by k_place and
                    // reset by k_cell_order (zero at once when nothing is placed)
                    cnt[key] = fits ? (int)(run >> 32) : 0;
                }
                run += pack_cnt(c[u]);
            }
        }
        carry += tot;
    }
}

__global__ void __launch_bounds__(kB) k_place(const unsigned* __restrict__ keys, const unsigned* __restrict__ ranks,
                                              const int* __restrict__ cnt, unsigned* __restrict__ skeys,
                                              unsigned* __restrict__ svals, long long max_cells,
                                              const ft_counters* ctr) {
    const long long C = ctr->C;
    if (ctr->M > max_cells) return;
    for (long long c = (long long)blockIdx.x * kB + threadIdx.x; c < C; c += (long long)gridDim.x * kB) {
        const unsigned k = keys[c];
        if (k == FT_SENTINEL) continue;
        const long long dst = (long long)cnt[k] + ranks[c];  // the cell's pair offset (k_cnt_down)
        skeys[dst] = k;
        svals[dst] = (unsigned)c;
    }
}

constexpr int kWarpSlots = 8;  // slots per lane of the warp path: cells of up to 256 pairs

// The pairs of a cell in slot order (slot order is triangle order; slots are
// distinct).  One warp per cell of up to 32 kWarpSlots pairs, each lane
// holding kWarpSlots of them: a pair's place is the number of smaller slots of
// the cell, counted by shuffles, and the warp writes in place.  A larger cell
// goes to a worklist for k_cell_order_big.
// The fragment records in sorted pair order (so that later kernels read a
// cell's fragments as one contiguous range), written by the per-cell ordering
// as soon as a cell's slots are in order; the float centroid entry carries the
// cell's key in w.  srec == NULL: a workspace without sorted copies.
struct Gather {
    const ft_frag* rec;
    const ft_frag32* rec32;
    ft_frag* srec;
    ft_frag32* srec32;
    float4* scen;
    int fp32;
    __device__ __forceinline__ void put(long long q, unsigned slot, unsigned key) const {
        if (fp32) {
            const ft_frag32 f = rec32[slot];
            srec32[q] = f;
            scen[q] = make_float4(f.c[0], f.c[1], f.c[2], __uint_as_float(key));
        } else {
            const ft_frag f = rec[slot];
            srec[q] = f;
            scen[q] = make_float4((float)f.c[0], (float)f.c[1], (float)f.c[2], __uint_as_float(key));
        }
    }
};

__global__ void __launch_bounds__(kB) k_cell_order(const int* __restrict__ cell_off, const unsigned* __restrict__ cells,
                                                   unsigned* __restrict__ svals, int* __restrict__ cnt,
                                                   int* __restrict__ big, long long max_cells, ft_counters* ctr,
                                                   Gather G) {
    const long long M = ctr->M;
    if (M > max_cells) return;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (kB / 32);
    for (long long m = ((long long)blockIdx.x * kB + threadIdx.x) >> 5; m < M; m += nw) {
        const int q0 = cell_off[m], n = cell_off[m + 1] - q0;
        const unsigned key = cells[m];
        if (lane == 0) cnt[key] = 0;  // back to zero for the next binning
        if (n > 32 * kWarpSlots) {
            if (lane == 0) big[atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->big), 1ull)] = (int)m;
            continue;
        }
        unsigned* v = svals + q0;
        if (n <= 32) {  // most cells: one slot per lane
            const unsigned x = (lane < n) ? v[lane] : 0xffffffffu;
            int r = 0;
            for (int o = 0; o < n; o++) r += (__shfl_sync(0xffffffffu, x, o) < x) ? 1 : 0;
            __syncwarp();
            if (lane < n) {
                v[r] = x;
                if (G.srec) G.put(q0 + r, x, key);
            }
            __syncwarp();
            continue;
        }
        const int J = (n + 31) >> 5;  // slots per lane in use (warp-uniform)
        unsigned x[kWarpSlots];
        int r[kWarpSlots];
#pragma unroll
        for (int j = 0; j < kWarpSlots; j++) {
            const int a = lane + 32 * j;
            x[j] = (j < J && a < n) ? v[a] : 0xffffffffu;  // padding sorts after every slot
            r[j] = 0;
        }
#pragma unroll
        for (int jj = 0; jj < kWarpSlots; jj++) {
            if (jj < J) {
                for (int o = 0; o < 32; o++) {
                    const unsigned y = __shfl_sync(0xffffffffu, x[jj], o);
#pragma unroll
                    for (int j = 0; j < kWarpSlots; j++) r[j] += (y < x[j]) ? 1 : 0;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kWarpSlots; j++) {
            const int a = lane + 32 * j;
            if (j < J && a < n) {
                v[r[j]] = x[j];
                if (G.srec) G.put(q0 + r[j], x[j], key);
            }
        }
        __syncwarp();
    }
}

constexpr int kSortCap = 4096;  // slots a block sorts in shared memory at once

// One block per cell of the worklist: chunks of up to kSortCap slots sorted in
// shared memory (bitonic network), then sorted runs merged pairwise through
// tmp (each slot's place: its offset in its run plus, by binary search, the
// number of smaller slots in the partner run).
__global__ void __launch_bounds__(kB) k_cell_order_big(const int* __restrict__ cell_off, unsigned* __restrict__ svals,
                                                       unsigned* __restrict__ tmp, const int* __restrict__ big,
                                                       long long max_cells, ft_counters* ctr,
                                                       const unsigned* __restrict__ cells, Gather G) {
    __shared__ unsigned sh[kSortCap];
    if (ctr->M > max_cells) {
        // the last kernel of the placement: flag the capacity and leave no cells.
        // A block that reads M after this reset finds no worklist (nothing was
        // placed or listed), so the order of the blocks does not matter.
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ft_flag(ctr, FT_ST_CAPACITY);
            ctr->M = 0;
            ctr->P = 0;
        }
        return;
    }
    const long long nbig = ctr->big;
    for (long long w = blockIdx.x; w < nbig; w += gridDim.x) {
        const int m = big[w];
        const int q0 = cell_off[m], n = cell_off[m + 1] - q0;
        unsigned* v = svals + q0;
        for (int c0 = 0; c0 < n; c0 += kSortCap) {
            const int len = min(kSortCap, n - c0);
            int N = 1;
            while (N < len) N <<= 1;
            for (int i = threadIdx.x; i < N; i += kB) sh[i] = (i < len) ? v[c0 + i] : 0xffffffffu;
            __syncthreads();
            for (int k = 2; k <= N; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = threadIdx.x; i < N; i += kB) {
                        const int l = i ^ j;
                        if (l > i) {
                            const unsigned a = sh[i], b = sh[l];
                            if ((a > b) == ((i & k) == 0)) {
                                sh[i] = b;
                                sh[l] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int i = threadIdx.x; i < len; i += kB) v[c0 + i] = sh[i];
            __syncthreads();
        }
        unsigned* src = v;
        unsigned* dst = tmp + q0;
        for (int L = kSortCap; L < n; L <<= 1) {
            for (int i = threadIdx.x; i < n; i += kB) {
                const int a0 = (i / L) * L;  // this slot's run
                const bool left = ((i / L) & 1) == 0;
                const int p0 = left ? a0 : a0 - L;  // the merged pair of runs starts here
                const int b0 = left ? a0 + L : a0 - L;  // the partner run
                const int bl = left ? min(L, n - b0) : L;
                const unsigned x = src[i];
                int lo = 0, hi = bl > 0 ? bl : 0;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (src[b0 + mid] < x)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                dst[p0 + (i - a0) + lo] = x;
            }
            __syncthreads();
            unsigned* sw = src;
            src = dst;
            dst = sw;
        }
        const unsigned key = cells[m];
        for (int i = threadIdx.x; i < n; i += kB) {
            const unsigned x = src[i];
            if (src != v) v[i] = x;
            if (G.srec) G.put(q0 + i, x, key);
        }
        __syncthreads();
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

cudaError_t launch_export_pairs(ft_workspace* ws, long long cap, unsigned* keys, int* tris, cudaStream_t s) {
    count_launches(1);
    k_export_pairs<<<ws->sm_count * 2, kB, 0, s>>>(ws->keys[ws->sorted_buf], ws->vals[ws->sorted_buf], ws->cand_tri,
                                                   cap, keys, tris, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_candidates(ft_workspace* ws, cudaStream_t s) {
    const int G = ws->tune.seg_blocks;
    long long* part = reinterpret_cast<long long*>(ws->partials);
    LoadCounts ld{ws->tri_cnt};
    count_launches(2);
    {
        Trace t(s, "k_scan_reduce");
        k_scan_reduce<<<G, kB, 0, s>>>(ld, &ws->ctr->T, part);
    }
    Trace t(s, "k_scan_expand");
    k_scan_expand<<<G, kB, 0, s>>>(ws->tri_cnt, &ws->ctr->T, part, ws->tri_off, ws->max_cand, ws->cand_tri, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_place_pairs(ft_workspace* ws, long long nkeys, cudaStream_t s) {
    // the key range is read once per scan kernel: four blocks per segment of
    // the tuning (up to 4 grid_blocks partials) keep enough loads in flight
    const int G = 4 * ws->tune.seg_blocks;
    long long* part = reinterpret_cast<long long*>(ws->partials);
    count_launches(5);
    {
        Trace t(s, "k_cnt_reduce");
        k_cnt_reduce<<<G, kB, 0, s>>>(ws->cell_cnt, nkeys, part);
    }
    {
        Trace t(s, "k_cnt_down");
        k_cnt_down<<<G, kB, 0, s>>>(ws->cell_cnt, nkeys, part, ws->cells, ws->cell_off, ws->idx_map, ws->max_cells,
                                    ws->ctr);
    }
    {
        Trace t(s, "k_place");
        k_place<<<ws->sm_count * 4, kB, 0, s>>>(ws->keys[0], ws->vals[0], ws->cell_cnt, ws->keys[1], ws->vals[1],
                                                ws->max_cells, ws->ctr);
    }
    // large cells: the ranks in vals[0] are spent once placed, so that buffer is
    // their merge scratch; cell_L (filled only by the volume fraction) holds the worklist
    int* big = reinterpret_cast<int*>(ws->cell_L);
    // the records follow their slots into cell order (a workspace without sorted
    // copies, as the allocation-free one, reads them through the slot instead)
    const bool gather = ws->srec && ws->srec32 && ws->scen;
    const Gather gat{ws->rec, ws->rec32, gather ? ws->srec : nullptr, ws->srec32, ws->scen,
                     ws->last_precision == FT_FP32C ? 1 : 0};
    {
        Trace t(s, "k_cell_order");
        k_cell_order<<<ws->sm_count * 8, kB, 0, s>>>(ws->cell_off, ws->cells, ws->vals[1], ws->cell_cnt, big,
                                                     ws->max_cells, ws->ctr, gat);
    }
    {
        Trace t(s, "k_cell_order_big");
        k_cell_order_big<<<ws->sm_count * 2, kB, 0, s>>>(ws->cell_off, ws->vals[1], ws->vals[0], big, ws->max_cells,
                                                         ws->ctr, ws->cells, gat);
    }
    ws->sorted_buf = 1;
    return cudaGetLastError();
}

cudaError_t launch_cell_ranges(ft_workspace* ws, long long* off, cudaStream_t s) {
    count_launches(1);
    k_cell_ranges<<<(ws->nf + 1 + kB - 1) / kB, kB, 0, s>>>(ws->cells, ws->fbase, ws->nf, off, ws->ctr);
    return cudaGetLastError();
}

}  // namespace ft
