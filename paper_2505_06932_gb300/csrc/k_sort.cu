// k_sort.cu -- front_bin, part 2: device-wide exclusive scans, the stable LSD
// radix sort of the (cell key, candidate slot) pairs and the run-length
// encoding into the interfacial-cell list.
//
// Element counts live in device memory (no host round trip), so every kernel
// here splits its range into gridDim.x contiguous segments computed on the
// device.  No kernel waits on another block: a scan is a reduce launch and a
// down-sweep launch, a radix pass a histogram launch and a scatter launch (the
// down-sweep and the scatter each combine the per-block partials themselves).
#include "ft_internal.cuh"

namespace {

constexpr int kB = 256;             // threads per block
constexpr int kKPT = 4;             // keys per thread and tile of the radix scatter
constexpr int kTile = kKPT * kB;    // keys per tile
constexpr int kRows = kKPT * (kB / 32);  // (row, warp) pairs of a tile

__device__ __forceinline__ long long seg_len(long long n, int G) {
    long long s = (n + G - 1) / G;
    return (s + kB - 1) / kB * kB;  // whole tiles per segment
}

// exclusive block scan of one int per thread; returns the block total
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
struct LoadHeads {
    const unsigned* keys;
    __device__ long long operator()(long long i) const { return (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0; }
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

// The down-sweep: each block sums the reduce partials of the blocks before it
// (gridDim <= kB, one per thread) for its carry, block 0 also writes the total;
// then its segment is scanned tile by tile.
template <class L>
__global__ void __launch_bounds__(kB) k_scan_down(L ld, const long long* n_ptr, const long long* partials,
                                                  int* out, long long* total) {
    __shared__ long long sm[kB / 32];
    const long long n = *n_ptr;
    const long long s = seg_len(n, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(n, b0 + s);
    long long carry;
    {
        const long long p = (threadIdx.x < gridDim.x) ? partials[threadIdx.x] : 0;
        long long excl;
        carry = block_excl_scan((threadIdx.x < blockIdx.x) ? p : 0, excl, sm);
        const long long all = block_excl_scan(p, excl, sm);
        if (blockIdx.x == 0 && threadIdx.x == 0) *total = all;
    }
    for (long long base = b0; base < b1; base += kB) {
        const long long i = base + threadIdx.x;
        const long long v = (i < b1) ? ld(i) : 0;
        long long excl;
        const long long tot = block_excl_scan(v, excl, sm);
        if (i < b1) out[i] = (int)(carry + excl);
        carry += tot;
    }
}

// ---------------------------------------------------------------------------
// radix sort: 8-bit digits, stable, segment per block
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kB) k_radix_hist(const unsigned* __restrict__ keys, const long long* n_ptr,
                                                   int shift, int* __restrict__ hist) {
    __shared__ int h[256];
    const long long n = *n_ptr;
    const long long s = seg_len(n, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(n, b0 + s);
    h[threadIdx.x] = 0;
    __syncthreads();
    long long i = b0 + threadIdx.x;
    for (; i + 3 * kB < b1; i += 4 * kB) {  // four loads in flight
        unsigned k[4];
#pragma unroll
        for (int u = 0; u < 4; u++) k[u] = keys[i + u * kB];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (k[u] != FT_SENTINEL) atomicAdd(&h[(k[u] >> shift) & 255u], 1);
    }
    for (; i < b1; i += kB) {
        const unsigned k = keys[i];
        if (k != FT_SENTINEL) atomicAdd(&h[(k >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];  // block-major (coalesced)
}

// Stable scatter: each block walks its segment in tiles of kTile keys in
// order; a key's destination is the digit's offset for this block + the count
// of the same digit earlier in the segment (earlier tiles, then earlier places
// in its own tile).
__global__ void __launch_bounds__(kB) k_radix_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                                                      unsigned* __restrict__ kout, unsigned* __restrict__ vout,
                                                      const long long* n_ptr, int shift,
                                                      const int* __restrict__ hist, long long* total) {
    __shared__ int base[256];
    __shared__ __align__(16) int wcnt[kRows][256];
    const long long n = *n_ptr;
    const long long s = seg_len(n, gridDim.x);
    const long long b0 = blockIdx.x * s, b1 = min(n, b0 + s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        // this block's offset for digit d = threadIdx.x: the keys of all smaller
        // digits plus the keys of digit d in earlier segments, from the
        // block-major histogram (one coalesced row per segment) and a block scan
        // of the digit totals
        // thread t adds four digits (4 (t % 64) ...) over the rows j = t / 64 mod 4
        // with 16-byte loads; the four row phases are then combined
        {
            const int ph = threadIdx.x >> 6, d4 = threadIdx.x & 63;
            int4 t4 = make_int4(0, 0, 0, 0), b4 = make_int4(0, 0, 0, 0);
            const int G = (int)gridDim.x, bid = (int)blockIdx.x;
            const int4* __restrict__ h4 = reinterpret_cast<const int4*>(hist) + d4;
            auto add = [&](const int4 c, int j) {
                t4.x += c.x;
                t4.y += c.y;
                t4.z += c.z;
                t4.w += c.w;
                if (j < bid) {
                    b4.x += c.x;
                    b4.y += c.y;
                    b4.z += c.z;
                    b4.w += c.w;
                }
            };
            int j = ph;
            for (; j + 60 < G; j += 64) {  // sixteen rows of this phase in flight together
                int4 c[16];
#pragma unroll
                for (int u = 0; u < 16; u++) c[u] = h4[(j + 4 * u) * 64];
#pragma unroll
                for (int u = 0; u < 16; u++) add(c[u], j + 4 * u);
            }
            for (; j + 28 < G; j += 32) {  // then eight
                int4 c[8];
#pragma unroll
                for (int u = 0; u < 8; u++) c[u] = h4[(j + 4 * u) * 64];
#pragma unroll
                for (int u = 0; u < 8; u++) add(c[u], j + 4 * u);
            }
            for (; j < G; j += 4) add(h4[j * 64], j);
            reinterpret_cast<int4*>(&wcnt[ph][0])[d4] = t4;
            reinterpret_cast<int4*>(&wcnt[4 + ph][0])[d4] = b4;
        }
        __syncthreads();
        int tot = 0, before = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            tot += wcnt[q][threadIdx.x];
            before += wcnt[4 + q][threadIdx.x];
        }
        __syncthreads();
        int x = tot;  // inclusive scan over the digits
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wcnt[0][w] = x;
        __syncthreads();
        int wbase = 0;
        for (int q = 0; q < w; q++) wbase += wcnt[0][q];
        const int excl = wbase + x - tot;
        base[threadIdx.x] = excl + before;
        if (blockIdx.x == 0 && threadIdx.x == kB - 1) *total = excl + tot;
        __syncthreads();
    }
    // Tiles of kTile = kKPT x 256 keys.  Row j of a tile is the 256 keys
    // t0 + 256 j + threadIdx.x (coalesced); a key's place in the tile is
    // (row, warp, lane), and its rank among the tile's keys of its digit counts
    // the earlier (row, warp) pairs and the lower lanes of its own.  Four rows
    // per tile cut the barriers per key fourfold.  The next tile's keys and
    // values are loaded while this one is ranked.
    unsigned kn[kKPT], vn[kKPT];
#pragma unroll
    for (int j = 0; j < kKPT; j++) {
        const long long i = b0 + j * kB + threadIdx.x;
        kn[j] = (i < b1) ? kin[i] : FT_SENTINEL;
        vn[j] = (i < b1) ? vin[i] : 0u;
    }
    for (long long t0 = b0; t0 < b1; t0 += kTile) {
        unsigned k[kKPT], v[kKPT];
#pragma unroll
        for (int j = 0; j < kKPT; j++) {
            k[j] = kn[j];
            v[j] = vn[j];
            const long long i = t0 + kTile + j * kB + threadIdx.x;
            kn[j] = (i < b1) ? kin[i] : FT_SENTINEL;
            vn[j] = (i < b1) ? vin[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kRows; r++) wcnt[r][threadIdx.x] = 0;
        __syncthreads();
        unsigned dig[kKPT];
        int rank[kKPT];
#pragma unroll
        for (int j = 0; j < kKPT; j++) {
            const bool valid = (k[j] != FT_SENTINEL);
            dig[j] = valid ? ((k[j] >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, dig[j]);
            rank[j] = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank[j] == 0) wcnt[j * (kB / 32) + w][dig[j]] = __popc(peers);
        }
        __syncthreads();
        // per digit (thread = digit): exclusive prefix over the (row, warp) pairs
        int run = 0;
#pragma unroll 8
        for (int r = 0; r < kRows; r++) {
            const int c = wcnt[r][threadIdx.x];
            wcnt[r][threadIdx.x] = run;
            run += c;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kKPT; j++) {
            if (dig[j] < 256u) {
                const int dst = base[dig[j]] + wcnt[j * (kB / 32) + w][dig[j]] + rank[j];
                kout[dst] = k[j];
                vout[dst] = v[j];
            }
        }
        __syncthreads();
        base[threadIdx.x] += run;  // the tile's keys of this digit; read after the next tile's first barrier
    }
}

// run-length encoding of the sorted keys: cells[m], cell_off[m], idx_map.
// Writes nothing when M exceeds the capacity (k_cap_cells then resets M).
__global__ void __launch_bounds__(kB) k_rle(const unsigned* __restrict__ keys, const int* __restrict__ head_idx,
                                            unsigned* __restrict__ cells, int* __restrict__ cell_off,
                                            int* __restrict__ idx_map, long long max_cells, const ft_counters* ctr) {
    const long long P = ctr->P;
    const long long M = ctr->M;  // computed by the head scan
    if (M > max_cells) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) cell_off[M] = (int)P;
    for (long long q = (long long)blockIdx.x * kB + threadIdx.x; q < P; q += (long long)gridDim.x * kB) {
        const unsigned k = keys[q];
        if (q == 0 || keys[q - 1] != k) {
            const int m = head_idx[q];
            cells[m] = k;
            cell_off[m] = (int)q;
            idx_map[k] = m;
        }
    }
}

__global__ void k_cap_cells(long long max_cells, ft_counters* ctr) {
    if (ctr->M > max_cells) {
        ft_flag(ctr, FT_ST_CAPACITY);
        ctr->M = 0;
        ctr->P = 0;
    }
}

// reset the index map entries of the previous bins
__global__ void __launch_bounds__(kB) k_clear_map(const unsigned* __restrict__ cells, int* __restrict__ idx_map,
                                                  const ft_counters* ctr) {
    const long long M = ctr->M;
    for (long long m = (long long)blockIdx.x * kB + threadIdx.x; m < M; m += (long long)gridDim.x * kB)
        idx_map[cells[m]] = -1;
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

cudaError_t launch_scan_counts(ft_workspace* ws, const int* in, int* out, const long long* n, long long* total,
                               cudaStream_t s) {
    const int G = ws->tune.seg_blocks;
    long long* part = reinterpret_cast<long long*>(ws->partials);
    LoadCounts ld{in};
    count_launches(2);
    k_scan_reduce<<<G, kB, 0, s>>>(ld, n, part);
    k_scan_down<<<G, kB, 0, s>>>(ld, n, part, out, total);
    return cudaGetLastError();
}

cudaError_t launch_scan_heads(ft_workspace* ws, const unsigned* keys, int* out, const long long* n,
                              long long* total, cudaStream_t s) {
    const int G = ws->tune.seg_blocks;
    long long* part = reinterpret_cast<long long*>(ws->partials);
    LoadHeads ld{keys};
    count_launches(2);
    k_scan_reduce<<<G, kB, 0, s>>>(ld, n, part);
    k_scan_down<<<G, kB, 0, s>>>(ld, n, part, out, total);
    return cudaGetLastError();
}

cudaError_t prepare_sort(int grid_blocks) {
    (void)grid_blocks;  // no kernel of the sort needs more than the default shared memory
    return cudaSuccess;
}

cudaError_t launch_sort(ft_workspace* ws, cudaStream_t s) {
    const int G = ws->tune.seg_blocks;
    const int passes = (ws->key_bits + 7) / 8;
    int src = 0;
    for (int p = 0; p < passes; p++) {
        // pass 0 reads the candidates (sentinels dropped) and counts the pairs
        const long long* n = (p == 0) ? &ws->ctr->C : &ws->ctr->P;
        long long* tot = (p == 0) ? &ws->ctr->P : &ws->ctr->scratch;
        count_launches(2);
        k_radix_hist<<<G, kB, 0, s>>>(ws->keys[src], n, 8 * p, ws->hist);
        k_radix_scatter<<<G, kB, 0, s>>>(ws->keys[src], ws->vals[src], ws->keys[src ^ 1], ws->vals[src ^ 1], n,
                                         8 * p, ws->hist, tot);
        src ^= 1;
    }
    ws->sorted_buf = src;
    return cudaGetLastError();
}

cudaError_t launch_rle(ft_workspace* ws, cudaStream_t s) {
    const unsigned* keys = ws->keys[ws->sorted_buf];
    cudaError_t e = launch_scan_heads(ws, keys, ws->heads, &ws->ctr->P, &ws->ctr->M, s);
    if (e != cudaSuccess) return e;
    count_launches(2);
    k_rle<<<ws->sm_count * 2, kB, 0, s>>>(keys, ws->heads, ws->cells, ws->cell_off, ws->idx_map, ws->max_cells,
                                          ws->ctr);
    k_cap_cells<<<1, 1, 0, s>>>(ws->max_cells, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_cell_ranges(ft_workspace* ws, long long* off, cudaStream_t s) {
    count_launches(1);
    k_cell_ranges<<<(ws->nf + 1 + kB - 1) / kB, kB, 0, s>>>(ws->cells, ws->fbase, ws->nf, off, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_clear_map(ft_workspace* ws, cudaStream_t s) {
    count_launches(1);
    k_clear_map<<<ws->sm_count * 2, kB, 0, s>>>(ws->cells, ws->idx_map, ws->ctr);
    return cudaGetLastError();
}

}  // namespace ft
