// k_csf.cu -- front_csf_force: S_P = sigma kappa_P grad alpha_P (Eq. csf) with
// the weighted curvature smoothing of Sec. 3.3 in cells next to the interface:
// kbar_P = sum_Q kappa_Q w_Q / sum_Q w_Q, w_Q = |s_Q . n_Q| / |s_Q|, over the
// interfacial cells Q among the 26 neighbours of P (plain mean if all w_Q = 0).
//
// Only cells next to the interface carry a force: grad alpha_P != 0 needs
// alpha_{P+e} != alpha_{P-e} along some axis, and two full/empty cells on
// either side differ only if the front passes through P; so P is interfacial
// or a face neighbour of an interfacial cell.  Hence:
//  * the force arrays are zeroed (a memset, or k_zero_force for a batch);
//  * k_csf_ring_list -- six threads per interfacial cell, each looking at one
//    face neighbour and listing it as a ring cell when it is not interfacial
//    and this cell is the smallest-key interfacial face neighbour it has (so
//    it is listed once); it needs only the binning, so a caller may run it
//    beside the PPIC fit (front_csf_prepare);
//  * k_csf_force -- one thread per interfacial cell (its force sigma kappa
//    grad alpha, central differences, alpha = 0 outside the grid) and per ring
//    cell (the smoothed curvature and the force), in one launch.
#include <type_traits>

#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;  // one block per column; 128 and 256 cell columns fill it

// Compact force output (one front): the interfacial cells first (slot m = the
// cell's row of front_curvature_ppic), then the ring cells; keys == NULL
// selects the dense force arrays of the front descriptor.
struct CsfOut {
    unsigned* keys;
    double* f;        // 3 per slot (x, y, z)
    long long cap;
    long long* count;
};

// zero the force arrays of every front (the batched form).  A block clears a
// tile of 8 x 128 consecutive cells of the batch-wide cell index (one front
// search per tile, then a step to the next front where the tile crosses one),
// each warp storing 3 x 256 contiguous bytes per row of the tile.
template <class F>
__global__ void __launch_bounds__(kThreads) k_zero_force(F fr) {
    constexpr int kTile = 8 * kThreads;
    const long long total = fr.ncells;
    for (long long t0 = (long long)blockIdx.x * kTile; t0 < total; t0 += (long long)gridDim.x * kTile) {
        int b = fr.by_key(t0);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const long long g = t0 + i * kThreads + threadIdx.x;
            if (g >= total) break;
            while (g >= fr.key_base(b + 1)) b++;
            const ft_fdesc& D = fr.desc(b);
            const long long NC = (long long)D.g.n[0] * D.g.n[1] * D.g.n[2];
            const long long c = g - fr.key_base(b);
            double* __restrict__ force = D.force;
            force[c] = 0.0;
            force[NC + c] = 0.0;
            force[2 * NC + c] = 0.0;
        }
    }
}

// Six tasks per interfacial cell (one thread each): task e looks at the face
// neighbour e and lists it as a ring cell when it is not interfacial and this
// cell is its smallest-key interfacial face neighbour (so that it is listed
// once).  Needs only the binning.
template <class F>
__global__ void __launch_bounds__(kThreads) k_csf_ring_list(F fr, const unsigned* __restrict__ cells,
                                                            const int* __restrict__ idx_map,
                                                            unsigned* __restrict__ ring, unsigned* __restrict__ nring,
                                                            long long ring_cap, ft_counters* ctr) {
    const long long M = ctr->M;
    for (long long w = (long long)blockIdx.x * kThreads + threadIdx.x; w < 6 * M; w += (long long)gridDim.x * kThreads) {
        const long long m = w / 6;
        const int e = (int)(w - 6 * m);
        const long long gkey = cells[m];
        const int b = fr.by_key(gkey);
        const ft_fdesc& D = fr.desc(b);
        const unsigned n0 = (unsigned)D.g.n[0], n1 = (unsigned)D.g.n[1], n2 = (unsigned)D.g.n[2];
        const long long kb = fr.key_base(b);
        const unsigned key = (unsigned)(gkey - kb);  // a front's keys fit 32 bits
        const unsigned col = key / n2, k = key - col * n2;
        const unsigned i = col / n1, j = col - i * n1;
        const long long s0 = (long long)n1 * n2, s1 = n2;
        const int c[3] = {(int)i, (int)j, (int)k}, n[3] = {(int)n0, (int)n1, (int)n2};
        const long long st[3] = {s0, s1, 1};
        const int ax = e >> 1, sg = (e & 1) ? -1 : 1;
        if (c[ax] + sg < 0 || c[ax] + sg >= n[ax]) continue;
        const long long q = (long long)key + sg * st[ax];
        if (idx_map[kb + q] >= 0) continue;
        // the interfacial face neighbours of q: is this cell the smallest key?
        bool own = true;
        int cq[3] = {c[0], c[1], c[2]};
        cq[ax] += sg;
        for (int e2 = 0; e2 < 6 && own; e2++) {
            const int ax2 = e2 >> 1, sg2 = (e2 & 1) ? -1 : 1;
            if (cq[ax2] + sg2 < 0 || cq[ax2] + sg2 >= n[ax2]) continue;
            const long long r = q + sg2 * st[ax2];
            if (r < (long long)key && idx_map[kb + r] >= 0) own = false;
        }
        if (!own) continue;
        const unsigned pos = atomicAdd(nring, 1u);
        if (pos < ring_cap)
            ring[pos] = (unsigned)(kb + q);
        else
            ft_flag(ctr, FT_ST_CAPACITY);
    }
}

// The force of interfacial cell m: sigma kappa_m grad alpha (central
// differences, alpha = 0 outside the grid), into slot m or the dense arrays.
template <class F>
__device__ __forceinline__ void cell_force(const F& fr, double sigma, const unsigned* __restrict__ cells,
                                           const double* __restrict__ kappa, long long m, const CsfOut& out) {
    const long long gkey = cells[m];
    const int b = fr.by_key(gkey);
    const ft_fdesc& D = fr.desc(b);
    const unsigned n0 = (unsigned)D.g.n[0], n1 = (unsigned)D.g.n[1], n2 = (unsigned)D.g.n[2];
    const long long kb = fr.key_base(b);
    const unsigned key = (unsigned)(gkey - kb);
    const unsigned col = key / n2, k = key - col * n2;
    const unsigned i = col / n1, j = col - i * n1;
    const long long s0 = (long long)n1 * n2, s1 = n2;
    const int c[3] = {(int)i, (int)j, (int)k}, n[3] = {(int)n0, (int)n1, (int)n2};
    const long long st[3] = {s0, s1, 1};
    const long long NC = (long long)n0 * n1 * n2;
    const double* __restrict__ alpha = D.alpha;
    double a[6];
#pragma unroll
    for (int e = 0; e < 6; e++) {
        const int ax = e >> 1, sg = (e & 1) ? -1 : 1;
        a[e] = (c[ax] + sg >= 0 && c[ax] + sg < n[ax]) ? alpha[key + sg * st[ax]] : 0.0;
    }
    const double ih2 = 0.5 * D.inv_h;
    const double f = sigma * kappa[m];
    const double fx = f * ((a[0] - a[1]) * ih2), fy = f * ((a[2] - a[3]) * ih2), fz = f * ((a[4] - a[5]) * ih2);
    if (out.keys) {
        if (m < out.cap) {
            out.keys[m] = key;
            out.f[3 * m] = fx;
            out.f[3 * m + 1] = fy;
            out.f[3 * m + 2] = fz;
        }
    } else {
        double* __restrict__ force = D.force;
        force[key] = fx;
        force[NC + key] = fy;
        force[2 * NC + key] = fz;
    }
}

// The force of ring cell r (slot M + r): the smoothed curvature over its
// interfacial neighbours times sigma grad alpha.  The 26 index-map lookups are
// issued together (independent loads) before the float64 smoothing sums, which
// then run once per cell instead of once per lane of a warp-wide reduction.
template <class F>
__device__ __forceinline__ void ring_force(const F& fr, double sigma, const int* __restrict__ idx_map,
                                           const double* __restrict__ kappa, const double* __restrict__ normal,
                                           const unsigned* __restrict__ ring, long long r, long long M,
                                           const CsfOut& out) {
    const long long gkey = ring[r];
    const int b = fr.by_key(gkey);
    const ft_fdesc& D = fr.desc(b);
    const int n0 = D.g.n[0], n1 = D.g.n[1], n2 = D.g.n[2];
    const long long NC = (long long)n0 * n1 * n2;
    const long long s1 = n2, s0 = (long long)n1 * n2;
    const double* __restrict__ alpha = D.alpha;
    const long long kb = fr.key_base(b);
    const long long key = gkey - kb;
    const unsigned ukey = (unsigned)key, ucol = ukey / (unsigned)n2;
    const int k = (int)(ukey - ucol * (unsigned)n2);
    const int i = (int)(ucol / (unsigned)n1);
    const int j = (int)(ucol - (unsigned)i * (unsigned)n1);
    int q[26];
#pragma unroll
    for (int c = 0; c < 26; c++) {
        const int code = c < 13 ? c : c + 1;  // the 27 offsets without the centre
        const int di = code / 9 - 1, dj = (code / 3) % 3 - 1, dk = code % 3 - 1;
        const int ii = i + di, jj = j + dj, kk = k + dk;
        const bool in = ii >= 0 && ii < n0 && jj >= 0 && jj < n1 && kk >= 0 && kk < n2;
        q[c] = in ? idx_map[kb + key + (long long)di * s0 + (long long)dj * s1 + dk] : -1;
    }
    const double axp = (i + 1 < n0) ? alpha[key + s0] : 0.0;
    const double axm = (i > 0) ? alpha[key - s0] : 0.0;
    const double ayp = (j + 1 < n1) ? alpha[key + s1] : 0.0;
    const double aym = (j > 0) ? alpha[key - s1] : 0.0;
    const double azp = (k + 1 < n2) ? alpha[key + 1] : 0.0;
    const double azm = (k > 0) ? alpha[key - 1] : 0.0;
    double num = 0.0, den = 0.0, ks = 0.0;
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < 26; c++) {
        if (q[c] < 0) continue;
        const int code = c < 13 ? c : c + 1;
        const int di = code / 9 - 1, dj = (code / 3) % 3 - 1, dk = code % 3 - 1;
        const int nsq = di * di + dj * dj + dk * dk;
        const double inv_len = nsq == 1 ? 1.0 : (nsq == 2 ? 0.70710678118654752440 : 0.57735026918962576451);
        const double* nq = normal + 3 * (long long)q[c];
        // s_Q . n_Q with the offset's zero components left out (c is a
        // compile-time constant here, so only the non-zero terms are formed:
        // for a finite normal the sum is the same, term for term, as the full
        // dot product, whose other products are zeros)
        double dot = 0.0;
        bool any = false;
        if (di != 0) {
            dot = di > 0 ? nq[0] : -nq[0];
            any = true;
        }
        if (dj != 0) {
            const double t = dj > 0 ? nq[1] : -nq[1];
            dot = any ? dot + t : t;
            any = true;
        }
        if (dk != 0) {
            const double t = dk > 0 ? nq[2] : -nq[2];
            dot = any ? dot + t : t;
        }
        const double w = nsq == 1 ? fabs(dot) : fabs(dot) * inv_len;
        const double kq = kappa[q[c]];
        num += kq * w;
        den += w;
        ks += kq;
        cnt++;
    }
    const double ih2 = 0.5 * D.inv_h;
    const double gx = (axp - axm) * ih2, gy = (ayp - aym) * ih2, gz = (azp - azm) * ih2;
    const double kp = (den > 0.0) ? num / den : (cnt ? ks / cnt : 0.0);
    const double f = sigma * kp;
    if (out.keys) {
        const long long slot = M + r;
        if (slot < out.cap) {
            out.keys[slot] = ukey;
            out.f[3 * slot] = f * gx;
            out.f[3 * slot + 1] = f * gy;
            out.f[3 * slot + 2] = f * gz;
        }
    } else {
        double* __restrict__ force = D.force;
        force[key] = f * gx;
        force[NC + key] = f * gy;
        force[2 * NC + key] = f * gz;
    }
}

// The CSF force of every interfacial cell (items [0, M)) and every listed ring
// cell (items [M, M + nring)) in one launch, after the PPIC fit; the ring
// list comes from k_csf_ring_list, which needs only the binning and so can run
// beside the fit.
template <class F>
__global__ void __launch_bounds__(kThreads) k_csf_force(F fr, double sigma, const unsigned* __restrict__ cells,
                                                        const int* __restrict__ idx_map,
                                                        const double* __restrict__ kappa,
                                                        const double* __restrict__ normal,
                                                        const unsigned* __restrict__ ring,
                                                        const unsigned* __restrict__ nring, long long ring_cap,
                                                        ft_counters* ctr, CsfOut out) {
    const long long M = ctr->M;
    const long long nr = min((long long)*nring, ring_cap);
    if (out.keys && blockIdx.x == 0 && threadIdx.x == 0) {
        const long long total = M + nr;
        *out.count = total;
        if (total > out.cap) ft_flag(ctr, FT_ST_CAPACITY);
    }
    for (long long w = (long long)blockIdx.x * kThreads + threadIdx.x; w < M + nr; w += (long long)gridDim.x * kThreads) {
        if (w < M)
            cell_force(fr, sigma, cells, kappa, w, out);
        else
            ring_force(fr, sigma, idx_map, kappa, normal, ring, w - M, M, out);
    }
}

// Compact volume fraction (one front): bit q % 32 of word q / 32 is set when
// alpha[q] > 1/2 (a warp per 32 consecutive cells, one ballot), and the values
// at the interfacial cells in cell order.
__global__ void __launch_bounds__(256) k_alpha_pack(const double* __restrict__ alpha, long long ncells,
                                                    const unsigned* __restrict__ cells, long long cap,
                                                    unsigned* __restrict__ bits, double* __restrict__ acells,
                                                    ft_counters* ctr) {
    const int lane = threadIdx.x & 31;
    const long long nwords = (ncells + 31) / 32;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = gw; w < nwords; w += nw) {
        const long long q = 32 * w + lane;
        const bool full = q < ncells && alpha[q] > 0.5;
        const unsigned b = __ballot_sync(0xffffffffu, full);
        if (lane == 0) bits[w] = b;
    }
    const long long M = ctr->M;
    if (M > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
        return;
    }
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x)
        acells[m] = alpha[cells[m]];
}

// Cell curvature of the surface-tension terms (Sec. 3.3): the cell's own kappa
// if it is interfacial, else the weighted mean of its interfacial neighbours'
// kappa (w_Q = |s_Q . n_Q| / |s_Q|; plain mean if every w_Q is 0; 0 if none).
template <class F>
__device__ double cell_kappa(const int* __restrict__ idx_map, const double* __restrict__ kappa,
                             const double* __restrict__ normal, long long kb, int n0, int n1, int n2, int i, int j,
                             int k) {
    const long long key = ((long long)i * n1 + j) * n2 + k;
    const int m = idx_map[kb + key];
    if (m >= 0) return kappa[m];
    double num = 0.0, den = 0.0, ks = 0.0;
    int cnt = 0;
    for (int c = 0; c < 27; c++) {
        if (c == 13) continue;
        const int di = c / 9 - 1, dj = (c / 3) % 3 - 1, dk = c % 3 - 1;
        const int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii < 0 || jj < 0 || kk < 0 || ii >= n0 || jj >= n1 || kk >= n2) continue;
        const int q = idx_map[kb + ((long long)ii * n1 + jj) * n2 + kk];
        if (q < 0) continue;
        const int nsq = di * di + dj * dj + dk * dk;
        const double inv_len = nsq == 1 ? 1.0 : (nsq == 2 ? 0.70710678118654752440 : 0.57735026918962576451);
        const double* nq = normal + 3 * (long long)q;
        const double w = fabs(di * nq[0] + dj * nq[1] + dk * nq[2]) * inv_len;
        num += kappa[q] * w;
        den += w;
        ks += kappa[q];
        cnt++;
    }
    return (den > 0.0) ? num / den : (cnt ? ks / cnt : 0.0);
}

// Balanced-force face term (Sec. 3.3, Eq. mwi_disc): S_f = sigma kbar_f
// (alpha_Q - alpha_P)/h on the face between P and Q = P + e_d, kbar_f the mean
// of the two cells' curvatures, alpha and kappa 0 outside the grid.  Block per
// (i, j) column, threads along k; cell (i, j, k) writes its three lower faces,
// the last cell of each direction also the upper boundary face.
template <class F>
__global__ void __launch_bounds__(kThreads) k_face_force(F fr, double sigma, const int* __restrict__ idx_map,
                                                         const double* __restrict__ kappa,
                                                         const double* __restrict__ normal) {
    for (long long gcol = blockIdx.x; gcol < fr.ncols; gcol += gridDim.x) {
        const int b = fr.by_col(gcol);
        const ft_fdesc& D = fr.desc(b);
        const int n0 = D.g.n[0], n1 = D.g.n[1], n2 = D.g.n[2];
        const long long kb = fr.key_base(b);
        const long long col = gcol - fr.col_base(b);
        const int i = (int)(col / n1), j = (int)(col - (long long)i * n1);
        const double* __restrict__ alpha = D.alpha;
        const double sh = 0.5 * sigma * D.inv_h;
        for (int k0 = 0; k0 <= n2; k0 += kThreads) {
            const int k = k0 + (int)threadIdx.x;
            if (k > n2) continue;
            const bool in = k < n2;
            const long long key = ((long long)i * n1 + j) * n2 + k;
            const double aq = in ? alpha[key] : 0.0;
            auto kap = [&](int a, int bb, int c) { return cell_kappa<F>(idx_map, kappa, normal, kb, n0, n1, n2, a, bb, c); };
            // z-face between (i, j, k-1) and (i, j, k): index (i, j, k) of (n0, n1, n2+1)
            {
                const double ap = (k > 0) ? alpha[key - 1] : 0.0;
                double f = 0.0;
                if (__double_as_longlong(ap) != __double_as_longlong(aq)) {
                    const double kp = (k > 0) ? kap(i, j, k - 1) : 0.0;
                    const double kq = in ? kap(i, j, k) : 0.0;
                    f = sh * (kp + kq) * (aq - ap);
                }
                D.fface[2][((long long)i * n1 + j) * (n2 + 1) + k] = f;
            }
            if (!in) continue;
            // x-faces (i, j, k) and, for the last i, (n0, j, k) of (n0+1, n1, n2)
            for (int up = 0; up < ((i == n0 - 1) ? 2 : 1); up++) {
                const int fi = i + up;  // face between cells fi-1 and fi
                const double a_lo = (fi > 0) ? alpha[key - (long long)(1 - up) * n1 * n2] : 0.0;
                const double a_hi = (fi < n0) ? alpha[key + (long long)up * n1 * n2] : 0.0;
                double f = 0.0;
                if (__double_as_longlong(a_lo) != __double_as_longlong(a_hi)) {
                    const double klo = (fi > 0) ? kap(fi - 1, j, k) : 0.0;
                    const double khi = (fi < n0) ? kap(fi, j, k) : 0.0;
                    f = sh * (klo + khi) * (a_hi - a_lo);
                }
                D.fface[0][((long long)fi * n1 + j) * n2 + k] = f;
            }
            // y-faces (i, j, k) and, for the last j, (i, n1, k) of (n0, n1+1, n2)
            for (int up = 0; up < ((j == n1 - 1) ? 2 : 1); up++) {
                const int fj = j + up;
                const double a_lo = (fj > 0) ? alpha[key - (long long)(1 - up) * n2] : 0.0;
                const double a_hi = (fj < n1) ? alpha[key + (long long)up * n2] : 0.0;
                double f = 0.0;
                if (__double_as_longlong(a_lo) != __double_as_longlong(a_hi)) {
                    const double klo = (fj > 0) ? kap(i, fj - 1, k) : 0.0;
                    const double khi = (fj < n1) ? kap(i, fj, k) : 0.0;
                    f = sh * (klo + khi) * (a_hi - a_lo);
                }
                D.fface[1][((long long)i * (n1 + 1) + fj) * n2 + k] = f;
            }
        }
    }
}

}  // namespace

namespace ft {

// the dense force arrays of every front of fr set to zero
template <class F>
cudaError_t clear_with(ft_workspace* ws, const F& fr, cudaStream_t s) {
    if constexpr (std::is_same<F, FrontsOne>::value) {
        Trace t(s, "force clear (memset)");
        const cudaError_t e = cudaMemsetAsync(fr.d0.force, 0, 3 * sizeof(double) * (size_t)fr.ncells, s);
        if (e != cudaSuccess) return e;
    } else {
        count_launches(1);
        Trace t(s, "k_zero_force");
        k_zero_force<F><<<ws->sm_count * ws->tune.csf_bps, kThreads, 0, s>>>(fr);
    }
    return cudaGetLastError();
}

// The ring list of the current binning (the face neighbours of interfacial
// cells that are not interfacial themselves), in the sort's spare key buffer
// (max_cand entries, free once the pairs are placed); its length in ctr->pad.
template <class F>
cudaError_t ring_with(ft_workspace* ws, const F& fr, cudaStream_t s) {
    unsigned* nring = &ws->ctr->pad;
    const cudaError_t e = cudaMemsetAsync(nring, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    Trace t(s, "k_csf_ring_list");
    k_csf_ring_list<F><<<ws->sm_count * 4, kThreads, 0, s>>>(fr, ws->cells, ws->idx_map, ws->keys[ws->sorted_buf ^ 1],
                                                             nring, ws->max_cand, ws->ctr);
    return cudaGetLastError();
}

// The force in the cells where it can be non-zero: the ring list made here
// (list) or by the caller beforehand for the same binning (!list), then the
// dense arrays cleared here (clear) or by the caller beforehand (!clear; the
// compact output has no dense array), then one launch over the interfacial
// and ring cells.
template <class F>
cudaError_t csf_with(ft_workspace* ws, const F& fr, const ft_params* p, const double* kappa, const double* normal,
                     cudaStream_t s, bool clear, bool list, CsfOut out = CsfOut{nullptr, nullptr, 0, nullptr}) {
    cudaError_t e = list ? ring_with(ws, fr, s) : cudaSuccess;
    if (e == cudaSuccess && clear && !out.keys) e = clear_with(ws, fr, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    Trace t(s, "k_csf_force");
    k_csf_force<F><<<ws->sm_count * 4, kThreads, 0, s>>>(fr, p->sigma, ws->cells, ws->idx_map, kappa, normal,
                                                         ws->keys[ws->sorted_buf ^ 1], &ws->ctr->pad, ws->max_cand,
                                                         ws->ctr, out);
    return cudaGetLastError();
}

cudaError_t launch_csf_compact(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                               const double* normal, long long cap, unsigned* keys, double* force, long long* count,
                               cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = const_cast<double*>(alpha);  // read only here
    return csf_with(ws, fr, p, kappa, normal, s, false, true, CsfOut{keys, force, cap, count});
}

cudaError_t launch_alpha_pack(ft_workspace* ws, const double* alpha, long long cap, unsigned* bits, double* acells,
                              cudaStream_t s) {
    count_launches(1);
    Trace t(s, "k_alpha_pack");
    k_alpha_pack<<<ws->sm_count * 8, 256, 0, s>>>(alpha, ws->ncells, ws->cells, cap, bits, acells, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_csf(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                       const double* normal, double* force, cudaStream_t s, bool clear, bool list) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = const_cast<double*>(alpha);  // read only here
    fr.d0.force = force;
    return csf_with(ws, fr, p, kappa, normal, s, clear, list);
}

cudaError_t launch_csf_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                             cudaStream_t s, bool clear, bool list) {
    return csf_with(ws, ft_many(ws), p, kappa, normal, s, clear, list);
}

cudaError_t launch_csf_prepare(ft_workspace* ws, cudaStream_t s) {
    if (ws->batch) return ring_with(ws, ft_many(ws), s);
    return ring_with(ws, ft_one(ws, nullptr, nullptr, 0, 0), s);
}

cudaError_t launch_force_clear(ft_workspace* ws, double* force, cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.force = force;
    return clear_with(ws, fr, s);
}

cudaError_t launch_force_clear_batch(ft_workspace* ws, cudaStream_t s) { return clear_with(ws, ft_many(ws), s); }

cudaError_t launch_face_force(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                              const double* normal, double* fx, double* fy, double* fz, cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = const_cast<double*>(alpha);  // read only here
    fr.d0.fface[0] = fx;
    fr.d0.fface[1] = fy;
    fr.d0.fface[2] = fz;
    count_launches(1);
    k_face_force<FrontsOne><<<ws->sm_count * ws->tune.csf_bps, kThreads, 0, s>>>(fr, p->sigma, ws->idx_map, kappa,
                                                                                 normal);
    return cudaGetLastError();
}

cudaError_t launch_face_force_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                                    cudaStream_t s) {
    count_launches(1);
    k_face_force<FrontsMany><<<ws->sm_count * ws->tune.csf_bps, kThreads, 0, s>>>(ft_many(ws), p->sigma,
                                                                                  ws->idx_map, kappa, normal);
    return cudaGetLastError();
}

}  // namespace ft
