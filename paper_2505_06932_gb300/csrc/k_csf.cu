// k_csf.cu -- front_csf_force: S_P = sigma kappa_P grad alpha_P (Eq. csf) with
// the weighted curvature smoothing of Sec. 3.3 in cells next to the interface:
// kbar_P = sum_Q kappa_Q w_Q / sum_Q w_Q, w_Q = |s_Q . n_Q| / |s_Q|, over the
// interfacial cells Q among the 26 neighbours of P (plain mean if all w_Q = 0).
//
// Two passes:
//  * k_csf_dense -- one block per (i, j) column, threads along k (coalesced):
//    the central-difference gradient (alpha = 0 outside the grid); flat
//    neighbourhoods (bitwise-equal neighbour pairs: full and empty cells hold
//    exactly 1 and 0) write zero force, interfacial cells write sigma kappa grad
//    alpha, and the remaining cells (the ring around the interface) are appended
//    to a compact list.
//  * k_csf_ring -- one thread per listed cell: the smoothed curvature and the
//    force.  Keeping the float64 smoothing out of the dense pass keeps that pass
//    bound by memory instead of by divergent float64 issue.
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;  // one block per column; 128 and 256 cell columns fill it

template <class F>
__global__ void __launch_bounds__(kThreads) k_csf_dense(F fr, double sigma, const int* __restrict__ idx_map,
                                                        const double* __restrict__ kappa,
                                                        unsigned* __restrict__ ring, unsigned* __restrict__ nring,
                                                        long long ring_cap, ft_counters* ctr) {
    const int lane = threadIdx.x & 31;
    for (long long gcol = blockIdx.x; gcol < fr.ncols; gcol += gridDim.x) {
        const int b = fr.by_col(gcol);
        const ft_fdesc& D = fr.desc(b);
        const int n0 = D.g.n[0], n1 = D.g.n[1], n2 = D.g.n[2];
        const long long NC = (long long)n0 * n1 * n2;
        const long long s1 = n2, s0 = (long long)n1 * n2;
        const double ih2 = 0.5 * D.inv_h;
        const double* __restrict__ alpha = D.alpha;
        double* __restrict__ force = D.force;
        const long long kb = fr.key_base(b);
        const long long col = gcol - fr.col_base(b);
        const int i = (int)(col / n1), j = (int)(col - (long long)i * n1);
        for (int k0 = 0; k0 < n2; k0 += kThreads) {
            const int k = k0 + (int)threadIdx.x;
            const bool valid = k < n2;
            const long long key = col * n2 + k;
            double axp = 0.0, axm = 0.0, ayp = 0.0, aym = 0.0, azp = 0.0, azm = 0.0;
            if (valid) {
                if (i + 1 < n0) axp = alpha[key + s0];
                if (i > 0) axm = alpha[key - s0];
                if (j + 1 < n1) ayp = alpha[key + s1];
                if (j > 0) aym = alpha[key - s1];
                if (k + 1 < n2) azp = alpha[key + 1];
                if (k > 0) azm = alpha[key - 1];
            }
            const bool flat = __double_as_longlong(axp) == __double_as_longlong(axm) &&
                              __double_as_longlong(ayp) == __double_as_longlong(aym) &&
                              __double_as_longlong(azp) == __double_as_longlong(azm);
            bool to_ring = false;
            if (__all_sync(0xffffffffu, flat)) {
                if (valid) {
                    force[key] = 0.0;
                    force[NC + key] = 0.0;
                    force[2 * NC + key] = 0.0;
                }
            } else if (valid) {
                const double gx = (axp - axm) * ih2, gy = (ayp - aym) * ih2, gz = (azp - azm) * ih2;
                double kp = 0.0;
                if (gx != 0.0 || gy != 0.0 || gz != 0.0) {
                    const int m = idx_map[kb + key];
                    if (m >= 0)
                        kp = kappa[m];
                    else
                        to_ring = true;
                }
                if (!to_ring) {
                    const double f = sigma * kp;
                    force[key] = f * gx;
                    force[NC + key] = f * gy;
                    force[2 * NC + key] = f * gz;
                }
            }
            // append this warp's ring cells (batch-global keys) with one atomic
            const unsigned bal = __ballot_sync(0xffffffffu, to_ring);
            if (bal) {
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(nring, (unsigned)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (to_ring) {
                    const unsigned pos = base + __popc(bal & ((1u << lane) - 1u));
                    if (pos < ring_cap)
                        ring[pos] = (unsigned)(kb + key);
                    else
                        ft_flag(ctr, FT_ST_CAPACITY);
                }
            }
        }
    }
}

// One thread per ring cell.  The 26 index-map lookups are issued together
// (independent loads) before the float64 smoothing sums, which then run once
// per cell instead of once per lane of a warp-wide reduction.
template <class F>
__global__ void __launch_bounds__(128) k_csf_ring(F fr, double sigma, const int* __restrict__ idx_map,
                                                  const double* __restrict__ kappa, const double* __restrict__ normal,
                                                  const unsigned* __restrict__ ring, const unsigned* __restrict__ nring,
                                                  long long ring_cap) {
    const long long nr = min((long long)*nring, ring_cap);
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (long long)gridDim.x * blockDim.x) {
        const long long gkey = ring[r];
        const int b = fr.by_key(gkey);
        const ft_fdesc& D = fr.desc(b);
        const int n0 = D.g.n[0], n1 = D.g.n[1], n2 = D.g.n[2];
        const long long NC = (long long)n0 * n1 * n2;
        const long long s1 = n2, s0 = (long long)n1 * n2;
        const double* __restrict__ alpha = D.alpha;
        const long long kb = fr.key_base(b);
        const long long key = gkey - kb;
        const int k = (int)(key % n2);
        const int j = (int)((key / n2) % n1);
        const int i = (int)(key / s0);
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
            const double w = fabs(di * nq[0] + dj * nq[1] + dk * nq[2]) * inv_len;
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
        double* __restrict__ force = D.force;
        force[key] = f * gx;
        force[NC + key] = f * gy;
        force[2 * NC + key] = f * gz;
    }
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

template <class F>
cudaError_t csf_with(ft_workspace* ws, const F& fr, const ft_params* p, const double* kappa, const double* normal,
                     cudaStream_t s) {
    // the ring list lives in the sort's spare key buffer (max_cand entries)
    unsigned* ring = ws->keys[ws->sorted_buf ^ 1];
    unsigned* nring = &ws->ctr->pad;
    cudaMemsetAsync(nring, 0, sizeof(unsigned), s);
    count_launches(2);
    k_csf_dense<F><<<ws->sm_count * ws->tune.csf_bps, kThreads, 0, s>>>(fr, p->sigma, ws->idx_map, kappa, ring, nring,
                                                                        ws->max_cand, ws->ctr);
    k_csf_ring<F><<<ws->sm_count * 4, 128, 0, s>>>(fr, p->sigma, ws->idx_map, kappa, normal, ring, nring,
                                                   ws->max_cand);
    return cudaGetLastError();
}

cudaError_t launch_csf(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                       const double* normal, double* force, cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = const_cast<double*>(alpha);  // read only here
    fr.d0.force = force;
    return csf_with(ws, fr, p, kappa, normal, s);
}

cudaError_t launch_csf_batch(ft_workspace* ws, const ft_params* p, const double* kappa, const double* normal,
                             cudaStream_t s) {
    return csf_with(ws, ft_many(ws), p, kappa, normal, s);
}

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
