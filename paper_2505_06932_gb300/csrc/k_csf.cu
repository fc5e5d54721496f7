// k_csf.cu -- front_csf_force: S_P = sigma kappa_P grad alpha_P (Eq. csf) with
// the weighted curvature smoothing of Sec. 3.3 in cells next to the interface:
// kbar_P = sum_Q kappa_Q w_Q / sum_Q w_Q, w_Q = |s_Q . n_Q| / |s_Q|, over the
// interfacial cells Q among the 26 neighbours of P (plain mean if all w_Q = 0).
// One block per (i, j) column (grid-stride), threads along k: alpha loads and
// force stores coalesce and no 64-bit division is needed per cell.
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;  // one block per column; 128 and 256 cell columns fill it

__global__ void __launch_bounds__(kThreads) k_csf(ft_grid g, double sigma, const double* __restrict__ alpha,
                                                  const int* __restrict__ idx_map, const double* __restrict__ kappa,
                                                  const double* __restrict__ normal, double* __restrict__ force) {
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long NC = (long long)n0 * n1 * n2;
    const long long s1 = n2, s0 = (long long)n1 * n2;
    const double ih2 = 0.5 / g.h;
    const double inv_len[4] = {0.0, 1.0, 0.70710678118654752440, 0.57735026918962576451};
    const long long ncol = (long long)n0 * n1;
    for (long long col = blockIdx.x; col < ncol; col += gridDim.x) {
        const int i = (int)(col / n1), j = (int)(col - (long long)i * n1);
        for (int k = threadIdx.x; k < n2; k += kThreads) {
            const long long key = col * n2 + k;
            const double axp = (i + 1 < n0) ? alpha[key + s0] : 0.0;
            const double axm = (i > 0) ? alpha[key - s0] : 0.0;
            const double ayp = (j + 1 < n1) ? alpha[key + s1] : 0.0;
            const double aym = (j > 0) ? alpha[key - s1] : 0.0;
            const double azp = (k + 1 < n2) ? alpha[key + 1] : 0.0;
            const double azm = (k > 0) ? alpha[key - 1] : 0.0;
            // equal neighbour pairs (bitwise: full and empty cells hold exactly 1 and 0)
            // give a zero gradient; a warp whose cells are all flat writes zeros
            // without issuing any float64 instruction
            const bool flat = __double_as_longlong(axp) == __double_as_longlong(axm) &&
                              __double_as_longlong(ayp) == __double_as_longlong(aym) &&
                              __double_as_longlong(azp) == __double_as_longlong(azm);
            if (__all_sync(__activemask(), flat)) {
                force[key] = 0.0;
                force[NC + key] = 0.0;
                force[2 * NC + key] = 0.0;
                continue;
            }
            const double gx = (axp - axm) * ih2, gy = (ayp - aym) * ih2, gz = (azp - azm) * ih2;
            double kp = 0.0;
            if (gx != 0.0 || gy != 0.0 || gz != 0.0) {
                const int m = idx_map[key];
                if (m >= 0) {
                    kp = kappa[m];
                } else {
                    double num = 0.0, den = 0.0, ks = 0.0;
                    int cnt = 0;
                    for (int di = -1; di <= 1; di++) {
                        const int ii = i + di;
                        if (ii < 0 || ii >= n0) continue;
                        for (int dj = -1; dj <= 1; dj++) {
                            const int jj = j + dj;
                            if (jj < 0 || jj >= n1) continue;
                            for (int dk = -1; dk <= 1; dk++) {
                                const int kk = k + dk;
                                if (kk < 0 || kk >= n2 || (di == 0 && dj == 0 && dk == 0)) continue;
                                const int q = idx_map[((long long)ii * n1 + jj) * n2 + kk];
                                if (q < 0) continue;
                                const double* nq = normal + 3 * (long long)q;
                                const double w = fabs(di * nq[0] + dj * nq[1] + dk * nq[2]) *
                                                 inv_len[di * di + dj * dj + dk * dk];
                                const double kq = kappa[q];
                                num += kq * w;
                                den += w;
                                ks += kq;
                                cnt++;
                            }
                        }
                    }
                    kp = (den > 0.0) ? num / den : (cnt ? ks / cnt : 0.0);
                }
            }
            const double f = sigma * kp;
            force[key] = f * gx;
            force[NC + key] = f * gy;
            force[2 * NC + key] = f * gz;
        }
    }
}

}  // namespace

namespace ft {

cudaError_t launch_csf(ft_workspace* ws, const ft_params* p, const double* alpha, const double* kappa,
                       const double* normal, double* force, cudaStream_t s) {
    count_launches(1);
    k_csf<<<ws->sm_count * 16, kThreads, 0, s>>>(ws->g, p->sigma, alpha, ws->idx_map, kappa, normal, force);
    return cudaGetLastError();
}

}  // namespace ft
