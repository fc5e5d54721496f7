// k_ppic.cu -- front_curvature_ppic: PPIC volume fit of a paraboloid
// z = a1 + a2 x + a3 y + a4 x^2 + a5 xy + a6 y^2 in every interfacial cell
// (Sec. 3.2, Eqs. volumefit, Wendland, volumefit2) and its curvature.
//
// One warp per fit cell.  In the local frame (t1, t2, n) centred at the cell
// centre (lengths in units of h), a fragment f with area vector AN, area
// centroid p and central second moment per unit area K contributes the signed
// projected moments (Green's theorem integrals over its projection Gamma_f):
//   m_f = (n . AN) [1, x, y, x^2 + t1.K.t1, x y + t1.K.t2, y^2 + t2.K.t2],
//   G_f = (n . AN) z,     (x, y, z) = (t1.p, t2.p, n.p),
// so that int_Gamma P dA = m_f . a and int_Gamma g_f dA = G_f.  The normal
// equations sum_f w_f m_f m_f^T a = sum_f w_f G_f m_f (Eq. volumefit2) are
// accumulated in registers, reduced over the warp and solved in float64.
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;

struct PpicArgs {
    ft_grid g;
    double delta_h, delta_growth, delta_max_h;
    int fit_min;
    long long cap;
};

// Tangents (t1, t2) completing the unit normal n: the branchless basis of Duff
// et al. 2017 ("Building an orthonormal basis, revisited") built for m = R n in
// a fixed rotated reference frame (third row of R: (sin 1 cos 1, sin 1 sin 1, cos 1), a
// direction with no small-integer relation to axes or symmetric fronts) and rotated
// back, so that the basis' switch on sign(m_z) does not fall on fronts with an
// exactly vertical normal.
__constant__ double kFrameR[3][3] = {{0.890670841215793, -0.3614406733922875, -0.2758008198422935},
                                     {0.0, 0.6066239971779142, -0.7949888842291382},
                                     {0.4546487134128409, 0.7080734182735712, 0.5403023058681398}};

__device__ __forceinline__ void basis(const double n[3], double t1[3], double t2[3]) {
    double m[3], u1[3], u2[3];
#pragma unroll
    for (int r = 0; r < 3; r++) m[r] = kFrameR[r][0] * n[0] + kFrameR[r][1] * n[1] + kFrameR[r][2] * n[2];
    const double sg = copysign(1.0, m[2]);
    const double a = -1.0 / (sg + m[2]);
    const double b = m[0] * m[1] * a;
    u1[0] = 1.0 + sg * m[0] * m[0] * a;
    u1[1] = sg * b;
    u1[2] = -sg * m[0];
    u2[0] = b;
    u2[1] = sg + m[1] * m[1] * a;
    u2[2] = -m[1];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        t1[c] = kFrameR[0][c] * u1[0] + kFrameR[1][c] * u1[1] + kFrameR[2][c] * u1[2];
        t2[c] = kFrameR[0][c] * u2[0] + kFrameR[1][c] * u2[1] + kFrameR[2][c] * u2[2];
    }
}

// coefficients c such that c . (Kxx,Kyy,Kzz,Kxy,Kxz,Kyz) = u . K . v
__device__ __forceinline__ void qform(const double u[3], const double v[3], double c[6]) {
    c[0] = u[0] * v[0];
    c[1] = u[1] * v[1];
    c[2] = u[2] * v[2];
    c[3] = u[0] * v[1] + u[1] * v[0];
    c[4] = u[0] * v[2] + u[2] * v[0];
    c[5] = u[1] * v[2] + u[2] * v[1];
}

// LDL^T solve of the 6x6 normal equations (upper triangle packed row-wise in S,
// right-hand side B).  Returns the smallest pivot relative to the trace.
__device__ double ldlt_solve(const double* S, const double* B, int n, double* a) {
    double Lm[6][6], d[6];
    auto at = [&](int i, int j) {  // packed upper triangle of the 6x6 matrix
        if (i > j) { int t = i; i = j; j = t; }
        return S[i * 6 - (i * (i - 1)) / 2 + (j - i)];
    };
    double tr = 0.0;
    for (int i = 0; i < n; i++) tr += at(i, i);
    double minp = INFINITY;
    for (int j = 0; j < n; j++) {
        double dj = at(j, j);
        for (int k = 0; k < j; k++) dj -= Lm[j][k] * Lm[j][k] * d[k];
        d[j] = dj;
        minp = fmin(minp, dj);
        if (!(dj > 0.0)) return -1.0;
        for (int i = j + 1; i < n; i++) {
            double v = at(i, j);
            for (int k = 0; k < j; k++) v -= Lm[i][k] * Lm[j][k] * d[k];
            Lm[i][j] = v / dj;
        }
    }
    double y[6];
    for (int i = 0; i < n; i++) {
        double v = B[i];
        for (int k = 0; k < i; k++) v -= Lm[i][k] * y[k];
        y[i] = v;
    }
    for (int i = n - 1; i >= 0; i--) {
        double v = y[i] / d[i];
        for (int k = i + 1; k < n; k++) v -= Lm[k][i] * a[k];
        a[i] = v;
    }
    return minp / tr;
}

__global__ void __launch_bounds__(kThreads) k_ppic(PpicArgs A, const unsigned* __restrict__ cells,
                                                   const int* __restrict__ cell_off, const unsigned* __restrict__ vals,
                                                   const ft_frag* __restrict__ rec, const int* __restrict__ idx_map,
                                                   ft_counters* ctr, unsigned* __restrict__ out_keys,
                                                   double* __restrict__ out_kappa, double* __restrict__ out_normal,
                                                   double* __restrict__ out_coeffs, int8_t* __restrict__ out_status) {
    const long long M = ctr->M;
    if (M > A.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
    const long long nw = (long long)gridDim.x * kWarps;
    long long pairs_total = 0;
    for (long long m = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); m < M; m += nw) {
        const unsigned key = cells[m];
        const int ck = (int)(key % (unsigned)n2);
        const int cj = (int)((key / (unsigned)n2) % (unsigned)n1);
        const int ci = (int)(key / ((unsigned)n2 * (unsigned)n1));
        int8_t st = 0;

        // 1. local normal: normalized sum of the cell's fragment area vectors
        double N[3] = {0.0, 0.0, 0.0}, sa = 0.0, best = -1.0;
        int bestq = 0x7fffffff;
        const int q0 = cell_off[m], q1 = cell_off[m + 1];
        for (int q = q0 + lane; q < q1; q += 32) {
            const ft_frag* f = rec + vals[q];
            const double ax = f->an[0], ay = f->an[1], az = f->an[2];
            N[0] += ax;
            N[1] += ay;
            N[2] += az;
            const double a = sqrt(ax * ax + ay * ay + az * az);
            sa += a;
            if (a > best) {
                best = a;
                bestq = q;
            }
        }
        for (int d = 0; d < 3; d++) N[d] = ft_warp_sum(N[d]);
        sa = ft_warp_sum(sa);
        double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        if (nn < 1e-3 * sa) {
            // opposing sheets: normal of the largest fragment (first on ties)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oq = __shfl_xor_sync(0xffffffffu, bestq, o);
                if (ob > best || (ob == best && oq < bestq)) {
                    best = ob;
                    bestq = oq;
                }
            }
            const ft_frag* f = rec + vals[bestq];
            N[0] = f->an[0];
            N[1] = f->an[1];
            N[2] = f->an[2];
            nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
            st |= FT_FIT_NORMAL;
        }
        const double n[3] = {N[0] / nn, N[1] / nn, N[2] / nn};
        double t1[3], t2[3];
        basis(n, t1, t2);
        double c11[6], c12[6], c22[6];
        qform(t1, t1, c11);
        qform(t1, t2, c12);
        qform(t2, t2, c22);

        // 2-4. weighted normal equations, support grown while too few fragments
        double delta = A.delta_h;
        double S[21], B[6];
        int count;
        for (;;) {
#pragma unroll
            for (int r = 0; r < 21; r++) S[r] = 0.0;
#pragma unroll
            for (int r = 0; r < 6; r++) B[r] = 0.0;
            count = 0;
            const double d2hi = delta * delta * (1.0 + 1e-12);
            const int R = (int)ceil(delta - 0.5);
            const int side = 2 * R + 1;
            const int nb = side * side * side;
            for (int cb = 0; cb < nb; cb += 32) {
                const int l = cb + lane;
                int f0 = 0, cnt = 0, dpack = 0;
                if (l < nb) {
                    const int di = l / (side * side) - R, dj = (l / side) % side - R, dk = l % side - R;
                    const int ii = ci + di, jj = cj + dj, kk = ck + dk;
                    if (ii >= 0 && jj >= 0 && kk >= 0 && ii < n0 && jj < n1 && kk < n2) {
                        const int m2 = idx_map[((long long)ii * n1 + jj) * n2 + kk];
                        if (m2 >= 0) {
                            f0 = cell_off[m2];
                            cnt = cell_off[m2 + 1] - f0;
                        }
                    }
                    dpack = ((di + 128) << 16) | ((dj + 128) << 8) | (dk + 128);
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = incl - cnt;
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                for (int fb = 0; fb < total; fb += 32) {
                    const int fi = fb + lane;
                    int o = 0;
#pragma unroll
                    for (int s = 16; s > 0; s >>= 1) {
                        const int e = __shfl_sync(0xffffffffu, excl, o + s);
                        if (e <= fi) o += s;
                    }
                    const int fo = __shfl_sync(0xffffffffu, f0, o);
                    const int eo = __shfl_sync(0xffffffffu, excl, o);
                    const int dp = __shfl_sync(0xffffffffu, dpack, o);
                    if (fi >= total) continue;
                    const ft_frag fr = rec[vals[fo + (fi - eo)]];
                    const double p[3] = {fr.c[0] + (double)(((dp >> 16) & 255) - 128),
                                         fr.c[1] + (double)(((dp >> 8) & 255) - 128),
                                         fr.c[2] + (double)((dp & 255) - 128)};
                    const double dd2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
                    if (!(dd2 < d2hi)) continue;
                    const double dist = sqrt(dd2);
                    if (!(dist < delta)) continue;
                    count++;
                    const double q = dist / delta;
                    const double om = 1.0 - q;
                    const double om2 = om * om;
                    const double w = (1.0 + 4.0 * q) * om2 * om2;
                    const double x = t1[0] * p[0] + t1[1] * p[1] + t1[2] * p[2];
                    const double y = t2[0] * p[0] + t2[1] * p[1] + t2[2] * p[2];
                    const double z = n[0] * p[0] + n[1] * p[1] + n[2] * p[2];
                    const double sA = n[0] * fr.an[0] + n[1] * fr.an[1] + n[2] * fr.an[2];
                    double q11 = 0.0, q12 = 0.0, q22 = 0.0;
#pragma unroll
                    for (int r = 0; r < 6; r++) {
                        q11 += c11[r] * fr.k[r];
                        q12 += c12[r] * fr.k[r];
                        q22 += c22[r] * fr.k[r];
                    }
                    const double mv[6] = {sA, sA * x, sA * y, sA * (x * x + q11), sA * (x * y + q12), sA * (y * y + q22)};
                    const double G = sA * z;
                    int r = 0;
#pragma unroll
                    for (int i = 0; i < 6; i++) {
                        const double wm = w * mv[i];
#pragma unroll
                        for (int j = i; j < 6; j++) S[r++] += wm * mv[j];
                        B[i] += wm * G;
                    }
                }
            }
            const int ctot = ft_warp_sum_i(count);
            if (ctot >= A.fit_min || delta >= A.delta_max_h) {
                count = ctot;
                break;
            }
            delta = fmin(delta * A.delta_growth, A.delta_max_h);
            st |= FT_FIT_GROWN;
        }
        pairs_total += count;
#pragma unroll
        for (int r = 0; r < 21; r++) S[r] = ft_warp_sum(S[r]);
#pragma unroll
        for (int r = 0; r < 6; r++) B[r] = ft_warp_sum(B[r]);

        // 5-6. solve (Eq. volumefit2) and take the curvature of z = P(x, y) at the origin
        if (lane == 0) {
            double Sl[21], Bl[6];  // copies, so that S and B stay in registers
#pragma unroll
            for (int r = 0; r < 21; r++) Sl[r] = S[r];
#pragma unroll
            for (int r = 0; r < 6; r++) Bl[r] = B[r];
            double a[6] = {0, 0, 0, 0, 0, 0};
            const double rel = ldlt_solve(Sl, Bl, 6, a);
            if (!(rel >= 1e-12)) {
                // singular: plane fit on the leading 3x3 block
                for (int r = 0; r < 6; r++) a[r] = 0.0;
                double a3[6];
                if (ldlt_solve(Sl, Bl, 3, a3) > 0.0) {
                    a[0] = a3[0];
                    a[1] = a3[1];
                    a[2] = a3[2];
                }
                st |= FT_FIT_SINGULAR;
            }
            const double g2 = 1.0 + a[1] * a[1] + a[2] * a[2];
            const double kl = -(2.0 * a[3] * (1.0 + a[2] * a[2]) - 2.0 * a[1] * a[2] * a[4] +
                                2.0 * a[5] * (1.0 + a[1] * a[1])) / (g2 * sqrt(g2));
            double nv[3];
            for (int d = 0; d < 3; d++) nv[d] = n[d] - a[1] * t1[d] - a[2] * t2[d];
            const double nl = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
            out_keys[m] = key;
            out_kappa[m] = kl / A.g.h;
            for (int d = 0; d < 3; d++) out_normal[3 * m + d] = nv[d] / nl;
            if (out_coeffs)
                for (int r = 0; r < 6; r++) out_coeffs[6 * m + r] = a[r];
            out_status[m] = st;
        }
    }
    if (lane == 0 && pairs_total) atomicAdd((unsigned long long*)&ctr->fit_pairs, (unsigned long long)pairs_total);
}

}  // namespace

namespace ft {

cudaError_t launch_ppic(ft_workspace* ws, const ft_params* p, long long cap, unsigned* cell_keys, double* kappa,
                        double* normal, double* coeffs, int8_t* fit_status, cudaStream_t s) {
    PpicArgs A;
    A.g = ws->g;
    A.delta_h = p->delta_h;
    A.delta_growth = p->delta_growth;
    A.delta_max_h = p->delta_max_h;
    A.fit_min = p->fit_min;
    A.cap = cap;
    cudaMemsetAsync(&ws->ctr->fit_pairs, 0, sizeof(long long), s);
    count_launches(1);
    k_ppic<<<ws->sm_count * 4, kThreads, 0, s>>>(A, ws->cells, ws->cell_off, ws->vals[ws->sorted_buf], ws->rec,
                                                 ws->idx_map, ws->ctr, cell_keys, kappa, normal, coeffs, fit_status);
    return cudaGetLastError();
}

}  // namespace ft
