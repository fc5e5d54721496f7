// k_parab.cu -- the paper's own cut-cell quantities from the fitted
// paraboloids (Sec. 3.2): alpha = V_P / V_C of the cell below its paraboloid,
// and the curvature and normal averaged over the paraboloid surface inside
// the cell (parab.cuh has the integration).  A group of kG = 8 lanes per cell
// (four cells per warp): every lane walks the cell's breakpoints and pieces,
// the lanes take different outer quadrature nodes of each piece side by side
// (lane g the nodes g, g + kG), and the group adds its shares with shuffles.
// One thread per cell would leave the GPU nearly empty (a front has tens of
// thousands of interfacial cells, a few warps per SM) with each thread running
// a long serial float64 chain.
//  * k_parab_cells -- from caller-given frames and coefficients (cell units);
//  * k_parab_ppic<F> -- from the last PPIC fit of a workspace (frame normal
//    from the stored normal equations, the tangents as the fit built them),
//    writing alpha_P into the front's alpha grid at the interfacial cells;
//  * k_ppic_frame -- the frames of the last fit.
#include "frame.cuh"
#include "ft_internal.cuh"
#include "parab.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kG = 8;                   // lanes per cell (divides parab::kNS and parab::kN8)
constexpr int kCellsPerWarp = 32 / kG;  // cells per warp and pass

struct ParabOut {
    double* alpha;  // per cell (k_parab_cells) or nullptr
    double* area;
    double* kappa;
    double* normal;
    int8_t* status;
};

// mean curvature and unit normal of z = P(x, y) at the frame origin
__device__ void point_values(const double t1[3], const double t2[3], const double n[3], const double a[6],
                             double& kappa, double nv[3]) {
    const double g2 = 1.0 + a[1] * a[1] + a[2] * a[2];
    kappa = -(2.0 * a[3] * (1.0 + a[2] * a[2]) - 2.0 * a[1] * a[2] * a[4] + 2.0 * a[5] * (1.0 + a[1] * a[1])) /
            (g2 * sqrt(g2));
    for (int d = 0; d < 3; d++) nv[d] = n[d] - a[1] * t1[d] - a[2] * t2[d];
    const double il = 1.0 / sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int d = 0; d < 3; d++) nv[d] *= il;
}

// this lane's share of a cell, added over the group (all 32 lanes call it)
__device__ void group_sum(parab::Out& o) {
#pragma unroll
    for (int off = kG / 2; off >= 1; off >>= 1) {
        o.V += __shfl_xor_sync(0xffffffffu, o.V, off);
        o.A += __shfl_xor_sync(0xffffffffu, o.A, off);
        o.K += __shfl_xor_sync(0xffffffffu, o.K, off);
        for (int d = 0; d < 3; d++) o.N[d] += __shfl_xor_sync(0xffffffffu, o.N[d], off);
    }
}

// from the cell totals (cell units): returns alpha; writes area, kbar, nbar and status
__device__ double finish(const double t1[3], const double t2[3], const double n[3], const double a[6],
                         const parab::Out& o, double& area, double& kbar, double nb[3], int& st) {
    area = o.A;
    const double nl = sqrt(o.N[0] * o.N[0] + o.N[1] * o.N[1] + o.N[2] * o.N[2]);
    if (o.A > 0.0 && nl > 0.0) {
        kbar = o.K / o.A;
        for (int d = 0; d < 3; d++) nb[d] = o.N[d] / nl;
        st = 0;
    } else {  // the surface misses the cell: the point values at the origin, and
              // the cell lies on one side of it (alpha exactly 0 or 1)
        area = 0.0;
        point_values(t1, t2, n, a, kbar, nb);
        st = FT_PARAB_MISS;
        return o.V > 0.5 ? 1.0 : 0.0;
    }
    return fmin(fmax(o.V, 0.0), 1.0);
}

__global__ void __launch_bounds__(kThreads, 4) k_parab_cells(const double* __restrict__ frame,
                                                          const double* __restrict__ coeffs, long long m,
                                                          parab::Rule R, ParabOut out) {
    const int lane = threadIdx.x & 31, g = lane % kG;
    // the strip plans of each group's cell (shared by its kG lanes)
    __shared__ unsigned long long plans[kThreads / kG][parab::kMaxStrips];
    const unsigned gmask = ((1u << kG) - 1u) << (lane - g);
    const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * kThreads) >> 5;
    // warp-uniform loop: all 32 lanes reach the shuffles of every pass
    for (long long base = warp * kCellsPerWarp; base < m; base += nwarps * kCellsPerWarp) {
        const long long c = base + lane / kG;
        double t1[3], t2[3], n[3], a[6];
        parab::Out o{0.0, 0.0, 0.0, {0.0, 0.0, 0.0}};
        if (c < m) {
            for (int d = 0; d < 3; d++) {
                t1[d] = frame[9 * c + d];
                t2[d] = frame[9 * c + 3 + d];
                n[d] = frame[9 * c + 6 + d];
            }
            for (int r = 0; r < 6; r++) a[r] = coeffs[6 * c + r];
            const parab::Split sp{g, kG};
            const parab::PlanShare ps{plans[threadIdx.x / kG], g, kG};
            parab::parab_cell(t1, t2, n, a, R, sp, ps, [&] { __syncwarp(gmask); }, o);
        }
        group_sum(o);
        if (c < m && g == 0) {
            double area, kbar, nb[3];
            int st;
            out.alpha[c] = finish(t1, t2, n, a, o, area, kbar, nb, st);
            if (out.area) out.area[c] = area;
            if (out.kappa) out.kappa[c] = kbar;
            if (out.normal)
                for (int d = 0; d < 3; d++) out.normal[3 * c + d] = nb[d];
            if (out.status) out.status[c] = (int8_t)st;
        }
    }
}

template <class F>
__global__ void __launch_bounds__(kThreads, 4) k_parab_ppic(F fr, const ft_cellsys* __restrict__ sys, int fp32,
                                                         const unsigned* __restrict__ cells,
                                                         const double* __restrict__ coeffs, long long cap,
                                                         ft_counters* ctr, parab::Rule R, ParabOut out) {
    const long long M = ctr->M;
    if (M > cap) {  // the caller's arrays are too short: write nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
        return;
    }
    const int lane = threadIdx.x & 31, g = lane % kG;
    // the strip plans of each group's cell (shared by its kG lanes)
    __shared__ unsigned long long plans[kThreads / kG][parab::kMaxStrips];
    const unsigned gmask = ((1u << kG) - 1u) << (lane - g);
    const long long warp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * kThreads) >> 5;
    for (long long base = warp * kCellsPerWarp; base < M; base += nwarps * kCellsPerWarp) {
        const long long m = base + lane / kG;
        double n[3], t1[3], t2[3], a[6];
        parab::Out o{0.0, 0.0, 0.0, {0.0, 0.0, 0.0}};
        if (m < M) {
            sys_normal(sys[m], fp32 != 0, n);
            basis<double>(n, t1, t2);
            for (int r = 0; r < 6; r++) a[r] = coeffs[6 * m + r];
            const parab::Split sp{g, kG};
            const parab::PlanShare ps{plans[threadIdx.x / kG], g, kG};
            parab::parab_cell(t1, t2, n, a, R, sp, ps, [&] { __syncwarp(gmask); }, o);
        }
        group_sum(o);
        if (m < M && g == 0) {
            double area, kbar, nb[3];
            int st;
            const double al = finish(t1, t2, n, a, o, area, kbar, nb, st);
            const long long gkey = cells[m];
            const int b = fr.by_key(gkey);
            const ft_fdesc& D = fr.desc(b);
            const double h = D.g.h;
            D.alpha[gkey - fr.key_base(b)] = al;
            if (out.area) out.area[m] = area * h * h;
            if (out.kappa) out.kappa[m] = kbar * D.inv_h;
            if (out.normal)
                for (int d = 0; d < 3; d++) out.normal[3 * m + d] = nb[d];
            if (out.status) out.status[m] = (int8_t)st;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_ppic_frame(const ft_cellsys* __restrict__ sys, int fp32, long long cap,
                                                         ft_counters* ctr, double* __restrict__ frame) {
    const long long M = ctr->M;
    if (M > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
        return;
    }
    for (long long m = (long long)blockIdx.x * kThreads + threadIdx.x; m < M; m += (long long)gridDim.x * kThreads) {
        double n[3], t1[3], t2[3];
        sys_normal(sys[m], fp32 != 0, n);
        basis<double>(n, t1, t2);
        for (int d = 0; d < 3; d++) {
            frame[9 * m + d] = t1[d];
            frame[9 * m + 3 + d] = t2[d];
            frame[9 * m + 6 + d] = n[d];
        }
    }
}

const parab::Rule& rule() {
    static const parab::Rule R = parab::make_rule();
    return R;
}

}  // namespace

namespace ft {

cudaError_t launch_parab_cells(const double* frame, const double* coeffs, long long m, double* alpha, double* area,
                               double* kappa, double* normal, int8_t* status, int sm_count, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    ParabOut out{alpha, area, kappa, normal, status};
    const long long blocks = (m * kG + kThreads - 1) / kThreads;
    count_launches(1);
    k_parab_cells<<<(unsigned)(blocks < 16LL * sm_count ? blocks : 16LL * sm_count), kThreads, 0, s>>>(
        frame, coeffs, m, rule(), out);
    return cudaGetLastError();
}

template <class F>
static cudaError_t parab_with(ft_workspace* ws, const F& fr, const double* coeffs, long long cap, double* area,
                              double* kappa, double* normal, int8_t* status, cudaStream_t s) {
    ParabOut out{nullptr, area, kappa, normal, status};
    count_launches(1);
    k_parab_ppic<F><<<ws->sm_count * 16, kThreads, 0, s>>>(fr, ws->sys, ws->sys_fp32 ? 1 : 0,
                                                          ws->cells, coeffs, cap, ws->ctr, rule(), out);
    return cudaGetLastError();
}

cudaError_t launch_parab_ppic(ft_workspace* ws, const double* coeffs, long long cap, double* alpha, double* area,
                              double* kappa, double* normal, int8_t* status, cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = alpha;
    return parab_with(ws, fr, coeffs, cap, area, kappa, normal, status, s);
}

cudaError_t launch_parab_ppic_batch(ft_workspace* ws, const double* coeffs, long long cap, double* area,
                                    double* kappa, double* normal, int8_t* status, cudaStream_t s) {
    return parab_with(ws, ft_many(ws), coeffs, cap, area, kappa, normal, status, s);
}

cudaError_t launch_ppic_frame(ft_workspace* ws, long long cap, double* frame, cudaStream_t s) {
    count_launches(1);
    k_ppic_frame<<<ws->sm_count * 4, kThreads, 0, s>>>(ws->sys, ws->sys_fp32 ? 1 : 0, cap,
                                                       ws->ctr, frame);
    return cudaGetLastError();
}

}  // namespace ft
