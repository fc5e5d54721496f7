// k_interp.cu -- front_interp_velocity: divergence-preserving interpolation of
// staggered face velocities to the front vertices (Sec. 3.1).  Inside cell
// [x-, x+] x [y-, y+] x [z-, z+]:
//   u(x) = xi (U+ + yt Uy+ + zt Uz+) + (1 - xi)(U- + yt Uy- + zt Uz-)
//          + (x+ - x)(x - x-)/(2h) (Vx+ - Vx- + Wx+ - Wx-)
// with xi = (x - x-)/h, yt = y - (y- + y+)/2, zt = z - (z- + z+)/2, and the
// same form for v and w.  Transverse face derivatives are central differences
// of the same face array (one-sided on the first and last rows).
// One thread per vertex; the face arrays are read through the read-only cache.
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;

struct FaceArr {
    const double* a;
    int e[3];  // extents
    __device__ __forceinline__ double at(int i, int j, int k) const {
        return __ldg(a + ((long long)i * e[1] + j) * e[2] + k);
    }
    // derivative along `dir` at face (i,j,k)
    __device__ __forceinline__ double grad(int dir, int i, int j, int k, double h) const {
        int idx[3] = {i, j, k};
        const int c = idx[dir], n = e[dir];
        int lo = c - 1, hi = c + 1;
        double inv = 0.5 / h;
        if (c == 0) {
            lo = 0;
            hi = 1;
            inv = 1.0 / h;
        } else if (c == n - 1) {
            lo = n - 2;
            hi = n - 1;
            inv = 1.0 / h;
        }
        idx[dir] = hi;
        const double vh = at(idx[0], idx[1], idx[2]);
        idx[dir] = lo;
        const double vl = at(idx[0], idx[1], idx[2]);
        return (vh - vl) * inv;
    }
};

__global__ void __launch_bounds__(kThreads) k_interp(ft_grid g, FaceArr U, FaceArr V, FaceArr W,
                                                     const double* __restrict__ pts, long long np,
                                                     double* __restrict__ vel) {
    const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (p >= np) return;
    const FaceArr F[3] = {U, V, W};
    const double h = g.h;
    double x[3], lo[3], hi[3];
    int c[3];
    for (int d = 0; d < 3; d++) {
        x[d] = pts[3 * p + d];
        const double f = floor(__ddiv_rn(__dsub_rn(x[d], g.origin[d]), h));
        const int n = g.n[d];
        c[d] = (f >= 0.0) ? ((f <= (double)(n - 1)) ? (int)f : n - 1) : 0;
        lo[d] = ft_plane(g.origin[d], h, c[d]);
        hi[d] = ft_plane(g.origin[d], h, c[d] + 1);
    }
    for (int d = 0; d < 3; d++) {
        const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
        const FaceArr& A = F[d];
        int ip[3] = {c[0], c[1], c[2]};
        ip[d] += 1;
        const double Am = A.at(c[0], c[1], c[2]);
        const double Ap = A.at(ip[0], ip[1], ip[2]);
        const double g1m = A.grad(e1, c[0], c[1], c[2], h);
        const double g2m = A.grad(e2, c[0], c[1], c[2], h);
        const double g1p = A.grad(e1, ip[0], ip[1], ip[2], h);
        const double g2p = A.grad(e2, ip[0], ip[1], ip[2], h);
        const double y1 = x[e1] - 0.5 * (lo[e1] + hi[e1]);
        const double y2 = x[e2] - 0.5 * (lo[e2] + hi[e2]);
        double corr = 0.0;
        for (int s = 1; s <= 2; s++) {
            const int o = (d + s) % 3;
            int bp[3] = {c[0], c[1], c[2]};
            bp[o] += 1;
            corr += F[o].grad(d, bp[0], bp[1], bp[2], h) - F[o].grad(d, c[0], c[1], c[2], h);
        }
        const double a = (x[d] - lo[d]) / h, b = (hi[d] - x[d]) / h;
        vel[3 * p + d] = a * (Ap + y1 * g1p + y2 * g2p) + b * (Am + y1 * g1m + y2 * g2m) +
                         0.5 * (hi[d] - x[d]) * a * corr;
    }
}

}  // namespace

namespace ft {

cudaError_t launch_interp(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                          long long nv, double* vel, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    FaceArr fu{U, {g->n[0] + 1, g->n[1], g->n[2]}};
    FaceArr fv{V, {g->n[0], g->n[1] + 1, g->n[2]}};
    FaceArr fw{W, {g->n[0], g->n[1], g->n[2] + 1}};
    const unsigned nb = (unsigned)((nv + kThreads - 1) / kThreads);
    count_launches(1);
    k_interp<<<nb, kThreads, 0, s>>>(*g, fu, fv, fw, verts, nv, vel);
    return cudaGetLastError();
}

}  // namespace ft
