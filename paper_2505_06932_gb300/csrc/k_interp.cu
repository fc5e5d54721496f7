// k_interp.cu -- front_interp_velocity and front_advect_rk4 (Sec. 3.1):
// divergence-preserving interpolation of staggered face velocities to the
// front vertices, and the RK4 step that advects them.  Inside cell
// [x-, x+] x [y-, y+] x [z-, z+]:
//   u(x) = xi (U+ + yt Uy+ + zt Uz+) + (1 - xi)(U- + yt Uy- + zt Uz-)
//          + (x+ - x)(x - x-)/(2h) (Vx+ - Vx- + Wx+ - Wx-)
// with xi = (x - x-)/h, yt = y - (y- + y+)/2, zt = z - (z- + z+)/2, and the
// same form for v and w.  Transverse face derivatives are central differences
// of the same face array (one-sided on the first and last rows).
// One thread per vertex (batch-global vertex index in the batched form); the
// face arrays are read through the read-only cache.
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
    __device__ __forceinline__ double grad(int dir, int i, int j, int k, double inv_h) const {
        int idx[3] = {i, j, k};
        const int c = idx[dir], n = e[dir];
        int lo = c - 1, hi = c + 1;
        double inv = 0.5 * inv_h;
        if (c == 0) {
            lo = 0;
            hi = 1;
            inv = inv_h;
        } else if (c == n - 1) {
            lo = n - 2;
            hi = n - 1;
            inv = inv_h;
        }
        idx[dir] = hi;
        const double vh = at(idx[0], idx[1], idx[2]);
        idx[dir] = lo;
        const double vl = at(idx[0], idx[1], idx[2]);
        return (vh - vl) * inv;
    }
};

// the interpolated velocity u at point x of front D
__device__ __forceinline__ void interp_at(const ft_fdesc& D, const FaceArr (&F)[3], const double x[3], double u[3]) {
    const ft_grid& g = D.g;
    const double h = g.h, ih = D.inv_h;
    double lo[3], hi[3];
    int c[3];
    for (int d = 0; d < 3; d++) {
        // floor((x - origin) / h) with the quotient rounded once: the product with
        // the rounded 1/h is within 3.4e-16 |q| of that quotient (three
        // roundings), under 4e-7 for |q| < 2^30, so its floor is the same unless
        // q lies within 1e-6 of an integer (or is that large), where the
        // division itself decides
        const double dx = __dsub_rn(x[d], g.origin[d]);
        const double q = __dmul_rn(dx, ih);
        double f = floor(q);
        const double r = q - f;
        if (!(r > 1e-6 && r < 1.0 - 1e-6 && fabs(q) < 1073741824.0)) f = floor(__ddiv_rn(dx, h));
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
        const double g1m = A.grad(e1, c[0], c[1], c[2], ih);
        const double g2m = A.grad(e2, c[0], c[1], c[2], ih);
        const double g1p = A.grad(e1, ip[0], ip[1], ip[2], ih);
        const double g2p = A.grad(e2, ip[0], ip[1], ip[2], ih);
        const double y1 = x[e1] - 0.5 * (lo[e1] + hi[e1]);
        const double y2 = x[e2] - 0.5 * (lo[e2] + hi[e2]);
        double corr = 0.0;
        for (int s = 1; s <= 2; s++) {
            const int o = (d + s) % 3;
            int bp[3] = {c[0], c[1], c[2]};
            bp[o] += 1;
            corr += F[o].grad(d, bp[0], bp[1], bp[2], ih) - F[o].grad(d, c[0], c[1], c[2], ih);
        }
        const double a = (x[d] - lo[d]) * ih, b = (hi[d] - x[d]) * ih;
        u[d] = a * (Ap + y1 * g1p + y2 * g2p) + b * (Am + y1 * g1m + y2 * g2m) + 0.5 * (hi[d] - x[d]) * a * corr;
    }
}

template <class Fr>
__global__ void __launch_bounds__(kThreads) k_interp(Fr fr, long long np) {
    const long long gp = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (gp >= np) return;
    const int b = fr.by_vert(gp);
    const ft_fdesc& D = fr.desc(b);
    const long long p = gp - fr.vert_base(b);
    const ft_grid g = D.g;
    const FaceArr F[3] = {FaceArr{D.U, {g.n[0] + 1, g.n[1], g.n[2]}}, FaceArr{D.V, {g.n[0], g.n[1] + 1, g.n[2]}},
                          FaceArr{D.W, {g.n[0], g.n[1], g.n[2] + 1}}};
    double x[3], u[3];
    for (int d = 0; d < 3; d++) x[d] = D.verts[3 * p + d];
    interp_at(D, F, x, u);
    for (int d = 0; d < 3; d++) D.vel[3 * p + d] = u[d];
}

// One classical fourth-order Runge-Kutta step of dx/dt = u(x) (Sec. 3.1) with
// the face field held fixed: k1 = u(x), k2 = u(x + dt/2 k1), k3 = u(x + dt/2 k2),
// k4 = u(x + dt k3), x_new = x + dt/6 (k1 + 2 k2 + 2 k3 + k4).  Every stage of a
// vertex reads only that vertex, so x_new may overwrite x.  vel (optional)
// receives k1, the velocity of front_interp_velocity.
template <class Fr>
__global__ void __launch_bounds__(kThreads) k_advect(Fr fr, long long np) {
    const long long gp = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (gp >= np) return;
    const int b = fr.by_vert(gp);
    const ft_fdesc& D = fr.desc(b);
    const double dt = D.dt;
    const long long p = gp - fr.vert_base(b);
    const ft_grid g = D.g;
    const FaceArr F[3] = {FaceArr{D.U, {g.n[0] + 1, g.n[1], g.n[2]}}, FaceArr{D.V, {g.n[0], g.n[1] + 1, g.n[2]}},
                          FaceArr{D.W, {g.n[0], g.n[1], g.n[2] + 1}}};
    double x[3], y[3], k[3], acc[3];
    for (int d = 0; d < 3; d++) x[d] = D.verts[3 * p + d];
    interp_at(D, F, x, k);
    if (D.vel)
        for (int d = 0; d < 3; d++) D.vel[3 * p + d] = k[d];
    for (int d = 0; d < 3; d++) {
        acc[d] = k[d];
        y[d] = x[d] + 0.5 * dt * k[d];
    }
    interp_at(D, F, y, k);
    for (int d = 0; d < 3; d++) {
        acc[d] += 2.0 * k[d];
        y[d] = x[d] + 0.5 * dt * k[d];
    }
    interp_at(D, F, y, k);
    for (int d = 0; d < 3; d++) {
        acc[d] += 2.0 * k[d];
        y[d] = x[d] + dt * k[d];
    }
    interp_at(D, F, y, k);
    double* out = D.verts_next;
    for (int d = 0; d < 3; d++) out[3 * p + d] = x[d] + dt / 6.0 * (acc[d] + k[d]);
}

}  // namespace

namespace ft {

cudaError_t launch_interp(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                          long long nv, double* vel, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    FrontsOne fr;
    fr.d0 = ft_fdesc{};
    fr.d0.g = *g;
    fr.d0.verts = verts;
    fr.d0.nv = nv;
    fr.d0.U = U;
    fr.d0.V = V;
    fr.d0.W = W;
    fr.d0.vel = vel;
    fr.d0.inv_h = 1.0 / g->h;
    fr.ncells = 0;
    fr.ncols = 0;
    const unsigned nb = (unsigned)((nv + kThreads - 1) / kThreads);
    count_launches(1);
    Trace t(s, "k_interp");
    k_interp<FrontsOne><<<nb, kThreads, 0, s>>>(fr, nv);
    return cudaGetLastError();
}

cudaError_t launch_advect(const ft_grid* g, const double* U, const double* V, const double* W, const double* verts,
                          long long nv, double dt, double* verts_out, double* vel, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    FrontsOne fr;
    fr.d0 = ft_fdesc{};
    fr.d0.g = *g;
    fr.d0.verts = verts;
    fr.d0.verts_next = verts_out;
    fr.d0.nv = nv;
    fr.d0.U = U;
    fr.d0.V = V;
    fr.d0.W = W;
    fr.d0.vel = vel;
    fr.d0.dt = dt;
    fr.d0.inv_h = 1.0 / g->h;
    fr.ncells = 0;
    fr.ncols = 0;
    const unsigned nb = (unsigned)((nv + kThreads - 1) / kThreads);
    count_launches(1);
    k_advect<FrontsOne><<<nb, kThreads, 0, s>>>(fr, nv);
    return cudaGetLastError();
}

cudaError_t launch_advect_batch(ft_workspace* ws, cudaStream_t s) {
    const long long nv = ws->nv_total;
    if (nv <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nv + kThreads - 1) / kThreads);
    count_launches(1);
    k_advect<FrontsMany><<<nb, kThreads, 0, s>>>(ft_many(ws), nv);
    return cudaGetLastError();
}

cudaError_t launch_interp_batch(ft_workspace* ws, cudaStream_t s) {
    const long long nv = ws->nv_total;
    if (nv <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nv + kThreads - 1) / kThreads);
    count_launches(1);
    Trace t(s, "k_interp");
    k_interp<FrontsMany><<<nb, kThreads, 0, s>>>(ft_many(ws), nv);
    return cudaGetLastError();
}

}  // namespace ft
