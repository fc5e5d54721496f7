// k_rough.cu -- local roughness detection and volume-conserving smoothing of
// the front mesh (Sec. 3.4): the geometric Laplacian GL(x_i) = x_i - sum w x_j /
// sum w (w = 1/|x_i - x_j| over the one-ring), the edge roughness
// R_e = 1 - n_1 . n_2 of the two triangles at an edge, its mean G_i and
// variance V_i over the edges of each vertex, the triangle roughness
// R_t = sum G_i V_i / sum V_i, the area-weighted one- and two-ring vertex
// roughness R^1, R^2 and R = max(R^1, R^2); then the edge move of Kuprat et al.
// (2001, Algorithm 4) on every edge with a rough endpoint (|GL| and R above
// their thresholds), in rounds of edges whose stars are disjoint.
//
// Mesh adjacency is built on the device: the triangles incident to each vertex
// (counted, scanned, filled, then sorted per vertex so that every sum runs in
// ascending triangle order).  All arithmetic is float64.
#include <math.h>
#include <stdlib.h>

#include "ft_internal.cuh"

struct ft_rough {
    int device;
    long long max_nv, max_nt;
    int* cnt;        // max_nv + 1
    int* off;        // max_nv + 1
    int* cur;        // max_nv
    int* inc;        // 3 max_nt: incident triangles per vertex
    int* part;       // scan partials
    double* nrm;     // 3 max_nt unit normals
    double* area;    // max_nt
    double* G;       // max_nv
    double* V;       // max_nv
    double* gl;      // 3 max_nv (smoothing: own copy)
    double* rough;   // max_nv
    double* r1;      // max_nv
    double* r2;      // max_nv
    double* rt;      // max_nt
    unsigned char* pend;  // 3 max_nt
    unsigned char* sel;   // 3 max_nt
    double* newpos;  // 6 x 3 max_nt
    unsigned long long* npend;  // device counter
    unsigned* status;
    size_t bytes;
};

namespace {

constexpr int kT = 256;
constexpr int kScanBlock = 1024;
constexpr int kRing2Cap = 512;  // triangles of a two-ring neighbourhood (status bit beyond)

__global__ void k_count(const int* __restrict__ tris, long long nt, long long nv, int* __restrict__ cnt,
                        unsigned* status) {
    const long long t = (long long)blockIdx.x * kT + threadIdx.x;
    if (t >= nt) return;
    for (int c = 0; c < 3; c++) {
        const int v = tris[3 * t + c];
        if (v < 0 || v >= nv) {
            atomicOr(status, FT_ST_BAD_INDEX);
            continue;
        }
        atomicAdd(cnt + v, 1);
    }
}

// exclusive scan of n ints in three passes (block sums, scan of the sums, down-sweep)
__global__ void k_scan_blocks(const int* __restrict__ in, long long n, int* __restrict__ part) {
    __shared__ int s[kScanBlock / 32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    int v = i < n ? in[i] : 0;
    v = ft_warp_sum_i(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int x = s[threadIdx.x];
        x = ft_warp_sum_i(x);
        if (threadIdx.x == 0) part[blockIdx.x] = x;
    }
}

__global__ void k_scan_part(int* part, int nb) {
    // one thread: nb <= a few thousand
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int b = 0; b < nb; b++) {
        const int v = part[b];
        part[b] = run;
        run += v;
    }
    part[nb] = run;
}

__global__ void k_scan_down(const int* __restrict__ in, long long n, const int* __restrict__ part,
                            int* __restrict__ out) {
    __shared__ int s[kScanBlock / 32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = s[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s[lane] = t;
    }
    __syncthreads();
    const int excl = part[blockIdx.x] + ((w > 0) ? s[w - 1] : 0) + x - v;
    if (i < n) out[i] = excl;
    if (i == n - 1) out[n] = excl + v;
}

__global__ void k_fill(const int* __restrict__ tris, long long nt, long long nv, int* __restrict__ cur,
                       int* __restrict__ inc) {
    const long long t = (long long)blockIdx.x * kT + threadIdx.x;
    if (t >= nt) return;
    for (int c = 0; c < 3; c++) {
        const int v = tris[3 * t + c];
        if (v < 0 || v >= nv) continue;
        inc[atomicAdd(cur + v, 1)] = (int)t;
    }
}

// every vertex's triangle list in ascending order (insertion sort: short lists)
__global__ void k_sort_lists(const int* __restrict__ off, long long nv, int* __restrict__ inc) {
    const long long v = (long long)blockIdx.x * kT + threadIdx.x;
    if (v >= nv) return;
    const int a = off[v], b = off[v + 1];
    for (int i = a + 1; i < b; i++) {
        const int x = inc[i];
        int j = i - 1;
        while (j >= a && inc[j] > x) {
            inc[j + 1] = inc[j];
            j--;
        }
        inc[j + 1] = x;
    }
}

__global__ void k_tri_geom(const double* __restrict__ verts, const int* __restrict__ tris, long long nt,
                           double* __restrict__ nrm, double* __restrict__ area) {
    const long long t = (long long)blockIdx.x * kT + threadIdx.x;
    if (t >= nt) return;
    const double* a = verts + 3 * (long long)tris[3 * t];
    const double* b = verts + 3 * (long long)tris[3 * t + 1];
    const double* c = verts + 3 * (long long)tris[3 * t + 2];
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double x[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double l = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    area[t] = 0.5 * l;
    for (int d = 0; d < 3; d++) nrm[3 * t + d] = l > 0.0 ? x[d] / l : 0.0;
}

__device__ __forceinline__ int slot_of(const int* tris, long long t, long long v) {
    return tris[3 * t] == v ? 0 : (tris[3 * t + 1] == v ? 1 : (tris[3 * t + 2] == v ? 2 : -1));
}

// the triangle holding the directed edge b -> a, among those incident to a
__device__ long long twin_of(const int* __restrict__ off, const int* __restrict__ inc, const int* __restrict__ tris,
                             long long a, long long b) {
    for (int r = off[a]; r < off[a + 1]; r++) {
        const long long t = inc[r];
        const int sb = slot_of(tris, t, b);
        if (sb >= 0 && tris[3 * t + (sb + 1) % 3] == a) return t;
    }
    return -1;
}

__global__ void k_vertex_metrics(const double* __restrict__ verts, long long nv, const int* __restrict__ tris,
                                 const int* __restrict__ off, const int* __restrict__ inc,
                                 const double* __restrict__ nrm, double* __restrict__ gl, double* __restrict__ G,
                                 double* __restrict__ V) {
    const long long i = (long long)blockIdx.x * kT + threadIdx.x;
    if (i >= nv) return;
    const double xi[3] = {verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]};
    double sw = 0.0, sx[3] = {0.0, 0.0, 0.0}, sum = 0.0, sum2 = 0.0;
    int ne = 0;
    for (int r = off[i]; r < off[i + 1]; r++) {
        const long long t = inc[r];
        const int s = slot_of(tris, t, i);
        for (int o = 1; o <= 2; o++) {
            const double* xj = verts + 3 * (long long)tris[3 * t + (s + o) % 3];
            const double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
            const double w = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
            sw += w;
            for (int d = 0; d < 3; d++) sx[d] += w * xj[d];
        }
        const long long j = tris[3 * t + (s + 1) % 3];
        const long long u = twin_of(off, inc, tris, i, j);
        if (u < 0) continue;
        const double re = 1.0 - (nrm[3 * t] * nrm[3 * u] + nrm[3 * t + 1] * nrm[3 * u + 1] + nrm[3 * t + 2] * nrm[3 * u + 2]);
        sum += re;
        sum2 += re * re;
        ne++;
    }
    for (int d = 0; d < 3; d++) gl[3 * i + d] = sw > 0.0 ? xi[d] - sx[d] / sw : 0.0;
    const double g = ne ? sum / ne : 0.0;
    double v = ne ? sum2 / ne - g * g : 0.0;
    G[i] = g;
    V[i] = v < 0.0 ? 0.0 : v;
}

__global__ void k_tri_rough(const int* __restrict__ tris, long long nt, const double* __restrict__ G,
                            const double* __restrict__ V, double* __restrict__ rt) {
    const long long t = (long long)blockIdx.x * kT + threadIdx.x;
    if (t >= nt) return;
    double num = 0.0, den = 0.0, gm = 0.0;
    for (int c = 0; c < 3; c++) {
        const long long v = tris[3 * t + c];
        num += G[v] * V[v];
        den += V[v];
        gm += G[v];
    }
    rt[t] = den > 0.0 ? num / den : gm / 3.0;
}

// one- and two-ring vertex roughness; the two-ring triangles are gathered in
// the oracle's order (incident triangles of i, and of each of their vertices)
// and counted once
__global__ void k_vertex_ring(long long nv, const int* __restrict__ tris, const int* __restrict__ off,
                              const int* __restrict__ inc, const double* __restrict__ area,
                              const double* __restrict__ rt, double* __restrict__ r1, double* __restrict__ r2,
                              double* __restrict__ rough, unsigned* status) {
    const long long i = (long long)blockIdx.x * kT + threadIdx.x;
    if (i >= nv) return;
    int seen[kRing2Cap];
    int ns = 0;
    double s1 = 0.0, s2 = 0.0;
    long long c1 = 0, c2 = 0;
    bool over = false;
    for (int r = off[i]; r < off[i + 1]; r++) {
        const long long t = inc[r];
        s1 += area[t] * rt[t];
        c1++;
        for (int c = 0; c < 3; c++) {
            const long long v = tris[3 * t + c];
            for (int r2i = off[v]; r2i < off[v + 1]; r2i++) {
                const int t2 = inc[r2i];
                bool dup = false;
                for (int q = 0; q < ns && !dup; q++) dup = (seen[q] == t2);
                if (dup) continue;
                if (ns < kRing2Cap) {
                    seen[ns++] = t2;
                } else {
                    over = true;
                    continue;
                }
                s2 += area[t2] * rt[t2];
                c2++;
            }
        }
    }
    if (over) atomicOr(status, FT_ST_CAPACITY);
    const double a = c1 ? s1 / c1 : 0.0, b = c2 ? s2 / c2 : 0.0;
    r1[i] = a;
    r2[i] = b;
    rough[i] = a > b ? a : b;
}

// SplitMix64 finalizer (Steele, Lea and Flood 2014): edge priorities
__device__ __forceinline__ unsigned long long priority(unsigned long long e) {
    unsigned long long z = e + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool is_rough(const double* gl, const double* rough, long long v, double gl_thr,
                                         double r_thr) {
    const double g = sqrt(gl[3 * v] * gl[3 * v] + gl[3 * v + 1] * gl[3 * v + 1] + gl[3 * v + 2] * gl[3 * v + 2]);
    return g > gl_thr && rough[v] > r_thr;
}

__global__ void k_flag(const int* __restrict__ tris, long long nt, const double* __restrict__ gl,
                       const double* __restrict__ rough, double gl_thr, double r_thr, unsigned char* __restrict__ pend,
                       unsigned long long* npend) {
    const long long e = (long long)blockIdx.x * kT + threadIdx.x;
    if (e >= 3 * nt) return;
    const long long t = e / 3;
    const int s = (int)(e % 3);
    const long long a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
    unsigned char f = 0;
    if (a < b && (is_rough(gl, rough, a, gl_thr, r_thr) || is_rough(gl, rough, b, gl_thr, r_thr))) f = 1;
    pend[e] = f;
    if (f) atomicAdd(npend, 1ull);
}

// an edge moves in this round when its priority is the smallest among the
// pending edges touching the closed one-rings of its endpoints
__global__ void k_select(const int* __restrict__ tris, long long nt, const int* __restrict__ off,
                         const int* __restrict__ inc, const unsigned char* __restrict__ pend,
                         unsigned char* __restrict__ sel) {
    const long long e = (long long)blockIdx.x * kT + threadIdx.x;
    if (e >= 3 * nt) return;
    unsigned char best = 0;
    if (pend[e]) {
        best = 1;
        const long long t = e / 3;
        const int s = (int)(e % 3);
        const long long a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
        const unsigned long long pe = priority((unsigned long long)e);
        for (int side = 0; side < 2 && best; side++) {
            const long long v = side ? b : a;
            for (int r = off[v]; r < off[v + 1] && best; r++) {
                const long long t1 = inc[r];
                for (int c = 0; c < 3 && best; c++) {
                    const long long w = tris[3 * t1 + c];
                    for (int r2 = off[w]; r2 < off[w + 1] && best; r2++) {
                        const long long t2 = inc[r2];
                        for (int s2 = 0; s2 < 3; s2++) {
                            const long long f = 3 * t2 + s2;
                            if (f == e || !pend[f]) continue;
                            const unsigned long long pf = priority((unsigned long long)f);
                            if (pf < pe || (pf == pe && f < e)) {
                                best = 0;
                                break;
                            }
                        }
                    }
                }
            }
        }
    }
    sel[e] = best;
}

// the volume-conserving edge move: simultaneous Laplacian smoothing of both
// endpoints, then a common shift h n with 6 dV = da.A_a + db.A_b + da.(db x y) = 0
__global__ void k_move(const double* __restrict__ verts, const int* __restrict__ tris, long long nt,
                       const int* __restrict__ off, const int* __restrict__ inc,
                       const unsigned char* __restrict__ sel, double* __restrict__ newpos) {
    const long long e = (long long)blockIdx.x * kT + threadIdx.x;
    if (e >= 3 * nt || !sel[e]) return;
    const long long t = e / 3;
    const int s = (int)(e % 3);
    const long long a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3], p = tris[3 * t + (s + 2) % 3];
    const long long u = twin_of(off, inc, tris, a, b);
    const long long q = u >= 0 ? tris[3 * u + (slot_of(tris, u, b) + 2) % 3] : p;
    double Sa[3] = {0, 0, 0}, Sb[3] = {0, 0, 0}, Aa[3] = {0, 0, 0}, Ab[3] = {0, 0, 0};
    long long na = 0, nb = 0;
    for (int side = 0; side < 2; side++) {
        const long long v = side ? b : a, other = side ? a : b;
        double* S = side ? Sb : Sa;
        double* A = side ? Ab : Aa;
        long long cnt = 0;
        for (int r = off[v]; r < off[v + 1]; r++) {
            const long long tt = inc[r];
            const int sv = slot_of(tris, tt, v);
            const long long jn = tris[3 * tt + (sv + 1) % 3];
            const double* xj = verts + 3 * jn;
            const double* xk = verts + 3 * (long long)tris[3 * tt + (sv + 2) % 3];
            A[0] += xj[1] * xk[2] - xj[2] * xk[1];
            A[1] += xj[2] * xk[0] - xj[0] * xk[2];
            A[2] += xj[0] * xk[1] - xj[1] * xk[0];
            cnt++;
            if (jn != other)
                for (int d = 0; d < 3; d++) S[d] += xj[d];
        }
        if (side)
            nb = cnt;
        else
            na = cnt;
    }
    double xsa[3], xsb[3], da[3], db[3], y[3], m[3];
    const double den = (double)na * (double)nb - 1.0;
    for (int d = 0; d < 3; d++) {
        xsa[d] = (Sb[d] + (double)nb * Sa[d]) / den;
        xsb[d] = (xsa[d] + Sb[d]) / (double)nb;
        da[d] = xsa[d] - verts[3 * a + d];
        db[d] = xsb[d] - verts[3 * b + d];
        y[d] = verts[3 * p + d] - verts[3 * q + d];
    }
    const double dd[3] = {da[0] - db[0], da[1] - db[1], da[2] - db[2]};
    m[0] = Aa[0] + Ab[0] + (y[1] * dd[2] - y[2] * dd[1]);
    m[1] = Aa[1] + Ab[1] + (y[2] * dd[0] - y[0] * dd[2]);
    m[2] = Aa[2] + Ab[2] + (y[0] * dd[1] - y[1] * dd[0]);
    const double ml = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    const double dbxy[3] = {db[1] * y[2] - db[2] * y[1], db[2] * y[0] - db[0] * y[2], db[0] * y[1] - db[1] * y[0]};
    const double c0 = da[0] * Aa[0] + da[1] * Aa[1] + da[2] * Aa[2] + db[0] * Ab[0] + db[1] * Ab[1] + db[2] * Ab[2] +
                      da[0] * dbxy[0] + da[1] * dbxy[1] + da[2] * dbxy[2];
    double h = 0.0, n[3] = {0.0, 0.0, 0.0};
    if (ml > 0.0) {
        for (int d = 0; d < 3; d++) n[d] = m[d] / ml;
        h = -c0 / ml;
    }
    for (int d = 0; d < 3; d++) {
        newpos[6 * e + d] = xsa[d] + h * n[d];
        newpos[6 * e + 3 + d] = xsb[d] + h * n[d];
    }
}

__global__ void k_apply(double* __restrict__ verts, const int* __restrict__ tris, long long nt,
                        const unsigned char* __restrict__ sel, const double* __restrict__ newpos,
                        unsigned char* __restrict__ pend, unsigned long long* npend) {
    const long long e = (long long)blockIdx.x * kT + threadIdx.x;
    if (e >= 3 * nt || !sel[e]) return;
    const long long t = e / 3;
    const int s = (int)(e % 3);
    const long long a = tris[3 * t + s], b = tris[3 * t + (s + 1) % 3];
    for (int d = 0; d < 3; d++) {
        verts[3 * a + d] = newpos[6 * e + d];
        verts[3 * b + d] = newpos[6 * e + 3 + d];
    }
    pend[e] = 0;
    atomicAdd(npend, ~0ull);  // -1
}

unsigned blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

// adjacency + metrics into r (r->gl, rough, r1, r2, rt, G, V).  The vertex
// indices are checked first (and the stream synchronized): every later kernel
// reads positions through them.  Returns FT_ERR_ARG for an index out of range.
int metrics(ft_rough* r, const double* verts, long long nv, const int* tris, long long nt, cudaStream_t s) {
    cudaMemsetAsync(r->cnt, 0, sizeof(int) * (size_t)(nv + 1), s);
    cudaMemsetAsync(r->status, 0, sizeof(unsigned), s);
    const unsigned nbs = (unsigned)((nv + kScanBlock - 1) / kScanBlock);
    ft::count_launches(1);
    k_count<<<blocks(nt), kT, 0, s>>>(tris, nt, nv, r->cnt, r->status);
    unsigned st = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, r->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FT_ERR_CUDA;
    if (st & FT_ST_BAD_INDEX) return FT_ERR_ARG;
    ft::count_launches(10);
    k_scan_blocks<<<nbs, kScanBlock, 0, s>>>(r->cnt, nv, r->part);
    k_scan_part<<<1, 32, 0, s>>>(r->part, (int)nbs);
    k_scan_down<<<nbs, kScanBlock, 0, s>>>(r->cnt, nv, r->part, r->off);
    cudaMemcpyAsync(r->cur, r->off, sizeof(int) * (size_t)nv, cudaMemcpyDeviceToDevice, s);
    k_fill<<<blocks(nt), kT, 0, s>>>(tris, nt, nv, r->cur, r->inc);
    k_sort_lists<<<blocks(nv), kT, 0, s>>>(r->off, nv, r->inc);
    k_tri_geom<<<blocks(nt), kT, 0, s>>>(verts, tris, nt, r->nrm, r->area);
    k_vertex_metrics<<<blocks(nv), kT, 0, s>>>(verts, nv, tris, r->off, r->inc, r->nrm, r->gl, r->G, r->V);
    k_tri_rough<<<blocks(nt), kT, 0, s>>>(tris, nt, r->G, r->V, r->rt);
    k_vertex_ring<<<blocks(nv), kT, 0, s>>>(nv, tris, r->off, r->inc, r->area, r->rt, r->r1, r->r2, r->rough,
                                            r->status);
    return cudaGetLastError() == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

bool front_ok(const ft_rough* r, const double* verts, long long nv, const int* tris, long long nt) {
    return r && nv >= 0 && nt >= 0 && nv <= r->max_nv && nt <= r->max_nt && (nt == 0 || (verts && tris));
}

}  // namespace

extern "C" {

int ft_rough_create(ft_rough** out, int64_t max_nv, int64_t max_nt, int device, size_t* bytes) {
    if (!out || max_nv < 1 || max_nt < 1 || max_nv > 0x7ffffffeLL || 3 * max_nt > 0x7ffffffeLL) return FT_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return FT_ERR_CUDA;
    ft_rough* r = (ft_rough*)calloc(1, sizeof(ft_rough));
    if (!r) return FT_ERR_ALLOC;
    r->device = device;
    r->max_nv = max_nv;
    r->max_nt = max_nt;
    const size_t V = (size_t)max_nv, T = (size_t)max_nt;
    size_t tot = 0;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, n);
        tot += n;
    };
    al((void**)&r->cnt, sizeof(int) * (V + 1));
    al((void**)&r->off, sizeof(int) * (V + 1));
    al((void**)&r->cur, sizeof(int) * V);
    al((void**)&r->inc, sizeof(int) * 3 * T);
    al((void**)&r->part, sizeof(int) * (V / kScanBlock + 2));
    al((void**)&r->nrm, sizeof(double) * 3 * T);
    al((void**)&r->area, sizeof(double) * T);
    al((void**)&r->G, sizeof(double) * V);
    al((void**)&r->V, sizeof(double) * V);
    al((void**)&r->gl, sizeof(double) * 3 * V);
    al((void**)&r->rough, sizeof(double) * V);
    al((void**)&r->r1, sizeof(double) * V);
    al((void**)&r->r2, sizeof(double) * V);
    al((void**)&r->rt, sizeof(double) * T);
    al((void**)&r->pend, 3 * T);
    al((void**)&r->sel, 3 * T);
    al((void**)&r->newpos, sizeof(double) * 18 * T);
    al((void**)&r->npend, sizeof(unsigned long long));
    al((void**)&r->status, sizeof(unsigned));
    if (e != cudaSuccess) {
        ft_rough_destroy(r);
        cudaGetLastError();
        return FT_ERR_ALLOC;
    }
    r->bytes = tot;
    if (bytes) *bytes = tot;
    *out = r;
    return FT_OK;
}

int ft_rough_destroy(ft_rough* r) {
    if (!r) return FT_ERR_ARG;
    cudaSetDevice(r->device);
    cudaDeviceSynchronize();
    void* p[] = {r->cnt, r->off, r->cur, r->inc, r->part, r->nrm, r->area, r->G, r->V, r->gl, r->rough,
                 r->r1, r->r2, r->rt, r->pend, r->sel, r->newpos, r->npend, r->status};
    for (void* q : p)
        if (q) cudaFree(q);
    free(r);
    return FT_OK;
}

int ft_rough_status(ft_rough* r, void* stream, uint32_t* bits) {
    if (!r || !bits) return FT_ERR_ARG;
    if (cudaSetDevice(r->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, r->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

int front_roughness(ft_rough* r, const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double* gl,
                    double* rough, double* r1, double* r2, double* rt, double* G, double* V, void* stream) {
    if (!front_ok(r, verts, nv, tris, nt) || !gl || !rough) return FT_ERR_ARG;
    if (nv == 0 || nt == 0) return FT_OK;
    if (cudaSetDevice(r->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rc = metrics(r, verts, nv, tris, nt, s);
    if (rc != FT_OK) return rc;
    cudaError_t e = cudaSuccess;
    auto cp = [&](double* dst, const double* src, size_t n) {
        if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    };
    cp(gl, r->gl, 3 * (size_t)nv);
    cp(rough, r->rough, (size_t)nv);
    cp(r1, r->r1, (size_t)nv);
    cp(r2, r->r2, (size_t)nv);
    cp(rt, r->rt, (size_t)nt);
    cp(G, r->G, (size_t)nv);
    cp(V, r->V, (size_t)nv);
    return e == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

int front_roughness_smooth(ft_rough* r, double* verts, int64_t nv, const int32_t* tris, int64_t nt, double gl_thr,
                           double r_thr, int32_t max_rounds, int32_t* rounds, int64_t* moved, uint32_t* status,
                           void* stream) {
    if (!front_ok(r, verts, nv, tris, nt) || max_rounds < 0) return FT_ERR_ARG;
    if (rounds) *rounds = 0;
    if (moved) *moved = 0;
    if (status) *status = 0;
    if (nv == 0 || nt == 0) return FT_OK;
    if (cudaSetDevice(r->device) != cudaSuccess) return FT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rc = metrics(r, verts, nv, tris, nt, s);
    if (rc != FT_OK) return rc;
    cudaError_t e = cudaMemsetAsync(r->npend, 0, sizeof(unsigned long long), s);
    ft::count_launches(1);
    if (e == cudaSuccess) {
        k_flag<<<blocks(3 * nt), kT, 0, s>>>(tris, nt, r->gl, r->rough, gl_thr, r_thr, r->pend, r->npend);
        e = cudaGetLastError();
    }
    unsigned long long pending = 0, start = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&pending, r->npend, sizeof(pending), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    start = pending;
    int k = 0;
    while (e == cudaSuccess && pending > 0 && k < max_rounds) {
        ft::count_launches(3);
        k_select<<<blocks(3 * nt), kT, 0, s>>>(tris, nt, r->off, r->inc, r->pend, r->sel);
        k_move<<<blocks(3 * nt), kT, 0, s>>>(verts, tris, nt, r->off, r->inc, r->sel, r->newpos);
        k_apply<<<blocks(3 * nt), kT, 0, s>>>(verts, tris, nt, r->sel, r->newpos, r->pend, r->npend);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&pending, r->npend, sizeof(pending), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        k++;
    }
    unsigned st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, r->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (rounds) *rounds = k;
    if (moved) *moved = (int64_t)(start - pending);
    if (status) *status = st;
    return e == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

}  // extern "C"

namespace ft {

// The triangles incident to each vertex of a front (CSR: off (nv + 1), inc
// (3 nt), each list ascending), built on `s` without a host synchronization;
// cnt, cur (nv + 1) and part (nv / 1024 + 2) are scratch.  Indices out of range
// are skipped and flagged in *status.
cudaError_t launch_incidence(const int* tris, long long nt, long long nv, int* cnt, int* off, int* cur, int* inc,
                             int* part, unsigned* status, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    const unsigned nbs = (unsigned)((nv + kScanBlock - 1) / kScanBlock);
    cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nv + 1), s);
    count_launches(6);
    {
        Trace t(s, "k_count (incidence)");
        k_count<<<blocks(nt > 0 ? nt : 1), kT, 0, s>>>(tris, nt, nv, cnt, status);
    }
    k_scan_blocks<<<nbs, kScanBlock, 0, s>>>(cnt, nv, part);
    k_scan_part<<<1, 32, 0, s>>>(part, (int)nbs);
    k_scan_down<<<nbs, kScanBlock, 0, s>>>(cnt, nv, part, off);
    cudaMemcpyAsync(cur, off, sizeof(int) * (size_t)nv, cudaMemcpyDeviceToDevice, s);
    k_fill<<<blocks(nt > 0 ? nt : 1), kT, 0, s>>>(tris, nt, nv, cur, inc);
    k_sort_lists<<<blocks(nv), kT, 0, s>>>(off, nv, inc);
    return cudaGetLastError();
}

}  // namespace ft
