// k_ppic.cu -- front_curvature_ppic: PPIC volume fit of a paraboloid
// z = a1 + a2 x + a3 y + a4 x^2 + a5 xy + a6 y^2 in every interfacial cell
// (Sec. 3.2, Eqs. volumefit, Wendland, volumefit2) and its curvature.
//
// In the local frame (t1, t2, n) centred at the cell centre (lengths in units
// of h), a fragment f with area vector AN, area centroid p and central second
// moment per unit area K contributes the signed projected moments (Green's
// theorem integrals over its projection Gamma_f):
//   m_f = (n . AN) v_f,  v_f = [1, x, y, x^2 + t1.K.t1, x y + t1.K.t2, y^2 + t2.K.t2],
//   G_f = (n . AN) z,    (x, y, z) = (t1.p, t2.p, n.p),
// so that int_Gamma P dA = m_f . a and int_Gamma g_f dA = G_f.  With
// u_f = w_f (n . AN)^2 the normal equations (Eq. volumefit2) read
//   sum_f u_f v_f v_f^T a = sum_f u_f z_f v_f.
//
// Two kernels:
//  * k_ppic_acc<T> -- one warp per cell (static interleaving or a global work
//    counter; kMinBlocks sets the occupancy the registers are fitted to); fragment
//    records are read in sorted pair
//    order, so a cell's fragments are one contiguous range): frame, candidate
//    fragments of the cells within ceil(delta - 1/2), a float32 support test
//    on a compact centroid array that appends the
//    fragments near or inside the support to a per-warp queue (so that the
//    expensive part runs on full warps), the exact test and the accumulation in
//    T (double: the plain path; float: the FP32 form), support growth, and a
//    warp reduction of the 27 sums (compensated hi/lo pairs for float).
//  * k_ppic_solve -- one thread per cell: the 6x6 LDL^T solve in float64, the
//    curvature of z = P(x, y) at the origin and the outputs.
#include <stddef.h>

#include <type_traits>

#include "frame.cuh"
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kQueue = 64;

struct PpicArgs {
    double delta_h, delta_growth, delta_max_h;
    int fit_min;
    int dynamic;  // 1: cells from the global work counter, 0: static interleaving
};

// coefficients c such that c . (Kxx,Kyy,Kzz,Kxy,Kxz,Kyz) = u . K . v
template <typename T>
__device__ __forceinline__ void qform(const T u[3], const T v[3], T c[6]) {
    c[0] = u[0] * v[0];
    c[1] = u[1] * v[1];
    c[2] = u[2] * v[2];
    c[3] = u[0] * v[1] + u[1] * v[0];
    c[4] = u[0] * v[2] + u[2] * v[0];
    c[5] = u[1] * v[2] + u[2] * v[1];
}

// fragment records of either precision, read as T
template <typename T> struct Rec;
template <> struct Rec<double> {
    const ft_frag* r;
    __device__ __forceinline__ void load(unsigned i, double an[3], double c[3], double k[6]) const {
        const ft_frag f = r[i];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            an[d] = f.an[d];
            c[d] = f.c[d];
        }
#pragma unroll
        for (int d = 0; d < 6; d++) k[d] = f.k[d];
    }
    __device__ __forceinline__ void load_an(unsigned i, double an[3]) const {
        an[0] = r[i].an[0];
        an[1] = r[i].an[1];
        an[2] = r[i].an[2];
    }
};
template <> struct Rec<float> {
    const ft_frag32* r;
    __device__ __forceinline__ void load(unsigned i, float an[3], float c[3], float k[6]) const {
        const ft_frag32 f = r[i];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            an[d] = f.an[d];
            c[d] = f.c[d];
        }
#pragma unroll
        for (int d = 0; d < 6; d++) k[d] = f.k[d];
    }
    __device__ __forceinline__ void load_an(unsigned i, float an[3]) const {
        an[0] = r[i].an[0];
        an[1] = r[i].an[1];
        an[2] = r[i].an[2];
    }
};

// error-free sum (Knuth's two-sum), each operation rounded on its own (no
// contraction with the surrounding code)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Transposed warp reduction of 32 values per lane: each round a lane keeps one
// half of its vector and adds the partner's copy of that half, so after five
// rounds lane l holds the warp total of value l (31 shuffles instead of 32 x 5).
__device__ __forceinline__ double warp_transpose_sum(double (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; i++) {
            const double send = up ? v[i] : v[i + o];
            const double keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// The same with float (hi, lo) pairs combined by two-sum: the lanes' rounding
// errors are carried along instead of being lost.  The lo parts start at zero,
// so the first round exchanges only the hi parts (lo = the two-sum error).
__device__ __forceinline__ void warp_transpose_sum2(float (&h)[32], float (&l)[32]) {
    const int lane = threadIdx.x & 31;
    {
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const float sh = up ? h[i] : h[i + 16];
            const float kh = up ? h[i + 16] : h[i];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, 16);
            float s, e;
            two_sum(kh, rh, s, e);
            h[i] = s;
            l[i] = e;
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; i++) {
            const float sh = up ? h[i] : h[i + o];
            const float sl = up ? l[i] : l[i + o];
            const float kh = up ? h[i + o] : h[i];
            const float kl = up ? l[i + o] : l[i];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, o);
            const float rl = __shfl_xor_sync(0xffffffffu, sl, o);
            float s, e;
            two_sum(kh, rh, s, e);
            h[i] = s;
            l[i] = kl + rl + e;
        }
    }
}

// The 27 sums of the normal equations: S (packed upper triangle of the 6x6
// matrix, row by row) and B.
template <typename T> struct Acc;

template <> struct Acc<double> {
    double S[21], B[6];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < 21; r++) S[r] = 0.0;
#pragma unroll
        for (int r = 0; r < 6; r++) B[r] = 0.0;
    }
    __device__ __forceinline__ void get(double (&s)[21], double (&b)[6]) const {
#pragma unroll
        for (int r = 0; r < 21; r++) s[r] = S[r];
#pragma unroll
        for (int r = 0; r < 6; r++) b[r] = B[r];
    }
};

// Float sums kept in pairs for the paired float instructions of this GPU
// (two fused multiply-adds per instruction): the packed entries 0..9, 11..16
// and 18..19 are nine adjacent pairs, entries 10 and 17 (rows 1 and 3, column
// 5) form one more, entry 20 stays single; B in three pairs.
template <> struct Acc<float> {
    float2 P[9], Q, Bp[3];
    float s20;
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int r = 0; r < 9; r++) P[r] = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 3; r++) Bp[r] = make_float2(0.f, 0.f);
        Q = make_float2(0.f, 0.f);
        s20 = 0.f;
    }
    __device__ __forceinline__ void get(float (&s)[21], float (&b)[6]) const {
        const int first[9] = {0, 2, 4, 6, 8, 11, 13, 15, 18};
#pragma unroll
        for (int r = 0; r < 9; r++) {
            s[first[r]] = P[r].x;
            s[first[r] + 1] = P[r].y;
        }
        s[10] = Q.x;
        s[17] = Q.y;
        s[20] = s20;
#pragma unroll
        for (int r = 0; r < 3; r++) {
            b[2 * r] = Bp[r].x;
            b[2 * r + 1] = Bp[r].y;
        }
    }
};

// The expensive part for one queued fragment: exact support test, weight,
// projected moments and the 27 accumulations.
// A queue entry (float4): the float form holds the fragment centroid relative
// to the fitted cell (x, y, z) and the record index (w); the float64 form the
// neighbour offset code (x) and the record index (w), the centroid being
// rebuilt exactly in float64.
template <typename T>
__device__ __forceinline__ void accumulate(const Rec<T>& rec, const float4 qe, T delta, T inv_delta,
                                          const T n[3], const T t1[3], const T t2[3], const T c11[6],
                                          const T c12[6], const T c22[6], T z0, Acc<T>& acc, int& count);

// One fit element (area vector an, centroid p relative to the cell centre and
// central second moment per unit area k, lengths in cells) into the float64
// normal equations, if its centroid lies inside the support.
__device__ __forceinline__ void accum_d(const double an[3], const double p[3], const double k[6], double delta,
                                        double inv_delta, const double n[3], const double t1[3], const double t2[3],
                                        const double c11[6], const double c12[6], const double c22[6], double z0,
                                        Acc<double>& acc, int& count) {
    const double d2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    const double dist = sqrt(d2);
    if (!(dist < delta)) return;
    count++;
    const double q = dist * inv_delta;
    const double om = 1.0 - q;
    const double om2 = om * om;
    const double w = (1.0 + 4.0 * q) * om2 * om2;
    const double x = t1[0] * p[0] + t1[1] * p[1] + t1[2] * p[2];
    const double y = t2[0] * p[0] + t2[1] * p[1] + t2[2] * p[2];
    const double z = n[0] * p[0] + n[1] * p[1] + n[2] * p[2] - z0;
    const double sA = n[0] * an[0] + n[1] * an[1] + n[2] * an[2];
    double q11 = 0, q12 = 0, q22 = 0;
#pragma unroll
    for (int r = 0; r < 6; r++) {
        q11 += c11[r] * k[r];
        q12 += c12[r] * k[r];
        q22 += c22[r] * k[r];
    }
    const double v[6] = {1.0, x, y, x * x + q11, x * y + q12, y * y + q22};
    const double u = w * sA * sA;
    int r = 0;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const double uv = (i == 0) ? u : u * v[i];
#pragma unroll
        for (int j = i; j < 6; j++) acc.S[r++] += uv * v[j];
        acc.B[i] += uv * z;
    }
}

template <>
__device__ __forceinline__ void accumulate<double>(const Rec<double>& rec, const float4 qe, double delta,
                                                   double inv_delta, const double n[3], const double t1[3],
                                                   const double t2[3], const double c11[6], const double c12[6],
                                                   const double c22[6], double z0, Acc<double>& acc, int& count) {
    const unsigned ri = __float_as_uint(qe.w);
    const int dcode = __float_as_int(qe.x);
    double an[3], c[3], k[6];
    rec.load(ri, an, c, k);
    const double p[3] = {c[0] + (double)(((dcode >> 8) & 15) - 8), c[1] + (double)(((dcode >> 4) & 15) - 8),
                         c[2] + (double)((dcode & 15) - 8)};
    accum_d(an, p, k, delta, inv_delta, n, t1, t2, c11, c12, c22, z0, acc, count);
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <>
__device__ __forceinline__ void accumulate<float>(const Rec<float>& rec, const float4 qe, float delta,
                                                  float inv_delta, const float n[3], const float t1[3],
                                                  const float t2[3], const float c11[6], const float c12[6],
                                                  const float c22[6], float z0, Acc<float>& acc, int& count) {
    float an[3], c[3], k[6];
    rec.load(__float_as_uint(qe.w), an, c, k);
    const float p[3] = {qe.x, qe.y, qe.z};
    const float d2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    // the support test on squared lengths; the distance from the fast reciprocal
    // square root (its rounding moves the weight by about 1e-7 of itself)
    if (!(d2 < delta * delta)) return;
    count++;
    const float q = (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f) * inv_delta;
    const float om = 1.f - q;
    const float om2 = om * om;
    const float w = (1.f + 4.f * q) * om2 * om2;
    // (x, y) = (t1 . p, t2 . p) and (z + z0, sA) = (n . p, n . AN), two lanes per instruction
    float2 xy = __fmul2_rn(f2(t1[0], t2[0]), f2(p[0], p[0]));
    xy = __ffma2_rn(f2(t1[1], t2[1]), f2(p[1], p[1]), xy);
    xy = __ffma2_rn(f2(t1[2], t2[2]), f2(p[2], p[2]), xy);
    float2 zs = __fmul2_rn(f2(n[0], n[0]), f2(p[0], an[0]));
    zs = __ffma2_rn(f2(n[1], n[1]), f2(p[1], an[1]), zs);
    zs = __ffma2_rn(f2(n[2], n[2]), f2(p[2], an[2]), zs);
    const float x = xy.x, y = xy.y, z = zs.x - z0, sA = zs.y;
    // (q11, q12) = (t1.K.t1, t1.K.t2); q22 = t2.K.t2 as two half sums
    float2 q1 = __fmul2_rn(f2(c11[0], c12[0]), f2(k[0], k[0]));
#pragma unroll
    for (int r = 1; r < 6; r++) q1 = __ffma2_rn(f2(c11[r], c12[r]), f2(k[r], k[r]), q1);
    float2 q2 = __fmul2_rn(f2(c22[0], c22[1]), f2(k[0], k[1]));
    q2 = __ffma2_rn(f2(c22[2], c22[3]), f2(k[2], k[3]), q2);
    q2 = __ffma2_rn(f2(c22[4], c22[5]), f2(k[4], k[5]), q2);
    const float q22 = q2.x + q2.y;
    // v = [1, x, y, x^2 + q11, xy + q12, y^2 + q22]
    const float2 v34 = __ffma2_rn(f2(x, x), f2(x, y), q1);
    const float v5 = y * y + q22;
    const float u = w * sA * sA;
    // uv_i = u v_i
    const float2 uv12 = __fmul2_rn(f2(u, u), f2(x, y));
    const float2 uv34 = __fmul2_rn(f2(u, u), v34);
    const float uv5 = u * v5;
    // row 0 (uv0 = u): entries 0..5
    acc.P[0] = __ffma2_rn(f2(u, u), f2(1.f, x), acc.P[0]);
    acc.P[1] = __ffma2_rn(f2(u, u), f2(y, v34.x), acc.P[1]);
    acc.P[2] = __ffma2_rn(f2(u, u), f2(v34.y, v5), acc.P[2]);
    // row 1: entries 6..9 (columns 1..4), entry 10 (column 5) in Q.x
    acc.P[3] = __ffma2_rn(f2(uv12.x, uv12.x), f2(x, y), acc.P[3]);
    acc.P[4] = __ffma2_rn(f2(uv12.x, uv12.x), v34, acc.P[4]);
    // row 2: entries 11..14 (columns 2..5)
    acc.P[5] = __ffma2_rn(f2(uv12.y, uv12.y), f2(y, v34.x), acc.P[5]);
    acc.P[6] = __ffma2_rn(f2(uv12.y, uv12.y), f2(v34.y, v5), acc.P[6]);
    // row 3: entries 15..16 (columns 3..4), entry 17 (column 5) in Q.y
    acc.P[7] = __ffma2_rn(f2(uv34.x, uv34.x), v34, acc.P[7]);
    acc.Q = __ffma2_rn(f2(uv12.x, uv34.x), f2(v5, v5), acc.Q);
    // row 4: entries 18..19 (columns 4..5); row 5: entry 20
    acc.P[8] = __ffma2_rn(f2(uv34.y, uv34.y), f2(v34.y, v5), acc.P[8]);
    acc.s20 += uv5 * v5;
    // B_i += uv_i z
    acc.Bp[0] = __ffma2_rn(f2(u, uv12.x), f2(z, z), acc.Bp[0]);
    acc.Bp[1] = __ffma2_rn(f2(uv12.y, uv34.x), f2(z, z), acc.Bp[1]);
    acc.Bp[2] = __ffma2_rn(f2(uv34.y, uv5), f2(z, z), acc.Bp[2]);
}

template <typename T, class F, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_ppic_acc(PpicArgs A, F fr, const unsigned* __restrict__ cells,
                                                       const int* __restrict__ cell_off, Rec<T> rec,
                                                       const float4* __restrict__ cen,
                                                       const int* __restrict__ idx_map, ft_counters* ctr,
                                                       ft_cellsys* __restrict__ sys, int* __restrict__ fit_info,
                                                       const double* __restrict__ n_over) {
    __shared__ float4 s_q[kWarps][kQueue];
    const long long M = ctr->M;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* qq = s_q[wid];
    unsigned long long pairs_total = 0;
    // Schedule: static interleaving (the warps of a block take consecutive
    // cells, which share most of their candidate fragments in L1), or a global
    // work counter (balances cells whose supports differ widely, as between the
    // fronts of a batch); lane 0 fetches the next index while a cell runs.
    const long long nw = (long long)gridDim.x * kWarps;
    // support radii in T (the default radii 2.5, 3.125, 3.90625, 4 are exact in float)
    const T d_start = (T)A.delta_h, d_growth = (T)A.delta_growth, d_max = (T)A.delta_max_h;
    unsigned long long next = 0;
    if (A.dynamic && lane == 0) next = atomicAdd((unsigned long long*)&ctr->work, 1ull);
    for (long long m0 = (long long)blockIdx.x * kWarps + wid;; m0 += nw) {
        long long m = m0;
        if (A.dynamic) {
            m = (long long)__shfl_sync(0xffffffffu, next, 0);
            if (m < M && lane == 0) next = atomicAdd((unsigned long long*)&ctr->work, 1ull);
        }
        if (m >= M) break;
        const unsigned gkey = cells[m];
        const int fb = fr.by_key(gkey);
        const ft_grid& G = fr.desc(fb).g;
        const int n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
        const long long kb = fr.key_base(fb);
        const unsigned key = (unsigned)(gkey - kb);
        const int ck = (int)(key % (unsigned)n2);
        const int cj = (int)((key / (unsigned)n2) % (unsigned)n1);
        const int ci = (int)(key / ((unsigned)n2 * (unsigned)n1));
        int st = 0;

        // 1. local normal: normalized sum of the cell's fragment area vectors
        T N[3] = {0, 0, 0}, sa = 0, best = -1, AC[3] = {0, 0, 0};
        int bestq = 0x7fffffff;
        const int q0 = cell_off[m], q1 = cell_off[m + 1];
        for (int q = q0 + lane; q < q1; q += 32) {
            T an[3];
            rec.load_an(q, an);
            const float4 cq = cen[q];
            N[0] += an[0];
            N[1] += an[1];
            N[2] += an[2];
            const T a = sqrt(an[0] * an[0] + an[1] * an[1] + an[2] * an[2]);
            sa += a;
            AC[0] += a * (T)cq.x;
            AC[1] += a * (T)cq.y;
            AC[2] += a * (T)cq.z;
            if (a > best) {
                best = a;
                bestq = q;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            N[0] += __shfl_xor_sync(0xffffffffu, N[0], o);
            N[1] += __shfl_xor_sync(0xffffffffu, N[1], o);
            N[2] += __shfl_xor_sync(0xffffffffu, N[2], o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            AC[0] += __shfl_xor_sync(0xffffffffu, AC[0], o);
            AC[1] += __shfl_xor_sync(0xffffffffu, AC[1], o);
            AC[2] += __shfl_xor_sync(0xffffffffu, AC[2], o);
        }
        T nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        bool given = false;
        if (n_over) {
            // the frame normal given per cell (the closest vertex's normal);
            // a zero vector keeps the fragment normal
            const double o0 = n_over[3 * m], o1 = n_over[3 * m + 1], o2 = n_over[3 * m + 2];
            if (o0 != 0.0 || o1 != 0.0 || o2 != 0.0) {
                N[0] = (T)o0;
                N[1] = (T)o1;
                N[2] = (T)o2;
                nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                given = true;
            } else {
                st |= FT_FIT_NORMAL;
            }
        }
        if (!given && nn < (T)1e-3 * sa) {
            // opposing sheets: normal of the largest fragment (first on ties)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oq = __shfl_xor_sync(0xffffffffu, bestq, o);
                if (ob > best || (ob == best && oq < bestq)) {
                    best = ob;
                    bestq = oq;
                }
            }
            rec.load_an(bestq, N);
            nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
            st |= FT_FIT_NORMAL;
        }
        const T n[3] = {N[0] / nn, N[1] / nn, N[2] / nn};
        // heights are fitted relative to the cell's own fragment centroid: a
        // shift of z that leaves a2..a6 (and so kappa and n) unchanged but keeps
        // the constant term small, which conditions the float32 form
        const T z0 = (sa > 0) ? (n[0] * AC[0] + n[1] * AC[1] + n[2] * AC[2]) / sa : (T)0;
        T t1[3], t2[3], c11[6], c12[6], c22[6];
        basis<T>(n, t1, t2);
        qform<T>(t1, t1, c11);
        qform<T>(t1, t2, c12);
        qform<T>(t2, t2, c22);

        // 2-4. normal equations; the support grows while too few fragments lie in it
        T delta = d_start;
        Acc<T> acc;
        int ctot;
        for (;;) {
            acc.zero();
            int count = 0;
            const T inv_delta = (T)1 / delta;
            // float pre-filter, slightly wider than the support; the exact test follows
            const float f_thr = (float)delta * (float)delta * 1.0001f;
            const int R = (int)ceil(delta - (T)0.5);
            const int side = 2 * R + 1;
            const int nrows = side * side;
            // row offsets decoded with a float reciprocal: (l + 1/2)/side stays at
            // least 1/(2 side) away from an integer for l < side^2, far beyond the
            // float rounding, so the truncation is exact
            const float inv_s = 1.0f / (float)side;
            int qn = 0;
            // Neighbour rows (i + di, j + dj, k - R .. k + R): keys are k-fastest, so a
            // row's interfacial cells are consecutive in the cell list and their
            // fragments one contiguous range.  Cells whose box lies beyond the
            // support hold no fragment in it (a fragment's centroid lies in its own
            // cell): each row keeps the cells |dk| <= dkmax that pass the box test.
            // Lane l takes row l of a round of 32 rows.
            for (int cb = 0; cb < nrows; cb += 32) {
                const int l = cb + lane;
                int f0 = 0, cnt = 0, dcode = 0;
                float ox = 0.f, oy = 0.f;
                unsigned rkey = 0;  // batch-global key of the row's cell at height ck
                if (l < nrows) {
                    const int a = (int)(((float)l + 0.5f) * inv_s);
                    const int di = a - R, dj = l - a * side - R;
                    const int ii = ci + di, jj = cj + dj;
                    const float bx = fmaxf(fabsf((float)di) - 0.5f, 0.0f), by = fmaxf(fabsf((float)dj) - 0.5f, 0.0f);
                    int dkmax = -1;
                    for (int t = 0; t <= R; t++) {
                        const float bz = fmaxf((float)t - 0.5f, 0.0f);
                        if (bx * bx + by * by + bz * bz <= f_thr) dkmax = t;
                    }
                    if (dkmax >= 0 && ii >= 0 && jj >= 0 && ii < n0 && jj < n1) {
                        const int k0 = max(ck - dkmax, 0), k1 = min(ck + dkmax, n2 - 1);
                        const long long base = kb + ((long long)ii * n1 + jj) * n2;
                        // the first and last interfacial cells of the row's k range (up to
                        // nine entries loaded at once; wider supports loop)
                        int mf = -1, ml = -1;
                        if (k1 - k0 < 9) {
                            int mm[9];
#pragma unroll
                            for (int t = 0; t < 9; t++) mm[t] = (k0 + t <= k1) ? __ldg(idx_map + base + k0 + t) : -1;
#pragma unroll
                            for (int t = 0; t < 9; t++)
                                if (mm[t] >= 0) {
                                    if (mf < 0) mf = mm[t];
                                    ml = mm[t];
                                }
                        } else {
                            for (int k = k0; k <= k1; k++) {
                                const int m2 = idx_map[base + k];
                                if (m2 >= 0) {
                                    if (mf < 0) mf = m2;
                                    ml = m2;
                                }
                            }
                        }
                        if (mf >= 0) {
                            f0 = cell_off[mf];
                            cnt = cell_off[ml + 1] - f0;
                        }
                        rkey = (unsigned)(base + ck);
                    }
                    dcode = ((di + 8) << 8) | ((dj + 8) << 4);
                    ox = (float)di;
                    oy = (float)dj;
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = incl - cnt;
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                // candidate fi of this round -> owning row lane o, record ri; dk from
                // the record's cell key (the w of its centroid entry); the next
                // batch's mapping and centroid load are issued before the current
                // batch is tested (software pipelining of the loads)
                auto map = [&](int fb, unsigned& ri, float& dx, float& dy, unsigned& rk, int& dc, bool& valid) {
                    const int fi = fb + lane;
                    int o = 0;
#pragma unroll
                    for (int s = 16; s > 0; s >>= 1) {
                        const int e = __shfl_sync(0xffffffffu, excl, o + s);
                        if (e <= fi) o += s;
                    }
                    const int fo = __shfl_sync(0xffffffffu, f0, o);
                    const int eo = __shfl_sync(0xffffffffu, excl, o);
                    rk = __shfl_sync(0xffffffffu, rkey, o);
                    if constexpr (sizeof(T) == 4) {
                        dx = __shfl_sync(0xffffffffu, ox, o);
                        dy = __shfl_sync(0xffffffffu, oy, o);
                        dc = 0;
                    } else {
                        // one shuffle of the offset code; the float64 form is issue-bound
                        dc = __shfl_sync(0xffffffffu, dcode, o);
                        dx = (float)(((dc >> 8) & 15) - 8);
                        dy = (float)(((dc >> 4) & 15) - 8);
                    }
                    valid = fi < total;
                    ri = valid ? (unsigned)(fo + (fi - eo)) : 0u;
                };
                unsigned ri_n = 0, rk_n = 0;
                float dx_n = 0.f, dy_n = 0.f;
                int dc_n = 0;
                bool v_n = false;
                float4 c4_n = make_float4(0.f, 0.f, 0.f, 0.f);
                if (total > 0) {
                    map(0, ri_n, dx_n, dy_n, rk_n, dc_n, v_n);
                    if (v_n) c4_n = cen[ri_n];
                }
                // (the float64 form maps each batch in turn: its registers are full)
                constexpr bool kPipe = sizeof(T) == 4;
                for (int fb = 0; fb < total; fb += 32) {
                    if (!kPipe && fb > 0) {
                        map(fb, ri_n, dx_n, dy_n, rk_n, dc_n, v_n);
                        if (v_n) c4_n = cen[ri_n];
                    }
                    const unsigned ri = ri_n, rk = rk_n;
                    const float dx = dx_n, dy = dy_n;
                    const int dc = dc_n;
                    const bool valid = v_n;
                    const float4 c4 = c4_n;
                    if (kPipe && fb + 32 < total) {
                        map(fb + 32, ri_n, dx_n, dy_n, rk_n, dc_n, v_n);
                        if (v_n) c4_n = cen[ri_n];
                    }
                    bool pass = false;
                    float4 entry = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid) {
                        // the fragment's cell lies in the row: dk = its key - the row's key at ck
                        const int dk = (int)(__float_as_uint(c4.w) - rk);
                        const float px = c4.x + dx, py = c4.y + dy, pz = c4.z + (float)dk;
                        pass = (px * px + py * py + pz * pz) < f_thr;
                        if (sizeof(T) == 4)
                            entry = make_float4(px, py, pz, __uint_as_float(ri));
                        else
                            entry = make_float4(__int_as_float(dc | (dk + 8)), 0.f, 0.f, __uint_as_float(ri));
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, pass);
                    if (pass) qq[qn + __popc(bal & ((1u << lane) - 1u))] = entry;
                    qn += __popc(bal);
                    __syncwarp();
                    if (qn >= 32) {
                        accumulate<T>(rec, qq[qn - 32 + lane], delta, inv_delta, n, t1, t2, c11, c12, c22, z0, acc,
                                      count);
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
            if (lane < qn)
                accumulate<T>(rec, qq[lane], delta, inv_delta, n, t1, t2, c11, c12, c22, z0, acc, count);
            __syncwarp();
            ctot = ft_warp_sum_i(count);
            if (ctot >= A.fit_min || delta >= d_max) break;
            delta = min(delta * d_growth, d_max);
            st |= FT_FIT_GROWN;
        }
        pairs_total += (unsigned long long)ctot;

        // 5. reduce the 27 sums over the warp (transposed: lane r ends with sum r)
        //    and leave them for the solve kernel
        ft_cellsys* out = sys + m;
        T S[21], B[6];
        acc.get(S, B);
        if (sizeof(T) == 8) {
            double v[32];
#pragma unroll
            for (int r = 0; r < 21; r++) v[r] = (double)S[r];
#pragma unroll
            for (int r = 0; r < 6; r++) v[21 + r] = (double)B[r];
#pragma unroll
            for (int r = 27; r < 32; r++) v[r] = 0.0;
            const double tot = warp_transpose_sum(v);
            if (lane < 27) out->v[lane] = tot;
            if (lane == 0) {
#pragma unroll
                for (int r = 0; r < 3; r++) out->v[27 + r] = (double)n[r];
                out->v[30] = (double)z0;
            }
        } else {
            float hv[32], lv[32];
#pragma unroll
            for (int r = 0; r < 21; r++) hv[r] = (float)S[r];
#pragma unroll
            for (int r = 0; r < 6; r++) hv[21 + r] = (float)B[r];
#pragma unroll
            for (int r = 27; r < 32; r++) hv[r] = 0.f;
            warp_transpose_sum2(hv, lv);
            float* o32 = reinterpret_cast<float*>(out->v);
            if (lane < 27) {
                o32[2 * lane] = hv[0];
                o32[2 * lane + 1] = lv[0];
            }
            if (lane == 0) {
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    o32[54 + 2 * r] = (float)n[r];
                    o32[55 + 2 * r] = 0.f;
                }
                o32[60] = (float)z0;
            }
        }
        if (lane == 0) {
            fit_info[2 * m] = ctot;
            fit_info[2 * m + 1] = st;
        }
    }
    if (lane == 0 && pairs_total) atomicAdd((unsigned long long*)&ctr->fit_pairs, pairs_total);
}

// LDL^T solve of the leading N x N block of the packed symmetric 6x6 system
// (N a compile-time size: every loop unrolls, the factors stay in registers).
// Returns the smallest pivot relative to the trace (-1 if a pivot is not > 0).
__device__ __forceinline__ constexpr int packed(int i, int j) {  // i <= j
    return i * 6 - (i * (i - 1)) / 2 + (j - i);
}

template <int N>
__device__ __forceinline__ double ldlt_solve(const double (&S)[21], const double (&B)[6], double (&a)[6]) {
    double Lm[N][N], d[N], inv_d[N];
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) tr += S[packed(i, i)];
    double minp = INFINITY;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; j++) {
        double dj = S[packed(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) dj -= Lm[j][k] * Lm[j][k] * d[k];
        d[j] = dj;
        minp = fmin(minp, dj);
        ok = ok && (dj > 0.0);
        inv_d[j] = 1.0 / dj;  // one float64 division per pivot
#pragma unroll
        for (int i = j + 1; i < N; i++) {
            double v = S[packed(j, i)];
#pragma unroll
            for (int k = 0; k < j; k++) v -= Lm[i][k] * Lm[j][k] * d[k];
            Lm[i][j] = v * inv_d[j];
        }
    }
    if (!ok) return -1.0;
    double y[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        double v = B[i];
#pragma unroll
        for (int k = 0; k < i; k++) v -= Lm[i][k] * y[k];
        y[i] = v;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        double v = y[i] * inv_d[i];
#pragma unroll
        for (int k = i + 1; k < N; k++) v -= Lm[k][i] * a[k];
        a[i] = v;
    }
    return minp / tr;
}

// Double-float numbers hi + lo (Dekker's double-length arithmetic: two-sum and
// the fused-multiply-add exact product, renormalised after every operation),
// about 48 significant bits on the float32 pipe.  The FP32 form solves its
// normal equations in them: their sums arrive as compensated float pairs, and
// on this GPU a float64 instruction costs the SM sub-partition as much as
// dozens of float32 ones.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl df_fast(float s, float e) {  // |s| >= |e|
    const float h = __fadd_rn(s, e);
    return dfl{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl df_norm(float a, float b) {
    float s, e;
    two_sum(a, b, s, e);
    return dfl{s, e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df_fast(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, dfl{-b.hi, -b.lo}); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // the product's rounding error, exactly
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast(p, e);
}
__device__ __forceinline__ dfl df_rcp(dfl b) {  // 1 / b: a float quotient and one correction
    const float q1 = 1.f / b.hi;
    const dfl r = df_sub(dfl{1.f, 0.f}, df_mul(dfl{q1, 0.f}, b));
    return df_fast(q1, __fmul_rn(r.hi, q1));
}

// ldlt_solve in double-float (same steps; the relative pivot in float).
template <int N>
__device__ __forceinline__ float ldlt_solve_df(const dfl (&S)[21], const dfl (&B)[6], dfl (&a)[6]) {
    dfl Lm[N][N], d[N], inv_d[N];
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < N; i++) tr += S[packed(i, i)].hi;
    float minp = INFINITY;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; j++) {
        dfl dj = S[packed(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) dj = df_sub(dj, df_mul(df_mul(Lm[j][k], Lm[j][k]), d[k]));
        d[j] = dj;
        minp = fminf(minp, dj.hi);
        ok = ok && (dj.hi > 0.f);
        inv_d[j] = df_rcp(dj);
#pragma unroll
        for (int i = j + 1; i < N; i++) {
            dfl v = S[packed(j, i)];
#pragma unroll
            for (int k = 0; k < j; k++) v = df_sub(v, df_mul(df_mul(Lm[i][k], Lm[j][k]), d[k]));
            Lm[i][j] = df_mul(v, inv_d[j]);
        }
    }
    if (!ok) return -1.f;
    dfl y[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        dfl v = B[i];
#pragma unroll
        for (int k = 0; k < i; k++) v = df_sub(v, df_mul(Lm[i][k], y[k]));
        y[i] = v;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        dfl v = df_mul(y[i], inv_d[i]);
#pragma unroll
        for (int k = i + 1; k < N; k++) v = df_sub(v, df_mul(Lm[k][i], a[k]));
        a[i] = v;
    }
    return minp / tr;
}

// One thread per cell on kSolveLanes lanes of each warp, in blocks of
// kSolveThreads.  The solve is bound by the float64 pipe of the SM
// sub-partition each warp runs on; spreading the cells over more warps with
// fewer active lanes does not help (a float64 warp instruction costs the same
// with 16 or 8 lanes active: the PPIC step took 4 % and 19 % longer), and
// one-warp blocks measured the same as blocks of four.
constexpr int kSolveThreads = 128;
constexpr int kSolveLanes = 32;

template <class F, bool FP32>
__global__ void __launch_bounds__(kSolveThreads) k_ppic_solve(F fr, const ft_cellsys* __restrict__ sys,
                                                              const int* __restrict__ fit_info,
                                                              const unsigned* __restrict__ cells, long long cap,
                                                              ft_counters* ctr, unsigned* __restrict__ out_keys,
                                                              double* __restrict__ out_kappa,
                                                              double* __restrict__ out_normal,
                                                              double* __restrict__ out_coeffs,
                                                              int8_t* __restrict__ out_status) {
    const long long M = ctr->M;
    if (M > cap) {  // the caller's arrays are too short: write nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) ft_flag(ctr, FT_ST_CAPACITY);
        return;
    }
    const int lane = threadIdx.x & 31;
    if (lane >= kSolveLanes) return;
    const long long wid = ((long long)blockIdx.x * kSolveThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kSolveThreads) >> 5;
    for (long long m = wid * kSolveLanes + lane; m < M; m += nw * kSolveLanes) {
        int st = fit_info[2 * m + 1];
        const unsigned key = cells[m];
        out_keys[m] = key;
        if constexpr (FP32) {
            // The FP32 form, without float64 instructions: the compensated pairs as
            // double-float numbers, the frame rebuilt in float from the stored float
            // normal exactly as the accumulation built it, the curvature and the
            // normal in float (their tolerance is 1e-4), widened by integer operations
            const float* v = reinterpret_cast<const float*>(sys[m].v);
            dfl S[21], B[6], ad[6];
#pragma unroll
            for (int r = 0; r < 21; r++) S[r] = df_norm(v[2 * r], v[2 * r + 1]);
#pragma unroll
            for (int r = 0; r < 6; r++) B[r] = df_norm(v[42 + 2 * r], v[43 + 2 * r]);
            const float z0 = v[60];
            const float n[3] = {v[54], v[56], v[58]};
#pragma unroll
            for (int r = 0; r < 6; r++) ad[r] = dfl{0.f, 0.f};
            const float rel = ldlt_solve_df<6>(S, B, ad);
            if (!(rel >= 1e-12f)) {
                // singular: plane fit on the leading 3x3 block, kappa = 0
                dfl a3[6];
#pragma unroll
                for (int r = 0; r < 6; r++) ad[r] = dfl{0.f, 0.f};
                if (ldlt_solve_df<3>(S, B, a3) > 0.f)
                    for (int r = 0; r < 3; r++) ad[r] = a3[r];
                st |= FT_FIT_SINGULAR;
            }
            ad[0] = df_add(ad[0], dfl{z0, 0.f});  // undo the height shift (it changes a1 only)
            float a[6];
#pragma unroll
            for (int r = 0; r < 6; r++) a[r] = __fadd_rn(ad[r].hi, ad[r].lo);
            float t1[3], t2[3];
            basis<float>(n, t1, t2);
            // mean curvature of the graph z = P(x, y) at the origin, kappa = div n
            const float g2 = 1.f + a[1] * a[1] + a[2] * a[2];
            const float kl = -(2.f * a[3] * (1.f + a[2] * a[2]) - 2.f * a[1] * a[2] * a[4] +
                               2.f * a[5] * (1.f + a[1] * a[1])) / (g2 * sqrtf(g2));
            float nv[3];
            for (int d = 0; d < 3; d++) nv[d] = n[d] - a[1] * t1[d] - a[2] * t2[d];
            const float il = 1.f / sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
            out_kappa[m] = ft_f2d(kl * (float)fr.desc(fr.by_key(key)).inv_h);
            for (int d = 0; d < 3; d++) out_normal[3 * m + d] = ft_f2d(nv[d] * il);
            if (out_coeffs)
                for (int r = 0; r < 6; r++) out_coeffs[6 * m + r] = ft_f2d(ad[r].hi) + ft_f2d(ad[r].lo);
        } else {
            double S[21], B[6], n[3];
            double a[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int r = 0; r < 21; r++) S[r] = sys[m].v[r];
#pragma unroll
            for (int r = 0; r < 6; r++) B[r] = sys[m].v[21 + r];
            const double z0 = sys[m].v[30];
            const double rel = ldlt_solve<6>(S, B, a);
            if (!(rel >= 1e-12)) {
                // singular: plane fit on the leading 3x3 block, kappa = 0
                for (int r = 0; r < 6; r++) a[r] = 0.0;
                double a3[6] = {0, 0, 0, 0, 0, 0};
                if (ldlt_solve<3>(S, B, a3) > 0.0) {
                    a[0] = a3[0];
                    a[1] = a3[1];
                    a[2] = a3[2];
                }
                st |= FT_FIT_SINGULAR;
            }
            sys_normal(sys[m], false, n);
            double t1[3], t2[3];
            basis<double>(n, t1, t2);
            a[0] += z0;  // undo the height shift (it changes a1 only)
            // mean curvature of the graph z = P(x, y) at the origin, kappa = div n
            const double g2 = 1.0 + a[1] * a[1] + a[2] * a[2];
            const double kl = -(2.0 * a[3] * (1.0 + a[2] * a[2]) - 2.0 * a[1] * a[2] * a[4] +
                                2.0 * a[5] * (1.0 + a[1] * a[1])) / (g2 * sqrt(g2));
            double nv[3];
            for (int d = 0; d < 3; d++) nv[d] = n[d] - a[1] * t1[d] - a[2] * t2[d];
            const double il = 1.0 / sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
            out_kappa[m] = kl * fr.desc(fr.by_key(key)).inv_h;
            for (int d = 0; d < 3; d++) out_normal[3 * m + d] = nv[d] * il;
            if (out_coeffs)
                for (int r = 0; r < 6; r++) out_coeffs[6 * m + r] = a[r];
        }
        out_status[m] = (int8_t)st;
    }
}

// ---------------------------------------------------------------------------
// The paper's own fit neighbourhood and frame (Sec. 3.2): the front vertex
// closest to the cell centre, its normal as the frame normal, and the whole
// triangles of the k-ring of triangles around it as the fit elements (the
// Wendland distance taken from each triangle's centre), in float64.
//  * k_edge_max -- the longest triangle edge of the front (squared), which
//    bounds how far the closest vertex can be from an interfacial cell centre;
//  * k_closest -- one warp per interfacial cell: the closest vertex among the
//    vertices of the triangles binned within that distance (|x - x_c|^2
//    rounded operation by operation, ties to the lowest index) and its normal,
//    the normalized sum of its triangles' area vectors in ascending order;
//  * k_ppic_ring -- one warp per cell: the k-ring (sorted, unique) in shared
//    memory, then the volume fit over its triangles as k_ppic_acc does over
//    fragments.
// ---------------------------------------------------------------------------
constexpr int kRingCap = 512;    // triangles of one k-ring
constexpr int kRingCand = 1024;  // incident-triangle entries gathered for one ring step

struct RingArgs {
    const double* verts;
    const int* tris;
    const int* inc_off;  // nv + 1
    const int* inc;      // 3 nt: triangles of each vertex, ascending
    long long nv;
    int ring;            // k (0: not used)
    int frame_vertex;
};

__global__ void k_edge_max(const double* __restrict__ verts, const int* __restrict__ tris, long long nt,
                           unsigned long long* out) {
    double best = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
        const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        const int e[3][2] = {{a, b}, {b, c}, {c, a}};
        for (int q = 0; q < 3; q++) {
            double l2 = 0.0;
            for (int d = 0; d < 3; d++) {
                const double x = verts[3 * (long long)e[q][1] + d] - verts[3 * (long long)e[q][0] + d];
                l2 += x * x;
            }
            best = fmax(best, l2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

__device__ __forceinline__ double cell_centre(double o, double h, int i) {
    return __dadd_rn(o, __dmul_rn((double)i + 0.5, h));
}

template <class F>
__global__ void __launch_bounds__(kThreads) k_closest(F fr, RingArgs R, const unsigned* __restrict__ cells,
                                                      const int* __restrict__ cell_off,
                                                      const unsigned* __restrict__ slot_of,
                                                      const int* __restrict__ cand_tri,
                                                      const int* __restrict__ idx_map, const ft_counters* ctr,
                                                      const unsigned long long* lmax2_bits, int* __restrict__ cv,
                                                      double* __restrict__ vn) {
    const long long M = ctr->M;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWarps;
    const ft_grid& G = fr.desc(0).g;
    const double h = G.h;
    // the closest vertex lies within D = (sqrt 3 / 2) h + L_max / sqrt 3 of the
    // centre of an interfacial cell (a front point lies in the cell; every point
    // of a triangle is within L_max / sqrt 3 of one of its vertices), so one of
    // its triangles is binned in a cell within r_v cells
    const double D = 0.8660254037844387 * h + sqrt(__longlong_as_double((long long)*lmax2_bits)) * 0.5773502691896258;
    const int rv = (int)floor(D / h + 0.5) + 1;
    for (long long m = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); m < M; m += nw) {
        const unsigned key = cells[m];
        const int n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
        const int ck = (int)(key % (unsigned)n2), cj = (int)((key / (unsigned)n2) % (unsigned)n1),
                  ci = (int)(key / ((unsigned)n2 * (unsigned)n1));
        const double xc[3] = {cell_centre(G.origin[0], h, ci), cell_centre(G.origin[1], h, cj),
                              cell_centre(G.origin[2], h, ck)};
        double bd = INFINITY;
        int bv = 0x7fffffff;
        const int side = 2 * rv + 1;
        const long long nb = (long long)side * side * side;
        for (long long l = lane; l < nb; l += 32) {
            const int di = (int)(l / (side * side)) - rv, dj = (int)((l / side) % side) - rv, dk = (int)(l % side) - rv;
            const int ii = ci + di, jj = cj + dj, kk = ck + dk;
            if (ii < 0 || jj < 0 || kk < 0 || ii >= n0 || jj >= n1 || kk >= n2) continue;
            const int m2 = idx_map[((long long)ii * n1 + jj) * n2 + kk];
            if (m2 < 0) continue;
            for (int q = cell_off[m2]; q < cell_off[m2 + 1]; q++) {
                const int t = cand_tri[slot_of[q]];
                for (int c = 0; c < 3; c++) {
                    const int v = R.tris[3 * (long long)t + c];
                    const double dx = __dsub_rn(R.verts[3 * (long long)v], xc[0]);
                    const double dy = __dsub_rn(R.verts[3 * (long long)v + 1], xc[1]);
                    const double dz = __dsub_rn(R.verts[3 * (long long)v + 2], xc[2]);
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    if (d2 < bd || (d2 == bd && v < bv)) {
                        bd = d2;
                        bv = v;
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
            if (od < bd || (od == bd && ov < bv)) {
                bd = od;
                bv = ov;
            }
        }
        if (lane == 0) {
            cv[m] = bv;
            // its normal: the sum of its triangles' area vectors, ascending order
            double s[3] = {0.0, 0.0, 0.0};
            if (bv >= 0 && bv < R.nv) {
                for (int q = R.inc_off[bv]; q < R.inc_off[bv + 1]; q++) {
                    const long long t = R.inc[q];
                    const double* a = R.verts + 3 * (long long)R.tris[3 * t];
                    const double* b = R.verts + 3 * (long long)R.tris[3 * t + 1];
                    const double* c = R.verts + 3 * (long long)R.tris[3 * t + 2];
                    const double e1[3] = {__dsub_rn(b[0], a[0]), __dsub_rn(b[1], a[1]), __dsub_rn(b[2], a[2])};
                    const double e2[3] = {__dsub_rn(c[0], a[0]), __dsub_rn(c[1], a[1]), __dsub_rn(c[2], a[2])};
                    s[0] = __dadd_rn(s[0], __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1])));
                    s[1] = __dadd_rn(s[1], __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2])));
                    s[2] = __dadd_rn(s[2], __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0])));
                }
            }
            const double l = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            for (int d = 0; d < 3; d++) vn[3 * m + d] = (l > 0.0) ? s[d] / l : 0.0;
        }
    }
}

// warp bitonic sort of s[0..n) ascending (n a power of two, <= kRingCand)
__device__ void warp_sort(int* s, int n) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const int a = s[i], b = s[p];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s[i] = b;
                        s[p] = a;
                    }
                }
            }
            __syncwarp();
        }
}

template <class F, typename TR>
__global__ void __launch_bounds__(kThreads) k_ppic_ring(PpicArgs A, F fr, RingArgs R, const unsigned* __restrict__ cells,
                                                        const int* __restrict__ cell_off, Rec<TR> rec,
                                                        ft_counters* ctr, const int* __restrict__ cv,
                                                        const double* __restrict__ vn, ft_cellsys* __restrict__ sys,
                                                        int* __restrict__ fit_info, unsigned* status) {
    __shared__ int s_ring[kWarps][kRingCap];
    __shared__ int s_cand[kWarps][kRingCand];
    const long long M = ctr->M;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* ring = s_ring[wid];
    int* cand = s_cand[wid];
    const long long nw = (long long)gridDim.x * kWarps;
    const ft_grid& G = fr.desc(0).g;
    const double h = G.h, inv_h = fr.desc(0).inv_h;
    unsigned long long pairs_total = 0;
    for (long long m = (long long)blockIdx.x * kWarps + wid; m < M; m += nw) {
        const unsigned key = cells[m];
        const int n1 = G.n[1], n2 = G.n[2];
        const int ck = (int)(key % (unsigned)n2), cj = (int)((key / (unsigned)n2) % (unsigned)n1),
                  ci = (int)(key / ((unsigned)n2 * (unsigned)n1));
        const double xc[3] = {cell_centre(G.origin[0], h, ci), cell_centre(G.origin[1], h, cj),
                              cell_centre(G.origin[2], h, ck)};
        int st = 0;
        // frame normal: the closest vertex's (frame_vertex) or the cell's fragments'
        double n[3];
        bool given = false;
        if (R.frame_vertex && (vn[3 * m] != 0.0 || vn[3 * m + 1] != 0.0 || vn[3 * m + 2] != 0.0)) {
            for (int d = 0; d < 3; d++) n[d] = vn[3 * m + d];
            given = true;
        }
        if (!given) {
            if (R.frame_vertex) st |= FT_FIT_NORMAL;
            double N[3] = {0, 0, 0}, sa = 0.0, best = -1.0;
            int bestq = 0x7fffffff;
            for (int q = cell_off[m] + lane; q < cell_off[m + 1]; q += 32) {
                TR at[3];
                rec.load_an(q, at);
                const double an[3] = {(double)at[0], (double)at[1], (double)at[2]};
                for (int d = 0; d < 3; d++) N[d] += an[d];
                const double a = sqrt(an[0] * an[0] + an[1] * an[1] + an[2] * an[2]);
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
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oq = __shfl_xor_sync(0xffffffffu, bestq, o);
                    if (ob > best || (ob == best && oq < bestq)) {
                        best = ob;
                        bestq = oq;
                    }
                }
                TR at[3];
                rec.load_an(bestq, at);
                for (int d = 0; d < 3; d++) N[d] = (double)at[d];
                nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                st |= FT_FIT_NORMAL;
            }
            for (int d = 0; d < 3; d++) n[d] = N[d] / nn;
        }
        double t1[3], t2[3], c11[6], c12[6], c22[6];
        basis<double>(n, t1, t2);
        qform<double>(t1, t1, c11);
        qform<double>(t1, t2, c12);
        qform<double>(t2, t2, c22);
        // the k-ring of the closest vertex: its triangles, then k - 1 times every
        // triangle sharing a vertex with the ring (sorted, duplicates removed)
        const int v0 = cv[m];
        int nr = 0;
        bool over = false;
        if (v0 >= 0 && v0 < R.nv) {
            const int b0 = R.inc_off[v0];
            nr = R.inc_off[v0 + 1] - b0;
            if (nr > kRingCap) {
                over = true;
                nr = kRingCap;
            }
            for (int q = lane; q < nr; q += 32) ring[q] = R.inc[b0 + q];
            __syncwarp();
            for (int r = 2; r <= R.ring; r++) {
                // gather, per ring triangle and corner, that vertex's triangles
                int nc = 0;
                for (int q0 = 0; q0 < 3 * nr; q0 += 32) {
                    const int q = q0 + lane;
                    int u = -1, deg = 0;
                    if (q < 3 * nr) {
                        u = R.tris[3 * (long long)ring[q / 3] + q % 3];
                        deg = R.inc_off[u + 1] - R.inc_off[u];
                    }
                    int incl = deg;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int base = nc + incl - deg;
                    for (int e = 0; e < deg; e++)
                        if (base + e < kRingCand) cand[base + e] = R.inc[R.inc_off[u] + e];
                    nc += __shfl_sync(0xffffffffu, incl, 31);
                }
                if (nc > kRingCand) {
                    over = true;
                    nc = kRingCand;
                }
                int np2 = 32;
                while (np2 < nc) np2 <<= 1;
                for (int q = nc + lane; q < np2; q += 32) cand[q] = 0x7fffffff;
                __syncwarp();
                warp_sort(cand, np2);
                // unique, in order, into the ring
                int nu = 0;
                for (int q0 = 0; q0 < nc; q0 += 32) {
                    const int q = q0 + lane;
                    const bool head = q < nc && (q == 0 || cand[q] != cand[q - 1]);
                    const unsigned bal = __ballot_sync(0xffffffffu, head);
                    const int pos = nu + __popc(bal & ((1u << lane) - 1u));
                    if (head && pos < kRingCap) ring[pos] = cand[q];
                    nu += __popc(bal);
                }
                if (nu > kRingCap) {
                    over = true;
                    nu = kRingCap;
                }
                nr = nu;
                __syncwarp();
            }
        }
        if (over && lane == 0) atomicOr(status, FT_ST_CAPACITY);
        // 2-4. normal equations over the ring's triangles; the support grows
        // while fewer than fit_min of them lie inside it
        double delta = A.delta_h;
        Acc<double> acc;
        int ctot;
        for (;;) {
            acc.zero();
            int count = 0;
            const double inv_delta = 1.0 / delta;
            for (int q = lane; q < nr; q += 32) {
                const long long t = ring[q];
                double p[3][3];
                for (int c = 0; c < 3; c++)
                    for (int d = 0; d < 3; d++)
                        p[c][d] = (R.verts[3 * (long long)R.tris[3 * t + c] + d] - xc[d]) * inv_h;
                double cen[3], an[3], k[6], e1[3], e2[3], r0[3], r1[3], r2[3];
                for (int d = 0; d < 3; d++) {
                    cen[d] = (p[0][d] + p[1][d] + p[2][d]) / 3.0;
                    e1[d] = p[1][d] - p[0][d];
                    e2[d] = p[2][d] - p[0][d];
                    r0[d] = p[0][d] - cen[d];
                    r1[d] = p[1][d] - cen[d];
                    r2[d] = p[2][d] - cen[d];
                }
                an[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
                an[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
                an[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
                // central second moment per unit area of a triangle: (1/12) sum_i r_i r_i^T
                const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
                for (int r = 0; r < 6; r++)
                    k[r] = (r0[ia[r]] * r0[ib[r]] + r1[ia[r]] * r1[ib[r]] + r2[ia[r]] * r2[ib[r]]) * (1.0 / 12.0);
                accum_d(an, cen, k, delta, inv_delta, n, t1, t2, c11, c12, c22, 0.0, acc, count);
            }
            ctot = ft_warp_sum_i(count);
            if (ctot >= A.fit_min || delta >= A.delta_max_h) break;
            delta = fmin(delta * A.delta_growth, A.delta_max_h);
            st |= FT_FIT_GROWN;
        }
        pairs_total += (unsigned long long)ctot;
        double S[21], B[6];
        acc.get(S, B);
        double v[32];
#pragma unroll
        for (int r = 0; r < 21; r++) v[r] = S[r];
#pragma unroll
        for (int r = 0; r < 6; r++) v[21 + r] = B[r];
#pragma unroll
        for (int r = 27; r < 32; r++) v[r] = 0.0;
        const double tot = warp_transpose_sum(v);
        ft_cellsys* out = sys + m;
        if (lane < 27) out->v[lane] = tot;
        if (lane == 0) {
            for (int r = 0; r < 3; r++) out->v[27 + r] = n[r];
            out->v[30] = 0.0;
            fit_info[2 * m] = ctot;
            fit_info[2 * m + 1] = st;
        }
        __syncwarp();
    }
    if (lane == 0 && pairs_total) atomicAdd((unsigned long long*)&ctr->fit_pairs, pairs_total);
}
}  // namespace

namespace ft {

template <class T>
cudaError_t grow(T** p, long long n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(n > 0 ? n : 1));
}

// Buffers of the paper-neighbourhood fit, allocated on first use and grown
// with the front (vertex incidence) or sized by the cell capacity.
cudaError_t ring_buffers(ft_workspace* ws) {
    cudaError_t e = cudaSuccess;
    if (ws->f_nv > ws->inc_nv_cap || !ws->inc_off) {
        const long long nv = ws->f_nv > 1 ? ws->f_nv : 1;
        e = e ? e : grow(&ws->inc_cnt, nv + 1);
        e = e ? e : grow(&ws->inc_off, nv + 1);
        e = e ? e : grow(&ws->inc_cur, nv + 1);
        e = e ? e : grow(&ws->inc_part, nv / 1024 + 2);
        if (e == cudaSuccess) ws->inc_nv_cap = nv;
    }
    if (ws->f_nt > ws->inc_nt_cap || !ws->inc) {
        const long long nt = ws->f_nt > 1 ? ws->f_nt : 1;
        e = e ? e : grow(&ws->inc, 3 * nt);
        if (e == cudaSuccess) ws->inc_nt_cap = nt;
    }
    if (!ws->cv) e = e ? e : grow(&ws->cv, ws->max_cells);
    if (!ws->vn) e = e ? e : grow(&ws->vn, 3 * ws->max_cells);
    return e;
}

template <class F>
cudaError_t ppic_with(ft_workspace* ws, const F& fr, const ft_params* p, long long cap, unsigned* cell_keys,
                      double* kappa, double* normal, double* coeffs, int8_t* fit_status, cudaStream_t s) {
    PpicArgs A;
    A.delta_h = p->delta_h;
    A.delta_growth = p->delta_growth;
    A.delta_max_h = p->delta_max_h;
    A.fit_min = p->fit_min;
    A.dynamic = ws->tune.ppic_dynamic;
    // fit_pairs and the work counter are adjacent: one reset
    static_assert(offsetof(ft_counters, work) == offsetof(ft_counters, fit_pairs) + sizeof(long long), "layout");
    cudaMemsetAsync(&ws->ctr->fit_pairs, 0, 2 * sizeof(long long), s);
    bool fp32 = ws->last_precision == FT_FP32C;
    const unsigned nb = (unsigned)(ws->sm_count * ws->tune.ppic_bps);
    const double* n_over = nullptr;
    if constexpr (std::is_same<F, FrontsOne>::value) {
        if (p->fit_ring > 0 || p->frame == FT_FRAME_VERTEX) {
            // the paper's own neighbourhood and frame: mesh incidence, the
            // longest edge, then the closest vertex of every cell and its normal
            cudaError_t e = ring_buffers(ws);
            if (e != cudaSuccess) return e;
            RingArgs R{ws->f_verts, ws->f_tris, ws->inc_off, ws->inc, ws->f_nv, p->fit_ring,
                       p->frame == FT_FRAME_VERTEX ? 1 : 0};
            e = launch_incidence(ws->f_tris, ws->f_nt, ws->f_nv, ws->inc_cnt, ws->inc_off, ws->inc_cur, ws->inc,
                                 ws->inc_part, &ws->ctr->status, s);
            if (e != cudaSuccess) return e;
            cudaMemsetAsync(&ws->ctr->lmax2_bits, 0, sizeof(unsigned long long), s);
            count_launches(2);
            {
                Trace t(s, "k_edge_max");
                k_edge_max<<<ws->sm_count * 2, 256, 0, s>>>(ws->f_verts, ws->f_tris, ws->f_nt, &ws->ctr->lmax2_bits);
            }
            {
                Trace t(s, "k_closest");
                k_closest<F><<<ws->sm_count * 4, kThreads, 0, s>>>(fr, R, ws->cells, ws->cell_off,
                                                                    ws->vals[ws->sorted_buf], ws->cand_tri,
                                                                    ws->idx_map, ws->ctr, &ws->ctr->lmax2_bits,
                                                                    ws->cv, ws->vn);
            }
            if (p->fit_ring > 0) {
                // the ring fit (float64 in both forms) writes float64 normal equations
                count_launches(2);
                {
                    Trace t(s, "k_ppic_ring");
                    // (the records only give the fragment normal when the frame is the fragments')
                    if (fp32)
                        k_ppic_ring<F, float><<<ws->sm_count * 4, kThreads, 0, s>>>(
                            A, fr, R, ws->cells, ws->cell_off, Rec<float>{ws->srec32}, ws->ctr, ws->cv, ws->vn,
                            ws->sys, ws->fit_info, &ws->ctr->status);
                    else
                        k_ppic_ring<F, double><<<ws->sm_count * 4, kThreads, 0, s>>>(
                            A, fr, R, ws->cells, ws->cell_off, Rec<double>{ws->srec}, ws->ctr, ws->cv, ws->vn,
                            ws->sys, ws->fit_info, &ws->ctr->status);
                }
                ws->sys_fp32 = false;
                Trace t(s, "k_ppic_solve");
                k_ppic_solve<F, false><<<ws->sm_count * (512 / kSolveThreads), kSolveThreads, 0, s>>>(
                    fr, ws->sys, ws->fit_info, ws->cells, cap, ws->ctr, cell_keys, kappa, normal, coeffs,
                    fit_status);
                return cudaGetLastError();
            }
            n_over = ws->vn;
        }
    }
    count_launches(2);
    // fragments are read in sorted pair order (front_bin gathers them)
    if (fp32) {
        Rec<float> r{ws->srec32};
        Trace t(s, "k_ppic_acc<float>");
        if (ws->tune.ppic_min_blocks >= 6)
            k_ppic_acc<float, F, 6><<<nb, kThreads, 0, s>>>(A, fr, ws->cells, ws->cell_off, r, ws->scen, ws->idx_map,
                                                           ws->ctr, ws->sys, ws->fit_info, n_over);
        else
            k_ppic_acc<float, F, 4><<<nb, kThreads, 0, s>>>(A, fr, ws->cells, ws->cell_off, r, ws->scen, ws->idx_map,
                                                           ws->ctr, ws->sys, ws->fit_info, n_over);
    } else {
        Rec<double> r{ws->srec};
        Trace t(s, "k_ppic_acc<double>");
        k_ppic_acc<double, F, 3><<<nb, kThreads, 0, s>>>(A, fr, ws->cells, ws->cell_off, r, ws->scen, ws->idx_map,
                                                        ws->ctr, ws->sys, ws->fit_info, n_over);
    }
    ws->sys_fp32 = fp32;
    Trace t(s, "k_ppic_solve");
    if (fp32)
        k_ppic_solve<F, true><<<ws->sm_count * (512 / kSolveThreads), kSolveThreads, 0, s>>>(
            fr, ws->sys, ws->fit_info, ws->cells, cap, ws->ctr, cell_keys, kappa, normal, coeffs, fit_status);
    else
        k_ppic_solve<F, false><<<ws->sm_count * (512 / kSolveThreads), kSolveThreads, 0, s>>>(
            fr, ws->sys, ws->fit_info, ws->cells, cap, ws->ctr, cell_keys, kappa, normal, coeffs, fit_status);
    return cudaGetLastError();
}

cudaError_t launch_ppic(ft_workspace* ws, const ft_params* p, long long cap, unsigned* cell_keys, double* kappa,
                        double* normal, double* coeffs, int8_t* fit_status, cudaStream_t s) {
    if (ws->batch)
        return ppic_with(ws, ft_many(ws), p, cap, cell_keys, kappa, normal, coeffs, fit_status, s);
    return ppic_with(ws, ft_one(ws, nullptr, nullptr, 0, 0), p, cap, cell_keys, kappa, normal, coeffs, fit_status,
                     s);
}

}  // namespace ft
