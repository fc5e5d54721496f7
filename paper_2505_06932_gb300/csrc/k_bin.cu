// k_bin.cu -- front_bin, part 1: candidate cells of every triangle and the
// canonical clip predicate (Sec. 3.2, "interfacial cells"), with the fragment
// moments that the volume fraction and the PPIC fit use later.
//
// The predicate is an exact definition, not an approximation: each arithmetic
// step is one IEEE binary64 operation with round-to-nearest (the __d*_rn
// intrinsics are never contracted into FMA), so every decision is reproducible
// bit for bit by any implementation that follows the same definition.
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Order-preserving integer key of a finite double: comparing keys as signed
// 64-bit integers gives exactly the result of comparing the doubles (-0 and +0
// map to the same key), on the integer pipe instead of the float64 one.
__device__ __forceinline__ long long okey(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

// Plane coordinates of one front: the table entry when the front has a table
// (identical values: the table is filled with the same canonical operations),
// else origin + i h computed here.
struct Planes {
    const double* t;
    int off1, off2;  // first Y and Z entries
    double o[3], h;
    __device__ __forceinline__ explicit Planes(const ft_fdesc& D)
        : t(D.planes), off1(D.g.n[0] + 1), off2(D.g.n[0] + D.g.n[1] + 2),
          o{D.g.origin[0], D.g.origin[1], D.g.origin[2]}, h(D.g.h) {}
    __device__ __forceinline__ double at(int ax, long long i) const {
        if (t) return __ldg(t + (ax == 0 ? 0 : (ax == 1 ? off1 : off2)) + i);
        return ft_plane(ax == 0 ? o[0] : (ax == 1 ? o[1] : o[2]), h, i);
    }
};

// Candidate range along one axis: cells whose closed extent [X_i, X_i+1] meets
// [lo, hi]: i0 = min{i : X_i+1 >= lo}, i1 = max{i : X_i <= hi}.  The product
// with 1/h is only a starting guess; the exact comparisons make the result exact.
__device__ __forceinline__ float d2f_rn(double x);

// first guess of the cell index of coordinate x along an axis: the offset
// from the origin in float64, the rest in float32 (the exact answer comes from
// the integer plane-key comparisons after it; a guess off by one cell costs
// one more comparison)
__device__ __forceinline__ int cell_guess(double x, double o, float inv_h, int n) {
    const float f = floorf(d2f_rn(x - o) * inv_h);
    return (f >= 0.0f) ? ((f <= (float)(n - 1)) ? (int)f : n - 1) : 0;
}

__device__ void cand_range(const Planes& P, int ax, double inv_h, int n, double lo, double hi, int& i0, int& i1) {
    const double o = ax == 0 ? P.o[0] : (ax == 1 ? P.o[1] : P.o[2]);  // (no dynamic index: registers)
    const float ihf = d2f_rn(inv_h);
    const long long klo = okey(lo), khi = okey(hi);
    int e = cell_guess(lo, o, ihf, n);
    while (e > 0 && okey(P.at(ax, e)) >= klo) e--;
    while (e < n - 1 && okey(P.at(ax, e + 1)) < klo) e++;
    i0 = e;
    e = cell_guess(hi, o, ihf, n);
    while (e < n - 1 && okey(P.at(ax, e + 1)) <= khi) e++;
    while (e > 0 && okey(P.at(ax, e)) > khi) e--;
    i1 = e;
}

// The plane table of front blockIdx.y (grid-stride over its entries).
template <class F>
__global__ void __launch_bounds__(kThreads) k_planes(F fr) {
    const ft_fdesc& D = fr.desc((int)blockIdx.y);
    double* out = const_cast<double*>(D.planes);
    const ft_grid g = D.g;
    const int n0 = g.n[0] + 1, n1 = g.n[1] + 1, n2 = g.n[2] + 1;
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < n0 + n1 + n2; e += gridDim.x * kThreads) {
        const int ax = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
        const int i = e - (ax == 0 ? 0 : (ax == 1 ? n0 : n0 + n1));
        out[e] = ft_plane(g.origin[ax], g.h, i);
    }
}

// The FP32 clip's view of a triangle (32 words, eight 16-byte loads): its
// vertices in cell units relative to the lower planes of its candidate box,
// t = (x - X_lo) / h in binary64, kept as the float pair hi + lo (hi = t
// rounded to float, lo = t - hi rounded to float); its normal direction in
// float; per vertex and axis the index A (relative to the box) of the last
// plane at or below the coordinate, X_{lo+A} <= x < X_{lo+A+1}; bit 3a+ax of
// eq set when x == X_{lo+A} exactly.  The exact inside flags of vertex a for
// candidate cell lo + o then follow from integers alone: x >= X_{lo+o} iff
// o <= A, x <= X_{lo+o+1} iff o >= A - eq.
struct __align__(16) Tri32 {
    float hi[9];  // vertex a, axis ax at 3a + ax
    float lo[9];
    float tn[3];  // normal direction
    int A[9];
    unsigned eq;
    int pad;
};
static_assert(sizeof(Tri32) == 32 * sizeof(float), "Tri32 is eight 16-byte words");

// Per triangle: the candidate box (cells whose closed extent meets the
// triangle's closed bounding box) and its size.  tri_box holds lo[3], ext[3]
// and the owning front per triangle (8 ints); tri32 (when given) the record
// above.
template <class F>
__global__ void __launch_bounds__(kThreads) k_tri_setup(F fr, long long T, int margin, long long max_cand,
                                                        int* __restrict__ tri_cnt, int* __restrict__ tri_box,
                                                        double* __restrict__ tri_nrm, float* __restrict__ tri32,
                                                        const unsigned* __restrict__ cells,
                                                        int* __restrict__ idx_map, ft_counters* ctr) {
    const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
    // first the index map entries of the previous binning's cells go back to -1
    const long long M_prev = ctr->M;
    for (long long m = t; m < M_prev; m += (long long)gridDim.x * kThreads) idx_map[cells[m]] = -1;
    if (t == 0) {
        ctr->T = T;
        ctr->clip_f64 = 0;
    }
    if (t >= T) return;
    const int b = fr.by_tri(t);
    const ft_fdesc& D = fr.desc(b);
    const ft_grid g = D.g;
    const long long tl = t - fr.tri_base(b);
    const long long nv = D.nv;
    const double* __restrict__ verts = D.verts;
    int cnt = 0;
    int box[6] = {0, 0, 0, 1, 1, 1};
    unsigned err = 0;
    int vi[3];
    for (int c = 0; c < 3; c++) {
        vi[c] = D.tris[3 * tl + c];
        if (vi[c] < 0 || vi[c] >= nv) err |= FT_ST_BAD_INDEX;
    }
    if (!err) {
        // extent per axis by exact integer-key comparisons (no float64 arithmetic)
        double mn[3], mx[3];
        bool finite = true;
        for (int ax = 0; ax < 3; ax++) {
            double lo = 0.0, hi = 0.0;
            long long klo = 0, khi = 0;
            for (int c = 0; c < 3; c++) {
                const double x = verts[3 * (long long)vi[c] + ax];
                const long long bits = __double_as_longlong(x);
                finite = finite && ((bits & 0x7ff0000000000000ll) != 0x7ff0000000000000ll);
                const long long kx = okey(x);
                if (c == 0 || kx < klo) { klo = kx; lo = x; }
                if (c == 0 || kx > khi) { khi = kx; hi = x; }
            }
            mn[ax] = lo;
            mx[ax] = hi;
        }
        if (!finite) err |= FT_ST_OUTSIDE_GRID;
        long long total = 1;
        const Planes P(D);
        for (int ax = 0; ax < 3 && !err; ax++) {
            int i0, i1;
            cand_range(P, ax, D.inv_h, g.n[ax], mn[ax], mx[ax], i0, i1);
            if (i0 < margin || i1 > g.n[ax] - 1 - margin) err |= FT_ST_OUTSIDE_GRID;
            box[ax] = i0;
            box[3 + ax] = i1 - i0 + 1;
            total *= (long long)(i1 - i0 + 1);
        }
        if (!err) {
            if (total > max_cand) {
                err |= FT_ST_CAPACITY;
                total = max_cand + 1;  // still counted so that the total exceeds the capacity
            }
            cnt = (int)total;
        }
    }
    if (err) {
        ft_flag(ctr, err);
        fr.flag(b, err);
    }
    tri_cnt[t] = (err & ~FT_ST_CAPACITY) ? 0 : cnt;
    // normal direction (orientation of every fragment of the triangle; zero if
    // degenerate): twice the area vector in units of h^2.  Only its direction
    // matters -- the moments use ratios of areas signed along it.  (The FP32
    // clip's record carries its own float normal instead.)
    double nrm[3] = {0.0, 0.0, 0.0};
    if (!err && !tri32) {
        double e1[3], e2[3];
        for (int d = 0; d < 3; d++) {
            e1[d] = (verts[3 * (long long)vi[1] + d] - verts[3 * (long long)vi[0] + d]) * D.inv_h;
            e2[d] = (verts[3 * (long long)vi[2] + d] - verts[3 * (long long)vi[0] + d]) * D.inv_h;
        }
        nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    }
    if (!tri32) {
        double2* nb = reinterpret_cast<double2*>(tri_nrm + 4 * t);
        nb[0] = make_double2(nrm[0], nrm[1]);
        nb[1] = make_double2(nrm[2], 0.0);
    }
    int4* bx = reinterpret_cast<int4*>(tri_box + 8 * t);
    bx[0] = make_int4(box[0], box[1], box[2], box[3]);
    bx[1] = make_int4(box[4], box[5], b, 0);
    if (tri32) {
        float hv[9], lv[9], tn[3] = {0.f, 0.f, 0.f};
        int A[9];
        unsigned eq = 0u;
#pragma unroll
        for (int q = 0; q < 9; q++) {
            hv[q] = lv[q] = 0.f;
            A[q] = 0;
        }
        if (!err) {
            const Planes P(D);
#pragma unroll
            for (int ax = 0; ax < 3; ax++) {
                const int lo = box[ax], ext = box[3 + ax];
                const double xlo = P.at(ax, lo);
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const double x = verts[3 * (long long)vi[a] + ax];
                    const double tt = __dmul_rn(__dsub_rn(x, xlo), D.inv_h);
                    const float f = d2f_rn(tt);
                    hv[3 * a + ax] = f;
                    lv[3 * a + ax] = d2f_rn(__dsub_rn(tt, ft_f2d(f)));
                    // Every vertex lies in [X_lo, X_{lo+ext}]: A in [0, ext - 1].  f is
                    // within 1e-7 (1 + |f|) of the exact plane-relative position (the
                    // planes are spaced h apart to within 1e-8 h), so away from an
                    // integer its floor is A and the coordinate lies on no plane;
                    // near one, the exact comparisons decide
                    const float fl = floorf(f), fr = f - fl;
                    const float m = 1e-5f + 1e-6f * fabsf(f);
                    int i = (int)fminf(fmaxf(fl, 0.f), (float)(ext - 1));
                    if (!(fr > m && fr < 1.f - m)) {
                        const long long kx = okey(x);
                        while (i > 0 && okey(P.at(ax, lo + i)) > kx) i--;
                        while (i < ext - 1 && okey(P.at(ax, lo + i + 1)) <= kx) i++;
                        if (okey(P.at(ax, lo + i)) == kx) eq |= 1u << (3 * a + ax);
                    }
                    A[3 * a + ax] = i;
                }
            }
            // the normal direction from the float-pair edges, each 2x2 determinant
            // with Kahan's fused-multiply-add correction (accurate despite cancellation)
            float e1[3], e2[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                e1[d] = __fadd_rn(__fsub_rn(hv[3 + d], hv[d]), __fsub_rn(lv[3 + d], lv[d]));
                e2[d] = __fadd_rn(__fsub_rn(hv[6 + d], hv[d]), __fsub_rn(lv[6 + d], lv[d]));
            }
            auto det2 = [](float a, float b, float c, float d) {  // a d - b c
                const float w = __fmul_rn(b, c);
                const float e = __fmaf_rn(-b, c, w);
                return __fadd_rn(__fmaf_rn(a, d, -w), e);
            };
            tn[0] = det2(e1[1], e1[2], e2[1], e2[2]);
            tn[1] = det2(e1[2], e1[0], e2[2], e2[0]);
            tn[2] = det2(e1[0], e1[1], e2[0], e2[1]);
        }
        float4* o4 = reinterpret_cast<float4*>(tri32 + 32 * t);
        int4* i4 = reinterpret_cast<int4*>(tri32 + 32 * t);
        o4[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
        o4[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
        o4[2] = make_float4(hv[8], lv[0], lv[1], lv[2]);
        o4[3] = make_float4(lv[3], lv[4], lv[5], lv[6]);
        o4[4] = make_float4(lv[7], lv[8], tn[0], tn[1]);
        o4[5] = make_float4(tn[2], __int_as_float(A[0]), __int_as_float(A[1]), __int_as_float(A[2]));
        i4[6] = make_int4(A[3], A[4], A[5], A[6]);
        i4[7] = make_int4(A[7], A[8], (int)eq, 0);
    }
}

// ---------------------------------------------------------------------------
// canonical clip
// ---------------------------------------------------------------------------

// One Sutherland-Hodgman step against coord[ax] >= pv (ge) or <= pv (!ge).
// Returns false if the output would exceed MAXV vertices.
template <int MAXV>
__device__ __forceinline__ bool clip_half(const double (*in)[3], int n, double (*out)[3], int& m, int ax,
                                          double pv, bool ge) {
    m = 0;
    const long long kp = okey(pv);
    const long long kl = okey(in[n - 1][ax]);
    bool pin = ge ? (kl >= kp) : (kl <= kp);
    for (int i = 0; i < n; i++) {
        const double* cur = in[i];
        const double* prev = in[i == 0 ? n - 1 : i - 1];
        const long long kc = okey(cur[ax]);
        const bool cin = ge ? (kc >= kp) : (kc <= kp);
        if (cin != pin) {
            if (m >= MAXV) return false;
            const double t = __ddiv_rn(__dsub_rn(pv, prev[ax]), __dsub_rn(cur[ax], prev[ax]));
#pragma unroll
            for (int c = 0; c < 3; c++)
                out[m][c] = (c == ax) ? pv : __dadd_rn(prev[c], __dmul_rn(t, __dsub_rn(cur[c], prev[c])));
            m++;
        }
        if (cin) {
            if (m >= MAXV) return false;
            out[m][0] = cur[0];
            out[m][1] = cur[1];
            out[m][2] = cur[2];
            m++;
        }
        pin = cin;
    }
    return true;
}

// The six clip stages of the canonical predicate for triangle v and cell idx,
// followed by the upper-face test.  Returns the vertex count (>= 3) of the
// surviving polygon in res, 0 if rejected, -1 if MAXV was too small.  The
// remaining condition (fan area vector not zero) is checked by the caller.
template <int MAXV>
__device__ int canon_stages(const double (*v)[3], const ft_grid& g, const int idx[3], double (*res)[3]) {
    double A[MAXV][3], B[MAXV][3];
    int n = 3;
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) A[c][d] = v[c][d];
    double(*src)[3] = A;
    double(*dst)[3] = B;
    for (int ax = 0; ax < 3; ax++) {
        for (int side = 0; side < 2; side++) {
            int m;
            const double pv = ft_plane(g.origin[ax], g.h, idx[ax] + side);
            if (!clip_half<MAXV>(src, n, dst, m, ax, pv, side == 0)) return -1;
            if (m < 3) return 0;
            n = m;
            double(*tmp)[3] = src;
            src = dst;
            dst = tmp;
        }
    }
    for (int ax = 0; ax < 3; ax++) {
        const long long ku = okey(ft_plane(g.origin[ax], g.h, idx[ax] + 1));
        bool all = true;
        for (int m = 0; m < n && all; m++) all = (okey(src[m][ax]) == ku);
        if (all) return 0;
    }
    for (int m = 0; m < n; m++)
        for (int d = 0; d < 3; d++) res[m][d] = src[m][d];
    return n;
}

// The canonical fan area vector sum_m (p_m - p_0) x (p_m+1 - p_0), exactly as
// defined (binary64, round to nearest, no contraction); true if not zero.
__device__ bool canon_area_nonzero(const double (*p)[3], int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int m = 1; m + 1 < n; m++) {
        const double e1x = __dsub_rn(p[m][0], p[0][0]), e1y = __dsub_rn(p[m][1], p[0][1]),
                     e1z = __dsub_rn(p[m][2], p[0][2]);
        const double e2x = __dsub_rn(p[m + 1][0], p[0][0]), e2y = __dsub_rn(p[m + 1][1], p[0][1]),
                     e2z = __dsub_rn(p[m + 1][2], p[0][2]);
        s0 = __dadd_rn(s0, __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y)));
        s1 = __dadd_rn(s1, __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z)));
        s2 = __dadd_rn(s2, __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x)));
    }
    return !(s0 == 0.0 && s1 == 0.0 && s2 == 0.0);
}

__device__ __noinline__ int canon_stages_wide(const double (*v)[3], const ft_grid& g, const int idx[3],
                                              double (*res)[3]) {
    return canon_stages<32>(v, g, idx, res);
}

// Fragment moments in units of h relative to the fragment cell's centre, in one
// pass over the fan triangles (p0, p_m, p_m+1) of the convex fragment polygon.
// Fan areas are signed along the triangle's normal direction tn (a fragment
// lies in its triangle's plane, with the triangle's orientation), so the
// centroid and second moment need no second pass; they are ratios of such
// areas, so the length of tn cancels.  q0 = (p0 - cell centre) / h.
__device__ void frag_moments(const double (*p)[3], int n, const double q0[3], const double tn[3], double inv_h,
                             ft_frag& f) {
    double an[3] = {0.0, 0.0, 0.0}, m1[3] = {0, 0, 0}, m2[6] = {0, 0, 0, 0, 0, 0}, As = 0.0;
    double e1[3], e2[3];
    for (int d = 0; d < 3; d++) e1[d] = (p[1][d] - p[0][d]) * inv_h;
    for (int m = 1; m + 1 < n; m++) {
        for (int d = 0; d < 3; d++) e2[d] = (p[m + 1][d] - p[0][d]) * inv_h;
        const double cr0 = e1[1] * e2[2] - e1[2] * e2[1];
        const double cr1 = e1[2] * e2[0] - e1[0] * e2[2];
        const double cr2 = e1[0] * e2[1] - e1[1] * e2[0];
        an[0] += 0.5 * cr0;
        an[1] += 0.5 * cr1;
        an[2] += 0.5 * cr2;
        const double a = 0.5 * (cr0 * tn[0] + cr1 * tn[1] + cr2 * tn[2]);
        As += a;
        const double s[3] = {e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]};
        const double a3 = a * (1.0 / 3.0), a12 = a * (1.0 / 12.0);
        for (int d = 0; d < 3; d++) m1[d] += a3 * s[d];
        // int x_i x_j over a triangle with one vertex at the origin:
        // (A/12) (s_i s_j + e1_i e1_j + e2_i e2_j)
        m2[0] += a12 * (s[0] * s[0] + e1[0] * e1[0] + e2[0] * e2[0]);
        m2[1] += a12 * (s[1] * s[1] + e1[1] * e1[1] + e2[1] * e2[1]);
        m2[2] += a12 * (s[2] * s[2] + e1[2] * e1[2] + e2[2] * e2[2]);
        m2[3] += a12 * (s[0] * s[1] + e1[0] * e1[1] + e2[0] * e2[1]);
        m2[4] += a12 * (s[0] * s[2] + e1[0] * e1[2] + e2[0] * e2[2]);
        m2[5] += a12 * (s[1] * s[2] + e1[1] * e1[2] + e2[1] * e2[2]);
        for (int d = 0; d < 3; d++) e1[d] = e2[d];
    }
    if (As > 0.0) {
        const double ia = 1.0 / As;
        const double c[3] = {m1[0] * ia, m1[1] * ia, m1[2] * ia};
        f.k[0] = m2[0] * ia - c[0] * c[0];
        f.k[1] = m2[1] * ia - c[1] * c[1];
        f.k[2] = m2[2] * ia - c[2] * c[2];
        f.k[3] = m2[3] * ia - c[0] * c[1];
        f.k[4] = m2[4] * ia - c[0] * c[2];
        f.k[5] = m2[5] * ia - c[1] * c[2];
        for (int d = 0; d < 3; d++) f.c[d] = q0[d] + c[d];
    } else {
        for (int d = 0; d < 6; d++) f.k[d] = 0.0;
        for (int d = 0; d < 3; d++) f.c[d] = q0[d];
    }
    for (int d = 0; d < 3; d++) f.an[d] = an[d];
}

// double -> float with round to nearest even, in integer operations: on this
// GPU the conversion instruction runs on the float64 pipe at the float64 rate,
// which the canonical clip already saturates.  Identical to the hardware
// conversion for zero and for results in the normal float range; anything
// else (float subnormals, overflow) takes the hardware conversion.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sign = hi & 0x80000000u;
    if (((hi << 1) | lo) == 0u) return __uint_as_float(sign);
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e < 1023 - 126 || e > 1023 + 127) return (float)x;
    const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rb = lo & 0x1fffffffu, half = 0x10000000u;
    unsigned r = sign | ((unsigned)(e - 1023 + 127) << 23) | m23;
    if (rb > half || (rb == half && (m23 & 1u))) r += 1u;  // a carry moves into the exponent, as it should
    return __uint_as_float(r);
}

// The same moments in float32 (the FP32 form): each vertex offset from p0 is
// formed in float64 and rounded once; all products and sums are float32.
__device__ void frag_moments32(const double (*p)[3], int n, const float q0[3], const float tn[3], float inv_h,
                               ft_frag32& f) {
    float an[3] = {0.f, 0.f, 0.f}, m1[3] = {0, 0, 0}, m2[6] = {0, 0, 0, 0, 0, 0}, As = 0.f;
    float e1[3], e2[3];
    for (int d = 0; d < 3; d++) e1[d] = d2f_rn(p[1][d] - p[0][d]) * inv_h;
    for (int m = 1; m + 1 < n; m++) {
        for (int d = 0; d < 3; d++) e2[d] = d2f_rn(p[m + 1][d] - p[0][d]) * inv_h;
        const float cr0 = e1[1] * e2[2] - e1[2] * e2[1];
        const float cr1 = e1[2] * e2[0] - e1[0] * e2[2];
        const float cr2 = e1[0] * e2[1] - e1[1] * e2[0];
        an[0] += 0.5f * cr0;
        an[1] += 0.5f * cr1;
        an[2] += 0.5f * cr2;
        const float a = 0.5f * (cr0 * tn[0] + cr1 * tn[1] + cr2 * tn[2]);
        As += a;
        const float s[3] = {e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]};
        const float a3 = a * (1.f / 3.f), a12 = a * (1.f / 12.f);
        for (int d = 0; d < 3; d++) m1[d] += a3 * s[d];
        m2[0] += a12 * (s[0] * s[0] + e1[0] * e1[0] + e2[0] * e2[0]);
        m2[1] += a12 * (s[1] * s[1] + e1[1] * e1[1] + e2[1] * e2[1]);
        m2[2] += a12 * (s[2] * s[2] + e1[2] * e1[2] + e2[2] * e2[2]);
        m2[3] += a12 * (s[0] * s[1] + e1[0] * e1[1] + e2[0] * e2[1]);
        m2[4] += a12 * (s[0] * s[2] + e1[0] * e1[2] + e2[0] * e2[2]);
        m2[5] += a12 * (s[1] * s[2] + e1[1] * e1[2] + e2[1] * e2[2]);
        for (int d = 0; d < 3; d++) e1[d] = e2[d];
    }
    if (As > 0.f) {
        const float ia = 1.f / As;
        const float c[3] = {m1[0] * ia, m1[1] * ia, m1[2] * ia};
        f.k[0] = m2[0] * ia - c[0] * c[0];
        f.k[1] = m2[1] * ia - c[1] * c[1];
        f.k[2] = m2[2] * ia - c[2] * c[2];
        f.k[3] = m2[3] * ia - c[0] * c[1];
        f.k[4] = m2[4] * ia - c[0] * c[2];
        f.k[5] = m2[5] * ia - c[1] * c[2];
        for (int d = 0; d < 3; d++) f.c[d] = q0[d] + c[d];
    } else {
        for (int d = 0; d < 6; d++) f.k[d] = 0.f;
        for (int d = 0; d < 3; d++) f.c[d] = q0[d];
    }
    for (int d = 0; d < 3; d++) f.an[d] = an[d];
}

// One queued edge-plane crossing: the edge prev -> cur of a lane's polygon and
// the plane value; the result q is written back for the owning lane.
struct ClipJob {
    double a[3], b[3], q[3], pv;
};

constexpr int kClipV = 12;     // polygon capacity of the warp-cooperative path
constexpr int kClipJobs = 64;  // <= 2 crossings per lane and stage
constexpr int kClipThreads = 256;

// Warp-cooperative canonical clip: lane l holds candidate cb + l.  Each stage
// computes the inside flags per lane, queues every crossing of the warp in
// shared memory and evaluates them on full lanes with the canonical operations
// (t = (pv - a)/(b - a), q = a + t (b - a), clipped coordinate set to pv), then
// each lane assembles its output in Sutherland-Hodgman order.  A stage with more
// than two crossings in some lane (degenerate) is done lane by lane with
// clip_half, and a polygon that outgrows kClipV is redone with the wide serial
// clip: both give the same result as this path would.
// The surviving polygon is left in A or B (or, after the wide fallback, in
// wide_res); *out points to it.
template <int MAXV>
__device__ int clip_warp(const double (*v)[3], const Planes& P, const ft_grid& g, const int idx[3], bool active,
                         ClipJob* jobs, double (*A)[3], double (*B)[3], double (*wide_res)[3],
                         const double (**out)[3]) {
    const int lane = threadIdx.x & 31;
    double(*src)[3] = A;
    double(*dst)[3] = B;
    int n = 3;
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) A[c][d] = v[c][d];
    bool alive = active, wide = false;
    for (int st = 0; st < 6; st++) {
        const int ax = st >> 1;
        const bool ge = (st & 1) == 0;
        const double pv = P.at(ax, idx[ax] + (st & 1));
        unsigned flags = 0, cross = 0;
        int ncross = 0;
        if (alive) {
            const long long kp = okey(pv);
            for (int i = 0; i < n; i++) {
                const long long kc = okey(src[i][ax]);
                if (ge ? (kc >= kp) : (kc <= kp)) flags |= 1u << i;
            }
            // edge (i-1 -> i) crosses iff the flags of its ends differ
            const unsigned prevf = (flags << 1 | flags >> (n - 1)) & ((1u << n) - 1u);
            cross = flags ^ prevf;
            ncross = __popc(cross);
        }
        if (__any_sync(0xffffffffu, ncross > 2)) {
            // degenerate stage somewhere in the warp: lane by lane, canonically
            if (alive) {
                int m;
                if (!clip_half<MAXV>(src, n, dst, m, ax, pv, ge)) {
                    wide = true;
                    alive = false;
                } else if (m < 3) {
                    alive = false;
                } else {
                    n = m;
                    double(*tmp)[3] = src;
                    src = dst;
                    dst = tmp;
                }
            }
            continue;
        }
        int incl = ncross;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int base = incl - ncross;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (ncross) {
            int k = 0;
            for (int i = 0; i < n; i++) {
                if (!((cross >> i) & 1u)) continue;
                const int pi = (i == 0) ? n - 1 : i - 1;
                ClipJob& J = jobs[base + k++];
                for (int d = 0; d < 3; d++) {
                    J.a[d] = src[pi][d];
                    J.b[d] = src[i][d];
                }
                J.pv = pv;
            }
        }
        __syncwarp();
        for (int j = lane; j < total; j += 32) {
            ClipJob& J = jobs[j];
            const double t = __ddiv_rn(__dsub_rn(J.pv, J.a[ax]), __dsub_rn(J.b[ax], J.a[ax]));
#pragma unroll
            for (int c = 0; c < 3; c++)
                J.q[c] = (c == ax) ? J.pv : __dadd_rn(J.a[c], __dmul_rn(t, __dsub_rn(J.b[c], J.a[c])));
        }
        __syncwarp();
        // (a lane whose vertices are all inside keeps its polygon as it is)
        if (alive && flags != (1u << n) - 1u) {
            int m = 0, k = 0;
            for (int i = 0; i < n && !wide; i++) {
                if ((cross >> i) & 1u) {
                    if (m >= MAXV) {
                        wide = true;
                        break;
                    }
                    const ClipJob& J = jobs[base + k++];
                    dst[m][0] = J.q[0];
                    dst[m][1] = J.q[1];
                    dst[m][2] = J.q[2];
                    m++;
                }
                if ((flags >> i) & 1u) {
                    if (m >= MAXV) {
                        wide = true;
                        break;
                    }
                    dst[m][0] = src[i][0];
                    dst[m][1] = src[i][1];
                    dst[m][2] = src[i][2];
                    m++;
                }
            }
            if (wide || m < 3) {
                alive = false;
            } else {
                n = m;
                double(*tmp)[3] = src;
                src = dst;
                dst = tmp;
            }
        }
        __syncwarp();
    }
    if (wide) {
        *out = wide_res;
        return canon_stages_wide(v, g, idx, wide_res);
    }
    *out = src;
    if (!alive) return 0;
    for (int ax = 0; ax < 3; ax++) {
        const long long ku = okey(P.at(ax, idx[ax] + 1));
        bool all = true;
        for (int m = 0; m < n && all; m++) all = (okey(src[m][ax]) == ku);
        if (all) return 0;
    }
    return n;
}

// The canonical clip of candidate slot c on every lane of a warp (warp-
// collective: lanes without a candidate pass active = false), its fragment
// record and its key and rank.
template <int MAXV, class F>
__device__ __forceinline__ void clip_slot_warp(const F& fr, long long c, bool active, ClipJob* jobs,
                                               const int* __restrict__ cand_tri, const int* __restrict__ tri_off,
                                               const int* __restrict__ tri_box, const double* __restrict__ tri_nrm,
                                               unsigned* __restrict__ keys, unsigned* __restrict__ ranks,
                                               int* __restrict__ cell_cnt, ft_frag* __restrict__ rec,
                                               ft_frag32* __restrict__ rec32, float4* __restrict__ cen32, int fp32,
                                               double (*bufA)[3], double (*bufB)[3]) {
    int idx[3] = {0, 0, 0};
    int b = 0;
    double v[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (active) {
        const int t = cand_tri[c];
        const int l = (int)(c - tri_off[t]);
        const int4* bx = reinterpret_cast<const int4*>(tri_box + 8 * (long long)t);
        const int4 b0 = bx[0], b1 = bx[1];
        const int e1 = b1.x, e2 = b1.y;
        b = b1.z;
        idx[0] = b0.x + l / (e1 * e2);
        idx[1] = b0.y + (l / e2) % e1;
        idx[2] = b0.z + l % e2;
        const ft_fdesc& D = fr.desc(b);
        const long long tl = t - fr.tri_base(b);
        for (int a = 0; a < 3; a++) {
            const long long vi = D.tris[3 * tl + a];
            for (int d = 0; d < 3; d++) v[a][d] = D.verts[3 * vi + d];
        }
    }
    const ft_fdesc& D = fr.desc(b);
    const ft_grid g = D.g;
    const Planes P(D);
    double wide[32][3];
    const double(*poly)[3] = bufA;
    const int n = clip_warp<MAXV>(v, P, g, idx, active, jobs, bufA, bufB, wide, &poly);
    if (!active) return;
    unsigned key = FT_SENTINEL;
    if (n >= 3) {
        const double inv_h = D.inv_h;
        const double2* tnp = reinterpret_cast<const double2*>(tri_nrm + 4 * (long long)cand_tri[c]);
        const double2 tn01 = tnp[0], tn2 = tnp[1];
        // The moments' own area vector certifies the canonical "area vector
        // is not zero" condition whenever it exceeds its rounding bound by
        // far (float32: 1e-4 h^2, float64: 1e-9 h^2); only smaller fragments
        // evaluate the canonical sum.
        bool accept;
        if (fp32) {
            ft_frag32 f;
            const float tn[3] = {d2f_rn(tn01.x), d2f_rn(tn01.y), d2f_rn(tn2.x)};
            const float ih = d2f_rn(inv_h);
            float q0[3];
            for (int d = 0; d < 3; d++) q0[d] = d2f_rn(poly[0][d] - P.at(d, idx[d])) * ih - 0.5f;
            frag_moments32(poly, n, q0, tn, ih, f);
            const float a = fmaxf(fabsf(f.an[0]), fmaxf(fabsf(f.an[1]), fabsf(f.an[2])));
            accept = (a > 1e-4f) || canon_area_nonzero(poly, n);
            if (accept) rec32[c] = f;
        } else {
            ft_frag f;
            const double tn[3] = {tn01.x, tn01.y, tn2.x};
            double q0[3];
            for (int d = 0; d < 3; d++) q0[d] = (poly[0][d] - P.at(d, idx[d])) * inv_h - 0.5;
            frag_moments(poly, n, q0, tn, inv_h, f);
            const double a = fmax(fabs(f.an[0]), fmax(fabs(f.an[1]), fabs(f.an[2])));
            accept = (a > 1e-9) || canon_area_nonzero(poly, n);
            if (accept) {
                rec[c] = f;
                if (cen32) cen32[c] = make_float4(d2f_rn(f.c[0]), d2f_rn(f.c[1]), d2f_rn(f.c[2]), 0.f);
            }
        }
        if (accept) key = (unsigned)(fr.key_base(b) + ((long long)idx[0] * g.n[1] + idx[1]) * g.n[2] + idx[2]);
    }
    keys[c] = key;
    // the pair's rank among its cell's pairs, in arrival order (k_cell_order
    // puts each cell's pairs back into slot order)
    if (key != FT_SENTINEL) ranks[c] = (unsigned)atomicAdd(&cell_cnt[key], 1);
}

// 80 registers (a few bytes of spills) let three blocks of 256 threads share
// an SM instead of two: 24 resident warps hide more of the float64 and local
// memory latency of the clip.  With a list, only the listed slots (their
// number in clip_f64: the pairs the FP32 clip's warps could not keep).
template <class F>
__global__ void __maxnreg__(80) k_clip(F fr, const int* __restrict__ cand_tri,
                                                   const int* __restrict__ tri_off, const int* __restrict__ tri_box,
                                                   const double* __restrict__ tri_nrm,
                                                   unsigned* __restrict__ keys, unsigned* __restrict__ ranks,
                                                   int* __restrict__ cell_cnt, ft_frag* __restrict__ rec,
                                                   ft_frag32* __restrict__ rec32, float4* __restrict__ cen32, int fp32,
                                                   const ft_counters* ctr, const unsigned* __restrict__ list) {
    __shared__ ClipJob s_jobs[kClipThreads / 32][kClipJobs];
    ClipJob* jobs = s_jobs[threadIdx.x >> 5];
    const long long C = list ? ctr->clip_f64 : ctr->C;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (kClipThreads / 32);
    for (long long cb = ((long long)blockIdx.x * (kClipThreads / 32) + (threadIdx.x >> 5)) * 32; cb < C; cb += nwarps * 32) {
        const bool active = cb + lane < C;
        const long long c = list ? (active ? (long long)list[cb + lane] : 0) : cb + lane;
        double bufA[kClipV][3], bufB[kClipV][3];
        clip_slot_warp<kClipV>(fr, c, active, jobs, cand_tri, tri_off, tri_box, tri_nrm, keys, ranks, cell_cnt, rec, rec32,
                       cen32, fp32, bufA, bufB);
    }
}

// The pairs the FP32 clip left to the binary64 clip (ctr->clip_f64 slots in
// list): few, so a segment of kSeg lanes per pair (four pairs per warp), the
// polygon one vertex per lane.  Each stage is the Sutherland-Hodgman step
// written lane-parallel: lane i of a segment owns the edge from vertex i-1
// (cyclically) to vertex i and computes its crossing with the canonical
// operations (t = (pv - a)/(b - a), q = a + t (b - a), the clipped coordinate
// set to pv); an exclusive scan of the per-lane output counts (crossing first,
// then the vertex if inside) places the outputs in exactly the serial order.  A
// polygon that would outgrow the segment (a triangle clipped by all six planes
// has up to nine vertices: rare) is redone by the wide serial clip on the
// segment's first lane.  The float32 record's moments are spread over the
// segment's lanes; the canonical area test runs on its first lane.  Several
// pairs per warp divide the float64 instructions per pair (a float64 warp
// instruction costs the same however few lanes it has): one pair per warp took
// 18.5 us for the ~1,300 pairs of a 128^3 front, two 17.4 us, four 17.0 us.
constexpr int kListWarps = 4;
constexpr int kSeg = 8;                  // lanes per listed pair (polygons up to 8 vertices)
constexpr int kSegPerWarp = 32 / kSeg;
// frag_moments32 spread over a segment of kSeg lanes (collective over the
// warp, each segment with its own polygon): lane m-1 of the segment takes fan
// triangle (p0, p_m, p_m+1), m = 1 .. n-2 (n <= kSeg + 1; n = 0: no polygon),
// and the thirteen sums are reduced over the segment; every lane of it ends
// with the record.  The terms are those of frag_moments32; only the order of
// their float32 sums differs.
__device__ void frag_moments32_seg(const double (*p)[3], int n, const float q0[3], const float tn[3], float inv_h,
                                   int lane, ft_frag32& f) {
    float v[13];
#pragma unroll
    for (int r = 0; r < 13; r++) v[r] = 0.f;
    const int m = lane + 1;
    if (m + 1 < n) {
        float e1[3], e2[3];
        for (int d = 0; d < 3; d++) {
            e1[d] = d2f_rn(p[m][d] - p[0][d]) * inv_h;
            e2[d] = d2f_rn(p[m + 1][d] - p[0][d]) * inv_h;
        }
        const float cr0 = e1[1] * e2[2] - e1[2] * e2[1];
        const float cr1 = e1[2] * e2[0] - e1[0] * e2[2];
        const float cr2 = e1[0] * e2[1] - e1[1] * e2[0];
        v[0] = 0.5f * cr0;
        v[1] = 0.5f * cr1;
        v[2] = 0.5f * cr2;
        const float a = 0.5f * (cr0 * tn[0] + cr1 * tn[1] + cr2 * tn[2]);
        v[3] = a;
        const float s[3] = {e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]};
        const float a3 = a * (1.f / 3.f), a12 = a * (1.f / 12.f);
        for (int d = 0; d < 3; d++) v[4 + d] = a3 * s[d];
        v[7] = a12 * (s[0] * s[0] + e1[0] * e1[0] + e2[0] * e2[0]);
        v[8] = a12 * (s[1] * s[1] + e1[1] * e1[1] + e2[1] * e2[1]);
        v[9] = a12 * (s[2] * s[2] + e1[2] * e1[2] + e2[2] * e2[2]);
        v[10] = a12 * (s[0] * s[1] + e1[0] * e1[1] + e2[0] * e2[1]);
        v[11] = a12 * (s[0] * s[2] + e1[0] * e1[2] + e2[0] * e2[2]);
        v[12] = a12 * (s[1] * s[2] + e1[1] * e1[2] + e2[1] * e2[2]);
    }
#pragma unroll
    for (int o = kSeg / 2; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < 13; r++) v[r] += __shfl_xor_sync(0xffffffffu, v[r], o);
    const float As = v[3];
    if (As > 0.f) {
        const float ia = 1.f / As;
        const float c[3] = {v[4] * ia, v[5] * ia, v[6] * ia};
        f.k[0] = v[7] * ia - c[0] * c[0];
        f.k[1] = v[8] * ia - c[1] * c[1];
        f.k[2] = v[9] * ia - c[2] * c[2];
        f.k[3] = v[10] * ia - c[0] * c[1];
        f.k[4] = v[11] * ia - c[0] * c[2];
        f.k[5] = v[12] * ia - c[1] * c[2];
        for (int d = 0; d < 3; d++) f.c[d] = q0[d] + c[d];
    } else {
        for (int d = 0; d < 6; d++) f.k[d] = 0.f;
        for (int d = 0; d < 3; d++) f.c[d] = q0[d];
    }
    for (int d = 0; d < 3; d++) f.an[d] = v[d];
}

template <class F>
__global__ void __launch_bounds__(kListWarps * 32) k_clip_list(F fr, const int* __restrict__ cand_tri,
                                                              const int* __restrict__ tri_off,
                                                              const int* __restrict__ tri_box,
                                                              const float* __restrict__ tri32,
                                                              unsigned* __restrict__ keys,
                                                              unsigned* __restrict__ ranks,
                                                              int* __restrict__ cell_cnt,
                                                              ft_frag32* __restrict__ rec32, const ft_counters* ctr,
                                                              const unsigned* __restrict__ list) {
    __shared__ double s_poly[kListWarps][2][32][3];
    __shared__ double s_wide[kListWarps][kSegPerWarp][32][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int seg = lane / kSeg, sl = lane % kSeg, base = seg * kSeg;
    const unsigned segmask = (kSeg == 32 ? 0xffffffffu : ((1u << kSeg) - 1u)) << base;
    const long long L = ctr->clip_f64;
    const long long step = (long long)gridDim.x * kListWarps * kSegPerWarp;
    for (long long j0 = ((long long)blockIdx.x * kListWarps + w) * kSegPerWarp; j0 < L; j0 += step) {
        const long long j = j0 + seg;
        const bool has = j < L;  // (the warp's second segment may have no pair)
        const long long c = has ? (long long)list[j] : 0;
        int t = 0, idx[3] = {0, 0, 0}, b = 0;
        if (has) {
            t = cand_tri[c];
            const int l = (int)(c - tri_off[t]);
            const int4* bx = reinterpret_cast<const int4*>(tri_box + 8 * (long long)t);
            const int4 b0 = bx[0], b1 = bx[1];
            const int e1 = b1.x, e2 = b1.y;
            b = b1.z;
            idx[0] = b0.x + l / (e1 * e2);
            idx[1] = b0.y + (l / e2) % e1;
            idx[2] = b0.z + l % e2;
        }
        const ft_fdesc& D = fr.desc(b);
        const ft_grid g = D.g;
        const Planes P(D);
        const long long tl = t - fr.tri_base(b);
        // lane i < n of the segment holds polygon vertex i; the triangle first
        double x[3] = {0.0, 0.0, 0.0};
        if (has && sl < 3) {
            const long long vi = D.tris[3 * tl + sl];
            for (int d = 0; d < 3; d++) x[d] = D.verts[3 * vi + d];
        }
        int n = 3;
        bool alive = has, wide = false;
        for (int st = 0; st < 6; st++) {
            // (every lane takes part in the shuffles; a finished segment's lanes idle)
            const bool go = alive && !wide;
            const int ax = st >> 1;
            const bool ge = (st & 1) == 0;
            const double pv = P.at(ax, idx[ax] + (st & 1));
            const long long kp = okey(pv);
            const bool act = go && sl < n;
            const long long kc = okey(x[ax]);
            const bool cin = act && (ge ? (kc >= kp) : (kc <= kp));
            const int pl = (sl == 0) ? n - 1 : sl - 1;  // the edge's first vertex (in the segment)
            double pr[3];
#pragma unroll
            for (int d = 0; d < 3; d++) pr[d] = __shfl_sync(0xffffffffu, x[d], pl, kSeg);
            const bool pin = __shfl_sync(0xffffffffu, cin ? 1 : 0, pl, kSeg) != 0;
            const bool cross = act && (cin != pin);
            double q[3] = {0.0, 0.0, 0.0};
            if (cross) {
                const double tt = __ddiv_rn(__dsub_rn(pv, pr[ax]), __dsub_rn(x[ax], pr[ax]));
#pragma unroll
                for (int d = 0; d < 3; d++)
                    q[d] = (d == ax) ? pv : __dadd_rn(pr[d], __dmul_rn(tt, __dsub_rn(x[d], pr[d])));
            }
            const int cnt = (cross ? 1 : 0) + (cin ? 1 : 0);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < kSeg; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o, kSeg);
                if (sl >= o) incl += y;
            }
            const int m = __shfl_sync(0xffffffffu, incl, kSeg - 1, kSeg);
            if (go && m > kSeg) wide = true;
            if (go && m < 3) alive = false;
            double(*dst)[3] = s_poly[w][st & 1] + base;
            if (go && alive && !wide) {
                const int pos = incl - cnt;
                if (cross)
                    for (int d = 0; d < 3; d++) dst[pos][d] = q[d];
                if (cin)
                    for (int d = 0; d < 3; d++) dst[pos + (cross ? 1 : 0)][d] = x[d];
            }
            __syncwarp();
            if (go && alive && !wide) {
                n = m;
                if (sl < n)
                    for (int d = 0; d < 3; d++) x[d] = dst[sl][d];
            }
            __syncwarp();
        }
        const double(*poly)[3] = s_poly[w][1] + base;  // the last stage's output
        if (wide) {
            // the wide serial clip of the triangle, on the segment's first lane
            int nw = 0;
            if (sl == 0) {
                double v[3][3];
                for (int a = 0; a < 3; a++) {
                    const long long vi = D.tris[3 * tl + a];
                    for (int d = 0; d < 3; d++) v[a][d] = D.verts[3 * vi + d];
                }
                nw = canon_stages_wide(v, g, idx, s_wide[w][seg]);
            }
            n = __shfl_sync(segmask, nw, base);
            alive = n >= 3;
            poly = s_wide[w][seg];
        }
        // a polygon lying in an upper face of the cell belongs to the next cell
        // (the wide clip has applied this test itself)
        for (int ax = 0; ax < 3; ax++) {
            const long long ku = okey(P.at(ax, idx[ax] + 1));
            const unsigned on = __ballot_sync(0xffffffffu, sl < n && okey(x[ax]) == ku) & segmask;
            const unsigned all = (n >= 32 ? 0xffffffffu : ((1u << n) - 1u)) << base;
            if (alive && !wide && on == (all & segmask)) alive = false;
        }
        __syncwarp();
        ft_frag32 f;
        {
            const float* tr = tri32 + 32 * (long long)t;
            const float tn[3] = {tr[18], tr[19], tr[20]};
            const float ih = d2f_rn(D.inv_h);
            float q0[3];
            for (int d = 0; d < 3; d++) q0[d] = alive ? d2f_rn(poly[0][d] - P.at(d, idx[d])) * ih - 0.5f : 0.f;
            frag_moments32_seg(poly, alive ? n : 0, q0, tn, ih, sl, f);
        }
        if (has && sl == 0) {
            unsigned key = FT_SENTINEL;
            if (alive) {
                // the moments' own area vector certifies the canonical "area vector
                // is not zero" condition whenever it exceeds its rounding bound by far
                const float a = fmaxf(fabsf(f.an[0]), fmaxf(fabsf(f.an[1]), fabsf(f.an[2])));
                if ((a > 1e-4f) || canon_area_nonzero(poly, n)) {
                    rec32[c] = f;
                    key = (unsigned)(fr.key_base(b) + ((long long)idx[0] * g.n[1] + idx[1]) * g.n[2] + idx[2]);
                }
            }
            keys[c] = key;
            if (key != FT_SENTINEL) ranks[c] = (unsigned)atomicAdd(&cell_cnt[key], 1);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// FP32 clip of the FP32-compensated form.
//
// The decision whether a (triangle, cell) pair is kept stays the binary64
// canonical predicate above; this kernel reaches the same decision without
// binary64 crossing points wherever a float32 computation certifies it:
//  * the triangle's own vertices are classified against the six planes exactly
//    (order-preserving integer keys of the binary64 values, as the predicate
//    does);
//  * the clip runs in float32 in cell units (x - X_i)/h, the polygons in
//    per-lane shared-memory buffers, each vertex carrying a bound on its
//    distance to the vertex of the exact-arithmetic clip (rounding of the
//    conversions and of every crossing, amplified by the conditioning of the
//    crossing, as derived below);
//  * a crossing vertex whose distance to a later plane does not exceed its
//    bound, a crossing edge too close to parallel to its plane, a stage with
//    more than two crossings or a polygon that outgrows its buffer makes the
//    pair undecided.
// When every classification is certain, the binary64 clip classifies every
// vertex the same way (its own errors are far below the float bounds, so both
// polygons have the same vertex sequence): a polygon that dies is rejected,
// and one whose float area exceeds its bound by far (and that does not lie
// within its bounds of an upper face) is kept.  Everything else -- undecided
// pairs, small areas, fragments near an upper face -- runs the binary64
// canonical clip (the plane-edge sign tests and crossings of near-degenerate
// vertices stay float64), so the kept set, the cell list and the parity fill are
// those of the float64 path bit for bit.  Kept fragments' float32 records come
// from the float32 polygon (or, for pairs decided in float64, from the binary64
// polygon).
// ---------------------------------------------------------------------------

constexpr int kClip32Threads = 128;
constexpr int kClip32Warps = kClip32Threads / 32;
constexpr int kPV = 9;           // float polygon capacity (the exact clip of a triangle has at most 9)
constexpr float kEps = 3e-7f;    // relative bound of a few float32 roundings (2^-24 = 6e-8 each)
// A kept fragment whose vertex bound exceeds this (crossings of edges nearly
// parallel to their plane) takes its record from the binary64 polygon, so that
// float32 records stay within about 1e-7 cells of the exact fragment's.
constexpr float kEmaxRecord = 3e-4f;

// Float32 fragment moments of the polygon buf[0..n) (cell units, lower corner
// at the origin; the x, y, z of each float4), as frag_moments32 computes them
// from a binary64 polygon.  tn: the triangle's normal direction.
__device__ void frag_moments_f(const float4 (*buf)[32], int lane, int n, const float tn[3], ft_frag32& f,
                               float& absum) {
    float an[3] = {0.f, 0.f, 0.f}, m1[3] = {0, 0, 0}, m2[6] = {0, 0, 0, 0, 0, 0}, As = 0.f;
    absum = 0.f;
    const float4 p0 = buf[0][lane];
    const float4 p1 = buf[1][lane];
    float e1[3] = {p1.x - p0.x, p1.y - p0.y, p1.z - p0.z}, e2[3];
    for (int m = 1; m + 1 < n; m++) {
        const float4 pm = buf[m + 1][lane];
        e2[0] = pm.x - p0.x;
        e2[1] = pm.y - p0.y;
        e2[2] = pm.z - p0.z;
        const float cr0 = e1[1] * e2[2] - e1[2] * e2[1];
        const float cr1 = e1[2] * e2[0] - e1[0] * e2[2];
        const float cr2 = e1[0] * e2[1] - e1[1] * e2[0];
        absum += fmaxf(fabsf(e1[0]), fmaxf(fabsf(e1[1]), fabsf(e1[2]))) *
                 fmaxf(fabsf(e2[0]), fmaxf(fabsf(e2[1]), fabsf(e2[2])));
        an[0] += 0.5f * cr0;
        an[1] += 0.5f * cr1;
        an[2] += 0.5f * cr2;
        const float a = 0.5f * (cr0 * tn[0] + cr1 * tn[1] + cr2 * tn[2]);
        As += a;
        const float s[3] = {e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2]};
        const float a3 = a * (1.f / 3.f), a12 = a * (1.f / 12.f);
        for (int d = 0; d < 3; d++) m1[d] += a3 * s[d];
        m2[0] += a12 * (s[0] * s[0] + e1[0] * e1[0] + e2[0] * e2[0]);
        m2[1] += a12 * (s[1] * s[1] + e1[1] * e1[1] + e2[1] * e2[1]);
        m2[2] += a12 * (s[2] * s[2] + e1[2] * e1[2] + e2[2] * e2[2]);
        m2[3] += a12 * (s[0] * s[1] + e1[0] * e1[1] + e2[0] * e2[1]);
        m2[4] += a12 * (s[0] * s[2] + e1[0] * e1[2] + e2[0] * e2[2]);
        m2[5] += a12 * (s[1] * s[2] + e1[1] * e1[2] + e2[1] * e2[2]);
        for (int d = 0; d < 3; d++) e1[d] = e2[d];
    }
    const float q0[3] = {p0.x - 0.5f, p0.y - 0.5f, p0.z - 0.5f};
    if (As > 0.f) {
        const float ia = 1.f / As;
        const float c[3] = {m1[0] * ia, m1[1] * ia, m1[2] * ia};
        f.k[0] = m2[0] * ia - c[0] * c[0];
        f.k[1] = m2[1] * ia - c[1] * c[1];
        f.k[2] = m2[2] * ia - c[2] * c[2];
        f.k[3] = m2[3] * ia - c[0] * c[1];
        f.k[4] = m2[4] * ia - c[0] * c[2];
        f.k[5] = m2[5] * ia - c[1] * c[2];
        for (int d = 0; d < 3; d++) f.c[d] = q0[d] + c[d];
    } else {
        for (int d = 0; d < 6; d++) f.k[d] = 0.f;
        for (int d = 0; d < 3; d++) f.c[d] = q0[d];
    }
    for (int d = 0; d < 3; d++) f.an[d] = an[d];
}

__device__ __forceinline__ float comp(const float4& v, int ax) { return ax == 0 ? v.x : (ax == 1 ? v.y : v.z); }

// Outcome of the float32 clip of one pair.
enum : int { kUndecided = 0, kRejected = 1, kKept = 2 };

// The float32 clip of triangle (tv, in cell units) against the cell [0, top]:
// exact flags of the triangle's vertices (bit st: inside for stage st), the
// polygon left in bufs[*res] (n vertices), its largest vertex bound (emax) and
// its S2 sum (below).  Vertex w: < 0 for a triangle
// vertex (-(1 + flags)), else the distance bound of a crossing vertex.  A
// triangle vertex's coordinates are within kEps (|x|max + W) of the exact ones
// (ew = kEps W, see k_clip32).
__device__ int clip_f32(const float tv[3][3], const unsigned vflags[3], const float top[3], float ew,
                        float4 (*b0)[32], float4 (*b1)[32], int lane, int& n_out, float4 (**res)[32],
                        float& emax, float& S2) {
    float4(*src)[32] = b0;
    float4(*dst)[32] = b1;
    for (int c = 0; c < 3; c++) src[c][lane] = make_float4(tv[c][0], tv[c][1], tv[c][2], -(float)(1 + vflags[c]));
    int n = 3;
    // Stages whose half-space holds all three triangle vertices by more than
    // 1e-5 cells plus 2e-6 of the coordinate (the float coordinates are within
    // kEps |x| + ew of the exact ones) keep every polygon derived from the
    // triangle as it is: its points
    // are convex combinations of the vertices, and the binary64 crossings lie
    // within 1e-12 cells of them, so the canonical stage finds every vertex
    // inside too.  Those stages are skipped without reading the polygon.
    unsigned skip = 0u;
#pragma unroll
    for (int st = 0; st < 6; st++) {
        const int ax = st >> 1;
        const bool ge = (st & 1) == 0;
        bool all = true;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float x = tv[c][ax], mg = 1e-5f + 2e-6f * fabsf(x);
            all = all && (ge ? x > mg : top[ax] - x > mg);
        }
        if (all) skip |= 1u << st;
    }
    // Each lane walks only its own remaining stages, in stage order (a skipped
    // stage leaves the polygon as it is): the warp's lanes run their first
    // remaining stage together, then their second, and so on, instead of each
    // stage idling the lanes that skip it.
    for (unsigned act = ~skip & 63u; act; act &= act - 1u) {
        const int st = __ffs(act) - 1;
        const int ax = st >> 1;
        const bool ge = (st & 1) == 0;
        const float pl = ge ? 0.f : top[ax];
        const float epl = kEps * fabsf(pl);
        // inside flags of the polygon's vertices
        unsigned in = 0;
        for (int i = 0; i < n; i++) {
            const float4 v = src[i][lane];
            bool ins;
            if (v.w < 0.f) {
                ins = (((unsigned)(-v.w) - 1u) >> st) & 1u;
            } else {
                const float x = comp(v, ax);
                const float d = x - pl;
                const float m = 1.01f * (v.w + epl + kEps * (fabsf(x) + fabsf(pl))) + 1e-30f;
                if (!(fabsf(d) > m)) return kUndecided;
                ins = ge ? (d > 0.f) : (d < 0.f);
            }
            if (ins) in |= 1u << i;
        }
        if (in == 0u) return kRejected;  // the polygon dies at this stage (every vertex outside)
        if (in == (1u << n) - 1u) continue;  // every vertex inside: the stage keeps the polygon as it is
        const unsigned prevf = (in << 1 | in >> (n - 1)) & ((1u << n) - 1u);
        const unsigned cross = in ^ prevf;
        if (__popc(cross) > 2) return kUndecided;
        // Exactly two crossings now (in is neither empty nor full), on the edges
        // i1-1 -> i1 and i2-1 -> i2; both are computed in straight-line code on
        // every lane (no per-vertex branch over which lanes cross where).  Each
        // crossing interpolates from the edge's end nearer to the plane (the
        // smaller step t (b - a) keeps the rounding of q small); a is that end.
        const int i1 = __ffs(cross) - 1, i2 = 31 - __clz(cross);
        const int nin = __popc(in);
        if (nin + 2 > kPV) return kUndecided;
        bool bad = false;
        float4 qv[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int i = k ? i2 : i1;
            float4 a = src[i == 0 ? n - 1 : i - 1][lane];
            float4 b = src[i][lane];
            if (fabsf(pl - comp(a, ax)) > fabsf(pl - comp(b, ax))) {
                const float4 tmp = a;
                a = b;
                b = tmp;
            }
            const float ea = a.w < 0.f ? kEps * fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))) + ew : a.w;
            const float eb = b.w < 0.f ? kEps * fmaxf(fabsf(b.x), fmaxf(fabsf(b.y), fabsf(b.z))) + ew : b.w;
            const float aa = comp(a, ax), ba = comp(b, ax);
            const float D = ba - aa;
            const float den = fabsf(D) - 1.01f * (ea + eb + kEps * (fabsf(aa) + fabsf(ba)));
            bad = bad || !(den > 0.f);
            const float t = __fdiv_rn(pl - aa, D);
            const float tt = fmaxf(fabsf(t), 1.f);
            // |t - t*| <= (errors of the numerator + |t*| errors of D) / |D*| + the division's rounding
            const float dt = ((ea + epl + kEps * (fabsf(aa) + fabsf(pl))) +
                              tt * (ea + eb + kEps * (fabsf(aa) + fabsf(ba)))) / den + 4.f * kEps * tt;
            const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
            const float L = fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz)));
            const float amax = fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z)));
            const float bmax = fmaxf(fabsf(b.x), fmaxf(fabsf(b.y), fabsf(b.z)));
            float4 q;
            q.x = (ax == 0) ? pl : __fadd_rn(a.x, __fmul_rn(t, dx));
            q.y = (ax == 1) ? pl : __fadd_rn(a.y, __fmul_rn(t, dy));
            q.z = (ax == 2) ? pl : __fadd_rn(a.z, __fmul_rn(t, dz));
            // |q - q*| <= max(ea, eb) + |b - a| |t - t*| + the roundings of q
            q.w = 1.01f * (fmaxf(ea, eb) + L * dt + 2.f * kEps * tt * (amax + bmax + 1.f));
            qv[k] = q;
        }
        if (bad) return kUndecided;
        // The output in Sutherland-Hodgman order (for i = 0 .. n-1: the crossing
        // of edge i-1 -> i, then vertex i if inside), each entry stored at the
        // position that order gives it.
        for (int i = 0; i < n; i++)
            if ((in >> i) & 1u) dst[__popc(in & ((1u << i) - 1u)) + (i1 <= i) + (i2 <= i)][lane] = src[i][lane];
        dst[__popc(in & ((1u << i1) - 1u))][lane] = qv[0];
        dst[__popc(in & ((1u << i2) - 1u)) + 1][lane] = qv[1];
        n = nin + 2;
        float4(*tmp)[32] = src;
        src = dst;
        dst = tmp;
    }
    // One pass over the surviving polygon: the largest vertex bound; S2, the
    // sum over vertices i of |p_i+1 - p_i-1| (max norm), which bounds the
    // area's error for the caller; and per axis whether every vertex lies within
    // its bounds of the upper face (such a fragment may lie in it exactly in
    // binary64).
    float e = 0.f, s2 = 0.f;
    bool on[3] = {true, true, true};
    float4 vp = src[n - 1][lane], v = src[0][lane];
    for (int i = 0; i < n; i++) {
        const float4 vn = src[i + 1 < n ? i + 1 : 0][lane];
        s2 += fmaxf(fabsf(vn.x - vp.x), fmaxf(fabsf(vn.y - vp.y), fabsf(vn.z - vp.z)));
        const bool tri = v.w < 0.f;
        e = fmaxf(e, tri ? kEps * fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))) + ew : v.w);
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            const float x = comp(v, ax);
            const float ev = tri ? kEps * fabsf(x) + ew : v.w;
            on[ax] = on[ax] && fabsf(x - top[ax]) <= 2.02f * (ev + kEps * (fabsf(x) + 2.f * fabsf(top[ax]))) + 1e-30f;
        }
        vp = v;
        v = vn;
    }
    if (on[0] || on[1] || on[2]) return kUndecided;
    n_out = n;
    *res = src;
    emax = e;
    S2 = s2;
    return kKept;
}

template <class F>
__global__ void __launch_bounds__(kClip32Threads, 6) k_clip32(F fr, const int* __restrict__ cand_tri,
                                                           const int* __restrict__ tri_off,
                                                           const int* __restrict__ tri_box,
                                                           const float* __restrict__ tri32,
                                                           unsigned* __restrict__ keys, unsigned* __restrict__ ranks,
                                                           int* __restrict__ cell_cnt, ft_frag32* __restrict__ rec32,
                                                           ft_counters* ctr, unsigned* __restrict__ undecided) {
    __shared__ float4 s_poly[kClip32Warps][2][kPV][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long C = ctr->C;
    const long long nthreads = (long long)gridDim.x * kClip32Threads;
    for (long long c = (long long)blockIdx.x * kClip32Threads + threadIdx.x; c < C; c += nthreads) {
        const int t = cand_tri[c];
        const int l = (int)(c - tri_off[t]);
        const int4* bx = reinterpret_cast<const int4*>(tri_box + 8 * (long long)t);
        const int4 bb0 = bx[0], bb1 = bx[1];
        const int e1 = bb1.x, e2 = bb1.y;
        const int b = bb1.z;
        const int o[3] = {l / (e1 * e2), (l / e2) % e1, l % e2};  // the cell within the box
        const ft_fdesc& D = fr.desc(b);
        const ft_grid g = D.g;
        const float4* tr = reinterpret_cast<const float4*>(tri32 + 32 * (long long)t);
        const int4* ti = reinterpret_cast<const int4*>(tri32 + 32 * (long long)t);
        const float4 r0 = tr[0], r1 = tr[1], r2 = tr[2], r3 = tr[3], r4 = tr[4], r5 = tr[5];
        const int4 A1 = ti[6], A2 = ti[7];
        const float hv[9] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x};
        const float lv[9] = {r2.y, r2.z, r2.w, r3.x, r3.y, r3.z, r3.w, r4.x, r4.y};
        const int A[9] = {__float_as_int(r5.y), __float_as_int(r5.z), __float_as_int(r5.w), A1.x, A1.y, A1.z,
                          A1.w, A2.x, A2.y};
        const unsigned eq = (unsigned)A2.z;
        // exact flags of the triangle's vertices (integer comparisons with the
        // record's plane indices) and their cell-unit coordinates (hi - o) + lo,
        // two roundings of about |x|.  Their error against (x - X_i) / h, X_i the
        // binary64 plane, is at most kEps |x| + ew: the pair carries the
        // box-relative position to about 4e-15 of W (the box's largest extent + 1),
        // and binary64 planes are spaced h apart to within 1e-8 cells (the far
        // plane (X_i+1 - X_i) / h is taken as 1, within its own bound kEps).
        float tv[3][3];
        const float top[3] = {1.f, 1.f, 1.f};
        unsigned vflags[3] = {0u, 0u, 0u};
        unsigned on_top = 7u;  // axes whose upper plane holds all three vertices
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int Aa = A[3 * a + ax];
                const int ea = (int)((eq >> (3 * a + ax)) & 1u);
                if (o[ax] <= Aa) vflags[a] |= 1u << (2 * ax);
                if (o[ax] >= Aa - ea) vflags[a] |= 1u << (2 * ax + 1);
                if (!(ea && Aa == o[ax] + 1)) on_top &= ~(1u << ax);
                tv[a][ax] = __fadd_rn(__fsub_rn(hv[3 * a + ax], (float)o[ax]), lv[3 * a + ax]);
            }
        }
        const float ew = 1e-8f + 4e-15f * (float)(max(max(bb0.w, bb1.x), bb1.y) + 1);
        int n = 0;
        float4(*poly)[32] = nullptr;
        float emax = 0.f, S2 = 0.f;
        int verdict = on_top ? kRejected : clip_f32(tv, vflags, top, ew, s_poly[w][0], s_poly[w][1], lane, n, &poly,
                                                    emax, S2);
        unsigned key = FT_SENTINEL;
        ft_frag32 f;
        const float tn[3] = {r4.z, r4.w, r5.x};
        if (verdict == kKept && emax > kEmaxRecord) verdict = kUndecided;  // ill-conditioned: record in float64
        if (verdict == kKept) {
            float absum;
            frag_moments_f(poly, lane, n, tn, f, absum);
            // Moving the vertices p_i by d_i changes the area vector by
            // (1/2) sum_i d_i x (p_i+1 - p_i-1) + O(d^2): at most emax S2 + n emax^2
            // per component, S2 = sum_i |p_i+1 - p_i-1| (max norm, widened by the
            // vertex errors; summed by clip_f32); the fan sum adds its own
            // rounding (a few ulps of its terms)
            const float a = fmaxf(fabsf(f.an[0]), fmaxf(fabsf(f.an[1]), fabsf(f.an[2])));
            const float bound = 1.01f * (emax * (S2 + 2.f * (float)n * emax) + (float)n * emax * emax) +
                                32.f * kEps * absum + 1e-30f;
            if (!(a > bound)) verdict = kUndecided;
        }
        if (verdict == kUndecided) {
            // the binary64 canonical clip decides this pair (and gives its record)
            // in a second launch over the listed slots
            const unsigned long long gp = atomicAdd((unsigned long long*)&ctr->clip_f64, 1ull);
            undecided[gp] = (unsigned)c;
            continue;
        }
        if (verdict == kKept) {
            rec32[c] = f;
            const int idx[3] = {bb0.x + o[0], bb0.y + o[1], bb0.z + o[2]};
            key = (unsigned)(fr.key_base(b) + ((long long)idx[0] * g.n[1] + idx[1]) * g.n[2] + idx[2]);
        }
        keys[c] = key;
        if (key != FT_SENTINEL) ranks[c] = (unsigned)atomicAdd(&cell_cnt[key], 1);
    }
}

}  // namespace

namespace ft {

template <class F>
cudaError_t bin_with(ft_workspace* ws, const F& fr, long long T, const ft_params* p, cudaStream_t s) {
    const int margin = 2 + (int)ceil(p->delta_max_h);
    const unsigned nb = (unsigned)((T + kThreads - 1) / kThreads);
    // the FP32 form needs float records; a workspace without them computes float64 records
    const bool fp32 = p->precision == FT_FP32C && ws->rec32 != nullptr;
    const bool clip32 = fp32 && ws->clip32_ok && ws->tri32 != nullptr;
    // (always launched: it also clears the index map of the previous binning, and sets T)
    count_launches(1);
    {
        Trace t(s, "k_tri_setup");
        k_tri_setup<F><<<nb ? nb : 1, kThreads, 0, s>>>(fr, T, margin, ws->max_cand, ws->tri_cnt, ws->tri_box,
                                                        ws->tri_nrm, clip32 ? ws->tri32 : nullptr, ws->cells,
                                                        ws->idx_map, ws->ctr);
    }
    // candidate ranges in triangle order, so that slot order is triangle order
    cudaError_t e = launch_candidates(ws, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    ws->last_precision = fp32 ? FT_FP32C : FT_FP64;
    if (clip32) {
        // a grid-stride loop: at most the blocks that are resident at once (the
        // polygon buffers limit them), so that no block waits for a second wave
        static int occ = 0;
        if (occ == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_clip32<F>, kClip32Threads, 0) !=
                             cudaSuccess || occ < 1))
            occ = 1;
        const int bps = min(occ, 2 * ws->tune.clip_bps);
        // the pairs it leaves undecided are listed in the spare key buffer (free
        // until the placement) and clipped by the binary64 kernel right after
        unsigned* undecided = ws->keys[1];
        count_launches(1);
        {
            Trace t(s, "k_clip32");
            k_clip32<F><<<ws->sm_count * bps, kClip32Threads, 0, s>>>(fr, ws->cand_tri, ws->tri_off, ws->tri_box,
                                                                      ws->tri32, ws->keys[0], ws->vals[0],
                                                                      ws->cell_cnt, ws->rec32, ws->ctr, undecided);
        }
        Trace t(s, "k_clip_list");
        k_clip_list<F><<<ws->sm_count * 8, kListWarps * 32, 0, s>>>(fr, ws->cand_tri, ws->tri_off, ws->tri_box,
                                                                    ws->tri32, ws->keys[0], ws->vals[0],
                                                                    ws->cell_cnt, ws->rec32, ws->ctr, undecided);
        return cudaGetLastError();
    }
    Trace t(s, "k_clip");
    k_clip<F><<<ws->sm_count * ws->tune.clip_bps, kClipThreads, 0, s>>>(fr, ws->cand_tri, ws->tri_off, ws->tri_box,
                                                                    ws->tri_nrm, ws->keys[0], ws->vals[0], ws->cell_cnt, ws->rec, ws->rec32,
                                                                    ws->cen32, fp32 ? 1 : 0, ws->ctr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_planes_one(ft_workspace* ws, cudaStream_t s) {
    const long long n = ft_plane_count(ws->g);
    count_launches(1);
    k_planes<FrontsOne><<<dim3((unsigned)((n + kThreads - 1) / kThreads), 1), kThreads, 0, s>>>(
        ft_one(ws, nullptr, nullptr, 0, 0));
    return cudaGetLastError();
}

cudaError_t launch_planes_batch(ft_workspace* ws, int max_planes, cudaStream_t s) {
    count_launches(1);
    k_planes<FrontsMany><<<dim3((unsigned)((max_planes + kThreads - 1) / kThreads), (unsigned)ws->nf), kThreads, 0, s>>>(
        ft_many(ws));
    return cudaGetLastError();
}

cudaError_t launch_bin(ft_workspace* ws, const ft_front* f, const ft_params* p, cudaStream_t s) {
    return bin_with(ws, ft_one(ws, f->verts, f->tris, f->nv, f->nt), f->nt, p, s);
}

cudaError_t launch_bin_batch(ft_workspace* ws, const ft_params* p, cudaStream_t s) {
    return bin_with(ws, ft_many(ws), ws->nt_total, p, s);
}

}  // namespace ft
