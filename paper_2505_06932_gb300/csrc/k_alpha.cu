// k_alpha.cu -- front_volume_fraction: alpha_C = (1/V_C) int_C I dx (Sec. 3.2).
//
// Divergence theorem along z: for a vertical line the length inside the
// enclosed region and inside [Z_k, Z_k+1] is sum over front crossings of
// sign(n_z)(clamp(z, Z_k, Z_k+1) - Z_k).  Integrated over the column cross-
// section, with fragments f of cell C and the column above C:
//   alpha_C h^3 = sum_{f in C} int_f (z - Z_k) n_z dA + h sum_{f above C} int_f n_z dA.
// In units of h the first term is AN_z (c_z + 1/2) per fragment (area vector
// AN, centroid c relative to the cell centre) and the second a suffix sum of
// AN_z over the column.  Cells without fragments get the rounded suffix sum,
// which is exactly 0 or 1 for a closed, outward-oriented front (the "column
// parity fill" standing in for the paper's ray casting / flood fill).
#include "ft_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// one warp per interfacial cell: L_C = sum AN_z (c_z + 1/2), P_C = sum AN_z
__global__ void __launch_bounds__(kThreads) k_alpha_cells(const int* __restrict__ cell_off, const unsigned* __restrict__ vals,
                                                          const ft_frag* __restrict__ rec, double* __restrict__ cell_L,
                                                          double* __restrict__ cell_P, const ft_counters* ctr) {
    const long long M = ctr->M;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long m = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); m < M; m += nw) {
        const int q0 = cell_off[m], q1 = cell_off[m + 1];
        double L = 0.0, P = 0.0;
        for (int q = q0 + lane; q < q1; q += 32) {
            const ft_frag* f = rec + (vals ? vals[q] : (unsigned)q);
            const double az = f->an[2];
            L += az * (f->c[2] + 0.5);
            P += az;
        }
        L = ft_warp_sum(L);
        P = ft_warp_sum(P);
        if (lane == 0) {
            cell_L[m] = L;
            cell_P[m] = P;
        }
    }
}

// error-free sum (Knuth's two-sum), every operation rounded on its own: with
// plain operators the compiler may fuse the caller's product into s = a + b, and
// e would then describe a differently rounded b
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// FP32 form: float fragment terms, combined over the warp with compensated
// (two-sum) accumulation, so each cell's L and P keep float64-like accuracy
__global__ void __launch_bounds__(kThreads) k_alpha_cells32(const int* __restrict__ cell_off,
                                                            const unsigned* __restrict__ vals,
                                                            const ft_frag32* __restrict__ rec,
                                                            double* __restrict__ cell_L, double* __restrict__ cell_P,
                                                            const ft_counters* ctr) {
    const long long M = ctr->M;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long m = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); m < M; m += nw) {
        const int q0 = cell_off[m], q1 = cell_off[m + 1];
        float Lh = 0.f, Ll = 0.f, Ph = 0.f, Pl = 0.f;
        for (int q = q0 + lane; q < q1; q += 32) {
            const ft_frag32* f = rec + (vals ? vals[q] : (unsigned)q);
            const float az = f->an[2];
            float s, e;
            two_sum(Lh, __fmul_rn(az, __fadd_rn(f->c[2], 0.5f)), s, e);
            Lh = s;
            Ll += e;
            two_sum(Ph, az, s, e);
            Ph = s;
            Pl += e;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float s, e;
            two_sum(Lh, __shfl_xor_sync(0xffffffffu, Lh, o), s, e);
            Ll += __shfl_xor_sync(0xffffffffu, Ll, o) + e;
            Lh = s;
            two_sum(Ph, __shfl_xor_sync(0xffffffffu, Ph, o), s, e);
            Pl += __shfl_xor_sync(0xffffffffu, Pl, o) + e;
            Ph = s;
        }
        if (lane == 0) {
            cell_L[m] = (double)Lh + (double)Ll;
            cell_P[m] = (double)Ph + (double)Pl;
        }
    }
}

// one warp per (i, j) column, walking k downwards in chunks of 32 cells
template <class F>
__global__ void __launch_bounds__(kThreads) k_alpha_fill(F fr, const int* __restrict__ idx_map,
                                                         const double* __restrict__ cell_L,
                                                         const double* __restrict__ cell_P, double closure_tol,
                                                         ft_counters* ctr) {
    const int lane = threadIdx.x & 31;
    const long long ncol = fr.ncols;
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long gcol = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); gcol < ncol; gcol += nw) {
        const int b = fr.by_col(gcol);
        const ft_fdesc& D = fr.desc(b);
        const int n2 = D.g.n[2];
        const long long col = gcol - fr.col_base(b);
        const long long base = col * n2;            // front-local key of the column's first cell
        const long long gbase = fr.key_base(b) + base;  // the same, batch-global (index map)
        double* __restrict__ alpha = D.alpha;
        unsigned err = 0;
        double carry = 0.0;
        // the index map of the chunk below is loaded while this chunk is processed
        int k0 = ((n2 - 1) / 32) * 32;
        int m_next = (k0 + lane < n2) ? idx_map[gbase + k0 + lane] : -1;
        for (; k0 >= 0; k0 -= 32) {
            const int k = k0 + lane;
            const bool valid = k < n2;
            const int m = m_next;
            if (k0 >= 32) m_next = idx_map[gbase + k0 - 32 + lane];
            if (__ballot_sync(0xffffffffu, m >= 0) == 0u) {
                // no interfacial cell in this chunk: every cell takes the parity above it
                const long long cb = __double_as_longlong(carry);
                double r;
                if (cb == __double_as_longlong(0.0) || cb == __double_as_longlong(1.0)) {
                    r = carry;  // already exact: no float64 arithmetic needed
                } else {
                    r = rint(carry);
                    if (fabs(carry - r) > closure_tol) err |= FT_ST_NOT_CLOSED;
                    if (r != 0.0 && r != 1.0) err |= FT_ST_ORIENTATION;
                    r = fmin(fmax(r, 0.0), 1.0);
                    // below a closed stretch of front the parity is exact again
                    if (fabs(carry - rint(carry)) <= closure_tol) carry = rint(carry);
                }
                if (valid) alpha[base + k] = r;
                continue;
            }
            const double Pz = (m >= 0) ? cell_P[m] : 0.0;
            const double L = (m >= 0) ? cell_L[m] : 0.0;
            double x = Pz;  // inclusive suffix sum within the chunk
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_down_sync(0xffffffffu, x, o);
                if (lane + o < 32) x += y;
            }
            double ex = __shfl_down_sync(0xffffffffu, x, 1);
            if (lane == 31) ex = 0.0;
            const double S = carry + ex;
            carry += __shfl_sync(0xffffffffu, x, 0);
            if (valid) {
                double a;
                if (m >= 0) {
                    a = L + S;
                } else {
                    const double r = rint(S);
                    if (fabs(S - r) > closure_tol) err |= FT_ST_NOT_CLOSED;
                    if (r != 0.0 && r != 1.0) err |= FT_ST_ORIENTATION;
                    a = r;
                }
                alpha[base + k] = fmin(fmax(a, 0.0), 1.0);
            }
        }
        err = __reduce_or_sync(0xffffffffu, err);
        if (err && lane == 0) {
            ft_flag(ctr, err);
            fr.flag(b, err);
        }
    }
}

}  // namespace

namespace ft {

template <class F>
cudaError_t alpha_with(ft_workspace* ws, const F& fr, cudaStream_t s) {
    const bool fp32 = ws->last_precision == FT_FP32C;
    // records in sorted pair order when front_bin gathered them, else through the slot index
    const bool sorted = fp32 ? ws->srec32 != nullptr : ws->srec != nullptr;
    const unsigned* vals = sorted ? nullptr : ws->vals[ws->sorted_buf];
    count_launches(2);
    if (fp32) {
        Trace t(s, "k_alpha_cells32");
        k_alpha_cells32<<<ws->sm_count * 8, kThreads, 0, s>>>(ws->cell_off, vals, sorted ? ws->srec32 : ws->rec32,
                                                              ws->cell_L, ws->cell_P, ws->ctr);
    } else {
        Trace t(s, "k_alpha_cells");
        k_alpha_cells<<<ws->sm_count * 8, kThreads, 0, s>>>(ws->cell_off, vals, sorted ? ws->srec : ws->rec,
                                                            ws->cell_L, ws->cell_P, ws->ctr);
    }
    // the column parity of a closed front is an integer up to rounding of the fragment terms
    const double closure_tol = fp32 ? 1e-5 : 1e-9;
    Trace t(s, "k_alpha_fill");
    k_alpha_fill<F><<<ws->sm_count * ws->tune.fill_bps, kThreads, 0, s>>>(fr, ws->idx_map, ws->cell_L, ws->cell_P,
                                                                          closure_tol, ws->ctr);
    return cudaGetLastError();
}

cudaError_t launch_alpha(ft_workspace* ws, double* alpha, cudaStream_t s) {
    FrontsOne fr = ft_one(ws, nullptr, nullptr, 0, 0);
    fr.d0.alpha = alpha;
    return alpha_with(ws, fr, s);
}

cudaError_t launch_alpha_batch(ft_workspace* ws, cudaStream_t s) { return alpha_with(ws, ft_many(ws), s); }

}  // namespace ft
