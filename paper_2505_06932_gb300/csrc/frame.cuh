// frame.cuh -- the tangents (t1, t2) of the PPIC cell frame [t1 t2 n]
// (Sec. 3.2), shared by the fit and by the kernels that read its paraboloids.
#pragma once

#include "ft_internal.cuh"

namespace {

// Tangents (t1, t2) completing the unit normal n: the branchless basis of Duff
// et al. 2017 ("Building an orthonormal basis, revisited") built for m = R n in
// a fixed rotated reference frame (third row of R: (sin 1 cos 1, sin 1 sin 1,
// cos 1), a direction with no small-integer relation to axes or symmetric
// fronts) and rotated back, so that the basis' switch on sign(m_z) does not
// fall on fronts with an exactly vertical normal.
__constant__ double kFrameR[3][3] = {{0.890670841215793, -0.3614406733922875, -0.2758008198422935},
                                     {0.0, 0.6066239971779142, -0.7949888842291382},
                                     {0.4546487134128409, 0.7080734182735712, 0.5403023058681398}};
// the same matrix rounded to float (the FP32 form reads it without conversions)
__constant__ float kFrameRf[3][3] = {{0.890670841215793f, -0.3614406733922875f, -0.2758008198422935f},
                                     {0.0f, 0.6066239971779142f, -0.7949888842291382f},
                                     {0.4546487134128409f, 0.7080734182735712f, 0.5403023058681398f}};

template <typename T> __device__ __forceinline__ T frame_r(int r, int c);
template <> __device__ __forceinline__ double frame_r<double>(int r, int c) { return kFrameR[r][c]; }
template <> __device__ __forceinline__ float frame_r<float>(int r, int c) { return kFrameRf[r][c]; }

template <typename T>
__device__ __forceinline__ void basis(const T n[3], T t1[3], T t2[3]) {
    T m[3], u1[3], u2[3];
#pragma unroll
    for (int r = 0; r < 3; r++)
        m[r] = frame_r<T>(r, 0) * n[0] + frame_r<T>(r, 1) * n[1] + frame_r<T>(r, 2) * n[2];
    const T sg = copysign((T)1, m[2]);
    const T a = (T)-1 / (sg + m[2]);
    const T b = m[0] * m[1] * a;
    u1[0] = (T)1 + sg * m[0] * m[0] * a;
    u1[1] = sg * b;
    u1[2] = -sg * m[0];
    u2[0] = b;
    u2[1] = sg + m[1] * m[1] * a;
    u2[2] = -m[1];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        t1[c] = frame_r<T>(0, c) * u1[0] + frame_r<T>(1, c) * u1[1] + frame_r<T>(2, c) * u1[2];
        t2[c] = frame_r<T>(0, c) * u2[0] + frame_r<T>(1, c) * u2[1] + frame_r<T>(2, c) * u2[2];
    }
}

// The frame normal n of an interfacial cell as the PPIC accumulation stored it
// with its normal equations: float64 and unit in the plain form; float sums in
// the FP32 form, widened (exactly) and renormalised in float64.
__device__ __forceinline__ void sys_normal(const ft_cellsys& S, bool fp32, double n[3]) {
    if (fp32) {
        const float* v = reinterpret_cast<const float*>(S.v);
#pragma unroll
        for (int r = 0; r < 3; r++) n[r] = (double)v[54 + 2 * r];
        const double il = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
#pragma unroll
        for (int r = 0; r < 3; r++) n[r] *= il;
    } else {
#pragma unroll
        for (int r = 0; r < 3; r++) n[r] = S.v[27 + r];
    }
}

}  // namespace
