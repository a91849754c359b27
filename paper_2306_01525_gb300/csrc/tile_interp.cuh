// Tile-staged own-stencil interpolation shared by the fused step and its adjoint (Sec. 2.3,
// eq. shape_vector): the halo of a tile of B Morton-ordered nodes is staged in shared memory as
// [slot][8] populations, and each node interpolates its eight moving populations over its
// stencil members, whose halo slots come packed two per 32-bit word.
//   FP32: fhat_k = f_k(i) + sum_{j>=1} W_k[j](i) (f_k(s_j(i)) - f_k(i)) -- differences to the
//         centre value, shape vectors [j-1][2][B][4 directions] as float4;
//   FP64: fhat_k = sum_{j>=0} W_k[j](i) f_k(s_j(i)) literally, [j][4][B][2 directions] double2.
// The adjoint calls the same routine, so it recomputes fhat with the forward's arithmetic.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace mlbm {

// Populations moved per shared-memory or shape-vector load: 4 directions in FP32 (16 B),
// 2 directions in FP64 (16 B).
template <typename T> struct V;
template <> struct V<float> {
    using type = float4;
    static constexpr int width = 4;
};
template <> struct V<double> {
    using type = double2;
    static constexpr int width = 2;
};

// acc += w (x - c) (difference form, FP32) or acc += w x (literal form, FP64)
template <bool kLiteral>
__device__ __forceinline__ void vfma(float4 &acc, const float4 w, const float4 x, const float4 c) {
    acc.x = fmaf(w.x, x.x - c.x, acc.x);
    acc.y = fmaf(w.y, x.y - c.y, acc.y);
    acc.z = fmaf(w.z, x.z - c.z, acc.z);
    acc.w = fmaf(w.w, x.w - c.w, acc.w);
}
template <bool kLiteral>
__device__ __forceinline__ void vfma(double2 &acc, const double2 w, const double2 x, const double2 c) {
    if constexpr (kLiteral) {
        acc.x = fma(w.x, x.x, acc.x);
        acc.y = fma(w.y, x.y, acc.y);
    } else {
        acc.x = fma(w.x, x.x - c.x, acc.x);
        acc.y = fma(w.y, x.y - c.y, acc.y);
    }
}
__device__ __forceinline__ void vmul(float4 &acc, const float4 w, const float4 x) {
    acc = make_float4(w.x * x.x, w.y * x.y, w.z * x.z, w.w * x.w);
}
__device__ __forceinline__ void vmul(double2 &acc, const double2 w, const double2 x) {
    acc = make_double2(w.x * x.x, w.y * x.y);
}
__device__ __forceinline__ void vunpack(float *d, const float4 &a) {
    d[0] = a.x;
    d[1] = a.y;
    d[2] = a.z;
    d[3] = a.w;
}
__device__ __forceinline__ void vunpack(double *d, const double2 &a) {
    d[0] = a.x;
    d[1] = a.y;
}
__device__ __forceinline__ void vzero(float4 &v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vzero(double2 &v) { v = make_double2(0.0, 0.0); }
__device__ __forceinline__ void vpack(float4 &v, const float *s) { v = make_float4(s[0], s[1], s[2], s[3]); }
__device__ __forceinline__ void vpack(double2 &v, const double *s) { v = make_double2(s[0], s[1]); }
__device__ __forceinline__ void vunpack_sum(float *d, const float4 &c, const float4 &a) {
    d[0] = c.x + a.x;
    d[1] = c.y + a.y;
    d[2] = c.z + a.z;
    d[3] = c.w + a.w;
}
__device__ __forceinline__ void vunpack_sum(double *d, const double2 &c, const double2 &a) {
    d[0] = c.x + a.x;
    d[1] = c.y + a.y;
}

__device__ __forceinline__ void vadd(float4 &a, const float4 w) {
    a.x += w.x;
    a.y += w.y;
    a.z += w.z;
    a.w += w.w;
}
__device__ __forceinline__ void vadd(double2 &a, const double2 w) {
    a.x += w.x;
    a.y += w.y;
}

// Stage f_k, k = 1..8, of the tile's U halo nodes (stored positions halo[u]) as sh[u][8].
template <typename T>
__device__ __forceinline__ void stage_halo(const int32_t *__restrict__ halo, int U, const T *__restrict__ f,
                                           int64_t N, typename V<T>::type *sh) {
    using VT = typename V<T>::type;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
        const int64_t node = __ldg(halo + u);
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldg(f + (int64_t)(k + 1) * N + node);
#pragma unroll
        for (int q = 0; q < NV; ++q) vpack(sh[u * NV + q], v + q * W);
    }
}

// The same halo staged direction-major, sh[k][U] (k = 0..7 for populations 1..8).
template <typename T>
__device__ __forceinline__ void stage_halo_dirmajor(const int32_t *__restrict__ halo, int U, const T *__restrict__ f,
                                                    int64_t N, T *sh) {
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
        const int64_t node = __ldg(halo + u);
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[k * U + u] = __ldg(f + (int64_t)(k + 1) * N + node);
    }
}

// Members 1..m1 of node b's own stencil: acc += W (x - c) (FP32) or acc += W x (FP64), with wp
// at the shape vectors of member 1 for node b and lp at its slot words.  kSum also adds the
// weights up in ws (the centre coefficient of the FP32 form is 1 - sum_{j>=1} W).
template <typename T, int B, bool kSum>
__device__ __forceinline__ void interp_own(const typename V<T>::type *__restrict__ wp,
                                           const uint32_t *__restrict__ lp, const typename V<T>::type *sh,
                                           const typename V<T>::type (&c)[8 / V<T>::width],
                                           typename V<T>::type (&acc)[8 / V<T>::width],
                                           typename V<T>::type (&ws)[8 / V<T>::width], int m1) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int NV = 8 / V<T>::width;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < m1; j += 2) {
        const uint32_t pr = __ldcs(lp + (int64_t)(j >> 1) * B);
        VT w0[NV], w1[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            w0[q] = __ldcs(wp + (int64_t)(j * NV + q) * B);
            w1[q] = __ldcs(wp + (int64_t)((j + 1) * NV + q) * B);
        }
        const int s0 = (int)(pr & 0xFFFFu), s1 = (int)(pr >> 16);
#pragma unroll
        for (int q = 0; q < NV; ++q) vfma<kLiteral>(acc[q], w0[q], sh[s0 * NV + q], c[q]);
#pragma unroll
        for (int q = 0; q < NV; ++q) vfma<kLiteral>(acc[q], w1[q], sh[s1 * NV + q], c[q]);
        if constexpr (kSum) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                vadd(ws[q], w0[q]);
                vadd(ws[q], w1[q]);
            }
        }
    }
    if (j < m1) {
        const uint32_t pr = __ldcs(lp + (int64_t)(j >> 1) * B);
        const int s0 = (int)(pr & 0xFFFFu);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const VT w0 = __ldcs(wp + (int64_t)(j * NV + q) * B);
            vfma<kLiteral>(acc[q], w0, sh[s0 * NV + q], c[q]);
            if constexpr (kSum) vadd(ws[q], w0);
        }
    }
}

}  // namespace mlbm
