// D2Q9 model pieces used inside the fused kernels (Sec. 2.1 velocity set and weights,
// eq. feq equilibrium, eq. LBM_collision BGK relaxation, Sec. 3 forcing term).
//
// Populations are handled in "storage form" s_k = f_k - omega_k * rho_ref: rho_ref = rho0 for
// the FP32 deviation storage and 0 for FP64 (then s_k = f_k).  Because sum_k omega_k e_k = 0,
// the momentum sum_k s_k e_k equals sum_k f_k e_k in both forms.
#pragma once

#include <cstdint>

namespace mlbm {

__host__ __device__ constexpr int ex_of(int k) {
    return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int k) {
    return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int k) {
    return k == 0 ? 0 : (k <= 4 ? ((k + 1) % 4) + 1 : ((k - 5 + 2) % 4) + 5);
}
template <typename T>
__host__ __device__ constexpr T omega_of(int k) {
    return k == 0 ? T(4) / T(9) : (k <= 4 ? T(1) / T(9) : T(1) / T(36));
}

static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 && opp_of(4) == 2, "opp");
static_assert(opp_of(5) == 7 && opp_of(6) == 8 && opp_of(7) == 5 && opp_of(8) == 6, "opp");
static_assert(ex_of(opp_of(6)) == -ex_of(6) && ey_of(opp_of(6)) == -ey_of(6), "opp");
// direction pairs of collide(): c_1 = (1,0), c_2 = (0,1), c_5 = (1,1), c_6 = (-1,1)
static_assert(ex_of(1) == 1 && ey_of(1) == 0 && ex_of(2) == 0 && ey_of(2) == 1, "axes");
static_assert(ex_of(5) == 1 && ey_of(5) == 1 && ex_of(6) == -1 && ey_of(6) == 1, "diagonals");

// Macroscopic fields of storage-form populations: drho = rho - rho_ref, and rho, u.
template <typename T>
__device__ __forceinline__ void moments_of(const T (&s)[9], T rho_ref, T &drho, T &rho, T &ux, T &uy) {
    drho = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8];
    T mx = (s[1] - s[3]) + (s[5] - s[6]) + (s[8] - s[7]);
    T my = (s[2] - s[4]) + (s[5] + s[6]) - (s[7] + s[8]);
    rho = rho_ref + drho;
    T ir = T(1) / rho;
    ux = mx * ir;
    uy = my * ir;
}

// Equilibrium in storage form: f^eq_k - omega_k rho_ref = omega_k (drho + rho (3 cu + 4.5 cu^2 - 1.5 u^2)).
template <typename T>
__device__ __forceinline__ T geq_of(int k, T drho, T rho, T ux, T uy, T usq15) {
    T cu = T(ex_of(k)) * ux + T(ey_of(k)) * uy;
    return omega_of<T>(k) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - usq15));
}

// In place: s <- s - (s - s^eq) / tau + omega_k e_k.g / c_s^2.  Returns the pre-collision
// moments through rho, ux, uy.
//
// Evaluated as s (1 - 1/tau) + s^eq / tau + F_k, direction pairs (k, opposite of k) together:
// c_k.u and e_k.g change sign between the two, so s^eq / tau splits into a common even part
// omega (drho + rho (4.5 cu^2 - 1.5 u^2)) / tau and an odd part 3 omega rho cu / tau, and the
// forcing term (odd as well) joins the odd part.  About half the arithmetic of evaluating the
// nine equilibria one by one, which matters where FP64 arithmetic bounds the step.
template <typename T>
__device__ __forceinline__ void collide(T (&s)[9], T rho_ref, T inv_tau, T gx, T gy, T &rho, T &ux,
                                        T &uy) {
    T drho;
    moments_of(s, rho_ref, drho, rho, ux, uy);
    const T usq15 = T(1.5) * (ux * ux + uy * uy);
    const T keep = T(1) - inv_tau;
    const T dt = drho * inv_tau, rt = rho * inv_tau;
    s[0] = fma(s[0], keep, omega_of<T>(0) * (dt - rt * usq15));
    // (k, opposite): c_k.u = cu, e_k.g = eg, weight w
    auto pair = [&](int k, int ko, T cu, T eg, T w) {
        const T even = w * fma(rt, fma(T(4.5) * cu, cu, -usq15), dt);
        const T odd = (T(3) * w) * fma(rt, cu, eg);
        s[k] = fma(s[k], keep, even + odd);
        s[ko] = fma(s[ko], keep, even - odd);
    };
    pair(1, 3, ux, gx, omega_of<T>(1));
    pair(2, 4, uy, gy, omega_of<T>(2));
    pair(5, 7, ux + uy, gx + gy, omega_of<T>(5));
    pair(6, 8, uy - ux, gy - gx, omega_of<T>(6));
}

// FP32 collision with exact conservation by construction.  With rounded lattice weights
// (fl(1/9), fl(1/36)) the equilibrium's mass and momentum differ from those of fhat by fixed
// relative amounts (3 (2 fl(1/9) + 4 fl(1/36)) = 1 + 7.45e-9 exactly, plus the rounding of the
// other constants), which would rescale the momentum of every node in the same direction at
// every step (a drift of order 1e-8 per step).  The non-equilibrium part n = fhat - f^eq
// is therefore projected onto zero mass and momentum with exact operations (its mass is taken
// from n_0, half of its x / y momentum from each of n_1, n_3 / n_2, n_4) before relaxing.
//
// The stored result is then rounded so that its mass and momentum are those of the collision in
// exact arithmetic (fhat's mass, fhat's momentum plus g) as closely as FP32 allows: the FP32
// updates leave a residual R = (sum D, sum e_x D - g_x, sum e_y D - g_y) of the changes
// D_k = s'_k - s_k, and the populations are re-rounded one at a time in the fixed order
// 1, 2, 3, 4, 5, 6, 7, 8, 0 at s'_k + delta_k, delta_k = -c_k . R, where c_k = (G + 0.01 I)^{-1}
// a_k is the minimum-norm feedback for a_k = (1, e_kx, e_ky) over the populations not yet
// re-rounded (G the sum of their a a^T; the rest population, last, takes the remaining mass).
// The rounding of the conserved moments, which the collision does not damp, would otherwise
// accumulate in the slowly decaying long-wave modes of large clouds.
__device__ __forceinline__ void conserve_rounding(float (&s)[9], const float (&s_in)[9], float gx, float gy) {
    constexpr int kOrder[9] = {1, 2, 3, 4, 5, 6, 7, 8, 0};
    constexpr float kC[9][3] = {{0.110987791f, 0.166389351f, 0.0f},
                                {0.128034429f, 0.0255557742f, 0.166389351f},
                                {0.121074514f, -0.175434229f, 0.0241665696f},
                                {0.137752876f, 0.0f, -0.172105214f},
                                {0.199600798f, 0.249376559f, 0.249376559f},
                                {0.331677695f, -0.08436278f, 0.414390337f},
                                {0.00487781084f, -0.497512438f, -0.492658895f},
                                {0.0049017205f, 0.495073771f, -0.495073771f},
                                {0.99009901f, 0.0f, 0.0f}};
    float d[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = s[k] - s_in[k];
    float r0 = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    float rx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]) - gx;
    float ry = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]) - gy;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int k = kOrder[p];
        const float delta = -((kC[p][0] * r0 + kC[p][1] * rx) + kC[p][2] * ry);
        const float v = s[k] + delta;
        const float dv = v - s[k];
        s[k] = v;
        r0 += dv;
        rx += float(ex_of(k)) * dv;
        ry += float(ey_of(k)) * dv;
    }
}

// kConserve = false leaves out the re-rounding (the lattice LBM comparison path, whose per-node
// arithmetic is small enough that it would cost throughput).
template <bool kConserve = true>
__device__ __forceinline__ void collide_projected(float (&s)[9], float rho_ref, float inv_tau, float gx, float gy,
                                                  float &rho, float &ux, float &uy) {
    float s_in[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s_in[k] = s[k];
    float drho;
    moments_of(s, rho_ref, drho, rho, ux, uy);
    const float usq15 = 1.5f * (ux * ux + uy * uy);
    float ne[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) ne[k] = s[k] - geq_of<float>(k, drho, rho, ux, uy, usq15);
    const float dm = ((ne[0] + ne[1]) + (ne[2] + ne[3])) + ((ne[4] + ne[5]) + (ne[6] + ne[7])) + ne[8];
    const float dx = (ne[1] - ne[3]) + (ne[5] - ne[6]) + (ne[8] - ne[7]);
    const float dy = (ne[2] - ne[4]) + (ne[5] + ne[6]) - (ne[7] + ne[8]);
    ne[0] -= dm;
    ne[1] -= 0.5f * dx;
    ne[3] += 0.5f * dx;
    ne[2] -= 0.5f * dy;
    ne[4] += 0.5f * dy;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float force = omega_of<float>(k) * 3.0f * (float(ex_of(k)) * gx + float(ey_of(k)) * gy);
        s[k] = s[k] - ne[k] * inv_tau + force;
    }
    if constexpr (kConserve) conserve_rounding(s, s_in, gx, gy);
}

}  // namespace mlbm
