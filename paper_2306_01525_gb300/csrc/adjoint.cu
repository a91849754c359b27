// Discrete adjoint of the fused step (reverse mode of pull-stream, bounce-back, collide) and of
// the initial state and the moments, for gradients of a loss on the macroscopic fields with
// respect to tau, the body force g and the initial fields.
//
// Forward step (storage form s, lattice units): fhat = B (S s), s' = C(fhat; tau, g) with
//   S  the interpolation fhat_k(i) = sum_j W_k[j](i) s_k(s_j(i))       (Sec. 2.3), in the form
//      the forward kernel evaluates it: FP64 literally, FP32 as s_k(i) + sum_{j>=1} W (s_k(s_j) -
//      s_k(i)), i.e. with centre coefficient 1 - sum_{j>=1} W_k[j](i)
//   B  the wall bounce-back fhat_k = fhat_k' on unknown populations      (Sec. 3)
//   C  the BGK collision with forcing                                    (eq. LBM_collision, Sec. 3)
// Reverse: mu = J_C^T lam, mut = B^T mu, lam_prev = S^T mut.  S^T is done as a pull over the
// transposed stencil (for node m, the pairs (i, j) with s_j(i) = m, the centre pair (m, 0)
// included), in a fixed order, so the result is deterministic without atomics.  Parameter
// gradients are reduced per tile and then per segment in a fixed order.
//
// J_C and dL/dtau need the moments and the non-equilibrium part of fhat.  When the caller
// passes the forward's output s' = C(fhat) they come from it: the collision keeps rho and adds
// exactly g to rho u, and s' - F - s^eq = (1 - 1/tau)(fhat - s^eq), so no shape vector is read.
// Near tau = 1 that division loses fhat (at tau = 1, s' = s^eq + F whatever fhat was), so with
// |1 - 1/tau| < 1/16 in any segment, or without s', fhat is recomputed from s with the forward's
// own tile interpolation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>

#include "d2q9_device.cuh"
#include "mlbm_internal.h"
#include "tile_interp.cuh"

namespace mlbm {

int set_params(mlbm_weights *w, const mlbm_params *params, cudaStream_t st);
int check_dtype(const mlbm_weights *w, int dtype);
int cuda_check_step(cudaError_t e, const char *what);

namespace {

constexpr int kThreads = 256;
// rows per CTA of the transposed pull: one row per thread, a CTA per 128 rows, so that the
// hardware's block scheduling balances the rows' uneven lengths
constexpr int kPullThreads = 128;

__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh) {
    sh[threadIdx.x] = a;
    sh[kThreads + threadIdx.x] = b;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[threadIdx.x] += sh[threadIdx.x + s];
            sh[kThreads + threadIdx.x] += sh[kThreads + threadIdx.x + s];
        }
        __syncthreads();
    }
    a = sh[0];
    b = sh[kThreads];
    __syncthreads();
}

// d f^eq_k / d rho and d f^eq_k / d u contracted with lam: returns A_rho, A_x, A_y.
template <typename T>
__device__ __forceinline__ void feq_vjp(const T (&lam)[9], T rho, T ux, T uy, T &Ar, T &Ax, T &Ay) {
    const T usq15 = T(1.5) * (ux * ux + uy * uy);
    Ar = Ax = Ay = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const T ex = T(ex_of(k)), ey = T(ey_of(k));
        const T cu = ex * ux + ey * uy;
        const T wl = omega_of<T>(k) * lam[k];
        Ar += wl * (T(1) + T(3) * cu + T(4.5) * cu * cu - usq15);
        const T c = wl * rho * (T(3) + T(9) * cu);
        Ax += c * ex - wl * rho * T(3) * ux;
        Ay += c * ey - wl * rho * T(3) * uy;
    }
}

template <typename T>
struct AdjArgs {
    const TileDev *__restrict__ tiles;
    const int32_t *__restrict__ halo;
    const uint32_t *__restrict__ lidx;
    const T *__restrict__ wt;           // tile-layout shape vectors of the forward step
    const uint16_t *__restrict__ mask;
    const T *__restrict__ fdir;         // [2][N]
    const T *__restrict__ params;       // [nseg][4]: tau, g, rho0, 1/tau in T
    const T *__restrict__ s_prev;
    const T *__restrict__ s_next;       // forward output C(fhat), or null (recompute fhat)
    const T *__restrict__ lam_next;
    T *__restrict__ lam_prev;
    T *__restrict__ mut;    // [N][8] node-major: bounce-back-transposed cotangent of fhat
    double *__restrict__ partials;  // [ntiles][2]
    const int64_t *__restrict__ slice;    // [ceil(N/32)+1] offsets of the sliced entry table
    const int32_t *__restrict__ tsrc;     // per entry slot: stored position of the reading node (-1: none)
    const T *__restrict__ tw;             // per entry slot [8]: its shape-vector values (0: none)
    int64_t N;
    int ntiles;
};

// Transposed collision Jacobian (with d f^eq / d(rho, u)) and transposed bounce-back at node p:
// mu = J_C^T lam at the moments (rho, u) of fhat, mut_l = [l not unknown] mu_l + [l' unknown]
// mu_l'.  Writes lam_prev_0 = mut_0 (population 0 is not interpolated), returns mut_1..8.
template <typename T>
__device__ __forceinline__ void adj_collide_node(const AdjArgs<T> &a, int64_t p, const T (&lam)[9], T rho, T ux,
                                                 T uy, T inv_tau, uint16_t mb, T (&out)[8]) {
    T Ar, Ax, Ay;
    feq_vjp<T>(lam, rho, ux, uy, Ar, Ax, Ay);
    const T ir = T(1) / rho;
    T mu[9];
#pragma unroll
    for (int l = 0; l < 9; ++l)
        mu[l] = (T(1) - inv_tau) * lam[l] +
                inv_tau * (Ar + (Ax * (T(ex_of(l)) - ux) + Ay * (T(ey_of(l)) - uy)) * ir);
    T mt[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        T v = (mb >> l & 1u) ? T(0) : mu[l];
        if (l > 0 && (mb >> opp_of(l) & 1u)) v += mu[opp_of(l)];
        mt[l] = v;
    }
    a.lam_prev[p] = mt[0];
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = mt[k + 1];
}

// Per-tile sums of the parameter-gradient terms in a fixed order: warps by shuffles in the
// step's precision (FP64 operations are scarce on this part), then the warps' sums in FP64 in
// index order.  Called by every thread of the block; ends with a barrier.
template <typename T, int B>
__device__ __forceinline__ void tile_partials(T dtau, T dg, double (&red)[2][B / 32], double *__restrict__ partials,
                                              int t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dtau += __shfl_xor_sync(0xffffffffu, dtau, o);
        dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    if (lane == 0) {
        red[0][warp] = (double)dtau;
        red[1][warp] = (double)dg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < B / 32; ++q) {
            s0 += red[0][q];
            s1 += red[1][q];
        }
        partials[2 * t] = s0;
        partials[2 * t + 1] = s1;
    }
    __syncthreads();
}

// Local part of the reverse step by recomputation, tile by tile like the forward step (B nodes
// per CTA, halo of s_prev staged in shared memory): fhat with the forward's own arithmetic, then
// the transposed collision and bounce-back; writes mut node-major for the scatter and the
// per-tile sums of dL/dtau and dL/dg.
template <typename T, int B>
__global__ void __launch_bounds__(B, 1) adj_local_kernel(AdjArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr bool kDev = std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *sh = reinterpret_cast<VT *>(smem_raw);  // [U][NV]
    __shared__ double red[2][B / 32];
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        stage_halo<T>(a.halo + tile.h_off, tile.U, a.s_prev, N, sh);
        __syncthreads();
        T dtau = T(0), dg = T(0);
        const int b = threadIdx.x;
        if (b < tile.count) {
            const int64_t p = tile.begin + b;
            VT c[NV], acc[NV], ws[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                c[q] = sh[b * NV + q];
                vzero(acc[q]);
            }
            const uint32_t *__restrict__ lp = a.lidx + tile.l_off + b;
            const VT *__restrict__ wp;
            if constexpr (!kDev) {
                wp = reinterpret_cast<const VT *>(a.wt + tile.w64_off) + b;
#pragma unroll
                for (int q = 0; q < NV; ++q) vmul(acc[q], __ldcs(wp + (int64_t)q * B), c[q]);
                wp += (int64_t)NV * B;
            } else {
                wp = reinterpret_cast<const VT *>(a.wt + tile.w_off) + b;
            }
            interp_own<T, B, false>(wp, lp, sh, c, acc, ws, tile.K - 1);
            T f[9];
            f[0] = a.s_prev[p];
            {
                T cv[8], av[8];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    vunpack(cv + q * W, c[q]);
                    vunpack(av + q * W, acc[q]);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) f[k + 1] = kDev ? cv[k] + av[k] : av[k];
            }
            const uint16_t mb = a.mask ? a.mask[p] : (uint16_t)0;
            if (mb) {
                T g[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) g[k] = f[k];
#pragma unroll
                for (int k = 1; k < 9; ++k)
                    if (mb >> k & 1u) f[k] = g[opp_of(k)];
            }
            const T *pr = a.params + 4 * tile.seg;
            const T inv_tau = pr[3];
            const T rho_ref = kDev ? pr[2] : T(0);
            T drho, rho, ux, uy;
            moments_of<T>(f, rho_ref, drho, rho, ux, uy);
            const T usq15 = T(1.5) * (ux * ux + uy * uy);
            T lam[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) lam[k] = a.lam_next[(int64_t)k * N + p];
            const T fx = a.fdir[p], fy = a.fdir[N + p];
            T st = T(0), sg = T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                T geq = geq_of<T>(k, drho, rho, ux, uy, usq15);
                st += lam[k] * (f[k] - geq);
                sg += lam[k] * omega_of<T>(k) * T(3) * (T(ex_of(k)) * fx + T(ey_of(k)) * fy);
            }
            dtau = st * inv_tau * inv_tau;
            dg = sg;
            T mt[8];
            adj_collide_node<T>(a, p, lam, rho, ux, uy, inv_tau, mb, mt);
            VT *mo = reinterpret_cast<VT *>(a.mut + p * 8);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                VT v;
                vpack(v, mt + q * W);
                mo[q] = v;
            }
        }
        tile_partials<T, B>(dtau, dg, red, a.partials, t);
    }
}

// The same local part from the forward's output s_next = C(fhat), one node per thread and no
// shape vector, halo or stencil read: rho is the moment of s_next, rho u that of s_next minus g
// (the forcing term adds exactly g), and sum_k lam_k (fhat_k - s^eq_k) = sum_k lam_k (s_next_k
// - F_k - s^eq_k) / (1 - 1/tau), with F_k = 3 omega_k e_k.g as the forward adds it.
template <typename T, int B>
__global__ void __launch_bounds__(B) adj_local_next_kernel(AdjArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr bool kDev = std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    __shared__ double red[2][B / 32];
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        T dtau = T(0), dg = T(0);
        const int b = threadIdx.x;
        if (b < tile.count) {
            const int64_t p = tile.begin + b;
            const T *pr = a.params + 4 * tile.seg;
            const T inv_tau = pr[3], gm = pr[1];
            const T rho_ref = kDev ? pr[2] : T(0);
            T s[9], lam[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                s[k] = __ldcs(a.s_next + (int64_t)k * N + p);
                lam[k] = __ldcs(a.lam_next + (int64_t)k * N + p);
            }
            const uint16_t mb = a.mask ? a.mask[p] : (uint16_t)0;
            const T fx = a.fdir[p], fy = a.fdir[N + p];
            T gx = T(0), gy = T(0);
            if (gm != T(0)) {
                gx = gm * fx;
                gy = gm * fy;
            }
            T drho, rho, ux, uy;
            moments_of<T>(s, rho_ref, drho, rho, ux, uy);
            const T ir = T(1) / rho;
            ux -= gx * ir;
            uy -= gy * ir;
            const T usq15 = T(1.5) * (ux * ux + uy * uy);
            T st = T(0), sg = T(0);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T w3 = omega_of<T>(k) * T(3);
                const T force = w3 * (T(ex_of(k)) * gx + T(ey_of(k)) * gy);
                st += lam[k] * ((s[k] - force) - geq_of<T>(k, drho, rho, ux, uy, usq15));
                sg += lam[k] * w3 * (T(ex_of(k)) * fx + T(ey_of(k)) * fy);
            }
            dtau = st * (inv_tau * inv_tau / (T(1) - inv_tau));
            dg = sg;
            T mt[8];
            adj_collide_node<T>(a, p, lam, rho, ux, uy, inv_tau, mb, mt);
            VT *mo = reinterpret_cast<VT *>(a.mut + p * 8);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                VT v;
                vpack(v, mt + q * W);
                mo[q] = v;
            }
        }
        tile_partials<T, B>(dtau, dg, red, a.partials, t);
    }
}

// lam_prev_k(m) = sum over the entries (i, j) of row m of the transposed stencil (s_j(i) = m) of
// c_kj(i) mut_k(i), k = 1..8: the transpose of the interpolation, pulled in the row's fixed order
// (j-major, so the centre entry (m, 0) comes first).  c_kj is the coefficient of s_k(s_j(i)) in
// the forward's fhat_k(i): W_k[j](i), except the centre of the FP32 difference form,
// 1 - sum_{j>=1} W_k[j](i).  The entries are tabulated sliced by 32 rows (a warp): entry
// t of row 32 s + l sits at slice_off[s] + 32 t + l, rows padded to the slice's longest with
// empty entries (src -1), so each warp reads 32 consecutive entries per pass (1 KB in FP32), and
// mut is node-major (one 32-byte sector per gathered node in FP32).
template <typename T>
__global__ void __launch_bounds__(kPullThreads) adj_transpose_kernel(AdjArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    const int64_t N = a.N;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < N; m += (int64_t)gridDim.x * blockDim.x) {
        T acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = T(0);
        const int64_t s = m >> 5, b1 = a.slice[s + 1];
        int64_t q = a.slice[s] + (m & 31);
        // entry e of the row; past its end: src -1
        auto load = [&](int64_t e, int32_t &src, VT (&w)[NV]) {
            src = -1;
            if (e < b1) {
                src = __ldcs(a.tsrc + e);
#pragma unroll
                for (int qq = 0; qq < NV; ++qq) w[qq] = __ldcs(reinterpret_cast<const VT *>(a.tw + e * 8) + qq);
            }
        };
        auto add = [&](int32_t src, const VT (&w)[NV]) {
            if (src < 0) return;
            const VT *mi = reinterpret_cast<const VT *>(a.mut + (int64_t)src * 8);
            T wv[8], mv[8];
#pragma unroll
            for (int qq = 0; qq < NV; ++qq) {
                vunpack(wv + qq * W, w[qq]);
                vunpack(mv + qq * W, __ldg(mi + qq));
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = fma(wv[k], mv[k], acc[k]);
        };
        // the next pair's table entries are in flight while the current pair's cotangents are
        // gathered (the rows of a slice share one length, so the loop is uniform over the warp)
        int32_t s0, s1;
        VT w0[NV], w1[NV];
        load(q, s0, w0);
        load(q + 32, s1, w1);
        for (; q < b1; q += 64) {
            int32_t n0, n1;
            VT v0[NV], v1[NV];
            load(q + 64, n0, v0);
            load(q + 96, n1, v1);
            add(s0, w0);
            add(s1, w1);
            s0 = n0;
            s1 = n1;
#pragma unroll
            for (int qq = 0; qq < NV; ++qq) {
                w0[qq] = v0[qq];
                w1[qq] = v1[qq];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) a.lam_prev[(int64_t)(k + 1) * N + m] = acc[k];
    }
}

// Sliced table of the transposed stencil (layout above): row m's entry q = j n + i (member j of
// node i, segment-local) gets the reading node's stored position and its coefficients c_kj(i),
// k = 1..8, in the step's precision (the FP32 values round the FP64 shape vectors as the
// forward's FP32 layout does, and the FP32 centre coefficient adds them up in member order as
// the forward's interpolation does); padding gets src -1 and zero coefficients.
template <typename T>
__global__ void adj_table_kernel(int64_t N, const int32_t *__restrict__ node_seg, const SegDev *__restrict__ seg,
                                 const double *__restrict__ w64c, const int32_t *__restrict__ csr_ptr,
                                 const int32_t *__restrict__ csr_ent, const int64_t *__restrict__ slice,
                                 int32_t *__restrict__ tsrc, T *__restrict__ tw) {
    constexpr bool kDev = std::is_same<T, float>::value;
    // rows N .. 32 ceil(N/32) - 1 of the last slice do not exist: their slots are filled empty
    const int64_t rows = (N + 31) & ~(int64_t)31;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < rows; m += (int64_t)gridDim.x * blockDim.x) {
        const bool row = m < N;
        const SegDev sd = seg[node_seg[row ? m : 0]];
        const int64_t s = m >> 5, base = slice[s] + (m & 31), len = (slice[s + 1] - slice[s]) >> 5;
        const int32_t e0 = row ? csr_ptr[m] : 0, e1 = row ? csr_ptr[m + 1] : 0;
        for (int64_t t = 0; t < len; ++t) {
            const int64_t q = base + 32 * t;
            int32_t src = -1;
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = T(0);
            if (e0 + t < e1) {
                const int64_t e = csr_ent[e0 + t];
                const int64_t j = e / sd.n, i = e - j * sd.n;
                src = (int32_t)(sd.off + i);
                const double *wk = w64c + sd.w_off + i;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (j > 0 || !kDev) {
                        v[k] = (T)wk[((int64_t)k * sd.K + j) * sd.n];
                    } else {
                        float ws = 0.f;
                        for (int jj = 1; jj < sd.K; ++jj) ws += (float)wk[((int64_t)k * sd.K + jj) * sd.n];
                        v[k] = (T)(1.f - ws);
                    }
                }
            }
            tsrc[q] = src;
#pragma unroll
            for (int k = 0; k < 8; ++k) tw[q * 8 + k] = v[k];
        }
    }
}

// grad[2 s + c] += sum over tiles of segment s (in tile order) of partials[2 t + c].
__global__ void __launch_bounds__(kThreads) grad_finalize_kernel(const TileDev *__restrict__ tiles, int ntiles,
                                                                  const double *__restrict__ partials,
                                                                  double *__restrict__ grad) {
    __shared__ double sh[2 * kThreads];
    const int s = blockIdx.x;
    double a0 = 0.0, a1 = 0.0;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        if (tiles[t].seg == s) {
            a0 += partials[2 * t];
            a1 += partials[2 * t + 1];
        }
    block_sum2(a0, a1, sh);
    if (threadIdx.x == 0) {
        grad[2 * s] += a0;
        grad[2 * s + 1] += a1;
    }
}

// Seed from a loss on (rho, u) of the level whose post-collision state is f.
template <typename T>
__global__ void __launch_bounds__(kThreads) moments_adjoint_kernel(
    const TileDev *__restrict__ tiles, int ntiles, const int64_t *__restrict__ perm,
    const double *__restrict__ fdir, const double *__restrict__ params, const T *__restrict__ f,
    const double *__restrict__ drho_in, const double *__restrict__ dux_in, const double *__restrict__ duy_in,
    T *__restrict__ lam, double *__restrict__ partials, int64_t N) {
    constexpr bool kDev = std::is_same<T, float>::value;
    __shared__ double sh[2 * kThreads];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        double dg = 0.0, zero = 0.0;
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
            const int64_t p = tile.begin + b;
            const double *pr = params + 4 * tile.seg;
            double s[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) s[k] = (double)f[(int64_t)k * N + p];
            double dr, rho, ux, uy;
            moments_of<double>(s, kDev ? pr[2] : 0.0, dr, rho, ux, uy);
            const double fx = fdir[p], fy = fdir[N + p];
            ux -= pr[1] * fx / rho;
            uy -= pr[1] * fy / rho;
            const int64_t o = perm[p];
            const double a = drho_in[o], bx = dux_in[o], by = duy_in[o];
#pragma unroll
            for (int l = 0; l < 9; ++l)
                lam[(int64_t)l * N + p] = (T)(a + (bx * (ex_of(l) - ux) + by * (ey_of(l) - uy)) / rho);
            dg += -(bx * fx + by * fy) / rho;
        }
        block_sum2(zero, dg, sh);
        if (threadIdx.x == 0) {
            partials[2 * t] = 0.0;
            partials[2 * t + 1] = dg;
        }
    }
}

// Reverse of the initial state s_k = f^eq_k(rho, u) - omega_k rho_ref + omega_k 3 e_k.g.
template <typename T>
__global__ void __launch_bounds__(kThreads) init_adjoint_kernel(
    const TileDev *__restrict__ tiles, int ntiles, const int64_t *__restrict__ perm,
    const double *__restrict__ fdir, const double *__restrict__ rho_in, const double *__restrict__ ux_in,
    const double *__restrict__ uy_in, const T *__restrict__ lam0, double *__restrict__ drho,
    double *__restrict__ dux, double *__restrict__ duy, double *__restrict__ partials, int64_t N) {
    __shared__ double sh[2 * kThreads];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        double dg = 0.0, zero = 0.0;
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
            const int64_t p = tile.begin + b;
            const int64_t o = perm[p];
            double lam[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) lam[k] = (double)lam0[(int64_t)k * N + p];
            double Ar, Ax, Ay;
            feq_vjp<double>(lam, rho_in[o], ux_in[o], uy_in[o], Ar, Ax, Ay);
            drho[o] = Ar;
            dux[o] = Ax;
            duy[o] = Ay;
            const double fx = fdir[p], fy = fdir[N + p];
#pragma unroll
            for (int k = 0; k < 9; ++k) dg += lam[k] * omega_of<double>(k) * 3.0 * (ex_of(k) * fx + ey_of(k) * fy);
        }
        block_sum2(zero, dg, sh);
        if (threadIdx.x == 0) {
            partials[2 * t] = 0.0;
            partials[2 * t + 1] = dg;
        }
    }
}

int ensure_adj_scratch(mlbm_weights *w) {
    size_t need = sizeof(double) * (8 * (size_t)w->N + 2 * (size_t)w->ntiles);
    if (w->d_scratch && w->scratch_bytes >= need) return MLBM_OK;
    cudaFree(w->d_scratch);
    w->d_scratch = nullptr;
    cudaError_t e = cudaMalloc(&w->d_scratch, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w->d_scratch = nullptr;
        w->scratch_bytes = 0;
        return fail(MLBM_ENOMEM, "adjoint scratch allocation failed");
    }
    w->scratch_bytes = need;
    return MLBM_OK;
}

int grid_of(const mlbm_weights *w, const void *fn) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
    return std::max(1, std::min(w->ntiles, std::max(1, per_sm) * w->num_sms));
}

template <typename T>
int ensure_adj_tables(mlbm_weights *w, cudaStream_t st) {
    const int i = std::is_same<T, float>::value ? 0 : 1;
    if (w->d_adj_tw[i]) return MLBM_OK;
    int rc = MLBM_OK;
    if (!w->d_adj_slice) {
        // slice offsets from the row lengths (host arithmetic on the downloaded row pointers)
        std::vector<int32_t> ptr((size_t)w->N + 1);
        if ((rc = cuda_check_step(cudaMemcpy(ptr.data(), w->d_csr_ptr, sizeof(int32_t) * ptr.size(),
                                             cudaMemcpyDeviceToHost), "row pointers")))
            return rc;
        const int64_t ns = (w->N + 31) / 32;
        std::vector<int64_t> off((size_t)ns + 1, 0);
        for (int64_t s = 0; s < ns; ++s) {
            int32_t len = 0;
            for (int64_t m = 32 * s; m < std::min<int64_t>(32 * s + 32, w->N); ++m) len = std::max(len, ptr[m + 1] - ptr[m]);
            off[s + 1] = off[s] + 32 * (int64_t)len;
        }
        w->adj_slots = off[ns];
        if (cudaMalloc(&w->d_adj_slice, sizeof(int64_t) * off.size()) != cudaSuccess ||
            cudaMalloc(&w->d_adj_tsrc, sizeof(int32_t) * std::max<int64_t>(1, w->adj_slots)) != cudaSuccess) {
            cudaGetLastError();
            return fail(MLBM_ENOMEM, "adjoint table allocation failed");
        }
        if ((rc = cuda_check_step(cudaMemcpy(w->d_adj_slice, off.data(), sizeof(int64_t) * off.size(),
                                             cudaMemcpyHostToDevice), "slice offsets")))
            return rc;
    }
    if (cudaMalloc(&w->d_adj_tw[i], sizeof(T) * 8 * std::max<int64_t>(1, w->adj_slots)) != cudaSuccess) {
        cudaGetLastError();
        w->d_adj_tw[i] = nullptr;
        return fail(MLBM_ENOMEM, "adjoint table allocation failed");
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((w->N + 31 + 255) / 256, 65536));
    adj_table_kernel<T><<<grid, 256, 0, st>>>(w->N, w->d_node_seg, w->d_seg, w->d_w64, w->d_csr_ptr, w->d_csr_ent,
                                              w->d_adj_slice, w->d_adj_tsrc, (T *)w->d_adj_tw[i]);
    return cuda_check_step(cudaGetLastError(), "adjoint table launch");
}

template <typename T, int B>
int launch_adj_local(mlbm_weights *w, const AdjArgs<T> &a, cudaStream_t st) {
    const size_t smem = (size_t)w->umax * 8 * sizeof(T);
    const void *fn = (const void *)adj_local_kernel<T, B>;
    int rc = cuda_check_step(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "adjoint shared memory");
    if (rc) return rc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, B, smem);
    if (per_sm < 1) return fail(MLBM_EINVAL, "a tile's halo does not fit in shared memory for the adjoint");
    const int grid = std::max(1, std::min(w->ntiles, per_sm * w->num_sms));
    adj_local_kernel<T, B><<<grid, B, smem, st>>>(a);
    return MLBM_OK;
}

template <typename T, int B>
int launch_adj_local_next(mlbm_weights *w, const AdjArgs<T> &a, cudaStream_t st) {
    const void *fn = (const void *)adj_local_next_kernel<T, B>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, B, 0);
    const int grid = std::max(1, std::min(w->ntiles, std::max(1, per_sm) * w->num_sms));
    adj_local_next_kernel<T, B><<<grid, B, 0, st>>>(a);
    return MLBM_OK;
}

template <typename T>
int adjoint_step_t(mlbm_weights *w, const void *s_prev, const void *s_next, const void *lam_next, void *lam_prev,
                   double *grad, cudaStream_t st) {
    constexpr bool kDev = std::is_same<T, float>::value;
    int rc = ensure_adj_tables<T>(w, st);
    if (rc) return rc;
    AdjArgs<T> a;
    a.tiles = w->d_tiles;
    a.halo = w->d_halo;
    a.lidx = w->d_lidx;
    a.wt = kDev ? (const T *)w->d_w32t : (const T *)w->d_w64t;
    a.mask = w->has_mask ? w->d_mask : nullptr;
    a.fdir = kDev ? (const T *)w->d_fdir32 : (const T *)w->d_fdir64;
    a.params = kDev ? (const T *)(w->d_params + 4 * (size_t)w->nseg) : (const T *)w->d_params;
    a.s_prev = (const T *)s_prev;
    a.s_next = (const T *)s_next;
    a.lam_next = (const T *)lam_next;
    a.lam_prev = (T *)lam_prev;
    a.mut = (T *)w->d_scratch;
    a.partials = (double *)((char *)w->d_scratch + sizeof(double) * 8 * (size_t)w->N);
    a.slice = w->d_adj_slice;
    a.tsrc = w->d_adj_tsrc;
    a.tw = (const T *)w->d_adj_tw[kDev ? 0 : 1];
    a.N = w->N;
    a.ntiles = w->ntiles;
    if (s_next)
        rc = w->tile_nodes == kTileNodes ? launch_adj_local_next<T, kTileNodes>(w, a, st)
                                         : launch_adj_local_next<T, kTileNodesSmall>(w, a, st);
    else
        rc = w->tile_nodes == kTileNodes ? launch_adj_local<T, kTileNodes>(w, a, st)
                                         : launch_adj_local<T, kTileNodesSmall>(w, a, st);
    if (rc) return rc;
    const int tgrid = (int)std::max<int64_t>(1, std::min<int64_t>((w->N + kPullThreads - 1) / kPullThreads, INT32_MAX));
    adj_transpose_kernel<T><<<tgrid, kPullThreads, 0, st>>>(a);
    grad_finalize_kernel<<<w->nseg, kThreads, 0, st>>>(w->d_tiles, w->ntiles, a.partials, grad);
    return cuda_check_step(cudaGetLastError(), "adjoint launch");
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" {

int mlbm_adjoint_step(const mlbm_weights *w, const mlbm_params *params, int dtype,
                      const void *s_prev, const void *s_next, const void *lam_next, void *lam_prev,
                      double *grad, void *stream) {
    set_error("");
    if (!w || !params || !s_prev || !lam_next || !lam_prev || !grad) return fail(MLBM_EINVAL, "NULL argument");
    if (lam_next == lam_prev) return fail(MLBM_EINVAL, "lam_next and lam_prev must not alias");
    if (s_next == lam_prev) return fail(MLBM_EINVAL, "s_next and lam_prev must not alias");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    if (w->any_nearest)
        return fail(MLBM_EINVAL, "the adjoint step supports own-stencil segments only (MLBM_STENCIL_OWN)");
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(wm, params, st))) return rc;
    if ((rc = ensure_adj_scratch(wm))) return rc;
    // fhat from s_next only where 1 - 1/tau keeps it recoverable (see the top of this file)
    for (int s = 0; s < w->nseg && s_next; ++s)
        if (!(std::fabs(1.0 - 1.0 / params[s].tau) >= 1.0 / 16)) s_next = nullptr;
    return dtype == MLBM_F32 ? adjoint_step_t<float>(wm, s_prev, s_next, lam_next, lam_prev, grad, st)
                             : adjoint_step_t<double>(wm, s_prev, s_next, lam_next, lam_prev, grad, st);
}

int mlbm_moments_adjoint(const mlbm_weights *w, const mlbm_params *params, int dtype,
                         const void *f, const double *drho, const double *dux,
                         const double *duy, void *lam, double *grad, void *stream) {
    set_error("");
    if (!w || !f || !drho || !dux || !duy || !lam || !grad) return fail(MLBM_EINVAL, "NULL argument");
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "bad dtype");
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = set_params(wm, params, st);
    if (rc) return rc;
    if ((rc = ensure_adj_scratch(wm))) return rc;
    double *partials = (double *)((char *)wm->d_scratch + sizeof(double) * 8 * (size_t)w->N);
    if (dtype == MLBM_F32)
        moments_adjoint_kernel<float><<<grid_of(w, (const void *)moments_adjoint_kernel<float>), kThreads, 0, st>>>(
            w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params, (const float *)f, drho, dux, duy, (float *)lam,
            partials, w->N);
    else
        moments_adjoint_kernel<double><<<grid_of(w, (const void *)moments_adjoint_kernel<double>), kThreads, 0, st>>>(
            w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params, (const double *)f, drho, dux, duy,
            (double *)lam, partials, w->N);
    grad_finalize_kernel<<<w->nseg, kThreads, 0, st>>>(w->d_tiles, w->ntiles, partials, grad);
    return cuda_check_step(cudaGetLastError(), "moments adjoint launch");
}

int mlbm_init_adjoint(const mlbm_weights *w, const mlbm_params *params, int dtype,
                      const double *rho, const double *ux, const double *uy, const void *lam0,
                      double *drho, double *dux, double *duy, double *grad, void *stream) {
    set_error("");
    if (!w || !rho || !ux || !uy || !lam0 || !drho || !dux || !duy || !grad)
        return fail(MLBM_EINVAL, "NULL argument");
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "bad dtype");
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = set_params(wm, params, st);
    if (rc) return rc;
    if ((rc = ensure_adj_scratch(wm))) return rc;
    double *partials = (double *)((char *)wm->d_scratch + sizeof(double) * 8 * (size_t)w->N);
    if (dtype == MLBM_F32)
        init_adjoint_kernel<float><<<grid_of(w, (const void *)init_adjoint_kernel<float>), kThreads, 0, st>>>(
            w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, rho, ux, uy, (const float *)lam0, drho, dux, duy, partials,
            w->N);
    else
        init_adjoint_kernel<double><<<grid_of(w, (const void *)init_adjoint_kernel<double>), kThreads, 0, st>>>(
            w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, rho, ux, uy, (const double *)lam0, drho, dux, duy, partials,
            w->N);
    grad_finalize_kernel<<<w->nseg, kThreads, 0, st>>>(w->d_tiles, w->ntiles, partials, grad);
    return cuda_check_step(cudaGetLastError(), "init adjoint launch");
}

}  // extern "C"
