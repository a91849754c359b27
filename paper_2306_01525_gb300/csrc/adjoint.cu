// Discrete adjoint of the fused step (reverse mode of pull-stream, bounce-back, collide) and of
// the initial state and the moments, for gradients of a loss on the macroscopic fields with
// respect to tau, the body force g and the initial fields.
//
// Forward step (storage form s, lattice units): fhat = B (S s), s' = C(fhat; tau, g) with
//   S  the interpolation fhat_k(i) = sum_j W_k[j](i) s_k(s_j(L))        (Sec. 2.3), L = i under
//      the own-node rule and L = L_k(i), the node nearest to the departure point, under the
//      nearest-node rule; in the form the forward kernel evaluates it: FP64 literally, FP32 as
//      s_k(L) + sum_{j>=1} W (s_k(s_j) - s_k(L)), i.e. with centre coefficient
//      1 - sum_{j>=1} W_k[j](i)
//   B  the wall bounce-back fhat_k = fhat_k' on unknown populations      (Sec. 3)
//   C  the BGK collision with forcing                                    (eq. LBM_collision, Sec. 3)
// Reverse: mu = J_C^T lam, mut = B^T mu, lam_prev = S^T mut.  S^T is done as a pull over the
// transposed stencil (for node m, the pairs (i, j) with s_j(i) = m, the centre pair (m, 0)
// included; under the nearest-node rule, every node i whose departure-node stencil holds m
// for some direction, with a coefficient per direction), in a fixed order, so the result is
// deterministic without atomics.  Parameter gradients are reduced per tile and then per
// segment in a fixed order.
//
// J_C and dL/dtau need the moments and the non-equilibrium part of fhat.  When the caller
// passes the forward's output s' = C(fhat) they come from it: the collision keeps rho and adds
// exactly g to rho u, and s' - F - s^eq = (1 - 1/tau)(fhat - s^eq), so no shape vector is read.
// Near tau = 1 that division loses fhat (at tau = 1, s' = s^eq + F whatever fhat was), so with
// |1 - 1/tau| < 1/16 in any segment, or without s', fhat is recomputed from s with the forward's
// own tile interpolation (own-node rule only; nearest-node clouds need s').
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "d2q9_device.cuh"
#include "mlbm_internal.h"
#include "tile_interp.cuh"

namespace mlbm {

int set_params(mlbm_weights *w, const mlbm_params *params, cudaStream_t st);
int check_dtype(const mlbm_weights *w, int dtype);
int cuda_check_step(cudaError_t e, const char *what);

namespace {

constexpr int kThreads = 256;

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
    // transposed interpolation, per forward tile (see ensure_adj_tables)
    const uint16_t *__restrict__ rowp;    // [ntiles][B] the tile's rows, longest first
    const int32_t *__restrict__ rhalo;    // reverse halos (stored positions)
    const int64_t *__restrict__ roff;     // [ntiles] offset of the tile's reverse halo
    const int32_t *__restrict__ rcnt;     // [ntiles] its size
    const int64_t *__restrict__ sbeg;     // [ntiles][B/32] first entry of each 32-row slice
    const int64_t *__restrict__ cbeg;     // [ntiles][B/32] its first coefficient
    const int32_t *__restrict__ slen;     // [ntiles][B/32] entries per row of the slice
    const int32_t *__restrict__ nlen;     // [ntiles][B/32][8] nearest rule: entries per direction
    const uint16_t *__restrict__ slot;    // per entry: reverse-halo slot of the reading node
    const T *__restrict__ coef;           // own rule: per entry [8] coefficients c_kj; nearest
                                          // rule: per entry its direction's coefficient
    int64_t N;
    int ntiles;
    // per-segment reduction of the tile sums folded into the pull kernel's last CTA (nullptr:
    // grad_finalize_kernel does it); done counts finished CTAs and is left at zero
    unsigned int *done;
    double *grad;
    int nseg;
};

// Transposed collision Jacobian (with d f^eq / d(rho, u)) and transposed bounce-back at node p:
// mu = J_C^T lam at the moments (rho, u) of fhat, mut_l = [l not unknown] mu_l + [l' unknown]
// mu_l'.  Writes lam_prev_0 = mut_0 (population 0 is not interpolated), returns mut_1..8.
template <typename T>
__device__ __forceinline__ void adj_collide_node(const AdjArgs<T> &a, int64_t p, const T (&lam)[9], T rho, T ux,
                                                 T uy, T inv_tau, uint16_t mb, T (&out)[8], bool write0 = true) {
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
    if (write0) a.lam_prev[p] = mt[0];
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

// The local part from the forward's output s_next = C(fhat) at node p, no shape vector, halo or
// stencil read: rho is the moment of s_next, rho u that of s_next minus g (the forcing term adds
// exactly g), and sum_k lam_k (fhat_k - s^eq_k) = sum_k lam_k (s_next_k - F_k - s^eq_k) / (1 -
// 1/tau), with F_k = 3 omega_k e_k.g as the forward adds it.  Returns mut_1..8 in mt; with own,
// also writes lam_prev_0 and adds the node's dL/dtau and dL/dg terms.
template <typename T>
__device__ __forceinline__ void local_from_next(const AdjArgs<T> &a, int64_t p, int seg, bool own, T (&mt)[8],
                                                T &dtau, T &dg) {
    constexpr bool kDev = std::is_same<T, float>::value;
    const int64_t N = a.N;
    const T *pr = a.params + 4 * seg;
    const T inv_tau = pr[3], gm = pr[1];
    const T rho_ref = kDev ? pr[2] : T(0);
    T s[9], lam[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        s[k] = a.s_next[(int64_t)k * N + p];
        lam[k] = a.lam_next[(int64_t)k * N + p];
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
    if (own) {
        const T usq15 = T(1.5) * (ux * ux + uy * uy);
        T st = T(0), sg = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const T w3 = omega_of<T>(k) * T(3);
            const T force = w3 * (T(ex_of(k)) * gx + T(ey_of(k)) * gy);
            st += lam[k] * ((s[k] - force) - geq_of<T>(k, drho, rho, ux, uy, usq15));
            sg += lam[k] * w3 * (T(ex_of(k)) * fx + T(ey_of(k)) * fy);
        }
        dtau += st * (inv_tau * inv_tau / (T(1) - inv_tau));
        dg += sg;
    }
    adj_collide_node<T>(a, p, lam, rho, ux, uy, inv_tau, mb, mt, own);
}

// Four consecutive coefficients (16-byte aligned in FP32, two 16-byte loads in FP64), streamed.
__device__ __forceinline__ void load4(float (&c)[4], const float *p) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    c[0] = v.x;
    c[1] = v.y;
    c[2] = v.z;
    c[3] = v.w;
}
__device__ __forceinline__ void load4(double (&c)[4], const double *p) {
    const double2 v0 = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    c[0] = v0.x;
    c[1] = v0.y;
    c[2] = v1.x;
    c[3] = v1.y;
}

// acc += w * m component-wise
__device__ __forceinline__ void vfma_acc(float4 &acc, const float4 w, const float4 m) {
    acc.x = fmaf(w.x, m.x, acc.x);
    acc.y = fmaf(w.y, m.y, acc.y);
    acc.z = fmaf(w.z, m.z, acc.z);
    acc.w = fmaf(w.w, m.w, acc.w);
}
__device__ __forceinline__ void vfma_acc(double2 &acc, const double2 w, const double2 m) {
    acc.x = fma(w.x, m.x, acc.x);
    acc.y = fma(w.y, m.y, acc.y);
}

// The transposed interpolation, tile by tile on the forward's tiles (B rows per CTA):
//   1. the cotangents mut of the tile's reverse halo (its own nodes, then every other node whose
//      stencil holds one of them) are staged in shared memory as [slot][8]: with kFromNext
//      computed there from s_next and lam_next (own nodes also give lam_prev_0 and the
//      parameter-gradient terms), otherwise read from the node-major buffer adj_local_kernel
//      wrote;
//   2. row m (thread b handles the tile's b-th longest row) sums c_kj(i) mut_k(i) over its
//      entries (i, j), s_j(i) = m, in its fixed order (j-major: the centre entry (m, 0) first):
//      lam_prev_k(m), k = 1..8.  c_kj is the coefficient of s_k(s_j(i)) in the forward's
//      fhat_k(i): W_k[j](i), except the centre of the FP32 difference form, 1 - sum_{j>=1}
//      W_k[j](i).  The entries are sliced by 32 rows (entry e of the slice's lane l at
//      sbeg + 32 e + l, rows padded to the slice's longest with slot 0 and zero coefficients;
//      the coefficients in planes, vector q of the 32 lanes' entries contiguous), so every
//      warp load is a contiguous run, and the gathered cotangents come from shared memory.
//      Nearest-node tiles: the cotangents are staged direction-major ([k][slot]) and each row
//      sums, direction by direction, its (slot, coefficient) entries, four per lane contiguous;
//   3. with the per-segment reduction folded in (a.done), the last CTA to finish adds every
//      segment's tile sums to grad in a fixed order.
//      No atomics in the sums: deterministic.
template <typename T, int B, bool kFromNext>
__global__ void __launch_bounds__(B) adj_pull_kernel(AdjArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *sh = reinterpret_cast<VT *>(smem_raw);  // [U][NV]
    __shared__ double red[2][B / 32];
    const int64_t N = a.N;
    const int b = threadIdx.x;
    T *shs = reinterpret_cast<T *>(smem_raw);  // nearest rule: [8][U], direction-major
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        const bool nearest = tile.mode == MLBM_STENCIL_NEAREST;
        const int U = a.rcnt[t];
        const int32_t *__restrict__ rh = a.rhalo + a.roff[t];
        T dtau = T(0), dg = T(0);
        // the next iteration's halo index is loaded one iteration ahead (its latency overlaps the
        // current node's loads)
        int32_t node_next = b < U ? rh[b] : 0;
        for (int u = b; u < U; u += B) {
            const int64_t node = node_next;
            if (u + B < U) node_next = rh[u + B];
            T mt[8];
            if constexpr (kFromNext) {
                local_from_next<T>(a, node, tile.seg, u < tile.count, mt, dtau, dg);
            } else {
                const VT *mi = reinterpret_cast<const VT *>(a.mut + node * 8);
#pragma unroll
                for (int q = 0; q < NV; ++q) vunpack(mt + q * W, mi[q]);
            }
            if (nearest) {
#pragma unroll
                for (int k = 0; k < 8; ++k) shs[k * U + u] = mt[k];
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) vpack(sh[u * NV + q], mt + q * W);
            }
        }
        __syncthreads();
        if (nearest && b < tile.count) {
            // the slice's entries direction by direction, each a (slot, coefficient) pair: row m
            // sums c(i) mut_k(i) over the nodes i whose departure-node stencil for k holds m
            const int64_t m = tile.begin + a.rowp[(int64_t)t * B + b];
            const int ws = t * (B / 32) + (b >> 5);
            const int32_t *__restrict__ nl = a.nlen + (int64_t)ws * 8;
            // quads of entries: four slots in one 8-byte word, four coefficients contiguous
            const uint2 *__restrict__ sp = reinterpret_cast<const uint2 *>(a.slot + a.sbeg[ws]) + (b & 31);
            const T *__restrict__ cp = a.coef + a.cbeg[ws] + 4 * (b & 31);
#pragma unroll 1
            for (int k = 0; k < 8; ++k) {
                const int L4 = nl[k] >> 2;
                const T *__restrict__ sk = shs + k * U;
                T acc = T(0);
                int e = 0;
                for (; e + 1 < L4; e += 2) {  // two quads per pass
                    const uint2 s0 = __ldcs(sp + 32 * e), s1 = __ldcs(sp + 32 * (e + 1));
                    T c0[4], c1[4];
                    load4(c0, cp + 128 * e);
                    load4(c1, cp + 128 * (e + 1));
                    acc = fma(c0[0], sk[s0.x & 0xFFFFu], acc);
                    acc = fma(c0[1], sk[s0.x >> 16], acc);
                    acc = fma(c0[2], sk[s0.y & 0xFFFFu], acc);
                    acc = fma(c0[3], sk[s0.y >> 16], acc);
                    acc = fma(c1[0], sk[s1.x & 0xFFFFu], acc);
                    acc = fma(c1[1], sk[s1.x >> 16], acc);
                    acc = fma(c1[2], sk[s1.y & 0xFFFFu], acc);
                    acc = fma(c1[3], sk[s1.y >> 16], acc);
                }
                if (e < L4) {
                    const uint2 s0 = __ldcs(sp + 32 * e);
                    T c0[4];
                    load4(c0, cp + 128 * e);
                    acc = fma(c0[0], sk[s0.x & 0xFFFFu], acc);
                    acc = fma(c0[1], sk[s0.x >> 16], acc);
                    acc = fma(c0[2], sk[s0.y & 0xFFFFu], acc);
                    acc = fma(c0[3], sk[s0.y >> 16], acc);
                }
                a.lam_prev[(int64_t)(k + 1) * N + m] = acc;
                sp += (int64_t)32 * L4;
                cp += (int64_t)128 * L4;
            }
        } else if (b < tile.count) {
            const int64_t m = tile.begin + a.rowp[(int64_t)t * B + b];
            const int ws = t * (B / 32) + (b >> 5);
            const int L = a.slen[ws];
            const int64_t q0 = a.sbeg[ws] + (b & 31);
            const uint16_t *__restrict__ sp = a.slot + q0;
            // coefficients in planes per 32-entry row of the slice: vector q of entry (e, lane)
            // at cbeg / W + 32 e NV + 32 q + lane, so each warp load is 512 contiguous bytes
            const VT *__restrict__ cp = reinterpret_cast<const VT *>(a.coef + a.cbeg[ws]) + (b & 31);
            VT acc[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) vzero(acc[q]);
            // kE entries per pass: their slots and coefficients are loaded before any is used.
            // Eight when the cotangents come from s_next, four when they are read from the
            // node-major buffer (the widths that measured fastest on each route)
            constexpr int kE = kFromNext ? 8 : 4;
            int e = 0;
            for (; e + kE - 1 < L; e += kE) {
                int sl[kE];
                VT c[kE][NV];
#pragma unroll
                for (int r = 0; r < kE; ++r) {
                    sl[r] = sp[(int64_t)32 * (e + r)];
#pragma unroll
                    for (int q = 0; q < NV; ++q) c[r][q] = __ldcs(cp + ((int64_t)32 * (e + r)) * NV + 32 * q);
                }
#pragma unroll
                for (int r = 0; r < kE; ++r)
#pragma unroll
                    for (int q = 0; q < NV; ++q) vfma_acc(acc[q], c[r][q], sh[sl[r] * NV + q]);
            }
            for (; e < L; ++e) {
                const int s0 = sp[(int64_t)32 * e];
#pragma unroll
                for (int q = 0; q < NV; ++q) vfma_acc(acc[q], __ldcs(cp + ((int64_t)32 * e) * NV + 32 * q), sh[s0 * NV + q]);
            }
            T v[8];
#pragma unroll
            for (int q = 0; q < NV; ++q) vunpack(v + q * W, acc[q]);
#pragma unroll
            for (int k = 0; k < 8; ++k) a.lam_prev[(int64_t)(k + 1) * N + m] = v[k];
        }
        if constexpr (kFromNext)
            tile_partials<T, B>(dtau, dg, red, a.partials, t);
        else
            __syncthreads();
    }
    if constexpr (kFromNext) {
        if (a.done) {
            // the last CTA to finish adds every segment's tile sums to grad: per thread the tiles
            // t = tid, tid + B, ... in order, then the warps' shuffle trees, then the warps in
            // order (a fixed order whichever CTA is last)
            __shared__ int last;
            if (threadIdx.x == 0) {
                __threadfence();
                last = atomicAdd(a.done, 1u) == gridDim.x - 1;
            }
            __syncthreads();
            if (last) {
                __threadfence();
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                for (int sg = 0; sg < a.nseg; ++sg) {
                    double s0 = 0.0, s1 = 0.0;
                    // the running gradient is read before the tile sums (its latency overlaps theirs)
                    double2 g_old = make_double2(0.0, 0.0);
                    if (threadIdx.x == 0) g_old = make_double2(__ldcg(a.grad + 2 * sg), __ldcg(a.grad + 2 * sg + 1));
                    // eight tiles' segments and sums loaded before any is added (one memory
                    // latency per eight tiles, not two per tile)
                    for (int t0 = threadIdx.x; t0 < a.ntiles; t0 += 8 * B) {
                        int sgv[8];
                        double2 pv[8];
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const int t = t0 + r * B;
                            sgv[r] = t < a.ntiles ? a.tiles[t].seg : -1;
                            pv[r] = t < a.ntiles ? __ldcg(reinterpret_cast<const double2 *>(a.partials) + t)
                                                 : make_double2(0.0, 0.0);
                        }
#pragma unroll
                        for (int r = 0; r < 8; ++r)
                            if (sgv[r] == sg) {
                                s0 += pv[r].x;
                                s1 += pv[r].y;
                            }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                    }
                    if (lane == 0) {
                        red[0][warp] = s0;
                        red[1][warp] = s1;
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double g0 = 0.0, g1 = 0.0;
                        for (int q = 0; q < B / 32; ++q) {
                            g0 += red[0][q];
                            g1 += red[1][q];
                        }
                        a.grad[2 * sg] = g_old.x + g0;
                        a.grad[2 * sg + 1] = g_old.y + g1;
                    }
                    __syncthreads();
                }
                if (threadIdx.x == 0) *a.done = 0u;
            }
        }
    }
}

// Coefficients of the sliced entry table: thread (t, b) fills the entries of the tile's b-th
// row m (slice b / 32, lane b % 32).  The entry at position q reads node i = src[q], and m is
// member j = jh[q] of the stencil that interpolates (i, k): the coefficient with which f_k(m)
// enters fhat_k(i) is c_kj(i) = W_k[j](i) in the step's precision (FP32: the rounded canonical
// FP32 shape vectors the forward's FP32 layout is made of), except the FP32 difference form's
// centre, 1 - sum_{j>=1} W_k[j](i) added up in member order as the forward does.  Own-node
// rule: all eight directions share the entry (m is member j of i's own stencil), coefficients
// in planes after cbeg.  Nearest-node rule: the slice's entries run direction by direction
// (nlen per direction, in quads of four entries per lane), one coefficient each at
// cbeg + (q - sbeg).  Padding (src -1) gets zeros.
template <typename T>
__device__ __forceinline__ T adj_coef_of(const SegDev &sd, const double *__restrict__ w64c,
                                         const float *__restrict__ w32c, int64_t i, int k, int j) {
    constexpr bool kDev = std::is_same<T, float>::value;
    const int64_t base = sd.w_off + (int64_t)k * sd.K * sd.n + i;
    if (!kDev) return (T)w64c[base + (int64_t)j * sd.n];
    if (j > 0) return (T)w32c[base + (int64_t)j * sd.n];
    float wsum = 0.f;
    for (int jj = 1; jj < sd.K; ++jj) wsum += w32c[base + (int64_t)jj * sd.n];
    return (T)(1.f - wsum);
}

template <typename T>
__global__ void adj_coef_kernel(const TileDev *__restrict__ tiles, int ntiles, int B, const SegDev *__restrict__ seg,
                                const int64_t *__restrict__ sbeg, const int64_t *__restrict__ cbeg,
                                const int32_t *__restrict__ slen, const int32_t *__restrict__ nlen,
                                const int32_t *__restrict__ srcs, const int8_t *__restrict__ jhs,
                                const double *__restrict__ w64c, const float *__restrict__ w32c,
                                T *__restrict__ coef) {
    constexpr int W = V<T>::width, NV = 8 / W;
    const int64_t total = (int64_t)ntiles * B;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(g / B), b = (int)(g - (int64_t)t * B);
        const TileDev tile = tiles[t];
        const int ws = t * (B / 32) + (b >> 5);
        const int L = slen[ws];
        if (L == 0) continue;
        const SegDev sd = seg[tile.seg];
        const int lane = b & 31;
        if (tile.mode == MLBM_STENCIL_NEAREST) {
            int64_t kb = sbeg[ws];
            for (int k = 0; k < 8; ++k) {
                const int Lk = nlen[(int64_t)ws * 8 + k];
                for (int e = 0; e < Lk; ++e) {
                    const int64_t q = kb + 128 * (e >> 2) + 4 * lane + (e & 3);
                    const int32_t src = b < tile.count ? srcs[q] : -1;
                    coef[cbeg[ws] + (q - sbeg[ws])] =
                        src >= 0 ? adj_coef_of<T>(sd, w64c, w32c, src - sd.off, k, jhs[q]) : T(0);
                }
                kb += (int64_t)32 * Lk;
            }
            continue;
        }
        for (int e = 0; e < L; ++e) {
            const int64_t q = sbeg[ws] + (int64_t)32 * e + lane;
            const int32_t src = b < tile.count ? srcs[q] : -1;
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = src >= 0 ? adj_coef_of<T>(sd, w64c, w32c, src - sd.off, k, jhs[q]) : T(0);
            // planes: vector h (directions h W .. h W + W - 1) of the lane at cbeg + (32 e NV + 32 h + lane) W
#pragma unroll
            for (int k = 0; k < 8; ++k) coef[cbeg[ws] + ((int64_t)32 * e * NV + 32 * (k / W) + lane) * W + k % W] = v[k];
        }
    }
}

// grad[2 s + c] += sum over tiles of segment s of partials[2 t + c], in a fixed order (thread
// tid adds tiles tid, tid + 1024, ...; then a tree over the threads).  The tile's segment and
// its partial sums are loaded together, so each pass costs one memory latency.
constexpr int kFinalizeThreads = 1024;
constexpr int kFoldSegments = 8;  // up to this many segments the pull kernel reduces the tile sums
__global__ void __launch_bounds__(kFinalizeThreads) grad_finalize_kernel(const TileDev *__restrict__ tiles, int ntiles,
                                                                          const double *__restrict__ partials,
                                                                          double *__restrict__ grad) {
    __shared__ double sh[2][kFinalizeThreads];
    const int s = blockIdx.x, tid = threadIdx.x;
    double a0 = 0.0, a1 = 0.0;
    for (int t = tid; t < ntiles; t += kFinalizeThreads) {
        const int sg = tiles[t].seg;
        const double p0 = partials[2 * t], p1 = partials[2 * t + 1];
        if (sg == s) {
            a0 += p0;
            a1 += p1;
        }
    }
    sh[0][tid] = a0;
    sh[1][tid] = a1;
    __syncthreads();
    for (int h = kFinalizeThreads / 2; h > 0; h >>= 1) {
        if (tid < h) {
            sh[0][tid] += sh[0][tid + h];
            sh[1][tid] += sh[1][tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        grad[2 * s] += sh[0][0];
        grad[2 * s + 1] += sh[1][0];
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

// Scratch of the reverse step: node-major cotangents [N][8] (8 doubles per node at most), the
// per-tile gradient sums [ntiles][2], then the finished-CTA counter of the pull kernel (zeroed
// here, left at zero by each launch).
size_t adj_done_offset(const mlbm_weights *w) { return sizeof(double) * (8 * (size_t)w->N + 2 * (size_t)w->ntiles); }

int ensure_adj_scratch(mlbm_weights *w) {
    size_t need = adj_done_offset(w) + 16;
    if (w->d_scratch && w->scratch_bytes >= need) return MLBM_OK;
    cudaFree(w->d_scratch);
    w->d_scratch = nullptr;
    cudaError_t e = cudaMalloc(&w->d_scratch, need);
    if (e == cudaSuccess) e = cudaMemset((char *)w->d_scratch + adj_done_offset(w), 0, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w->d_scratch);
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

template <typename V_>
int upload_vec(V_ **dst, const std::vector<V_> &v, const char *what) {
    if (cudaMalloc(dst, sizeof(V_) * std::max<size_t>(1, v.size())) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return fail(MLBM_ENOMEM, std::string(what) + " allocation failed");
    }
    return cuda_check_step(cudaMemcpy(*dst, v.data(), sizeof(V_) * v.size(), cudaMemcpyHostToDevice), what);
}

// Tables of the transposed interpolation, per forward tile (host arithmetic on the downloaded
// tile table and transposed stencil): the tile's rows ordered by entry count, longest first
// (stable), so that the 32 rows of a slice have similar lengths; its reverse halo (own nodes in
// order, then every other reading node, sorted); per 32-row slice the entry count of its longest
// row and the slice's first entry; per entry the reading node's reverse-halo slot (0 for
// padding).  Then the coefficients of the dtype, in a kernel.
template <typename T>
int ensure_adj_tables(mlbm_weights *w, cudaStream_t st) {
    int rc = MLBM_OK;
    const int B = w->tile_nodes, WPT = B / 32, nt = w->ntiles;
    if (!w->d_adj_slot) {
        std::vector<TileDev> tiles((size_t)nt);
        std::vector<int32_t> ptr((size_t)w->N + 1), ent((size_t)w->idx_total);
        if ((rc = cuda_check_step(cudaMemcpy(tiles.data(), w->d_tiles, sizeof(TileDev) * tiles.size(),
                                             cudaMemcpyDeviceToHost), "tile table")) ||
            (rc = cuda_check_step(cudaMemcpy(ptr.data(), w->d_csr_ptr, sizeof(int32_t) * ptr.size(),
                                             cudaMemcpyDeviceToHost), "transposed stencil")) ||
            (rc = cuda_check_step(cudaMemcpy(ent.data(), w->d_csr_ent, sizeof(int32_t) * ent.size(),
                                             cudaMemcpyDeviceToHost), "transposed stencil")))
            return rc;
        // nearest-node segments: which nodes depart to each node, per direction (inverse of the
        // departure map), [seg] -> per direction k: offsets [n + 1] and readers
        std::vector<int32_t> near;
        std::vector<std::vector<std::vector<int32_t>>> inv_ptr(w->nseg), inv_ent(w->nseg);
        if (w->any_nearest) {
            near.resize((size_t)8 * w->N);
            if ((rc = cuda_check_step(cudaMemcpy(near.data(), w->d_near, sizeof(int32_t) * near.size(),
                                                 cudaMemcpyDeviceToHost), "departure nodes")))
                return rc;
            for (int sg = 0; sg < w->nseg; ++sg) {
                const SegmentHost &h = w->seg[sg];
                if (h.d.stencil_mode != MLBM_STENCIL_NEAREST) continue;
                inv_ptr[sg].assign(8, {});
                inv_ent[sg].assign(8, {});
                for (int k = 0; k < 8; ++k) {
                    const int32_t *nk = &near[(size_t)8 * h.off + (size_t)k * h.n];
                    std::vector<int32_t> &pt = inv_ptr[sg][k], &en = inv_ent[sg][k];
                    pt.assign((size_t)h.n + 1, 0);
                    for (int64_t i = 0; i < h.n; ++i) pt[nk[i] - h.off + 1]++;
                    for (int64_t L = 0; L < h.n; ++L) pt[L + 1] += pt[L];
                    en.resize((size_t)h.n);
                    std::vector<int32_t> fill(pt.begin(), pt.end() - 1);
                    for (int64_t i = 0; i < h.n; ++i) en[fill[nk[i] - h.off]++] = (int32_t)(h.off + i);
                }
            }
        }
        std::vector<uint16_t> rowp((size_t)nt * B, 0);
        std::vector<int32_t> slen((size_t)nt * WPT, 0);
        std::vector<int32_t> nlen((size_t)nt * WPT * 8, 0);  // nearest-rule slices: entries per direction
        std::vector<std::vector<int32_t>> rh(nt);
        std::vector<std::vector<uint16_t>> sl(nt);
        std::vector<std::vector<int32_t>> ps(nt);  // per tile, per position: reading node (-1 padding)
        std::vector<std::vector<int8_t>> pj(nt);   // per tile, per position: member index
        std::vector<int> bad(nt, 0);
        auto work = [&](int t0, int t1) {
            std::vector<int32_t> others;
            std::vector<int> ord;
            std::vector<std::vector<int32_t>> rs;  // per row of the tile: reading nodes
            std::vector<std::vector<int8_t>> rj;   // and member indices
            std::vector<std::array<int32_t, 9>> rk;  // nearest rule: start of direction k's readers in rs
            std::vector<std::pair<int32_t, int8_t>> tmp;
            for (int t = t0; t < t1; ++t) {
                const TileDev &T_ = tiles[t];
                const SegmentHost &h = w->seg[T_.seg];
                const bool nearest = h.d.stencil_mode == MLBM_STENCIL_NEAREST;
                const int64_t m0 = T_.begin;
                rs.assign(T_.count, {});
                rj.assign(T_.count, {});
                rk.assign(T_.count, {});
                for (int b = 0; b < T_.count; ++b) {
                    const int64_t m = m0 + b;
                    std::vector<int32_t> &R = rs[b];
                    if (!nearest) {  // the transposed stencil's entries (i, j), j-major: centre first
                        for (int32_t q = ptr[m]; q < ptr[m + 1]; ++q) {
                            R.push_back((int32_t)(h.off + ent[q] % h.n));
                            rj[b].push_back((int8_t)(ent[q] / h.n));
                        }
                    } else {
                        // per direction k, the nodes i whose departure node L_k(i) has m in its
                        // stencil (as member j), by increasing i: each i at most once per direction
                        for (int k = 0; k < 8; ++k) {
                            rk[b][k] = (int32_t)R.size();
                            tmp.clear();
                            for (int32_t q = ptr[m]; q < ptr[m + 1]; ++q) {
                                const int64_t L = ent[q] % h.n;
                                const int8_t j = (int8_t)(ent[q] / h.n);
                                for (int32_t r = inv_ptr[T_.seg][k][L]; r < inv_ptr[T_.seg][k][L + 1]; ++r)
                                    tmp.emplace_back(inv_ent[T_.seg][k][r], j);
                            }
                            std::sort(tmp.begin(), tmp.end());
                            for (auto &e : tmp) {
                                R.push_back(e.first);
                                rj[b].push_back(e.second);
                            }
                        }
                        rk[b][8] = (int32_t)R.size();
                    }
                }
                ord.resize(T_.count);
                for (int b = 0; b < T_.count; ++b) ord[b] = b;
                std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return rs[x].size() > rs[y].size(); });
                others.clear();
                for (int b = 0; b < T_.count; ++b) {
                    rowp[(size_t)t * B + b] = (uint16_t)ord[b];
                    for (int32_t s_ : rs[b])
                        if (s_ < m0 || s_ >= m0 + T_.count) others.push_back(s_);
                }
                std::sort(others.begin(), others.end());
                others.erase(std::unique(others.begin(), others.end()), others.end());
                if ((int64_t)T_.count + (int64_t)others.size() > 65535) {
                    bad[t] = 1;
                    continue;
                }
                std::vector<int32_t> &RH = rh[t];
                RH.resize((size_t)T_.count + others.size());
                for (int b = 0; b < T_.count; ++b) RH[b] = (int32_t)(m0 + b);
                std::copy(others.begin(), others.end(), RH.begin() + T_.count);
                auto slot_of = [&](int32_t s_) -> uint16_t {
                    if (s_ >= m0 && s_ < m0 + T_.count) return (uint16_t)(s_ - m0);
                    return (uint16_t)(T_.count + (std::lower_bound(others.begin(), others.end(), s_) - others.begin()));
                };
                // slices of 32 rows: entry e of lane l at position 32 e + l; under the nearest
                // rule the directions follow one another, each padded to the slice's longest
                // rounded up to a multiple of 4, entry e of lane l at 128 (e / 4) + 4 l + e % 4
                // (four consecutive entries of a lane are one 8-byte slot load and one
                // 16-byte FP32 coefficient load)
                int64_t n_ent = 0;
                for (int ws = 0; ws < WPT; ++ws) {
                    int L = 0;
                    if (!nearest) {
                        for (int l = 0; l < 32 && 32 * ws + l < T_.count; ++l)
                            L = std::max(L, (int)rs[ord[32 * ws + l]].size());
                    } else {
                        for (int k = 0; k < 8; ++k) {
                            int Lk = 0;
                            for (int l = 0; l < 32 && 32 * ws + l < T_.count; ++l) {
                                const int r = ord[32 * ws + l];
                                Lk = std::max(Lk, rk[r][k + 1] - rk[r][k]);
                            }
                            Lk = (Lk + 3) & ~3;  // whole quads
                            nlen[((size_t)t * WPT + ws) * 8 + k] = Lk;
                            L += Lk;
                        }
                    }
                    slen[(size_t)t * WPT + ws] = L;
                    n_ent += 32 * (int64_t)L;
                }
                std::vector<uint16_t> &S = sl[t];
                S.assign((size_t)n_ent, 0);
                ps[t].assign((size_t)n_ent, -1);
                pj[t].assign((size_t)n_ent, (int8_t)-1);
                int64_t base = 0;
                for (int ws = 0; ws < WPT; ++ws) {
                    const int L = slen[(size_t)t * WPT + ws];
                    for (int l = 0; l < 32 && 32 * ws + l < T_.count; ++l) {
                        const int r = ord[32 * ws + l];
                        if (!nearest) {
                            for (size_t e = 0; e < rs[r].size(); ++e) {
                                const int64_t q = base + 32 * (int64_t)e + l;
                                S[q] = slot_of(rs[r][e]);
                                ps[t][q] = rs[r][e];
                                pj[t][q] = rj[r][e];
                            }
                        } else {
                            int64_t kb = base;
                            for (int k = 0; k < 8; ++k) {
                                for (int32_t e = rk[r][k]; e < rk[r][k + 1]; ++e) {
                                    const int32_t ee = e - rk[r][k];  // quad ee / 4, lane l, place ee % 4
                                    const int64_t q = kb + 128 * (int64_t)(ee >> 2) + 4 * l + (ee & 3);
                                    S[q] = slot_of(rs[r][e]);
                                    ps[t][q] = rs[r][e];
                                    pj[t][q] = rj[r][e];
                                }
                                kb += 32 * (int64_t)nlen[((size_t)t * WPT + ws) * 8 + k];
                            }
                        }
                    }
                    base += 32 * (int64_t)L;
                }
            }
        };
        {
            unsigned hw = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
            std::vector<std::thread> th;
            const int chunk = (nt + (int)hw - 1) / (int)hw;
            for (int t0 = 0; t0 < nt; t0 += chunk) th.emplace_back(work, t0, std::min(nt, t0 + chunk));
            for (auto &x : th) x.join();
        }
        for (int t = 0; t < nt; ++t)
            if (bad[t]) return fail(MLBM_EINVAL, "a tile's reverse halo exceeds 65535 nodes (stencils too spread out)");
        // coefficients: eight per position of an own-rule slice (planes), one per position of
        // a nearest-rule slice (its direction's)
        std::vector<int64_t> roff((size_t)nt), sbeg((size_t)nt * WPT), cbeg((size_t)nt * WPT);
        std::vector<int32_t> rcnt((size_t)nt), rall, srcs;
        std::vector<uint16_t> slots;
        std::vector<int8_t> jhs;
        int rmax = 0;
        int64_t cbase = 0;
        for (int t = 0; t < nt; ++t) {
            roff[t] = (int64_t)rall.size();
            rcnt[t] = (int32_t)rh[t].size();
            rmax = std::max(rmax, rcnt[t]);
            rall.insert(rall.end(), rh[t].begin(), rh[t].end());
            int64_t base = (int64_t)slots.size();
            const bool nearest = tiles[t].mode == MLBM_STENCIL_NEAREST;
            for (int ws = 0; ws < WPT; ++ws) {
                sbeg[(size_t)t * WPT + ws] = base;
                cbeg[(size_t)t * WPT + ws] = cbase;
                base += 32 * (int64_t)slen[(size_t)t * WPT + ws];
                cbase += 32 * (int64_t)slen[(size_t)t * WPT + ws] * (nearest ? 1 : 8);
            }
            slots.insert(slots.end(), sl[t].begin(), sl[t].end());
            srcs.insert(srcs.end(), ps[t].begin(), ps[t].end());
            jhs.insert(jhs.end(), pj[t].begin(), pj[t].end());
            std::vector<int32_t>().swap(rh[t]);
            std::vector<uint16_t>().swap(sl[t]);
            std::vector<int32_t>().swap(ps[t]);
            std::vector<int8_t>().swap(pj[t]);
        }
        w->adj_positions = (int64_t)slots.size();
        w->adj_coefs = cbase;
        w->adj_rmax = rmax;
        if ((rc = upload_vec(&w->d_adj_rowp, rowp, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_rhalo, rall, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_roff, roff, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_rcnt, rcnt, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_sbeg, sbeg, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_cbeg, cbeg, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_slen, slen, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_nlen, nlen, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_slot, slots, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_src, srcs, "adjoint tables")) ||
            (rc = upload_vec(&w->d_adj_jh, jhs, "adjoint tables")))
            return rc;
    }
    const int i = std::is_same<T, float>::value ? 0 : 1;
    if (w->d_adj_coef[i]) return MLBM_OK;
    if (i == 0 && !w->d_w32c) return fail(MLBM_EINVAL, "weights built without MLBM_KEEP_W32");
    if (cudaMalloc(&w->d_adj_coef[i], sizeof(T) * (size_t)std::max<int64_t>(1, w->adj_coefs)) != cudaSuccess) {
        cudaGetLastError();
        w->d_adj_coef[i] = nullptr;
        return fail(MLBM_ENOMEM, "adjoint table allocation failed");
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nt * B + 255) / 256, 65536));
    adj_coef_kernel<T><<<grid, 256, 0, st>>>(w->d_tiles, nt, B, w->d_seg, w->d_adj_sbeg, w->d_adj_cbeg, w->d_adj_slen,
                                             w->d_adj_nlen, w->d_adj_src, w->d_adj_jh, w->d_w64, w->d_w32c,
                                             (T *)w->d_adj_coef[i]);
    return cuda_check_step(cudaGetLastError(), "adjoint table launch");
}

template <typename T, int B>
int launch_adj_local(mlbm_weights *w, const AdjArgs<T> &a, cudaStream_t st) {
    const size_t smem = (size_t)w->umax * 8 * sizeof(T);
    const void *fn = (const void *)adj_local_kernel<T, B>;
    int rc = allow_dynamic_smem(fn);
    if (rc) return rc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, B, smem);
    if (per_sm < 1) return fail(MLBM_EINVAL, "a tile's halo does not fit in shared memory for the adjoint");
    const int grid = std::max(1, std::min(w->ntiles, per_sm * w->num_sms));
    adj_local_kernel<T, B><<<grid, B, smem, st>>>(a);
    return MLBM_OK;
}

template <typename T, int B, bool kFromNext>
int launch_adj_pull(mlbm_weights *w, const AdjArgs<T> &a, cudaStream_t st) {
    const size_t smem = (size_t)w->adj_rmax * 8 * sizeof(T);
    const void *fn = (const void *)adj_pull_kernel<T, B, kFromNext>;
    int rc = allow_dynamic_smem(fn);
    if (rc) return rc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, B, smem);
    if (per_sm < 1) return fail(MLBM_EINVAL, "a tile's reverse halo does not fit in shared memory for the adjoint");
    const int grid = std::max(1, std::min(w->ntiles, per_sm * w->num_sms));
    adj_pull_kernel<T, B, kFromNext><<<grid, B, smem, st>>>(a);
    return MLBM_OK;
}

template <typename T, int B>
int launch_reverse(mlbm_weights *w, const AdjArgs<T> &a, cudaStream_t st) {
    if (a.s_next) return launch_adj_pull<T, B, true>(w, a, st);
    int rc = launch_adj_local<T, B>(w, a, st);
    return rc ? rc : launch_adj_pull<T, B, false>(w, a, st);
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
    a.rowp = w->d_adj_rowp;
    a.rhalo = w->d_adj_rhalo;
    a.roff = w->d_adj_roff;
    a.rcnt = w->d_adj_rcnt;
    a.sbeg = w->d_adj_sbeg;
    a.cbeg = w->d_adj_cbeg;
    a.slen = w->d_adj_slen;
    a.nlen = w->d_adj_nlen;
    a.slot = w->d_adj_slot;
    a.coef = (const T *)w->d_adj_coef[kDev ? 0 : 1];
    a.N = w->N;
    a.ntiles = w->ntiles;
    // few segments: the pull kernel's last CTA reduces the tile sums (one launch fewer)
    const bool fold = s_next && w->nseg <= kFoldSegments;
    a.done = fold ? (unsigned int *)((char *)w->d_scratch + adj_done_offset(w)) : nullptr;
    a.grad = grad;
    a.nseg = w->nseg;
    rc = with_tile_nodes(w->tile_nodes, [&](auto Bc) { return launch_reverse<T, decltype(Bc)::value>(w, a, st); });
    if (rc) return rc;
    if (!fold) grad_finalize_kernel<<<w->nseg, kFinalizeThreads, 0, st>>>(w->d_tiles, w->ntiles, a.partials, grad);
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
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(wm, params, st))) return rc;
    if ((rc = ensure_adj_scratch(wm))) return rc;
    // fhat from s_next only where 1 - 1/tau keeps it recoverable (see the top of this file)
    for (int s = 0; s < w->nseg && s_next; ++s)
        if (!(std::fabs(1.0 - 1.0 / params[s].tau) >= 1.0 / 16)) s_next = nullptr;
    if (!s_next && w->any_nearest)
        return fail(MLBM_EINVAL, "the adjoint of nearest-node stencils needs the forward's next state (s_next) and "
                                 "|1 - 1/tau| >= 1/16 in every segment");
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
    grad_finalize_kernel<<<w->nseg, kFinalizeThreads, 0, st>>>(w->d_tiles, w->ntiles, partials, grad);
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
    grad_finalize_kernel<<<w->nseg, kFinalizeThreads, 0, st>>>(w->d_tiles, w->ntiles, partials, grad);
    return cuda_check_step(cudaGetLastError(), "init adjoint launch");
}

}  // extern "C"
