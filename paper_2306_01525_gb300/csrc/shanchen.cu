// Shan-Chen single-component multiphase extension of the meshless step.  The paper's discussion
// names this model as one whose particle interactions sit in the local collision and so carry
// over to the meshless streaming unchanged; it gives no formulas, and the model is Shan & Chen
// (1993):
//   psi(rho) = rho_psi (1 - exp(-rho / rho_psi)),
//   F(x)     = -G psi(x) sum_k omega_k psi(x + e_k dx_ml) e_k,
//   collision towards the equilibrium at the shifted velocity u + tau F / rho.
// On a node cloud the point x + e_k dx_ml is the departure point of the opposite direction, so
// psi there is interpolated with the shape vectors the streaming already holds; no new weights.
//
// A step is two passes, because the force at a node needs psi at its neighbours after they
// have streamed:
//   1. sc_stream_kernel: pull-stream (the step kernel's tile interpolation), store the streamed
//      state fhat in f_out and psi(rho of fhat) in a scratch array;
//   2. sc_collide_kernel: stage psi of the tile's halo, interpolate it at the eight departure
//      points with the same tile-layout shape vectors, form F, collide fhat in place.
// The velocity shift is applied as (s^eq(u + tau F / rho) - s^eq(u)) / tau on top of the plain
// collision (the same thing written as a difference), so the FP32 path keeps its exact mass
// and momentum projection.  Both stencil rules: under the nearest-node rule (Sec. 2.3) psi at
// the departure point of direction k is interpolated in that point's own stencil (that of its
// nearest node), with the streaming's per-direction slots and shape vectors.  Periodic segments
// only (no walls: the model needs a wall value of psi, a wetting choice, that the method leaves
// open).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
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

template <typename T>
struct ScArgs {
    const TileDev *__restrict__ tiles;
    const int32_t *__restrict__ halo;
    const uint32_t *__restrict__ lidx;
    const T *__restrict__ wt;       // tile-layout shape vectors of the step's precision
    const T *__restrict__ fdir;     // [2][N] body-force direction
    const T *__restrict__ params;   // [nseg][4] tau, g, rho0, 1/tau in T
    const T *__restrict__ sc;       // [nseg][2] G, rho_psi in T
    const T *__restrict__ fin;
    T *__restrict__ fout;
    T *__restrict__ psi;            // [N] scratch
    T *__restrict__ mom;            // optional [3][N]
    int64_t N;
    int ntiles;
};

template <typename T>
__device__ __forceinline__ T sc_exp(T x) {
    if constexpr (std::is_same<T, float>::value)
        return expf(x);
    else
        return exp(x);
}

// Values at the departure points x_b - e_k dx_ml of node b, k = 1..8 (out[k - 1]), under the
// nearest-node rule: direction k is interpolated in the stencil of its departure node, member 0
// being that node, through the per-direction halo slots ([ceil(K/2)][B][8] packed pairs) and
// the tile-layout shape vectors.  val(k, slot) reads direction k's value at a halo slot.
// Members are taken in the order, and in the forms, of the step kernel's nearest-node
// interpolation (FP32: differences to the departure node's value; FP64: the literal sum), so a
// step without interaction gives the plain step's populations bit for bit.
template <typename T, int B, typename Val>
__device__ __forceinline__ void interp_departure(const uint32_t *__restrict__ lidx, const T *__restrict__ wt,
                                                 const TileDev &tile, int b, Val val, T (&out)[8]) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    const int K = tile.K, JP = (K + 1) / 2;
    const uint4 *__restrict__ lp = reinterpret_cast<const uint4 *>(lidx + tile.l_off) + 2 * b;
    const VT *__restrict__ wbase = reinterpret_cast<const VT *>(wt + (kLiteral ? tile.w64_off : tile.w_off)) + b;
    auto slot_words = [&](int jp, uint32_t (&pr)[8]) {
        const uint4 lo = __ldcs(lp + (int64_t)jp * 2 * B), hi = __ldcs(lp + (int64_t)jp * 2 * B + 1);
        pr[0] = lo.x; pr[1] = lo.y; pr[2] = lo.z; pr[3] = lo.w;
        pr[4] = hi.x; pr[5] = hi.y; pr[6] = hi.z; pr[7] = hi.w;
    };
    T acc[8], c[8];
    {
        uint32_t pr[8];
        slot_words(0, pr);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = val(k, (int)(pr[k] & 0xFFFFu));
            acc[k] = T(0);
        }
    }
    for (int jp = 0; jp < JP; ++jp) {
        uint32_t pr[8];
        slot_words(jp, pr);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * jp + h;
            if (j >= K) break;
            if (!kLiteral && j == 0) continue;
            const VT *__restrict__ wr = wbase + (int64_t)(kLiteral ? j : j - 1) * NV * B;
            T wk[8];
#pragma unroll
            for (int q = 0; q < NV; ++q) vunpack(wk + q * W, __ldcs(wr + (int64_t)q * B));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const T x = val(k, h ? (int)(pr[k] >> 16) : (int)(pr[k] & 0xFFFFu));
                acc[k] = kLiteral ? fma(wk[k], x, acc[k]) : fma(wk[k], x - c[k], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = kLiteral ? acc[k] : c[k] + acc[k];
}

// The streamed populations f (storage form) of node p into fout, psi(rho of f) into psi.
template <typename T>
__device__ __forceinline__ void sc_store_streamed(const ScArgs<T> &a, int seg, int64_t p, const T (&f)[9]) {
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    const T *pr = a.params + 4 * seg;
    const T rho_ref = kLiteral ? T(0) : pr[2];
    const T drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const T rho = rho_ref + drho;
    const T rp = a.sc[2 * seg + 1];
    a.psi[p] = rp * (T(1) - sc_exp(-rho / rp));
#pragma unroll
    for (int k = 0; k < 9; ++k) a.fout[(int64_t)k * a.N + p] = f[k];
}

// Pass 1: fhat of every node of the tile (storage form) into fout, psi(rho of fhat) into psi.
// kNear: some tiles use nearest-node stencils (their halo staged direction-major, [8][U]).
template <typename T, int B, bool kNear>
__global__ void __launch_bounds__(B, tile_min_blocks(B, (int)sizeof(T))) sc_stream_kernel(ScArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *sh = reinterpret_cast<VT *>(smem_raw);  // [U][NV]
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        const bool near = kNear && tile.mode == MLBM_STENCIL_NEAREST;
        if (near)
            stage_halo_dirmajor<T>(a.halo + tile.h_off, tile.U, a.fin, N, reinterpret_cast<T *>(sh));
        else
            stage_halo<T>(a.halo + tile.h_off, tile.U, a.fin, N, sh);
        __syncthreads();
        const int b = threadIdx.x;
        if (b < tile.count && near) {
            if constexpr (kNear) {
                const int64_t p = tile.begin + b;
                const T *shs = reinterpret_cast<const T *>(sh);
                const int U = tile.U;
                T f[9], fk[8];
                f[0] = a.fin[p];
                interp_departure<T, B>(a.lidx, a.wt, tile, b, [&](int k, int sl) { return shs[k * U + sl]; }, fk);
#pragma unroll
                for (int k = 0; k < 8; ++k) f[k + 1] = fk[k];
                sc_store_streamed<T>(a, tile.seg, p, f);
            }
        } else if (b < tile.count) {
            const int64_t p = tile.begin + b;
            T f[9];
            f[0] = a.fin[p];
            VT c[NV], acc[NV], unused[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                c[q] = sh[b * NV + q];
                vzero(acc[q]);
            }
            const uint32_t *__restrict__ lp = a.lidx + tile.l_off + b;
            const VT *__restrict__ wp;
            if constexpr (kLiteral) {
                wp = reinterpret_cast<const VT *>(a.wt + tile.w64_off) + b;
#pragma unroll
                for (int q = 0; q < NV; ++q) vmul(acc[q], __ldcs(wp + (int64_t)q * B), c[q]);
                wp += (int64_t)NV * B;
            } else {
                wp = reinterpret_cast<const VT *>(a.wt + tile.w_off) + b;
            }
            interp_own<T, B, false>(wp, lp, sh, c, acc, unused, tile.K - 1);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if constexpr (kLiteral)
                    vunpack(f + 1 + q * W, acc[q]);
                else
                    vunpack_sum(f + 1 + q * W, c[q], acc[q]);
            }
            sc_store_streamed<T>(a, tile.seg, p, f);
        }
        __syncthreads();
    }
}

// Pass 2: psi at the eight departure points of every node, the interaction force, and the
// collision of fhat (read from and written back to fout) towards the shifted equilibrium.
template <typename T, int B, bool kNear>
__global__ void __launch_bounds__(B, tile_min_blocks(B, (int)sizeof(T))) sc_collide_kernel(ScArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *shp = reinterpret_cast<T *>(smem_raw);  // [U] psi of the halo
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        for (int u = threadIdx.x; u < tile.U; u += blockDim.x) shp[u] = a.psi[__ldg(a.halo + tile.h_off + u)];
        __syncthreads();
        const int b = threadIdx.x;
        if (b < tile.count) {
            const int64_t p = tile.begin + b;
            const T pc = shp[b];
            // psi_k = psi at x - e_k dx_ml, k = 1..8: FP32 as differences to the centre value,
            // FP64 as the literal sum (the forms of the streaming)
            T psik[8];
            if (kNear && tile.mode == MLBM_STENCIL_NEAREST) {
                if constexpr (kNear)
                    interp_departure<T, B>(a.lidx, a.wt, tile, b, [&](int, int sl) { return shp[sl]; }, psik);
            } else {
                T acc[8];
                const uint32_t *__restrict__ lp = a.lidx + tile.l_off + b;
                const VT *__restrict__ wp;
                if constexpr (kLiteral) {
                    wp = reinterpret_cast<const VT *>(a.wt + tile.w64_off) + b;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        T w0[W];
                        vunpack(w0, __ldcs(wp + (int64_t)q * B));
#pragma unroll
                        for (int r = 0; r < W; ++r) acc[q * W + r] = w0[r] * pc;
                    }
                    wp += (int64_t)NV * B;
                } else {
                    wp = reinterpret_cast<const VT *>(a.wt + tile.w_off) + b;
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc[k] = T(0);
                }
                const int m1 = tile.K - 1;
                for (int j = 0; j < m1; ++j) {
                    const uint32_t pr = __ldcs(lp + (int64_t)(j >> 1) * B);
                    const int sl = (j & 1) ? (int)(pr >> 16) : (int)(pr & 0xFFFFu);
                    const T x = kLiteral ? shp[sl] : shp[sl] - pc;
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        T wv[W];
                        vunpack(wv, __ldcs(wp + (int64_t)(j * NV + q) * B));
#pragma unroll
                        for (int r = 0; r < W; ++r) acc[q * W + r] = fma(wv[r], x, acc[q * W + r]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) psik[k] = kLiteral ? acc[k] : pc + acc[k];
            }
            // F = -G psi sum_k omega_k psi(x + e_k dx) e_k = G psi sum_k omega_k e_k psi_k, since
            // x - e_k dx = x + e_k' dx with e_k' = -e_k
            T sx = T(0), sy = T(0);
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                const T pk = psik[k - 1];
                sx += omega_of<T>(k) * T(ex_of(k)) * pk;
                sy += omega_of<T>(k) * T(ey_of(k)) * pk;
            }
            const T G = a.sc[2 * tile.seg];
            const T Fx = G * pc * sx, Fy = G * pc * sy;
            // collision of fhat with the body force, then the velocity shift as a difference
            T f[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) f[k] = a.fout[(int64_t)k * N + p];
            const T *pr = a.params + 4 * tile.seg;
            const T tau = pr[0], gm = pr[1], inv_tau = pr[3];
            T gx = T(0), gy = T(0);
            if (gm != T(0)) {
                gx = gm * a.fdir[p];
                gy = gm * a.fdir[N + p];
            }
            T rho, ux, uy;
            if constexpr (kLiteral)
                collide<T>(f, T(0), inv_tau, gx, gy, rho, ux, uy);
            else
                collide_projected(f, pr[2], inv_tau, gx, gy, rho, ux, uy);
            const T dux = tau * Fx / rho, duy = tau * Fy / rho;
            const T vx = ux + dux, vy = uy + duy;
            const T dsq15 = T(1.5) * ((vx * vx + vy * vy) - (ux * ux + uy * uy));
            const T rt = rho * inv_tau;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const T cu = T(ex_of(k)) * ux + T(ey_of(k)) * uy;
                const T dc = T(ex_of(k)) * dux + T(ey_of(k)) * duy;
                // s^eq(v) - s^eq(u) = omega rho (3 dc + 4.5 dc (2 cu + dc) - 1.5 (v^2 - u^2))
                f[k] += omega_of<T>(k) * rt * (T(3) * dc + T(4.5) * dc * (T(2) * cu + dc) - dsq15);
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) a.fout[(int64_t)k * N + p] = f[k];
            if (a.mom) {
                a.mom[p] = rho;
                a.mom[N + p] = ux;
                a.mom[2 * N + p] = uy;
            }
        }
        __syncthreads();
    }
}

template <typename T, int B, bool kNear>
int launch_sc_t(mlbm_weights *w, const ScArgs<T> &a, cudaStream_t st) {
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, w->device);
    const size_t sm1 = (size_t)w->umax * 8 * sizeof(T), sm2 = (size_t)w->umax * sizeof(T);
    if (sm1 > (size_t)maxsm) return fail(MLBM_EINVAL, "a tile's halo does not fit in shared memory at this precision");
    const void *k1 = (const void *)sc_stream_kernel<T, B, kNear>, *k2 = (const void *)sc_collide_kernel<T, B, kNear>;
    int rc = allow_dynamic_smem(k1);
    if (!rc) rc = allow_dynamic_smem(k2);
    if (rc) return rc;
    int per1 = 0, per2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k1, B, sm1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, B, sm2);
    const int g1 = std::max(1, std::min(w->ntiles, std::max(1, per1) * w->num_sms));
    const int g2 = std::max(1, std::min(w->ntiles, std::max(1, per2) * w->num_sms));
    sc_stream_kernel<T, B, kNear><<<g1, B, sm1, st>>>(a);
    sc_collide_kernel<T, B, kNear><<<g2, B, sm2, st>>>(a);
    return cuda_check_step(cudaGetLastError(), "Shan-Chen step launch");
}

// Per-segment (G, rho_psi) on the device, FP64 then an FP32 copy; uploaded when they change.
int set_sc_params(mlbm_weights *w, const mlbm_sc_params *sc, cudaStream_t st) {
    std::vector<double> v(2 * (size_t)w->nseg);
    for (int s = 0; s < w->nseg; ++s) {
        if (!std::isfinite(sc[s].G) || !(sc[s].rho_psi > 0) || !std::isfinite(sc[s].rho_psi))
            return fail(MLBM_EINVAL, "Shan-Chen parameters need a finite G and rho_psi > 0");
        v[2 * s] = sc[s].G;
        v[2 * s + 1] = sc[s].rho_psi;
    }
    if (w->d_sc && v == w->sc_cache) return MLBM_OK;
    if (!w->d_sc) {
        cudaError_t e = cudaMalloc(&w->d_sc, sizeof(double) * 3 * (size_t)w->nseg);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w->d_sc = nullptr;
            return fail(MLBM_ENOMEM, "Shan-Chen parameter allocation failed");
        }
    }
    std::vector<double> buf(3 * (size_t)w->nseg, 0.0);
    std::copy(v.begin(), v.end(), buf.begin());
    float *f32 = reinterpret_cast<float *>(buf.data() + 2 * (size_t)w->nseg);
    for (size_t i = 0; i < v.size(); ++i) f32[i] = (float)v[i];
    int rc = cuda_check_step(cudaMemcpyAsync(w->d_sc, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                             "Shan-Chen parameter upload");
    // the pageable source may be read after return: wait for the copy before buf dies
    if (!rc) rc = cuda_check_step(cudaStreamSynchronize(st), "Shan-Chen parameter upload");
    if (!rc) w->sc_cache = v;
    return rc;
}

template <typename T>
int sc_step_t(mlbm_weights *w, const void *fin, void *fout, void *mom, cudaStream_t st) {
    constexpr bool kDev = std::is_same<T, float>::value;
    ScArgs<T> a;
    a.tiles = w->d_tiles;
    a.halo = w->d_halo;
    a.lidx = w->d_lidx;
    a.wt = kDev ? (const T *)w->d_w32t : (const T *)w->d_w64t;
    a.fdir = kDev ? (const T *)w->d_fdir32 : (const T *)w->d_fdir64;
    a.params = kDev ? (const T *)(w->d_params + 4 * (size_t)w->nseg) : (const T *)w->d_params;
    a.sc = kDev ? (const T *)(w->d_sc + 2 * (size_t)w->nseg) : (const T *)w->d_sc;
    a.fin = (const T *)fin;
    a.fout = (T *)fout;
    a.psi = (T *)w->d_sc_psi;
    a.mom = (T *)mom;
    a.N = w->N;
    a.ntiles = w->ntiles;
    return with_tile_nodes(w->tile_nodes, [&](auto Bc) {
        return w->any_nearest ? launch_sc_t<T, decltype(Bc)::value, true>(w, a, st)
                              : launch_sc_t<T, decltype(Bc)::value, false>(w, a, st);
    });
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" int mlbm_sc_step(mlbm_weights *w, const mlbm_params *params, const mlbm_sc_params *sc, int dtype,
                            const void *f_in, void *f_out, void *moments, void *stream) {
    set_error("");
    if (!w || !f_in || !f_out || !sc) return fail(MLBM_EINVAL, "NULL argument");
    if (f_in == f_out) return fail(MLBM_EINVAL, "f_in and f_out must not alias");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    if (w->has_mask)
        return fail(MLBM_EINVAL, "Shan-Chen steps need periodic segments (no walls)");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(w, params, st))) return rc;
    if ((rc = set_sc_params(w, sc, st))) return rc;
    if (!w->d_sc_psi) {
        cudaError_t e = cudaMalloc(&w->d_sc_psi, sizeof(double) * std::max<int64_t>(1, w->N));
        if (e != cudaSuccess) {
            cudaGetLastError();
            w->d_sc_psi = nullptr;
            return fail(MLBM_ENOMEM, "Shan-Chen scratch allocation failed");
        }
    }
    return dtype == MLBM_F32 ? sc_step_t<float>(w, f_in, f_out, moments, st)
                             : sc_step_t<double>(w, f_in, f_out, moments, st);
}
