// Fused meshless-LBM time step and its companions (appendix algorithm COLLIDE/STREAM reordered
// as a pull; Sec. 2.3 semi-Lagrangian streaming; Sec. 3 forcing and wall bounce-back),
// initial state, moments, norms and the CUDA-graph step loop.
//
// Step kernel: persistent CTAs walk a tile table (tiles = runs of 512, 128 or 32 stored nodes of
// one segment, largest stencils first), one thread per node (one per 16-byte direction vector
// in 32-node tiles).  A tile's halo of f^post is staged in shared memory; for node i each stencil
// member's 16-bit halo slot is loaded once and reused by all eight moving directions, and the
// shape vectors are stored per tile as [member][direction vector][node] so that every warp load
// is a contiguous 512-byte run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "d2q9_device.cuh"
#include "mlbm_internal.h"
#include "tile_interp.cuh"

namespace mlbm {

int cuda_check_step(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MLBM_OK;
    return fail(MLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int allow_dynamic_smem(const void *fn) {
    int dev = 0, maxsm = 0;
    cudaFuncAttributes fa;
    int rc = cuda_check_step(cudaGetDevice(&dev), "current device");
    if (!rc) rc = cuda_check_step(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                                  "shared-memory limit");
    if (!rc) rc = cuda_check_step(cudaFuncGetAttributes(&fa, fn), "kernel attributes");
    // the dynamic part may use what the kernel's static shared memory leaves of the maximum
    if (!rc)
        rc = cuda_check_step(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  maxsm - (int)fa.sharedSizeBytes),
                             "shared-memory attribute");
    return rc;
}

namespace {

template <typename T>
struct StepArgs {
    const TileDev *__restrict__ tiles;
    const int32_t *__restrict__ halo;
    const uint32_t *__restrict__ lidx;
    const T *__restrict__ wt;           // tile layout shape vectors
    const uint16_t *__restrict__ mask;  // NULL when no segment has wall populations
    const T *__restrict__ fdir;         // [2][N]
    const T *__restrict__ params;  // [nseg][4]: tau, g, rho0, 1/tau in the step's precision
    const T *__restrict__ fin;
    T *__restrict__ fout;
    T *__restrict__ mom;  // optional [3][N]
    int64_t N;
    int ntiles;
    int umax;  // largest halo (slots): split tiles keep their hand-over buffer after it
};

// Nearest-node stencils (Sec. 2.3, appendix algorithm): population k of node b is interpolated
// in the stencil of its departure node L_k, so every direction has its own members; their halo
// slots are packed [ceil(K/2)][B][8], member 0 being L_k itself.  Same forms as the own-stencil
// path: FP32 differences to the centre value f_k(L_k) (members 1..K-1), FP64 the literal sum.
// The halo is staged direction-major, shs[k][U]: a warp reading direction k at scattered slots
// then spreads over all banks instead of the four that [U][8] would leave it.
template <typename T, int B>
__device__ __forceinline__ void interp_nearest(const StepArgs<T> &a, const TileDev &tile, int b,
                                               const T *__restrict__ shs, T (&f)[9]) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;
    const int K = tile.K, JP = (K + 1) / 2, U = tile.U;
    // slot words of a node for one member pair: eight directions, two 16-byte loads
    const uint4 *__restrict__ lp = reinterpret_cast<const uint4 *>(a.lidx + tile.l_off) + 2 * b;
    const VT *__restrict__ wbase = reinterpret_cast<const VT *>(a.wt + (kLiteral ? tile.w64_off : tile.w_off)) + b;
    T acc[8], c[8];
    auto load_pairs = [&](int jp, uint32_t (&pr)[8]) {
        const uint4 lo = __ldcs(lp + (int64_t)jp * 2 * B), hi = __ldcs(lp + (int64_t)jp * 2 * B + 1);
        pr[0] = lo.x; pr[1] = lo.y; pr[2] = lo.z; pr[3] = lo.w;
        pr[4] = hi.x; pr[5] = hi.y; pr[6] = hi.z; pr[7] = hi.w;
    };
    {
        uint32_t pr[8];
        load_pairs(0, pr);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = shs[k * U + (int)(pr[k] & 0xFFFFu)];
            acc[k] = T(0);
        }
    }
    for (int jp = 0; jp < JP; ++jp) {
        uint32_t pr[8];
        load_pairs(jp, pr);
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
                const int sl = h ? (int)(pr[k] >> 16) : (int)(pr[k] & 0xFFFFu);
                const T x = shs[k * U + sl];
                acc[k] = kLiteral ? fma(wk[k], x, acc[k]) : fma(wk[k], x - c[k], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k + 1] = kLiteral ? acc[k] : c[k] + acc[k];
}

// Own-stencil interpolation of the direction vectors Q0 .. Q0 + NQ - 1 of node b over members
// 1..m1, in interp_own's order (members in sequence, two per slot word), so a node whose
// directions are split over two threads gets the same sums as one thread computing all.
template <typename T, int B, int Q0, int NQ>
__device__ __forceinline__ void interp_own_part(const typename V<T>::type *__restrict__ wp,
                                                const uint32_t *__restrict__ lp, const typename V<T>::type *sh,
                                                const typename V<T>::type (&c)[8 / V<T>::width],
                                                typename V<T>::type (&acc)[8 / V<T>::width], int m1) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int NV = 8 / V<T>::width;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < m1; j += 2) {
        const uint32_t pr = __ldcs(lp + (int64_t)(j >> 1) * B);
        VT w0[NQ], w1[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            w0[q] = __ldcs(wp + (int64_t)(j * NV + Q0 + q) * B);
            w1[q] = __ldcs(wp + (int64_t)((j + 1) * NV + Q0 + q) * B);
        }
        const int s0 = (int)(pr & 0xFFFFu), s1 = (int)(pr >> 16);
#pragma unroll
        for (int q = 0; q < NQ; ++q) vfma<kLiteral>(acc[Q0 + q], w0[q], sh[s0 * NV + Q0 + q], c[Q0 + q]);
#pragma unroll
        for (int q = 0; q < NQ; ++q) vfma<kLiteral>(acc[Q0 + q], w1[q], sh[s1 * NV + Q0 + q], c[Q0 + q]);
    }
    if (j < m1) {
        const uint32_t pr = __ldcs(lp + (int64_t)(j >> 1) * B);
        const int s0 = (int)(pr & 0xFFFFu);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            vfma<kLiteral>(acc[Q0 + q], __ldcs(wp + (int64_t)(j * NV + Q0 + q) * B), sh[s0 * NV + Q0 + q], c[Q0 + q]);
    }
}

// Threads per node of the step kernel: one, except in one-warp tiles, whose nodes get one thread
// per 16-byte vector of their eight directions (two in FP32, four in FP64), so that small
// clouds, a few warps per SM, hide the latency of their dependent operations with more warps.
__host__ __device__ constexpr int step_split(int B, int elem_bytes) {
    return B == kTileNodesTiny ? (elem_bytes == 8 ? 4 : 2) : 1;
}
__host__ __device__ constexpr int step_threads(int B, int elem_bytes) { return B * step_split(B, elem_bytes); }
__host__ __device__ constexpr int step_min_blocks(int B, int elem_bytes) {
    return B == kTileNodesTiny ? 16 / step_split(B, elem_bytes) : tile_min_blocks(B, elem_bytes);
}

// One fused time step over all tiles (persistent CTAs, one node per thread, B threads per CTA
// and B nodes per tile; for one-warp tiles two threads per node, see step_threads):
//   1. stage f^post_k (k = 1..8) of the tile's halo in shared memory as [slot][8];
//   2. FP32: fhat_k(i) = f_k(i) + sum_{j>=1} W_k[j](i) (f_k(s_j(i)) - f_k(i)) -- the shape vector
//      sums to one (constant reproduction), so the centre weight is implied and never loaded,
//      and rounding of the FP32 weights only touches the small differences;
//      FP64: fhat_k(i) = sum_{j>=0} W_k[j](i) f_k(s_j(i)) as written in eq. (shape_vector);
//   3. bounce-back of unknown wall populations; 4. BGK collision with forcing; 5. store.
template <typename T, int B>
__global__ void __launch_bounds__(step_threads(B, (int)sizeof(T)), step_min_blocks(B, (int)sizeof(T)))
    step_kernel(StepArgs<T> a) {
    using VT = typename V<T>::type;
    constexpr bool kLiteral = !std::is_same<T, float>::value;
    constexpr int W = V<T>::width;
    constexpr int NV = 8 / W;  // vectors per 8 moving populations
    constexpr int S = step_split(B, (int)sizeof(T));  // threads per node
    constexpr bool kSplit = S > 1;
    constexpr int NQ = NV / S;  // direction vectors per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *sh = reinterpret_cast<VT *>(smem_raw);  // [U][NV]
    const int64_t N = a.N;
    // split tiles: the other threads' interpolated populations, handed to the first, [B][NV]
    VT *hand = sh + (size_t)a.umax * NV;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        // 1. halo staging (own nodes first, then the other members sorted: mostly coalesced)
        if (tile.mode == MLBM_STENCIL_NEAREST)
            stage_halo_dirmajor<T>(a.halo + tile.h_off, tile.U, a.fin, N, reinterpret_cast<T *>(sh));
        else
            stage_halo<T>(a.halo + tile.h_off, tile.U, a.fin, N, sh);
        __syncthreads();
        if constexpr (kSplit) {
            // S threads per node: thread part r interpolates the direction vectors r NQ ..
            // (r + 1) NQ - 1 over all members, in the one-thread order; part 0 collects the
            // others' populations from hand[] and collides
            const int b = (int)threadIdx.x % B;
            const int part = (int)threadIdx.x / B;
            const bool own = tile.mode != MLBM_STENCIL_NEAREST;
            T f[9];
            if (b < tile.count && own) {
                VT c[NV], acc[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    c[q] = sh[b * NV + q];
                    vzero(acc[q]);
                }
                const uint32_t *__restrict__ lp = a.lidx + tile.l_off + b;
                const VT *__restrict__ wp;
                if constexpr (kLiteral) {
                    // FP64: literal sum over members 0..K-1; row 0 holds the centre weight
                    wp = reinterpret_cast<const VT *>(a.wt + tile.w64_off) + b;
#pragma unroll
                    for (int q = 0; q < NV; ++q)
                        if (q / NQ == part) vmul(acc[q], __ldcs(wp + (int64_t)q * B), c[q]);
                    wp += (int64_t)NV * B;
                } else {
                    wp = reinterpret_cast<const VT *>(a.wt + tile.w_off) + b;
                }
                // 2. interpolation over stencil members 1..K-1, two members per packed slot word
                switch (part) {
                    case 0: interp_own_part<T, B, 0, NQ>(wp, lp, sh, c, acc, tile.K - 1); break;
                    case 1: interp_own_part<T, B, 1 * NQ, NQ>(wp, lp, sh, c, acc, tile.K - 1); break;
                    case 2: interp_own_part<T, B, (2 * NQ) % NV, NQ>(wp, lp, sh, c, acc, tile.K - 1); break;
                    default: interp_own_part<T, B, (3 * NQ) % NV, NQ>(wp, lp, sh, c, acc, tile.K - 1); break;
                }
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    if (q / NQ != part) continue;
                    VT v = acc[q];
                    if constexpr (!kLiteral)
                        v = make_float4(c[q].x + v.x, c[q].y + v.y, c[q].z + v.z, c[q].w + v.w);
                    if (part == 0)
                        vunpack(f + 1 + q * W, v);
                    else
                        hand[b * NV + q] = v;
                }
            }
            __syncthreads();  // the other parts' populations are in hand[]
            if (b < tile.count && part == 0) {
                const int64_t p = tile.begin + b;
                f[0] = a.fin[p];
                if (!own) {
                    interp_nearest<T, B>(a, tile, b, reinterpret_cast<const T *>(sh), f);
                } else {
#pragma unroll
                    for (int q = NQ; q < NV; ++q) vunpack(f + 1 + q * W, hand[b * NV + q]);
                }
                // 3. wall bounce-back: unknown populations take the streamed opposite population
                if (a.mask) {
                    const uint16_t mb = a.mask[p];
                    if (mb) {
                        T g[9];
#pragma unroll
                        for (int k = 0; k < 9; ++k) g[k] = f[k];
#pragma unroll
                        for (int k = 1; k < 9; ++k)
                            if (mb >> k & 1u) f[k] = g[opp_of(k)];
                    }
                }
                // 4. collision
                const T *pr = a.params + 4 * tile.seg;
                const T inv_tau = pr[3];
                const T gm = pr[1];
                T gx = T(0), gy = T(0);
                if (gm != T(0)) {
                    gx = gm * a.fdir[p];
                    gy = gm * a.fdir[N + p];
                }
                T rho, ux, uy;
                if constexpr (std::is_same<T, float>::value)
                    collide_projected(f, pr[2], inv_tau, gx, gy, rho, ux, uy);
                else
                    collide<T>(f, T(0), inv_tau, gx, gy, rho, ux, uy);
                // 5. store
#pragma unroll
                for (int k = 0; k < 9; ++k) a.fout[(int64_t)k * N + p] = f[k];
                if (a.mom) {
                    a.mom[p] = rho;
                    a.mom[N + p] = ux;
                    a.mom[2 * N + p] = uy;
                }
            }
        } else {
            const int b = threadIdx.x;
            if (b < tile.count) {
                const int64_t p = tile.begin + b;
                T f[9];
                f[0] = a.fin[p];
                if (tile.mode == MLBM_STENCIL_NEAREST) {
                    interp_nearest<T, B>(a, tile, b, reinterpret_cast<const T *>(sh), f);
                } else {
                    VT c[NV], acc[NV];
    #pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        c[q] = sh[b * NV + q];
                        vzero(acc[q]);
                    }
                    const uint32_t *__restrict__ lp = a.lidx + tile.l_off + b;
                    const VT *__restrict__ wp;
                    if constexpr (kLiteral) {
                        // FP64: literal sum over members 0..K-1; row 0 holds the centre weight
                        wp = reinterpret_cast<const VT *>(a.wt + tile.w64_off) + b;
    #pragma unroll
                        for (int q = 0; q < NV; ++q) vmul(acc[q], __ldcs(wp + (int64_t)q * B), c[q]);
                        wp += (int64_t)NV * B;
                    } else {
                        wp = reinterpret_cast<const VT *>(a.wt + tile.w_off) + b;
                    }
                    // 2. interpolation over stencil members 1..K-1, two members per packed slot word
                    VT unused[NV];
                    interp_own<T, B, false>(wp, lp, sh, c, acc, unused, tile.K - 1);
    #pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        if constexpr (kLiteral)
                            vunpack(f + 1 + q * W, acc[q]);
                        else
                            vunpack_sum(f + 1 + q * W, c[q], acc[q]);
                    }
                }  // own-stencil interpolation
                // 3. wall bounce-back: unknown populations take the streamed opposite population
                if (a.mask) {
                    const uint16_t mb = a.mask[p];
                    if (mb) {
                        T g[9];
    #pragma unroll
                        for (int k = 0; k < 9; ++k) g[k] = f[k];
    #pragma unroll
                        for (int k = 1; k < 9; ++k)
                            if (mb >> k & 1u) f[k] = g[opp_of(k)];
                    }
                }
                // 4. collision
                const T *pr = a.params + 4 * tile.seg;
                const T inv_tau = pr[3];
                const T gm = pr[1];
                T gx = T(0), gy = T(0);
                if (gm != T(0)) {
                    gx = gm * a.fdir[p];
                    gy = gm * a.fdir[N + p];
                }
                T rho, ux, uy;
                if constexpr (std::is_same<T, float>::value)
                    collide_projected(f, pr[2], inv_tau, gx, gy, rho, ux, uy);
                else
                    collide<T>(f, T(0), inv_tau, gx, gy, rho, ux, uy);
                // 5. store
    #pragma unroll
                for (int k = 0; k < 9; ++k) a.fout[(int64_t)k * N + p] = f[k];
                if (a.mom) {
                    a.mom[p] = rho;
                    a.mom[N + p] = ux;
                    a.mom[2 * N + p] = uy;
                }
            }
        }
        __syncthreads();
    }
}

// Initial state: equilibrium at (rho, u) plus the forcing term (its post-collision value).
template <typename T>
__global__ void init_kernel(const TileDev *__restrict__ tiles, int ntiles, const int64_t *__restrict__ perm,
                            const double *__restrict__ fdir, const double *__restrict__ params,
                            const double *__restrict__ rho_in, const double *__restrict__ ux_in,
                            const double *__restrict__ uy_in, T *__restrict__ f, int64_t N) {
    constexpr bool kDev = std::is_same<T, float>::value;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
        const int64_t p = tile.begin + b;
        const int64_t o = perm[p];
        const double *pr = params + 4 * tile.seg;
        const double rho_ref = kDev ? pr[2] : 0.0;
        const double rho = rho_in[o], ux = ux_in[o], uy = uy_in[o];
        const double gx = pr[1] * fdir[p], gy = pr[1] * fdir[N + p];
        const double usq15 = 1.5 * (ux * ux + uy * uy);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double s = geq_of<double>(k, rho - rho_ref, rho, ux, uy, usq15) +
                       omega_of<double>(k) * 3.0 * (ex_of(k) * gx + ey_of(k) * gy);
            f[(int64_t)k * N + p] = (T)s;
        }
        }
    }
}

// Macroscopic fields of the level whose post-collision state is f (collision keeps rho and
// adds g to rho u), FP64, scattered to original order.
template <typename T>
__global__ void moments_kernel(const TileDev *__restrict__ tiles, int ntiles, const int64_t *__restrict__ perm,
                               const double *__restrict__ fdir, const double *__restrict__ params,
                               const T *__restrict__ f, double *__restrict__ rho_out,
                               double *__restrict__ ux_out, double *__restrict__ uy_out, int64_t N) {
    constexpr bool kDev = std::is_same<T, float>::value;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
        const int64_t p = tile.begin + b;
        const double *pr = params + 4 * tile.seg;
        double s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = (double)f[(int64_t)k * N + p];
        double drho, rho, ux, uy;
        moments_of<double>(s, kDev ? pr[2] : 0.0, drho, rho, ux, uy);
        // remove the body force the collision added
        ux -= pr[1] * fdir[p] / rho;
        uy -= pr[1] * fdir[N + p] / rho;
        const int64_t o = perm[p];
        rho_out[o] = rho;
        ux_out[o] = ux;
        uy_out[o] = uy;
        }
    }
}

constexpr int kNormBlocks = 1024;
constexpr int kNormThreads = 256;

template <int NT>
__device__ __forceinline__ void block_sum3(double v[3], double *sh) {
    for (int c = 0; c < 3; ++c) {
        sh[threadIdx.x] = v[c];
        __syncthreads();
        for (int s = NT / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        v[c] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kNormThreads) norms_pass1(const double *__restrict__ a, const double *__restrict__ b,
                                                             const double *__restrict__ c, const double *__restrict__ d,
                                                             int64_t n, double *__restrict__ partial) {
    __shared__ double sh[kNormThreads];
    double v[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double e = a[i] - b[i];
        v[0] += e * e;
        v[1] += b[i] * b[i];
        v[2] += a[i] * a[i];
        if (c) {
            double e2 = c[i] - d[i];
            v[0] += e2 * e2;
            v[1] += d[i] * d[i];
            v[2] += c[i] * c[i];
        }
    }
    block_sum3<kNormThreads>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[3 * blockIdx.x + k] = v[k];
}

__global__ void __launch_bounds__(kNormThreads) norms_pass2(const double *__restrict__ partial, int nparts,
                                                             double *__restrict__ out) {
    __shared__ double sh[kNormThreads];
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
        for (int k = 0; k < 3; ++k) v[k] += partial[3 * i + k];
    block_sum3<kNormThreads>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k] = v[k];
}

int grid_for(const mlbm_weights *w, const void *fn, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    per_sm = std::max(1, per_sm);
    return std::max(1, std::min(w->ntiles, per_sm * w->num_sms));
}

}  // namespace

// Stream-ordered refresh of the device copy of the step parameters.
int set_params(mlbm_weights *w, const mlbm_params *params, cudaStream_t st) {
    if (!params) return fail(MLBM_EINVAL, "params is NULL");
    std::vector<double> v(4 * w->nseg);
    for (int s = 0; s < w->nseg; ++s) {
        if (!(params[s].tau > 0.5)) return fail(MLBM_EINVAL, "tau must be > 0.5 (positive viscosity)");
        if (!std::isfinite(params[s].g) || !std::isfinite(params[s].rho0))
            return fail(MLBM_EINVAL, "non-finite parameter");
        v[4 * s] = params[s].tau;
        v[4 * s + 1] = params[s].g;
        v[4 * s + 2] = params[s].rho0;
        v[4 * s + 3] = 1.0 / params[s].tau;  // 1/tau once here, not per node
    }
    if (v == w->params_cache) return MLBM_OK;
    // device buffer: [nseg][4] float64 followed by an FP32 copy [nseg][4] for the FP32 kernels
    // (conversions from float64 would run on the FP64 unit once per node)
    std::vector<double> buf(6 * (size_t)w->nseg, 0.0);
    std::copy(v.begin(), v.end(), buf.begin());
    float *f32 = reinterpret_cast<float *>(buf.data() + 4 * (size_t)w->nseg);
    for (size_t i = 0; i < v.size(); ++i) f32[i] = (float)v[i];
    int rc = cuda_check_step(cudaMemcpyAsync(w->d_params, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                             "parameter upload");
    if (rc) return rc;
    // the pageable source may be read after return: wait for the copy before v dies
    rc = cuda_check_step(cudaStreamSynchronize(st), "parameter upload");
    if (rc) return rc;
    w->params_cache = v;
    return MLBM_OK;
}

int check_dtype(const mlbm_weights *w, int dtype) {
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "dtype must be MLBM_F32 or MLBM_F64");
    const int i = dtype == MLBM_F32 ? 0 : 1;
    if (!(i == 0 ? (const void *)w->d_w32t : (const void *)w->d_w64t))
        return fail(MLBM_EINVAL, i == 0 ? "weights built without MLBM_KEEP_W32" : "weights built without MLBM_KEEP_W64");
    if (!w->step_grid[i])
        return fail(MLBM_EINVAL, "a tile's halo (" + std::to_string(w->umax) +
                                     " nodes) does not fit in shared memory at this precision");
    return MLBM_OK;
}

template <typename T>
size_t step_smem(const mlbm_weights *w) {
    const size_t hand = w->tile_nodes == kTileNodesTiny ? (size_t)kTileNodesTiny * 8 * sizeof(T) : 0;
    return (size_t)w->umax * 8 * sizeof(T) + hand;
}

template <typename T>
int launch_step_t(const mlbm_weights *w, const TileDev *tiles, int ntiles, const void *fin, void *fout, void *mom,
                  cudaStream_t st) {
    StepArgs<T> a;
    a.tiles = tiles;
    a.halo = w->d_halo;
    a.lidx = w->d_lidx;
    a.wt = std::is_same<T, float>::value ? (const T *)w->d_w32t : (const T *)w->d_w64t;
    a.mask = w->has_mask ? w->d_mask : nullptr;
    a.fdir = std::is_same<T, float>::value ? (const T *)w->d_fdir32 : (const T *)w->d_fdir64;
    a.params = std::is_same<T, float>::value ? (const T *)(w->d_params + 4 * (size_t)w->nseg) : (const T *)w->d_params;
    a.fin = (const T *)fin;
    a.fout = (T *)fout;
    a.mom = (T *)mom;
    a.N = w->N;
    a.ntiles = ntiles;
    a.umax = w->umax;
    const int grid = std::max(1, std::min(ntiles, w->step_grid[std::is_same<T, float>::value ? 0 : 1]));
    const size_t smem = step_smem<T>(w);
    return with_tile_nodes(w->tile_nodes, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        step_kernel<T, B><<<grid, step_threads(B, (int)sizeof(T)), smem, st>>>(a);
        return cuda_check_step(cudaGetLastError(), "step_kernel launch");
    });
}

// Persistent grids of the step kernels: CTAs resident per SM x SMs, capped by the tile count.
// A precision whose halo does not fit in shared memory gets grid 0 and is refused by the step.
int prepare_step_grids(mlbm_weights *w) {
    const void *fns[2] = {nullptr, nullptr};
    with_tile_nodes(w->tile_nodes, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        fns[0] = (const void *)step_kernel<float, B>;
        fns[1] = (const void *)step_kernel<double, B>;
        return 0;
    });
    const size_t sm[2] = {step_smem<float>(w), step_smem<double>(w)};
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, w->device);
    for (int i = 0; i < 2; ++i) {
        w->step_grid[i] = 0;
        if (sm[i] > (size_t)maxsm) continue;
        int rc = allow_dynamic_smem(fns[i]);
        if (rc) return rc;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[i], step_threads(w->tile_nodes, i == 0 ? 4 : 8), sm[i]);
        w->step_grid[i] = std::max(1, std::min(w->ntiles, std::max(1, per_sm) * w->num_sms));
    }
    return MLBM_OK;
}

// One step over the first ntiles tiles of a tile table (the weights' own, or a re-sorted copy).
int launch_step_tiles(const mlbm_weights *w, int dtype, const TileDev *tiles, int ntiles, const void *fin,
                      void *fout, void *mom, cudaStream_t st) {
    return dtype == MLBM_F32 ? launch_step_t<float>(w, tiles, ntiles, fin, fout, mom, st)
                             : launch_step_t<double>(w, tiles, ntiles, fin, fout, mom, st);
}

int launch_step(const mlbm_weights *w, int dtype, const void *fin, void *fout, void *mom, cudaStream_t st) {
    return launch_step_tiles(w, dtype, w->d_tiles, w->ntiles, fin, fout, mom, st);
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the norms reduction.
//
// The per-block partial sums live in a fixed array in the library's own device memory instead
// of a buffer from cudaMalloc, so the call allocates nothing.  Each block reduces at most
// kNoallocChunk elements, so the array bounds n.  Host code cannot use the array's name as a
// device address; the address is looked up once per device with cudaGetSymbolAddress.
constexpr int kNoallocChunk = kNormThreads * 16;                             // elements per block
constexpr int kNoallocMaxBlocks = 4096;                                      // 96 KiB of partials
constexpr int64_t kNoallocMaxN = (int64_t)kNoallocMaxBlocks * kNoallocChunk;  // 16,777,216

static __device__ __align__(256) double g_norms_scratch[3 * kNoallocMaxBlocks];

namespace {
constexpr int kMaxDevicesNoalloc = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevicesNoalloc] = {nullptr};

// Device address of g_norms_scratch on the current device (looked up on first use).
int noalloc_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MLBM_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevicesNoalloc) return fail(MLBM_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_norms_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(MLBM_ECUDA, std::string("cudaGetSymbolAddress(norms scratch): ") + cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = (double *)ptr;
    }
    *out = g_noalloc_ptr[dev];
    return MLBM_OK;
}
}  // namespace

}  // namespace mlbm

using namespace mlbm;

extern "C" {

int mlbm_init(const mlbm_weights *w, const mlbm_params *params, int dtype, const double *rho,
              const double *ux, const double *uy, void *f_out, void *stream) {
    set_error("");
    if (!w || !rho || !ux || !uy || !f_out) return fail(MLBM_EINVAL, "NULL argument");
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "bad dtype");
    cudaStream_t st = (cudaStream_t)stream;
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    int rc = set_params(wm, params, st);
    if (rc) return rc;
    if (dtype == MLBM_F32) {
        int grid = grid_for(w, (const void *)init_kernel<float>, 256, 0);
        init_kernel<float><<<grid, 256, 0, st>>>(w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params, rho, ux,
                                                 uy, (float *)f_out, w->N);
    } else {
        int grid = grid_for(w, (const void *)init_kernel<double>, 256, 0);
        init_kernel<double><<<grid, 256, 0, st>>>(w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params, rho, ux,
                                                  uy, (double *)f_out, w->N);
    }
    return cuda_check_step(cudaGetLastError(), "init_kernel launch");
}

int mlbm_step(const mlbm_weights *w, const mlbm_params *params, int dtype, const void *f_in,
              void *f_out, void *moments, void *stream) {
    set_error("");
    if (!w || !f_in || !f_out) return fail(MLBM_EINVAL, "NULL argument");
    if (f_in == f_out) return fail(MLBM_EINVAL, "f_in and f_out must not alias");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(const_cast<mlbm_weights *>(w), params, st))) return rc;
    return launch_step(w, dtype, f_in, f_out, moments, st);
}

}  // extern "C"

namespace mlbm {
namespace {

// nsteps steps ping-ponging f_a -> f_b -> f_a ... over the first ntiles tiles of a tile table:
// 64-step CUDA graphs (cached per buffers, dtype and tile table prefix) and the remainder as
// single launches.
int run_steps(mlbm_weights *w, int dtype, const TileDev *tiles, int ntiles, void *f_a, void *f_b, int64_t nsteps,
              cudaStream_t st) {
    int rc = MLBM_OK;
    const int64_t G = 64;  // steps per captured graph (even: the graph maps f_a back to f_a)
    int64_t reps = nsteps / G, rem = nsteps % G;
    if (reps > 0) {
        GraphKey key{f_a, f_b, dtype, G, {}, tiles, ntiles};
        cudaGraphExec_t exec = nullptr;
        auto it = w->graphs.find(key);
        if (it != w->graphs.end()) {
            exec = (cudaGraphExec_t)it->second;
        } else {
            cudaStream_t cs;
            if ((rc = cuda_check_step(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream")))
                return rc;
            rc = cuda_check_step(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int64_t i = 0; i < G && !rc; ++i)
                rc = launch_step_tiles(w, dtype, tiles, ntiles, (i & 1) ? f_b : f_a, (i & 1) ? f_a : f_b, nullptr, cs);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &graph);
            if (!rc) rc = cuda_check_step(e, "end capture");
            if (!rc) rc = cuda_check_step(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
            if (rc) return rc;
            w->graphs[key] = (void *)exec;
        }
        for (int64_t r = 0; r < reps; ++r)
            if ((rc = cuda_check_step(cudaGraphLaunch(exec, st), "graph launch"))) return rc;
    }
    for (int64_t i = 0; i < rem; ++i)
        if ((rc = launch_step_tiles(w, dtype, tiles, ntiles, (i & 1) ? f_b : f_a, (i & 1) ? f_a : f_b, nullptr, st)))
            return rc;
    return MLBM_OK;
}

}  // namespace
}  // namespace mlbm

extern "C" {

int mlbm_run(mlbm_weights *w, const mlbm_params *params, int dtype, void *f_a, void *f_b,
             int64_t nsteps, void *stream) {
    set_error("");
    if (!w || !f_a || !f_b) return fail(MLBM_EINVAL, "NULL argument");
    if (f_a == f_b) return fail(MLBM_EINVAL, "f_a and f_b must differ");
    if (nsteps < 0) return fail(MLBM_EINVAL, "nsteps < 0");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(w, params, st))) return rc;
    return run_steps(w, dtype, w->d_tiles, w->ntiles, f_a, f_b, nsteps, st);
}

int mlbm_run_until(mlbm_weights *w, const mlbm_params *params, int dtype, void *f_a, void *f_b,
                   const int64_t *seg_steps, void *stream) {
    set_error("");
    if (!w || !f_a || !f_b || !seg_steps) return fail(MLBM_EINVAL, "NULL argument");
    if (f_a == f_b) return fail(MLBM_EINVAL, "f_a and f_b must differ");
    int64_t S = 0;
    for (int s = 0; s < w->nseg; ++s) {
        if (seg_steps[s] < 0) return fail(MLBM_EINVAL, "negative step count");
        S = std::max(S, seg_steps[s]);
    }
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(w, params, st))) return rc;
    if (S == 0) return MLBM_OK;
    // the tile table sorted by the segments' step counts, longest first (stable: within a count
    // the weights' own order, largest stencils first), so each step's active tiles are a prefix
    if (w->tiles_host.empty()) {
        w->tiles_host.resize((size_t)w->ntiles);
        if ((rc = cuda_check_step(cudaMemcpy(w->tiles_host.data(), w->d_tiles, sizeof(TileDev) * w->ntiles,
                                             cudaMemcpyDeviceToHost), "tile table")))
            return rc;
        if (cudaMalloc(&w->d_tiles_run, sizeof(TileDev) * w->ntiles) != cudaSuccess) {
            cudaGetLastError();
            w->d_tiles_run = nullptr;
            w->tiles_host.clear();
            return fail(MLBM_ENOMEM, "tile table allocation failed");
        }
    }
    std::vector<TileDev> sorted(w->tiles_host);
    std::stable_sort(sorted.begin(), sorted.end(), [&](const TileDev &p, const TileDev &q) {
        return seg_steps[p.seg] > seg_steps[q.seg];
    });
    // stream-ordered: earlier steps still reading the table finish before it changes
    if ((rc = cuda_check_step(cudaMemcpyAsync(w->d_tiles_run, sorted.data(), sizeof(TileDev) * sorted.size(),
                                              cudaMemcpyHostToDevice, st), "tile table")) ||
        (rc = cuda_check_step(cudaStreamSynchronize(st), "tile table")))
        return rc;
    // intervals between the distinct step counts: steps done .. v - 1 run the tiles of the
    // segments with at least v steps
    std::vector<int64_t> ends;
    for (int s = 0; s < w->nseg; ++s)
        if (seg_steps[s] > 0) ends.push_back(seg_steps[s]);
    std::sort(ends.begin(), ends.end());
    ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
    int64_t done = 0;
    for (int64_t v : ends) {
        int active = 0;
        while (active < w->ntiles && seg_steps[sorted[active].seg] >= v) ++active;
        void *cur = (done & 1) ? f_b : f_a, *oth = (done & 1) ? f_a : f_b;
        if ((rc = run_steps(w, dtype, w->d_tiles_run, active, cur, oth, v - done, st))) return rc;
        done = v;
    }
    // a segment that stopped at a step count of the other parity left its state in the other
    // buffer: copy its rows of the nine populations over
    const size_t es = dtype == MLBM_F32 ? sizeof(float) : sizeof(double);
    char *res = (char *)((S & 1) ? f_b : f_a), *other = (char *)((S & 1) ? f_a : f_b);
    for (int s = 0; s < w->nseg; ++s) {
        if (((S - seg_steps[s]) & 1) == 0) continue;
        const SegmentHost &h = w->seg[s];
        if ((rc = cuda_check_step(cudaMemcpy2DAsync(res + h.off * es, w->N * es, other + h.off * es, w->N * es,
                                                    h.n * es, 9, cudaMemcpyDeviceToDevice, st),
                                  "segment state copy")))
            return rc;
    }
    return MLBM_OK;
}

int mlbm_step_host(mlbm_weights *w, const mlbm_params *params, int dtype, int64_t nbatch, const void *const *f_in,
                   void *const *f_out, void *stream) {
    set_error("");
    if (!w || !f_in || !f_out) return fail(MLBM_EINVAL, "NULL argument");
    if (nbatch < 1) return fail(MLBM_EINVAL, "nbatch < 1");
    for (int64_t b = 0; b < nbatch; ++b)
        if (!f_in[b] || !f_out[b]) return fail(MLBM_EINVAL, "NULL state pointer");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(w, params, st))) return rc;
    const size_t bytes = (size_t)9 * w->N * (dtype == MLBM_F32 ? sizeof(float) : sizeof(double));
    // staging buffers and copy streams, kept for later calls
    if (w->stage_bytes < bytes) {
        for (void *&p : w->d_stage) {
            cudaFree(p);
            p = nullptr;
        }
        w->stage_bytes = 0;
        for (void *&p : w->d_stage) {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e == cudaErrorMemoryAllocation) {
                cudaGetLastError();
                return fail(MLBM_ENOMEM, "device allocation of the host-step buffers failed");
            }
            if ((rc = cuda_check_step(e, "host-step buffers"))) return rc;
        }
        w->stage_bytes = bytes;
    }
    for (void *&q : w->copy_stream)
        if (!q && (rc = cuda_check_step(cudaStreamCreateWithFlags((cudaStream_t *)&q, cudaStreamNonBlocking),
                                        "copy stream")))
            return rc;
    for (void *&e : w->stage_event)
        if (!e && (rc = cuda_check_step(cudaEventCreateWithFlags((cudaEvent_t *)&e, cudaEventDisableTiming),
                                        "copy event")))
            return rc;
    cudaStream_t s_in = (cudaStream_t)w->copy_stream[0], s_out = (cudaStream_t)w->copy_stream[1];
    cudaEvent_t *ev = (cudaEvent_t *)w->stage_event;  // [0,1] copied in, [2,3] stepped, [4,5] copied out, [6] start
    // the copies start after the work already queued on the caller's stream
    rc = cuda_check_step(cudaEventRecord(ev[6], st), "event");
    if (!rc) rc = cuda_check_step(cudaStreamWaitEvent(s_in, ev[6], 0), "event wait");
    if (!rc) rc = cuda_check_step(cudaStreamWaitEvent(s_out, ev[6], 0), "event wait");
    // state b uses buffers k = b mod 2: its copy in overlaps the step of b - 1 and the copy out
    // of b - 2
    for (int64_t b = 0; b < nbatch && !rc; ++b) {
        const int k = (int)(b & 1);
        void *din = w->d_stage[k], *dout = w->d_stage[2 + k];
        if (b >= 2) rc = cuda_check_step(cudaStreamWaitEvent(s_in, ev[2 + k], 0), "event wait");
        if (!rc) rc = cuda_check_step(cudaMemcpyAsync(din, f_in[b], bytes, cudaMemcpyHostToDevice, s_in), "copy in");
        if (!rc) rc = cuda_check_step(cudaEventRecord(ev[k], s_in), "event");
        if (!rc) rc = cuda_check_step(cudaStreamWaitEvent(st, ev[k], 0), "event wait");
        if (!rc && b >= 2) rc = cuda_check_step(cudaStreamWaitEvent(st, ev[4 + k], 0), "event wait");
        if (!rc) rc = launch_step(w, dtype, din, dout, nullptr, st);
        if (!rc) rc = cuda_check_step(cudaEventRecord(ev[2 + k], st), "event");
        if (!rc) rc = cuda_check_step(cudaStreamWaitEvent(s_out, ev[2 + k], 0), "event wait");
        if (!rc) rc = cuda_check_step(cudaMemcpyAsync(f_out[b], dout, bytes, cudaMemcpyDeviceToHost, s_out), "copy out");
        if (!rc) rc = cuda_check_step(cudaEventRecord(ev[4 + k], s_out), "event");
    }
    // every copy and step has finished when the call returns
    cudaError_t e1 = cudaStreamSynchronize(s_in), e2 = cudaStreamSynchronize(s_out);
    if (!rc) rc = cuda_check_step(e1, "copy in");
    if (!rc) rc = cuda_check_step(e2, "copy out");
    if (!rc) rc = cuda_check_step(cudaStreamSynchronize(st), "mlbm_step_host");
    return rc;
}

int mlbm_moments(const mlbm_weights *w, const mlbm_params *params, int dtype, const void *f,
                 double *rho, double *ux, double *uy, void *stream) {
    set_error("");
    if (!w || !f || !rho || !ux || !uy) return fail(MLBM_EINVAL, "NULL argument");
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "bad dtype");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = set_params(const_cast<mlbm_weights *>(w), params, st);
    if (rc) return rc;
    if (dtype == MLBM_F32) {
        int grid = grid_for(w, (const void *)moments_kernel<float>, 256, 0);
        moments_kernel<float><<<grid, 256, 0, st>>>(w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params,
                                                    (const float *)f, rho, ux, uy, w->N);
    } else {
        int grid = grid_for(w, (const void *)moments_kernel<double>, 256, 0);
        moments_kernel<double><<<grid, 256, 0, st>>>(w->d_tiles, w->ntiles, w->d_perm, w->d_fdir64, w->d_params,
                                                     (const double *)f, rho, ux, uy, w->N);
    }
    return cuda_check_step(cudaGetLastError(), "moments_kernel launch");
}

int mlbm_norms(const mlbm_weights *w, const double *a, const double *b, const double *c,
               const double *d, int64_t n, double *out, void *stream) {
    set_error("");
    if (!w || !a || !b || !out || n < 0) return fail(MLBM_EINVAL, "bad argument");
    if ((c == nullptr) != (d == nullptr)) return fail(MLBM_EINVAL, "c and d must both be given or both NULL");
    cudaStream_t st = (cudaStream_t)stream;
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    if (!wm->d_partials) {
        cudaError_t e = cudaMalloc((void **)&wm->d_partials, sizeof(double) * (3 * kNormBlocks + 3));
        if (e != cudaSuccess) {
            cudaGetLastError();
            wm->d_partials = nullptr;
            return fail(MLBM_ENOMEM, "scratch allocation failed");
        }
    }
    norms_pass1<<<kNormBlocks, kNormThreads, 0, st>>>(a, b, c, d, n, wm->d_partials);
    norms_pass2<<<1, kNormThreads, 0, st>>>(wm->d_partials, kNormBlocks, wm->d_partials + 3 * kNormBlocks);
    int rc = cuda_check_step(cudaGetLastError(), "norms launch");
    if (rc) return rc;
    rc = cuda_check_step(cudaMemcpyAsync(out, wm->d_partials + 3 * kNormBlocks, 3 * sizeof(double),
                                         cudaMemcpyDeviceToHost, st),
                         "norms copy");
    if (rc) return rc;
    return cuda_check_step(cudaStreamSynchronize(st), "norms");
}

int mlbm_norms_noalloc(const double *a, const double *b, const double *c, const double *d, int64_t n,
                       double *out, void *stream) {
    set_error("");
    if (!a || !b || !out || n < 0) return fail(MLBM_EINVAL, "bad argument");
    if ((c == nullptr) != (d == nullptr)) return fail(MLBM_EINVAL, "c and d must both be given or both NULL");
    if (n > kNoallocMaxN)
        return fail(MLBM_EINVAL, "n = " + std::to_string(n) + " exceeds the limit of mlbm_norms_noalloc (" +
                                     std::to_string(kNoallocMaxN) + " elements); use mlbm_norms");
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::max<int64_t>(1, (n + kNoallocChunk - 1) / kNoallocChunk);
    // every partial slot read by the second pass is written by the first, so nothing to clear
    norms_pass1<<<blocks, kNormThreads, 0, st>>>(a, b, c, d, n, scratch);
    norms_pass2<<<1, kNormThreads, 0, st>>>(scratch, blocks, out);
    return cuda_check_step(cudaGetLastError(), "norms (no allocation) launch");
}

}  // extern "C"
