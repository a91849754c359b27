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
// transposed stencil (for node m, the pairs (i, j) with s_j(i) = m), in a fixed order, so the
// result is deterministic without atomics.  Parameter gradients are reduced per tile and then
// per segment in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "d2q9_device.cuh"
#include "mlbm_internal.h"

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
    const SegDev *__restrict__ seg;
    const TileDev *__restrict__ tiles;
    const int32_t *__restrict__ idx;
    const double *__restrict__ w64;  // canonical [8][K][n] per segment
    const uint16_t *__restrict__ mask;
    const T *__restrict__ fdir;
    const double *__restrict__ params;
    const T *__restrict__ s_prev;
    const T *__restrict__ lam_next;
    T *__restrict__ lam_prev;
    T *__restrict__ mut;    // [8][N] scratch: bounce-back-transposed cotangent of fhat
    T *__restrict__ selfc;  // [8][N] scratch: centre contribution (1 - sum_{j>=1} w) mut
    double *__restrict__ partials;  // [ntiles][2]
    const int32_t *__restrict__ csr_ptr;
    const int32_t *__restrict__ csr_ent;
    int64_t N;
    int ntiles;
};

// Local part of the reverse step at every node: recompute fhat (difference-form interpolation of
// s_prev as in the forward kernel, then bounce-back), apply the transposed collision Jacobian to
// lam_next, then the transposed bounce-back; accumulate dL/dtau and dL/dg per tile.
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_local_kernel(AdjArgs<T> a) {
    constexpr bool kDev = std::is_same<T, float>::value;
    __shared__ double sh[2 * kThreads];
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        double dtau = 0.0, dg = 0.0;
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
            const int64_t p = tile.begin + b;
            const SegDev &sd = a.seg[tile.seg];
            const int64_t n = sd.n, il = p - sd.off, KN = (int64_t)sd.K * n;
            const int K = sd.K;
            T f[9], wsum[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                f[k] = a.s_prev[(int64_t)k * N + p];
                wsum[k] = T(0);
            }
            T acc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = T(0);
            for (int j = 1; j < K; ++j) {
                const int32_t nb = a.idx[sd.idx_off + (int64_t)j * n + il];
                const double *wj = a.w64 + sd.w_off + (int64_t)j * n + il;
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    const T wk = (T)wj[(int64_t)(k - 1) * KN];
                    acc[k] = fma(wk, a.s_prev[(int64_t)k * N + nb] - f[k], acc[k]);
                    wsum[k] += wk;
                }
            }
            if constexpr (kDev) {
                // FP32 forward: difference form, centre coefficient 1 - sum_{j>=1} w
#pragma unroll
                for (int k = 1; k < 9; ++k) f[k] += acc[k];
            } else {
                // FP64 forward: literal form, centre coefficient w_0
                const double *w0 = a.w64 + sd.w_off + il;
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    const T c0 = (T)w0[(int64_t)(k - 1) * KN];
                    f[k] = c0 * f[k] + (acc[k] + wsum[k] * f[k]);
                    wsum[k] = T(1) - c0;
                }
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
            const double *pr = a.params + 4 * tile.seg;
            const T tau = T(pr[0]), inv_tau = T(pr[3]);
            const T rho_ref = kDev ? T(pr[2]) : T(0);
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
            dtau += (double)st / ((double)tau * (double)tau);
            dg += (double)sg;
            T Ar, Ax, Ay;
            feq_vjp<T>(lam, rho, ux, uy, Ar, Ax, Ay);
            const T ir = T(1) / rho;
            T mu[9];
#pragma unroll
            for (int l = 0; l < 9; ++l)
                mu[l] = (T(1) - inv_tau) * lam[l] +
                        inv_tau * (Ar + (Ax * (T(ex_of(l)) - ux) + Ay * (T(ey_of(l)) - uy)) * ir);
            // bounce-back transpose: mut_l = [l not unknown] mu_l + [l' unknown] mu_l'
            T mt[9];
#pragma unroll
            for (int l = 0; l < 9; ++l) {
                T v = (mb >> l & 1u) ? T(0) : mu[l];
                if (l > 0 && (mb >> opp_of(l) & 1u)) v += mu[opp_of(l)];
                mt[l] = v;
            }
            a.lam_prev[p] = mt[0];
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                a.mut[(int64_t)(k - 1) * N + p] = mt[k];
                a.selfc[(int64_t)(k - 1) * N + p] = (T(1) - wsum[k]) * mt[k];
            }
        }
        block_sum2(dtau, dg, sh);
        if (threadIdx.x == 0) {
            a.partials[2 * t] = dtau;
            a.partials[2 * t + 1] = dg;
        }
    }
}

// lam_prev_k(m) = (1 - sum_{j>=1} W_k[j](m)) mut_k(m) + sum over (i, j >= 1) with s_j(i) = m of
// W_k[j](i) mut_k(i), k = 1..8: the transpose of the difference-form interpolation.
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_transpose_kernel(AdjArgs<T> a) {
    const int64_t N = a.N;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDev tile = a.tiles[t];
        for (int b = threadIdx.x; b < tile.count; b += blockDim.x) {
            const int64_t mnode = tile.begin + b;
            const SegDev &sd = a.seg[tile.seg];
            const int64_t n = sd.n, KN = (int64_t)sd.K * n;
            T acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = a.selfc[(int64_t)k * N + mnode];
            const int32_t e0 = a.csr_ptr[mnode], e1 = a.csr_ptr[mnode + 1];
            for (int32_t q = e0; q < e1; ++q) {
                const int32_t ent = a.csr_ent[q];
                if (ent < n) continue;  // member 0: the node itself, counted in selfc
                const int64_t i = sd.off + (int64_t)(ent % n);
                const double *wq = a.w64 + sd.w_off + ent;
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = fma((T)wq[(int64_t)k * KN], a.mut[(int64_t)k * N + i], acc[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) a.lam_prev[(int64_t)(k + 1) * N + mnode] = acc[k];
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
    size_t need = sizeof(double) * (16 * (size_t)w->N + 2 * (size_t)w->ntiles);
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
int adjoint_step_t(mlbm_weights *w, const void *s_prev, const void *lam_next, void *lam_prev, double *grad,
                   cudaStream_t st) {
    AdjArgs<T> a;
    a.seg = w->d_seg;
    a.tiles = w->d_tiles;
    a.idx = w->d_idx;
    a.w64 = w->d_w64;
    a.mask = w->has_mask ? w->d_mask : nullptr;
    a.fdir = std::is_same<T, float>::value ? (const T *)w->d_fdir32 : (const T *)w->d_fdir64;
    a.params = w->d_params;
    a.s_prev = (const T *)s_prev;
    a.lam_next = (const T *)lam_next;
    a.lam_prev = (T *)lam_prev;
    a.mut = (T *)w->d_scratch;
    a.selfc = (T *)w->d_scratch + 8 * (size_t)w->N;
    a.partials = (double *)((char *)w->d_scratch + sizeof(double) * 16 * (size_t)w->N);
    a.csr_ptr = w->d_csr_ptr;
    a.csr_ent = w->d_csr_ent;
    a.N = w->N;
    a.ntiles = w->ntiles;
    adj_local_kernel<T><<<grid_of(w, (const void *)adj_local_kernel<T>), kThreads, 0, st>>>(a);
    adj_transpose_kernel<T><<<grid_of(w, (const void *)adj_transpose_kernel<T>), kThreads, 0, st>>>(a);
    grad_finalize_kernel<<<w->nseg, kThreads, 0, st>>>(w->d_tiles, w->ntiles, a.partials, grad);
    return cuda_check_step(cudaGetLastError(), "adjoint launch");
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" {

int mlbm_adjoint_step(const mlbm_weights *w, const mlbm_params *params, int dtype,
                      const void *s_prev, const void *lam_next, void *lam_prev, double *grad,
                      void *stream) {
    set_error("");
    if (!w || !s_prev || !lam_next || !lam_prev || !grad) return fail(MLBM_EINVAL, "NULL argument");
    if (lam_next == lam_prev) return fail(MLBM_EINVAL, "lam_next and lam_prev must not alias");
    int rc = check_dtype(w, dtype);
    if (rc) return rc;
    if (w->any_nearest)
        return fail(MLBM_EINVAL, "the adjoint step supports own-stencil segments only (MLBM_STENCIL_OWN)");
    mlbm_weights *wm = const_cast<mlbm_weights *>(w);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = set_params(wm, params, st))) return rc;
    if ((rc = ensure_adj_scratch(wm))) return rc;
    return dtype == MLBM_F32 ? adjoint_step_t<float>(wm, s_prev, lam_next, lam_prev, grad, st)
                             : adjoint_step_t<double>(wm, s_prev, lam_next, lam_prev, grad, st);
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
    double *partials = (double *)((char *)wm->d_scratch + sizeof(double) * 16 * (size_t)w->N);
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
    double *partials = (double *)((char *)wm->d_scratch + sizeof(double) * 16 * (size_t)w->N);
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
