// Standard lattice LBM on a periodic nx x ny lattice (Sec. 2.1): the special case of the method
// where nodes sit on a lattice with spacing dx_ml and streaming is the index shift of
// eq. (LBM_streaming), f_k(x) <- f^post_k(x - e_k).  Same state conventions as the meshless
// step (post-collision state, FP32 deviations f - omega_k rho0 or FP64 populations, SoA
// [9][nx*ny] with node index iy * nx + ix) and the same collision code.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "d2q9_device.cuh"
#include "mlbm_internal.h"

namespace mlbm {

int cuda_check_step(cudaError_t e, const char *what);

namespace {

struct LatticeParams {
    double tau, g, rho0, inv_tau;  // inv_tau = 1 / tau, computed once on the host
    float g32, rho032, inv_tau32;  // FP32 copies (no per-node conversion on the FP64 unit)
};

// One pull step: gather the eight moving populations from the upstream neighbours (periodic
// wrap), collide (BGK + forcing along +x), store.  2-D launch: threads along x within one
// lattice row (blockIdx.y = row), so every gather of a direction is a contiguous run of the
// source row, shifted by at most one element.
template <typename T>
__global__ void __launch_bounds__(256) lattice_step_kernel(int64_t nx, int64_t ny, LatticeParams prm,
                                                           const T *__restrict__ fin, T *__restrict__ fout,
                                                           T *__restrict__ mom) {
    const int64_t N = nx * ny;
    const T inv_tau = std::is_same<T, float>::value ? T(prm.inv_tau32) : T(prm.inv_tau);
    const T rho_ref = std::is_same<T, float>::value ? T(prm.rho032) : T(0);
    const T gx = std::is_same<T, float>::value ? T(prm.g32) : T(prm.g), gy = T(0);
    const int64_t iy = blockIdx.y;
    const int64_t rowm = (iy == 0 ? ny - 1 : iy - 1) * nx;  // row iy - 1
    const int64_t row0 = iy * nx;
    const int64_t rowp = (iy == ny - 1 ? 0 : iy + 1) * nx;  // row iy + 1
    for (int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ix < nx; ix += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xm = ix == 0 ? nx - 1 : ix - 1, xp = ix == nx - 1 ? 0 : ix + 1;
        const int64_t i = row0 + ix;
        T f[9];
        // source of population k at (ix, iy) is (ix - ex_k, iy - ey_k)
        f[0] = __ldg(fin + i);
        f[1] = __ldg(fin + 1 * N + row0 + xm);
        f[2] = __ldg(fin + 2 * N + rowm + ix);
        f[3] = __ldg(fin + 3 * N + row0 + xp);
        f[4] = __ldg(fin + 4 * N + rowp + ix);
        f[5] = __ldg(fin + 5 * N + rowm + xm);
        f[6] = __ldg(fin + 6 * N + rowm + xp);
        f[7] = __ldg(fin + 7 * N + rowp + xp);
        f[8] = __ldg(fin + 8 * N + rowp + xm);
        T rho, ux, uy;
        if constexpr (std::is_same<T, float>::value)
            collide_projected<false>(f, rho_ref, inv_tau, gx, gy, rho, ux, uy);
        else
            collide<T>(f, rho_ref, inv_tau, gx, gy, rho, ux, uy);
#pragma unroll
        for (int k = 0; k < 9; ++k) fout[(int64_t)k * N + i] = f[k];
        if (mom) {
            mom[i] = rho;
            mom[N + i] = ux;
            mom[2 * N + i] = uy;
        }
    }
}

// FP32 step with four consecutive nodes of a row per thread (nx a multiple of 4, 16-byte aligned
// arrays): every direction is one 16-byte load of the source row; the x-shifted directions take
// the one value that crosses into the neighbouring quad from the adjacent lane by a shuffle,
// and only the edge lanes of a warp (or the row's end, with periodic wrap) load it themselves.
// blockIdx.y = row; all 32 lanes of a warp stay in the loop so the shuffles see every lane.
__global__ void __launch_bounds__(256) lattice_step4_kernel(int nx, int ny, LatticeParams prm,
                                                            const float *__restrict__ fin,
                                                            float *__restrict__ fout, float *__restrict__ mom) {
    const int64_t N = (int64_t)nx * ny;
    const int nq = nx >> 2;
    const int iy = blockIdx.y;
    const int64_t rowm = (int64_t)(iy == 0 ? ny - 1 : iy - 1) * nx, row0 = (int64_t)iy * nx;
    const int64_t rowp = (int64_t)(iy == ny - 1 ? 0 : iy + 1) * nx;
    const int lane = threadIdx.x & 31;
    for (int q0 = blockIdx.x * blockDim.x; q0 < nq; q0 += gridDim.x * blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool valid = q < nq;
        const int x0 = (valid ? q : nq - 1) << 2;
        // source rows of each direction: k with ey = +1 read row iy - 1, ey = -1 read row iy + 1
        auto ld4 = [&](int k, int64_t row) {
            return __ldg(reinterpret_cast<const float4 *>(fin + (size_t)k * N + row + x0));
        };
        auto ld1 = [&](int k, int64_t row, int x) {
            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            return __ldg(fin + (size_t)k * N + row + x);
        };
        // ex = +1: value at x0 - 1 from the previous lane's last element; ex = -1: value at x0 + 4
        // from the next lane's first element
        auto prev = [&](const float4 &v, int k, int64_t row) {
            float p = __shfl_up_sync(0xffffffffu, v.w, 1);
            if (lane == 0 || !valid) p = ld1(k, row, x0 - 1);
            return p;
        };
        auto next = [&](const float4 &v, int k, int64_t row) {
            float n = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (lane == 31 || x0 + 4 >= nx || !valid) n = ld1(k, row, x0 + 4);
            return n;
        };
        const float4 a0 = ld4(0, row0), a1 = ld4(1, row0), a2 = ld4(2, rowm), a3 = ld4(3, row0), a4 = ld4(4, rowp);
        const float4 a5 = ld4(5, rowm), a6 = ld4(6, rowm), a7 = ld4(7, rowp), a8 = ld4(8, rowp);
        const float p1 = prev(a1, 1, row0), p5 = prev(a5, 5, rowm), p8 = prev(a8, 8, rowp);
        const float n3 = next(a3, 3, row0), n6 = next(a6, 6, rowm), n7 = next(a7, 7, rowp);
        // population k of node x0 + r comes from x0 + r - ex_k
        const float f1[4] = {p1, a1.x, a1.y, a1.z}, f5[4] = {p5, a5.x, a5.y, a5.z}, f8[4] = {p8, a8.x, a8.y, a8.z};
        const float f3[4] = {a3.y, a3.z, a3.w, n3}, f6[4] = {a6.y, a6.z, a6.w, n6}, f7[4] = {a7.y, a7.z, a7.w, n7};
        const float f0[4] = {a0.x, a0.y, a0.z, a0.w}, f2[4] = {a2.x, a2.y, a2.z, a2.w}, f4[4] = {a4.x, a4.y, a4.z, a4.w};
        float o[9][4], m[3][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float f[9] = {f0[r], f1[r], f2[r], f3[r], f4[r], f5[r], f6[r], f7[r], f8[r]};
            float rho, ux, uy;
            collide_projected<false>(f, prm.rho032, prm.inv_tau32, prm.g32, 0.0f, rho, ux, uy);
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k][r] = f[k];
            m[0][r] = rho;
            m[1][r] = ux;
            m[2][r] = uy;
        }
        if (valid) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                *reinterpret_cast<float4 *>(fout + (size_t)k * N + row0 + x0) = make_float4(o[k][0], o[k][1], o[k][2], o[k][3]);
            if (mom) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<float4 *>(mom + (size_t)c * N + row0 + x0) = make_float4(m[c][0], m[c][1], m[c][2], m[c][3]);
            }
        }
    }
}

// Equilibrium at (rho, u) plus the forcing term, as mlbm_init, in lattice order.
template <typename T>
__global__ void lattice_init_kernel(int64_t N, LatticeParams prm, const double *__restrict__ rho_in,
                                    const double *__restrict__ ux_in, const double *__restrict__ uy_in,
                                    T *__restrict__ f) {
    const double rho_ref = std::is_same<T, float>::value ? prm.rho0 : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double rho = rho_in[i], ux = ux_in[i], uy = uy_in[i];
        const double usq15 = 1.5 * (ux * ux + uy * uy);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            f[(int64_t)k * N + i] = (T)(geq_of<double>(k, rho - rho_ref, rho, ux, uy, usq15) +
                                        omega_of<double>(k) * 3.0 * ex_of(k) * prm.g);
    }
}

int lattice_grid(const void *fn, int64_t N) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
    const int64_t need = (N + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(1, per_sm) * sms));
}

int check_lattice_args(int64_t nx, int64_t ny, const mlbm_params *params, int dtype) {
    if (nx < 1 || ny < 1 || nx > (1LL << 31) / ny) return fail(MLBM_EINVAL, "bad lattice size");
    if (!params) return fail(MLBM_EINVAL, "params is NULL");
    if (!(params->tau > 0.5)) return fail(MLBM_EINVAL, "tau must be > 0.5 (positive viscosity)");
    if (dtype != MLBM_F32 && dtype != MLBM_F64) return fail(MLBM_EINVAL, "bad dtype");
    return MLBM_OK;
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" {

int mlbm_lattice_init(int64_t nx, int64_t ny, const mlbm_params *params, int dtype, const double *rho,
                      const double *ux, const double *uy, void *f_out, void *stream) {
    set_error("");
    int rc = check_lattice_args(nx, ny, params, dtype);
    if (rc) return rc;
    if (!rho || !ux || !uy || !f_out) return fail(MLBM_EINVAL, "NULL argument");
    const int64_t N = nx * ny;
    LatticeParams prm{params->tau, params->g, params->rho0, 1.0 / params->tau, (float)params->g,
                      (float)params->rho0, (float)(1.0 / params->tau)};
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MLBM_F32)
        lattice_init_kernel<float><<<lattice_grid((const void *)lattice_init_kernel<float>, N), 256, 0, st>>>(
            N, prm, rho, ux, uy, (float *)f_out);
    else
        lattice_init_kernel<double><<<lattice_grid((const void *)lattice_init_kernel<double>, N), 256, 0, st>>>(
            N, prm, rho, ux, uy, (double *)f_out);
    return cuda_check_step(cudaGetLastError(), "lattice_init launch");
}

int mlbm_lattice_step(int64_t nx, int64_t ny, const mlbm_params *params, int dtype, const void *f_in,
                      void *f_out, void *moments, void *stream) {
    set_error("");
    int rc = check_lattice_args(nx, ny, params, dtype);
    if (rc) return rc;
    if (!f_in || !f_out) return fail(MLBM_EINVAL, "NULL argument");
    if (f_in == f_out) return fail(MLBM_EINVAL, "f_in and f_out must not alias");
    LatticeParams prm{params->tau, params->g, params->rho0, 1.0 / params->tau, (float)params->g,
                      (float)params->rho0, (float)(1.0 / params->tau)};
    cudaStream_t st = (cudaStream_t)stream;
    if (ny > 65535) return fail(MLBM_EINVAL, "lattice step supports ny <= 65535");
    const dim3 grid((unsigned)std::min<int64_t>((nx + 255) / 256, 1 << 16), (unsigned)ny);
    const bool aligned = ((uintptr_t)f_in | (uintptr_t)f_out | (uintptr_t)moments) % 16 == 0;
    if (dtype == MLBM_F32 && nx % 4 == 0 && aligned) {
        const dim3 g4((unsigned)std::min<int64_t>((nx / 4 + 255) / 256, 1 << 16), (unsigned)ny);
        lattice_step4_kernel<<<g4, 256, 0, st>>>((int)nx, (int)ny, prm, (const float *)f_in, (float *)f_out,
                                                 (float *)moments);
    } else if (dtype == MLBM_F32)
        lattice_step_kernel<float><<<grid, 256, 0, st>>>(nx, ny, prm, (const float *)f_in, (float *)f_out,
                                                         (float *)moments);
    else
        lattice_step_kernel<double><<<grid, 256, 0, st>>>(nx, ny, prm, (const double *)f_in, (double *)f_out,
                                                          (double *)moments);
    return cuda_check_step(cudaGetLastError(), "lattice_step launch");
}

}  // extern "C"
