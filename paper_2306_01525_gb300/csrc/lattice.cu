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
            collide_projected(f, rho_ref, inv_tau, gx, gy, rho, ux, uy);
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
    if (dtype == MLBM_F32)
        lattice_step_kernel<float><<<grid, 256, 0, st>>>(nx, ny, prm, (const float *)f_in, (float *)f_out,
                                                         (float *)moments);
    else
        lattice_step_kernel<double><<<grid, 256, 0, st>>>(nx, ny, prm, (const double *)f_in, (double *)f_out,
                                                          (double *)moments);
    return cuda_check_step(cudaGetLastError(), "lattice_step launch");
}

}  // extern "C"
