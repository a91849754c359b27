// Device build of a node cloud (Sec. 2.2 stencils X^L, Sec. 2.3 departure nodes, Sec. 3 periodic
// stencil search and wall bounce-back): the cloud mlbm_build_cloud makes on the host, bit for bit,
// made on the GPU.
//   * Morton order: 16-bit quantised coordinates interleaved into a 32-bit code, stable LSD radix
//     sort (4 passes of 8 bits) of (code, node) pairs, so equal codes keep the original order.
//   * N_L nearest neighbours by (d^2, original index) over a uniform bucket grid, one thread per
//     query, ring by ring until no unscanned cell can hold a closer node.
//   * departure nodes (nearest-node stencil rule), bounce-back masks, force directions.
//   * the transposed stencil, each row in increasing (member slot, node) order.
// Every floating-point step that decides an index or a mask bit is written with explicitly
// rounded operations (__dmul_rn, __dadd_rn, ...), which the compiler never fuses into an FMA, so it
// rounds exactly as the host build (compiled without contraction) does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "mlbm_internal.h"

namespace mlbm {

int cuda_check_step(cudaError_t e, const char *what);

namespace {

__constant__ int c_ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads = kThreads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 1 << 20));
}

// ---------------------------------------------------------------------------------------------
// Exclusive prefix sum of int32 counts, in place (reduce, scan of the block totals, add).

constexpr int kScanThreads = 1024, kScanItems = 4, kScanChunk = kScanThreads * kScanItems;

// Exclusive scan of one block's chunk; the chunk total goes to block_sum[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) scan_chunk_kernel(int32_t *data, int64_t n, int32_t *block_sum) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        v[t] = base + t < n ? data[base + t] : 0;
        s += v[t];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0, wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31 && block_sum) block_sum[blockIdx.x] = wi;
    }
    __syncthreads();
    int32_t run = warp_tot[warp] + incl - s;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        if (base + t < n) data[base + t] = run;
        run += v[t];
    }
}

__global__ void scan_add_kernel(int32_t *data, int64_t n, const int32_t *block_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) data[i] += block_off[i / kScanChunk];
}

// Scratch ints needed by exclusive_scan for n items.
int64_t scan_scratch(int64_t n) {
    int64_t need = 0;
    while (n > kScanChunk) {
        n = (n + kScanChunk - 1) / kScanChunk;
        need += n;
    }
    return need + 1;
}

void exclusive_scan(int32_t *data, int64_t n, int32_t *scratch, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb == 1) {
        scan_chunk_kernel<<<1, kScanThreads, 0, st>>>(data, n, nullptr);
        return;
    }
    scan_chunk_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, scratch);
    exclusive_scan(scratch, nb, scratch + nb, st);
    scan_add_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(data, n, scratch);
}

// ---------------------------------------------------------------------------------------------
// Stable LSD radix sort of 32-bit keys with an int32 payload, 8 bits per pass.

constexpr int kSortThreads = 256, kSortTiles = 8, kSortChunk = kSortThreads * kSortTiles, kRadix = 256;

// counts[digit * nblk + block] = items of the block's chunk with that digit.
__global__ void __launch_bounds__(kSortThreads) radix_count_kernel(const uint32_t *key, int64_t n, int shift,
                                                                  int32_t *counts, int nblk) {
    __shared__ int32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kSortChunk;
    for (int t = 0; t < kSortTiles; ++t) {
        const int64_t i = b0 + t * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Scatter of one block's chunk to its digit offsets.  Items are ranked in chunk order (tile,
// warp, lane): within a warp by the lanes below with the same digit, across warps by a prefix
// over per-warp digit counts, across tiles by a running offset per digit.  Stable.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint32_t *key_in, const int32_t *val_in,
                                                                    int64_t n, int shift, const int32_t *offsets,
                                                                    int nblk, uint32_t *key_out, int32_t *val_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int32_t base[kRadix];
    __shared__ int32_t wcnt[kWarps][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblk + blockIdx.x];
    const int64_t b0 = (int64_t)blockIdx.x * kSortChunk;
    for (int t = 0; t < kSortTiles; ++t) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = b0 + t * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint32_t k = 0;
        int32_t v = 0;
        int digit = kRadix;  // invalid items form their own group and are dropped
        if (valid) {
            k = key_in[i];
            v = val_in[i];
            digit = (int)((k >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = s;
                s += c;
            }
            // s = items of digit threadIdx.x in this tile; applied after the scatter
            __syncthreads();
            if (valid) {
                const int64_t pos = (int64_t)base[digit] + wcnt[warp][digit] + rank;
                key_out[pos] = k;
                val_out[pos] = v;
            }
            __syncthreads();
            base[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// Sorts (key, val) in place using the second buffers; four passes leave the result in the
// first buffers.
void radix_sort(uint32_t *key, int32_t *val, uint32_t *key2, int32_t *val2, int64_t n, int32_t *counts,
                int32_t *scratch, cudaStream_t st) {
    const int nblk = (int)((n + kSortChunk - 1) / kSortChunk);
    uint32_t *ka = key, *kb = key2;
    int32_t *va = val, *vb = val2;
    for (int shift = 0; shift < 32; shift += 8) {
        radix_count_kernel<<<nblk, kSortThreads, 0, st>>>(ka, n, shift, counts, nblk);
        exclusive_scan(counts, (int64_t)kRadix * nblk, scratch, st);
        radix_scatter_kernel<<<nblk, kSortThreads, 0, st>>>(ka, va, n, shift, counts, nblk, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
}

// ---------------------------------------------------------------------------------------------
// Morton order and the stored arrays.

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// u - L floor(u / L): the coordinate folded into the periodic box [0, L).
__device__ __forceinline__ double fold(double u, double L) { return __dsub_rn(u, __dmul_rn(L, floor(__ddiv_rn(u, L)))); }

// d - L round(d / L): the minimum-image difference (L = 0: none).
__device__ __forceinline__ double min_image(double d, double L) {
    return L > 0.0 ? __dsub_rn(d, __dmul_rn(L, round(__ddiv_rn(d, L)))) : d;
}

struct MortonGeom {
    double x0, y0, sx, sy, lx, ly;
    int periodic;
};

__global__ void morton_kernel(int64_t ns, const double *__restrict__ X, const double *__restrict__ Y, MortonGeom g,
                              uint32_t *__restrict__ key, int32_t *__restrict__ val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        double xx = X[i], yy = Y[i];
        if (g.periodic) {
            xx = fold(xx, g.lx);
            yy = fold(yy, g.ly);
        }
        const double fx = fmin(65535.0, fmax(0.0, floor(__dmul_rn(__dsub_rn(xx, g.x0), g.sx))));
        const double fy = fmin(65535.0, fmax(0.0, floor(__dmul_rn(__dsub_rn(yy, g.y0), g.sy))));
        key[i] = spread16((uint32_t)fx) | (spread16((uint32_t)fy) << 1);
        val[i] = (int32_t)i;
    }
}

// Stored arrays of segment s from the sorted payload: stored position o + p holds original node
// o + val[p].
__global__ void gather_kernel(int64_t ns, int64_t o, int s, const int32_t *__restrict__ val,
                              const double *__restrict__ X, const double *__restrict__ Y, int64_t *__restrict__ perm,
                              double *__restrict__ x, double *__restrict__ y, int32_t *__restrict__ node_seg) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ns; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t src = val[p];
        perm[o + p] = o + src;
        x[o + p] = X[src];
        y[o + p] = Y[src];
        node_seg[o + p] = s;
    }
}

// ---------------------------------------------------------------------------------------------
// Bucket grid and nearest-neighbour queries.

struct GridDev {
    int ncx, ncy;
    double x0, y0, cw, ch, lx, ly;  // lx = ly = 0 unless periodic
    int periodic;
    const int32_t *start;  // [ncx*ncy + 1]
    const int32_t *items;  // segment-local stored indices, bucketed by cell
};

__device__ __forceinline__ int cell_x(const GridDev &g, double x) {
    double u = g.periodic ? fold(x, g.lx) : x;
    const double c = floor(__ddiv_rn(__dsub_rn(u, g.x0), g.cw));
    return (int)fmin(fmax(c, 0.0), (double)(g.ncx - 1));
}

__device__ __forceinline__ int cell_y(const GridDev &g, double y) {
    double u = g.periodic ? fold(y, g.ly) : y;
    const double c = floor(__ddiv_rn(__dsub_rn(u, g.y0), g.ch));
    return (int)fmin(fmax(c, 0.0), (double)(g.ncy - 1));
}

__global__ void cell_count_kernel(int64_t ns, const double *__restrict__ x, const double *__restrict__ y, GridDev g,
                                  int32_t *__restrict__ cell, int32_t *__restrict__ count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell_y(g, y[i]) * g.ncx + cell_x(g, x[i]);
        cell[i] = c;
        atomicAdd(&count[c], 1);
    }
}

// Bucket fill; the order inside a cell does not matter (queries rank by a total order).
__global__ void cell_fill_kernel(int64_t ns, const int32_t *__restrict__ cell, const int32_t *__restrict__ start,
                                 int32_t *__restrict__ cursor, int32_t *__restrict__ items) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[i];
        items[start[c] + atomicAdd(&cursor[c], 1)] = (int32_t)i;
    }
}

// The K nodes nearest to (qx, qy) by (d^2, original index), d the minimum-image difference in a
// periodic segment; out[j * stride] = segment-local stored index of the j-th.  KC >= K bounds
// the candidate list held in registers / local memory.
#pragma nv_diag_suppress 549  // the candidate lists are read only once filled (cnt == K)
template <int KC>
__device__ void knn(const GridDev &g, const double *__restrict__ x, const double *__restrict__ y,
                    const int32_t *__restrict__ orig, double qx, double qy, int K, int32_t *out, int64_t stride) {
    double bd[KC];
    int32_t bo[KC], bl[KC];
    int cnt = 0;
    auto consider = [&](int32_t j) {
        const double dx = min_image(__dsub_rn(x[j], qx), g.lx);
        const double dy = min_image(__dsub_rn(y[j], qy), g.ly);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const int32_t o = orig[j];
        if (cnt == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && o > bo[K - 1]))) return;
        int pos = cnt < K ? cnt : K - 1;
        while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bo[pos - 1] > o))) {
            bd[pos] = bd[pos - 1];
            bo[pos] = bo[pos - 1];
            bl[pos] = bl[pos - 1];
            --pos;
        }
        bd[pos] = d2;
        bo[pos] = o;
        bl[pos] = j;
        if (cnt < K) ++cnt;
    };
    auto scan_cell = [&](int cx, int cy) {
        const int c = cy * g.ncx + cx;
        const int32_t e = g.start[c + 1];
        for (int32_t t = g.start[c]; t < e; ++t) consider(g.items[t]);
    };
    const int cx = cell_x(g, qx), cy = cell_y(g, qy);
    const double ux = g.periodic ? fold(qx, g.lx) : qx, uy = g.periodic ? fold(qy, g.ly) : qy;
    for (int ring = 0;; ++ring) {
        const bool full = g.periodic ? (2 * ring + 1 >= g.ncx || 2 * ring + 1 >= g.ncy)
                                     : (ring > g.ncx && ring > g.ncy);
        if (full && g.periodic) {
            // the block of scanned cells wraps onto itself: scan every cell once
            cnt = 0;
            for (int yy = 0; yy < g.ncy; ++yy)
                for (int xx = 0; xx < g.ncx; ++xx) scan_cell(xx, yy);
            break;
        }
        if (full) break;
        // the cells at Chebyshev distance `ring` from (cx, cy): whole top and bottom rows, the two
        // end cells of the rows between
        for (int dy = -ring; dy <= ring; ++dy) {
            const bool edge_row = dy == -ring || dy == ring;
            for (int dx = -ring; dx <= ring; dx += edge_row ? 1 : 2 * ring) {
                int xx = cx + dx, yy = cy + dy;
                if (g.periodic) {
                    xx = ((xx % g.ncx) + g.ncx) % g.ncx;
                    yy = ((yy % g.ncy) + g.ncy) % g.ncy;
                } else if (xx < 0 || yy < 0 || xx >= g.ncx || yy >= g.ncy) {
                    continue;
                }
                scan_cell(xx, yy);
            }
        }
        if (cnt == K) {
            const double bx0 = __dadd_rn(g.x0, __dmul_rn((double)(cx - ring), g.cw));
            const double bx1 = __dadd_rn(g.x0, __dmul_rn((double)(cx + ring + 1), g.cw));
            const double by0 = __dadd_rn(g.y0, __dmul_rn((double)(cy - ring), g.ch));
            const double by1 = __dadd_rn(g.y0, __dmul_rn((double)(cy + ring + 1), g.ch));
            const double dmin = fmin(fmin(__dsub_rn(ux, bx0), __dsub_rn(bx1, ux)),
                                     fmin(__dsub_rn(uy, by0), __dsub_rn(by1, uy)));
            if (dmin > 0 && __dmul_rn(dmin, dmin) > __dmul_rn(bd[K - 1], 1.0 + 1e-12)) break;
        }
    }
    for (int j = 0; j < K; ++j) out[j * stride] = bl[j];
}

// Stencils of segment s: idx[j * ns + i] = o + (j-th nearest node of node i); a node that is not
// the first member of its own stencil (a duplicate position) raises *dup.
template <int KC>
__global__ void __launch_bounds__(128) stencil_kernel(int64_t ns, int64_t o, int K, GridDev g,
                                                      const double *__restrict__ x, const double *__restrict__ y,
                                                      const int32_t *__restrict__ orig, int32_t *__restrict__ idx,
                                                      int32_t *__restrict__ dup) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int32_t *out = idx + i;
    knn<KC>(g, x, y, orig, x[i], y[i], K, out, ns);
    const int32_t first = out[0];
    for (int j = 0; j < K; ++j) out[(int64_t)j * ns] += (int32_t)o;
    if (first != (int32_t)i) atomicExch(dup, 1);
}

// Departure nodes (nearest-node stencil rule): near[(k-1) * ns + i] = o + the node nearest to
// x_i - e_k dx_ml, k = 1..8.
__global__ void __launch_bounds__(128) departure_kernel(int64_t ns, int64_t o, double dx_ml, GridDev g,
                                                        const double *__restrict__ x, const double *__restrict__ y,
                                                        const int32_t *__restrict__ orig, int32_t *__restrict__ near) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * ns) return;
    const int k = 1 + (int)(t / ns);
    const int64_t i = t - (int64_t)(k - 1) * ns;
    const double qx = __dsub_rn(x[i], __dmul_rn((double)c_ex[k], dx_ml));
    const double qy = __dsub_rn(y[i], __dmul_rn((double)c_ey[k], dx_ml));
    int32_t nn;
    knn<1>(g, x, y, orig, qx, qy, 1, &nn, 1);
    near[t] = (int32_t)(o + nn);
}

// Own-stencil segments: every departure node is the node itself.
__global__ void own_departure_kernel(int64_t ns, int64_t o, int32_t *__restrict__ near) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 8 * ns; t += (int64_t)gridDim.x * blockDim.x)
        near[t] = (int32_t)(o + t % ns);
}

// Bounce-back mask and force direction (Sec. 3).  Annulus: bit k set when the departure point
// x_i - e_k dx_ml lies outside r_in <= r <= r_out (relative slack 1e-12 on r^2); force direction
// the azimuthal unit vector (-y, x) / r.  Periodic box: no walls, force along +x.
__global__ void mask_kernel(int64_t ns, int64_t o, int64_t N, mlbm_segment_desc d, const double *__restrict__ x,
                            const double *__restrict__ y, uint16_t *__restrict__ mask, double *__restrict__ fdir) {
    const bool annulus = d.geometry == MLBM_GEOM_ANNULUS;
    const double lo = __dmul_rn(__dmul_rn(d.r_in, d.r_in), 1.0 - 1e-12);
    const double hi = __dmul_rn(__dmul_rn(d.r_out, d.r_out), 1.0 + 1e-12);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const double xx = x[o + i], yy = y[o + i];
        uint16_t m = 0;
        double fx = 1.0, fy = 0.0;
        if (annulus) {
#pragma unroll
            for (int k = 1; k < kQ; ++k) {
                const double Dx = __dsub_rn(xx, __dmul_rn((double)c_ex[k], d.dx_ml));
                const double Dy = __dsub_rn(yy, __dmul_rn((double)c_ey[k], d.dx_ml));
                const double r2 = __dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy));
                if (r2 < lo || r2 > hi) m |= (uint16_t)(1u << k);
            }
            const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(xx, xx), __dmul_rn(yy, yy)));
            fx = r > 0 ? __ddiv_rn(-yy, r) : 0.0;
            fy = r > 0 ? __ddiv_rn(xx, r) : 0.0;
        }
        mask[o + i] = m;
        fdir[o + i] = fx;
        fdir[N + o + i] = fy;
    }
}

// ---------------------------------------------------------------------------------------------
// Transposed stencil: row m lists the entries t = j * ns + i (member slot j of node i) with
// idx[t] = o + m, in increasing t.

__global__ void csr_count_kernel(int64_t nt, int64_t o, const int32_t *__restrict__ idx, int32_t *__restrict__ cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[idx[t] - o], 1);
}

__global__ void csr_fill_kernel(int64_t nt, int64_t o, const int32_t *__restrict__ idx, const int32_t *__restrict__ rs,
                                int32_t *__restrict__ cursor, int32_t *__restrict__ ent) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = idx[t] - o;
        ent[rs[m] + atomicAdd(&cursor[m], 1)] = (int32_t)t;
    }
}

// Rows into increasing order (insertion sort; rows hold about N_L entries), and the global row
// pointers ptr[o + m] = csr_off + rs[m], m = 0..ns.
__global__ void csr_sort_kernel(int64_t ns, int64_t o, int64_t csr_off, const int32_t *__restrict__ rs,
                                int32_t *__restrict__ ent, int32_t *__restrict__ ptr) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m <= ns; m += (int64_t)gridDim.x * blockDim.x) {
        ptr[o + m] = (int32_t)(csr_off + rs[m]);
        if (m == ns) continue;
        int32_t *row = ent + rs[m];
        const int len = rs[m + 1] - rs[m];
        for (int a = 1; a < len; ++a) {
            const int32_t v = row[a];
            int b = a;
            while (b > 0 && row[b - 1] > v) {
                row[b] = row[b - 1];
                --b;
            }
            row[b] = v;
        }
    }
}

// ---------------------------------------------------------------------------------------------

struct DevMem {
    std::vector<void *> p;
    ~DevMem() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(int64_t n, cudaError_t &err) {
        void *q = nullptr;
        if (err == cudaSuccess) err = cudaMalloc(&q, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
        if (err == cudaSuccess) p.push_back(q);
        return (T *)q;
    }
};

#define MLBM_TRY(expr, what)                                       \
    do {                                                           \
        int rc_ = cuda_check_step((expr), what);                   \
        if (rc_) return rc_;                                       \
    } while (0)

template <int KC>
void launch_stencil(int64_t ns, int64_t o, int K, const GridDev &g, const double *x, const double *y,
                    const int32_t *orig, int32_t *idx, int32_t *dup, cudaStream_t st) {
    stencil_kernel<KC><<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(ns, o, K, g, x, y, orig, idx, dup);
}

int build_on_device(mlbm_cloud *c, const double *xy, cudaStream_t st) {
    const int64_t n = c->N;
    int64_t nsmax = 0;
    for (const SegmentHost &sh : c->seg) nsmax = std::max(nsmax, sh.n);
    // bucket grids of every segment (host arithmetic, identical to the host build's)
    std::vector<GridGeom> geo(c->nseg);
    std::vector<BBox> box(c->nseg);
    int64_t cells_max = 1;
    for (int s = 0; s < c->nseg; ++s) {
        const SegmentHost &sh = c->seg[s];
        box[s] = segment_bbox(xy + sh.off, xy + n + sh.off, sh.n, sh.d);
        geo[s] = grid_geom(sh.n, box[s], sh.d);
        cells_max = std::max(cells_max, (int64_t)geo[s].ncx * geo[s].ncy);
    }
    const int64_t nblk_max = (nsmax + kSortChunk - 1) / kSortChunk;
    const int64_t scan_max = std::max({(int64_t)kRadix * nblk_max, cells_max + 1, nsmax + 1});

    cudaError_t err = cudaSuccess;
    DevMem mem;
    double *d_xy = mem.get<double>(2 * n, err);
    double *d_x = mem.get<double>(n, err), *d_y = mem.get<double>(n, err);
    int64_t *d_perm = mem.get<int64_t>(n, err);
    int32_t *d_node_seg = mem.get<int32_t>(n, err);
    int32_t *d_idx = mem.get<int32_t>(c->idx_total, err);
    int32_t *d_near = mem.get<int32_t>(8 * n, err);
    uint16_t *d_mask = mem.get<uint16_t>(n, err);
    double *d_fdir = mem.get<double>(2 * n, err);
    int32_t *d_ptr = mem.get<int32_t>(n + 1, err);
    int32_t *d_ent = mem.get<int32_t>(c->idx_total, err);
    uint32_t *d_key = mem.get<uint32_t>(nsmax, err), *d_key2 = mem.get<uint32_t>(nsmax, err);
    int32_t *d_val = mem.get<int32_t>(nsmax, err), *d_val2 = mem.get<int32_t>(nsmax, err);
    int32_t *d_counts = mem.get<int32_t>(scan_max, err);
    int32_t *d_scan = mem.get<int32_t>(scan_scratch(scan_max), err);
    int32_t *d_cell = mem.get<int32_t>(nsmax, err);
    int32_t *d_start = mem.get<int32_t>(cells_max + 1, err);
    int32_t *d_cursor = mem.get<int32_t>(std::max(cells_max, nsmax) + 1, err);
    int32_t *d_items = mem.get<int32_t>(nsmax, err);
    int32_t *d_rs = mem.get<int32_t>(nsmax + 1, err);
    int32_t *d_dup = mem.get<int32_t>(1, err);
    if (err == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(MLBM_ENOMEM, "device allocation failed in the device cloud build");
    }
    MLBM_TRY(err, "device cloud build allocation");
    MLBM_TRY(cudaMemcpyAsync(d_xy, xy, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st), "coordinate upload");
    MLBM_TRY(cudaMemsetAsync(d_dup, 0, sizeof(int32_t), st), "memset");

    for (int s = 0; s < c->nseg; ++s) {
        const SegmentHost &sh = c->seg[s];
        const mlbm_segment_desc &d = sh.d;
        const int64_t ns = sh.n, o = sh.off;
        const double *X = d_xy + o, *Y = d_xy + n + o;
        // Morton order
        const BBox &bb = box[s];
        MortonGeom mg;
        mg.x0 = bb.x0;
        mg.y0 = bb.y0;
        mg.sx = (bb.x1 > bb.x0) ? 65536.0 / (bb.x1 - bb.x0) : 0.0;
        mg.sy = (bb.y1 > bb.y0) ? 65536.0 / (bb.y1 - bb.y0) : 0.0;
        mg.lx = d.lx;
        mg.ly = d.ly;
        mg.periodic = d.geometry == MLBM_GEOM_PERIODIC;
        morton_kernel<<<grid_for(ns), kThreads, 0, st>>>(ns, X, Y, mg, d_key, d_val);
        radix_sort(d_key, d_val, d_key2, d_val2, ns, d_counts, d_scan, st);
        gather_kernel<<<grid_for(ns), kThreads, 0, st>>>(ns, o, s, d_val, X, Y, d_perm, d_x, d_y, d_node_seg);
        // bucket grid over the stored order
        const GridGeom &gg = geo[s];
        const int64_t cells = (int64_t)gg.ncx * gg.ncy;
        GridDev g;
        g.ncx = gg.ncx;
        g.ncy = gg.ncy;
        g.x0 = gg.x0;
        g.y0 = gg.y0;
        g.cw = gg.cw;
        g.ch = gg.ch;
        g.periodic = gg.periodic;
        g.lx = gg.periodic ? gg.lx : 0.0;
        g.ly = gg.periodic ? gg.ly : 0.0;
        g.start = d_start;
        g.items = d_items;
        MLBM_TRY(cudaMemsetAsync(d_start, 0, sizeof(int32_t) * (cells + 1), st), "memset");
        MLBM_TRY(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * cells, st), "memset");
        cell_count_kernel<<<grid_for(ns), kThreads, 0, st>>>(ns, d_x + o, d_y + o, g, d_cell, d_start);
        exclusive_scan(d_start, cells + 1, d_scan, st);
        cell_fill_kernel<<<grid_for(ns), kThreads, 0, st>>>(ns, d_cell, d_start, d_cursor, d_items);
        // stencils (d_val holds the original index, segment-local, of each stored node)
        int32_t *idx = d_idx + sh.idx_off;
        const int K = sh.K;
        if (K <= 16)
            launch_stencil<16>(ns, o, K, g, d_x + o, d_y + o, d_val, idx, d_dup, st);
        else if (K <= 32)
            launch_stencil<32>(ns, o, K, g, d_x + o, d_y + o, d_val, idx, d_dup, st);
        else if (K <= 64)
            launch_stencil<64>(ns, o, K, g, d_x + o, d_y + o, d_val, idx, d_dup, st);
        else
            launch_stencil<kMaxK>(ns, o, K, g, d_x + o, d_y + o, d_val, idx, d_dup, st);
        // departure nodes
        if (d.stencil_mode == MLBM_STENCIL_NEAREST)
            departure_kernel<<<(unsigned)((8 * ns + 127) / 128), 128, 0, st>>>(ns, o, d.dx_ml, g, d_x + o, d_y + o,
                                                                             d_val, d_near + 8 * o);
        else
            own_departure_kernel<<<grid_for(8 * ns), kThreads, 0, st>>>(ns, o, d_near + 8 * o);
        mask_kernel<<<grid_for(ns), kThreads, 0, st>>>(ns, o, n, d, d_x, d_y, d_mask, d_fdir);
        // transposed stencil
        const int64_t nt = (int64_t)K * ns;
        MLBM_TRY(cudaMemsetAsync(d_rs, 0, sizeof(int32_t) * (ns + 1), st), "memset");
        MLBM_TRY(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * ns, st), "memset");
        csr_count_kernel<<<grid_for(nt), kThreads, 0, st>>>(nt, o, idx, d_rs);
        exclusive_scan(d_rs, ns + 1, d_scan, st);
        csr_fill_kernel<<<grid_for(nt), kThreads, 0, st>>>(nt, o, idx, d_rs, d_cursor, d_ent + sh.csr_off);
        csr_sort_kernel<<<grid_for(ns + 1), kThreads, 0, st>>>(ns, o, sh.csr_off, d_rs, d_ent + sh.csr_off, d_ptr);
        MLBM_TRY(cudaGetLastError(), "device cloud build launch");
    }
    int32_t dup = 0;
    MLBM_TRY(cudaMemcpyAsync(&dup, d_dup, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->x.data(), d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->y.data(), d_y, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->perm.data(), d_perm, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->node_seg.data(), d_node_seg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st),
             "download");
    MLBM_TRY(cudaMemcpyAsync(c->idx.data(), d_idx, sizeof(int32_t) * c->idx_total, cudaMemcpyDeviceToHost, st),
             "download");
    MLBM_TRY(cudaMemcpyAsync(c->near.data(), d_near, sizeof(int32_t) * 8 * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->mask.data(), d_mask, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->fdir.data(), d_fdir, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st), "download");
    MLBM_TRY(cudaMemcpyAsync(c->csr_ptr.data(), d_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st),
             "download");
    MLBM_TRY(cudaMemcpyAsync(c->csr_ent.data(), d_ent, sizeof(int32_t) * c->idx_total, cudaMemcpyDeviceToHost, st),
             "download");
    MLBM_TRY(cudaStreamSynchronize(st), "device cloud build");
    if (dup) {
        for (int s = 0; s < c->nseg; ++s) {
            const SegmentHost &sh = c->seg[s];
            for (int64_t i = 0; i < sh.n; ++i)
                if (c->idx[sh.idx_off + i] != (int32_t)(sh.off + i))
                    return fail(MLBM_EINVAL, "duplicate nodes in segment " + std::to_string(s) +
                                                 " (a node must be the first member of its own stencil)");
        }
        return fail(MLBM_EINVAL, "duplicate nodes");
    }
    return MLBM_OK;
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" int mlbm_build_cloud_device(const double *xy, int64_t n, const mlbm_segment_desc *segs,
                                       const int64_t *seg_offsets, int nseg, void *stream, mlbm_cloud **out) {
    set_error("");
    if (!out) return fail(MLBM_EINVAL, "out is NULL");
    *out = nullptr;
    int64_t idx_total = 0, w_total = 0;
    int rc = check_cloud_args(xy, n, segs, seg_offsets, nseg, &idx_total, &w_total);
    if (rc) return rc;
    mlbm_cloud *c = nullptr;
    try {
        c = new_cloud(n, segs, seg_offsets, nseg, idx_total, w_total);
    } catch (const std::bad_alloc &) {
        return fail(MLBM_ENOMEM, "host allocation failed");
    }
    rc = build_on_device(c, xy, (cudaStream_t)stream);
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return MLBM_OK;
}
