// Internal structures of the GB300 meshless LBM library (not part of the C ABI).
#pragma once

#include <algorithm>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/mlbm.h"

namespace mlbm {

constexpr int kQ = 9;
constexpr int kMaxDegree = 8;
constexpr int kMaxK = 128;

// Monomials of total degree <= d in two variables.
inline int num_monomials(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

// One segment (independent simulation) as laid out in device arrays.
struct SegmentHost {
    mlbm_segment_desc d;
    int64_t orig_off = 0;  // first original index of the segment
    int64_t off = 0;       // first stored position (global)
    int64_t n = 0;         // nodes in the segment
    int K = 0;             // stencil size
    int m = 0;             // monomials
    int64_t idx_off = 0;   // offset of the [K][n] stencil block (int32 entries)
    int64_t w_off = 0;     // offset of the [8][K][n] shape-vector block
    int64_t csr_off = 0;   // offset of the segment's transposed-stencil entries
};

struct mlbm_cloud_impl {
    int nseg = 0;
    int64_t N = 0;
    std::vector<SegmentHost> seg;
    std::vector<double> x, y;           // stored order
    std::vector<int64_t> perm;          // stored position -> original index
    std::vector<int32_t> idx;           // per segment [K][n], global stored positions
    std::vector<uint16_t> mask;         // stored order
    std::vector<double> fdir;           // [2][N] force direction, stored order
    std::vector<int32_t> csr_ptr;       // [N+1] transposed stencil row pointers (global)
    std::vector<int32_t> csr_ent;       // entries e = j * n_seg + i_local (segment-local)
    std::vector<int32_t> node_seg;      // stored position -> segment
    std::vector<int32_t> near;          // per segment [8][n]: departure node of (i, k), stored positions
    int64_t idx_total = 0, w_total = 0;
};

// Device-side segment descriptor (plain old data, copied to the device).
struct SegDev {
    int64_t off, n, idx_off, w_off;
    int K, m, deg, geometry;
    double lx, ly, dx_ml, pad;
};

// Nodes per tile of the fused step (one CTA pass over a contiguous Morton run): large tiles
// for clouds with enough tiles to fill the GPU, small tiles otherwise, and one-warp tiles for
// clouds so small that 128-node tiles would leave SMs idle or doubly loaded (a 20 k-node cloud
// makes 156 such tiles for 152 SMs).
constexpr int kTileNodes = 512;
constexpr int kTileNodesSmall = 128;
constexpr int kTileNodesTiny = 32;

// Functions evaluated both by host code and inside kernels' launch bounds.
#ifdef __CUDACC__
#define MLBM_HOST_DEVICE __host__ __device__
#else
#define MLBM_HOST_DEVICE
#endif

// CTAs per SM that the tile kernels' register budget is set for: two 512-node CTAs per SM in
// FP32 (one in FP64), the same threads per SM for 128-node tiles, at most 16 one-warp CTAs.
MLBM_HOST_DEVICE constexpr int tile_min_blocks(int B, int elem_bytes) {
    return (elem_bytes == 4 ? 2 : 1) * (kTileNodes / B) < 16 ? (elem_bytes == 4 ? 2 : 1) * (kTileNodes / B) : 16;
}

// Tile size for a cloud whose segments have the given node counts.
inline int choose_tile_nodes(const std::vector<int64_t> &seg_nodes, int num_sms) {
    int64_t big = 0, small = 0;
    for (int64_t n : seg_nodes) {
        big += (n + kTileNodes - 1) / kTileNodes;
        small += (n + kTileNodesSmall - 1) / kTileNodesSmall;
    }
    const int64_t sms = std::max(1, num_sms);
    if (big >= 4 * sms) return kTileNodes;
    if (small >= 2 * sms) return kTileNodesSmall;
    return kTileNodesTiny;
}

// Let kernel fn use up to the device's opt-in maximum of dynamic shared memory.  The attribute
// belongs to the function, not to a weights object: setting it to one object's own need would
// lower it under another object's launches (and under graphs captured for them), so every
// launcher that needs more than the default sets it to the maximum.  Defined in step.cu.
int allow_dynamic_smem(const void *fn);

// f(std::integral_constant<int, B>{}) for the tile size B of the weights (kernel dispatch).
template <typename F>
int with_tile_nodes(int tile_nodes, F &&f) {
    if (tile_nodes == kTileNodes) return f(std::integral_constant<int, kTileNodes>{});
    if (tile_nodes == kTileNodesSmall) return f(std::integral_constant<int, kTileNodesSmall>{});
    return f(std::integral_constant<int, kTileNodesTiny>{});
}

// A tile: a contiguous run of stored nodes of one segment processed by one CTA pass.
// Its halo (the tile's own nodes first, then every other node its stencils read, sorted) is
// staged in shared memory; the stencil members are 16-bit slots into that halo.
struct TileDev {
    int64_t begin;  // first stored position
    int64_t w_off;    // element offset of the tile's FP32 shape vectors (members 1..K-1)
    int64_t w64_off;  // element offset of the tile's FP64 shape vectors (members 0..K-1)
    int64_t l_off;  // offset of the tile's packed slot pairs: own mode [ceil((K-1)/2)][B] for
                    // members 1..K-1; nearest mode [ceil(K/2)][B][8] for members 0..K-1 of the
                    // departure node's stencil, per direction
    int64_t h_off;  // offset of the tile's halo list (int32 stored positions)
    int32_t count;  // nodes in tile
    int32_t seg;    // segment index
    int32_t K;      // stencil size of the segment
    int32_t U;      // halo size (slots)
    int32_t mode;   // MLBM_STENCIL_OWN or MLBM_STENCIL_NEAREST
    int32_t pad;
};

struct GraphKey {
    const void *a, *b;
    int dtype;
    int64_t chunk;
    std::vector<double> params;
    const void *tiles = nullptr;  // tile table the captured steps walk, and its length
    int64_t ntiles = 0;
    bool operator<(const GraphKey &o) const {
        return std::tie(a, b, dtype, chunk, params, tiles, ntiles) <
               std::tie(o.a, o.b, o.dtype, o.chunk, o.params, o.tiles, o.ntiles);
    }
};

struct mlbm_weights_impl {
    int nseg = 0;
    int64_t N = 0;
    std::vector<SegmentHost> seg;
    std::vector<int64_t> perm;  // host copy
    // device arrays
    SegDev *d_seg = nullptr;
    TileDev *d_tiles = nullptr;
    int ntiles = 0;
    int tile_nodes = 0;
    int32_t *d_idx = nullptr;
    double *d_w64 = nullptr;    // canonical FP64 shape vectors, per segment [8][K][n]
    float *d_w32c = nullptr;    // canonical FP32 shape vectors, per segment [8][K][n], rounded so that
                                // the polynomial reproduction holds as closely as FP32 allows
    double *d_x = nullptr, *d_y = nullptr;  // node coordinates, stored order (for that rounding)
    float *d_w32t = nullptr;    // tile layout, FP32: [j-1][2][kTileNodes][4 directions], j = 1..K-1
    double *d_w64t = nullptr;   // tile layout, FP64: [j][4][kTileNodes][2 directions], j = 0..K-1
    uint32_t *d_lidx = nullptr; // packed 16-bit halo slots of stencil members 1..K-1
    int32_t *d_halo = nullptr;  // halo lists
    int umax = 0;               // largest halo of any tile
    int64_t wt_total = 0, wt64_total = 0, l_total = 0, h_total = 0;
    uint16_t *d_mask = nullptr;
    float *d_fdir32 = nullptr;
    double *d_fdir64 = nullptr;
    int64_t *d_perm = nullptr;  // stored -> original
    int32_t *d_node_seg = nullptr;
    int32_t *d_csr_ptr = nullptr;
    int32_t *d_csr_ent = nullptr;
    int64_t idx_total = 0, w_total = 0;
    bool has_mask = false;
    // scratch (lazily allocated)
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    double *d_partials = nullptr;
    int partial_slots = 0;
    double *d_params = nullptr;  // [nseg][4] step parameters (tau, g, rho0, 1/tau) in FP64, then
                                 // the same [nseg][4] in FP32 (float view at d_params + 4 nseg)
    std::vector<double> params_cache;
    int num_sms = 0;
    int step_grid[2] = {0, 0};  // persistent grid of the step kernel, [FP32, FP64]
    int solve_wpb = 0;          // warps per CTA the solver ran with (autotuned)
    bool any_nearest = false;   // some segment interpolates in departure-node stencils
    // solver system table during the build (nearest-node stencils), freed afterwards
    int32_t *d_sys_node = nullptr;
    double *d_sys_q = nullptr;
    int32_t *d_sys_tgt = nullptr;
    int64_t nsys = 0;
    int device = 0;
    std::map<GraphKey, void *> graphs;  // cudaGraphExec_t
    // mlbm_run_until: host copy of the tile table, and a device table re-sorted per call by the
    // segments' step counts (longest first), so the active tiles of any step are a prefix
    std::vector<TileDev> tiles_host;
    TileDev *d_tiles_run = nullptr;
    // adjoint, built on first use: per forward tile its rows ordered by transposed-stencil
    // length ([ntiles][B] offsets), its reverse halo (own nodes, then every other node that reads
    // one of them, sorted; offset and size per tile), per 32-row slice of that order its first
    // entry and entries per row ([ntiles][B/32]), per entry the reading node's reverse-halo slot,
    // and the entries' coefficients in FP32 / FP64 (own-node rule: eight per entry; nearest-node
    // rule: the slice's entries are listed direction by direction, one coefficient each)
    uint16_t *d_adj_rowp = nullptr;
    int32_t *d_adj_rhalo = nullptr;
    int64_t *d_adj_roff = nullptr;
    int32_t *d_adj_rcnt = nullptr;
    int64_t *d_adj_sbeg = nullptr;
    int64_t *d_adj_cbeg = nullptr;  // [ntiles][B/32] first coefficient of each slice
    int32_t *d_adj_slen = nullptr;
    int32_t *d_adj_nlen = nullptr;  // [ntiles][B/32][8] nearest-rule slices: entries per direction
    uint16_t *d_adj_slot = nullptr;
    int32_t *d_adj_src = nullptr;  // per entry: reading node (stored position; -1 padding)
    int8_t *d_adj_jh = nullptr;    // per entry: row node's member index in the reader's stencil
    int32_t *d_near = nullptr;     // nearest-node clouds: per segment [8][n] departure nodes (stored positions)
    void *d_adj_coef[2] = {nullptr, nullptr};
    int64_t adj_positions = 0;
    int64_t adj_coefs = 0;
    int adj_rmax = 0;  // largest reverse halo
    // Shan-Chen steps: [nseg][2] (G, rho_psi) in FP64 then FP32, and the psi scratch [N]
    double *d_sc = nullptr;
    std::vector<double> sc_cache;
    void *d_sc_psi = nullptr;
    // host-buffer steps (mlbm_step_host): two input and two output state buffers, one copy
    // stream per direction and their events, created on first use
    void *d_stage[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t stage_bytes = 0;
    void *copy_stream[2] = {nullptr, nullptr};  // cudaStream_t: host->device, device->host
    void *stage_event[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // cudaEvent_t
};

}  // namespace mlbm

struct mlbm_cloud : mlbm::mlbm_cloud_impl {};
struct mlbm_weights : mlbm::mlbm_weights_impl {};

namespace mlbm {

// Helpers shared by the host build (cloud.cpp) and the device build (cloud_gpu.cu) of a cloud.

// Argument checks of mlbm_build_cloud; on success the stencil and shape-vector totals.
int check_cloud_args(const double *xy, int64_t n, const mlbm_segment_desc *segs, const int64_t *seg_offsets,
                     int nseg, int64_t *idx_total, int64_t *w_total);
// A cloud with every array sized and the segment table filled (throws std::bad_alloc).
mlbm_cloud *new_cloud(int64_t n, const mlbm_segment_desc *segs, const int64_t *seg_offsets, int nseg,
                      int64_t idx_total, int64_t w_total);

// Bounding box of a segment: the periodic box, else the extent of its nodes (unpadded).
struct BBox {
    double x0, x1, y0, y1;
};
BBox segment_bbox(const double *x, const double *y, int64_t n, const mlbm_segment_desc &d);

// Uniform bucket grid of a segment (about two nodes per cell) for nearest-neighbour queries.
struct GridGeom {
    int ncx, ncy;
    double x0, y0, cw, ch;
    bool periodic;
    double lx, ly;
};
GridGeom grid_geom(int64_t n, const BBox &b, const mlbm_segment_desc &d);

}  // namespace mlbm
