// Host-side stencil build (Sec. 2.2 stencils X^L, Sec. 3 periodic stencil search and wall
// bounce-back): Morton reorder, grid-bucket k-nearest neighbours, bounce-back masks, force
// directions and the transposed stencil used by the adjoint.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "mlbm_internal.h"

namespace mlbm {

static thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }
int fail(int code, const std::string &m) {
    g_err = m;
    return code;
}

namespace {

// D2Q9 directions of Sec. 2.1.
const int kEx[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kEy[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

double wrap(double d, double L) {
    if (L > 0.0) d -= L * std::round(d / L);
    return d;
}

uint32_t spread16(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

template <typename F>
void parallel_for(int64_t n, F &&fn) {
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::max(1u, std::min(hw, 64u));
    if (n < 4096) nt = 1;
    if (nt == 1) {
        fn(0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        th.emplace_back([&fn, b, e] { fn(b, e); });
    }
    for (auto &t : th) t.join();
}

// Uniform bucket grid over one segment (stored order), for nearest-neighbour queries.
struct Grid : GridGeom {
    std::vector<int32_t> start;  // [ncx*ncy + 1]
    std::vector<int32_t> items;  // segment-local stored indices

    void build(const double *x, const double *y, int64_t n, const mlbm_segment_desc &d) {
        static_cast<GridGeom &>(*this) = grid_geom(n, segment_bbox(x, y, n, d), d);
        start.assign((size_t)ncx * ncy + 1, 0);
        std::vector<int32_t> cell(n);
        for (int64_t i = 0; i < n; ++i) {
            int c = cell_of(x[i], y[i]);
            cell[i] = c;
            start[c + 1]++;
        }
        for (size_t c = 0; c < (size_t)ncx * ncy; ++c) start[c + 1] += start[c];
        items.resize(n);
        std::vector<int32_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < n; ++i) items[fill[cell[i]]++] = (int32_t)i;
    }
    int cx_of(double x) const {
        double u = x;
        if (periodic) u -= lx * std::floor(u / lx);
        int c = (int)std::floor((u - x0) / cw);
        return std::min(std::max(c, 0), ncx - 1);
    }
    int cy_of(double y) const {
        double u = y;
        if (periodic) u -= ly * std::floor(u / ly);
        int c = (int)std::floor((u - y0) / ch);
        return std::min(std::max(c, 0), ncy - 1);
    }
    int cell_of(double x, double y) const { return cy_of(y) * ncx + cx_of(x); }
};

// K nearest nodes of query node q (segment-local stored index) by (d^2, original index).
void knn_query(const Grid &g, const double *x, const double *y, const int64_t *orig, double qx, double qy,
               int K, int32_t *out_local) {
    double bd[kMaxK];
    int64_t bo[kMaxK];
    int32_t bl[kMaxK];
    int cnt = 0;
    auto consider = [&](int32_t j) {
        double dx = wrap(x[j] - qx, g.periodic ? g.lx : 0.0);
        double dy = wrap(y[j] - qy, g.periodic ? g.ly : 0.0);
        double d2 = dx * dx + dy * dy;
        int64_t o = orig[j];
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
        int c = cy * g.ncx + cx;
        for (int32_t t = g.start[c]; t < g.start[c + 1]; ++t) consider(g.items[t]);
    };
    int cx = g.cx_of(qx), cy = g.cy_of(qy);
    double ux = qx, uy = qy;
    if (g.periodic) {
        ux -= g.lx * std::floor(ux / g.lx);
        uy -= g.ly * std::floor(uy / g.ly);
    }
    for (int ring = 0;; ++ring) {
        bool full = g.periodic ? (2 * ring + 1 >= g.ncx || 2 * ring + 1 >= g.ncy)
                               : (ring > g.ncx && ring > g.ncy);
        if (full && g.periodic) {
            // the block wraps onto itself: scan everything once
            cnt = 0;
            for (int yy = 0; yy < g.ncy; ++yy)
                for (int xx = 0; xx < g.ncx; ++xx) scan_cell(xx, yy);
            break;
        }
        if (full) break;
        for (int dy = -ring; dy <= ring; ++dy) {
            for (int dx = -ring; dx <= ring; ++dx) {
                if (std::max(std::abs(dx), std::abs(dy)) != ring) continue;
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
            double bx0 = g.x0 + (cx - ring) * g.cw, bx1 = g.x0 + (cx + ring + 1) * g.cw;
            double by0 = g.y0 + (cy - ring) * g.ch, by1 = g.y0 + (cy + ring + 1) * g.ch;
            double dmin = std::min(std::min(ux - bx0, bx1 - ux), std::min(uy - by0, by1 - uy));
            if (dmin > 0 && dmin * dmin > bd[K - 1] * (1.0 + 1e-12)) break;
        }
    }
    for (int j = 0; j < K; ++j) out_local[j] = bl[j];
}

}  // namespace

BBox segment_bbox(const double *x, const double *y, int64_t n, const mlbm_segment_desc &d) {
    if (d.geometry == MLBM_GEOM_PERIODIC) return BBox{0.0, d.lx, 0.0, d.ly};
    return BBox{*std::min_element(x, x + n), *std::max_element(x, x + n), *std::min_element(y, y + n),
                *std::max_element(y, y + n)};
}

GridGeom grid_geom(int64_t n, const BBox &b, const mlbm_segment_desc &d) {
    GridGeom g;
    g.periodic = d.geometry == MLBM_GEOM_PERIODIC;
    g.lx = g.periodic ? d.lx : 0.0;
    g.ly = g.periodic ? d.ly : 0.0;
    double x0 = b.x0, x1 = b.x1, y0 = b.y0, y1 = b.y1;
    if (!g.periodic) {
        double pad = 1e-9 * std::max(1.0, std::max(x1 - x0, y1 - y0));
        x0 -= pad;
        y0 -= pad;
        x1 += pad;
        y1 += pad;
    }
    g.x0 = x0;
    g.y0 = y0;
    double W = std::max(x1 - x0, 1e-300), H = std::max(y1 - y0, 1e-300);
    // about two nodes per cell; degenerate (thin) clouds get a single row of cells
    double cells = std::max(1.0, (double)n / 2.0);
    double csz = std::sqrt(W * H / cells);
    g.ncx = (int)std::min(std::min(cells, 32768.0), std::max(1.0, std::floor(W / csz)));
    g.ncy = (int)std::min(std::min(cells, 32768.0), std::max(1.0, std::floor(cells / g.ncx)));
    g.cw = W / g.ncx;
    g.ch = H / g.ncy;
    return g;
}

int check_cloud_args(const double *xy, int64_t n, const mlbm_segment_desc *segs, const int64_t *seg_offsets,
                     int nseg, int64_t *idx_total_out, int64_t *w_total_out) {
    if (!xy || !segs || !seg_offsets || n < 1 || nseg < 1)
        return fail(MLBM_EINVAL, "bad arguments to mlbm_build_cloud");
    if (seg_offsets[0] != 0 || seg_offsets[nseg] != n)
        return fail(MLBM_EINVAL, "seg_offsets must start at 0 and end at n");
    int64_t idx_total = 0, w_total = 0;
    for (int s = 0; s < nseg; ++s) {
        const mlbm_segment_desc &d = segs[s];
        int64_t ns = seg_offsets[s + 1] - seg_offsets[s];
        if (ns < 1) return fail(MLBM_EINVAL, "empty segment " + std::to_string(s));
        if (d.k < 1 || d.k > kMaxK || d.k > ns)
            return fail(MLBM_EINVAL, "stencil size k out of range in segment " + std::to_string(s));
        if (d.degree < 0 || d.degree > kMaxDegree || num_monomials(d.degree) > d.k)
            return fail(MLBM_EINVAL,
                        "degree out of range or more monomials than stencil nodes in segment " +
                            std::to_string(s));
        if (!(d.dx_ml > 0)) return fail(MLBM_EINVAL, "dx_ml must be > 0");
        if (d.stencil_mode != MLBM_STENCIL_OWN && d.stencil_mode != MLBM_STENCIL_NEAREST)
            return fail(MLBM_EINVAL, "unknown stencil mode");
        if (d.geometry == MLBM_GEOM_PERIODIC) {
            if (!(d.lx > 0 && d.ly > 0)) return fail(MLBM_EINVAL, "periodic box needs lx, ly > 0");
        } else if (d.geometry == MLBM_GEOM_ANNULUS) {
            if (!(d.r_in >= 0 && d.r_out > d.r_in)) return fail(MLBM_EINVAL, "annulus needs 0 <= r_in < r_out");
        } else {
            return fail(MLBM_EINVAL, "unknown geometry");
        }
        idx_total += (int64_t)d.k * ns;
        w_total += 8LL * d.k * ns;
    }
    if (idx_total >= (1LL << 31)) return fail(MLBM_EINVAL, "N_L * N must stay below 2^31");
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(xy[i])) return fail(MLBM_EINVAL, "non-finite coordinate");
    *idx_total_out = idx_total;
    *w_total_out = w_total;
    return MLBM_OK;
}

mlbm_cloud *new_cloud(int64_t n, const mlbm_segment_desc *segs, const int64_t *seg_offsets, int nseg,
                      int64_t idx_total, int64_t w_total) {
    mlbm_cloud *c = new mlbm_cloud();
    try {
        c->nseg = nseg;
        c->N = n;
        c->idx_total = idx_total;
        c->w_total = w_total;
        c->x.resize(n);
        c->y.resize(n);
        c->perm.resize(n);
        c->idx.resize(idx_total);
        c->mask.assign(n, 0);
        c->fdir.assign(2 * n, 0.0);
        c->node_seg.resize(n);
        c->near.resize((size_t)8 * n);
        c->csr_ptr.assign(n + 1, 0);
        c->csr_ent.resize(idx_total);
        int64_t io = 0, wo = 0;
        for (int s = 0; s < nseg; ++s) {
            SegmentHost sh;
            sh.d = segs[s];
            sh.orig_off = seg_offsets[s];
            sh.off = seg_offsets[s];
            sh.n = seg_offsets[s + 1] - seg_offsets[s];
            sh.K = segs[s].k;
            sh.m = num_monomials(segs[s].degree);
            sh.idx_off = io;
            sh.w_off = wo;
            sh.csr_off = io;
            io += (int64_t)sh.K * sh.n;
            wo += 8LL * sh.K * sh.n;
            c->seg.push_back(sh);
        }
    } catch (...) {
        delete c;
        throw;
    }
    return c;
}

static int build_cloud_impl(const double *xy, int64_t n, const mlbm_segment_desc *segs,
                            const int64_t *seg_offsets, int nseg, mlbm_cloud **out) {
    if (!out) return fail(MLBM_EINVAL, "out is NULL");
    *out = nullptr;
    int64_t idx_total = 0, w_total = 0;
    int rc = check_cloud_args(xy, n, segs, seg_offsets, nseg, &idx_total, &w_total);
    if (rc) return rc;
    mlbm_cloud *c = nullptr;
    try {
        c = new_cloud(n, segs, seg_offsets, nseg, idx_total, w_total);
        const double *X = xy, *Y = xy + n;
        for (int s = 0; s < nseg; ++s) {
            SegmentHost &sh = c->seg[s];
            const mlbm_segment_desc &d = sh.d;
            int64_t ns = sh.n, o = sh.off;
            // Morton order of the segment: 16-bit quantised coordinates, interleaved.
            const BBox bb = segment_bbox(X + o, Y + o, ns, d);
            const double x0 = bb.x0, x1 = bb.x1, y0 = bb.y0, y1 = bb.y1;
            double sx = (x1 > x0) ? 65536.0 / (x1 - x0) : 0.0;
            double sy = (y1 > y0) ? 65536.0 / (y1 - y0) : 0.0;
            std::vector<std::pair<uint64_t, int64_t>> key(ns);
            for (int64_t i = 0; i < ns; ++i) {
                double xx = X[o + i], yy = Y[o + i];
                if (d.geometry == MLBM_GEOM_PERIODIC) {
                    xx -= d.lx * std::floor(xx / d.lx);
                    yy -= d.ly * std::floor(yy / d.ly);
                }
                uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, std::floor((xx - x0) * sx)));
                uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, std::floor((yy - y0) * sy)));
                uint64_t code = (uint64_t)(spread16(qx) | (spread16(qy) << 1));
                key[i] = {code, o + i};
            }
            std::sort(key.begin(), key.end());
            for (int64_t p = 0; p < ns; ++p) {
                int64_t src = key[p].second;
                c->perm[o + p] = src;
                c->x[o + p] = X[src];
                c->y[o + p] = Y[src];
                c->node_seg[o + p] = s;
            }
            // k-nearest-neighbour stencils (segment-local stored indices -> global positions)
            Grid g;
            g.build(&c->x[o], &c->y[o], ns, d);
            const double *sxp = &c->x[o], *syp = &c->y[o];
            const int64_t *orig = &c->perm[o];
            int K = sh.K;
            int32_t *idx = &c->idx[sh.idx_off];
            std::atomic<int> dup{0};
            parallel_for(ns, [&](int64_t b, int64_t e) {
                int32_t tmp[kMaxK];
                for (int64_t i = b; i < e; ++i) {
                    knn_query(g, sxp, syp, orig, sxp[i], syp[i], K, tmp);
                    if (tmp[0] != (int32_t)i) dup = 1;
                    for (int j = 0; j < K; ++j) idx[(int64_t)j * ns + i] = (int32_t)(o + tmp[j]);
                }
            });
            // departure nodes: the node nearest to x_i - e_k dx_ml (Sec. 2.3, appendix algorithm)
            if (d.stencil_mode == MLBM_STENCIL_NEAREST) {
                int32_t *near = &c->near[(size_t)8 * o];
                parallel_for(ns, [&](int64_t b, int64_t e) {
                    int32_t nn[1];
                    for (int64_t i = b; i < e; ++i)
                        for (int k = 1; k < kQ; ++k) {
                            knn_query(g, sxp, syp, orig, sxp[i] - kEx[k] * d.dx_ml, syp[i] - kEy[k] * d.dx_ml, 1, nn);
                            near[(int64_t)(k - 1) * ns + i] = (int32_t)(o + nn[0]);
                        }
                });
            } else {
                int32_t *near = &c->near[(size_t)8 * o];
                for (int k = 1; k < kQ; ++k)
                    for (int64_t i = 0; i < ns; ++i) near[(int64_t)(k - 1) * ns + i] = (int32_t)(o + i);
            }
            if (dup.load()) {
                delete c;
                return fail(MLBM_EINVAL, "duplicate nodes in segment " + std::to_string(s) +
                                             " (a node must be the first member of its own stencil)");
            }
            // bounce-back mask and force direction (Sec. 3)
            for (int64_t i = 0; i < ns; ++i) {
                double xx = sxp[i], yy = syp[i];
                uint16_t m = 0;
                if (d.geometry == MLBM_GEOM_ANNULUS) {
                    for (int k = 1; k < kQ; ++k) {
                        double Dx = xx - kEx[k] * d.dx_ml, Dy = yy - kEy[k] * d.dx_ml;
                        double r2 = Dx * Dx + Dy * Dy;
                        if (r2 < d.r_in * d.r_in * (1.0 - 1e-12) || r2 > d.r_out * d.r_out * (1.0 + 1e-12))
                            m |= (uint16_t)(1u << k);
                    }
                    double r = std::sqrt(xx * xx + yy * yy);
                    c->fdir[o + i] = r > 0 ? -yy / r : 0.0;
                    c->fdir[n + o + i] = r > 0 ? xx / r : 0.0;
                } else {
                    c->fdir[o + i] = 1.0;
                    c->fdir[n + o + i] = 0.0;
                }
                c->mask[o + i] = m;
            }
            // transposed stencil: for every node, the (member slot j, node i) pairs that read it
            std::vector<int32_t> cnt(ns + 1, 0);
            for (int64_t t = 0; t < (int64_t)K * ns; ++t) cnt[idx[t] - o + 1]++;
            for (int64_t i = 0; i < ns; ++i) cnt[i + 1] += cnt[i];
            std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
            int32_t *ent = &c->csr_ent[sh.csr_off];
            for (int j = 0; j < K; ++j)
                for (int64_t i = 0; i < ns; ++i) {
                    int64_t m = idx[(int64_t)j * ns + i] - o;
                    ent[fill[m]++] = (int32_t)((int64_t)j * ns + i);
                }
            for (int64_t i = 0; i <= ns; ++i) c->csr_ptr[o + i] = (int32_t)(sh.csr_off + cnt[i]);
        }
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(MLBM_ENOMEM, "host allocation failed");
    }
    *out = c;
    return MLBM_OK;
}

}  // namespace mlbm

using namespace mlbm;

extern "C" {

const char *mlbm_last_error(void) { return g_err.c_str(); }

int mlbm_abi_version(void) { return 6; }

int mlbm_build_cloud(const double *xy, int64_t n, const mlbm_segment_desc *segs,
                     const int64_t *seg_offsets, int nseg, mlbm_cloud **out) {
    set_error("");
    return build_cloud_impl(xy, n, segs, seg_offsets, nseg, out);
}

void mlbm_cloud_free(mlbm_cloud *c) { delete c; }

int64_t mlbm_cloud_size(const mlbm_cloud *c) { return c ? c->N : -1; }

int mlbm_cloud_perm(const mlbm_cloud *c, int64_t *perm) {
    if (!c || !perm) return fail(MLBM_EINVAL, "NULL argument");
    std::memcpy(perm, c->perm.data(), sizeof(int64_t) * c->N);
    return MLBM_OK;
}

int mlbm_cloud_stencil(const mlbm_cloud *c, int seg, int32_t *idx_out) {
    if (!c || !idx_out) return fail(MLBM_EINVAL, "NULL argument");
    if (seg < 0 || seg >= c->nseg) return fail(MLBM_EINVAL, "segment out of range");
    const SegmentHost &sh = c->seg[seg];
    int64_t ns = sh.n;
    for (int j = 0; j < sh.K; ++j)
        for (int64_t i = 0; i < ns; ++i) {
            int64_t io = c->perm[sh.off + i] - sh.orig_off;
            int64_t member = c->idx[sh.idx_off + (int64_t)j * ns + i];
            idx_out[(int64_t)j * ns + io] = (int32_t)(c->perm[member] - sh.orig_off);
        }
    return MLBM_OK;
}

int mlbm_cloud_departure_nodes(const mlbm_cloud *c, int seg, int32_t *near) {
    if (!c || !near) return fail(MLBM_EINVAL, "NULL argument");
    if (seg < 0 || seg >= c->nseg) return fail(MLBM_EINVAL, "segment out of range");
    const SegmentHost &sh = c->seg[seg];
    for (int k = 0; k < 8; ++k)
        for (int64_t i = 0; i < sh.n; ++i) {
            int64_t io = c->perm[sh.off + i] - sh.orig_off;
            int64_t L = c->near[(size_t)8 * sh.off + (int64_t)k * sh.n + i];
            near[(int64_t)k * sh.n + io] = (int32_t)(c->perm[L] - sh.orig_off);
        }
    return MLBM_OK;
}

int mlbm_cloud_bounce_mask(const mlbm_cloud *c, uint16_t *mask) {
    if (!c || !mask) return fail(MLBM_EINVAL, "NULL argument");
    for (int64_t p = 0; p < c->N; ++p) mask[c->perm[p]] = c->mask[p];
    return MLBM_OK;
}

}  // extern "C"
