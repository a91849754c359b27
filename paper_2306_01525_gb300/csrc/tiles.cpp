// Tile tables of the fused step: for each run of B (kTileNodes or kTileNodesSmall) stored nodes of one segment, the
// halo of nodes its stencils read (own nodes first, then the others sorted), and the 16-bit halo
// slot of every stencil member j = 1..K-1 (member 0 is the node itself, Sec. 2.2), packed two per
// 32-bit word as [ceil((K-1)/2)][B].  In nearest-node mode each direction k has its own stencil
// (that of the node nearest to the departure point, Sec. 2.3): slots of all K members per
// direction, [ceil(K/2)][B][8] so that a node's eight directions are one 32-byte run.
#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "mlbm_internal.h"

namespace mlbm {

int build_tiles(const mlbm_cloud *c, int B, std::vector<TileDev> &tiles, std::vector<int32_t> &halo,
                std::vector<uint32_t> &lidx, int &umax, int64_t &wt_total, int64_t &wt64_total) {
    tiles.clear();
    int64_t w_off = 0, w64_off = 0, l_off = 0;
    for (int s = 0; s < c->nseg; ++s) {
        const SegmentHost &h = c->seg[s];
        for (int64_t b = 0; b < h.n; b += B) {
            TileDev t{};
            t.begin = h.off + b;
            t.count = (int32_t)std::min<int64_t>(B, h.n - b);
            t.seg = s;
            t.K = h.K;
            t.mode = h.d.stencil_mode;
            t.w_off = w_off;
            t.w64_off = w64_off;
            t.l_off = l_off;
            w_off += (int64_t)(h.K - 1) * 8 * B;
            w64_off += (int64_t)h.K * 8 * B;
            if (t.mode == MLBM_STENCIL_NEAREST)
                l_off += (int64_t)8 * ((h.K + 1) / 2) * B;
            else
                l_off += (int64_t)((h.K - 1 + 1) / 2) * B;
            tiles.push_back(t);
        }
    }
    wt_total = w_off;
    wt64_total = w64_off;
    lidx.assign((size_t)l_off, 0u);
    const int nt = (int)tiles.size();
    std::vector<std::vector<int32_t>> halos(nt);
    std::vector<int> bad(nt, 0);
    unsigned hw = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    auto work = [&](int t0, int t1) {
        std::vector<int32_t> others;
        for (int t = t0; t < t1; ++t) {
            TileDev &T = tiles[t];
            const SegmentHost &h = c->seg[T.seg];
            const int32_t *idx = &c->idx[h.idx_off];
            const int64_t il0 = T.begin - h.off;
            const int32_t *near = &c->near[(size_t)8 * h.off];
            const bool nearest = T.mode == MLBM_STENCIL_NEAREST;
            // member j of the stencil that interpolates direction k (1..8) at tile node b
            auto member = [&](int k, int j, int b) -> int32_t {
                if (!nearest) return idx[(int64_t)j * h.n + il0 + b];
                const int64_t L = near[(int64_t)(k - 1) * h.n + il0 + b] - h.off;
                return idx[(int64_t)j * h.n + L];
            };
            others.clear();
            for (int k = 1; k <= (nearest ? 8 : 1); ++k)
                for (int j = nearest ? 0 : 1; j < T.K; ++j)
                    for (int b = 0; b < T.count; ++b) {
                        int32_t m = member(k, j, b);
                        if (m < T.begin || m >= T.begin + T.count) others.push_back(m);
                    }
            std::sort(others.begin(), others.end());
            others.erase(std::unique(others.begin(), others.end()), others.end());
            std::vector<int32_t> &H = halos[t];
            H.resize((size_t)T.count + others.size());
            for (int b = 0; b < T.count; ++b) H[b] = (int32_t)(T.begin + b);
            std::copy(others.begin(), others.end(), H.begin() + T.count);
            if (H.size() > 65535) {
                bad[t] = 1;
                continue;
            }
            T.U = (int32_t)H.size();
            auto slot = [&](int32_t m) -> uint32_t {
                if (m >= T.begin && m < T.begin + T.count) return (uint32_t)(m - T.begin);
                return (uint32_t)(T.count + (std::lower_bound(others.begin(), others.end(), m) - others.begin()));
            };
            if (!nearest) {
                for (int j = 1; j < T.K; ++j) {
                    const int jp = (j - 1) >> 1, hi = (j - 1) & 1;
                    for (int b = 0; b < T.count; ++b) {
                        uint32_t sl = slot(member(0, j, b));
                        lidx[T.l_off + (int64_t)jp * B + b] |= hi ? (sl << 16) : sl;
                    }
                }
            } else {
                for (int k = 1; k <= 8; ++k)
                    for (int j = 0; j < T.K; ++j) {
                        const int jp = j >> 1, hi = j & 1;
                        for (int b = 0; b < T.count; ++b) {
                            uint32_t sl = slot(member(k, j, b));
                            lidx[T.l_off + ((int64_t)jp * B + b) * 8 + (k - 1)] |= hi ? (sl << 16) : sl;
                        }
                    }
            }
        }
    };
    std::vector<std::thread> th;
    int chunk = (nt + (int)hw - 1) / (int)hw;
    for (int t0 = 0; t0 < nt; t0 += chunk) th.emplace_back(work, t0, std::min(nt, t0 + chunk));
    for (auto &x : th) x.join();
    for (int t = 0; t < nt; ++t)
        if (bad[t]) return fail(MLBM_EINVAL, "a tile's halo exceeds 65535 nodes (stencils too spread out)");
    halo.clear();
    umax = 0;
    for (int t = 0; t < nt; ++t) {
        tiles[t].h_off = (int64_t)halo.size();
        halo.insert(halo.end(), halos[t].begin(), halos[t].end());
        umax = std::max(umax, tiles[t].U);
    }
    // largest stencils first so that the persistent grid ends evenly
    std::stable_sort(tiles.begin(), tiles.end(), [](const TileDev &p, const TileDev &q) { return p.K > q.K; });
    return MLBM_OK;
}

}  // namespace mlbm
