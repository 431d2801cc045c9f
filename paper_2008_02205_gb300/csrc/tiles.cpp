// Row tiles of the batched transport operator apply (host, once per point set).
//
// The rows of the overlap pattern are taken in the Morton order of their
// points and cut into tiles of `rows_per_tile` consecutive rows, so that the
// rows of one tile are close in space and share most of their overlap
// partners.  For every tile:
//   * the halo: the sorted union of the pattern columns of its rows, whose
//     angular-flux rows a CTA stages in shared memory once and reuses for
//     every entry of the tile;
//   * sliced-ELL record slots: entry k of row slot s sits at slot
//     base[t] + k * rows_per_tile + s, for k below the tile's width (its
//     longest row, rounded up to width_multiple so that the apply's inner
//     loop has no remainder), so that the rows handled by one warp read adjacent
//     records; a row shorter than the width is padded with empty slots
//     (perm = -1, halo index 0, zero operator values);
//   * for every slot, the pattern entry it holds (perm) and that entry's
//     column as an index into the halo (lcol).
#include <algorithm>
#include <exception>
#include <thread>

#include "internal.h"

namespace mlpg {

namespace {
// threads for the per-tile passes: the host cores, fewer when their n-sized
// scratch (12 bytes a point each) would pass 256 MB
int tile_threads(int64_t n, int64_t ntile) {
    int64_t T = std::max(1u, std::thread::hardware_concurrency());
    T = std::min<int64_t>(T, std::max<int64_t>(1, (int64_t(256) << 20) / std::max<int64_t>(1, 12 * n)));
    return (int)std::max<int64_t>(1, std::min<int64_t>(T, ntile / 8));
}
// f(first tile, end tile, worker) over T workers; an exception thrown by a worker (an
// allocation that fails) is rethrown here, on the calling thread, after every worker ended
template <typename F>
void over_tiles(int64_t ntile, int T, F &&f) {
    if (T <= 1) {
        f(int64_t(0), ntile, 0);
        return;
    }
    std::vector<std::exception_ptr> errs(T);
    std::vector<std::thread> th;
    for (int w = 0; w < T; ++w)
        th.emplace_back([&, w]() {
            try {
                f(ntile * w / T, ntile * (w + 1) / T, w);
            } catch (...) {
                errs[w] = std::current_exception();
            }
        });
    for (auto &x : th) x.join();
    for (auto &e : errs)
        if (e) std::rethrow_exception(e);
}
}  // namespace

int64_t build_tiles(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *order, int rows_per_tile,
                    int width_multiple, TileLayout &out) {
    const int64_t TR = rows_per_tile;
    out = TileLayout{};
    out.rows_per_tile = rows_per_tile;
    out.ntile = (n + TR - 1) / TR;
    const int64_t ntile = out.ntile;
    out.base.assign(ntile + 1, 0);
    out.width.assign(ntile, 0);
    out.row.assign(ntile * TR, -1);
    out.hptr.assign(ntile + 1, 0);
    const int T = tile_threads(n, ntile);
    // 1. per tile: rows, width and halo.  The halo is collected with a stamp per column
    //    (stamp[c] == t: already in it), then sorted; linear in the pattern entries.
    std::vector<std::vector<int32_t>> halo(ntile);
    over_tiles(ntile, T, [&](int64_t t0, int64_t t1, int) {
        std::vector<int64_t> stamp(n, -1);
        for (int64_t t = t0; t < t1; ++t) {
            int32_t w = 0;
            std::vector<int32_t> &h = halo[t];
            for (int64_t s = 0; s < TR && t * TR + s < n; ++s) {
                const int32_t i = order[t * TR + s];
                out.row[t * TR + s] = i;
                w = std::max(w, rowptr[i + 1] - rowptr[i]);
                for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                    if (stamp[col[p]] != t) {
                        stamp[col[p]] = t;
                        h.push_back(col[p]);
                    }
            }
            std::sort(h.begin(), h.end());
            out.width[t] = (w + width_multiple - 1) / width_multiple * width_multiple;
        }
    });
    for (int64_t t = 0; t < ntile; ++t) {
        out.base[t + 1] = out.base[t] + (int64_t)out.width[t] * TR;
        out.hptr[t + 1] = out.hptr[t] + (int64_t)halo[t].size();
        out.max_halo = std::max<int64_t>(out.max_halo, (int64_t)halo[t].size());
        out.max_width = std::max<int32_t>(out.max_width, out.width[t]);
    }
    out.hcol.resize(out.hptr[ntile]);
    const int64_t nslot = out.base[ntile];
    out.perm.assign(nslot, -1);
    out.lcol.assign(nslot, 0);
    // 2. per tile: the halo into place and every slot's entry and halo index (pos[c]: the
    //    column's index in the tile's halo), slots in memory order
    over_tiles(ntile, T, [&](int64_t t0, int64_t t1, int) {
        std::vector<int32_t> pos(n, 0);
        for (int64_t t = t0; t < t1; ++t) {
            const std::vector<int32_t> &h = halo[t];
            std::copy(h.begin(), h.end(), out.hcol.begin() + out.hptr[t]);
            for (int32_t k = 0; k < (int32_t)h.size(); ++k) pos[h[k]] = k;
            const int32_t *rows = out.row.data() + t * TR;
            for (int32_t k = 0; k < out.width[t]; ++k) {
                int32_t *pe = out.perm.data() + out.base[t] + (int64_t)k * TR;
                int32_t *le = out.lcol.data() + out.base[t] + (int64_t)k * TR;
                for (int64_t s = 0; s < TR; ++s) {
                    const int32_t i = rows[s];
                    if (i < 0 || k >= rowptr[i + 1] - rowptr[i]) continue;
                    const int32_t p = rowptr[i] + k;
                    pe[s] = p;
                    le[s] = pos[col[p]];
                }
            }
        }
    });
    return nslot;
}

}  // namespace mlpg
