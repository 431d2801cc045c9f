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

#include "internal.h"

namespace mlpg {

int64_t build_tiles(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *order, int rows_per_tile,
                    int width_multiple, TileLayout &out) {
    const int64_t TR = rows_per_tile;
    out = TileLayout{};
    out.rows_per_tile = rows_per_tile;
    out.ntile = (n + TR - 1) / TR;
    out.base.assign(out.ntile + 1, 0);
    out.width.assign(out.ntile, 0);
    out.row.assign(out.ntile * TR, -1);
    out.hptr.assign(out.ntile + 1, 0);
    // widths, halo sizes and the total slot count
    std::vector<int32_t> h;
    for (int64_t t = 0; t < out.ntile; ++t) {
        int32_t w = 0;
        h.clear();
        for (int64_t s = 0; s < TR && t * TR + s < n; ++s) {
            const int32_t i = order[t * TR + s];
            out.row[t * TR + s] = i;
            w = std::max(w, rowptr[i + 1] - rowptr[i]);
            h.insert(h.end(), col + rowptr[i], col + rowptr[i + 1]);
        }
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
        w = (w + width_multiple - 1) / width_multiple * width_multiple;
        out.width[t] = w;
        out.base[t + 1] = out.base[t] + (int64_t)w * TR;
        out.hptr[t + 1] = out.hptr[t] + (int64_t)h.size();
        out.hcol.insert(out.hcol.end(), h.begin(), h.end());
        out.max_halo = std::max<int64_t>(out.max_halo, (int64_t)h.size());
        out.max_width = std::max<int32_t>(out.max_width, w);
    }
    const int64_t nslot = out.base[out.ntile];
    out.perm.assign(nslot, -1);
    out.lcol.assign(nslot, 0);
    for (int64_t t = 0; t < out.ntile; ++t) {
        const int32_t *hb = out.hcol.data() + out.hptr[t], *he = out.hcol.data() + out.hptr[t + 1];
        for (int64_t s = 0; s < TR; ++s) {
            const int32_t i = out.row[t * TR + s];
            if (i < 0) continue;
            for (int32_t p = rowptr[i], k = 0; p < rowptr[i + 1]; ++p, ++k) {
                const int64_t e = out.base[t] + (int64_t)k * TR + s;
                out.perm[e] = p;
                out.lcol[e] = (int32_t)(std::lower_bound(hb, he, col[p]) - hb);
            }
        }
    }
    return nslot;
}

}  // namespace mlpg
