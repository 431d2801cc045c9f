// Voronoi-like integration cells on the host (Sec. 3.1), built once per point
// set.  Each cell starts as the kernel-extent square [x_i - R_i, x_i + R_i]^2
// cut to the domain box and is clipped by the perpendicular bisector of every
// overlap neighbour; what is left is the part of space closer to x_i than to
// any neighbour.  Cells are independent, so they are built in parallel on the
// host cores.  Edge labels record where each edge came from so that edges on
// the domain boundary receive the surface quadrature (Alg. 1).
#include <algorithm>
#include <cmath>
#include <thread>

#include "internal.h"

namespace mlpg {

namespace {
struct Vtx {
    double x, y;
    int32_t lab;  // label of the edge that starts at this vertex
};

// Keep {p : a p.x + b p.y <= c}; edges created by the cut get label j.
void clip(std::vector<Vtx> &poly, std::vector<Vtx> &tmp, double a, double b, double c, int32_t j) {
    const size_t nv = poly.size();
    bool any_out = false;
    for (const Vtx &v : poly)
        if (a * v.x + b * v.y - c > 0.0) { any_out = true; break; }
    if (!any_out) return;
    tmp.clear();
    for (size_t k = 0; k < nv; ++k) {
        const Vtx &p = poly[k], &qv = poly[(k + 1) % nv];
        double sp = a * p.x + b * p.y - c, sq = a * qv.x + b * qv.y - c;
        bool pin = sp <= 0.0, qin = sq <= 0.0;
        if (pin) tmp.push_back(p);
        if (pin != qin) {
            double t = sp / (sp - sq);
            Vtx r{p.x + t * (qv.x - p.x), p.y + t * (qv.y - p.y), pin ? j : p.lab};
            tmp.push_back(r);
        }
    }
    poly.swap(tmp);
}

struct Chunk {
    std::vector<int32_t> nvert;
    std::vector<double> verts;
    std::vector<int32_t> labels;
    int64_t nbedges = 0;
    int64_t bad = -1;
};
}  // namespace

int64_t build_cells_2d(int64_t n, const double *x, const double *R, const double *lo,
                       const double *hi, const int32_t *rowptr, const int32_t *col,
                       int tri_points, int line_points, HostCells &out) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 4096) nt = 1;
    std::vector<Chunk> chunks(nt);
    out.volume.assign(n, 0.0);
    auto work = [&](unsigned t) {
        int64_t i0 = n * t / nt, i1 = n * (t + 1) / nt;
        Chunk &ch = chunks[t];
        std::vector<Vtx> poly, tmp;
        poly.reserve(64);
        tmp.reserve(64);
        for (int64_t i = i0; i < i1; ++i) {
            const double xi = x[2 * i], yi = x[2 * i + 1], r = R[i];
            double x0 = xi - r, x1 = xi + r, y0 = yi - r, y1 = yi + r;
            bool bx0 = x0 <= lo[0], bx1 = x1 >= hi[0], by0 = y0 <= lo[1], by1 = y1 >= hi[1];
            x0 = bx0 ? lo[0] : x0;
            x1 = bx1 ? hi[0] : x1;
            y0 = by0 ? lo[1] : y0;
            y1 = by1 ? hi[1] : y1;
            poly.clear();
            poly.push_back({x0, y0, by0 ? -3 : kLabelExtent});  // face 2 (-y)
            poly.push_back({x1, y0, bx1 ? -2 : kLabelExtent});  // face 1 (+x)
            poly.push_back({x1, y1, by1 ? -4 : kLabelExtent});  // face 3 (+y)
            poly.push_back({x0, y1, bx0 ? -1 : kLabelExtent});  // face 0 (-x)
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int32_t j = col[p];
                if (j == i) continue;
                double ax = x[2 * j] - xi, ay = x[2 * j + 1] - yi;
                double c = ax * 0.5 * (x[2 * j] + xi) + ay * 0.5 * (x[2 * j + 1] + yi);
                clip(poly, tmp, ax, ay, c, j);
                if (poly.empty()) break;
            }
            if (poly.size() < 3 && ch.bad < 0) ch.bad = i;
            double area2 = 0.0;
            for (size_t k = 0; k < poly.size(); ++k) {
                const Vtx &p = poly[k], &qv = poly[(k + 1) % poly.size()];
                area2 += p.x * qv.y - qv.x * p.y;
                if (p.lab < 0 && p.lab != kLabelExtent) ++ch.nbedges;
            }
            out.volume[i] = 0.5 * area2;
            if (!(out.volume[i] > 0.0) && ch.bad < 0) ch.bad = i;
            ch.nvert.push_back((int32_t)poly.size());
            for (const Vtx &p : poly) {
                ch.verts.push_back(p.x);
                ch.verts.push_back(p.y);
                ch.labels.push_back(p.lab);
            }
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &t : th) t.join();
    out.cptr.assign(n + 1, 0);
    out.verts.clear();
    out.labels.clear();
    int64_t nb = 0, nvtot = 0, k = 0;
    for (auto &ch : chunks) {
        if (ch.bad >= 0) return ch.bad;
        for (int32_t c : ch.nvert) {
            out.cptr[k + 1] = out.cptr[k] + c;
            nvtot += c;
            ++k;
        }
        out.verts.insert(out.verts.end(), ch.verts.begin(), ch.verts.end());
        out.labels.insert(out.labels.end(), ch.labels.begin(), ch.labels.end());
        nb += ch.nbedges;
    }
    out.n_volume_qp = nvtot * (int64_t)tri_points;
    out.n_boundary_qp = nb * (int64_t)line_points;
    return -1;
}

}  // namespace mlpg
