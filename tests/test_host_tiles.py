"""The row tiles of the FP32 transport-operator apply (csrc/tiles.cpp, host
code run once per point set), compiled with g++ and checked on the CPU
against the overlap pattern the oracle builds (Sec. 3.4).

The tiled apply reads the operator through these tables only, so every
pattern entry must sit in exactly one record slot, in its own row's slot
column, with a halo index that leads back to its column; padding slots must
be marked and point at a valid halo row; each halo must be the sorted union
of its tile's columns."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_02205_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include <cstdio>
#include <vector>
#include "internal.h"
template <class T> static void rd(FILE *f, T *p, size_t k) { if (fread(p, sizeof(T), k, f) != k) throw 1; }
template <class T> static void wr(FILE *f, const T *p, size_t k) { fwrite(p, sizeof(T), k, f); }
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int64_t n, nnz, tr;
    rd(f, &n, 1); rd(f, &nnz, 1); rd(f, &tr, 1);
    std::vector<int32_t> rowptr(n + 1), col(nnz), order(n);
    rd(f, rowptr.data(), n + 1); rd(f, col.data(), nnz); rd(f, order.data(), n);
    fclose(f);
    mlpg::TileLayout t;
    int64_t nslot = mlpg::build_tiles(n, rowptr.data(), col.data(), order.data(), (int)tr, 4, t);
    FILE *o = fopen(argv[2], "wb");
    wr(o, &nslot, 1); wr(o, &t.ntile, 1); wr(o, &t.max_halo, 1);
    int64_t nh = (int64_t)t.hcol.size();
    wr(o, &nh, 1);
    wr(o, t.base.data(), t.ntile + 1); wr(o, t.width.data(), t.ntile); wr(o, t.row.data(), t.ntile * tr);
    wr(o, t.hptr.data(), t.ntile + 1); wr(o, t.hcol.data(), nh);
    wr(o, t.perm.data(), nslot); wr(o, t.lcol.data(), nslot);
    fclose(o);
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("tiles")
    src = d / "main.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run(["g++", "-O2", "-std=c++17", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{CUDA_INC}", str(src), os.path.join(CSRC, "tiles.cpp"), "-o", str(exe)],
                   check=True, capture_output=True)
    return d, exe


def _run(harness, rowptr, col, order, tr):
    d, exe = harness
    n = len(rowptr) - 1
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        np.array([n, len(col), tr], np.int64).tofile(f)
        np.asarray(rowptr, np.int32).tofile(f)
        np.asarray(col, np.int32).tofile(f)
        np.asarray(order, np.int32).tofile(f)
    subprocess.run([str(exe), str(inp), str(out)], check=True, timeout=120)
    b = open(out, "rb").read()
    pos = 0

    def take(dtype, k):
        nonlocal pos
        a = np.frombuffer(b, dtype, k, pos)
        pos += a.nbytes
        return a
    nslot, ntile, max_halo, nh = (int(v) for v in take(np.int64, 4))
    r = dict(nslot=nslot, ntile=ntile, max_halo=max_halo)
    r["base"], r["width"] = take(np.int64, ntile + 1), take(np.int32, ntile)
    r["row"] = take(np.int32, ntile * tr).reshape(ntile, tr)
    r["hptr"], r["hcol"] = take(np.int64, ntile + 1), take(np.int32, nh)
    r["perm"], r["lcol"] = take(np.int32, nslot), take(np.int32, nslot)
    return r


def _morton(x):
    """Points sorted along a Morton curve (the tiles only need some order
    of nearby points; the library uses its own)."""
    q = np.clip((x - x.min(0)) / (np.ptp(x, 0) + 1e-300), 0, 1)
    q = (q * 1023).astype(np.int64)
    code = np.zeros(len(x), np.int64)
    for b in range(10):
        for a in range(x.shape[1]):
            code |= ((q[:, a] >> b) & 1) << (x.shape[1] * b + a)
    return np.argsort(code, kind="stable").astype(np.int32)


# the larger cases have enough tiles to run the builder on several host threads
@pytest.mark.parametrize("dim,side,tr", [(2, 13, 64), (2, 30, 64), (2, 30, 16), (3, 7, 64), (3, 6, 8),
                                         (2, 48, 8), (3, 9, 4)])
def test_tiles_cover_the_pattern_once(harness, dim, side, tr):
    x, h = mi.jittered_lattice(side, dim, 77 + side)
    R = np.full(len(x), 2.0 * h)
    rowptr, col = O.neighbors(x, R)
    n = len(x)
    order = _morton(x)
    r = _run(harness, rowptr, col, order, tr)
    assert r["ntile"] == -(-n // tr)
    # rows: the given order, -1 past n
    rows = r["row"].ravel()
    assert np.array_equal(rows[:n], order) and np.all(rows[n:] == -1)
    rowlen = np.diff(rowptr)
    seen = np.zeros(len(col), np.int64)
    for t in range(r["ntile"]):
        b0, b1, w = r["base"][t], r["base"][t + 1], r["width"][t]
        live = r["row"][t][r["row"][t] >= 0]
        assert w == -(-rowlen[live].max() // 4) * 4 and b1 - b0 == w * tr   # longest row, rounded up to 4
        halo = r["hcol"][r["hptr"][t]:r["hptr"][t + 1]]
        assert np.array_equal(halo, np.unique(np.concatenate([col[rowptr[i]:rowptr[i + 1]] for i in live])))
        perm = r["perm"][b0:b1].reshape(w, tr)
        lcol = r["lcol"][b0:b1].reshape(w, tr)
        assert np.all((lcol >= 0) & (lcol < len(halo)))
        for s in range(tr):
            i = r["row"][t][s]
            if i < 0:
                assert np.all(perm[:, s] == -1)
                continue
            k = rowlen[i]
            # entry k of row slot s holds pattern entry rowptr[i] + k, in column order
            assert np.array_equal(perm[:k, s], np.arange(rowptr[i], rowptr[i + 1]))
            assert np.array_equal(halo[lcol[:k, s]], col[rowptr[i]:rowptr[i + 1]])
            assert np.all(perm[k:, s] == -1) and np.all(lcol[k:, s] == 0)
        seen[perm[perm >= 0]] += 1
    assert np.all(seen == 1)
    assert r["max_halo"] == max(r["hptr"][t + 1] - r["hptr"][t] for t in range(r["ntile"]))
