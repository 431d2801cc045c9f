"""3D cells on the device (Sec. 3.1): the device builder (one thread per
cell, cells3d.cu, the default) against the host builder (geometry.cpp,
pinned against the oracle on the CPU in test_host_geometry.py).

Both run the same clipping in the same arithmetic (no floating-point
contraction), so the volumes and the element counts are identical, bit for
bit, and the integrated forms agree to the rounding of the assembly's atomic
sums; the oracle's forms on the same points are checked in test_gpu_3d.py.
Jittered and regular lattices, boundary-dominated and interior cells, and
the full 40^3 configuration."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402


def _build(prob, where):
    tp = pkg.TransportProblem.from_problem(prob, cells_3d=where)
    t0 = time.perf_counter()
    tp.integrate()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return tp, dt


@pytest.mark.parametrize("side,jitter", [(5, 0.2), (6, 0.0), (12, 0.2), (40, 0.2)])
def test_device_cells_equal_host_cells(side, jitter):
    prob = mi.make_problem(f"3d-{side}", side, 3, 4, 3300 + side, 1.0, 0.5, 1.0, 0.01, 1, jitter=jitter)
    dev, t_dev = _build(prob, 0)
    host, t_host = _build(prob, 1)
    try:
        sd, sh = dev.stats(), host.stats()
        print(f"{side}^3 jitter {jitter}: cells in {t_dev:.3f} s on the device, {t_host:.3f} s on the host; "
              f"{sd['n_volume_qp'] // 8} tetrahedra")
        assert sd["n_volume_qp"] == sh["n_volume_qp"] and sd["n_boundary_qp"] == sh["n_boundary_qp"]
        Vd, Vh = dev.volumes(), host.volumes()
        assert np.array_equal(Vd, Vh)
        assert abs(Vd.sum() - 1.0) < 1e-12
        if side <= 12:
            dev.assemble()
            host.assemble()
            md, vd = dev.forms()
            mh, vh = host.forms()
            for k in range(md.shape[0]):
                assert np.abs(md[k] - mh[k]).max() <= 1e-13 * max(np.abs(mh[k]).max(), 1e-300), k
            for k in range(vd.shape[0]):
                assert np.abs(vd[k] - vh[k]).max() <= 1e-13 * max(np.abs(vh[k]).max(), 1e-300), k
    finally:
        dev.close()
        host.close()
