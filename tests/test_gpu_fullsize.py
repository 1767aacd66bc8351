"""Parity at the full sphere-LES size (2,001,176 elements, the bench's launch configuration), on
outputs the oracle computes one by one:

* markers of a seeded sample of 20,000 elements and the sub-cell points of 40 Intercepted elements:
  bit-exact;
* R and J v rows of a seeded sample of 3,000 nodes (the oracle evaluates every element touching
  them, through the hanging-node operator), with the autotuned tile shapes the bench uses:
  <= 1e-10 relative (float64 path), <= 2e-5 (mixed);
* graph replay of the mixed J v equals the direct call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


@pytest.fixture(scope="module")
def les():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    w = I.sphere_les(0)
    tri = w.triangles()
    g = api.Mesh.from_workload(w, device=0, triangles=tri)
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)
    assert g.n_elem == o.n_elem == 2001176 and g.n_nodes == o.n_nodes
    return w, g, o


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_sampled_markers_and_cut_points_bit_exact(les):
    w, g, o = les
    mk, cf = g.markers()
    sel = np.unique(I.splitmix64(5, 20000) % g.n_elem).astype(np.int64)
    omk, ocf, _ = o.markers(sel)
    assert np.array_equal(mk[sel], omk) and np.array_equal(cf[sel], ocf)
    off, pts = g.cut_points()
    cut = np.where(mk == 2)[0]
    assert cut.size == g.info["n_cut"] > 1000
    for e in cut[np.unique(I.splitmix64(6, 40) % cut.size)]:
        q = o.cut_points(e)
        assert np.array_equal(pts[off[e]:off[e + 1]], q), e


def test_sampled_residual_and_jvp(les):
    w, g, o = les
    dev = torch.device("cuda:0")
    u, up, v = I.state(g.n_nodes, 0)
    sel = np.unique(I.splitmix64(7, 3000) % g.n_nodes).astype(np.int64)
    Ro, Jo = o.residual_jvp(w.physics, u, up, up, v=v, nodes=sel)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ud, upd, vd = T(u), T(up), T(v)
    g.autotune(True)   # the bench's launch configuration: tuned Intercepted-element tile shapes
    for prec, tol in ((api.PRECISION_FP64, 1e-10), (api.PRECISION_MIXED, 2e-5)):
        R = g.residual(w.physics, ud, upd, upd, precision=prec).cpu().numpy()
        J = g.jvp(w.physics, ud, upd, vd, upd, precision=prec).cpu().numpy()
        assert rel(R[sel], Ro[sel]) <= tol, (prec, rel(R[sel], Ro[sel]))
        assert rel(J[sel], Jo[sel]) <= tol, (prec, rel(J[sel], Jo[sel]))
    direct = g.jvp(w.physics, ud, upd, vd, upd, precision=api.PRECISION_MIXED).cpu().numpy()
    g.use_graphs(True)
    for _ in range(2):
        rep = g.jvp(w.physics, ud, upd, vd, upd, precision=api.PRECISION_MIXED).cpu().numpy()
        assert rel(rep, direct) <= 1e-6
    g.use_graphs(False)
