"""Bluff-body pair: two trucks (each a filleted cab and trailer, two disjoint closed surfaces) in
tandem in a 16 L x 2 L x 2 L box, Re 1e6, BDF2.

* Reduced levels (same geometry, levels 5-8, ~30 k elements, 6,912 triangles): the oracle checks
  everything -- mesh tables, markers and corner flags, sub-cell and surface points bit-exact;
  R and J v within 1e-10 (float64) and 2e-5 (mixed).
* Full size (19,791,080 elements, 397,488 triangles), where the oracle is too slow, properties that
  hold at any size: uniform flow with both bodies moving with it gives R = 0; the mixed J v
  agrees with the float64 J v within the mixed bound; graph replay equals the direct call; the
  Intercepted elements carry at most 4096 sub-cell points (none where all fell inside a body).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    return torch.device("cuda:0")


def test_reduced_pair_matches_oracle(dev):
    w = I.bluff_pair(0, levels=-3, n_per_edge=12)
    tri = w.triangles()
    assert tri.shape[0] == 4 * 12 * 12 * 12
    g = api.Mesh.from_workload(w, device=0, triangles=tri)
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)
    ex = g.export()
    assert np.array_equal(ex["conn"], o.conn) and np.array_equal(ex["node_ijk"], o.node_ijk)
    mk, cf = g.markers()
    omk, ocf, _ = o.markers()
    assert np.array_equal(mk, omk) and np.array_equal(cf, ocf)
    assert (mk == 2).sum() > 300 and (mk == 1).sum() > 100
    off, pts = g.cut_points()
    for e in np.where(mk == 2)[0]:
        assert np.array_equal(pts[off[e]:off[e + 1]], o.cut_points(e)), e
    assert np.array_equal(g.surface_points(), o.surface_points())
    u, up, v = I.state(g.n_nodes, 3)
    up2 = up.copy()
    up2[:, :3] += I.normal(9, 3 * g.n_nodes, 0.01).reshape(-1, 3)
    R_o, J_o = o.residual_jvp(w.physics, u, up, up2, v=v)
    for prec, tol in ((api.PRECISION_FP64, 1e-10), (api.PRECISION_MIXED, 2e-5)):
        R = g.residual(w.physics, T(u, dev), T(up, dev), T(up2, dev), precision=prec).cpu().numpy()
        J = g.jvp(w.physics, T(u, dev), T(up, dev), T(v, dev), T(up2, dev), precision=prec).cpu().numpy()
        assert rel(R, R_o) <= tol and rel(J, J_o) <= tol, (prec, rel(R, R_o), rel(J, J_o))


def test_full_size_pair_properties(dev):
    w = I.bluff_pair(0)
    g = api.Mesh.from_workload(w, device=0)
    assert g.n_elem == 19791080 and g.n_nodes == 19520852
    info = g.info
    assert info["n_tri"] == 397488 and info["n_cut"] > 10000
    off, _ = g.cut_points()
    mk, _ = g.markers()
    cnt = np.diff(off)[mk == 2]
    # 0 where every sub-cell Gauss point fell inside a body; at most 8^(L_max + 1)
    assert cnt.min() >= 0 and cnt.max() <= 4096 and (cnt > 8).mean() > 0.5, (cnt.min(), cnt.max(), cnt.mean())
    # uniform flow, both bodies moving with it: every term of R vanishes
    ub = (0.8, 0.3, -0.2)
    ph = I.Physics(rho=1.0, mu=w.physics.mu, dt=0.01, scheme=I.SCHEME_BDF2, g=ub, uinf=ub)
    U = torch.zeros((g.n_nodes, 4), dtype=torch.float64, device=dev)
    U[:, :3] = torch.tensor(ub, dtype=torch.float64)
    for prec, tol in ((api.PRECISION_FP64, 1e-12), (api.PRECISION_MIXED, 1e-6)):
        assert g.residual(ph, U, U, U, precision=prec).abs().max().item() <= tol
    del U
    u, up, v = I.state(g.n_nodes, 1)
    ud, upd, vd = T(u, dev), T(up, dev), T(v, dev)
    J64 = g.jvp(w.physics, ud, upd, vd, upd, precision=api.PRECISION_FP64).cpu().numpy()
    J32 = g.jvp(w.physics, ud, upd, vd, upd, precision=api.PRECISION_MIXED).cpu().numpy()
    assert rel(J32, J64) <= 2e-5, rel(J32, J64)
    g.use_graphs(True)
    for _ in range(2):
        Jg = g.jvp(w.physics, ud, upd, vd, upd, precision=api.PRECISION_MIXED).cpu().numpy()
        assert rel(Jg, J32) <= 1e-6
    g.close()
