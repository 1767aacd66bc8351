"""GPU: the volume buckets in one persistent launch (IMGA_OPT_FUSED).

One kernel drains a device work queue: the Intercepted elements by decreasing point count (Eq.
Wpart's volume cost), then the Out elements; the surface kernels run beside it.  The per-item
arithmetic is the bucketed kernels', so:

* with the deterministic scatter, the fused R and J v equal the bucketed ones row by row to the
  last bits that FMA contraction may change (relative 1e-13 in float64, 1e-6 in mixed), repeated
  fused calls give identical bits, and the result matches the oracle;
* with the atomic scatter, both agree to rounding;
* on a batched mesh (many problems, one queue) and inside the solvers (Newton-GMRES with the whole
  solve as one graph) the fused launch gives the same answers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


def rowmax(a, b):
    """largest row error relative to the largest reference entry"""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


@pytest.fixture(scope="module")
def sphere(dev):
    w = I.small_sphere()
    tri = w.triangles()
    g = api.Mesh.from_workload(w, device=0, triangles=tri)
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)
    return w, g, o


def both(g, ph, u, up, up2, v, prec):
    return (g.residual(ph, u, up, up2, precision=prec).cpu().numpy(),
            g.jvp(ph, u, up, v, up2, precision=prec).cpu().numpy())


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
@pytest.mark.parametrize("det", [True, False])
def test_fused_equals_bucketed_and_oracle(dev, sphere, prec, det):
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 21)
    up2 = up.copy()
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=I.SCHEME_BDF2)
    ut, upt, up2t, vt = T(u, dev), T(up, dev), T(up2, dev), T(v, dev)
    g.deterministic(det)
    try:
        Rb, Jb = both(g, ph, ut, upt, up2t, vt, prec)
        g.fused(True)
        info = g.fused_info()
        Rf, Jf = both(g, ph, ut, upt, up2t, vt, prec)
        Rf2, Jf2 = both(g, ph, ut, upt, up2t, vt, prec)
    finally:
        g.fused(False)
        g.deterministic(True)
    mk, _ = g.markers()
    assert info["on"] and info["cut_items"] == int((mk == 2).sum()) and info["out_elements"] == int((mk == 0).sum())
    assert info["dense_surface_elements"] + info["sparse_surface_points"] > 0
    tol = 1e-13 if prec == api.PRECISION_FP64 else 1e-6
    print(f"prec {prec} det {det}: fused vs bucketed R {rowmax(Rf, Rb):.2e} J v {rowmax(Jf, Jb):.2e}")
    assert rowmax(Rf, Rb) <= tol and rowmax(Jf, Jb) <= tol
    if det:
        assert np.array_equal(Rf2, Rf) and np.array_equal(Jf2, Jf)
    Ro, Jo = o.residual_jvp(ph, u, up, up2, v=v)
    bar = 1e-10 if prec == api.PRECISION_FP64 else 2e-5
    assert np.linalg.norm(Rf - Ro) <= bar * np.linalg.norm(Ro)
    assert np.linalg.norm(Jf - Jo) <= bar * np.linalg.norm(Jo)


def test_fused_on_batched_mesh(dev):
    ws = [wl for wl, _, _ in I.batched_spheres(6)]
    b = api.Mesh.batch(ws, device=0)
    u, up, v = I.state(b.n_nodes, 22)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01)
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    for prec in (api.PRECISION_FP64, api.PRECISION_MIXED):
        Rb = b.residual(ph, ut, upt, precision=prec).cpu().numpy()
        Jb = b.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy()
        b.fused(True)
        try:
            Rf = b.residual(ph, ut, upt, precision=prec).cpu().numpy()
            Jf = b.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy()
            b.use_graphs(True)
            Jg = b.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy()
        finally:
            b.use_graphs(False)
            b.fused(False)
        tol = 1e-13 if prec == api.PRECISION_FP64 else 1e-6
        assert rowmax(Rf, Rb) <= tol and rowmax(Jf, Jb) <= tol, (prec, rowmax(Rf, Rb), rowmax(Jf, Jb))
        assert np.array_equal(Jg, Jf)


def test_fused_inside_the_whole_graph_newton_solve(dev, sphere):
    w, g, o = sphere
    u, up, _ = I.state(g.n_nodes, 23)
    R0 = np.linalg.norm(o.residual(w.physics, u, up))
    kw = dict(precision=api.PRECISION_MIXED, precond=1, rtol=1e-8, gmres_m=50, max_krylov=1000, max_newton=12)
    out = {}
    try:
        for fused in (False, True):
            g.fused(fused)
            g.use_graphs(True)
            ud = T(u, dev)
            st = g.newton_step(w.physics, ud, T(up, dev), **kw)
            assert st["converged"], (fused, st)
            assert np.linalg.norm(o.residual(w.physics, ud.cpu().numpy(), up)) <= 1.5e-8 * R0
            out[fused] = st
    finally:
        g.use_graphs(False)
        g.fused(False)
    assert out[True]["newton_its"] == out[False]["newton_its"]
    assert abs(out[True]["krylov_its"] - out[False]["krylov_its"]) <= 0.02 * out[False]["krylov_its"] + 2


def test_fused_split_gives_the_same_bits(dev, sphere):
    """However many warps per block start on the Intercepted elements, every item is evaluated once by the
    same code: with the deterministic scatter the result is the same bit for bit."""
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 24)
    ph = w.physics
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    out = {}
    g.fused(True)
    try:
        for hw in (4, 3, 2, 1):
            g.fused_split(hw)
            assert g.fused_info()["heavy_first_warps"] == hw
            out[hw] = g.jvp(ph, ut, upt, vt, precision=api.PRECISION_MIXED).cpu().numpy()
    finally:
        g.fused_split(4)
        g.fused(False)
    for hw in (3, 2, 1):
        assert np.array_equal(out[hw], out[4]), hw
