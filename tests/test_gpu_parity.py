"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, same seeded inputs.

Bars:
* integer / flag / index work (markers, corner flags, in/out flags, sub-cell point lists,
  surface points): bit-exact;
* FP64 residual and J v: relative L2 error <= 1e-10 (and max-abs reported);
* mixed precision (FP32 element arithmetic, FP64 gathers / accumulation / Nitsche penalty):
  relative L2 error <= 2e-5 for R and J v, a bound from FP32 rounding (~6e-8 per operation, a few
  hundred dependent operations per element, cancellation in the momentum rows bounded by the
  ratio of term magnitudes to the row norm).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def sphere(dev):
    w = I.small_sphere()
    tri = w.triangles()
    g = api.Mesh.from_workload(w, device=0, triangles=tri)
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)
    return w, g, o


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def test_mesh_tables_match(sphere):
    w, g, o = sphere
    ex = g.export()
    assert np.array_equal(ex["conn"], o.conn) and np.array_equal(ex["node_ijk"], o.node_ijk)


def test_markers_and_corner_flags_bit_exact(sphere):
    w, g, o = sphere
    mk, cf = g.markers()
    omk, ocf, _ = o.markers()
    assert np.array_equal(mk, omk)
    assert np.array_equal(cf, ocf)
    assert (mk == 2).sum() > 100 and (mk == 1).sum() > 10


def test_cut_points_bit_exact(sphere):
    w, g, o = sphere
    off, pts = g.cut_points()
    mk, _ = g.markers()
    for e in np.where(mk == 2)[0]:
        q = o.cut_points(e)
        assert off[e + 1] - off[e] == q.shape[0], e
        assert np.array_equal(pts[off[e]:off[e + 1]], q), e


def test_surface_points_bit_exact(sphere):
    w, g, o = sphere
    assert np.array_equal(g.surface_points(), o.surface_points())


def _classify_points():
    pts = I.uniform(99, 3 * 20000).reshape(-1, 3)
    # concentrate half of the points around the sphere surface, where the test is hardest
    r = 0.1 + 0.01 * (I.uniform(98, 10000) - 0.5)
    d = I.normal(97, 30000).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1)[:, None]
    pts[:10000] = 0.5 + r[:, None] * d
    pts[0] = (-0.1, 0.5, 0.5)        # outside the box
    return pts


def test_classify_bit_exact(sphere, dev):
    w, g, o = sphere
    pts = _classify_points()
    f = g.classify(T(pts, dev)).cpu().numpy()
    assert np.array_equal(f, o.classify(pts))
    assert g.classify(T(np.zeros((0, 3)), dev)).numel() == 0


def test_classify_counts_and_ray_only_mode(sphere, dev):
    """Points in elements without background triangles take the stored marker; the normal test of
    Algorithm 6 is given to, and decides, exactly the points the oracle's is given and decides;
    rays go to the undecided ones only.  The ray-only mode (the conventional test of Table in-out)
    sends every point in the box to a ray and gives the same flags."""
    w, g, o = sphere
    pts = _classify_points()
    n_box = int(np.all((pts >= 0.0) & (pts < 1.0), axis=1).sum())
    P = T(pts, dev)
    g.classify_counts(reset=True)
    f = g.classify(P).cpu().numpy()
    cnt = g.classify_counts(reset=True)
    c0 = o.counters()
    of = o.classify(pts)
    c1 = o.counters()
    assert np.array_equal(f, of)
    assert cnt["marker"] + cnt["normal_tests"] == n_box
    assert cnt["normal_tests"] == c1["normal_tests"] - c0["normal_tests"]
    assert cnt["normal_decided"] == c1["normal_decided"] - c0["normal_decided"]
    assert cnt["rays"] == cnt["normal_tests"] - cnt["normal_decided"]
    # the oracle casts a ray for every point of an element without triangles as well
    assert c1["rays"] - c0["rays"] == cnt["rays"] + cnt["marker"]
    assert cnt["marker"] > 1000 and cnt["normal_decided"] > 0.5 * cnt["normal_tests"] and cnt["rays"] > 0
    g.classify_rays_only(True)
    try:
        fr = g.classify(P).cpu().numpy()
        cr = g.classify_counts(reset=True)
    finally:
        g.classify_rays_only(False)
    assert np.array_equal(fr, of)
    assert cr == {"marker": 0, "normal_tests": 0, "normal_decided": 0, "rays": n_box}


@pytest.mark.parametrize("seed", [0, 1])
def test_residual_and_jvp_fp64(sphere, dev, seed):
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, seed)
    R_o, J_o = o.residual_jvp(w.physics, u, up, v=v)
    R = g.residual(w.physics, T(u, dev), T(up, dev)).cpu().numpy()
    J = g.jvp(w.physics, T(u, dev), T(up, dev), T(v, dev)).cpu().numpy()
    assert rel(R, R_o) <= FP64_TOL, rel(R, R_o)
    assert rel(J, J_o) <= FP64_TOL, rel(J, J_o)


def test_residual_and_jvp_mixed(sphere, dev):
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 2)
    R_o, J_o = o.residual_jvp(w.physics, u, up, v=v)
    R = g.residual(w.physics, T(u, dev), T(up, dev), precision=api.PRECISION_MIXED).cpu().numpy()
    J = g.jvp(w.physics, T(u, dev), T(up, dev), T(v, dev), precision=api.PRECISION_MIXED).cpu().numpy()
    assert rel(R, R_o) <= MIXED_TOL, rel(R, R_o)
    assert rel(J, J_o) <= MIXED_TOL, rel(J, J_o)


@pytest.mark.parametrize("scheme", [I.SCHEME_CN, I.SCHEME_BDF2])
def test_time_schemes_fp64(sphere, dev, scheme):
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 4)
    up2 = up.copy()
    up2[:, :3] += I.normal(5, 3 * g.n_nodes, 0.01).reshape(-1, 3)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=scheme, g=(0.1, 0.0, 0.0))
    R_o, J_o = o.residual_jvp(ph, u, up, up2, v=v)
    R = g.residual(ph, T(u, dev), T(up, dev), T(up2, dev)).cpu().numpy()
    J = g.jvp(ph, T(u, dev), T(up, dev), T(v, dev), T(up2, dev)).cpu().numpy()
    assert rel(R, R_o) <= FP64_TOL and rel(J, J_o) <= FP64_TOL, (rel(R, R_o), rel(J, J_o))


def test_hanging_mesh_body_force_and_user_dirichlet(dev):
    regs = [I.Region(I.REGION_SPHERE_BAND, 5, (0.4, 0.55, 0.5, 0.2, 0.03))]
    g = api.Mesh((0, 0, 0), (1, 1, 1), 2, regs, None, 3, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 2, regs)
    assert g.n_hang > 0
    u, up, v = I.state(g.n_nodes, 6, sigma=0.3)
    f = np.zeros((g.n_nodes, 4))
    f[:, :3] = I.normal(8, 3 * g.n_nodes).reshape(-1, 3)
    ph = I.Physics(rho=1.3, mu=0.05, dt=0.02, drop_visc=0)
    R_o, J_o = o.residual_jvp(ph, u, up, f=f, v=v)
    R = g.residual(ph, T(u, dev), T(up, dev), f=T(f, dev)).cpu().numpy()
    J = g.jvp(ph, T(u, dev), T(up, dev), T(v, dev), f=T(f, dev)).cpu().numpy()
    assert rel(R, R_o) <= FP64_TOL and rel(J, J_o) <= FP64_TOL
    mask = (np.arange(g.n_nodes) % 7 == 0).astype(np.uint8) * 9
    vals = I.normal(12, 4 * g.n_nodes).reshape(-1, 4)
    o.set_dirichlet(mask, vals)
    g.set_dirichlet(torch.from_numpy(mask).to(dev), T(vals, dev))
    R_o = o.residual(ph, u, up, f=f)
    R = g.residual(ph, T(u, dev), T(up, dev), f=T(f, dev)).cpu().numpy()
    assert rel(R, R_o) <= FP64_TOL
    g.set_dirichlet(None, None)


def test_uniform_flow_with_moving_body_is_zero(sphere, dev):
    w, g, o = sphere
    ub = (0.8, 0.3, -0.2)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, g=ub, uinf=ub)
    U = np.zeros((g.n_nodes, 4))
    U[:, :3] = ub
    for prec in (api.PRECISION_FP64, api.PRECISION_MIXED):
        R = g.residual(ph, T(U, dev), T(U, dev), precision=prec).cpu().numpy()
        assert np.abs(R).max() <= (1e-13 if prec == 0 else 1e-6)


def test_bad_arguments_return_status(sphere, dev):
    w, g, o = sphere
    u = torch.zeros((g.n_nodes, 4), dtype=torch.float64, device=dev)
    with pytest.raises(_lib.ImgaError):
        g.residual(I.Physics(dt=-1.0), u, u)
    with pytest.raises(_lib.ImgaError):
        g.residual(I.Physics(scheme=I.SCHEME_BDF2), u, u)       # BDF2 without u_prev2
