"""GPU: the deterministic scatter (o2n of Algorithm 2 in a fixed order, IMGA_OPT_DETERMINISTIC).

Element kernels write their contributions to slots and one pass over the nodes sums them in the
order of the mesh's incidence list, so repeated calls give the same bits: R and J v in float64 and
in mixed precision, on an ordinary and on a batched mesh, and Krylov solves (same iterates).  The atomic scatter (option off) agrees with it to rounding, and both agree
with the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_repeated_calls_are_bitwise_identical(dev, sphere, prec):
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 2)
    up2 = up.copy()
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=I.SCHEME_BDF2)
    ut, upt, up2t, vt = T(u, dev), T(up, dev), T(up2, dev), T(v, dev)
    R = [g.residual(ph, ut, upt, up2t, precision=prec).cpu().numpy() for _ in range(3)]
    J = [g.jvp(ph, ut, upt, vt, up2t, precision=prec).cpu().numpy() for _ in range(3)]
    for k in (1, 2):
        assert np.array_equal(R[k], R[0]) and np.array_equal(J[k], J[0])
    # graphs replay the same launches: same bits
    g.use_graphs(True)
    try:
        Jg = [g.jvp(ph, ut, upt, vt, up2t, precision=prec).cpu().numpy() for _ in range(2)]
    finally:
        g.use_graphs(False)
    assert np.array_equal(Jg[0], J[0]) and np.array_equal(Jg[1], J[0])
    # the atomic scatter: the same sums in another order
    g.deterministic(False)
    try:
        Ra = g.residual(ph, ut, upt, up2t, precision=prec).cpu().numpy()
        Ja = g.jvp(ph, ut, upt, vt, up2t, precision=prec).cpu().numpy()
    finally:
        g.deterministic(True)
    tol = 1e-13 if prec == api.PRECISION_FP64 else 1e-6
    print(f"precision {prec}: deterministic vs atomic R {rel(R[0], Ra):.2e} J v {rel(J[0], Ja):.2e}")
    assert rel(R[0], Ra) <= tol and rel(J[0], Ja) <= tol
    Ro, Jo = o.residual_jvp(ph, u, up, up2, v=v)
    bar = 1e-10 if prec == api.PRECISION_FP64 else 2e-5
    print(f"precision {prec}: vs oracle R {rel(R[0], Ro):.2e} J v {rel(J[0], Jo):.2e}")
    assert rel(R[0], Ro) <= bar and rel(J[0], Jo) <= bar


def test_batched_mesh_bitwise_identical(dev):
    ws = [wl for wl, _, _ in I.batched_spheres(6)]
    b = api.Mesh.batch(ws, device=0)
    u, up, v = I.state(b.n_nodes, 4)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01)
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    for prec in (api.PRECISION_FP64, api.PRECISION_MIXED):
        J = [b.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy() for _ in range(3)]
        assert np.array_equal(J[1], J[0]) and np.array_equal(J[2], J[0])


@pytest.mark.parametrize("graphs", [False, True])
def test_krylov_solves_repeat_exactly(dev, sphere, graphs):
    """One Newton iteration with 40 unpreconditioned GMRES iterations, twice: J v, the Gram-Schmidt
    reductions (fixed grids) and the residual are all reproducible, so the iterates are too.  (The
    block-Jacobi diagonal and the assembled matrix still add with atomics.)"""
    w, g, o = sphere
    u0, up, _ = I.state(g.n_nodes, 14)
    upt = T(up, dev)
    runs = []
    g.use_graphs(graphs)
    try:
        for _ in range(2):
            u = T(u0, dev)
            st = g.newton_step(w.physics, u, upt, precision=api.PRECISION_MIXED, precond=0, max_newton=1,
                               max_krylov=40, krylov_rtol=1e-12, raise_on_failure=False)
            runs.append((st, u.cpu().numpy()))
    finally:
        g.use_graphs(False)
    (s0, u0r), (s1, u1r) = runs
    print(f"graphs {graphs}: Krylov {s0['krylov_per_newton']} |R| {s0['res_norm']}")
    assert s0["krylov_per_newton"] == s1["krylov_per_newton"] and s0["res_norm"] == s1["res_norm"]
    assert np.array_equal(u0r, u1r)


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_side_streams_give_the_same_bits(dev, sphere, prec):
    """The Intercepted-element and surface kernels on side streams beside the Out-element kernel
    (IMGA_OPT_CONCURRENT, the default) or all on the caller's stream: the same slots, the same sums."""
    w, g, o = sphere
    u, up, v = I.state(g.n_nodes, 5)
    ph = w.physics
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    out = {}
    try:
        for conc in (True, False):
            g.concurrent(conc)
            out[conc] = (g.residual(ph, ut, upt, precision=prec).cpu().numpy(),
                         g.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy())
            g.use_graphs(True)
            out[(conc, "graph")] = g.jvp(ph, ut, upt, vt, precision=prec).cpu().numpy()
            g.use_graphs(False)
    finally:
        g.use_graphs(False)
        g.concurrent(True)
    assert np.array_equal(out[True][0], out[False][0]) and np.array_equal(out[True][1], out[False][1])
    assert np.array_equal(out[(True, "graph")], out[True][1]) and np.array_equal(out[(False, "graph")], out[True][1])
