"""GPU element Jacobians and Newton-GMRES against the oracle.

* k_e (32 x 32, volume + Nitsche) of Out, Intercepted and In elements against the oracle's
  element matrix (built column by column from its exact tangent): FP64 <= 1e-10 relative.
* Newton-GMRES (FP64 and mixed J v, block-Jacobi): the oracle's own float64 residual evaluated at
  the GPU solution is below 1e-8 of its value at the start (the oracle judges convergence).
* On a small mesh the GPU solution equals the oracle Newton-GMRES solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.krylov import newton as oracle_newton
from oracle.oracle import OracleMesh
from tests.oracle_assembly import assemble_jacobian
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


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
    return w, api.Mesh.from_workload(w, device=0, triangles=tri), OracleMesh(w.lo, w.hi, w.base_level, w.regions, tri,
                                                                             w.lmax)


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_element_jacobians_match_oracle(sphere, dev):
    w, g, o = sphere
    u, up, _ = I.state(g.n_nodes, 11)
    mk, _ = g.markers()
    sq = g.surface_points()
    with_surface = np.unique(sq[:, 8].astype(np.int64))
    outs = np.where(mk == 0)[0]
    elems = np.concatenate([outs[:: max(1, outs.size // 40)], np.where(mk == 2)[0][:25], with_surface[:15],
                            np.where(mk == 1)[0][:3]])
    elems = np.unique(elems).astype(np.int32)
    for prec, tol in ((api.PRECISION_FP64, 1e-10), (api.PRECISION_MIXED, 5e-5)):
        K = g.element_jacobians(w.physics, T(u, dev), T(up, dev), T(elems, dev), precision=prec).cpu().numpy()
        for i, e in enumerate(elems):
            Ko, _ = o.element_matrix(w.physics, u, up, int(e))
            scale = max(np.linalg.norm(Ko), 1e-300)
            assert np.linalg.norm(K[i] - Ko) <= tol * scale, (prec, int(e), mk[e], np.linalg.norm(K[i] - Ko) / scale)


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_newton_converges_judged_by_oracle(sphere, dev, prec):
    w, g, o = sphere
    u, up, _ = I.state(g.n_nodes, 12)
    R0 = np.linalg.norm(o.residual(w.physics, u, up))
    ud = T(u, dev)
    st = g.newton_step(w.physics, ud, T(up, dev), precision=prec, precond=1, rtol=1e-8, gmres_m=50)
    assert st["converged"] and st["newton_its"] >= 1
    Rg = np.linalg.norm(o.residual(w.physics, ud.cpu().numpy(), up))
    assert Rg <= 1.5e-8 * R0, (Rg / R0, st)


def strong_mask(o):
    """Rows the residual replaces (box Dirichlet rows and nodes of In elements only)."""
    ijk = o.node_ijk.astype(np.int64)
    outlet = ijk[:, 0] == o.hiI[0]
    other = (ijk == 0).any(1) | (ijk[:, 1] == o.hiI[1]) | (ijk[:, 2] == o.hiI[2])
    mask = np.where(other, 7, 0).astype(np.uint8) | np.where(outlet, 8, 0).astype(np.uint8)
    mk, _, _ = o.markers()
    active = np.zeros(o.n_nodes, bool)
    for el in np.where(mk != 1)[0]:
        for cc in range(8):
            idx = o.conn[el, cc]
            if idx < o.n_nodes:
                active[idx] = True
            else:
                active[o.hang_parents[idx - o.n_nodes, :o.hang_np[idx - o.n_nodes]]] = True
    mask[~active] = 15
    return mask


def test_newton_matches_oracle_solver(dev):
    c = (0.5, 0.5, 0.5)
    regs = [I.Region(I.REGION_SPHERE_BAND, 4, (*c, 0.2, 0.05))]
    tri = I.icosphere(2, 0.2, c, 1e-4, 1)
    g = api.Mesh((0, 0, 0), (1, 1, 1), 2, regs, tri, 2, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 2, regs, tri, 2)
    ph = I.Physics(rho=1.0, mu=0.05, dt=0.02)
    u, up, _ = I.state(g.n_nodes, 13)
    ud = T(u, dev)
    g.newton_step(ph, ud, T(up, dev), precision=api.PRECISION_FP64, precond=1, rtol=1e-10, krylov_rtol=1e-6)
    R = lambda x: o.residual(ph, x.reshape(-1, 4), up).ravel()
    J = lambda x, v: o.jvp(ph, x.reshape(-1, 4), up, v.reshape(-1, 4)).ravel()

    def exact_inverse(x):   # sparse LU of the oracle's assembled Jacobian: GMRES then needs ~1 iteration
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        Jx = assemble_jacobian(o, ph, x.reshape(-1, 4), up, None, strong_mask(o)).tocsr()
        # dofs of Intercepted elements whose sub-cell points are all In have empty rows (R = 0
        # there); a unit diagonal keeps them fixed, as GMRES started from zero does
        empty = np.diff(Jx.indptr) == 0
        empty |= np.asarray(abs(Jx).sum(axis=1)).ravel() == 0.0
        Jx = Jx + sp.diags(empty.astype(float))
        return spla.splu(Jx.tocsc()).solve

    uo, st = oracle_newton(R, J, u.ravel(), rtol=1e-10, gmres_m=20, gmres_rtol=1e-6, precond_factory=exact_inverse)
    assert st["converged"]
    ug = ud.cpu().numpy().ravel()
    assert np.linalg.norm(ug - uo) <= 1e-7 * np.linalg.norm(uo)


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_graph_replayed_gmres_matches_host_driven(sphere, dev, prec):
    """With CUDA graphs on, GMRES keeps its Hessenberg matrix and rotations on the device and replays
    one captured Arnoldi step; the Newton solve is the same as the host-driven one."""
    w, g, o = sphere
    u, up, _ = I.state(g.n_nodes, 14)
    R0 = np.linalg.norm(o.residual(w.physics, u, up))
    out = {}
    try:
        for graphs in (False, True):
            g.use_graphs(graphs)
            ud = T(u, dev)
            st = g.newton_step(w.physics, ud, T(up, dev), precision=prec, precond=1, rtol=1e-8, gmres_m=50)
            assert st["converged"], (graphs, st)
            assert np.linalg.norm(o.residual(w.physics, ud.cpu().numpy(), up)) <= 1.5e-8 * R0
            out[graphs] = st
    finally:
        g.use_graphs(False)
    assert out[True]["newton_its"] == out[False]["newton_its"]
    # J v is bitwise reproducible (deterministic scatter); the two drivers differ only in where the
    # Givens rotations and reductions are computed (host against device arithmetic)
    assert abs(out[True]["krylov_its"] - out[False]["krylov_its"]) <= 0.02 * out[False]["krylov_its"] + 2, out


@pytest.mark.parametrize("precond", [1, 4])
def test_whole_newton_solve_as_one_graph(sphere, dev, precond):
    """With CUDA graphs on, the whole Newton solve is one graph launch: WHILE nodes for the Newton
    iterations, the GMRES restart cycles, the Arnoldi steps and the line search, their conditions set
    on the device.  It takes the same steps as the host-driven solver, up to the last bits of the
    preconditioner (its setup adds with atomics)."""
    w, g, o = sphere
    u, up, _ = I.state(g.n_nodes, 15)
    R0 = np.linalg.norm(o.residual(w.physics, u, up))
    out = {}
    kw = dict(precision=api.PRECISION_MIXED, precond=precond, rtol=1e-8, gmres_m=50,
              max_krylov=1000, max_newton=12)
    try:
        for graphs in (False, True):
            g.use_graphs(graphs)
            ud = T(u, dev)
            st = g.newton_step(w.physics, ud, T(up, dev), **kw)
            assert st["converged"], (graphs, st)
            assert np.linalg.norm(o.residual(w.physics, ud.cpu().numpy(), up)) <= 1.5e-8 * R0
            out[graphs] = (st, ud.cpu().numpy())
    finally:
        g.use_graphs(False)
    (sh, uh), (sg, ug) = out[False], out[True]
    print(f"precond {precond}: host {sh['krylov_per_newton']} {sh['time_ms']:.0f} ms; "
          f"graph {sg['krylov_per_newton']} {sg['time_ms']:.0f} ms")
    assert sg["newton_its"] == sh["newton_its"]
    assert abs(sg["krylov_its"] - sh["krylov_its"]) <= 0.02 * sh["krylov_its"] + 2
    assert np.linalg.norm(ug - uh) <= 1e-6 * np.linalg.norm(uh)
