"""GPU parity of the Nitsche terms of Eq. (weakbc), row by row.

* The exact linear flow past an immersed box (the oracle pin of test_oracle_nitsche.py) through the
  C ABI: with g = u_exact per surface point (imga_physics.g_points) every free row of the device
  residual vanishes, in float64 and in mixed precision, and R and J v at a perturbed state match
  the oracle row by row.
* A velocity per surface point (a rotating body) on the small sphere: R and J v against the
  oracle, relative L2 and the largest row error relative to the largest row.
* Sliver cut cells: a box body 0.005 h from element faces, so h_b sits on its floor 0.01 h and
  tau_B = 100 C_b mu / h.  The mixed path keeps the jump and the penalty in float64; its error on
  the rows of surface-hosting elements is bounded relative to those rows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sparse as S
from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I
from tests.test_oracle_nitsche import A_LIN, BODY_HI, BODY_LO, U0, _box_face_nodes, _linear_state

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def row_err(a, b, rows=None):
    """Largest |a - b| over the rows (node, component) relative to the largest |b| there."""
    d, r = np.abs(a - b), np.abs(b)
    if rows is not None:
        d, r = d[rows], r[rows]
    return float(d.max() / max(r.max(), 1e-300))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def _pair(dev, lo, hi, base, regions, tri, lmax=3):
    g = api.Mesh(lo, hi, base, regions, tri, lmax, device=0)
    o = OracleMesh(lo, hi, base, regions, tri, lmax)
    assert np.array_equal(g.surface_points(), o.surface_points())
    return g, o


@pytest.fixture(scope="module")
def box_body(dev):
    reg = [I.Region(I.REGION_BOX, 4, (0.25, 0.25, 0.25, 0.75, 0.75, 0.75))]
    tri = I.grid_box(BODY_LO, BODY_HI, 1 / 16)
    return _pair(dev, (0, 0, 0), (1, 1, 1), 3, reg, tri)


def test_exact_linear_flow_rows_vanish_on_the_device(dev, box_body):
    g, o = box_body
    U, F = _linear_state(o, 0.4)
    face = _box_face_nodes(o)
    mask = np.where(face, 7, 0).astype(np.uint8)
    o.set_dirichlet(mask, U)
    g.set_dirichlet(torch.from_numpy(mask).to(dev), T(U, dev))
    free = ((S.strong_mask(o)[:, None] >> np.arange(4)[None, :]) & 1) == 0
    sq = g.surface_points()
    gp = T(U0 + sq[:, :3] @ A_LIN.T, dev)
    ph = I.Physics(rho=1.2, mu=0.05, dt=0.02, scheme=I.SCHEME_BDF2)
    Ut, Ft = T(U, dev), T(F, dev)
    scale = np.abs(g.residual(ph, Ut, Ut, Ut, f=Ft).cpu().numpy()[free]).max()    # g = 0 on the body
    assert scale > 1e-4
    R64 = g.residual(ph, Ut, Ut, Ut, f=Ft, g_points=gp).cpu().numpy()
    R32 = g.residual(ph, Ut, Ut, Ut, f=Ft, precision=api.PRECISION_MIXED, g_points=gp).cpu().numpy()
    e64, e32 = np.abs(R64[free]).max() / scale, np.abs(R32[free]).max() / scale
    print(f"exact linear flow: free rows / scale  fp64 {e64:.2e}  mixed {e32:.2e}")
    assert e64 <= 1e-12
    assert e32 <= 1e-5
    # a perturbed state, row by row against the oracle (same per-point g on both sides)
    Up = U.copy()
    Up[:, :3] += 0.05 * I.normal(3, 3 * o.n_nodes).reshape(-1, 3)
    V = I.normal(4, 4 * o.n_nodes).reshape(-1, 4)
    o.set_surface_velocity(U0 + o.surface_points()[:, :3] @ A_LIN.T)
    try:
        Ro, Jo = o.residual_jvp(ph, Up, U, U, f=F, v=V)
    finally:
        o.set_surface_velocity(None)
    Upt, Vt = T(Up, dev), T(V, dev)
    for prec, tol in ((api.PRECISION_FP64, FP64_TOL), (api.PRECISION_MIXED, MIXED_TOL)):
        R = g.residual(ph, Upt, Ut, Ut, f=Ft, precision=prec, g_points=gp).cpu().numpy()
        J = g.jvp(ph, Upt, Ut, Vt, Ut, f=Ft, precision=prec, g_points=gp).cpu().numpy()
        print(f"perturbed, precision {prec}: R rel {rel(R, Ro):.2e} row {row_err(R, Ro):.2e}  "
              f"J v rel {rel(J, Jo):.2e} row {row_err(J, Jo):.2e}")
        assert rel(R, Ro) <= tol and rel(J, Jo) <= tol
        assert row_err(R, Ro) <= 10 * tol and row_err(J, Jo) <= 10 * tol
    g.set_dirichlet()


@pytest.fixture(scope="module")
def sphere(dev):
    w = I.small_sphere()
    tri = w.triangles()
    return (w,) + _pair(dev, w.lo, w.hi, w.base_level, w.regions, tri, w.lmax)


def _rotating(x, c=(0.5, 0.5, 0.5), omega=(0.3, -1.1, 0.7), vel=(0.2, 0.0, -0.1)):
    return np.asarray(vel) + np.cross(np.asarray(omega), x - np.asarray(c))


@pytest.mark.parametrize("scheme", [I.SCHEME_BE, I.SCHEME_CN])
def test_point_velocity_rotating_body_matches_oracle(dev, sphere, scheme):
    w, g, o = sphere
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=scheme)
    u, up, v = I.state(g.n_nodes, 5)
    o.set_surface_velocity(_rotating(o.surface_points()[:, :3]))
    try:
        Ro, Jo = o.residual_jvp(ph, u, up, v=v)
    finally:
        o.set_surface_velocity(None)
    gp = T(_rotating(g.surface_points()[:, :3]), dev)
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    for prec, tol in ((api.PRECISION_FP64, FP64_TOL), (api.PRECISION_MIXED, MIXED_TOL)):
        R = g.residual(ph, ut, upt, precision=prec, g_points=gp).cpu().numpy()
        J = g.jvp(ph, ut, upt, vt, precision=prec, g_points=gp).cpu().numpy()
        print(f"rotating body, precision {prec}: R rel {rel(R, Ro):.2e} row {row_err(R, Ro):.2e}  "
              f"J v rel {rel(J, Jo):.2e} row {row_err(J, Jo):.2e}")
        assert rel(R, Ro) <= tol and rel(J, Jo) <= tol
        assert row_err(R, Ro) <= 10 * tol and row_err(J, Jo) <= 10 * tol
    # without g_points the residual differs (the per-point velocity is read; the volume terms
    # dominate R, so the difference is a few 1e-4 of it)
    R0 = g.residual(ph, ut, upt).cpu().numpy()
    assert rel(R0, Ro) > 1e-4


# a box body whose faces are 0.005 h (level-4 h = 1/16) inside element faces: sliver cut cells
SLIVER_LO = (12.01 / 32, 10.01 / 32, 14.01 / 32)
SLIVER_HI = (19.99 / 32, 17.99 / 32, 21.99 / 32)


@pytest.fixture(scope="module")
def sliver(dev):
    reg = [I.Region(I.REGION_BOX, 4, (0.25, 0.25, 0.25, 0.75, 0.75, 0.75))]
    tri = I.grid_box(SLIVER_LO, SLIVER_HI, 1 / 16)
    return _pair(dev, (0, 0, 0), (1, 1, 1), 3, reg, tri)


def test_sliver_cut_cells_mixed_penalty_rows(dev, sliver):
    g, o = sliver
    sq = g.surface_points()
    h4 = 1 / 16
    # 56 Intercepted elements keep no volume point; h_b is on its floor at the points of the 24
    # elements inside the faces (the others reach a corner beyond a body edge)
    assert sq.shape[0] > 1000 and (np.abs(sq[:, 7] - 0.01 * h4) <= 1e-15).mean() >= 0.2
    hosts = np.unique(sq[:, 8].astype(np.int64))
    ex = g.export()
    rows = np.zeros((g.n_nodes, 4), bool)
    for e in hosts:
        for c in range(8):
            idx = ex["conn"][e, c]
            if idx < g.n_nodes:
                rows[idx, :3] = True
            else:
                h = idx - g.n_nodes
                rows[ex["hang_parents"][h, :ex["hang_np"][h]], :3] = True
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01)
    u, up, v = I.state(g.n_nodes, 11)
    Ro, Jo = o.residual_jvp(ph, u, up, v=v)
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    R64 = g.residual(ph, ut, upt).cpu().numpy()
    J64 = g.jvp(ph, ut, upt, vt).cpu().numpy()
    R32 = g.residual(ph, ut, upt, precision=api.PRECISION_MIXED).cpu().numpy()
    J32 = g.jvp(ph, ut, upt, vt, precision=api.PRECISION_MIXED).cpu().numpy()
    er64, ej64 = row_err(R64, Ro, rows), row_err(J64, Jo, rows)
    er32, ej32 = row_err(R32, Ro, rows), row_err(J32, Jo, rows)
    print(f"sliver rows ({rows.sum()}): fp64 R {er64:.2e} J v {ej64:.2e}; mixed R {er32:.2e} J v {ej32:.2e}")
    assert er64 <= 1e-12 and ej64 <= 1e-12
    assert er32 <= 1e-6 and ej32 <= 1e-6
