"""Degenerate meshes through the C ABI against the oracle: a single element, a body smaller than an
element (invisible to the corner markers, present through its surface points), and a body that
encloses the whole box (every element In, every row a Dirichlet row)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check(g, o, ph, dev, seed):
    u, up, v = I.state(g.n_nodes, seed)
    R_o, J_o = o.residual_jvp(ph, u, up, v=v)
    for prec, tol in ((api.PRECISION_FP64, 1e-10), (api.PRECISION_MIXED, 2e-5)):
        R = g.residual(ph, T(u, dev), T(up, dev), precision=prec).cpu().numpy()
        J = g.jvp(ph, T(u, dev), T(up, dev), T(v, dev), precision=prec).cpu().numpy()
        assert rel(R, R_o) <= tol and rel(J, J_o) <= tol, (prec, rel(R, R_o), rel(J, J_o))


def test_single_element(dev):
    g = api.Mesh((0, 0, 0), (1, 1, 1), 0, [], None, 3, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 0, [])
    assert g.n_elem == 1 and g.n_nodes == 8
    _check(g, o, I.Physics(), dev, 1)


def test_body_inside_one_element(dev):
    tri = I.icosphere(2, 0.05, (0.3, 0.3, 0.3), 1e-4, 3)
    g = api.Mesh((0, 0, 0), (1, 1, 1), 1, [], tri, 3, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 1, [], tri, 3)
    mk, cf = g.markers()
    omk, ocf, _ = o.markers()
    assert np.array_equal(mk, omk) and np.array_equal(cf, ocf)
    # Algorithm 5 judges an element by its corners: all 8 are Out, so no element is Intercepted and
    # the body is seen only through its surface points (Nitsche terms inside an Out element)
    assert (mk == 0).all()
    assert np.array_equal(g.surface_points(), o.surface_points()) and len(o.surface_points()) == 960
    _check(g, o, I.Physics(), dev, 2)


def test_body_enclosing_the_box(dev):
    tri = I.rounded_box((-0.5, -0.5, -0.5), (1.5, 1.5, 1.5), 0.1, 6, 1e-4, 5)   # jittered: no grazing rays
    g = api.Mesh((0, 0, 0), (1, 1, 1), 2, [], tri, 2, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 2, [], tri, 2)
    mk, _ = g.markers()
    omk, _, _ = o.markers()
    assert np.array_equal(mk, omk) and (mk == 1).all()
    _check(g, o, I.Physics(g=(0.2, 0.0, 0.0)), dev, 3)
