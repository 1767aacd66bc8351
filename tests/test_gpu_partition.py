"""GPU: residual and J v computed as k weighted parts with explicit halo exchange (imga_partition_*)
against the same calls on the whole mesh, and the Eq. (Wpart) balance of the parts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
    return w, api.Mesh.from_workload(w, device=0)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_partitioned_calls_equal_whole_mesh(dev, sphere, k):
    w, g = sphere
    P = api.Partition(g, k, ts_over_tv=0.5)
    # Eq. (Wpart) weights: every part within one heaviest element of the mean
    assert P.weight.sum() > 0
    assert np.abs(P.weight - P.weight.mean()).max() <= 0.05 * P.weight.mean() + 64.0
    u, up, v = I.state(g.n_nodes, 6)
    up2 = up.copy()
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=I.SCHEME_BDF2)
    ut, upt, up2t, vt = T(u, dev), T(up, dev), T(up2, dev), T(v, dev)
    for prec, tol in ((api.PRECISION_FP64, 1e-13), (api.PRECISION_MIXED, 1e-6)):
        R = g.residual(ph, ut, upt, up2t, precision=prec).cpu().numpy()
        J = g.jvp(ph, ut, upt, vt, up2t, precision=prec).cpu().numpy()
        Rp = P.residual(ph, ut, upt, up2t, precision=prec).cpu().numpy()
        Jp = P.jvp(ph, ut, upt, vt, up2t, precision=prec).cpu().numpy()
        print(f"k {k} precision {prec}: ghosts {list(P.n_ghost)}; R {rel(Rp, R):.2e} J v {rel(Jp, J):.2e}")
        assert rel(Rp, R) <= tol and rel(Jp, J) <= tol
    P.close()
