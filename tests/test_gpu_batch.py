"""Batched meshes and CUDA-graph execution against the plain per-problem path (and the oracle).

* A batched mesh of independent sphere problems with different viscosities gives, for residual and
  J v, the concatenation of the problems' own results (<= 1e-12 relative, FP64; atomics reorder sums);
  one problem is also checked against the oracle (<= 1e-10).
* Graph replay equals the direct call, also after the input vectors change in place.
"""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_batched_equals_separate(dev):
    probs = [wl for wl, t, Re in I.batched_spheres(40) if t < 15000][:5]
    assert len(probs) == 5
    B = api.Mesh.batch(probs, device=0)
    assert B.n_problems == 5
    sep = [api.Mesh.from_workload(w, device=0) for w in probs]
    assert B.n_elem == sum(m.n_elem for m in sep) and B.n_nodes == sum(m.n_nodes for m in sep)
    us, ups, vs = [], [], []
    for k, m in enumerate(sep):
        u, up, v = I.state(m.n_nodes, 50 + k)
        us.append(u); ups.append(up); vs.append(v)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ph = probs[0].physics          # mu is taken per problem from the batch
    Rb = B.residual(ph, T(np.concatenate(us)), T(np.concatenate(ups))).cpu().numpy()
    Jb = B.jvp(ph, T(np.concatenate(us)), T(np.concatenate(ups)), T(np.concatenate(vs))).cpu().numpy()
    for k, m in enumerate(sep):
        a, b = B.node_off[k], B.node_off[k + 1]
        R = m.residual(probs[k].physics, T(us[k]), T(ups[k])).cpu().numpy()
        J = m.jvp(probs[k].physics, T(us[k]), T(ups[k]), T(vs[k])).cpu().numpy()
        assert rel(Rb[a:b], R) <= 1e-12 and rel(Jb[a:b], J) <= 1e-12, k
    w = probs[1]
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax)
    Ro, Jo = o.residual_jvp(w.physics, us[1], ups[1], v=vs[1])
    a, b = B.node_off[1], B.node_off[2]
    assert rel(Rb[a:b], Ro) <= 1e-10 and rel(Jb[a:b], Jo) <= 1e-10


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_graph_replay_equals_direct(dev, prec):
    w = I.small_sphere()
    m = api.Mesh.from_workload(w, device=0)
    g = api.Mesh.from_workload(w, device=0)
    g.use_graphs(True)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    u, up, v = I.state(m.n_nodes, 3)
    ud, upd, vd = T(u), T(up), T(v)
    out = torch.empty_like(ud)
    for k in range(3):
        vd.copy_(T(I.normal(200 + k, v.size).reshape(v.shape)))       # new content, same pointers
        ref = m.jvp(w.physics, ud, upd, vd, precision=prec).cpu().numpy()
        got = g.jvp(w.physics, ud, upd, vd, precision=prec, out=out).cpu().numpy()
        assert rel(got, ref) <= (1e-12 if prec == 0 else 1e-6), k
    R = g.residual(w.physics, ud, upd, precision=prec).cpu().numpy()
    assert rel(R, m.residual(w.physics, ud, upd, precision=prec).cpu().numpy()) <= (1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_autotuned_cut_bucket_equals_default(dev, prec):
    """The autotuner times every tile shape of the Intercepted-element kernel and keeps one; the
    result does not depend on the shape (sums reorder only)."""
    probs = [wl for wl, t, Re in I.batched_spheres(12) if t < 40000][:3]
    B = api.Mesh.batch(probs, device=0)
    u, up, v = I.state(B.n_nodes, 21)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ph = probs[0].physics
    ref = B.jvp(ph, T(u), T(up), T(v), precision=prec).cpu().numpy()
    B.autotune(True)
    got = B.jvp(ph, T(u), T(up), T(v), precision=prec).cpu().numpy()
    wpb, lpt, ms = B.tuning()[(prec, "jvp")]
    assert wpb in ((2, 4, 8) if prec == api.PRECISION_MIXED else (2, 4)) and lpt in (0, 1)
    assert all(t > 0 for t in ms[: (6 if prec == api.PRECISION_MIXED else 4)])
    assert rel(got, ref) <= (1e-12 if prec == api.PRECISION_FP64 else 1e-6)
    again = B.jvp(ph, T(u), T(up), T(v), precision=prec).cpu().numpy()
    assert rel(again, ref) <= (1e-12 if prec == api.PRECISION_FP64 else 1e-6)
    B.close()
