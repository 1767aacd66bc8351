"""GPU: the matrix-based path and the multilevel preconditioner through the C ABI.

* imga_bsr_assemble equals the oracle's assembly sum_e M_e^T k_e M_e with identity rows
  (oracle/sparse.py, Algorithms 2 and 4) entry by entry, and imga_bsr_spmv with it equals the
  matrix-free J v.
* One V-cycle of imga_multilevel_apply equals the oracle's vcycle over hierarchy() built from the
  oracle's assembled matrix with the same parameters (float64; the float32 hierarchy within its
  rounding).
* Newton with the multilevel preconditioner converges on the small sphere with fewer Krylov
  iterations than block-Jacobi; Newton-BiCGStab on the assembled matrix reaches the same solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sparse as S
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
def small(dev):
    """the smoke mesh (2,696 elements, hanging nodes, Intercepted elements, surface points)"""
    c = (0.5, 0.5, 0.5)
    regs = [I.Region(I.REGION_SPHERE_BAND, 5, (*c, 0.15, 0.04))]
    tri = I.icosphere(2, 0.15, c, 1e-4, 0)
    g = api.Mesh((0, 0, 0), (1, 1, 1), 3, regs, tri, 2, device=0)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 3, regs, tri, 2)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01)
    u, up, v = I.state(g.n_nodes, 3)
    A = S.assemble_bsr(o, ph, u, up)
    return g, o, ph, u, up, v, A


def _dev_matrix(g, vals):
    import scipy.sparse as sp
    ptr, idx = g.bsr_pattern()
    return sp.bsr_matrix((vals.cpu().numpy(), idx, ptr), shape=(4 * g.n_nodes, 4 * g.n_nodes))


def test_assembly_matches_oracle_entry_by_entry(dev, small):
    g, o, ph, u, up, v, A = small
    vals = g.bsr_assemble(ph, T(u, dev), T(up, dev))
    Ad = _dev_matrix(g, vals).tocsr()
    D = (Ad - A.tocsr()).tocoo()
    scale = np.abs(A.data).max()
    err = np.abs(D.data).max() if D.nnz else 0.0
    print(f"assembly: max entry error / max entry {err / scale:.2e}, blocks {vals.shape[0]}")
    assert err <= 1e-12 * scale
    # mixed: float32 element arithmetic, float64 accumulation
    vals32 = g.bsr_assemble(ph, T(u, dev), T(up, dev), precision=api.PRECISION_MIXED)
    D32 = (_dev_matrix(g, vals32).tocsr() - A.tocsr()).tocoo()
    e32 = np.abs(D32.data).max() / scale
    print(f"assembly mixed: {e32:.2e}")
    assert e32 <= 1e-5


def test_spmv_equals_matrix_free_jvp(dev, small):
    g, o, ph, u, up, v, A = small
    ut, upt, vt = T(u, dev), T(up, dev), T(v, dev)
    vals = g.bsr_assemble(ph, ut, upt)
    y = g.bsr_spmv(vals, vt).cpu().numpy()
    J = g.jvp(ph, ut, upt, vt).cpu().numpy()
    print(f"spmv vs jvp: {rel(y, J):.2e}")
    assert rel(y, J) <= 1e-12
    assert rel(y.ravel(), A @ v.ravel()) <= 1e-12


@pytest.mark.parametrize("sweeps,omega", [(1, 0.5), (2, 0.5)])
def test_vcycle_matches_oracle(dev, small, sweeps, omega):
    g, o, ph, u, up, v, A = small
    levels = S.hierarchy(A, agg_size=6, coarse_max=16)
    r = I.normal(7, 4 * g.n_nodes)
    z_or = S.vcycle(levels, r, nu=sweeps, omega=omega)
    ut, upt = T(u, dev), T(up, dev)
    g.multilevel_setup(ph, ut, upt, agg=6, coarse_max=16, sweeps=sweeps, omega=omega)
    rows, singular = g.multilevel_info()
    assert not singular
    assert list(rows) == [L["n"] for L in levels]
    z = g.multilevel_apply(T(r.reshape(-1, 4), dev)).cpu().numpy().ravel()
    print(f"V-cycle ({sweeps} sweeps), levels {list(rows)}: float64 {rel(z, z_or):.2e}")
    assert rel(z, z_or) <= 1e-9
    g.multilevel_setup(ph, ut, upt, precision=api.PRECISION_MIXED, agg=6, coarse_max=16, sweeps=sweeps, omega=omega)
    z32 = g.multilevel_apply(T(r.reshape(-1, 4), dev)).cpu().numpy().ravel()
    print(f"V-cycle ({sweeps} sweeps): float32 hierarchy {rel(z32, z_or):.2e}")
    assert rel(z32, z_or) <= 1e-3


@pytest.fixture(scope="module")
def sphere(dev):
    w = I.small_sphere(16)
    g = api.Mesh.from_workload(w, device=0)
    return w, g


@pytest.mark.parametrize("precision", [api.PRECISION_FP64, api.PRECISION_MIXED])
def test_newton_multilevel_converges_with_fewer_iterations(dev, sphere, precision):
    w, g = sphere
    u0, up, _ = I.state(g.n_nodes, 16)
    upt = T(up, dev)
    out = {}
    for pc in (1, 4):
        u = T(u0, dev)
        st = g.newton_step(w.physics, u, upt, precision=precision, precond=pc, max_krylov=2000)
        out[pc] = (st, u.cpu().numpy())
        print(f"precision {precision} precond {pc}: Newton {st['newton_its']} Krylov {st['krylov_its']} "
              f"{st['time_ms']:.0f} ms, |R| {st['res_norm'][-1] / st['res_norm'][0]:.2e}")
        assert st["converged"]
    assert out[4][0]["krylov_its"] < out[1][0]["krylov_its"]
    assert rel(out[4][1], out[1][1]) <= 1e-6


def test_newton_bicgstab_on_assembled_matrix(dev, sphere):
    """Newton with BiCGStab on the assembled matrix (multilevel or block-Jacobi) reaches the same
    tolerance as Newton-GMRES, judged by the oracle's float64 residual.  (The solutions themselves
    are not compared: rows that no equation constrains -- dofs of Intercepted elements whose points
    are all In -- keep whatever the linear solvers leave there, and differ between them.)"""
    w, g = sphere
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax)
    u0, up, _ = I.state(g.n_nodes, 16)
    R0 = np.linalg.norm(o.residual(w.physics, u0, up))
    upt = T(up, dev)
    res = {}
    for ls, pc in ((0, 4), (1, 4), (1, 1)):
        u = T(u0, dev)
        st = g.newton_step(w.physics, u, upt, precond=pc, linear_solver=ls, max_krylov=3000)
        res[(ls, pc)] = u.cpu().numpy()
        print(f"linear solver {ls} precond {pc}: Newton {st['newton_its']} Krylov {st['krylov_its']} {st['time_ms']:.0f} ms")
        assert st["converged"]
        assert np.linalg.norm(o.residual(w.physics, res[(ls, pc)], up)) <= 1.5e-8 * R0, (ls, pc)
    print("solutions differ by", rel(res[(1, 4)], res[(0, 4)]), rel(res[(1, 1)], res[(0, 4)]))
