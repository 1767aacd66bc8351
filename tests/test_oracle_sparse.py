"""Pins of the oracle's matrix-based solver path (oracle/sparse.py): the assembled block-sparse
Jacobian of Algorithms 2 and 4, and BiCGStab.

What is fixed independently of the code under test:
* BiCGStab against dense LU (numpy.linalg.solve) on random nonsymmetric systems; with the exact
  inverse as preconditioner it must finish in one iteration;
* the assembled matrix times v against the matrix-free J v of the dual-number element code, and
  against a second assembly written with sparse Kronecker products (tests/oracle_assembly.py);
* the block pattern against the node pairs enumerated directly from the element corners;
* BiCGStab with block-Jacobi on the assembled system against scipy's sparse direct solver.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import sparse as S
from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import inputs as I
from tests.oracle_assembly import assemble_jacobian


def _dense_system(n, seed):
    A = I.normal(seed, n * n).reshape(n, n) / np.sqrt(n)
    A += np.diag(2.0 + I.uniform(seed + 1, n))                 # nonsymmetric, well conditioned
    b = I.normal(seed + 2, n)
    return A, b


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bicgstab_matches_dense_solve(seed):
    A, b = _dense_system(80, 10 * seed)
    x_ref = np.linalg.solve(A, b)
    for pre in (None, lambda z: z / np.diag(A)):
        x, its, ok, hist = S.bicgstab(lambda z: A @ z, b, rtol=1e-12, maxiter=500, precond=pre)
        assert ok and its < 80
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
        assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001


def test_bicgstab_exact_preconditioner_one_iteration():
    A, b = _dense_system(40, 7)
    Ainv = np.linalg.inv(A)
    x, its, ok, _ = S.bicgstab(lambda z: A @ z, b, rtol=1e-10, precond=lambda z: Ainv @ z)
    assert ok and its == 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


@pytest.fixture(scope="module")
def body_mesh():
    c = (0.5, 0.5, 0.5)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, [I.Region(I.REGION_SPHERE_BAND, 4, (*c, 0.2, 0.05))],
                   I.icosphere(2, 0.2, c, 1e-4, 3), 3)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=I.SCHEME_BDF2)
    u, up, v = I.state(m.n_nodes, 4)
    up2 = up + I.normal(13, m.n_nodes * 4, 0.01).reshape(-1, 4)
    A = S.assemble_bsr(m, ph, u, up, up2)
    mk, _, _ = m.markers()
    assert m.n_hang > 0 and (mk == 2).sum() > 20 and (mk == 1).sum() > 0
    return m, ph, u, up, up2, v, A


def test_assembled_matvec_equals_matrix_free_jvp(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    Jv = m.jvp(ph, u, up, v, u_prev2=up2)
    Av = (A @ v.reshape(-1)).reshape(-1, 4)
    assert np.linalg.norm(Av - Jv) <= 1e-12 * np.linalg.norm(Jv)


def test_assembly_equals_kronecker_assembly(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    C = _kron_assembly(m, ph, u, up, up2, S.strong_mask(m))
    D = (A.tocsr() - C).tocoo()
    assert np.abs(D.data).max(initial=0.0) <= 1e-12 * np.abs(C.data).max()


def _kron_assembly(m, ph, u, up, up2, mask):
    # tests/oracle_assembly.assemble_jacobian takes (U, Up, F) for one previous level; BDF2 needs two,
    # so the same Kronecker construction is repeated here with u_prev2 passed through
    import scipy.sparse as sp
    n = m.n_nodes * 4
    rows, cols, vals = [], [], []
    mk, _, _ = m.markers()
    for el in range(m.n_elem):
        if mk[el] == 1:
            continue
        Ke, _ = m.element_matrix(ph, u, up, el, u_prev2=up2)
        P = sp.csr_matrix(np.kron(m.gather_matrix(el), np.eye(4)))
        Jl = (P.T @ sp.csr_matrix(Ke) @ P).tocoo()
        rows.append(Jl.row); cols.append(Jl.col); vals.append(Jl.data)
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    fixed = np.zeros(n, bool)
    for k in range(4):
        fixed[k::4] = (mask >> k) & 1
    return (sp.diags((~fixed).astype(float)) @ J + sp.diags(fixed.astype(float))).tocsr()


def test_kron_helper_agrees_for_one_step_schemes():
    # the shared helper (used by the GPU solver tests) and the block assembly agree for BE
    c = (0.5, 0.5, 0.5)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, [I.Region(I.REGION_SPHERE_BAND, 3, (*c, 0.2, 0.05))],
                   I.icosphere(1, 0.2, c, 1e-4, 5), 2)
    ph = I.Physics(rho=1.0, mu=0.05, dt=0.02, scheme=I.SCHEME_BE)
    u, up, _ = I.state(m.n_nodes, 6)
    mask = S.strong_mask(m)
    A = S.assemble_bsr(m, ph, u, up, mask=mask).tocsr()
    C = assemble_jacobian(m, ph, u, up, None, mask).tocsr()
    assert np.abs((A - C).tocoo().data).max(initial=0.0) <= 1e-12 * np.abs(C.data).max()


def test_block_pattern_is_element_adjacency(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    want = set()
    for el in range(m.n_elem):
        nodes = set()
        for c in range(8):
            idx = int(m.conn[el, c])
            nodes |= {idx} if idx < m.n_nodes else set(int(p) for p in m.hang_parents[idx - m.n_nodes, :m.hang_np[idx - m.n_nodes]])
        want |= {(i, j) for i in nodes for j in nodes}
    assert all((i, i) in want for i in range(m.n_nodes))      # every node is in some element
    got = set()
    for i in range(m.n_nodes):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0)                       # sorted, no duplicates
        got |= {(i, int(j)) for j in cols}
    assert got == want


def test_strong_rows_are_identity_rows(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    mask = S.strong_mask(m)
    B = A.tocsr()
    for i in np.where(mask != 0)[0][:200]:
        for k in range(4):
            if (mask[i] >> k) & 1:
                row = B.getrow(4 * i + k).toarray().ravel()
                e = np.zeros_like(row)
                e[4 * i + k] = 1.0
                assert np.array_equal(row, e)
    assert (mask == 15).sum() > 0                              # In-only nodes present


def test_decoupled_nodes_have_empty_rows_and_columns(body_mesh):
    """A node touched only by In elements and by Intercepted elements that kept no quadrature
    point has R rows that do not depend on U, and no other row depends on it: J has zero rows and
    columns there.  Krylov iterations started from 0 on a right-hand side -R never leave the
    complement, so the Newton systems stay consistent."""
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    zr = np.where(np.abs(B).sum(1).A.ravel() == 0)[0]
    zc = np.where(np.abs(B).sum(0).A.ravel() == 0)[0]
    assert zr.size > 0 and np.array_equal(zr, zc)
    R = m.residual(ph, u, up, up2).reshape(-1)
    assert np.all(R[zr] == 0.0)


def test_bicgstab_block_jacobi_solves_assembled_system(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    live = np.abs(B).sum(1).A.ravel() != 0
    b = I.normal(31, B.shape[0])
    b[~live] = 0.0                                             # consistent right-hand side
    x_ref = np.zeros_like(b)
    x_ref[live] = spla.spsolve(B[live][:, live].tocsc(), b[live])
    x, its, ok, hist = S.bicgstab(lambda z: B @ z, b, rtol=1e-10, maxiter=4000, precond=S.block_jacobi(A))
    assert ok, (its, hist[-1] / hist[0])
    assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    assert np.all(x[~live] == 0.0)
    # the preconditioner helps: fewer iterations than without it
    _, its0, ok0, _ = S.bicgstab(lambda z: B @ z, b, rtol=1e-10, maxiter=4000)
    assert (not ok0) or its0 > its


# ---------------------------------------------------------------------------------------
# two-level preconditioner (piecewise constants on octants)
# ---------------------------------------------------------------------------------------
def test_octant_aggregates_contain_their_nodes(body_mesh):
    m = body_mesh[0]
    for lev in (1, 2, 3):
        agg, na = S.octant_aggregates(m, lev)
        assert agg.min() == 0 and agg.max() == na - 1 and np.unique(agg).size == na
        s = 1 << (20 - lev)
        ijk = m.node_ijk.astype(np.int64)
        for a in range(na):
            pts = ijk[agg == a]
            lo = (pts.min(0) // s) * s
            # every node of the aggregate lies in one closed octant of edge s
            assert np.all(pts - lo[None, :] <= s)


def test_coarse_correction_is_galerkin_orthogonal(body_mesh):
    import scipy.sparse.linalg as spla
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    agg, na = S.octant_aggregates(m, 3)
    P, Ac = S.coarse_space(A, agg, na)
    r = I.normal(3, B.shape[0])
    r[np.abs(B).sum(1).A.ravel() == 0] = 0.0
    x = P @ spla.splu(Ac).solve(P.T @ r)
    # the residual after the coarse correction has no component in the coarse space
    assert np.abs(P.T @ (r - B @ x)).max() <= 1e-12 * np.abs(r).max()


def test_two_level_beats_block_jacobi_and_is_exact_at_the_finest_level(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    b = -m.residual(ph, u, up, up2).reshape(-1)
    _, its_bj, ok, _ = S.bicgstab(lambda z: B @ z, b, rtol=1e-8, maxiter=3000, precond=S.block_jacobi(A))
    assert ok
    its = {}
    for lev in (2, 3, 20):                          # level 20: every node its own aggregate
        agg, na = S.octant_aggregates(m, lev)
        P, Ac = S.coarse_space(A, agg, na)
        x, its[lev], ok, _ = S.bicgstab(lambda z: B @ z, b, rtol=1e-8, maxiter=3000,
                                        precond=S.two_level(A, P, Ac, "multiplicative"))
        assert ok and np.linalg.norm(b - B @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
    assert its[20] == 1                             # the coarse solve is exact on the free unknowns
    assert its[3] <= its[2] < its_bj, (its, its_bj)


def test_morton_range_aggregates(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    agg, na = S.morton_aggregates(m.n_nodes, 512)
    cnt = np.bincount(agg)
    assert na == 512 and cnt.size == 512 and cnt.max() - cnt.min() <= 1
    assert np.all(np.diff(agg) >= 0)                             # contiguous ranges
    B = A.tocsr()
    b = -m.residual(ph, u, up, up2).reshape(-1)
    _, its_bj, _, _ = S.bicgstab(lambda z: B @ z, b, rtol=1e-8, maxiter=3000, precond=S.block_jacobi(A))
    P, Ac = S.coarse_space(A, agg, na)
    x, its, ok, _ = S.bicgstab(lambda z: B @ z, b, rtol=1e-8, maxiter=3000, precond=S.two_level(A, P, Ac))
    assert ok and its < its_bj


# ---------------------------------------------------------------------------------------
# multilevel preconditioner
# ---------------------------------------------------------------------------------------
def _consistent_rhs(B, seed):
    b = I.normal(seed, B.shape[0])
    b[np.abs(B).sum(1).A.ravel() == 0] = 0.0
    return b


def test_single_level_hierarchy_is_an_exact_solve(body_mesh):
    from oracle.krylov import gmres
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    lv = S.hierarchy(A, coarse_max=10 ** 6)
    assert len(lv) == 1
    b = _consistent_rhs(B, 41)
    x, k, _ = gmres(lambda z: B @ z, b, m=20, rtol=1e-10, maxiter=20, precond=lambda r: S.vcycle(lv, r))
    assert k == 1 and np.linalg.norm(b - B @ x) <= 1e-9 * np.linalg.norm(b)


def test_vcycle_is_linear_and_its_coarse_correction_galerkin_orthogonal(body_mesh):
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    lv = S.hierarchy(A, agg_size=6, coarse_max=300)
    assert len(lv) == 2                                          # 1,147 -> 192 blocks
    r1, r2 = _consistent_rhs(B, 42), _consistent_rhs(B, 43)
    V = lambda r: S.vcycle(lv, r, nu=1, omega=0.5)
    lhs, rhs = V(2.0 * r1 - 0.5 * r2), 2.0 * V(r1) - 0.5 * V(r2)
    assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs)
    # with no smoothing the V-cycle is the coarse correction P A_c^-1 P^T r
    P = lv[0]["P"]
    x = S.vcycle(lv, r1, nu=0)
    assert np.abs(P.T @ (r1 - B @ x)).max() <= 1e-10 * np.abs(r1).max()


def test_multilevel_needs_fewer_iterations_than_block_jacobi(body_mesh):
    from oracle.krylov import gmres
    m, ph, u, up, up2, v, A = body_mesh
    B = A.tocsr()
    b = -m.residual(ph, u, up, up2).reshape(-1)
    _, k_bj, _ = gmres(lambda z: B @ z, b, m=50, rtol=1e-8, maxiter=3000, precond=S.block_jacobi(A))
    x, k_ml, _ = gmres(lambda z: B @ z, b, m=50, rtol=1e-8, maxiter=3000,
                       precond=S.multilevel(A, agg_size=6, coarse_max=50))
    assert np.linalg.norm(b - B @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
    assert k_ml < k_bj, (k_ml, k_bj)
