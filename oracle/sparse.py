"""Matrix-based linear-solver path of the method, for the oracle: the global Jacobian assembled in
4 x 4 blocks and BiCGStab.

TEST INFRASTRUCTURE ONLY: the tests use this module; the product never imports it.

* Assembly (Algorithms 2 and 4): K = sum_e M_e^T k_e M_e, where k_e is the 32 x 32 element
  Jacobian (8 corners x 4 unknowns, row a*4+i, column b*4+k) and M_e the corner-to-node operator
  with the hanging-node interpolation of Algorithm 3 (weights 1/2 on edges, 1/4 on faces).
  Rows that the residual replaces by U - g (strong Dirichlet rows on the box, Algorithm 1's nodes
  touched by In elements only) become identity rows.  Stored as a block-sparse matrix with 4 x 4
  blocks, block columns sorted within each block row.
* BiCGStab (appendix "Details of solver selection": the linear systems of the Newton steps are
  solved by BiCGStab), in the form of van der Vorst (1992) with right preconditioning, float64.
* Preconditioners: nodal block-Jacobi, and a two-level one that adds a coarse space of piecewise
  constants on aggregates of nodes (octants, or equal ranges of the Morton node order), with the
  Galerkin coarse matrix P^T A P.  The paper preconditions with additive Schwarz; its conclusion
  asks for preconditioners suited to the method.
"""
import numpy as np
import scipy.sparse as sp


def strong_mask(m):
    """Bit k of mask[i] set: row (i, k) of the residual is U - g (box faces but the outlet carry
    the velocity, the outlet x = hi the pressure; every unknown of a node touched by no active
    element).  A mask set with set_dirichlet replaces the box rows."""
    if getattr(m, "_bc", None) is not None:
        mask = np.array(m._bc[0], dtype=np.uint8)
    else:
        ijk = m.node_ijk.astype(np.int64)
        outlet = ijk[:, 0] == m.hiI[0]
        other = (ijk == 0).any(1) | (ijk[:, 1] == m.hiI[1]) | (ijk[:, 2] == m.hiI[2])
        mask = np.where(other, 7, 0).astype(np.uint8) | np.where(outlet, 8, 0).astype(np.uint8)
    mk, _, _ = m.markers()
    active = np.zeros(m.n_nodes, bool)
    for el in np.where(mk != 1)[0]:
        for c in range(8):
            idx = m.conn[el, c]
            if idx < m.n_nodes:
                active[idx] = True
            else:
                h = idx - m.n_nodes
                active[m.hang_parents[h, :m.hang_np[h]]] = True
    mask[~active] = 15
    return mask


def corner_operator(m, e):
    """(nodes, weights) of the 8 corners of element e: corner c is sum_p weights[c][p] * node
    nodes[c][p] (one node with weight 1, or the 2 / 4 parents of a hanging node)."""
    out = []
    for c in range(8):
        idx = int(m.conn[e, c])
        if idx < m.n_nodes:
            out.append(([idx], [1.0]))
        else:
            h = idx - m.n_nodes
            k = int(m.hang_np[h])
            out.append(([int(p) for p in m.hang_parents[h, :k]], [1.0 / k] * k))
    return out


def assemble_bsr(m, phys, u, u_prev, u_prev2=None, f=None, mask=None):
    """The assembled Jacobian dR/dU as a scipy bsr_matrix with 4 x 4 blocks (n_nodes x n_nodes
    blocks).  The block pattern is structural and depends on the octree alone: every pair of nodes
    reached from the corners of a common element through M_e, In elements included.  In elements
    contribute zeros (Algorithm 1).  The rows of `mask` (default strong_mask(m)) are identity
    rows; their other entries stay in the pattern as zeros."""
    n = m.n_nodes
    if mask is None:
        mask = strong_mask(m)
    mk, _, _ = m.markers()
    blocks = {}
    for e in range(m.n_elem):
        K = np.zeros((32, 32)) if mk[e] == 1 else m.element_matrix(phys, u, u_prev, e, u_prev2=u_prev2, f=f)[0]
        ops = corner_operator(m, e)
        for a in range(8):
            for b in range(8):
                kab = K[4 * a:4 * a + 4, 4 * b:4 * b + 4]
                for ni, wi in zip(*ops[a]):
                    for nj, wj in zip(*ops[b]):
                        key = (ni, nj)
                        if key not in blocks:
                            blocks[key] = np.zeros((4, 4))
                        blocks[key] += (wi * wj) * kab
    # strong rows: zero the row, then a 1 on the diagonal
    fixed = ((mask[:, None] >> np.arange(4)[None, :]) & 1).astype(bool)
    for (i, j), B in blocks.items():
        B[fixed[i], :] = 0.0
    for i in np.where(fixed.any(1))[0]:
        B = blocks.setdefault((int(i), int(i)), np.zeros((4, 4)))
        for k in np.where(fixed[i])[0]:
            B[k, k] = 1.0
    keys = sorted(blocks)
    rows = np.array([k[0] for k in keys], dtype=np.int64)
    cols = np.array([k[1] for k in keys], dtype=np.int64)
    data = np.stack([blocks[k] for k in keys]) if keys else np.zeros((0, 4, 4))
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return sp.bsr_matrix((data, cols, indptr), shape=(4 * n, 4 * n))


def bicgstab(matvec, b, x0=None, rtol=1e-8, atol=0.0, maxiter=1000, precond=None):
    """BiCGStab (van der Vorst 1992) for A x = b, A given by matvec, with right preconditioning:
    the directions p and s are mapped by M^-1 = precond before each product with A, so the
    recurrence runs on the true residual b - A x.  Stops when ||b - A x|| <= max(rtol ||b||,
    atol).  Returns (x, iterations, converged, residual norms)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    Minv = (lambda z: z) if precond is None else precond
    r = b - matvec(x)
    tol = max(rtol * np.linalg.norm(b), atol)
    hist = [np.linalg.norm(r)]
    if hist[-1] <= tol:
        return x, 0, True, hist
    r_hat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxiter + 1):
        rho = float(r_hat @ r)
        if rho == 0.0:
            return x, it - 1, False, hist          # breakdown: r orthogonal to the shadow residual
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        p_hat = Minv(p)
        v = matvec(p_hat)
        alpha = rho / float(r_hat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol:
            x = x + alpha * p_hat
            hist.append(np.linalg.norm(s))
            return x, it, True, hist
        s_hat = Minv(s)
        t = matvec(s_hat)
        tt = float(t @ t)
        omega = float(t @ s) / tt if tt > 0.0 else 0.0
        x = x + alpha * p_hat + omega * s_hat
        r = s - omega * t
        hist.append(np.linalg.norm(r))
        if hist[-1] <= tol:
            return x, it, True, hist
        if omega == 0.0:
            return x, it, False, hist              # stagnation
        rho_old = rho
    return x, maxiter, False, hist


def block_jacobi(A):
    """Inverse of the 4 x 4 diagonal blocks of a block-sparse matrix, as a preconditioner.  A block
    whose smallest singular value is at most 1e-14 of its largest entry (all zero, for a node that
    only Intercepted elements without quadrature points touch) is replaced by the identity."""
    A = A.tobsr(blocksize=(4, 4))
    n = A.shape[0] // 4
    D = np.zeros((n, 4, 4))
    for i in range(n):
        for q in range(A.indptr[i], A.indptr[i + 1]):
            if A.indices[q] == i:
                D[i] = A.data[q]
    scale = np.abs(D).max(axis=(1, 2))
    smin = np.linalg.svd(D, compute_uv=False)[:, -1]
    singular = ~(smin > 1e-14 * scale)
    D[singular] = np.eye(4)
    Dinv = np.linalg.inv(D)
    return lambda z: np.einsum("nij,nj->ni", Dinv, z.reshape(n, 4)).reshape(-1)


# ------------------------------------------------------------------------------------------
# Two-level preconditioner: piecewise constants on octants as the coarse space
# ------------------------------------------------------------------------------------------
def octant_aggregates(m, level):
    """Aggregate of every node: the level-`level` octant that contains it (a node on an octant's
    upper face or on the box's upper boundary goes to the octant below it in that direction).
    Returns (agg [n_nodes] in 0 .. n_agg - 1, numbered in Morton order of the octants, n_agg)."""
    shift = 20 - level
    ijk = m.node_ijk.astype(np.int64)
    top = (np.asarray(m.hiI, dtype=np.int64) - 1) >> shift
    o = np.minimum(ijk >> shift, top[None, :])

    def spread(v):
        out = np.zeros_like(v)
        for b in range(21):
            out |= ((v >> b) & 1) << (3 * b)
        return out

    key = spread(o[:, 0]) | (spread(o[:, 1]) << 1) | (spread(o[:, 2]) << 2)
    uniq, agg = np.unique(key, return_inverse=True)
    return agg.astype(np.int64), int(uniq.size)


def morton_aggregates(n_nodes, n_agg):
    """Aggregates of equal size: nodes are numbered in Morton order of their coordinates, so
    contiguous ranges of that order are spatially compact.  Node i goes to aggregate
    floor(i n_agg / n_nodes).  Returns (agg, n_agg)."""
    n_agg = max(1, min(int(n_agg), n_nodes))
    return (np.arange(n_nodes, dtype=np.int64) * n_agg // n_nodes), n_agg


def coarse_space(A, agg, n_agg):
    """Prolongation P [4 n x 4 n_agg], one constant per aggregate and unknown, zero on the rows
    that A holds fixed (identity rows) or that are empty (decoupled nodes), and the Galerkin
    coarse matrix A_c = P^T A P (scipy sparse)."""
    import scipy.sparse as sp
    B = A.tocsr()
    n4 = B.shape[0]
    diag = B.diagonal()
    nnz_row = np.diff(B.indptr)
    absrow = np.asarray(np.abs(B).sum(axis=1)).ravel()
    fixed = (nnz_row > 0) & (diag == 1.0) & (absrow == 1.0)
    empty = absrow == 0.0
    free = ~(fixed | empty)
    rows = np.arange(n4)[free]
    cols = 4 * agg[rows // 4] + rows % 4
    P = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(n4, 4 * n_agg))
    keep = np.asarray(P.sum(axis=0)).ravel() > 0                 # drop coarse unknowns with no free row
    P = P[:, np.where(keep)[0]]
    Ac = (P.T @ B @ P).tocsc()
    return P.tocsr(), Ac


def two_level(A, P, Ac, mode="multiplicative"):
    """Preconditioner from block-Jacobi and the coarse correction Q r = P A_c^-1 P^T r:
    additive, z = D^-1 r + Q r; multiplicative (coarse first), x = Q r, z = x + D^-1 (r - A x)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(Ac)
    Dinv = block_jacobi(A)
    B = A.tocsr()

    def Q(r):
        return P @ lu.solve(P.T @ r)

    if mode == "additive":
        return lambda r: Dinv(r) + Q(r)

    def mult(r):
        x = Q(r)
        return x + Dinv(r - B @ x)

    return mult


# ------------------------------------------------------------------------------------------
# Multilevel preconditioner: the two-level construction applied recursively
# ------------------------------------------------------------------------------------------
def _block_diag_inverse(A, n):
    """Inverses of the 4 x 4 diagonal blocks of A (n blocks); a singular block becomes the identity
    (the reading of block_jacobi)."""
    coo = A.tocoo()
    sel = (coo.row // 4) == (coo.col // 4)
    D = np.zeros((n, 4, 4))
    np.add.at(D, (coo.row[sel] // 4, coo.row[sel] % 4, coo.col[sel] % 4), coo.data[sel])
    scale = np.abs(D).max(axis=(1, 2))
    smin = np.linalg.svd(D, compute_uv=False)[:, -1]
    D[~(smin > 1e-14 * scale)] = np.eye(4)
    return np.linalg.inv(D)


def hierarchy(A, agg_size=6, coarse_max=200):
    """Levels of the multilevel preconditioner.  Level 0 is A (4 x 4 blocks, one per node, nodes
    in Morton order).  Each coarser level aggregates agg_size consecutive unknown-blocks of the
    level above (Morton ranges, so aggregates stay compact), with a piecewise-constant
    prolongation per unknown that leaves out the fixed and empty rows of level 0 and the dead
    rows of coarser levels; A_{l+1} = P_l^T A_l P_l, and a coarse unknown that no free row
    reaches gets an identity row.  The last level (at most coarse_max blocks) is factorised."""
    import scipy.sparse.linalg as spla
    A = A.tocsr()
    n = A.shape[0] // 4
    diag = A.diagonal()
    absrow = np.asarray(np.abs(A).sum(axis=1)).ravel()
    free = ~(((diag == 1.0) & (absrow == 1.0)) | (absrow == 0.0))
    levels = []
    while True:
        Dinv = _block_diag_inverse(A, n)
        if n <= coarse_max:
            Ad = A.toarray()
            dead = np.abs(Ad).sum(axis=1) == 0
            Ad[dead, dead] = 1.0
            levels.append({"A": A, "Dinv": Dinv, "n": n, "lu": spla.splu(sp.csc_matrix(Ad))})
            return levels
        na = (n + agg_size - 1) // agg_size
        agg = np.minimum(np.arange(n) // agg_size, na - 1)
        rows = np.where(free)[0]
        P = sp.csr_matrix((np.ones(rows.size), (rows, 4 * agg[rows // 4] + rows % 4)), shape=(4 * n, 4 * na))
        Ac = (P.T @ A @ P).tocsr()
        dead = np.asarray(np.abs(Ac).sum(axis=1)).ravel() == 0
        levels.append({"A": A, "Dinv": Dinv, "n": n, "P": P})
        A, n, free = (Ac + sp.diags(dead.astype(float))).tocsr(), na, ~dead


def vcycle(levels, r, nu=1, omega=0.5, level=0):
    """One V-cycle applied to r: nu damped block-Jacobi sweeps (weight omega), the coarse
    correction of the level below, nu more sweeps; the last level is solved exactly.  Damping
    matters: the Jacobian is an indefinite saddle-point matrix, on which undamped block-Jacobi
    is not a convergent smoother."""
    L = levels[level]
    if "lu" in L:
        return L["lu"].solve(r)
    A, Dinv, n = L["A"], L["Dinv"], L["n"]

    def smooth(z):
        return omega * np.einsum("nij,nj->ni", Dinv, z.reshape(n, 4)).reshape(-1)

    x = np.zeros_like(r)
    for _ in range(nu):
        x = x + smooth(r - A @ x)
    x = x + L["P"] @ vcycle(levels, L["P"].T @ (r - A @ x), nu, omega, level + 1)
    for _ in range(nu):
        x = x + smooth(r - A @ x)
    return x


def multilevel(A, agg_size=6, coarse_max=200, nu=1, omega=0.5):
    """Preconditioner r -> vcycle(r) over hierarchy(A)."""
    levels = hierarchy(A, agg_size, coarse_max)
    return lambda r: vcycle(levels, r, nu, omega)
