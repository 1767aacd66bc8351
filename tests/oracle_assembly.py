"""Global Jacobian assembled from the oracle's element matrices (test helper, CPU)."""
import numpy as np


def assemble_jacobian(m, ph, U, Up, F, mask):
    """Global Jacobian  sum_e M_e^T k_e M_e  (Algorithm 2) with Dirichlet rows replaced by I."""
    import scipy.sparse as sp
    n = m.n_nodes * 4
    Ks = np.stack([m.element_matrix(ph, U, Up, el, f=F)[0] for el in range(m.n_elem)])
    if m.n_hang == 0:
        dof = (m.conn[:, :, None] * 4 + np.arange(4)[None, None, :]).reshape(m.n_elem, 32)
        rows = np.repeat(dof[:, :, None], 32, axis=2).ravel()
        cols = np.repeat(dof[:, None, :], 32, axis=1).ravel()
        J = sp.coo_matrix((Ks.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    else:
        rows, cols, vals = [], [], []
        for el in range(m.n_elem):
            Me = m.gather_matrix(el)
            P = np.kron(Me, np.eye(4))             # [32, n]
            Jl = sp.csr_matrix(P).T @ sp.csr_matrix(Ks[el]) @ sp.csr_matrix(P)
            Jl = Jl.tocoo()
            rows.append(Jl.row); cols.append(Jl.col); vals.append(Jl.data)
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    fixed = np.zeros(n, bool)
    for k in range(4):
        fixed[k::4] = (mask >> k) & 1
    D = sp.diags((~fixed).astype(float))
    J = D @ J + sp.diags(fixed.astype(float))
    return J
