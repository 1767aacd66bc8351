"""Textbook closed forms for trilinear (Q1) hexahedra, used to pin the oracle.

Every integral over a cube element [0, h]^3 of products of Q1 basis functions and their
first derivatives factors into 1-D integrals of linear shape functions on [0, h]:

    mass      int phi_a phi_b      = h/6 [[2, 1], [1, 2]]
    stiffness int phi_a' phi_b'    = 1/h [[1, -1], [-1, 1]]
    mixed     int phi_a' phi_b     = [[-1/2, -1/2], [1/2, 1/2]]   (and its transpose)

so  int D^alpha phi_a D^beta phi_b = prod_k T[alpha_k][beta_k][a_k][b_k]  for multi-indices
alpha, beta in {0, 1}^3 (a second mixed derivative d_i d_j phi, i != j, is the multi-index
e_i + e_j).  Corner a has bits (a & 1, a >> 1 & 1, a >> 2 & 1) along x, y, z.  The 2x2x2
Gauss rule integrates all of these exactly, so the oracle must reproduce them to rounding.
"""
import numpy as np


def tables(h):
    m1 = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k1 = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    c1 = np.array([[-0.5, -0.5], [0.5, 0.5]])       # int phi_a' phi_b
    return {(0, 0): m1, (1, 0): c1, (0, 1): c1.T, (1, 1): k1}


def integral(h, alpha, beta):
    """8 x 8 matrix  int_cube D^alpha phi_a D^beta phi_b."""
    T = tables(h)
    M = np.ones((8, 8))
    for a in range(8):
        for b in range(8):
            v = 1.0
            for k in range(3):
                v *= T[(alpha[k], beta[k])][(a >> k) & 1, (b >> k) & 1]
            M[a, b] = v
    return M


def e(k):
    v = [0, 0, 0]
    v[k] = 1
    return tuple(v)


def ee(i, j):
    v = [0, 0, 0]
    v[i] += 1
    v[j] += 1
    return tuple(v)


Z = (0, 0, 0)


def mass(h):
    return integral(h, Z, Z)


def laplace(h):
    return sum(integral(h, e(k), e(k)) for k in range(3))


def int_phi(h):
    """int phi_a (vector of 8)."""
    return np.full(8, (h / 2.0) ** 3)


def int_dphi(h, j):
    """int d_j phi_a (vector of 8)."""
    return np.array([(1.0 if (a >> j) & 1 else -1.0) * (h / 2.0) ** 2 for a in range(8)])
