"""Pins of the oracle by symmetry: the residual and J v commute with the rigid motions that map
the box onto itself.

The weak form of Eq. (vms) with the Nitsche terms of Eq. (weakbc) is built from vectors and
tensors only, and the octree (Sec. "Octree based Mesh Generation"), the element markers
(Algorithm 5), the sub-cell quadrature (Sec. "Adaptive Quadrature") and the surface rule are
defined geometrically.  So if the body, the refinement regions, the body force and g_body and
the state are moved by a rigid motion T of the box, every node's row must move with it: a
velocity row by T, the continuity row unchanged.  A slip that touches one axis or one
velocity component only -- a wrong derivative direction, a swapped normal component, a
one-sided sign in the Nitsche or sub-cell terms -- breaks this, which the closed forms at
u = 0 and constant u do not all see.

The box is [-0.5, 0.5]^3, so its integer grid is symmetric and x -> -x and the cyclic axis
permutation map every coordinate exactly (no rounding of the inputs).  Rows of box-face nodes,
which hold strong Dirichlet values with an outlet at x = hi, are left out.
"""
import numpy as np
import pytest

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import inputs as I

LO, HI = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
CENTRE = np.array([0.07, -0.04, 0.03])


class Motion:
    """x' = sign * x[perm] (a rotation if det = +1, else a reflection)."""

    def __init__(self, perm, sign):
        self.perm = np.array(perm)
        self.sign = np.array(sign, dtype=np.float64)
        P = np.zeros((3, 3))
        P[np.arange(3), self.perm] = 1.0
        self.det = round(np.linalg.det(np.diag(self.sign) @ P))

    def vec(self, a):
        a = np.asarray(a, dtype=np.float64)
        return self.sign * a[..., self.perm]

    def triangles(self, tri):
        t = self.vec(tri)
        return t if self.det > 0 else t[:, [0, 2, 1], :]     # keep outward = counter-clockwise

    def region(self, r):
        par = np.array(r.par, dtype=np.float64)
        if r.kind == I.REGION_SPHERE_BAND:
            return I.Region(r.kind, r.level, (*self.vec(par[:3]), *par[3:]))
        assert r.kind == I.REGION_BOX
        a, b = self.vec(par[:3]), self.vec(par[3:6])
        return I.Region(r.kind, r.level, (*np.minimum(a, b), *np.maximum(a, b)))

    def ijk(self, ijk, hi):
        src = ijk.astype(np.int64)[:, self.perm]
        return np.where(self.sign[None, :] < 0, hi[None, :] - src, src)


def _regions():
    return [I.Region(I.REGION_SPHERE_BAND, 5, (*CENTRE, 0.2, 0.04)),
            I.Region(I.REGION_BOX, 4, (-0.3, -0.1, -0.2, 0.05, 0.35, 0.1))]


def _body():
    return I.icosphere(2, 0.2, CENTRE, 1e-3, 7)


def _key(ijk):
    ijk = ijk.astype(np.int64)
    return (ijk[:, 0] << 42) | (ijk[:, 1] << 21) | ijk[:, 2]


def _face(m):
    ijk = m.node_ijk.astype(np.int64)
    return np.any((ijk == 0) | (ijk == m.hiI[None, :]), axis=1)


@pytest.fixture(scope="module")
def original():
    return OracleMesh(LO, HI, 2, _regions(), _body(), 3)


def _fields(n, seed):
    u = np.zeros((n, 4))
    u[:, 0] = 0.6
    u[:, :4] += I.normal(seed, n * 4, 0.2).reshape(n, 4)
    up = u + I.normal(seed + 1, n * 4, 0.05).reshape(n, 4)
    up2 = up + I.normal(seed + 2, n * 4, 0.05).reshape(n, 4)
    f = I.normal(seed + 3, n * 4, 1.0).reshape(n, 4)
    v = I.normal(seed + 4, n * 4, 1.0).reshape(n, 4)
    return u, up, up2, f, v


def _move_nodal(T, a):
    b = a.copy()
    b[:, :3] = T.vec(a[:, :3])
    return b


@pytest.mark.parametrize("T", [Motion((2, 0, 1), (1, 1, 1)),       # cyclic axis permutation
                               Motion((0, 1, 2), (-1, 1, 1)),      # reflection x -> -x
                               Motion((1, 0, 2), (1, 1, -1))],     # swap x, y and reflect z
                         ids=["rotate_xyz", "reflect_x", "swap_xy_reflect_z"])
def test_residual_and_jvp_commute_with_rigid_motions(original, T):
    A = original
    B = OracleMesh(LO, HI, 2, [T.region(r) for r in _regions()], T.triangles(_body()), 3)
    # the two meshes are images of each other
    assert (A.n_elem, A.n_nodes, A.n_hang) == (B.n_elem, B.n_nodes, B.n_hang)
    assert np.array_equal(A.hiI, B.hiI)
    mkA, mkB = A.markers()[0], B.markers()[0]
    assert np.array_equal(np.bincount(mkA, minlength=3), np.bincount(mkB, minlength=3))
    assert (mkA == 2).sum() > 20 and A.n_hang > 0
    sA, sB = A.surface_points(), B.surface_points()
    assert sA.shape == sB.shape
    keyB = _key(B.node_ijk)
    order = np.argsort(keyB)
    pos = np.searchsorted(keyB[order], _key(T.ijk(A.node_ijk, A.hiI)))
    assert (pos < B.n_nodes).all()
    img = order[pos]                                    # node i of A sits at node img[i] of B
    assert np.array_equal(B.node_ijk[img].astype(np.int64), T.ijk(A.node_ijk, A.hiI))

    u, up, up2, f, v = _fields(A.n_nodes, 40)
    g = np.array([0.1, -0.3, 0.2])

    def moved(a):
        out = np.empty_like(a)
        out[img] = _move_nodal(T, a)
        return out

    for scheme in (I.SCHEME_BE, I.SCHEME_CN, I.SCHEME_BDF2):
        phA = I.Physics(rho=1.1, mu=0.015, dt=0.02, scheme=scheme, Cb=4.0, g=tuple(g), uinf=(0.0, 0.0, 0.0))
        phB = I.Physics(rho=1.1, mu=0.015, dt=0.02, scheme=scheme, Cb=4.0, g=tuple(T.vec(g)),
                        uinf=(0.0, 0.0, 0.0))
        RA, JA = A.residual_jvp(phA, u, up, up2, f=f, v=v)
        RB, JB = B.residual_jvp(phB, moved(u), moved(up), moved(up2), f=moved(f), v=moved(v))
        keep = ~_face(A)
        for XA, XB in ((RA, RB), (JA, JB)):
            want = _move_nodal(T, XA)[keep]
            got = XB[img[keep]]
            assert np.abs(got - want).max() <= 1e-12 * np.abs(XA).max(), scheme
        # the force on the body moves with it (a polar vector: reflected with the body)
        FA, FB = A.surface_force(phA, u, up), B.surface_force(phB, moved(u), moved(up))
        assert np.abs(FB - T.vec(FA)).max() <= 1e-12 * np.abs(FA).max(), scheme


def test_symmetry_pin_detects_a_one_axis_slip(original):
    """The pin fails when one axis is treated differently: moving the state but not the body
    (the body is not symmetric under the motion) must change the interior rows."""
    A = original
    T = Motion((2, 0, 1), (1, 1, 1))
    B = OracleMesh(LO, HI, 2, [T.region(r) for r in _regions()], _body(), 3)   # body not moved
    u, up, up2, f, v = _fields(A.n_nodes, 40)
    ph = I.Physics(rho=1.1, mu=0.015, dt=0.02, scheme=I.SCHEME_BE, uinf=(0.0, 0.0, 0.0))
    RA = A.residual(ph, u, up, f=f)
    assert (A.n_elem, A.n_nodes) == (B.n_elem, B.n_nodes)     # the octree follows the moved regions
    keyB = _key(B.node_ijk)
    order = np.argsort(keyB)
    pos = np.clip(np.searchsorted(keyB[order], _key(T.ijk(A.node_ijk, A.hiI))), 0, B.n_nodes - 1)
    img = order[pos]
    moved = np.empty_like(u)
    moved[img] = _move_nodal(T, u)
    mp = np.empty_like(up)
    mp[img] = _move_nodal(T, up)
    mf = np.empty_like(f)
    mf[img] = _move_nodal(T, f)
    RB = B.residual(ph, moved, mp, f=mf)
    keep = ~_face(A)
    assert np.abs(RB[img[keep]] - _move_nodal(T, RA)[keep]).max() > 1e-6 * np.abs(RA).max()
