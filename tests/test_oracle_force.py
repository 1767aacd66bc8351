"""Pins of the oracle's force on the body (the weak-boundary terms of Eq. (weakbc) tested with
w = e_i, the conservative force of weak Dirichlet conditions).

What is fixed independently of the oracle:
* hydrostatics: u = 0, g = 0 and a linear pressure p = c.x leave only the pressure traction, and
  the divergence theorem over the triangulated body gives F = -c V, V the polyhedron's volume
  (the surface rule integrates p n exactly on flat triangles);
* a body moving with a uniform flow feels no force;
* with no strong rows, every node's momentum rows summed equal F in the hydrostatic state: the
  volume terms cancel by partition of unity (sum_a phi_a = 1, sum_a grad phi_a = 0);
* under Crank-Nicolson the force is the backward-Euler force at the midpoint velocity, with the
  pressure at n+1.
"""
import numpy as np
import pytest

from paper_2009_00706_gb300 import inputs as I


def _volume(tri):
    return float(np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0)


@pytest.mark.parametrize("c", [(0.7, -0.2, 0.4), (0.0, 0.0, 1.0)])
def test_hydrostatic_force_is_minus_c_times_volume(small_sphere_oracle, c):
    w, m = small_sphere_oracle
    tri = w.triangles()
    assert m.surface_points().shape[0] == 3 * tri.shape[0]      # every surface point kept
    c = np.asarray(c)
    U = np.zeros((m.n_nodes, 4))
    U[:, 3] = m.node_xyz @ c + 0.3
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, g=(0.0, 0.0, 0.0))
    F = m.surface_force(ph, U, U)
    V = _volume(tri)
    assert np.abs(F + c * V).max() <= 1e-12 * max(np.abs(c).max() * V, 1e-300)


def test_body_moving_with_uniform_flow_feels_no_force(small_sphere_oracle):
    w, m = small_sphere_oracle
    ub = (0.8, 0.3, -0.2)
    U = np.zeros((m.n_nodes, 4))
    U[:, :3] = ub
    for scheme in (I.SCHEME_BE, I.SCHEME_CN, I.SCHEME_BDF2):
        F = m.surface_force(I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=scheme, g=ub), U, U)
        assert np.abs(F).max() <= 1e-14


def test_force_equals_summed_momentum_rows_without_strong_rows():
    c = (0.5, 0.5, 0.5)
    from oracle.oracle import OracleMesh
    tri = I.icosphere(2, 0.2, c, 1e-4, 3)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, [I.Region(I.REGION_SPHERE_BAND, 4, (*c, 0.2, 0.05))], tri, 3)
    m.set_dirichlet(np.zeros(m.n_nodes, np.uint8), np.zeros((m.n_nodes, 4)))   # no box rows
    cp = np.array([0.3, -0.6, 0.25])
    U = np.zeros((m.n_nodes, 4))
    U[:, 3] = m.node_xyz @ cp
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, g=(0.0, 0.0, 0.0))
    R = m.residual(ph, U, U)
    F = m.surface_force(ph, U, U)
    # In-only nodes hold U - g = 0 in their momentum rows; every other row is the residual
    assert np.abs(R[:, :3].sum(axis=0) - F).max() <= 1e-12 * np.abs(F).max()
    if m.surface_points().shape[0] == 3 * tri.shape[0]:
        assert np.abs(F + cp * _volume(tri)).max() <= 1e-12 * np.abs(F).max()


def test_crank_nicolson_force_sees_the_midpoint_velocity(small_sphere_oracle):
    """Under CN the surface terms are evaluated at u_s = (u + u_prev) / 2 with the pressure at
    n+1: the CN force at (u, u_prev) equals the BE force at that state."""
    w, m = small_sphere_oracle
    u, up, _ = I.state(m.n_nodes, 12)
    u[:, 3] = I.normal(23, m.n_nodes, 0.2)
    up[:, :3] += I.normal(24, m.n_nodes * 3, 0.05).reshape(-1, 3)
    mid = u.copy()
    mid[:, :3] = 0.5 * (u[:, :3] + up[:, :3])
    g = (0.1, 0.0, -0.05)
    F_cn = m.surface_force(I.Physics(scheme=I.SCHEME_CN, g=g), u, up)
    F_be = m.surface_force(I.Physics(scheme=I.SCHEME_BE, g=g), mid, mid)
    assert np.abs(F_cn - F_be).max() <= 1e-13 * np.abs(F_be).max()
