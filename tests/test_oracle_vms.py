"""Pins of the oracle's VMS residual and Jacobian against closed forms and invariants.

What is fixed independently of the oracle's code:
* at three special states the element Jacobian reduces to textbook Q1 matrices (tests/
  fem_closed_form.py): u = 0 (Stokes-like), constant u (Galerkin convection + SUPG/PSPG), and
  u = 0 with a non-zero time derivative (fine scales u' != 0 with grad u = 0), which isolates
  the cross-stress and Reynolds-stress terms (6), (7), (8) of Eq. (vms);
* the local residual at the last state in closed form;
* a linear patch test (R = 0 at interior nodes, also across hanging faces/edges);
* uniform flow gives R = 0, with and without an immersed body moving with the flow;
* J v against central finite differences of R, and linearity of J in v;
* second-order L2 convergence on a manufactured solution.
"""
import numpy as np
import pytest

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import inputs as I
from tests import fem_closed_form as cf
from tests.fem_closed_form import Z, e, ee, integral
from tests.oracle_assembly import assemble_jacobian


def K_idx(a, i):
    return a * 4 + i


def tau_m(rho, mu, dt, h, CI, u2):
    g2 = (2.0 / h) ** 2
    nu = mu / rho
    return 1.0 / np.sqrt(4.0 / dt ** 2 + g2 * u2 + CI * nu ** 2 * 3.0 * g2 ** 2)


def tau_c(tm, h):
    return 1.0 / (tm * 3.0 * (2.0 / h) ** 2)


def base_blocks(h, rho, mu, dt, tm, tc):
    """Jacobian blocks common to the special states (u' = 0 parts)."""
    M, L = cf.mass(h), cf.laplace(h)
    K = np.zeros((32, 32))
    for i in range(3):
        for j in range(3):
            blk = mu * integral(h, e(j), e(i)) + rho * tc * integral(h, e(i), e(j))
            if i == j:
                blk = blk + rho / dt * M + mu * L
            K[i::4, j::4] += blk
        K[i::4, 3::4] += -integral(h, e(i), Z)
    for j in range(3):
        visc = sum(integral(h, e(k), ee(k, j)) for k in range(3) if k != j)
        K[3::4, j::4] += integral(h, Z, e(j)) + tm / dt * integral(h, e(j), Z) - tm * mu / rho * visc
    K[3::4, 3::4] += tm / rho * L
    return K


@pytest.fixture(scope="module")
def cube8():
    # eight level-1 elements of the unit cube, no immersed body: element 0 is [0, 0.5]^3
    return OracleMesh((0, 0, 0), (1, 1, 1), 1, [])


PH = dict(rho=1.3, mu=0.07, dt=0.05, CI=36.0)


def phys(**kw):
    d = dict(PH)
    d.update(kw)
    return I.Physics(rho=d["rho"], mu=d["mu"], dt=d["dt"], scheme=I.SCHEME_BE, CI=d["CI"])


def test_jacobian_rest_state_is_textbook(cube8):
    m = cube8
    ph = phys()
    h = 0.5
    U = np.zeros((m.n_nodes, 4))
    K, mk = m.element_matrix(ph, U, U, 0)
    assert mk == 0
    tm = tau_m(ph.rho, ph.mu, ph.dt, h, ph.CI, 0.0)
    Kx = base_blocks(h, ph.rho, ph.mu, ph.dt, tm, tau_c(tm, h))
    assert np.abs(K - Kx).max() <= 1e-13 * np.abs(Kx).max()


def test_jacobian_uniform_flow_is_galerkin_plus_supg_pspg(cube8):
    m = cube8
    ph = phys()
    h = 0.5
    ub = np.array([0.7, -0.4, 0.25])
    U = np.zeros((m.n_nodes, 4))
    U[:, :3] = ub
    K, _ = m.element_matrix(ph, U, U, 0)
    tm = tau_m(ph.rho, ph.mu, ph.dt, h, ph.CI, ub @ ub)
    Kx = base_blocks(h, ph.rho, ph.mu, ph.dt, tm, tau_c(tm, h))
    A = sum(ub[k] * integral(h, Z, e(k)) for k in range(3))              # int phi_a u.grad phi_b
    Sa = sum(ub[k] * integral(h, e(k), Z) for k in range(3))             # int (u.grad phi_a) phi_b
    SS = sum(ub[k] * ub[l] * integral(h, e(k), e(l)) for k in range(3) for l in range(3))
    rho, mu, dt = ph.rho, ph.mu, ph.dt
    for i in range(3):
        for j in range(3):
            blk = np.zeros((8, 8))
            if i == j:
                blk += rho * A + tm * (rho / dt * Sa + rho * SS)
            else:
                blk += -tm * mu * sum(ub[k] * integral(h, e(k), ee(i, j)) for k in range(3))
            Kx[i::4, j::4] += blk
        Kx[i::4, 3::4] += tm * sum(ub[k] * integral(h, e(k), e(i)) for k in range(3))
    for j in range(3):
        Kx[3::4, j::4] += tm * sum(ub[k] * integral(h, e(j), e(k)) for k in range(3))
    assert np.abs(K - Kx).max() <= 1e-13 * np.abs(Kx).max()


def _state_c(m):
    """u = 0, p = 0, u_prev = c: du/dt = -c/dt, u' = tau_M rho c / dt, grad u = 0."""
    c = np.array([0.3, 0.5, -0.2])
    U = np.zeros((m.n_nodes, 4))
    Up = np.zeros((m.n_nodes, 4))
    Up[:, :3] = c
    return c, U, Up


def test_residual_time_derivative_state_closed_form(cube8):
    m = cube8
    ph = phys()
    h = 0.5
    c, U, Up = _state_c(m)
    r = m.element_residual(ph, U, Up, 0)
    tm = tau_m(ph.rho, ph.mu, ph.dt, h, ph.CI, 0.0)
    a = -c / ph.dt
    up = tm * ph.rho * c / ph.dt
    rx = np.zeros((8, 4))
    dphi = np.stack([cf.int_dphi(h, j) for j in range(3)], axis=1)   # [8, 3]
    for i in range(3):
        rx[:, i] = ph.rho * a[i] * cf.int_phi(h) - up[i] * (dphi @ up) / ph.rho
    rx[:, 3] = -(dphi @ up) / ph.rho
    assert np.abs(r - rx).max() <= 1e-13 * np.abs(rx).max()


def test_jacobian_time_derivative_state_isolates_terms_6_7_8(cube8):
    m = cube8
    ph = phys()
    h = 0.5
    rho, mu, dt = ph.rho, ph.mu, ph.dt
    c, U, Up = _state_c(m)
    K, _ = m.element_matrix(ph, U, Up, 0)
    tm = tau_m(rho, mu, dt, h, ph.CI, 0.0)
    Kx = base_blocks(h, rho, mu, dt, tm, tau_c(tm, h))
    up = tm * rho * c / dt
    taubar = 1.0 / np.sqrt((2.0 / h) ** 2 * (up @ up))
    for i in range(3):
        for j in range(3):
            blk = -up[i] * integral(h, e(j), Z)                                        # term (4), delta u-bar
            if i == j:
                blk = blk + sum(up[k] * integral(h, Z, e(k)) for k in range(3))          # term (6)
                blk = blk + taubar * sum(up[k] * up[l] * integral(h, e(k), e(l))         # term (8)
                                         for k in range(3) for l in range(3))
            # term (7): -(1/rho) grad w : (du' x u' + u' x du'), du' = -tau_M d r_M
            t7 = np.zeros((8, 8))
            for k in range(3):
                dri = (rho / dt * integral(h, e(k), Z) if i == j else 0.0) - \
                      (mu * integral(h, e(k), ee(i, j)) if i != j else 0.0)
                drk = (rho / dt * integral(h, e(k), Z) if k == j else 0.0) - \
                      (mu * integral(h, e(k), ee(k, j)) if k != j else 0.0)
                t7 = t7 + dri * up[k] + up[i] * drk
            blk = blk + tm / rho * t7
            Kx[i::4, j::4] += blk
        t7p = sum(integral(h, e(k), e(i)) * up[k] + up[i] * integral(h, e(k), e(k)) for k in range(3))
        Kx[i::4, 3::4] += tm / rho * t7p
    assert np.abs(K - Kx).max() <= 1e-12 * np.abs(Kx).max()


def _box_face_nodes(m):
    ijk = m.node_ijk.astype(np.int64)
    return np.any((ijk == 0) | (ijk == m.hiI[None, :]), axis=1)


def test_linear_patch_test_with_hanging_nodes():
    # adaptive mesh with hanging faces and edges; no body
    reg = [I.Region(I.REGION_SPHERE_BAND, 4, (0.4, 0.55, 0.5, 0.2, 0.03))]
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, reg)
    assert m.n_hang > 0
    rho, mu = 1.3, 0.07
    ph = I.Physics(rho=rho, mu=mu, dt=0.05, scheme=I.SCHEME_BE)
    A = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [0.25, 0.15, -0.7]])   # trace 0
    b = np.array([1.0, 0.2, -0.1])
    cp = np.array([0.5, -1.0, 0.3])
    X = m.node_xyz
    U = np.zeros((m.n_nodes, 4))
    U[:, :3] = X @ A.T + b
    U[:, 3] = X @ cp + 0.2
    F = (U[:, :3] @ A.T) + cp / rho
    R = m.residual(ph, U, U, f=F)
    inner = ~_box_face_nodes(m)
    scale = np.abs(U).max() * (1.0 / 16) ** 2
    assert np.abs(R[inner]).max() <= 1e-12 * scale


def test_uniform_flow_zero_residual_no_body():
    reg = [I.Region(I.REGION_SPHERE_BAND, 4, (0.5, 0.5, 0.5, 0.2, 0.05))]
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, reg)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, uinf=(1.0, 0.0, 0.0))
    U = np.zeros((m.n_nodes, 4))
    U[:, 0] = 1.0
    R = m.residual(ph, U, U)
    assert np.abs(R).max() <= 1e-14


def test_uniform_flow_zero_residual_body_moving_with_flow(small_sphere_oracle):
    w, m = small_sphere_oracle
    ub = (0.8, 0.3, -0.2)
    ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, g=ub, uinf=ub)
    U = np.zeros((m.n_nodes, 4))
    U[:, :3] = ub
    R = m.residual(ph, U, U)
    assert np.abs(R).max() <= 1e-13


def test_nitsche_sum_closed_form(small_sphere_oracle):
    """Constant u = ub, p = 0, no-slip body: the volume terms vanish and, by partition of unity,
    the momentum rows summed over all nodes equal sum_q w_q (tau_B ub - [ub.n < 0] rho (ub.n) ub)."""
    w, m = small_sphere_oracle
    ub = np.array([0.8, 0.3, -0.2])
    rho, mu, Cb = 1.0, 0.02, 4.0
    ph = I.Physics(rho=rho, mu=mu, dt=0.01, g=(0, 0, 0), uinf=tuple(ub), Cb=Cb)
    U = np.zeros((m.n_nodes, 4))
    U[:, :3] = ub
    R = m.residual(ph, U, U)
    sq = m.surface_points()
    n, wq, hb = sq[:, 3:6], sq[:, 6], sq[:, 7]
    un = n @ ub
    exp = (wq * Cb * mu / hb)[:, None] * ub[None, :] - (wq * np.where(un < 0, rho * un, 0.0))[:, None] * ub[None, :]
    exp = exp.sum(axis=0)
    mk, _, _ = m.markers()
    active = np.zeros(m.n_nodes, bool)
    for el in np.where(mk != 1)[0]:
        for c in range(8):
            idx = m.conn[el, c]
            if idx < m.n_nodes:
                active[idx] = True
            else:
                active[m.hang_parents[idx - m.n_nodes, :m.hang_np[idx - m.n_nodes]]] = True
    rows = active & ~_box_face_nodes(m)
    got = R[rows, :3].sum(axis=0)
    assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max()


def test_jvp_matches_central_differences(small_sphere_oracle):
    w, m = small_sphere_oracle
    u, up, v = I.state(m.n_nodes, 3)
    ph = w.physics
    R, J = m.residual_jvp(ph, u, up, v=v)
    d = 1e-6 * np.linalg.norm(u) / np.linalg.norm(v)
    Rp = m.residual(ph, u + d * v, up)
    Rm = m.residual(ph, u - d * v, up)
    fd = (Rp - Rm) / (2 * d)
    assert np.linalg.norm(fd - J) <= 1e-6 * np.linalg.norm(J)


def test_jvp_linear_in_v(small_sphere_oracle):
    w, m = small_sphere_oracle
    u, up, v = I.state(m.n_nodes, 5)
    v2 = I.normal(77, m.n_nodes * 4).reshape(m.n_nodes, 4)
    ph = w.physics
    J1 = m.jvp(ph, u, up, v)
    J2 = m.jvp(ph, u, up, v2)
    J3 = m.jvp(ph, u, up, 2.5 * v - 0.75 * v2)
    assert np.linalg.norm(J3 - (2.5 * J1 - 0.75 * J2)) <= 1e-13 * np.linalg.norm(J3)


def test_bdf2_and_cn_jvp_match_central_differences():
    reg = [I.Region(I.REGION_SPHERE_BAND, 4, (0.5, 0.5, 0.5, 0.2, 0.05))]
    m = OracleMesh((0, 0, 0), (1, 1, 1), 2, reg)
    u, up, v = I.state(m.n_nodes, 9)
    up2 = up.copy()
    up2[:, :3] += I.normal(11, m.n_nodes * 3, 0.01).reshape(-1, 3)
    for scheme in (I.SCHEME_CN, I.SCHEME_BDF2):
        ph = I.Physics(rho=1.0, mu=0.01, dt=0.01, scheme=scheme)
        R, J = m.residual_jvp(ph, u, up, up2, v=v)
        d = 1e-6 * np.linalg.norm(u) / np.linalg.norm(v)
        fd = (m.residual(ph, u + d * v, up, up2) - m.residual(ph, u - d * v, up, up2)) / (2 * d)
        assert np.linalg.norm(fd - J) <= 1e-6 * np.linalg.norm(J)


# ---------------------------------------------------------------------------------------
# manufactured solution: second-order convergence of the discrete solution
# ---------------------------------------------------------------------------------------
def _exact(X, A=1.0):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    pi = np.pi
    u = np.stack([A * np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * z),
                  -A * np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * z),
                  np.zeros_like(x)], axis=1)
    p = np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z)
    # grad u, grad p analytically
    G = np.zeros((X.shape[0], 3, 3))
    G[:, 0, 0] = A * pi * np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z)
    G[:, 0, 1] = -A * pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)
    G[:, 0, 2] = -A * pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z)
    G[:, 1, 0] = A * pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)
    G[:, 1, 1] = -A * pi * np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z)
    G[:, 1, 2] = A * pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z)
    gp = np.stack([-pi * np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * z),
                   -pi * np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * z),
                   -pi * np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * z)], axis=1)
    lap = -3.0 * pi ** 2 * u
    return u, p, G, gp, lap


def mms_error(level, rho=1.0, mu=0.1):
    import scipy.sparse.linalg as spla
    m = OracleMesh((0, 0, 0), (1, 1, 1), level, [])
    X = m.node_xyz
    u, p, G, gp, lap = _exact(X)
    conv = np.einsum("nij,nj->ni", G, u)
    F = conv + (-mu * lap + gp) / rho
    face = _box_face_nodes(m)
    mask = np.where(face, 7, 0).astype(np.uint8)
    mask[0] |= 8
    vals = np.zeros((m.n_nodes, 4))
    vals[:, :3] = u
    vals[:, 3] = p
    m.set_dirichlet(mask, vals)
    ph = I.Physics(rho=rho, mu=mu, dt=1e12, scheme=I.SCHEME_BE)
    Up = np.zeros((m.n_nodes, 4))
    U = np.zeros((m.n_nodes, 4))
    U[face, :3] = u[face]
    U[0, 3] = p[0]
    for _ in range(12):
        R = m.residual(ph, U, Up, f=F)
        if np.linalg.norm(R) < 1e-11:
            break
        J = assemble_jacobian(m, ph, U, Up, F, mask)
        U = U - spla.spsolve(J.tocsc(), R.ravel()).reshape(-1, 4)
    assert np.linalg.norm(m.residual(ph, U, Up, f=F)) < 1e-9
    return np.sqrt(np.mean(np.sum((U[:, :3] - u) ** 2, axis=1)))


@pytest.mark.slow
def test_manufactured_solution_second_order():
    e2, e3, e4 = mms_error(2), mms_error(3), mms_error(4)
    assert e3 / e4 > 3.2, (e2, e3, e4)
    assert e2 / e3 > 2.5, (e2, e3, e4)


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_jvp_matches_complex_step(scheme):
    """The dual-number J v against the complex step Im R(u + i eps v) / eps, a derivative with no
    difference quotient: agreement to 1e-12 on a mesh with hanging nodes, Intercepted elements
    and surface points, for BE, CN and BDF2."""
    from oracle.oracle import OracleMesh
    from paper_2009_00706_gb300 import inputs as I
    c = (0.5, 0.5, 0.5)
    regs = [I.Region(I.REGION_SPHERE_BAND, 4, (*c, 0.2, 0.05))]
    tri = I.icosphere(2, 0.2, c, 1e-4, 1)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 2, regs, tri, 2)
    u, up, v = I.state(o.n_nodes, 9, sigma=0.2)
    up2 = up.copy()
    up2[:, :3] += I.normal(10, 3 * o.n_nodes, 0.05).reshape(-1, 3)
    ph = I.Physics(rho=1.0, mu=0.03, dt=0.02, scheme=scheme, g=(0.1, 0.0, 0.0))
    _, Jd = o.residual_jvp(ph, u, up, up2, v=v)
    Jc = o.jvp_complex_step(ph, u, up, v, up2)
    assert np.linalg.norm(Jc - Jd) <= 1e-12 * np.linalg.norm(Jd), np.linalg.norm(Jc - Jd) / np.linalg.norm(Jd)


def test_steady_velocity_makes_the_time_schemes_agree(small_sphere_oracle):
    """With the velocity unchanged between time levels (u = u_prev = u_prev2) the time derivative
    vanishes and the spatial terms see the same velocity under BE, CN (theta = 1/2) and BDF2.
    The pressure differs from p_prev: with the pressure taken at n+1 (reading of the CN scheme)
    the three residuals coincide; an averaged or lagged pressure would break this.  (J v differs:
    the schemes weight the tangent by theta and by their time coefficient.)"""
    w, m = small_sphere_oracle
    u, up, v = I.state(m.n_nodes, 8)
    u[:, :3] = up[:, :3]
    u[:, 3] = I.normal(21, m.n_nodes, 0.3)                      # p != p_prev = 0
    out = {}
    for scheme in (I.SCHEME_BE, I.SCHEME_CN, I.SCHEME_BDF2):
        ph = I.Physics(rho=1.0, mu=0.02, dt=0.01, scheme=scheme)
        out[scheme] = m.residual(ph, u, up, up)
    for scheme in (I.SCHEME_CN, I.SCHEME_BDF2):
        assert np.abs(out[scheme] - out[I.SCHEME_BE]).max() <= 1e-13 * np.abs(out[I.SCHEME_BE]).max(), scheme
