"""Pins of the oracle's Newton-GMRES against dense Gaussian elimination and closed forms."""
import numpy as np

from oracle.krylov import gmres, newton
from paper_2009_00706_gb300 import inputs as I


def _system(n, seed):
    A = I.normal(seed, n * n).reshape(n, n) / np.sqrt(n) + 3.0 * np.eye(n)
    b = I.normal(seed + 1, n)
    return A, b


def test_gmres_full_krylov_equals_dense_solve():
    A, b = _system(40, 3)
    x, its, _ = gmres(lambda z: A @ z, b, m=40, rtol=1e-13)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    assert its <= 40


def test_gmres_restarted_and_right_preconditioned():
    A, b = _system(60, 5)
    D = np.diag(A)
    x, its, hist = gmres(lambda z: A @ z, b, m=8, rtol=1e-10, precond=lambda z: z / D)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.0001
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-8 * np.linalg.norm(x)


def test_gmres_exact_preconditioner_one_iteration():
    A, b = _system(30, 7)
    Ainv = np.linalg.inv(A)
    x, its, _ = gmres(lambda z: A @ z, b, m=10, rtol=1e-12, precond=lambda z: Ainv @ z)
    assert its == 1


def test_newton_linear_problem_converges_in_one_step():
    A, b = _system(25, 9)
    u, st = newton(lambda u: A @ u - b, lambda u, v: A @ v, np.zeros(25), rtol=1e-10, gmres_m=25, gmres_rtol=1e-13)
    assert st["newton_its"] == 1 and st["converged"]


def test_newton_quadratic_convergence():
    A, b = _system(20, 11)
    R = lambda u: A @ u + 0.3 * u ** 3 - b
    J = lambda u, v: A @ v + 0.9 * u ** 2 * v
    u, st = newton(R, J, np.zeros(20), rtol=1e-14, gmres_m=20, gmres_rtol=1e-14)
    h = st["res_hist"]
    assert st["converged"]
    # once in the quadratic regime the residual roughly squares each step
    k = next(i for i in range(1, len(h)) if h[i] < 1e-3 * h[0])
    if k + 1 < len(h) and h[k + 1] > 1e-15 * h[0]:
        assert h[k + 1] <= 10.0 * h[k] ** 2 / h[0]
