"""Pins of the oracle's H-LU factorisation and direct solver (Sec. 3.2,
"H-LU factorization and direct solver"; the estimator of Sec. 3.3,
Eq. est_direct).  Without admissible blocks the recursion must reproduce the
(unique) LU factorisation without pivoting of the dense matrix; with them the
factors must reproduce the H-matrix to the truncation tolerance eps_LU and the
solve must converge to the exact solve of A_H as eps_LU -> 0."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

NC = 240


def setup(oracle, kernel, eta, eps=1e-6):
    pts = inputs.fibonacci_sphere(NC)
    nrm = inputs.sphere_normals(pts) if kernel == "T" else None
    w = np.full(NC, 4 * np.pi / NC)
    pb = oracle.problem(1, 2, 1, 4.0, kernel, 1.0, w)
    H = oracle.HMatrix(pb, pts, nrm, eps=eps, eta=eta, leaf=16)
    N = 3 * NC
    AH = np.stack([H.matvec(e) for e in np.eye(N)], 1)  # original order
    perm = H.perm()
    dof = (3 * perm[:, None] + np.arange(3)).ravel()
    return pb, pts, nrm, H, AH, AH[np.ix_(dof, dof)]


def test_dense_limit_is_lu_without_pivoting(oracle):
    """eta -> 0: every block is dense, the recursive 2 x 2 steps are block
    Gaussian elimination, and L U = A with L unit lower, U upper (the LU
    factorisation without pivoting is unique); the solve is the exact one."""
    pb, pts, nrm, H, AH, At = setup(oracle, "U", 1e-9)
    F = oracle.HLU(H, 1e-9, 1e-8)
    assert F.status == 0
    L, U = F.dense()
    assert np.allclose(np.diag(L), 1.0) and np.abs(np.triu(L, 1)).max() == 0.0
    assert np.abs(np.tril(U, -1)).max() == 0.0
    assert np.linalg.norm(L @ U - At) <= 1e-12 * np.linalg.norm(At)
    b = inputs.random_rhs(3 * NC, seed=1)
    x = F.solve(b)
    xs = np.linalg.solve(AH, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("kernel", ["U", "T"])
@pytest.mark.parametrize("eps_lu", [1e-4, 1e-6])
def test_factors_reproduce_A_H(oracle, kernel, eps_lu):
    """eta = 3: ||L U - A_H||_F <= eps_LU ||A_H||_F (the updates of low-rank
    blocks are truncated with eps_LU), triangular factors, and the direct solve
    has a relative residual below eps_LU."""
    pb, pts, nrm, H, AH, At = setup(oracle, kernel, 3.0)
    F = oracle.HLU(H, 3.0, eps_lu)
    assert F.status == 0
    L, U = F.dense()
    assert np.abs(np.triu(L, 1)).max() == 0.0 and np.abs(np.tril(U, -1)).max() == 0.0
    assert np.linalg.norm(L @ U - At) <= eps_lu * np.linalg.norm(At)
    b = inputs.random_rhs(3 * NC, seed=2)
    x = F.solve(b)
    assert np.linalg.norm(AH @ x - b) <= eps_lu * np.linalg.norm(b)


def test_solve_converges_as_eps_lu_decreases(oracle):
    """eps_LU -> 0: the direct solution tends to the exact solution of
    A_H x = b (numpy solve), error proportional to eps_LU."""
    pb, pts, nrm, H, AH, At = setup(oracle, "U", 3.0)
    b = inputs.random_rhs(3 * NC, seed=3)
    xs = np.linalg.solve(AH, b)
    errs = []
    for e in (1e-4, 1e-7, 1e-10):
        x = oracle.HLU(H, 3.0, e).solve(b)
        errs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert errs[2] <= 1e-9 and errs[0] > errs[1] > errs[2]


def test_estimator_bound_of_the_direct_solver(oracle):
    """Eq. est_direct: ||b - A x0|| <= ||b - A_H x0|| + ||A_H - A||_F ||x0||
    for the H-LU solution x0 (A the exact dense matrix)."""
    pb, pts, nrm, H, AH, At = setup(oracle, "U", 3.0, eps=1e-3)
    A = oracle.dense_matrix(pb, pts, nrm)
    x0 = oracle.HLU(H, 3.0, 1e-4).solve(inputs.random_rhs(3 * NC, seed=4))
    b = inputs.random_rhs(3 * NC, seed=4)
    lhs = np.linalg.norm(b - A @ x0)
    delta = np.linalg.norm(b - AH @ x0)
    dH = np.linalg.norm(AH - A)
    assert lhs <= delta + dH * np.linalg.norm(x0)
    assert dH > 0 and lhs > delta  # the H approximation error is what the bound adds
