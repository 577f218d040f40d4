"""Pins of the oracle's H-matrix (Sec. 2-3.1) and GMRES: the all-dense limit
equals the dense product, H vs dense within 3 eps at config 1, linearity,
GMRES vs a dense solve, and the a-posteriori bound Eq. est_direct."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs


@pytest.fixture(scope="module")
def cfg1(oracle):
    pts = inputs.fibonacci_sphere(1536)
    nrm = inputs.sphere_normals(pts)
    out = {}
    for kern in ("U", "T"):
        pb = oracle.problem(1, 2, 1, 4.0, kern)
        out[kern] = (pb, oracle.dense_matrix(pb, pts, nrm),
                     oracle.HMatrix(pb, pts, nrm, eps=1e-4, eta=3.0, leaf=32))
    return pts, nrm, out


def test_all_dense_limit(oracle):
    """eta -> 0: no block is admissible, the H-matvec is the dense product."""
    pts = inputs.fibonacci_sphere(700)
    pb = oracle.problem(1, 2, 1, 4.0, "U")
    H = oracle.HMatrix(pb, pts, eps=1e-4, eta=1e-12, leaf=32)
    blk, _, _ = H.blocks()
    assert blk["admissible"].sum() == 0
    x = inputs.random_rhs(3 * 700, seed=3)
    yd = oracle.dense_matrix(pb, pts) @ x
    assert np.linalg.norm(H.matvec(x) - yd) <= 1e-13 * np.linalg.norm(yd)


@pytest.mark.parametrize("kern", ["U", "T"])
def test_hmatvec_vs_dense(oracle, cfg1, kern):
    """Config 1: ||A_H x - A x|| <= 3 eps ||A x|| for a N(0,1) right-hand side."""
    pts, nrm, d = cfg1
    pb, A, H = d[kern]
    x = inputs.random_rhs(3 * len(pts), seed=0)
    yd = A @ x
    assert np.linalg.norm(H.matvec(x) - yd) <= 3e-4 * np.linalg.norm(yd)


def test_hmatvec_linear(oracle, cfg1):
    pts, nrm, d = cfg1
    _, _, H = d["U"]
    x1 = inputs.random_rhs(3 * len(pts), seed=1)
    x2 = inputs.random_rhs(3 * len(pts), seed=2)
    a = 0.3 - 1.1j
    y = H.matvec(a * x1 + x2)
    assert np.linalg.norm(y - (a * H.matvec(x1) + H.matvec(x2))) <= 1e-13 * np.linalg.norm(y)


def test_dense_rows_matvec(oracle, cfg1):
    pts, nrm, d = cfg1
    _, A, _ = d["T"]
    x = inputs.random_rhs(3 * len(pts), seed=4)
    rows = np.array([0, 5, 17, 400, 3 * len(pts) - 1])
    out = oracle.dense_rows_matvec(d["T"][0], pts, nrm, rows, x)
    assert np.allclose(out, (A @ x)[rows], rtol=1e-13, atol=0)


def test_gmres_dense_vs_solve(oracle):
    rng = np.random.default_rng(5)
    n = 120
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, rr, st = oracle.gmres_dense(A, b, restart=10, tol=1e-10, maxit=500)
    assert st == 0 and rr <= 1e-10
    assert np.linalg.norm(A @ x - b) <= 1.01e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(x)


def assemble(H, nc):
    """Dense matrix of A_H in original order, from the oracle's block data."""
    perm = H.perm()
    cl = H.clusters()
    blk, _, r = H.blocks()
    AH = np.zeros((3 * nc, 3 * nc), complex)
    for b in range(len(blk)):
        t, s = cl[blk[b]["tau"]], cl[blk[b]["sigma"]]
        ri = (3 * perm[t["begin"]:t["end"]][:, None] + np.arange(3)).ravel()
        ci = (3 * perm[s["begin"]:s["end"]][:, None] + np.arange(3)).ravel()
        data = H.block_data(b, blk, cl, r)
        AH[np.ix_(ri, ci)] = data if not blk[b]["admissible"] else data[0] @ data[1].conj().T
    return AH


def test_gmres_hmatrix_and_estimator(oracle):
    """GMRES on A_H reaches its tolerance (checked against the assembled A_H);
    Eq. est_direct: ||b - A x0||/||b|| <= (delta + delta_H,F ||x0||)/||b||."""
    nc = 600
    pts = inputs.fibonacci_sphere(nc)
    pb = oracle.problem(1, 2, 1, 4.0, "U")
    H = oracle.HMatrix(pb, pts, eps=1e-4, eta=3.0, leaf=32)
    b = inputs.random_rhs(3 * nc, seed=0)
    x0, it, rr, st = H.gmres(b, restart=50, tol=1e-6, maxit=3000)
    assert st == 0
    AH = assemble(H, nc)
    A = oracle.dense_matrix(pb, pts)
    bn = np.linalg.norm(b)
    delta = np.linalg.norm(b - AH @ x0)
    assert delta <= 1.01e-6 * bn
    dHF = np.linalg.norm(AH - A)
    true = np.linalg.norm(b - A @ x0) / bn
    assert true <= (delta + dHF * np.linalg.norm(x0)) / bn
    assert np.linalg.norm(AH @ np.ones(3 * nc) - H.matvec(np.ones(3 * nc))) < 1e-12 * np.linalg.norm(AH @ np.ones(3 * nc))


def test_uniform_weights_scale_the_offdiagonal(oracle):
    """A = K W_y (Sec. 4) with uniform w_j = c equals c times the unweighted
    matrix whose diagonal is diag/c: the tree, the partition, every ACA pivot
    and the truncation are scale invariant, so the H-matvecs agree to rounding."""
    nc, c = 900, 4 * np.pi / 900
    pts = inputs.fibonacci_sphere(nc)
    x = inputs.random_rhs(3 * nc, seed=6)
    Hw = oracle.HMatrix(oracle.problem(1, 2, 1, 4.0, "U", 1.0, np.full(nc, c)), pts, leaf=32)
    H1 = oracle.HMatrix(oracle.problem(1, 2, 1, 4.0, "U", 1.0 / c), pts, leaf=32)
    y1 = c * H1.matvec(x)
    assert np.linalg.norm(Hw.matvec(x) - y1) <= 1e-13 * np.linalg.norm(y1)
    assert np.array_equal(Hw.blocks()[1], H1.blocks()[1])


def test_weighted_hmatvec_vs_dense(oracle):
    nc = 1200
    pts, nrm = inputs.ellipsoid(nc)
    w = np.random.default_rng(8).uniform(0.5, 1.5, nc) * 4 * np.pi / nc
    for kern in ("U", "T"):
        pb = oracle.problem(1, 2, 1, 6.0, kern, 1.0, w)
        H = oracle.HMatrix(pb, pts, nrm, eps=1e-4, eta=3.0, leaf=32)
        x = inputs.random_rhs(3 * nc, seed=7)
        yd = oracle.dense_matrix(pb, pts, nrm) @ x
        assert np.linalg.norm(H.matvec(x) - yd) <= 3e-4 * np.linalg.norm(yd)


