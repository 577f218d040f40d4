"""Pins of the oracle's H-matrix between two clouds (targets x_i, sources y_j;
the paper's collocation points and integration points, Sec. 4): the same
recursion (Sec. 2.1), blocks and compression as the square case, which it must
reproduce exactly when both clouds are one; the partition of X x Y tiles the
index set; eta -> 0 is the dense product; distinct clouds are approximated to
the ACA tolerance; the U tensor is reciprocal, U(x, y) = U(y, x)^T."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs


def sphere(n, radius=1.0):
    return inputs.fibonacci_sphere(n, radius)


@pytest.mark.parametrize("kernel", ["U", "T"])
def test_one_cloud_reproduces_the_square_case(oracle, kernel):
    X = sphere(400)
    nrm = inputs.sphere_normals(X)
    w = np.full(len(X), 4 * np.pi / len(X))
    pb = oracle.problem(1, 2, 1, 4.0, kernel, 1.0, w)
    nrmY = nrm if kernel == "T" else None
    assert np.array_equal(oracle.dense_matrix2(pb, X, X, nrmY), oracle.dense_matrix(pb, X, nrmY))
    H1 = oracle.HMatrix(pb, X, nrmY, eps=1e-5, eta=3.0, leaf=16)
    H2 = oracle.HMatrix2(pb, X, X, nrmY, eps=1e-5, eta=3.0, leaf=16)
    b1, _, r1 = H1.blocks()
    b2, r2 = H2.blocks()
    assert np.array_equal(b1, b2) and np.array_equal(r1, r2)
    x = inputs.random_rhs(3 * len(X), seed=3)
    assert np.array_equal(H2.matvec(x), H1.matvec(x))


def test_partition_of_two_trees_tiles_the_index_set(oracle):
    X = sphere(700)
    Y, _ = inputs.cube_surface(500, seed=2)
    pb = oracle.problem(1, 2, 1, 4.0, "U")
    H = oracle.HMatrix2(pb, X, Y, eps=1e-4, eta=3.0, leaf=24)
    clX, clY = H.clusters()
    blk, _ = H.blocks()
    cover = np.zeros((len(X), len(Y)), np.int32)
    for b in blk:
        t, s = clX[b["tau"]], clY[b["sigma"]]
        cover[t["begin"]:t["end"], s["begin"]:s["end"]] += 1
        if b["admissible"]:
            dx = np.linalg.norm(t["hi"] - t["lo"])
            dy = np.linalg.norm(s["hi"] - s["lo"])
            gap = np.maximum(0.0, np.maximum(t["lo"] - s["hi"], s["lo"] - t["hi"]))
            assert min(dx, dy) < 3.0 * np.linalg.norm(gap)  # the box admissibility (Eq. admissibility_cond_bis)
        else:
            assert t["is_leaf"] or s["is_leaf"]
    assert cover.min() == 1 and cover.max() == 1  # every (x_i, y_j) in exactly one block


@pytest.mark.parametrize("kernel", ["U", "T"])
def test_eta_to_zero_is_the_dense_product(oracle, kernel):
    X = sphere(300)
    Y = sphere(240, 1.7)
    nrmY = inputs.sphere_normals(Y) if kernel == "T" else None
    pb = oracle.problem(1, 2, 1, 4.0, kernel)
    H = oracle.HMatrix2(pb, X, Y, nrmY, eps=1e-4, eta=1e-9, leaf=16)
    blk, _ = H.blocks()
    assert not blk["admissible"].any()
    A = oracle.dense_matrix2(pb, X, Y, nrmY)
    x = inputs.random_rhs(3 * len(Y), seed=4)
    y = A @ x
    assert np.linalg.norm(H.matvec(x) - y) <= 1e-13 * np.linalg.norm(y)


@pytest.mark.parametrize("kernel", ["U", "T"])
def test_distinct_clouds_within_the_tolerance(oracle, kernel):
    X = sphere(900)
    Y = sphere(700, 1.6)
    nrmY = inputs.sphere_normals(Y) if kernel == "T" else None
    w = np.full(len(Y), 4 * np.pi * 1.6 ** 2 / len(Y))
    eps = 1e-4
    pb = oracle.problem(1, 2, 1, 4.0, kernel, 1.0, w)
    H = oracle.HMatrix2(pb, X, Y, nrmY, eps=eps, eta=3.0, leaf=24)
    blk, r = H.blocks()
    assert blk["admissible"].any() and (r[blk["admissible"] == 1] > 0).all()
    A = oracle.dense_matrix2(pb, X, Y, nrmY)
    for seed in range(2):
        x = inputs.random_rhs(3 * len(Y), seed=seed)
        y = A @ x
        assert np.linalg.norm(H.matvec(x) - y) <= 3 * eps * np.linalg.norm(y)


def test_reciprocity_of_U(oracle):
    """U(x, y) = U(y, x)^T (the Green's tensor of the Navier equation is
    symmetric and even in x - y): the matrix from X to Y is the transpose of
    the one from Y to X."""
    X = sphere(120)
    Y, _ = inputs.cube_surface(90, seed=5)
    pb = oracle.problem(1, 2, 1, 4.0, "U")
    AXY = oracle.dense_matrix2(pb, X, Y)
    AYX = oracle.dense_matrix2(pb, Y, X)
    assert np.linalg.norm(AXY - AYX.T) <= 1e-14 * np.linalg.norm(AXY)
