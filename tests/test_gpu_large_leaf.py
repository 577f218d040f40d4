"""Leaves above 64 points: the paper's own N_leaf = 100 (Sec. 7).  The tree
and the partition follow N_leaf; the stored blocks are cut along segments of
at most 64 points of each leaf.  Parity against the oracle built with the same
N_leaf (whose blocks are not cut at all) and the dense product, in both
storage forms and for the tensor-core block product."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-4
U16 = 2.0 ** -8


@pytest.fixture(scope="module")
def hm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1706_09384_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("kern", ["U", "T"])
def test_leaf100_tree_partition_and_products(hm, oracle, kern):
    nc, leaf = 3000, 100
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    rho, lam, mu, om = inputs.material(6.0)
    pb = oracle.problem(rho, lam, mu, om, kern)
    ref = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=leaf)
    nn = nrm if kern == "T" else None
    H = hm.HMatrix.build(pts, nn, rho, lam, mu, om, kern, EPS, 3.0, leaf)
    perm_g, cl_g = H.tree()
    assert np.array_equal(perm_g, ref.perm())
    sizes = cl_g["end"] - cl_g["begin"]
    assert sizes[cl_g["is_leaf"] == 1].max() > 64  # leaves above one storage segment
    A = oracle.dense_matrix(pb, pts, nrm)
    for seed in (0, 1):
        x = inputs.random_rhs(3 * nc, seed=seed)
        y = H.matvec(cuda(x)).cpu().numpy()
        yo, yd = ref.matvec(x), A @ x
        assert np.linalg.norm(y - yo) <= 1e-5 * np.linalg.norm(yo)
        assert np.linalg.norm(y - yd) <= 3 * EPS * np.linalg.norm(yd)
    # mixed form: one-vector product and the tensor-core block product
    H16 = hm.HMatrix.build(pts, nn, rho, lam, mu, om, kern, EPS, 3.0, leaf,
                           opts=hm.hm_opts_default(storage=hm.HM_STORE_BF16))
    x = inputs.random_rhs(3 * nc, seed=3)
    y = H16.matvec(cuda(x)).cpu().numpy()
    yo = ref.matvec(x)
    assert np.linalg.norm(y - yo) <= U16 * np.linalg.norm(yo)
    X = inputs.random_rhs(3 * nc, nrhs=hm.HM_NRHS_BLOCK, seed=4)
    Y = H16.matvec(cuda(np.asfortranarray(X))).cpu().numpy()
    for c in (0, 13, 31):
        yo = ref.matvec(np.ascontiguousarray(X[:, c]))
        assert np.linalg.norm(Y[:, c] - yo) <= 2 * U16 * np.linalg.norm(yo)


def test_leaf100_gmres_and_block_data(hm, oracle):
    """GMRES on the weighted leaf-100 system reaches 1e-6; a dense block read
    back from the cut storage equals the oracle's dense matrix."""
    nc, leaf = 2500, 100
    pts = inputs.fibonacci_sphere(nc)
    w = np.full(nc, 4 * np.pi / nc)
    rho, lam, mu, om = inputs.material(8.0)
    pb = oracle.problem(rho, lam, mu, om, "U", 1.0, w)
    H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, leaf,
                         opts=hm.hm_opts_default(weights=w))
    A = oracle.dense_matrix(pb, pts)
    perm, cl = H.tree()
    blk = H.blocks()
    for b in np.nonzero(blk["admissible"] == 0)[0][::11]:
        t, s = cl[blk[b]["tau"]], cl[blk[b]["sigma"]]
        ri = (3 * perm[t["begin"]:t["end"]][:, None] + np.arange(3)).ravel()
        ci = (3 * perm[s["begin"]:s["end"]][:, None] + np.arange(3)).ravel()
        Ab = A[np.ix_(ri, ci)]
        assert np.abs(H.block_data(b, blk, cl) - Ab).max() <= 1e-6 * np.abs(Ab).max()
    b = inputs.random_rhs(3 * nc, seed=2)
    x, it, rr, st = H.gmres(cuda(b), restart=50, tol=1e-6, maxit=500)
    assert st == 0 and rr <= 1e-6
    r = b - A @ x.cpu().numpy()
    assert np.linalg.norm(r) <= (1e-6 + 3 * EPS) * np.linalg.norm(b)
