"""Approximation error of the stored H-matrix for the a-posteriori bound of
Sec. 3.3 (Eq. est_direct): every-pair evaluation against the oracle's dense
matrix and the GPU's exported blocks, the sampled estimate against it, and
the bound itself for a GMRES solution."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1706_09384_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def assemble(H, nc):
    perm, cl = H.tree()
    blk = H.blocks()
    A = np.zeros((3 * nc, 3 * nc), complex)
    for b in range(len(blk)):
        t, s = cl[blk[b]["tau"]], cl[blk[b]["sigma"]]
        ri = (3 * perm[t["begin"]:t["end"]][:, None] + np.arange(3)).ravel()
        ci = (3 * perm[s["begin"]:s["end"]][:, None] + np.arange(3)).ravel()
        d = H.block_data(b, blk, cl)
        A[np.ix_(ri, ci)] = d[0] @ d[1].conj().T if blk[b]["admissible"] else d
    return A


@pytest.mark.parametrize("kern", ["U", "T"])
def test_every_pair_matches_dense(hm, oracle, kern):
    nc = 1000
    pts, nrm = inputs.ellipsoid(nc)
    rho, lam, mu, om = inputs.material(8.0)
    w = np.full(nc, 5.46 / nc)
    H = hm.HMatrix.build(pts, nrm if kern == "T" else None, rho, lam, mu, om, kern, 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=w))
    A = oracle.dense_matrix(oracle.problem(rho, lam, mu, om, kern, 1.0, w), pts,
                            nrm if kern == "T" else None)
    dF = np.linalg.norm(A - assemble(H, nc))
    aF = np.linalg.norm(A)
    d, a = H.estimate_error(0)
    assert abs(a - aF) <= 1e-9 * aF
    assert abs(d - dF) <= 1e-6 * dF
    assert d <= 3e-2 * a  # the blocks' eps-accuracy, summed in Frobenius norm
    # the unbiased sampled estimate of the squared norms, 20 % of the pairs
    ds, as_ = H.estimate_error(200000, seed=5)
    assert abs(as_ - aF) <= 0.05 * aF
    assert abs(ds - dF) <= 0.25 * dF


def test_a_posteriori_bound(hm, oracle):
    """Eq. est_direct: ||b - A x|| <= ||b - A_H x|| + ||A - A_H||_F ||x||."""
    nc = 900
    pts = inputs.fibonacci_sphere(nc)
    rho, lam, mu, om = inputs.material(6.0)
    w = np.full(nc, 4 * np.pi / nc)
    H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=w))
    b = inputs.random_rhs(3 * nc, seed=3)
    x, it, rr, st = H.gmres(torch.from_numpy(b).cuda(), restart=50, tol=1e-8, maxit=500)
    assert st == 0
    x = x.cpu().numpy()
    A = oracle.dense_matrix(oracle.problem(rho, lam, mu, om, "U", 1.0, w), pts)
    d, _ = H.estimate_error(0)
    true = np.linalg.norm(b - A @ x)
    assert true <= rr * np.linalg.norm(b) + d * np.linalg.norm(x)
    assert true >= 0.5 * rr * np.linalg.norm(b)  # and it is not vacuous below the solver
