"""The accurate product of the GMRES restarts (FP32-stored entries,
double-float sums): a solve to 1e-11, far below the FP32 summation noise of
the fast product, checked with an FP64 residual of the operator the GPU
stores (its blocks exported and assembled in numpy)."""
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


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_restart_residuals_reach_fp64_level(hm, storage):
    nc = 700
    pts = inputs.fibonacci_sphere(nc)
    rho, lam, mu, om = inputs.material(6.0)
    st = hm.HM_STORE_BF16 if storage == "bf16" else hm.HM_STORE_FP32
    H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=np.full(nc, 4 * np.pi / nc), storage=st))
    b = inputs.random_rhs(3 * nc, seed=4)
    x, it, rr, status = H.gmres(torch.from_numpy(b).cuda(), restart=30, tol=1e-11, maxit=600)
    assert status == 0 and rr <= 1e-11
    A = assemble(H, nc)  # the FP32-stored operator the restarts use, in FP64
    r = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert r <= 1.05e-11
    assert abs(r - rr) <= 1e-13
