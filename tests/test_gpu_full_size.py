"""Full-size workloads checked on sampled outputs against the FP64 oracle
(dense rows of the exact operator, computed one by one): the precision +
multi-RHS workload (131 072-point sphere, T kernel, 32 plane waves, BF16
tensor-core products inside lockstep GMRES with FP64-grade refinement) and the
16-problem batch build."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-4


@pytest.fixture(scope="module")
def hm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1706_09384_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_plane_waves_T_131072(hm, oracle):
    nc, ks = 131072, 16.0
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    rho, lam, mu, om = inputs.material(ks)
    w = np.full(nc, 4 * np.pi / nc)
    H = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, "T", EPS, 3.0, 64,
                         opts=hm.hm_opts_default(weights=w, storage=hm.HM_STORE_BF16))
    B = inputs.plane_wave_rhs(pts, ks / 2, ks, 32, seed=0)
    X, it, rr, st = H.gmres_multi(cuda(B), restart=100, tol=1e-6, maxit=2000)
    assert st == 0 and rr.max() <= 1e-6
    X = X.cpu().numpy()
    H.free()
    pb = oracle.problem(rho, lam, mu, om, "T", 1.0, w)
    rows = np.random.default_rng(1).choice(3 * nc, 96, replace=False)
    for s in range(0, 32, 4):  # P and S waves
        Ax = oracle.dense_rows_matvec(pb, pts, nrm, rows, X[:, s])
        # residual of the exact operator: GMRES tolerance + the H-matrix error
        assert np.linalg.norm(B[rows, s] - Ax) <= 3 * EPS * np.linalg.norm(B[rows, s]), s


def test_batch_16_problems(hm, oracle):
    P = inputs.batch_problems(16, seed=0)
    Hs = hm.HMatrix.build_batch([dict(p, eta=3.0, leaf_size=64) for p in P], eps=EPS)
    try:
        for q, (p, H) in enumerate(zip(P, Hs)):
            assert H.stats()["batch_problems"] == 16
            n = 3 * len(p["points"])
            x = inputs.random_rhs(n, seed=q)
            y = H.matvec(cuda(x)).cpu().numpy()
            pb = oracle.problem(p["rho"], p["lam"], p["mu"], p["omega"], p["kernel"], 1.0,
                                p["weights"])
            rows = np.random.default_rng(q).choice(n, 48, replace=False)
            yo = oracle.dense_rows_matvec(pb, p["points"], p["normals"], rows, x)
            # U: the 3 eps of the configs; T: the paper reports 19-27 eps for its T matrices
            tol = 3 * EPS if p["kernel"] == "U" else 30 * EPS
            assert np.linalg.norm(y[rows] - yo) <= tol * np.linalg.norm(yo), q
            if p["kernel"] == "U":
                b = cuda(inputs.random_rhs(n, seed=100 + q))
                _, it, rr, st = H.gmres(b, restart=100, tol=1e-6, maxit=500)
                assert st == 0 and rr <= 1e-6, q
    finally:
        for H in Hs:
            H.free()
