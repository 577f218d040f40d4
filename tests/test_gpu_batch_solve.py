"""Independent problems joined into one block-diagonal operator
(hm_batch_join) and solved by lockstep GMRES, one per problem, with one
product of the joined operator per Arnoldi step (hm_gmres_batch).  The
joined product equals the problems' own products; every problem converges to
the tolerance on its own residual, and its solution agrees with a solve of
that problem alone."""
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


def problems():
    out = []
    for q, (nc, shape, ks, kern) in enumerate([(2500, "sphere", 6.0, "U"), (4000, "ellipsoid", 9.0, "T"),
                                                (1500, "cube", 3.0, "U"), (3000, "sphere", 12.0, "T")]):
        if shape == "sphere":
            pts = inputs.fibonacci_sphere(nc)
            nrm = inputs.sphere_normals(pts)
        elif shape == "cube":
            pts, nrm = inputs.cube_surface(nc, seed=q)
        else:
            pts, nrm = inputs.ellipsoid(nc)
        rho, lam, mu, om = inputs.material(ks)
        area = inputs.SURFACE_AREA[shape]
        out.append(dict(points=pts, normals=nrm if kern == "T" else None, rho=rho, lam=lam, mu=mu,
                        omega=om, kernel=kern, weights=np.full(nc, area / nc), eta=3.0, leaf_size=32))
    return out


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_join_product_and_lockstep_solve(hm, storage):
    P = problems()
    st = hm.HM_STORE_BF16 if storage == "bf16" else hm.HM_STORE_FP32
    Hs = hm.HMatrix.build_batch(P, eps=EPS, opts=hm.hm_opts_default(storage=st))
    J = hm.HMatrix.join(Hs)
    sizes = [3 * len(p["points"]) for p in P]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert J.n_c == sum(len(p["points"]) for p in P)
    # the joined product is the problems' products, concatenated
    x = inputs.random_rhs(int(offs[-1]), seed=1)
    y = J.matvec(cuda(x)).cpu().numpy()
    for q, H in enumerate(Hs):
        yq = H.matvec(cuda(x[offs[q]:offs[q + 1]])).cpu().numpy()
        assert np.linalg.norm(y[offs[q]:offs[q + 1]] - yq) <= 1e-6 * np.linalg.norm(yq), q
    # lockstep GMRES, one per problem, against solves of each problem alone
    b = inputs.random_rhs(int(offs[-1]), seed=2)
    X, it, rr, status = J.gmres_batch(cuda(b), restart=50, tol=1e-6, maxit=600)
    assert status == 0 and (rr <= 1e-6).all(), (it, rr)
    gm = J.stats()["gmres_last"]
    assert gm["fast_products"] == it.max()  # one product of the joined operator per step
    X = X.cpu().numpy()
    for q, H in enumerate(Hs):
        bq = b[offs[q]:offs[q + 1]]
        xq, itq, rrq, stq = H.gmres(cuda(bq), restart=50, tol=1e-6, maxit=600)
        assert stq == 0
        xq = xq.cpu().numpy()
        # both solutions solve A_q x = b_q to 1e-6; they agree to the conditioning of A_q
        assert np.linalg.norm(X[offs[q]:offs[q + 1]] - xq) <= 1e-4 * np.linalg.norm(xq), q
        if storage == "fp32":  # a BF16 handle's own product carries its 2^-8 rounding
            r = bq - H.matvec(cuda(X[offs[q]:offs[q + 1]])).cpu().numpy()
            assert np.linalg.norm(r) <= 2e-6 * np.linalg.norm(bq), q
    with pytest.raises(hm.HmError) as e:
        J.estimate_error(nsample=100)
    assert e.value.status == hm.HM_ERR_UNSUPPORTED
    with pytest.raises(hm.HmError) as e:
        hm.HMatrix.join([J, Hs[0]])
    assert e.value.status == hm.HM_ERR_ARG
