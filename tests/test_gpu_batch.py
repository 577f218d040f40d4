"""Batch build of independent problems (one ACA / recompression launch serves
the blocks of every problem): each handle equals the H-matrix built alone,
mixed U / T kernels, shapes, sizes, wavenumbers and weights; a T problem of
the batch against the oracle; GMRES on every handle."""
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
    specs = [("sphere", 3000, "U", 4.0, True), ("cube", 2000, "T", 8.0, False),
             ("ellipsoid", 2500, "U", 6.0, True), ("sphere", 1500, "T", 3.0, True),
             ("cube", 4000, "U", 10.0, False)]
    for shape, nc, kern, ks, weighted in specs:
        if shape == "sphere":
            pts = inputs.fibonacci_sphere(nc)
            nrm = inputs.sphere_normals(pts)
        elif shape == "cube":
            pts, nrm = inputs.cube_surface(nc, seed=nc)
        else:
            pts, nrm = inputs.ellipsoid(nc)
        rho, lam, mu, om = inputs.material(ks)
        out.append(dict(points=pts, normals=nrm if kern == "T" else None, rho=rho, lam=lam, mu=mu,
                        omega=om, kernel=kern, eta=3.0, leaf_size=32,
                        weights=np.full(nc, 4 * np.pi / nc) if weighted else None))
    return out


@pytest.fixture(scope="module")
def batch(hm):
    P = problems()
    return P, hm.HMatrix.build_batch(P, eps=EPS)


def test_batch_equals_single_builds(hm, batch):
    P, Hb = batch
    for q, p in enumerate(P):
        Hs = hm.HMatrix.build(p["points"], p["normals"], p["rho"], p["lam"], p["mu"], p["omega"],
                              p["kernel"], EPS, p["eta"], p["leaf_size"],
                              opts=hm.hm_opts_default(weights=p["weights"]))
        bb, bs = Hb[q].blocks(), Hs.blocks()
        assert np.array_equal(bb, bs), q
        assert Hb[q].stats()["batch_problems"] == len(P)
        n = 3 * len(p["points"])
        x = cuda(inputs.random_rhs(n, seed=q))
        yb, ys = Hb[q].matvec(x).cpu().numpy(), Hs.matvec(x).cpu().numpy()
        assert np.linalg.norm(yb - ys) <= 1e-6 * np.linalg.norm(ys), q
        Hs.free()


def test_batch_T_problem_vs_oracle(hm, oracle, batch):
    P, Hb = batch
    q = 1
    p = P[q]
    pb = oracle.problem(p["rho"], p["lam"], p["mu"], p["omega"], p["kernel"], 1.0, p["weights"])
    Ho = oracle.HMatrix(pb, p["points"], p["normals"], eps=EPS, eta=3.0, leaf=32)
    x = inputs.random_rhs(3 * len(p["points"]), seed=9)
    yo = Ho.matvec(x)
    y = Hb[q].matvec(cuda(x)).cpu().numpy()
    assert np.linalg.norm(y - yo) <= 1e-5 * np.linalg.norm(yo)


def test_batch_gmres_each(hm, batch):
    P, Hb = batch
    for q, p in enumerate(P):
        if p["weights"] is None:
            continue  # the unweighted systems are the badly scaled ones (see the readings)
        b = cuda(inputs.random_rhs(3 * len(p["points"]), seed=20 + q))
        x, it, rr, st = Hb[q].gmres(b, restart=100, tol=1e-6, maxit=2000)
        assert st == 0 and rr <= 1e-6, q


def test_batch_rejects_bad_problem(hm):
    P = problems()[:2]
    P[1] = dict(P[1], normals=None)  # T kernel without normals
    with pytest.raises(hm.HmError):
        hm.HMatrix.build_batch(P, eps=EPS)
