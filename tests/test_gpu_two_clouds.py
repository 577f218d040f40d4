"""The H-matrix between two clouds on the GPU (hm_build2): targets x_i as rows,
sources y_j with normals and weights as columns (Sec. 4), a cluster tree per
cloud and the partition from the two roots (Sec. 2.1).  Against the oracle's
two-cloud H-matrix: the same trees and block set, the H-matvec within 1e-5,
and the dense product within 3 eps; the BF16 form within its rounding."""
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


def clouds(kind):
    X = inputs.fibonacci_sphere(1500)
    if kind == "sphere":
        Y = inputs.fibonacci_sphere(1800, radius=1.6)
        nY = inputs.sphere_normals(Y)
        w = np.full(len(Y), 4 * np.pi * 1.6 ** 2 / len(Y))
    else:
        Y, nY = inputs.cube_surface(2000, seed=5)
        Y = 3.0 * (Y - 0.5)  # the cube [-1.5, 1.5]^3 enclosing the unit sphere
        w = np.full(len(Y), 6 * 3.0 ** 2 / len(Y))
    return X, Y, nY, w


def block_set(blk, clX, clY):
    return {(int(clX[b["tau"]]["begin"]), int(clX[b["tau"]]["end"]), int(clY[b["sigma"]]["begin"]),
             int(clY[b["sigma"]]["end"]), int(b["admissible"])) for b in blk}


@pytest.mark.parametrize("kind,kern", [("sphere", "U"), ("sphere", "T"), ("cube", "T")])
def test_two_clouds_vs_oracle(hm, oracle, kind, kern):
    X, Y, nY, w = clouds(kind)
    nx, ny = len(X), len(Y)
    rho, lam, mu, om = inputs.material(5.0)
    pb = oracle.problem(rho, lam, mu, om, kern, 1.0, w)
    nn = nY if kern == "T" else None
    ref = oracle.HMatrix2(pb, X, Y, nn, eps=EPS, eta=3.0, leaf=32)
    H = hm.HMatrix.build2(X, Y, nn, rho, lam, mu, om, kern, EPS, 3.0, 32,
                          opts=hm.hm_opts_default(weights=w))
    assert H.stats()["n_targets"] == nx
    # trees and partition: the GPU's clusters are the targets' then the sources'
    perm, cl = H.tree()
    clX_o, clY_o = ref.clusters()
    cx = len(clX_o)
    clX, clY = cl[:cx].copy(), cl[cx:].copy()
    clY["begin"] -= nx
    clY["end"] -= nx
    assert len(cl) == cx + len(clY_o)
    assert np.array_equal(perm[:nx], oracle.tree_build(X, 32)[0])
    assert np.array_equal(perm[nx:] - nx, oracle.tree_build(Y, 32)[0])
    blk = H.blocks()
    blk_g = blk.copy()
    blk_g["sigma"] -= cx
    blk_o, _ = ref.blocks()
    assert block_set(blk_g, clX, clY) == block_set(blk_o, clX_o, clY_o)
    # products
    A = oracle.dense_matrix2(pb, X, Y, nn)
    for seed in (0, 1):
        x = inputs.random_rhs(3 * ny, seed=seed)
        y = H.matvec_sources(cuda(x)).cpu().numpy()
        yo, yd = ref.matvec(x), A @ x
        assert np.linalg.norm(y - yo) <= 1e-5 * np.linalg.norm(yo), np.linalg.norm(y - yo) / np.linalg.norm(yo)
        assert np.linalg.norm(y - yd) <= 3 * EPS * np.linalg.norm(yd)
    # the embedded square product: the source part of y stays zero
    xf = np.concatenate([inputs.random_rhs(3 * nx, seed=4), x])
    yf = H.matvec(cuda(xf)).cpu().numpy()
    assert not yf[3 * nx:].any()
    assert np.linalg.norm(yf[:3 * nx] - A @ x) <= 3 * EPS * np.linalg.norm(A @ x)
    # mixed form
    H16 = hm.HMatrix.build2(X, Y, nn, rho, lam, mu, om, kern, EPS, 3.0, 32,
                            opts=hm.hm_opts_default(weights=w, storage=hm.HM_STORE_BF16))
    y16 = H16.matvec_sources(cuda(x)).cpu().numpy()
    assert np.linalg.norm(y16 - yo) <= U16 * np.linalg.norm(yo)


def test_two_cloud_refusals(hm):
    X, Y, nY, w = clouds("sphere")
    H = hm.HMatrix.build2(X, Y, None, 1.0, 2.0, 1.0, 4.0, "U", EPS, 3.0, 32)
    b = cuda(inputs.random_rhs(3 * H.n_c, seed=0))
    _, _, _, st = H.gmres(b, restart=20, tol=1e-6, maxit=20, check=False)
    assert st == hm.HM_ERR_UNSUPPORTED
    Y2 = Y.copy()
    Y2[17] = X[5]
    with pytest.raises(hm.HmError) as e:
        hm.HMatrix.build2(X, Y2, None, 1.0, 2.0, 1.0, 4.0, "U", EPS, 3.0, 32)
    assert e.value.status == hm.HM_ERR_ARG and "17" in str(e.value)
    with pytest.raises(hm.HmError) as e:
        hm.HMatrix.build2(X, Y, None, 1.0, 2.0, 1.0, 4.0, "T", EPS, 3.0, 32)  # T needs normals
    assert e.value.status == hm.HM_ERR_ARG
