"""Tensor-core product for blocks of 32 right-hand sides (BF16 storage): each
column of A_H X against the one-vector products and the FP64 oracle, ragged
leaves, a partial last block, the all-dense limit, and the T kernel with
plane-wave right-hand sides."""
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


def block_product(H, X):
    """A_H X for X of shape (n, nrhs) through one hm_matvec call."""
    return H.matvec(cuda(X)).cpu().numpy()


def colerr(Y, Yref):
    return np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)


def build_pair(hm, pts, nrm, ks, kern, leaf, eta=3.0):
    rho, lam, mu, om = inputs.material(ks)
    w = np.full(len(pts), 4 * np.pi / len(pts))
    H32 = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, kern, EPS, eta, leaf,
                           opts=hm.hm_opts_default(weights=w))
    H16 = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, kern, EPS, eta, leaf,
                           opts=hm.hm_opts_default(weights=w, storage=hm.HM_STORE_BF16))
    return H32, H16


@pytest.mark.parametrize("nrhs", [2, 32, 37])
def test_block_product_matches_one_vector_products(hm, nrhs):
    nc = 4000
    pts = inputs.fibonacci_sphere(nc)
    H32, H16 = build_pair(hm, pts, None, 8.0, "U", 32)
    X = inputs.random_rhs(3 * nc, nrhs, seed=5)
    Y = block_product(H16, X)
    Y32 = np.stack([H32.matvec(cuda(X[:, s])).cpu().numpy() for s in range(nrhs)], axis=1)
    Y16 = np.stack([H16.matvec(cuda(X[:, s])).cpu().numpy() for s in range(nrhs)], axis=1)
    # BF16 storage alone: 2^-8 (one-vector test); BF16 X and T add about as much
    assert colerr(Y, Y32).max() <= 2.0 ** -7
    assert colerr(Y, Y16).max() <= 2.0 ** -8
    # the columns are independent: a permuted block gives the permuted result
    perm = np.random.default_rng(0).permutation(nrhs)
    Yp = block_product(H16, X[:, perm])
    assert colerr(Yp, Y[:, perm]).max() <= 2.0 ** -8


def test_block_product_ragged_leaves_vs_oracle(hm, oracle):
    """Leaves of up to 20 points (rows 3..60: partial k-steps and m-tiles)."""
    nc = 2311
    pts, nrm = inputs.ellipsoid(nc)
    H32, H16 = build_pair(hm, pts, nrm, 6.0, "T", 20)
    X = inputs.random_rhs(3 * nc, 33, seed=7)
    Y = block_product(H16, X)
    rho, lam, mu, om = inputs.material(6.0)
    pb = oracle.problem(rho, lam, mu, om, "T", 1.0, np.full(nc, 4 * np.pi / nc))
    Ho = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=20)
    for s in (0, 17, 31, 32):
        yo = Ho.matvec(X[:, s])
        assert np.linalg.norm(Y[:, s] - yo) <= 2.0 ** -7 * np.linalg.norm(yo), s


def test_block_product_all_dense(hm):
    """eta -> 0: no admissible block, phase 2 only."""
    nc = 700
    pts = inputs.fibonacci_sphere(nc)
    H32, H16 = build_pair(hm, pts, None, 4.0, "U", 32, eta=1e-12)
    assert H16.blocks()["admissible"].sum() == 0
    X = inputs.random_rhs(3 * nc, 32, seed=1)
    Y = block_product(H16, X)
    Y32 = np.stack([H32.matvec(cuda(X[:, s])).cpu().numpy() for s in range(32)], axis=1)
    assert colerr(Y, Y32).max() <= 2.0 ** -7


def test_block_product_plane_waves_T(hm, oracle):
    """T kernel with outward normals, 32 plane-wave right-hand sides (P and S
    waves alternating): every column against the oracle's H-matvec."""
    nc = 3000
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    ks = 8.0
    H32, H16 = build_pair(hm, pts, nrm, ks, "T", 32)
    X = inputs.plane_wave_rhs(pts, ks / 2, ks, 32, seed=0)
    Y = block_product(H16, X)
    rho, lam, mu, om = inputs.material(ks)
    pb = oracle.problem(rho, lam, mu, om, "T", 1.0, np.full(nc, 4 * np.pi / nc))
    Ho = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=32)
    Yo = np.stack([Ho.matvec(X[:, s]) for s in range(32)], axis=1)
    assert colerr(Y, Yo).max() <= 2.0 ** -7


def test_block_profile_reports_kernels(hm):
    nc = 4000
    pts = inputs.fibonacci_sphere(nc)
    _, H16 = build_pair(hm, pts, None, 8.0, "U", 32)
    before = hm.hm_kernel_launches()
    p = H16.profile_matvec_multi(3)
    assert hm.hm_kernel_launches() - before >= 4 * 4
    assert p["bytes"] > H16.stats()["stored_bytes"]
    assert all(v > 0 for v in p["ms"].values())


@pytest.mark.parametrize("storage", ["bf16", "fp32"])
def test_gmres_multi_matches_single(hm, storage):
    """Lockstep GMRES for 33 columns (two blocks of the tensor-core product with
    BF16 storage; one product per column with FP32 storage): every column
    converges and agrees with the one-column solver on FP32 storage."""
    nc = 4000
    pts = inputs.fibonacci_sphere(nc)
    H32, H16 = build_pair(hm, pts, None, 8.0, "U", 32)
    H = H16 if storage == "bf16" else H32
    nrhs = 33 if storage == "bf16" else 3
    B = inputs.random_rhs(3 * nc, nrhs, seed=11)
    X, it, rr, st = H.gmres_multi(cuda(B), restart=50, tol=1e-6, maxit=500)
    assert st == 0 and (rr <= 1e-6).all() and (it > 0).all()
    X = X.cpu().numpy()
    for s in sorted({0, min(5, nrhs - 1), nrhs - 1}):
        xs, its, rrs, sts = H32.gmres(cuda(B[:, s]), restart=50, tol=1e-6, maxit=500)
        xs = xs.cpu().numpy()
        assert sts == 0
        assert np.linalg.norm(X[:, s] - xs) <= 1e-5 * np.linalg.norm(xs), s
        r = B[:, s] - H32.matvec(cuda(X[:, s])).cpu().numpy()
        assert np.linalg.norm(r) <= 2e-6 * np.linalg.norm(B[:, s])


def test_gmres_multi_plane_waves_T_vs_oracle(hm, oracle):
    """Scaled-down precision + multi-RHS workload: T kernel with outward
    normals, 32 plane-wave right-hand sides, BF16 tensor-core products inside
    GMRES with FP64 refinement; solutions against the FP64 oracle's GMRES on its
    own H-matrix, per right-hand side."""
    nc = 2500
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    ks = 8.0
    _, H16 = build_pair(hm, pts, nrm, ks, "T", 32)
    B = inputs.plane_wave_rhs(pts, ks / 2, ks, 32, seed=0)
    X, it, rr, st = H16.gmres_multi(cuda(B), restart=50, tol=1e-8, maxit=1000)
    assert st == 0 and (rr <= 1e-8).all()
    X = X.cpu().numpy()
    rho, lam, mu, om = inputs.material(ks)
    pb = oracle.problem(rho, lam, mu, om, "T", 1.0, np.full(nc, 4 * np.pi / nc))
    Ho = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=32)
    for s in (0, 1, 30, 31):
        xo, ito, rro, sto = Ho.gmres(B[:, s], restart=50, tol=1e-10, maxit=2000)
        assert sto == 0
        # the GPU operator carries FP32-stored entries: relative distance ~1e-7 x condition
        assert np.linalg.norm(X[:, s] - xo) <= 1e-5 * np.linalg.norm(xo), s
