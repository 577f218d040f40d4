"""H-LU factorisation and direct solver on the GPU (Sec. 3.2) against the
oracle's H-LU (same block tree, same four recursive steps, same eps_LU
recompression), the dense limit, the GPU's own operator, and the certificate
of Eq. est_direct (Sec. 3.3)."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs
from test_gpu_parity import oracle_export

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NC = 240
U32 = 2.0 ** -24  # unit roundoff of the FP32 storage


@pytest.fixture(scope="module")
def hm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1706_09384_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problem(oracle, kernel):
    pts = inputs.fibonacci_sphere(NC)
    nrm = inputs.sphere_normals(pts) if kernel == "T" else None
    w = np.full(NC, 4 * np.pi / NC)
    return pts, nrm, w, oracle.problem(1, 2, 1, 4.0, kernel, 1.0, w)


@pytest.mark.parametrize("kernel,eps_lu", [("U", 1e-7), ("T", 1e-7), ("U", 1e-5), ("T", 1e-5)])
def test_hlu_on_oracle_factors(hm, oracle, kernel, eps_lu):
    """The oracle's H-matrix imported on the GPU (FP32 storage) and factored
    there: the solve meets the oracle's H-LU solve to the truncation and the
    storage rounding, kappa (2 eps_LU + 4 u_32).  eps_LU = 1e-7 takes the
    Householder recompression, 1e-5 the Gram form."""
    pts, nrm, w, pb = problem(oracle, kernel)
    Ho = oracle.HMatrix(pb, pts, nrm, eps=1e-6, eta=3.0, leaf=16)
    perm, cl, blk, data = oracle_export(Ho)
    H = hm.HMatrix.import_(NC, perm, cl, blk, data)
    H.lu_factor(eps_lu)
    Fo = oracle.HLU(Ho, 3.0, eps_lu)
    assert Fo.status == 0
    A = oracle.dense_matrix(pb, pts, nrm)
    kappa = np.linalg.cond(A)
    b = inputs.random_rhs(3 * NC, 3, seed=5)
    x = H.lu_solve(cuda(b)).cpu().numpy()
    for j in range(3):
        xo = Fo.solve(b[:, j])
        err = np.linalg.norm(x[:, j] - xo) / np.linalg.norm(xo)
        assert err <= kappa * (2 * eps_lu + 4 * U32), (j, err, kappa)
    sec, entries, launches = H.lu_info()
    assert sec > 0 and entries > 0 and launches > 0
    assert abs(entries - Fo.stored) <= 0.1 * Fo.stored


@pytest.mark.parametrize("kernel", ["U", "T"])
def test_hlu_on_gpu_build(hm, oracle, kernel):
    """Factors of the GPU-built H-matrix: the residual with the GPU's own
    operator is at the truncation level, and the solution meets the oracle's
    H-LU solution within kappa times the two approximation errors."""
    pts, nrm, w, pb = problem(oracle, kernel)
    eps, eps_lu = 1e-6, 1e-6
    H = hm.HMatrix.build(pts, nrm, 1.0, 2.0, 1.0, 4.0, kernel, eps, 3.0, 16,
                         opts=hm.hm_opts_default(weights=w))
    H.lu_factor(eps_lu)
    Ho = oracle.HMatrix(pb, pts, nrm, eps=eps, eta=3.0, leaf=16)
    Fo = oracle.HLU(Ho, 3.0, eps_lu)
    kappa = np.linalg.cond(oracle.dense_matrix(pb, pts, nrm))
    b = inputs.random_rhs(3 * NC, 2, seed=6)
    x = H.lu_solve(cuda(b)).cpu().numpy()
    for j in range(2):
        r = b[:, j] - H.matvec(cuda(x[:, j])).cpu().numpy()
        assert np.linalg.norm(r) <= 20 * eps_lu * np.linalg.norm(b[:, j])
        xo = Fo.solve(b[:, j])
        err = np.linalg.norm(x[:, j] - xo) / np.linalg.norm(xo)
        assert err <= kappa * (4 * eps + 4 * eps_lu), (j, err, kappa)


def test_hlu_dense_limit(hm, oracle):
    """eta -> 0: every block dense; the factorisation is the LU without
    pivoting of the FP32-stored matrix and the solve meets the exact solve of
    A to kappa times the storage rounding."""
    pts, nrm, w, pb = problem(oracle, "U")
    H = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-6, 1e-9, 16,
                         opts=hm.hm_opts_default(weights=w))
    H.lu_factor(1e-8)
    assert H.stats()["lowrank_blocks"] == 0
    A = oracle.dense_matrix(pb, pts, None)
    b = inputs.random_rhs(3 * NC, seed=7)
    x = H.lu_solve(cuda(b)).cpu().numpy()
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 8 * np.linalg.cond(A) * U32 * np.linalg.norm(xs)


def test_hlu_certified_by_the_estimator(hm, oracle):
    """Eq. est_direct with the direct solution x0: ||b - A x0|| <= delta +
    delta_H,F ||x0||, delta = ||b - A_H x0|| (GPU product), delta_H,F from the
    every-pair evaluation on the GPU, A the exact dense matrix."""
    pts, nrm, w, pb = problem(oracle, "U")
    H = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-3, 3.0, 16,
                         opts=hm.hm_opts_default(weights=w))
    H.lu_factor(1e-4)
    b = inputs.random_rhs(3 * NC, seed=8)
    x0 = H.lu_solve(cuda(b)).cpu().numpy()
    delta = np.linalg.norm(b - H.matvec(cuda(x0)).cpu().numpy())
    dH, _ = H.estimate_error(0)
    A = oracle.dense_matrix(pb, pts, None)
    lhs = np.linalg.norm(b - A @ x0)
    assert lhs <= (delta + dH * np.linalg.norm(x0)) * (1 + 1e-9)


def test_hlu_needs_factors(hm):
    pts = inputs.fibonacci_sphere(NC)
    H = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-4, 3.0, 16)
    with pytest.raises(hm.HmError):
        H.lu_solve(cuda(inputs.random_rhs(3 * NC, seed=1)))
    with pytest.raises(hm.HmError):
        H.lu_factor(0.0)


def test_hlu_storage_rhs_and_refactor(hm, oracle):
    """The factorisation reads the FP32 copy of the stored operator, which a
    BF16-storage handle keeps as well: both handles give the same solution.
    Several right-hand sides at once equal the one-by-one solves; a second
    lu_factor replaces the factors (a smaller eps_LU, a smaller residual); the
    caller's output buffer is filled in place."""
    pts, nrm, w, pb = problem(oracle, "U")
    b = inputs.random_rhs(3 * NC, 3, seed=11)
    H32 = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-6, 3.0, 16,
                           opts=hm.hm_opts_default(weights=w))
    H16 = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-6, 3.0, 16,
                           opts=hm.hm_opts_default(weights=w, storage=hm.HM_STORE_BF16))
    H32.lu_factor(1e-4)
    H16.lu_factor(1e-4)
    x32 = H32.lu_solve(cuda(b)).cpu().numpy()
    x16 = H16.lu_solve(cuda(b)).cpu().numpy()
    assert np.linalg.norm(x16 - x32) <= 1e-12 * np.linalg.norm(x32)
    for j in range(3):
        xj = H32.lu_solve(cuda(b[:, j])).cpu().numpy()
        assert np.linalg.norm(xj - x32[:, j]) <= 1e-13 * np.linalg.norm(xj)
    res = lambda H, x, j: np.linalg.norm(b[:, j] - H.matvec(cuda(x)).cpu().numpy()) / np.linalg.norm(b[:, j])  # noqa: E731
    r4 = res(H32, x32[:, 0], 0)
    H32.lu_factor(1e-8)
    out = torch.empty(3 * NC, dtype=torch.complex128, device="cuda")
    ret = H32.lu_solve(cuda(b[:, 0]), x=out)
    assert ret.data_ptr() == out.data_ptr()
    r8 = res(H32, out.cpu().numpy(), 0)
    assert r8 < r4 and r8 <= 1e-5, (r4, r8)


def test_hlu_larger_cores(hm):
    """1 024 points, leaf 32: recompression cores above 128 columns (one-CTA
    Jacobi) and dense updates of large low-rank targets (randomized range
    finder) occur; the direct solution meets the GPU operator to the truncation
    level, and the factors stay below the operator's storage bound."""
    nc = 1024
    pts = inputs.fibonacci_sphere(nc)
    w = np.full(nc, 4 * np.pi / nc)
    H = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=w))
    H.lu_factor(1e-4)
    b = inputs.random_rhs(3 * nc, seed=21)
    x = H.lu_solve(cuda(b))
    r = np.linalg.norm(b - H.matvec(x).cpu().numpy()) / np.linalg.norm(b)
    assert np.isfinite(r) and r <= 1e-4, r
    _, entries, _ = H.lu_info()
    assert 0 < entries <= 1.5 * H.stats()["N_s"]
