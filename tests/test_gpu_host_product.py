"""hm_matvec_host: the product with host buffers (pinned or pageable, one or
several right-hand sides) gives the device product; overlapping buffers are
refused before any work is queued."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_host_product_mapped_and_copied(hm, storage):
    nc = 6000
    pts = inputs.fibonacci_sphere(nc)
    rho, lam, mu, om = inputs.material(10.0)
    st = hm.HM_STORE_BF16 if storage == "bf16" else hm.HM_STORE_FP32
    H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 64,
                         opts=hm.hm_opts_default(storage=st))
    x = inputs.random_rhs(3 * nc, seed=11)
    y_dev = H.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    # pageable numpy buffers
    assert rel(H.matvec_host(x), y_dev) <= 1e-6
    # pinned buffers
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.full_like(xh, complex(np.nan, np.nan)).pin_memory()
    for _ in range(2):
        assert hm.lib().hm_matvec_host(H.h, 1, xh.data_ptr(), yh.data_ptr(), None) == hm.HM_OK
        assert rel(yh.numpy(), y_dev) <= 1e-6
    # two right-hand sides (column-major)
    X = np.asfortranarray(np.stack([x, inputs.random_rhs(3 * nc, seed=12)], axis=1))
    Y_dev = H.matvec(torch.from_numpy(np.ascontiguousarray(X)).cuda()).cpu().numpy()
    Y = H.matvec_host(X)
    for c in range(2):
        assert rel(Y[:, c], Y_dev[:, c]) <= (2.0 ** -7 if storage == "bf16" else 1e-6)
    # overlapping host buffers are refused before any work is queued
    assert hm.lib().hm_matvec_host(H.h, 1, xh.data_ptr(), xh.data_ptr() + 16, None) == hm.HM_ERR_ARG
    H.free()
