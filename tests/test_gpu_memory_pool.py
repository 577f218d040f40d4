"""The build's workspaces (the ACA factors with their double-float copies, the
staged factors) come from the library's stream-ordered pool: after a build
and the handle's free the pool keeps them, a second build reuses them and
gives the same H-matrix, and hm_release_cached_memory returns them."""
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


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_build_workspace_pooled_reused_and_released(hm):
    nc = 8192
    pts = inputs.fibonacci_sphere(nc)
    rho, lam, mu, om = inputs.material(12.0)
    x = torch.from_numpy(inputs.random_rhs(3 * nc, seed=3)).cuda()

    def build():
        return hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 64)

    hm.hm_release_cached_memory()
    free0 = free_bytes()
    H1 = build()
    ws = H1.stats()["aca_workspace_peak_bytes"]
    assert ws > 256 << 20
    y1 = H1.matvec(x)
    b1 = H1.blocks()
    H1.free()
    held = free0 - free_bytes()
    assert held >= 0.9 * ws, (held, ws)  # the workspace stays reserved for reuse
    H2 = build()
    y2 = H2.matvec(x)
    b2 = H2.blocks()
    assert free0 - free_bytes() < held + H2.stats()["stored_bytes"] + (512 << 20)  # reused
    assert np.array_equal(b1["rank_aca"], b2["rank_aca"]) and np.array_equal(b1["rank"], b2["rank"])
    assert torch.linalg.norm(y1 - y2) <= 1e-6 * torch.linalg.norm(y1)
    H2.free()
    hm.hm_release_cached_memory()
    assert abs(free_bytes() - free0) < (256 << 20)
