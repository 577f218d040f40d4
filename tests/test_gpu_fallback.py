"""Blocks the vector ACA cannot pivot (rows whose 3x3 blocks are all
singular: the T kernel on coplanar points) are stored dense on the GPU exactly
where the oracle stores them dense; the H-matvec then meets the oracle and the
dense product."""
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


def keyed(blk, cl):
    return {(int(cl[b["tau"]]["begin"]), int(cl[b["tau"]]["end"]), int(cl[b["sigma"]]["begin"]),
             int(cl[b["sigma"]]["end"])): int(b["admissible"]) for b in blk}


@pytest.mark.parametrize("shape", ["plate", "cube"])
def test_fallback_matches_oracle(hm, oracle, shape):
    if shape == "plate":
        pts = inputs.plate(36)
        nrm = np.tile([0.0, 0.0, 1.0], (len(pts), 1))
        area = 4.0
    else:
        pts, nrm = inputs.cube_surface(2500, seed=4)
        area = 6.0
    nc = len(pts)
    rho, lam, mu, om = inputs.material(8.0)
    w = np.full(nc, area / nc)
    H = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, "T", 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=w))
    pb = oracle.problem(rho, lam, mu, om, "T", 1.0, w)
    Ho = oracle.HMatrix(pb, pts, nrm, eps=1e-4, eta=3.0, leaf=32)
    _, cl = H.tree()
    blk_o, _, _ = Ho.blocks()
    g, o = keyed(H.blocks(), cl), keyed(blk_o, Ho.clusters())
    assert g == o  # same partition, and the same blocks fell back to dense
    assert H.stats()["aca_dense_fallback"] > 0
    x = inputs.random_rhs(3 * nc, seed=1)
    y = H.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = Ho.matvec(x)
    assert np.linalg.norm(y - yo) <= 1e-5 * np.linalg.norm(yo)
    yd = oracle.dense_matrix(pb, pts, nrm) @ x
    assert np.linalg.norm(y - yd) <= 3e-4 * np.linalg.norm(yd)
