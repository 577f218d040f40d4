"""The learned rank predictor: GPU inference and gradient against the FP64
oracle restatement, training lowers the loss, and the trained model changes
the build's workspace sizing but not the H-matrix."""
import os

import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rm():
    from paper_1706_09384_gb300 import build, hm, rank_model
    build.build()
    hm.lib()
    return rank_model


def data(n=600, seed=1):
    rng = np.random.default_rng(seed)
    F = np.column_stack([rng.uniform(0, 60, n), rng.uniform(0, 30, n), rng.uniform(0.3, 5, n),
                         rng.uniform(4, 12, n), rng.uniform(4, 12, n),
                         rng.choice([-3.0, -4.0, -5.0], n)]).astype(np.float32)
    T = np.log1p(0.2 * F[:, 0] + 0.1 * F[:, 3] + 2.0 / F[:, 2] - F[:, 5]).astype(np.float32)
    return F, T


def standardised(rm, F, T):
    P = rm.init_params(seed=3)
    P[0:6] = F.mean(0)
    P[6:12] = F.std(0)
    P[12], P[13] = T.mean(), T.std()
    return P


def test_forward_and_gradient_match_oracle(rm):
    from oracle import mlp
    F, T = data()
    P = standardised(rm, F, T)
    out = rm.predict(P, F)
    ref, _ = mlp.forward(P.astype(np.float64), F.astype(np.float64))
    assert np.abs(out - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    loss, g = rm.grad(P, F, T)
    lref, gref = mlp.loss_and_grad(P.astype(np.float64), F.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * lref
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_training_lowers_loss(rm):
    F, T = data(4000)
    P, losses = rm.train(F, T, steps=600, batch=512, lr=3e-3, seed=0)
    assert losses[-50:].mean() < 0.2 * losses[:50].mean()
    pred = rm.predict(P, F) * P[13] + P[12]
    assert np.corrcoef(pred, T)[0, 1] > 0.95


def test_trained_model_sizes_workspace_not_result(rm):
    """The committed model (trained on cube-surface builds) on an unseen sphere:
    the ACA ranks, the recompressed ranks and the product are unchanged, while
    the ACA workspace and, under a fixed workspace bound per batch, the number of
    ACA batches shrink."""
    from paper_1706_09384_gb300 import hm
    assert os.path.exists(rm.DEFAULT_WEIGHTS)
    P = rm.load()
    nc = 32768
    pts = inputs.fibonacci_sphere(nc)
    rho, lam, mu, om = inputs.material(12.0)
    o0, o1 = hm.hm_opts_default(), hm.hm_opts_default(rank_model=P)
    o0.workspace_bytes = o1.workspace_bytes = 8 << 30
    H0 = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 64, opts=o0)
    H1 = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 64, opts=o1)
    b0, b1 = H0.blocks(), H1.blocks()
    assert np.array_equal(b0["rank_aca"], b1["rank_aca"])
    assert np.array_equal(b0["rank"], b1["rank"])
    s0, s1 = H0.stats(), H1.stats()
    assert s0["rank_model"] == 0 and s1["rank_model"] == 1
    # the gain: ACA workspace (summed over batches) and the number of batches
    assert s1["aca_workspace_total_bytes"] <= 0.75 * s0["aca_workspace_total_bytes"]
    assert s1["aca_batches"] < s0["aca_batches"]
    x = torch.from_numpy(inputs.random_rhs(3 * nc, seed=0)).cuda()
    y0, y1 = H0.matvec(x).cpu().numpy(), H1.matvec(x).cpu().numpy()
    assert np.linalg.norm(y0 - y1) <= 1e-6 * np.linalg.norm(y0)
