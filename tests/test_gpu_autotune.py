"""The autotuner of the H-matvec launch parameters (hm_opts.tune_cache): a
first build times the candidates on its own handle and records the fastest
in the cache file; a second build of the same workload class reads it back
without timing; malformed lines are ignored.  Tuned and default parameters
give the same product up to the FP32 rounding of a different summation
order (items regrouped; the phase-1 partial sums reach t through atomics in
an order the schedule decides)."""
import os

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


def workload(nc=12000):
    pts = inputs.fibonacci_sphere(nc)
    return pts, inputs.material(12.0), np.full(nc, 4 * np.pi / nc)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_sweep_then_cache(hm, tmp_path, storage):
    pts, (rho, lam, mu, om), w = workload()
    st = hm.HM_STORE_BF16 if storage == "bf16" else hm.HM_STORE_FP32
    cache = str(tmp_path / "tune.txt")
    H0 = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, 64,
                          opts=hm.hm_opts_default(weights=w, storage=st))
    assert H0.stats()["tune"]["source"] == "default"
    H1 = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, 64,
                          opts=hm.hm_opts_default(weights=w, storage=st, tune_cache=cache))
    t1 = H1.stats()["tune"]
    assert t1["source"] == "sweep" and len(t1["trials"]) == (3 if storage == "bf16" else 4)
    assert min(t["ms"] for t in t1["trials"]) == pytest.approx(t1["ms"], rel=1e-5)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and t1["key"] in lines[0] and ("storage=" + storage) in lines[0]
    H2 = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, 64,
                          opts=hm.hm_opts_default(weights=w, storage=st, tune_cache=cache))
    t2 = H2.stats()["tune"]
    assert t2["source"] == "cache" and t2["trials"] == []
    assert (t2["nstage"], t2["item_bytes"]) == (t1["nstage"], t1["item_bytes"])
    for seed in (0, 1):
        x = cuda(inputs.random_rhs(3 * len(pts), seed=seed))
        y0, y1, y2 = (H.matvec(x).cpu().numpy() for H in (H0, H1, H2))
        assert np.linalg.norm(y1 - y0) <= 1e-6 * np.linalg.norm(y0)
        assert np.linalg.norm(y2 - y0) <= 1e-6 * np.linalg.norm(y0)
    # the tuned handle's product graph and solver work
    b = cuda(inputs.random_rhs(3 * len(pts), seed=4))
    _, it, rr, status = H2.gmres(b, restart=50, tol=1e-6, maxit=500)
    assert status == 0 and rr <= 1e-6


def test_malformed_lines_are_ignored(hm, tmp_path):
    pts, (rho, lam, mu, om), w = workload(6000)
    cache = str(tmp_path / "tune.txt")
    other = "hm-tune-1 gpu=other;storage=fp32;ld=192;log2bytes=30 nstage=3 item_bytes=524288 ms=1.5"
    with open(cache, "w") as f:
        f.write("garbage line\nhm-tune-1 onlythree fields\n" + other + "\n"
                "hm-tune-1 gpu=x nstage=9 item_bytes=1 ms=-1\n")
    H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, 64,
                         opts=hm.hm_opts_default(weights=w, tune_cache=cache))
    t = H.stats()["tune"]
    assert t["source"] == "sweep"
    lines = open(cache).read().splitlines()
    assert other in lines and sum(t["key"] in s for s in lines) == 1


def test_unwritable_cache_is_an_argument_error(hm, tmp_path):
    pts, (rho, lam, mu, om), w = workload(3000)
    bad = str(tmp_path / "no_such_dir" / "tune.txt")
    with pytest.raises(hm.HmError) as e:
        hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", EPS, 3.0, 64,
                         opts=hm.hm_opts_default(weights=w, tune_cache=bad))
    assert e.value.status == hm.HM_ERR_ARG
    assert not os.path.exists(bad)
