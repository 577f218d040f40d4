"""The allocation-free single-block ACA (hm_aca_block_noalloc) against the
allocating path.

Some callers cannot allocate device memory (their memory belongs to another
allocator, or a latency-sensitive loop must avoid cudaMalloc's implicit
synchronisation); they compress a block with this entry point, whose scratch
is a fixed device array inside the library.  Its result must equal what
hm_build computes for the same block.  With recompression switched off the
build stores the ACA factors themselves.  The build computes its residual
rows and columns in double-float arithmetic while this entry point keeps
them in FP64 (double-float copies of the factors would not fit the fixed
scratch), so near the stopping threshold the two may stop one rank-3 step
apart: ranks agree within 3 and the products U V^H within eps of each other.
The block is also compressed by the oracle's vector ACA (Sec. 2.2 with the
sigma_3 pivot of Sec. 2.3), whose rank and product it must match the same
way, and both stay within 10 eps of the exact block.  Two calls in a row
check that the shared scratch carries nothing from one call into the next.
"""
import numpy as np
import pytest

import oracle as O
from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-4
TOL = 1e-5  # the GPU-vs-oracle tolerance of the parity tests


@pytest.mark.parametrize("kern", ["U", "T"])
def test_noalloc_aca_matches_build(kern):
    assert torch.cuda.is_available()
    from paper_1706_09384_gb300 import build, hm
    build.build()
    nc = 3000
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    rho, lam, mu, om = inputs.material(8.0)
    k = hm.HM_KERNEL_U if kern == "U" else hm.HM_KERNEL_T
    H = hm.HMatrix.build(pts, nrm if kern == "T" else None, rho, lam, mu, om, kern, 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(recompress=0))
    perm, cl = H.tree()
    blk = H.blocks()
    adm = np.nonzero(blk["admissible"])[0]
    size = lambda b: cl[blk[b]["tau"]]["end"] - cl[blk[b]["tau"]]["begin"]  # noqa: E731
    largest = max(adm, key=size)
    picks = [largest, adm[len(adm) // 2], largest]  # two different blocks, then the first again
    for b in picks:
        t, s = cl[blk[b]["tau"]], cl[blk[b]["sigma"]]
        m, n = int(t["end"] - t["begin"]), int(s["end"] - s["begin"])
        x = torch.from_numpy(np.ascontiguousarray(pts[perm[t["begin"]:t["end"]]])).cuda()
        y = torch.from_numpy(np.ascontiguousarray(pts[perm[s["begin"]:s["end"]]])).cuda()
        ny = (torch.from_numpy(np.ascontiguousarray(nrm[perm[s["begin"]:s["end"]]])).cuda()
              if kern == "T" else None)
        cap = min(3 * min(m, n), 768)
        uv = torch.full(((3 * m + 3 * n) * cap,), complex(np.nan, np.nan), dtype=torch.complex128,
                        device="cuda")
        r = hm.hm_aca_block_noalloc(k, rho, lam, mu, om, x, y, ny, EPS, cap, uv)
        assert r % 3 == 0 and abs(r - blk[b]["rank_aca"]) <= 3
        w = uv.cpu().numpy()
        U = w[:3 * m * cap].reshape(cap, 3 * m).T[:, :r]
        V = w[3 * m * cap:].reshape(cap, 3 * n).T[:, :r]
        Ug, Vg = H.block_data(b, blk, cl)
        B, Bg = U @ V.conj().T, Ug @ Vg.conj().T
        # the exact block and the oracle's ACA of it
        pb = O.problem(rho, lam, mu, om, kern)
        A = O.dense_matrix2(pb, x.cpu().numpy(), y.cpu().numpy(),
                            ny.cpu().numpy() if ny is not None else None)
        Uo, Vo, _ = O.aca_dense(A, EPS)
        Bo = Uo @ Vo.conj().T
        nA = np.linalg.norm(A)
        assert abs(r - Uo.shape[1]) <= 3
        if r == blk[b]["rank_aca"]:
            assert np.linalg.norm(B - Bg) <= TOL * np.linalg.norm(Bg)
        else:
            assert np.linalg.norm(B - Bg) <= EPS * nA
        if r == Uo.shape[1]:
            assert np.linalg.norm(B - Bo) <= TOL * nA
        assert np.linalg.norm(B - A) <= 10 * EPS * nA


def test_noalloc_binding_rejects_bad_buffers_before_the_call():
    """An undersized, mistyped or strided buffer is refused by the binding
    before any launch (the library writes through raw device pointers)."""
    from paper_1706_09384_gb300 import build, hm
    build.build()
    x = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    y = torch.ones((8, 3), dtype=torch.float64, device="cuda")
    cap = 12
    need = (3 * 10 + 3 * 8) * cap
    cases = [
        (x, y, None, torch.zeros(need - 1, dtype=torch.complex128, device="cuda")),
        (x, y, None, torch.zeros(need, dtype=torch.complex64, device="cuda")),
        (x.t().contiguous().t(), y, None, torch.zeros(need, dtype=torch.complex128, device="cuda")),
        (x.float(), y, None, torch.zeros(need, dtype=torch.complex128, device="cuda")),
        (x, y, torch.ones((7, 3), dtype=torch.float64, device="cuda"),
         torch.zeros(need, dtype=torch.complex128, device="cuda")),
    ]
    before = hm.hm_kernel_launches()
    for xx, yy, nn, uv in cases:
        with pytest.raises(hm.HmError) as e:
            hm.hm_aca_block_noalloc(hm.HM_KERNEL_U, 1.0, 2.0, 1.0, 4.0, xx, yy, nn, EPS, cap, uv)
        assert e.value.status == hm.HM_ERR_ARG
    assert hm.hm_kernel_launches() == before


def test_noalloc_rejects_oversized_blocks():
    from paper_1706_09384_gb300 import build, hm
    build.build()
    big = hm.HM_NOALLOC_MAX_POINTS + 1
    x = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
    y = torch.ones((4, 3), dtype=torch.float64, device="cuda")
    uv = torch.zeros((3 * big + 12) * 12, dtype=torch.complex128, device="cuda")
    with pytest.raises(hm.HmError) as e:
        hm.hm_aca_block_noalloc(hm.HM_KERNEL_U, 1.0, 2.0, 1.0, 4.0, x, y, None, 1e-4, 12, uv)
    assert e.value.status == hm.HM_ERR_ARG
