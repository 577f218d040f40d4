"""The allocation-free single-block ACA (hm_aca_block_noalloc) against the
allocating path.

Some callers cannot allocate device memory (their memory belongs to another
allocator, or a latency-sensitive loop must avoid cudaMalloc's implicit
synchronisation); they compress a block with this entry point, whose scratch
is a fixed device array inside the library.  Its result must equal what
hm_build computes for the same block: with recompression switched off the
build stores the ACA factors themselves, so the ranks must be equal and the
products U V^H equal up to the FP32 rounding of the stored factors.  Two
calls in a row check that the shared scratch carries nothing from one call
into the next.
"""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
        r = hm.hm_aca_block_noalloc(k, rho, lam, mu, om, x, y, ny, 1e-4, cap, uv)
        assert r == blk[b]["rank_aca"]
        w = uv.cpu().numpy()
        U = w[:3 * m * cap].reshape(cap, 3 * m).T[:, :r]
        V = w[3 * m * cap:].reshape(cap, 3 * n).T[:, :r]
        Ug, Vg = H.block_data(b, blk, cl)
        B, Bg = U @ V.conj().T, Ug @ Vg.conj().T
        assert np.linalg.norm(B - Bg) <= TOL * np.linalg.norm(Bg)


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
