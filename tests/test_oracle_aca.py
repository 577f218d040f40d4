"""Pins of the oracle's small linear algebra, vector ACA (Sec. 2.2 + Sec. 2.3)
and recompression (Sec. 3.2): library routines (numpy SVD/QR), exact
recovery of synthetic low-rank blocks, Eckart-Young (Sec. 2.2), the
Frobenius tail of the truncation, and the scalar-ACA failure on coplanar
clouds that motivates the sigma_3 pivot (Sec. 2.3)."""
import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_sv3_matches_numpy(oracle):
    rng = np.random.default_rng(0)
    for i in range(300):
        M = crandn(rng, 3, 3)
        if i % 3 == 1:       # rank 2
            M[:, 2] = M[:, 0] * (0.3 - 0.2j) + M[:, 1] * 1.7
        if i % 3 == 2:       # ill-conditioned
            M[:, 2] = M[:, 0] + 1e-9 * crandn(rng, 3)
        s = oracle.sv3(M)
        ref = np.linalg.svd(M, compute_uv=False)
        assert np.allclose(s, ref, rtol=0, atol=1e-14 * ref[0])


def test_svd_jacobi_matches_numpy(oracle):
    rng = np.random.default_rng(1)
    for M, N in ((20, 12), (7, 7), (40, 3), (30, 30)):
        A = crandn(rng, M, N)
        U, s, V = oracle.svd_jacobi(A)
        assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
        assert np.abs(U * s @ V.conj().T - A).max() < 1e-13 * s[0]
        assert np.abs(V.conj().T @ V - np.eye(N)).max() < 1e-13
        assert np.abs(U.conj().T @ U - np.eye(N)).max() < 1e-12


def test_qr(oracle):
    rng = np.random.default_rng(2)
    for M, N in ((50, 9), (9, 9), (300, 40)):
        A = crandn(rng, M, N)
        A[:, N // 2] = 0  # a zero column is allowed
        Q, R = oracle.qr(A)
        assert np.allclose(np.triu(R), R)
        assert np.abs(Q @ R - A).max() < 1e-13 * np.abs(A).max()
        assert np.abs(Q.conj().T @ Q - np.eye(N)).max() < 1e-13
        # full rank: |diag R| is unique, so it equals numpy's
        B = crandn(rng, M, N)
        Q, R = oracle.qr(B)
        Rn = np.linalg.qr(B, mode="r")
        assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rn)), rtol=1e-12)


@pytest.mark.parametrize("m,n,k", [(40, 30, 1), (50, 60, 4), (64, 64, 9), (20, 100, 6)])
def test_aca_exact_recovery(oracle, m, n, k):
    """A block of rank 3k is reproduced exactly after k rank-3 steps."""
    rng = np.random.default_rng(m * n + k)
    X = crandn(rng, 3 * m, 3 * k)
    Y = crandn(rng, 3 * n, 3 * k)
    A = X @ Y.conj().T
    U, V, piv = oracle.aca_dense(A, 1e-10)
    assert U.shape[1] == 3 * k
    assert np.linalg.norm(A - U @ V.conj().T) <= 1e-11 * np.linalg.norm(A)
    # pivots never repeat a row or a column
    assert len(set(piv[:, 0])) == len(piv) and len(set(piv[:, 1])) == len(piv)


def block_of(A, perm, t, s):
    ri = (3 * perm[t["begin"]:t["end"]][:, None] + np.arange(3)).ravel()
    ci = (3 * perm[s["begin"]:s["end"]][:, None] + np.arange(3)).ravel()
    return A[np.ix_(ri, ci)]


@pytest.fixture(scope="module")
def cfg1(oracle):
    pts = inputs.fibonacci_sphere(1536)
    pb = oracle.problem(1, 2, 1, 4.0, "U")
    A = oracle.dense_matrix(pb, pts)
    perm, cl = oracle.tree_build(pts, 32)
    blk = oracle.partition(cl, 3.0)
    return pb, pts, A, perm, cl, blk


def svd_rank_fro(s, eps):
    """Smallest r with sqrt(sum_{i>=r} s_i^2) <= eps ||s||."""
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    ok = np.nonzero(tail <= eps * np.linalg.norm(s))[0]
    return int(ok[0]) if len(ok) else len(s)


def test_aca_vs_dense_svd(oracle, cfg1):
    """Per admissible block of config 1: ACA error <= 3 eps (95th pct) and
    <= 10 eps (max) in the Frobenius norm; ACA rank is a multiple of 3 and
    not below the optimal (SVD) rank at the same eps (Eckart-Young)."""
    pb, pts, A, perm, cl, blk = cfg1
    eps = 1e-4
    adm = np.nonzero(blk["admissible"])[0]
    errs = []
    for b in adm[::6]:
        Ab = block_of(A, perm, cl[blk[b]["tau"]], cl[blk[b]["sigma"]])
        U, V, _ = oracle.aca_dense(Ab, eps)
        k = U.shape[1]
        assert k % 3 == 0
        s = np.linalg.svd(Ab, compute_uv=False)
        assert k >= svd_rank_fro(s, eps)
        errs.append(np.linalg.norm(Ab - U @ V.conj().T) / np.linalg.norm(Ab))
    errs = np.array(errs)
    assert np.percentile(errs, 95) <= 3 * eps and errs.max() <= 10 * eps


def test_recompression(oracle, cfg1):
    """Sec. 3.2: U'V'^H is the eps-truncated SVD of U V^H: same Frobenius tail
    rule, ||U'V'^H - UV^H||_F <= eps ||UV^H||_F, r' = SVD rank of U V^H, and the
    singular values of the core equal those of U V^H."""
    pb, pts, A, perm, cl, blk = cfg1
    eps = 1e-4
    adm = np.nonzero(blk["admissible"])[0]
    for b in adm[::25]:
        Ab = block_of(A, perm, cl[blk[b]["tau"]], cl[blk[b]["sigma"]])
        U, V, _ = oracle.aca_dense(Ab, eps)
        B = U @ V.conj().T
        U2, V2, s = oracle.recompress(U, V, eps)
        sref = np.linalg.svd(B, compute_uv=False)[:U.shape[1]]
        assert np.allclose(s, sref, rtol=1e-9, atol=1e-13 * sref[0])
        assert U2.shape[1] == svd_rank_fro(sref, eps)
        assert np.linalg.norm(B - U2 @ V2.conj().T) <= eps * np.linalg.norm(B) * (1 + 1e-9)
        # U' = Q_U P S^{1/2}: U'^H U' = S (diagonal), same for V'
        G = U2.conj().T @ U2
        assert np.allclose(G, np.diag(s[:U2.shape[1]]), atol=1e-10 * s[0])


def test_recompress_rank_zero(oracle):
    U = np.zeros((9, 3), complex)
    V = np.zeros((6, 3), complex)
    U2, V2, s = oracle.recompress(U, V, 1e-4)
    assert U2.shape[1] == 0


def scalar_aca(A, eps):
    """Plain scalar partially pivoted ACA, the six steps of Sec. 2.2 on the
    interleaved matrix (the approach Sec. 2.3 shows to fail)."""
    m, n = A.shape
    us, vs = [], []
    i = 0
    used_r, used_c = set(), set()
    nb2 = 0.0
    while len(us) < min(m, n):
        row = A[i].copy() - sum(u[i] * v.conj() for u, v in zip(us, vs))
        cand = [j for j in range(n) if j not in used_c]
        j = max(cand, key=lambda c: abs(row[c]))
        if abs(row[j]) < 1e-14:
            used_r.add(i)
            rest = [r for r in range(m) if r not in used_r]
            if not rest:
                break
            i = rest[0]
            continue
        col = A[:, j].copy() - sum(u * v[j].conj() for u, v in zip(us, vs))
        used_r.add(i)
        used_c.add(j)
        rest = [r for r in range(m) if r not in used_r]
        inext = max(rest, key=lambda r: abs(col[r])) if rest else None
        u, v = col / row[j], row.conj()
        nb2 += 2 * sum((uu.conj() @ u) * (v.conj() @ vv) for uu, vv in zip(us, vs)).real \
            + np.linalg.norm(u) ** 2 * np.linalg.norm(v) ** 2
        us.append(u)
        vs.append(v)
        if np.linalg.norm(u) * np.linalg.norm(v) <= eps * np.sqrt(nb2) or inext is None:
            break
        i = inext
    return np.array(us).T, np.array(vs).T


def test_scalar_aca_fails_on_plate_vector_aca_does_not(oracle):
    """Negative control (Sec. 2.3, E1): on the coplanar plate the matrix is
    reducible (Eq. FSplane), scalar partially pivoted ACA covers only part of
    it, while the vector ACA with the sigma_3 pivot reaches eps."""
    pts = inputs.plate(24)
    pb = oracle.problem(1, 2, 1, 5 * np.pi, "U")
    A = oracle.dense_matrix(pb, pts)
    perm, cl = oracle.tree_build(pts, 72)
    blk = oracle.partition(cl, 3.0)
    adm = [b for b in blk if b["admissible"]]
    b = max(adm, key=lambda b: (cl[b["tau"]]["end"] - cl[b["tau"]]["begin"]) *
            (cl[b["sigma"]]["end"] - cl[b["sigma"]]["begin"]))
    Ab = block_of(A, perm, cl[b["tau"]], cl[b["sigma"]])
    eps = 1e-4
    Us, Vs = scalar_aca(Ab, eps)
    err_scalar = np.linalg.norm(Ab - Us @ Vs.conj().T) / np.linalg.norm(Ab)
    U, V, _ = oracle.aca_dense(Ab, eps)
    err_vec = np.linalg.norm(Ab - U @ V.conj().T) / np.linalg.norm(Ab)
    assert err_vec <= 3 * eps
    assert err_scalar > 0.1
