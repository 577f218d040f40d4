"""Pins of the oracle's randomized SVD (the remark closing Sec. 2.3: blocks
whose 3x3 sub-blocks are all singular are compressed by the randomized SVD
instead of the vector ACA).  The range finder is pinned by exact recovery of
low-rank matrices, orthonormality, the certified error bound against the
optimal (numpy) SVD error and Eckart-Young; its test matrix by the published
splitmix64 outputs and the moments of the Box-Muller normals."""
import os

import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs

HERE = os.path.dirname(__file__)
EPS = 1e-4


def test_generator_matches_published_splitmix64(oracle):
    """The generator restates splitmix64: its outputs from state 1234567 are
    the published ones (tests/golden/splitmix64_seed1234567.txt)."""
    gold = [int(l) for l in open(os.path.join(HERE, "golden", "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    state = 1234567
    for g in gold:
        assert oracle.splitmix64(state) == g  # or_splitmix64 adds gamma, then mixes
        state = (state + gamma) & ((1 << 64) - 1)


def test_test_matrix_moments(oracle):
    """Box-Muller normals: mean 0, E|w|^2 = 1, independent real and imaginary
    parts of variance 1/2, no correlation between neighbouring counters."""
    z = oracle.gauss(oracle.rsvd_key(5, 77), range(40000))
    assert abs(z.mean()) < 0.02
    assert abs((abs(z) ** 2).mean() - 1.0) < 0.02
    assert abs(z.real.var() - 0.5) < 0.015 and abs(z.imag.var() - 0.5) < 0.015
    assert abs(np.mean(z.real * z.imag)) < 0.01
    assert abs(np.mean(z[1:] * np.conj(z[:-1]))) < 0.02
    # a different key draws a different matrix
    z2 = oracle.gauss(oracle.rsvd_key(6, 77), range(1000))
    assert np.max(np.abs(z2 - z[:1000])) > 1.0


def low_rank(m3, n3, k, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m3, k)) + 1j * rng.standard_normal((m3, k))
    Y = rng.standard_normal((n3, k)) + 1j * rng.standard_normal((n3, k))
    return X @ Y.conj().T


@pytest.mark.parametrize("k", [0, 1, 9, 40])
def test_exact_recovery_of_low_rank(oracle, k):
    """rank(A) = k < l: range(A Omega) = range(A) almost surely, so Q B = A to
    rounding, Q is orthonormal and the probes certify at the first l."""
    A = low_rank(96, 135, k, seed=k) if k else np.zeros((96, 135), np.complex128)
    U, V, ok = oracle.rsvd_dense(A, EPS, key=3)
    assert ok and U.shape[1] == 64
    assert np.linalg.norm(U.conj().T @ U - np.eye(64)) < 1e-12
    err = np.linalg.norm(U @ V.conj().T - A)
    assert err <= 1e-12 * max(np.linalg.norm(A), 1.0)


def test_full_rank_small_block_is_exact(oracle):
    """min(3m, 3n) <= 64: l takes the whole rank and Q Q^H A = A."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 48)) + 1j * rng.standard_normal((30, 48))
    U, V, ok = oracle.rsvd_dense(A, EPS, key=9)
    assert U.shape[1] == 30
    assert np.linalg.norm(U @ V.conj().T - A) <= 1e-12 * np.linalg.norm(A)


def test_samples_grow_until_certified(oracle):
    """A spectrum s_i = 0.95^i needs about 190 directions for eps / 2: l doubles
    from 64 until the probes certify, and the true range error ||A - Q Q^H A||_F
    is then below eps / 2 ||A||_F (it is at least the optimal tail of the SVD
    with l terms, Eckart-Young)."""
    rng = np.random.default_rng(11)
    n = 330
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = 0.95 ** np.arange(n)
    A = (Qa * s) @ Qb.conj().T
    U, V, ok = oracle.rsvd_dense(A, EPS, key=1)
    l = U.shape[1]
    assert ok and l == 256
    err = np.linalg.norm(A - U @ V.conj().T)
    assert err <= EPS / 2 * np.linalg.norm(A)
    assert err >= np.sqrt(np.sum(s[l:] ** 2)) * (1 - 1e-9)


def test_recompressed_rsvd_meets_eps_and_eckart_young(oracle):
    """Range finder, then the recompression of Sec. 3.2 with eps sqrt(3)/2: the
    factors meet eps against A, and their rank is at least the eps-rank of A's
    own SVD (Eckart-Young)."""
    rng = np.random.default_rng(5)
    n = 240
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((270, n)) + 1j * rng.standard_normal((270, n)))
    s = 0.9 ** np.arange(n)
    A = (Qa * s) @ Qb.conj().T
    U, V, ok = oracle.rsvd_dense(A, EPS, key=2)
    U2, V2, _ = oracle.recompress(U, V, EPS * np.sqrt(3) / 2)
    err = np.linalg.norm(A - U2 @ V2.conj().T)
    assert err <= EPS * np.linalg.norm(A)
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])  # tail[r] = ||s[r:]||
    r_opt = int(np.argmax(tail <= EPS * np.linalg.norm(s)))
    assert U2.shape[1] >= r_opt


def test_T_on_a_plane_is_compressed_by_rsvd(oracle):
    """Coplanar points with the plane's normal: every 3x3 candidate pivot of a
    same-plane block is singular, so every admissible block goes to the
    randomized SVD; each meets eps against its dense block and the H-matvec
    meets 3 eps of the dense product."""
    pts = inputs.plate(30)
    nrm = np.tile([0.0, 0.0, 1.0], (len(pts), 1))
    nc = len(pts)
    pb = oracle.problem(1, 2, 1, 6.0, "T", 1.0, np.full(nc, 4.0 / nc))
    H = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=32)
    blk, ra, r = H.blocks()
    meth = H.block_methods()
    adm = blk["admissible"] == 1
    assert adm.sum() > 0 and np.all(meth[adm] == 1)
    A = oracle.dense_matrix(pb, pts, nrm)
    perm, cl = H.perm(), H.clusters()
    for b in np.nonzero(adm)[0][:12]:
        t, s = cl[blk[b]["tau"]], cl[blk[b]["sigma"]]
        ri = (3 * perm[t["begin"]:t["end"]][:, None] + np.arange(3)).ravel()
        ci = (3 * perm[s["begin"]:s["end"]][:, None] + np.arange(3)).ravel()
        Ab = A[np.ix_(ri, ci)]
        U, V = H.block_data(b, blk, cl, r)
        assert np.linalg.norm(Ab - U @ V.conj().T) <= EPS * np.linalg.norm(Ab)
        assert r[b] <= min(Ab.shape)
    x = inputs.random_rhs(3 * nc, seed=2)
    yd = A @ x
    assert np.linalg.norm(H.matvec(x) - yd) <= 3 * EPS * np.linalg.norm(yd)


def test_T_on_cube_faces_mixes_aca_and_rsvd(oracle):
    """Cube surface, T kernel: same-face blocks go to the randomized SVD, the
    others keep their vector-ACA factors; the H-matvec meets 3 eps."""
    nc = 1500
    pts, nrm = inputs.cube_surface(nc, seed=2)
    pb = oracle.problem(1, 2, 1, 8.0, "T", 1.0, np.full(nc, 6.0 / nc))
    H = oracle.HMatrix(pb, pts, nrm, eps=EPS, eta=3.0, leaf=32)
    blk, _, _ = H.blocks()
    meth = H.block_methods()
    adm = blk["admissible"] == 1
    assert (meth[adm] == 1).sum() > 0 and (meth[adm] == 0).sum() > 0
    x = inputs.random_rhs(3 * nc, seed=3)
    yd = oracle.dense_matrix(pb, pts, nrm) @ x
    assert np.linalg.norm(H.matvec(x) - yd) <= 3 * EPS * np.linalg.norm(yd)


def test_acceptance_threshold_is_a_quarter_eps(oracle):
    """A spectrum 0.914^i: a Gaussian sketch of 128 columns leaves a range error
    of about 5e-5 ||A||_F (numpy QR of the sketch, several draws: 4.8e-5 to
    5.1e-5), between eps/4 and eps, so the probes must reject l = 128
    (threshold (eps/4)^2 on the mean probe residual) and accept l = 256."""
    rng = np.random.default_rng(21)
    n = 330
    rho = 0.914
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = rho ** np.arange(n)
    A = (Qa * s) @ Qb.conj().T
    U, V, ok = oracle.rsvd_dense(A, EPS, key=4)
    assert ok and U.shape[1] == 256
    assert np.linalg.norm(A - U @ V.conj().T) <= EPS / 2 * np.linalg.norm(A)
