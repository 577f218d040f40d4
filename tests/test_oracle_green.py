"""Pins of the oracle's Green's tensors (Eq. elasto_U, Eq. elasto_T) against
what the mathematics fixes: symmetry, the Navier equation (Eq. NE) by finite
differences, the static Kelvin limit, the far field, the coplanar zero
pattern (Eq. FSplane), the traction operator applied by finite differences,
and a 50-digit evaluation of the radial functions."""
import math
import os

import mpmath as mp
import numpy as np
import pytest

MATS = [  # (rho, lam, mu, omega)
    (1.0, 2.0, 1.0, 4.0),     # config-1 material, k_s = 4, k_p = 2 (nu = 1/3)
    (1.0, 2.0, 1.0, 16.0),    # k_s = 16
    (2.5, 0.7, 1.3, 3.0),     # a generic material
]


def rnd_pair(rng, r):
    x = rng.standard_normal(3)
    d = rng.standard_normal(3)
    d *= r / np.linalg.norm(d)
    return x, x - d


def test_symmetry(oracle):
    """U(x,y) = U(y,x) = U(x,y)^T (U depends on x - y through even functions)."""
    rng = np.random.default_rng(1)
    for rho, lam, mu, om in MATS:
        pb = oracle.problem(rho, lam, mu, om, "U")
        for r in (0.01, 0.3, 2.0, 7.0):
            x, y = rnd_pair(rng, r)
            G = oracle.green(pb, x, y)
            assert np.abs(G - oracle.green(pb, y, x)).max() <= 1e-15 * np.abs(G).max()
            assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()


# 4th-order central stencils
C1 = {-2: 1 / 12, -1: -2 / 3, 1: 2 / 3, 2: -1 / 12}          # first derivative
C2 = {-2: -1 / 12, -1: 4 / 3, 0: -5 / 2, 1: 4 / 3, 2: -1 / 12}  # second derivative


def d2(f, x, a, b, h):
    """4th-order FD of d^2 f / dx_a dx_b (f returns an array)."""
    if a == b:
        return sum(c * f(x + i * h * np.eye(3)[a]) for i, c in C2.items()) / h ** 2
    return sum(ci * cj * f(x + i * h * np.eye(3)[a] + j * h * np.eye(3)[b])
               for i, ci in C1.items() for j, cj in C1.items()) / h ** 2


@pytest.mark.parametrize("mat", MATS)
def test_navier_equation(oracle, mat):
    """Each column u = U(., y) e_b solves mu Lap u + (lam+mu) grad div u + rho w^2 u = 0
    (Eq. NE with sigma(u) = lam div u I + 2 mu eps(u)) away from the source."""
    rho, lam, mu, om = mat
    pb = oracle.problem(rho, lam, mu, om, "U")
    rng = np.random.default_rng(2)
    for r in (0.2, 0.9, 2.5):
        x0, y = rnd_pair(rng, r)
        h = 1e-3 * r
        f = lambda x: oracle.green(pb, x, y)  # noqa: E731
        H = {(a, b): d2(f, x0, a, b, h) for a in range(3) for b in range(a, 3)}
        Hs = lambda a, b: H[(min(a, b), max(a, b))]  # noqa: E731
        U = f(x0)
        # res[alpha, beta] = mu sum_g d_gg U_ab + (lam+mu) sum_g d_a d_g U_gb + rho w^2 U_ab
        res = np.zeros((3, 3), complex)
        for al in range(3):
            for be in range(3):
                lap = sum(Hs(g, g)[al, be] for g in range(3))
                gd = sum(Hs(al, g)[g, be] for g in range(3))
                res[al, be] = mu * lap + (lam + mu) * gd + rho * om ** 2 * U[al, be]
        scale = rho * om ** 2 * np.abs(U).max() + mu * np.abs(Hs(0, 0)).max()
        assert np.abs(res).max() <= 1e-6 * scale, (r, np.abs(res).max() / scale)


def kelvin(lam, mu, x, y):
    d = x - y
    r = np.linalg.norm(d)
    rh = d / r
    return ((lam + 3 * mu) * np.eye(3) + (lam + mu) * np.outer(rh, rh)) / (8 * math.pi * mu * (lam + 2 * mu) * r)


def test_kelvin_limit(oracle):
    """w -> 0: U -> Kelvin's static tensor plus the constant imaginary term
    i w (2/c_s^3 + 1/c_p^3)/(12 pi rho) I; the remainder is O((k r)^2)."""
    rho, lam, mu = 1.7, 2.2, 0.9
    x, y = np.array([0.3, -0.2, 0.1]), np.array([-0.4, 0.5, 0.35])
    r = np.linalg.norm(x - y)
    K = kelvin(lam, mu, x, y)
    errs = []
    for om in (1e-2, 1e-3):
        ks, kp = om * math.sqrt(rho / mu), om * math.sqrt(rho / (lam + 2 * mu))
        c0 = (2 * ks ** 3 + kp ** 3) / (12 * math.pi * mu * ks ** 2)
        G = oracle.green(oracle.problem(rho, lam, mu, om, "U"), x, y)
        e = np.abs(G - K - 1j * c0 * np.eye(3)).max() / np.abs(K).max()
        errs.append(e)
        assert e <= 2 * (ks * r) ** 2
        assert np.abs(G.real - K).max() <= 2 * (ks * r) ** 2 * np.abs(K).max()
    assert 50 < errs[0] / errs[1] < 200  # quadratic in w


def test_far_field(oracle):
    """k r >> 1: U = G_s (I - rr)/mu + G_p rr/(lam + 2 mu) + O(1/r^2)."""
    rho, lam, mu, om = 1.0, 2.0, 1.0, 5.0
    ks, kp = om * math.sqrt(rho / mu), om * math.sqrt(rho / (lam + 2 * mu))
    pb = oracle.problem(rho, lam, mu, om, "U")
    x = np.zeros(3)
    rh = np.array([2.0, -1.0, 0.5])
    rh /= np.linalg.norm(rh)
    errs = []
    for r in (1e2, 1e3):
        y = x - r * rh
        Gs = np.exp(1j * ks * r) / (4 * math.pi * r)
        Gp = np.exp(1j * kp * r) / (4 * math.pi * r)
        ff = Gs * (np.eye(3) - np.outer(rh, rh)) / mu + Gp * np.outer(rh, rh) / (lam + 2 * mu)
        G = oracle.green(pb, x, y)
        errs.append(np.abs(G - ff).max() / np.abs(ff).max())
    assert errs[1] < 5 / (kp * 1e3)
    assert 5 < errs[0] / errs[1] < 20  # O(1/(k r))


def read_pattern():
    path = os.path.join(os.path.dirname(__file__), "golden", "fsplane_pattern.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    iu, it = rows.index(["U"]), rows.index(["T"])
    U = np.array(rows[iu + 1:iu + 4], int)
    T = np.array(rows[it + 1:it + 4], int)
    return U, T


def test_coplanar_pattern(oracle):
    """Eq. FSplane: for x_3 = y_3 (and n = e_3 for T) the listed entries vanish."""
    Upat, Tpat = read_pattern()
    rng = np.random.default_rng(3)
    n = np.array([0.0, 0.0, 1.0])
    for rho, lam, mu, om in MATS:
        for kern, pat in (("U", Upat), ("T", Tpat)):
            pb = oracle.problem(rho, lam, mu, om, kern)
            for _ in range(5):
                x = np.r_[rng.standard_normal(2), 0.7]
                y = np.r_[rng.standard_normal(2), 0.7]
                G = oracle.green(pb, x, y, n)
                assert np.all(G[pat == 0] == 0)
                assert np.all(np.abs(G[pat == 1]) > 1e-8 * np.abs(G).max())


@pytest.mark.parametrize("mat", MATS)
def test_traction_by_finite_differences(oracle, mat):
    """T_ab(x,y) = C_{a g t s} d/dy_s U_bt(x,y) n_g(y) (Sec. 5.3 component form
    of Eq. elasto_T) with C = lam d_ag d_ts + mu (d_at d_gs + d_as d_gt)."""
    rho, lam, mu, om = mat
    pu = oracle.problem(rho, lam, mu, om, "U")
    pt = oracle.problem(rho, lam, mu, om, "T")
    rng = np.random.default_rng(4)
    for r in (0.3, 1.1, 3.0):
        x, y0 = rnd_pair(rng, r)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        h = 1e-3 * r
        dU = np.zeros((3, 3, 3), complex)  # dU[s] = d/dy_s U
        for s in range(3):
            e = np.eye(3)[s]
            dU[s] = sum(c * oracle.green(pu, x, y0 + i * h * e) for i, c in C1.items()) / h
        d = np.eye(3)
        Cten = (lam * np.einsum("ag,ts->agts", d, d)
                + mu * (np.einsum("at,gs->agts", d, d) + np.einsum("as,gt->agts", d, d)))
        Tfd = np.einsum("agts,sbt,g->ab", Cten, dU, n)
        T = oracle.green(pt, x, y0, n)
        assert np.abs(T - Tfd).max() <= 1e-7 * np.abs(T).max()


def test_radial_high_precision(oracle):
    """psi, chi and their derivatives against a 50-digit evaluation of the same
    closed form; pins cancellation at small k r (config 2 reaches k_s r ~ 0.2)."""
    mp.mp.dps = 50
    rho, lam, mu, om = 1.0, 2.0, 1.0, 16.0
    ks = mp.mpf(om) * mp.sqrt(mp.mpf(rho) / mu)
    kp = mp.mpf(om) * mp.sqrt(mp.mpf(rho) / (lam + 2 * mu))

    def G(k, r):
        return mp.exp(1j * k * r) / (4 * mp.pi * r)

    def psi(r):
        return (G(ks, r) + mp.diff(lambda t: G(ks, t) - G(kp, t), r) / (ks ** 2 * r)) / mu

    def chi(r):
        F = lambda t: G(ks, t) - G(kp, t)  # noqa: E731
        return (mp.diff(F, r, 2) - mp.diff(F, r) / r) / (ks ** 2 * mu)

    for r in (1e-3, 1e-2, 0.2, 1.0, 4.0):
        o = oracle.radial(r, rho, lam, mu, om)
        ref = [psi(mp.mpf(r)), chi(mp.mpf(r)), mp.diff(psi, mp.mpf(r)), mp.diff(chi, mp.mpf(r))]
        for val, rv in zip(o, ref):
            rv = complex(rv)
            tol = 1e-13 / min(1.0, (float(ks) * r) ** 2) + 1e-13
            assert abs(val - rv) <= tol * abs(rv), (r, val, rv)


def test_diagonal_block(oracle):
    """The i = j block of A is diag_value * I3 (the configs' choice)."""
    from paper_1706_09384_gb300 import inputs
    pts = inputs.fibonacci_sphere(20)
    A = oracle.dense_matrix(oracle.problem(1, 2, 1, 4.0, "U", diag_value=1.0), pts)
    for i in range(20):
        assert np.array_equal(A[3 * i:3 * i + 3, 3 * i:3 * i + 3], np.eye(3))
