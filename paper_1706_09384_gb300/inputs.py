"""Seeded synthetic inputs: point clouds, normals and right-hand sides.

This module holds none of the method's arithmetic; it only makes inputs, and
it is the one module that both the CUDA path's tests/bench and the FP64
oracle use.  The clouds stand in for the paper's BEM meshes (icosphere
vertices of a unit sphere, Sec. 7-8, and the plate of Sec. 2.1) with the same
size, shape and density regime.
"""
import math

import numpy as np


def fibonacci_sphere(nc: int, radius: float = 1.0) -> np.ndarray:
    """Quasi-uniform points on a sphere: z_k = 1 - (2k+1)/nc, phi_k = k*pi*(3 - sqrt 5)."""
    k = np.arange(nc, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / nc
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return radius * np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def sphere_normals(pts: np.ndarray) -> np.ndarray:
    """Outward unit normals of a sphere centred at the origin."""
    return pts / np.linalg.norm(pts, axis=1, keepdims=True)


def ellipsoid(nc: int, axes=(1.0, 2.0 / 3.0, 1.0 / 3.0)):
    """Fibonacci points scaled to an ellipsoid (non-uniform density), with normals."""
    s = fibonacci_sphere(nc)
    a = np.asarray(axes, dtype=np.float64)
    pts = s * a
    n = s / a
    return pts, n / np.linalg.norm(n, axis=1, keepdims=True)


def plate(nd: int = 50, a: float = 1.0) -> np.ndarray:
    """Uniform nd x nd grid on [-a, a]^2 x {0} (the illustrative plate of Sec. 2.1)."""
    g = np.linspace(-a, a, nd)
    X, Y = np.meshgrid(g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(nd * nd)], axis=1)


def cube_surface(nc: int, seed: int = 0):
    """Points on the surface of [0,1]^3: each face gets floor or ceil(nc/6) points
    from the 2-D R2 low-discrepancy sequence with a seeded offset.  Returns
    (points, outward normals)."""
    rng = np.random.default_rng(seed)
    g = 1.32471795724474602596  # plastic number: R2 sequence alpha = (1/g, 1/g^2)
    alpha = np.array([1.0 / g, 1.0 / (g * g)])
    counts = [nc // 6 + (1 if f < nc % 6 else 0) for f in range(6)]
    pts, nrm = [], []
    for f, cnt in enumerate(counts):
        off = rng.random(2)
        k = np.arange(1, cnt + 1, dtype=np.float64)[:, None]
        uv = np.mod(off + k * alpha, 1.0)
        axis, side = f // 2, f % 2
        p = np.zeros((cnt, 3))
        others = [a for a in range(3) if a != axis]
        p[:, others[0]] = uv[:, 0]
        p[:, others[1]] = uv[:, 1]
        p[:, axis] = float(side)
        n = np.zeros((cnt, 3))
        n[:, axis] = 1.0 if side else -1.0
        pts.append(p)
        nrm.append(n)
    return np.concatenate(pts), np.concatenate(nrm)


def random_rhs(n: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """complex128 right-hand sides with N(0,1) + i N(0,1) entries, DOF order.
    Shape (n,) for nrhs == 1, else (n, nrhs) column-major values."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))
    return b[0].copy() if nrhs == 1 else np.asfortranarray(b.T)


def plane_wave_directions(nrhs: int, seed: int = 0):
    """Propagation directions d_s uniform on S^2 and unit polarisations p_s _|_ d_s."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((nrhs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    q = rng.standard_normal((nrhs, 3))
    p = q - np.sum(q * d, axis=1, keepdims=True) * d
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return d, p


def material(kappa_s: float, rho: float = 1.0, mu: float = 1.0, lam: float = 2.0):
    """(rho, lam, mu, omega) with omega chosen so that k_s = omega sqrt(rho/mu) = kappa_s."""
    return rho, lam, mu, kappa_s / math.sqrt(rho / mu)


def plane_wave_rhs(points: np.ndarray, kappa_p: float, kappa_s: float, nrhs: int, seed: int = 0):
    """Incident plane waves sampled at the points, DOF order, shape (3 n_c, nrhs)
    column-major: even s a P wave d_s exp(i k_p d_s.x), odd s an S wave
    p_s exp(i k_s d_s.x), with d_s, p_s from plane_wave_directions."""
    d, p = plane_wave_directions(nrhs, seed)
    out = np.empty((3 * len(points), nrhs), dtype=np.complex128, order="F")
    for s in range(nrhs):
        if s % 2 == 0:
            u = d[s][None, :] * np.exp(1j * kappa_p * (points @ d[s]))[:, None]
        else:
            u = p[s][None, :] * np.exp(1j * kappa_s * (points @ d[s]))[:, None]
        out[:, s] = u.reshape(-1)
    return out


SURFACE_AREA = {"sphere": 4.0 * math.pi, "cube": 6.0, "ellipsoid": 5.46}  # ellipsoid: Thomsen's estimate


def batch_problems(count: int = 16, seed: int = 0):
    """Independent problems of mixed size, shape, wavenumber and kernel: n_c from
    {4096, ..., 131072}, shape sphere : cube : ellipsoid = 3 : 2 : 1, k_s ~ U[2, 24],
    U or T by a fair coin, column weights area / n_c.  Returns a list of dicts with
    points, normals (None for U), rho, lam, mu, omega, kernel, weights, shape, ks."""
    rng = np.random.default_rng(seed)
    sizes = [4096 * 2 ** k for k in range(6)]
    shapes = ["sphere"] * 3 + ["cube"] * 2 + ["ellipsoid"]
    out = []
    for q in range(count):
        nc = int(rng.choice(sizes))
        shape = shapes[int(rng.integers(6))]
        ks = float(rng.uniform(2.0, 24.0))
        kern = "U" if rng.random() < 0.5 else "T"
        if shape == "sphere":
            pts = fibonacci_sphere(nc)
            nrm = sphere_normals(pts)
        elif shape == "cube":
            pts, nrm = cube_surface(nc, seed=q)
        else:
            pts, nrm = ellipsoid(nc)
        rho, lam, mu, om = material(ks)
        out.append(dict(points=pts, normals=nrm if kern == "T" else None, rho=rho, lam=lam, mu=mu,
                        omega=om, kernel=kern, weights=np.full(nc, SURFACE_AREA[shape] / nc),
                        shape=shape, ks=ks))
    return out


def icosphere(level: int):
    """Vertices of the icosahedron subdivided `level` times (edge midpoints pushed
    to the unit sphere): 10 * 4^level + 2 points, the vertex counts of the
    paper's sphere meshes (642, 2562, 10242, 40962 for levels 3-6).  Returns
    (points, outward normals), deterministic order."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    pts = np.array(verts)
    return pts, pts.copy()
