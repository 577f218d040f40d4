"""Pins of the oracle's cluster tree (Sec. 2.1), admissibility (Sec. 6.1,
Eq. admissibility_cond / admissibility_cond_bis) and partition P
(Sec. 2.1 "Subdivision of the matrix"): invariants, brute force on tiny
clouds and the storage bound of Sec. 5.1."""
import math

import numpy as np
import pytest

from paper_1706_09384_gb300 import inputs


def clouds():
    rng = np.random.default_rng(7)
    yield "sphere", inputs.fibonacci_sphere(1536), 32
    yield "plate", inputs.plate(30), 16
    yield "cube", inputs.cube_surface(900, seed=1)[0], 20
    yield "random", rng.random((500, 3)) * np.array([3.0, 1.0, 0.2]), 10
    dup = np.repeat(rng.random((40, 3)), 5, axis=0)  # coincident points
    yield "duplicates", dup, 4


@pytest.mark.parametrize("name,pts,leaf", list(clouds()), ids=lambda v: v if isinstance(v, str) else "")
def test_tree_invariants(oracle, name, pts, leaf):
    perm, cl = oracle.tree_build(pts, leaf)
    nc = len(pts)
    assert np.array_equal(np.sort(perm), np.arange(nc))            # bijection
    assert cl[0]["begin"] == 0 and cl[0]["end"] == nc and cl[0]["level"] == 0
    for c in cl:
        P = pts[perm[c["begin"]:c["end"]]]
        assert np.array_equal(c["lo"], P.min(0)) and np.array_equal(c["hi"], P.max(0))  # tight box
        if c["is_leaf"]:
            ext = c["hi"] - c["lo"]
            assert c["end"] - c["begin"] <= leaf or ext.max() == 0.0
            continue
        assert c["end"] - c["begin"] > leaf
        a, b = cl[c["child0"]], cl[c["child1"]]
        assert a["begin"] == c["begin"] and a["end"] == b["begin"] and b["end"] == c["end"]
        assert a["level"] == b["level"] == c["level"] + 1
        ext = c["hi"] - c["lo"]
        axis = int(np.argmax(ext))                                   # largest extent, lowest axis on ties
        mid = (c["lo"][axis] + c["hi"][axis]) * 0.5
        assert np.all(pts[perm[a["begin"]:a["end"]], axis] < mid)
        assert np.all(pts[perm[b["begin"]:b["end"]], axis] >= mid)
        # stable: children keep the parent's relative order
        seg = perm[c["begin"]:c["end"]]
        left = seg[pts[seg, axis] < mid]
        assert np.array_equal(perm[a["begin"]:a["end"]], left)


def test_tree_depth_matches_L(oracle):
    """Sec. 2.1: for uniform clouds the tree is balanced, L(I) = ceil(log2(|I|/N_leaf))."""
    for nc, leaf in ((1536, 32), (6000, 64), (20000, 100)):
        _, cl = oracle.tree_build(inputs.fibonacci_sphere(nc), leaf)
        L = math.ceil(math.log2(nc / leaf))
        depth = int(cl["level"].max())
        assert L <= depth <= L + 2, (nc, leaf, depth, L)


def test_box_bounds_brute_force(oracle):
    """diam_box >= diam and dist_box <= dist (Sec. 6.1); overlapping boxes have
    dist_box = 0 (the positive-part reading of the printed formula)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        X = rng.random((6, 3)) * rng.random(3) * 2
        Y = rng.random((5, 3)) * rng.random(3) * 2 + rng.standard_normal(3)
        dX = max(np.linalg.norm(p - q) for p in X for q in X)
        dist = min(np.linalg.norm(p - q) for p in X for q in Y)
        assert oracle.diam_box(X.min(0), X.max(0)) >= dX * (1 - 1e-15)
        db = oracle.dist_box(X.min(0), X.max(0), Y.min(0), Y.max(0))
        assert db <= dist * (1 + 1e-15)
        if np.all(X.min(0) <= Y.max(0)) and np.all(Y.min(0) <= X.max(0)):
            assert db == 0.0
        for eta in (0.5, 3.0):
            if oracle.admissible_box(X.min(0), X.max(0), Y.min(0), Y.max(0), eta):
                assert oracle.admissible_exact(X, Y, eta)
    # strict "<": coincident boxes are never admissible
    lo, hi = np.zeros(3), np.ones(3)
    assert not oracle.admissible_box(lo, hi, lo, hi, 1e9)


@pytest.mark.parametrize("name,pts,leaf", list(clouds()), ids=lambda v: v if isinstance(v, str) else "")
def test_partition_tiles_matrix(oracle, name, pts, leaf):
    """P tiles I x I exactly once; admissible blocks pass the exact condition;
    non-admissible blocks have a leaf on one side (Sec. 2.1, Sec. 5.1)."""
    eta = 3.0
    perm, cl = oracle.tree_build(pts, leaf)
    blk = oracle.partition(cl, eta)
    nc = len(pts)
    cover = np.zeros((nc, nc), np.int32)
    for b in blk:
        t, s = cl[b["tau"]], cl[b["sigma"]]
        cover[t["begin"]:t["end"], s["begin"]:s["end"]] += 1
        if b["admissible"]:
            X, Y = pts[perm[t["begin"]:t["end"]]], pts[perm[s["begin"]:s["end"]]]
            if len(X) * len(Y) < 4000:
                assert oracle.admissible_exact(X, Y, eta)
        else:
            assert t["is_leaf"] or s["is_leaf"]
            assert not oracle.admissible_box(t["lo"], t["hi"], s["lo"], s["hi"], eta)
    assert np.all(cover == 1)


def test_storage_bound(oracle):
    """Sec. 5.1: N_st <= 2 C_sp max(r_max, N_leaf) N_c (log2 N_c - log2 N_leaf + 1)
    with C_sp the sparsity constant of Sec. 2.1."""
    nc, leaf = 1536, 32
    pts = inputs.fibonacci_sphere(nc)
    H = oracle.HMatrix(oracle.problem(1, 2, 1, 4.0, "U"), pts, eps=1e-4, eta=3.0, leaf=leaf)
    blk, ra, r = H.blocks()
    cl = H.clusters()
    rows = np.bincount(blk["tau"], minlength=len(cl))
    cols = np.bincount(blk["sigma"], minlength=len(cl))
    csp = max(rows.max(), cols.max())
    sz = cl["end"] - cl["begin"]
    m, n = sz[blk["tau"]], sz[blk["sigma"]]
    # storage counted per point pair as in Sec. 5.1 (ranks in points: r/3)
    nst = np.where(blk["admissible"] == 1, (r / 3.0) * (m + n), m * n).sum()
    rmax = ra.max() / 3.0
    bound = 2 * csp * max(rmax, leaf) * nc * (math.log2(nc) - math.log2(leaf) + 1)
    assert nst <= bound
    assert nst < nc * nc  # compression happens at all


def test_icosphere_vertices():
    """10 * 4^l + 2 distinct unit vectors, nearest-neighbour spacing within a
    factor 1.5 of its mean (a quasi-uniform mesh), normals = positions."""
    import numpy as np
    from scipy.spatial import cKDTree
    from paper_1706_09384_gb300 import inputs
    for level in range(0, 5):
        p, n = inputs.icosphere(level)
        assert len(p) == 10 * 4 ** level + 2
        assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-15)
        assert np.array_equal(p, n)
        d, _ = cKDTree(p).query(p, k=2)
        nn = d[:, 1]
        assert nn.min() > 0 and nn.max() < 1.5 * nn.mean() and nn.min() > nn.mean() / 1.5
