"""ctypes binding of the FP64 oracle (test infrastructure only).

Arrays cross as numpy complex128 (interleaved re/im doubles) or float64/int64.
"""
import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


class Problem(C.Structure):
    _fields_ = [("rho", C.c_double), ("lam", C.c_double), ("mu", C.c_double),
                ("omega", C.c_double), ("kernel", C.c_int32), ("pad_", C.c_int32),
                ("diag_value", C.c_double), ("weights", C.c_void_p)]


class Cluster(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64), ("child0", C.c_int64),
                ("child1", C.c_int64), ("parent", C.c_int64), ("level", C.c_int32),
                ("is_leaf", C.c_int32), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class Block(C.Structure):
    _fields_ = [("tau", C.c_int64), ("sigma", C.c_int64), ("admissible", C.c_int32),
                ("pad_", C.c_int32)]


CLUSTER_DTYPE = np.dtype([("begin", "<i8"), ("end", "<i8"), ("child0", "<i8"),
                          ("child1", "<i8"), ("parent", "<i8"), ("level", "<i4"),
                          ("is_leaf", "<i4"), ("lo", "<f8", (3,)), ("hi", "<f8", (3,))])
BLOCK_DTYPE = np.dtype([("tau", "<i8"), ("sigma", "<i8"), ("admissible", "<i4"),
                        ("pad_", "<i4")])

_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
_INT = C.c_int


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        sig = {
            "or_radial": (None, [_D, _D, _D, _D, _D, _P]),
            "or_green": (None, [_P, _P, _P, _P, _P]),
            "or_dense_matrix": (None, [_P, _P, _P, _I64, _P]),
            "or_dense_rows_matvec": (None, [_P, _P, _P, _I64, _P, _I64, _P, _P, _INT]),
            "or_tree_build": (_I64, [_P, _I64, _I64, _P, _P]),
            "or_diam_box": (_D, [_P, _P]),
            "or_dist_box": (_D, [_P, _P, _P, _P]),
            "or_admissible_box": (_INT, [_P, _P, _P, _P, _D]),
            "or_admissible_exact": (_INT, [_P, _I64, _P, _I64, _D]),
            "or_partition": (_I64, [_P, _I64, _D, _P]),
            "or_sv3": (None, [_P, _P]),
            "or_svd_jacobi": (_INT, [_P, _I64, _I64, _P, _P, _P]),
            "or_qr_householder": (_INT, [_P, _I64, _I64, _P, _P]),
            "or_aca_dense": (_I64, [_P, _I64, _I64, _D, _I64, _P, _P, _P]),
            "or_recompress": (_I64, [_P, _P, _I64, _I64, _I64, _D, _P, _P, _P]),
            "or_rsvd_dense": (_I64, [_P, _I64, _I64, _D, C.c_uint64, _I64, _P, _P, _P]),
            "or_gauss": (None, [C.c_uint64, C.c_uint64, _P]),
            "or_rsvd_key": (C.c_uint64, [_I64, _I64]),
            "or_splitmix64": (C.c_uint64, [C.c_uint64]),
            "or_hmat_block_methods": (None, [_P, _P]),
            "or_hmat_build": (_P, [_P, _P, _P, _I64, _D, _D, _I64, _INT, _I64, _INT]),
            "or_hlu_factor": (_P, [_P, _D, _D, _P]),
            "or_hlu_free": (None, [_P]),
            "or_hlu_solve": (None, [_P, _P, _P]),
            "or_hlu_dense": (None, [_P, _P, _P]),
            "or_hlu_seconds": (_D, [_P]),
            "or_hlu_stored": (_I64, [_P]),
            "or_hmat_free": (None, [_P]),
            "or_hmat_nclusters": (_I64, [_P]),
            "or_hmat_clusters": (None, [_P, _P]),
            "or_hmat_perm": (None, [_P, _P]),
            "or_hmat_nblocks": (_I64, [_P]),
            "or_hmat_blocks": (None, [_P, _P, _P, _P]),
            "or_hmat_block_data": (None, [_P, _I64, _P, _P]),
            "or_hmat_matvec": (None, [_P, _P, _P]),
            "or_dense_matrix2": (None, [_P, _P, _I64, _P, _I64, _P, _P]),
            "or_partition2": (_I64, [_P, _I64, _P, _I64, _D, _P]),
            "or_hmat2_build": (_P, [_P, _P, _I64, _P, _I64, _P, _D, _D, _I64, _INT]),
            "or_hmat2_free": (None, [_P]),
            "or_hmat2_nblocks": (_I64, [_P]),
            "or_hmat2_blocks": (None, [_P, _P, _P]),
            "or_hmat2_nclusters": (_I64, [_P, _INT]),
            "or_hmat2_clusters": (None, [_P, _P, _P]),
            "or_hmat2_matvec": (None, [_P, _P, _P]),
            "or_hmat_build_seconds": (_D, [_P]),
            "or_gmres_hmat": (_INT, [_P, _P, _P, _INT, _D, _INT, _P, _P]),
            "or_gmres_dense": (_INT, [_P, _I64, _P, _P, _INT, _D, _INT, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def problem(rho=1.0, lam=2.0, mu=1.0, omega=4.0, kernel="U", diag_value=1.0, weights=None):
    """Problem definition; `weights` (n_c column weights w_j) are kept alive on
    the returned object."""
    k = {"U": 0, "T": 1}[kernel] if isinstance(kernel, str) else int(kernel)
    pb = Problem(rho, lam, mu, omega, k, 0, diag_value, None)
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        pb._w = w
        pb.weights = w.ctypes.data
    return pb


def radial(r, rho, lam, mu, omega):
    out = np.zeros(4, np.complex128)
    lib().or_radial(r, rho, lam, mu, omega, _ptr(out))
    return out  # psi, chi, dpsi, dchi


def green(pb, x, y, ny=None):
    """3x3 complex K(x, y) (row-major alpha, beta)."""
    G = np.zeros((3, 3), np.complex128)
    x, y = _f64(x), _f64(y)
    nyv = _f64(ny) if ny is not None else np.zeros(3)
    lib().or_green(C.byref(pb), _ptr(x), _ptr(y), _ptr(nyv), _ptr(G))
    return G


def dense_matrix(pb, pts, nrm=None):
    pts = _f64(pts)
    nc = pts.shape[0]
    A = np.zeros((3 * nc, 3 * nc), np.complex128)
    lib().or_dense_matrix(C.byref(pb), _ptr(pts), _ptr(_f64(nrm)) if nrm is not None else None,
                          nc, _ptr(A))
    return A


def dense_rows_matvec(pb, pts, nrm, rows, x, nthreads=0):
    pts = _f64(pts)
    rows = np.ascontiguousarray(rows, np.int64)
    x = _c128(x)
    out = np.zeros(len(rows), np.complex128)
    lib().or_dense_rows_matvec(C.byref(pb), _ptr(pts), _ptr(_f64(nrm)) if nrm is not None else None,
                               pts.shape[0], _ptr(rows), len(rows), _ptr(x), _ptr(out), nthreads)
    return out


def tree_build(pts, leaf):
    pts = _f64(pts)
    nc = pts.shape[0]
    perm = np.zeros(nc, np.int64)
    cl = np.zeros(2 * nc + 1, CLUSTER_DTYPE)
    n = lib().or_tree_build(_ptr(pts), nc, leaf, _ptr(perm), _ptr(cl))
    return perm, cl[:n].copy()


def diam_box(lo, hi):
    return lib().or_diam_box(_ptr(_f64(lo)), _ptr(_f64(hi)))


def dist_box(lo1, hi1, lo2, hi2):
    return lib().or_dist_box(_ptr(_f64(lo1)), _ptr(_f64(hi1)), _ptr(_f64(lo2)), _ptr(_f64(hi2)))


def admissible_box(lo1, hi1, lo2, hi2, eta):
    return bool(lib().or_admissible_box(_ptr(_f64(lo1)), _ptr(_f64(hi1)), _ptr(_f64(lo2)),
                                        _ptr(_f64(hi2)), eta))


def admissible_exact(X, Y, eta):
    X, Y = _f64(X), _f64(Y)
    return bool(lib().or_admissible_exact(_ptr(X), X.shape[0], _ptr(Y), Y.shape[0], eta))


def dense_matrix2(pb, X, Y, nrmY=None):
    """The 3 nx x 3 ny matrix between targets X and sources Y (normals at Y)."""
    X, Y = _f64(X), _f64(Y)
    A = np.zeros((3 * X.shape[0], 3 * Y.shape[0]), np.complex128)
    lib().or_dense_matrix2(C.byref(pb), _ptr(X), X.shape[0], _ptr(Y), Y.shape[0],
                           _ptr(_f64(nrmY)) if nrmY is not None else None, _ptr(A))
    return A


def partition2(clX, clY, eta):
    a = np.ascontiguousarray(clX, CLUSTER_DTYPE)
    b = np.ascontiguousarray(clY, CLUSTER_DTYPE)
    n = lib().or_partition2(_ptr(a), len(a), _ptr(b), len(b), eta, None)
    out = np.zeros(n, BLOCK_DTYPE)
    lib().or_partition2(_ptr(a), len(a), _ptr(b), len(b), eta, _ptr(out))
    return out


def partition(clusters, eta):
    cl = np.ascontiguousarray(clusters, CLUSTER_DTYPE)
    n = lib().or_partition(_ptr(cl), len(cl), eta, None)
    out = np.zeros(n, BLOCK_DTYPE)
    lib().or_partition(_ptr(cl), len(cl), eta, _ptr(out))
    return out


def sv3(M):
    M = _c128(M)
    s = np.zeros(3)
    lib().or_sv3(_ptr(M), _ptr(s))
    return s


def svd_jacobi(A):
    """A (M x N, M >= N) -> (U, s, V) with A = U diag(s) V^H."""
    A = np.asfortranarray(A, dtype=np.complex128)
    M, N = A.shape
    s = np.zeros(N)
    U = np.zeros((M, N), np.complex128, order="F")
    V = np.zeros((N, N), np.complex128, order="F")
    lib().or_svd_jacobi(_ptr(A), M, N, _ptr(s), _ptr(U), _ptr(V))
    return U, s, V


def qr(A):
    A = np.asfortranarray(A, dtype=np.complex128)
    M, N = A.shape
    Q = np.zeros((M, N), np.complex128, order="F")
    R = np.zeros((N, N), np.complex128, order="F")
    lib().or_qr_householder(_ptr(A), M, N, _ptr(Q), _ptr(R))
    return Q, R


def aca_dense(A, eps, kcap=None):
    """Vector ACA of an explicit 3m x 3n matrix.  Returns (U, V, pivots)."""
    A = _c128(A)
    m3, n3 = A.shape
    m, n = m3 // 3, n3 // 3
    kcap = kcap if kcap is not None else 3 * min(m, n)
    U = np.zeros((kcap, m3), np.complex128)  # col-major storage as rows of U^T
    V = np.zeros((kcap, n3), np.complex128)
    piv = np.zeros(2 * (kcap // 3 + 1), np.int64)
    k = lib().or_aca_dense(_ptr(A), m, n, eps, kcap, _ptr(U), _ptr(V), _ptr(piv))
    if k < 0:
        raise RuntimeError("ACA rank exceeded capacity")
    return U[:k].T.copy(), V[:k].T.copy(), piv[:2 * (k // 3)].reshape(-1, 2)


def recompress(U, V, eps):
    U = np.asfortranarray(U, dtype=np.complex128)
    V = np.asfortranarray(V, dtype=np.complex128)
    M, k = U.shape
    N = V.shape[0]
    U2 = np.zeros((max(k, 1), M), np.complex128)
    V2 = np.zeros((max(k, 1), N), np.complex128)
    s = np.zeros(max(k, 1))
    r = lib().or_recompress(_ptr(U), _ptr(V), M, N, k, eps, _ptr(U2), _ptr(V2), _ptr(s))
    return U2[:r].T.copy(), V2[:r].T.copy(), s[:k].copy()


def gauss(key, counters):
    """Entries of the randomized SVD's test matrix for the given counters."""
    out = np.zeros(2, np.float64)
    z = np.zeros(len(counters), np.complex128)
    for i, c in enumerate(counters):
        lib().or_gauss(int(key), int(c), _ptr(out))
        z[i] = out[0] + 1j * out[1]
    return z


def splitmix64(z):
    return int(lib().or_splitmix64(int(z) & ((1 << 64) - 1)))


def rsvd_key(tau_begin, sigma_begin):
    return int(lib().or_rsvd_key(int(tau_begin), int(sigma_begin)))


def rsvd_dense(A, eps, key=0):
    """Randomized range finder of an explicit 3m x 3n matrix.  Returns (U, V, ok)
    with U = Q (orthonormal columns) and V = (Q^H A)^H, before recompression."""
    A = _c128(A)
    m3, n3 = A.shape
    lcap = min(m3, n3, 768)
    U = np.zeros((lcap, m3), np.complex128)
    V = np.zeros((lcap, n3), np.complex128)
    ok = C.c_int(0)
    l = lib().or_rsvd_dense(_ptr(A), m3 // 3, n3 // 3, eps, int(key), lcap, _ptr(U), _ptr(V),
                            C.byref(ok))
    return U[:l].T.copy(), V[:l].T.copy(), bool(ok.value)


class HMatrix:
    """Oracle H-matrix (tree, partition, dense blocks, ACA + recompression)."""

    def __init__(self, pb, pts, nrm=None, eps=1e-4, eta=3.0, leaf=32, recompress=True,
                 sample_stride=1, nthreads=0):
        self.pts = _f64(pts)
        self.nrm = _f64(nrm) if nrm is not None else None
        self.pb = pb
        self.nc = self.pts.shape[0]
        self.h = lib().or_hmat_build(C.byref(pb), _ptr(self.pts), _ptr(self.nrm), self.nc, eps,
                                     eta, leaf, 1 if recompress else 0, sample_stride, nthreads)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_hmat_free(self.h)
            self.h = None

    @property
    def build_seconds(self):
        return lib().or_hmat_build_seconds(self.h)

    def perm(self):
        p = np.zeros(self.nc, np.int64)
        lib().or_hmat_perm(self.h, _ptr(p))
        return p

    def clusters(self):
        n = lib().or_hmat_nclusters(self.h)
        cl = np.zeros(n, CLUSTER_DTYPE)
        lib().or_hmat_clusters(self.h, _ptr(cl))
        return cl

    def blocks(self):
        n = lib().or_hmat_nblocks(self.h)
        b = np.zeros(n, BLOCK_DTYPE)
        ra = np.zeros(n, np.int64)
        r = np.zeros(n, np.int64)
        lib().or_hmat_blocks(self.h, _ptr(b), _ptr(ra), _ptr(r))
        return b, ra, r

    def block_methods(self):
        """0 dense or vector ACA, 1 randomized SVD, 2 randomized SVD at its cap."""
        m = np.zeros(lib().or_hmat_nblocks(self.h), np.int32)
        lib().or_hmat_block_methods(self.h, _ptr(m))
        return m

    def block_data(self, b, blocks=None, clusters=None, ranks=None):
        """dense -> D (3m x 3n); low rank -> (U, V) with block = U V^H."""
        if blocks is None:
            blocks, _, ranks = self.blocks()
        if clusters is None:
            clusters = self.clusters()
        t, s = clusters[blocks[b]["tau"]], clusters[blocks[b]["sigma"]]
        m3, n3 = 3 * (t["end"] - t["begin"]), 3 * (s["end"] - s["begin"])
        if not blocks[b]["admissible"]:
            D = np.zeros((n3, m3), np.complex128)
            lib().or_hmat_block_data(self.h, b, _ptr(D), None)
            return D.T.copy()
        r = int(ranks[b])
        U = np.zeros((max(r, 1), m3), np.complex128)
        V = np.zeros((max(r, 1), n3), np.complex128)
        lib().or_hmat_block_data(self.h, b, _ptr(U), _ptr(V))
        return U[:r].T.copy(), V[:r].T.copy()

    def matvec(self, x):
        x = _c128(x)
        y = np.zeros_like(x)
        lib().or_hmat_matvec(self.h, _ptr(x), _ptr(y))
        return y

    def gmres(self, b, restart=50, tol=1e-6, maxit=1000):
        b = _c128(b)
        x = np.zeros_like(b)
        it = C.c_int(0)
        rr = C.c_double(0)
        st = lib().or_gmres_hmat(self.h, _ptr(b), _ptr(x), restart, tol, maxit, C.byref(it),
                                 C.byref(rr))
        return x, it.value, rr.value, st


def gmres_dense(A, b, restart=50, tol=1e-6, maxit=1000):
    A = _c128(A)
    b = _c128(b)
    x = np.zeros_like(b)
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib().or_gmres_dense(_ptr(A), A.shape[0], _ptr(b), _ptr(x), restart, tol, maxit,
                              C.byref(it), C.byref(rr))
    return x, it.value, rr.value, st




class HMatrix2:
    """Oracle H-matrix between two clouds: targets X (rows), sources Y
    (columns, with normals and the problem's weights)."""

    def __init__(self, pb, X, Y, nrmY=None, eps=1e-4, eta=3.0, leaf=32, nthreads=0):
        self.pb = pb
        self.X, self.Y = _f64(X), _f64(Y)
        self.nrmY = _f64(nrmY) if nrmY is not None else None
        self.nx, self.ny = self.X.shape[0], self.Y.shape[0]
        self.h = lib().or_hmat2_build(C.byref(pb), _ptr(self.X), self.nx, _ptr(self.Y), self.ny,
                                      _ptr(self.nrmY), eps, eta, leaf, nthreads)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_hmat2_free(self.h)
            self.h = None

    def blocks(self):
        n = lib().or_hmat2_nblocks(self.h)
        blk = np.zeros(n, BLOCK_DTYPE)
        r = np.zeros(n, np.int64)
        lib().or_hmat2_blocks(self.h, _ptr(blk), _ptr(r))
        return blk, r

    def clusters(self):
        a = np.zeros(lib().or_hmat2_nclusters(self.h, 0), CLUSTER_DTYPE)
        b = np.zeros(lib().or_hmat2_nclusters(self.h, 1), CLUSTER_DTYPE)
        lib().or_hmat2_clusters(self.h, _ptr(a), _ptr(b))
        return a, b

    def matvec(self, x):
        """y = A_H x for x of 3 ny complex entries (original source order)."""
        x = _c128(x)
        y = np.zeros(3 * self.nx, np.complex128)
        lib().or_hmat2_matvec(self.h, _ptr(x), _ptr(y))
        return y


class HLU:
    """H-LU factors of an oracle H-matrix (Sec. 3.2); solve() is the direct solver."""

    def __init__(self, H, eta, eps_lu):
        self.H = H  # keeps the H-matrix alive
        self.nc = H.nc
        st = C.c_int(0)
        self.f = lib().or_hlu_factor(H.h, eta, eps_lu, C.byref(st))
        self.status = st.value

    def __del__(self):
        if getattr(self, "f", None):
            lib().or_hlu_free(self.f)
            self.f = None

    def solve(self, b):
        b = _c128(b)
        x = np.zeros_like(b)
        lib().or_hlu_solve(self.f, _ptr(b), _ptr(x))
        return x

    def dense(self):
        N = 3 * self.nc
        L = np.zeros((N, N), np.complex128)
        U = np.zeros((N, N), np.complex128)
        lib().or_hlu_dense(self.f, _ptr(L), _ptr(U))
        return L.T.copy(), U.T.copy()  # col-major buffers

    @property
    def seconds(self):
        return lib().or_hlu_seconds(self.f)

    @property
    def stored(self):
        return lib().or_hlu_stored(self.f)


__all__ = [n for n in dir() if not n.startswith("_")]
