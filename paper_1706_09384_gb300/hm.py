"""Thin ctypes binding of ``libhm.so`` (the C ABI in ``include/hm.h``).

Names follow the C entry points.  Only argument marshalling happens here:
every step of the build, the product and the solver runs in the library's
CUDA kernels.  Device buffers are torch tensors (PyTorch supplies device
memory and streams).  If ``libhm.so`` cannot be loaded this module raises:
there is no fallback path.
"""
import ctypes as C
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhm.so")

HM_OK, HM_ERR_ARG, HM_ERR_CUDA, HM_ERR_OOM, HM_ERR_NOCONV, HM_ERR_TIMEOUT, HM_ERR_NUMERIC, \
    HM_ERR_UNSUPPORTED = range(8)
HM_KERNEL_U, HM_KERNEL_T = 0, 1
HM_STORE_FP32, HM_STORE_BF16 = 0, 1


class HmError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s failed: %s (%s)" % (where, msg, _status_name(status)))
        self.status = status


class hm_opts(C.Structure):
    _fields_ = [("storage", C.c_int32), ("aca_fp32", C.c_int32), ("diag_value", C.c_double),
                ("fp64_switch_ksr", C.c_double), ("recompress", C.c_int32),
                ("aca_max_rank", C.c_int32), ("workspace_bytes", C.c_int64),
                ("verbose", C.c_int32), ("pad_", C.c_int32), ("weights", C.c_void_p),
                ("rank_model", C.c_void_p), ("tune_cache", C.c_char_p)]


class hm_problem(C.Structure):
    _fields_ = [("points", C.c_void_p), ("normals", C.c_void_p), ("n_c", C.c_int64),
                ("rho", C.c_double), ("lambda_", C.c_double), ("mu", C.c_double),
                ("omega", C.c_double), ("kernel", C.c_int32), ("pad_", C.c_int32),
                ("eta", C.c_double), ("leaf_size", C.c_int64), ("weights", C.c_void_p)]


class hm_cluster(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64), ("child0", C.c_int64),
                ("child1", C.c_int64), ("level", C.c_int32), ("is_leaf", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class hm_block(C.Structure):
    _fields_ = [("tau", C.c_int64), ("sigma", C.c_int64), ("admissible", C.c_int32),
                ("rank_aca", C.c_int32), ("rank", C.c_int32), ("pad_", C.c_int32)]


CLUSTER_DTYPE = np.dtype([("begin", "<i8"), ("end", "<i8"), ("child0", "<i8"), ("child1", "<i8"),
                          ("level", "<i4"), ("is_leaf", "<i4"), ("lo", "<f8", (3,)),
                          ("hi", "<f8", (3,))])
BLOCK_DTYPE = np.dtype([("tau", "<i8"), ("sigma", "<i8"), ("admissible", "<i4"),
                        ("rank_aca", "<i4"), ("rank", "<i4"), ("pad_", "<i4")])
assert CLUSTER_DTYPE.itemsize == C.sizeof(hm_cluster)
assert BLOCK_DTYPE.itemsize == C.sizeof(hm_block)

_P, _I64, _I32, _D, _SZ = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_size_t
SIGNATURES = {
    "hm_opts_default": (None, [_P]),
    "hm_build": (_I32, [_P, _P, _I64, _D, _D, _D, _D, _I32, _D, _D, _I64, _P, _P, _P]),
    "hm_build_batch": (_I32, [_I32, _P, _D, _P, _P, _P]),
    "hm_build2": (_I32, [_P, _I64, _P, _P, _I64, _D, _D, _D, _D, _I32, _D, _D, _I64, _P, _P, _P]),
    "hm_batch_join": (_I32, [_I32, _P, _P, _P]),
    "hm_gmres_batch": (_I32, [_P, _P, _P, _I32, _D, _I32, _P, _P, _P]),
    "hm_matvec": (_I32, [_P, _I32, _P, _P, _P]),
    "hm_matvec_host": (_I32, [_P, _I32, _P, _P, _P]),
    "hm_gmres": (_I32, [_P, _P, _P, _I32, _D, _I32, _P, _P, _P]),
    "hm_gmres_multi": (_I32, [_P, _I32, _P, _P, _I32, C.c_double, _I32, _P, _P, _P]),
    "hm_estimate_error": (_I32, [_P, _I64, C.c_uint64, _P, _P, _P]),
    "hm_lu_factor": (_I32, [_P, _D, _P]),
    "hm_lu_solve": (_I32, [_P, _I32, _P, _P, _P]),
    "hm_lu_info": (_I32, [_P, _P, _P, _P]),
    "hm_stats": (_I32, [_P, C.c_char_p, _SZ, _P]),
    "hm_sizes": (_I32, [_P, _P, _P, _P]),
    "hm_get_tree": (_I32, [_P, _P, _P]),
    "hm_get_blocks": (_I32, [_P, _P]),
    "hm_get_block_data": (_I32, [_P, _I64, _P, _P]),
    "hm_green_eval": (_I32, [_I32, _D, _D, _D, _D, _D, _P, _P, _P, _I64, _P, _P]),
    "hm_import": (_I32, [_I64, _P, _I64, _P, _I64, _P, _P, _P, _P, _P]),
    "hm_aca_block_noalloc": (_I32, [_I32, _D, _D, _D, _D, _P, _I64, _P, _P, _I64, _D, _I32, _P,
                                    _P, _P]),
    "hm_rank_samples": (_I32, [_P, _P, _P, _P]),
    "hm_rank_model_train": (_I32, [_P, _P, _I64, _I32, _I32, C.c_float, C.c_uint64, _P, _P, _P]),
    "hm_rank_model_predict": (_I32, [_P, _P, _I64, _P, _P]),
    "hm_rank_model_grad": (_I32, [_P, _P, _P, _I64, _P, _P, _P]),
    "hm_profile_matvec": (_I32, [_P, _I32, _P, _P, _P]),
    "hm_profile_matvec_multi": (_I32, [_P, _I32, _P, _P, _P]),
    "hm_kernel_launches": (_I64, []),
    "hm_release_cached_memory": (_I32, []),
    "hm_free": (None, [_P]),
    "hm_status_string": (C.c_char_p, [_I32]),
    "hm_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libhm.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhm.so not built (run __graft_entry__.build()): " + LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _status_name(s):
    try:
        return lib().hm_status_string(s).decode()
    except Exception:  # noqa: BLE001
        return str(s)


def _check(st, where):
    if st != HM_OK:
        raise HmError(st, where, lib().hm_last_error().decode())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def hm_kernel_launches():
    return lib().hm_kernel_launches()


def hm_release_cached_memory():
    """Return the memory the library's pools keep for later builds and solves."""
    _check(lib().hm_release_cached_memory(), "hm_release_cached_memory")


def hm_opts_default(**kw):
    """Default options; weights=<array of n_c floats> is kept alive on the object."""
    o = hm_opts()
    lib().hm_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "weights" and v is not None:
            w = np.ascontiguousarray(v, dtype=np.float64)
            o._w = w
            o.weights = w.ctypes.data
        elif k == "tune_cache" and v is not None:
            b = os.fsencode(v)
            o._tc = b
            o.tune_cache = b
        elif k == "rank_model" and v is not None:
            m = np.ascontiguousarray(v, dtype=np.float32)
            assert m.size == HM_RANK_MODEL_PARAMS
            o._m = m
            o.rank_model = m.ctypes.data
        else:
            setattr(o, k, v)
    return o


def hm_green_eval(kernel, rho, lam, mu, omega, x, y, ny=None, diag_value=1.0, stream=None):
    """Green's tensors K(x_q, y_q) on the GPU.  x, y, ny: cuda float64 (n, 3).
    Returns a cuda complex128 tensor (n, 3, 3)."""
    import torch
    n = x.shape[0]
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=x.device)
    _check(lib().hm_green_eval(kernel, rho, lam, mu, omega, diag_value, x.data_ptr(),
                               y.data_ptr(), ny.data_ptr() if ny is not None else None, n,
                               out.data_ptr(), _stream_ptr(stream)), "hm_green_eval")
    return out


HM_NOALLOC_MAX_POINTS = 8192
HM_NRHS_BLOCK = 32  # right-hand sides per tensor-core block product (include/hm.h)
HM_RANK_MODEL_PARAMS = 4687


def _require(cond, what):
    if not cond:
        raise HmError(HM_ERR_ARG, "hm_aca_block_noalloc", what)


def _check_noalloc_args(x, y, ny, cap, uv):
    """The library reads x, y, ny and writes (3m + 3n) cap entries of uv through
    raw device pointers: reject anything that would make it touch memory
    outside those tensors before the call is made."""
    import torch
    pts = (("x", x), ("y", y)) + ((("ny", ny),) if ny is not None else ())
    for name, t in pts:
        _require(isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.dim() == 2
                 and t.shape[1] == 3 and t.is_contiguous(),
                 "%s must be a contiguous float64 tensor of shape (., 3)" % name)
    if ny is not None:
        _require(ny.shape[0] == y.shape[0], "ny must have the shape of y")
    _require(isinstance(uv, torch.Tensor) and uv.dtype == torch.complex128
             and uv.is_contiguous(), "uv must be a contiguous complex128 tensor")
    _require(isinstance(cap, int) and cap > 0, "cap must be a positive int")
    need = (3 * x.shape[0] + 3 * y.shape[0]) * cap
    _require(uv.numel() >= need, "uv holds %d entries, (3m + 3n) cap = %d are written"
             % (uv.numel(), need))
    tensors = [t for _, t in pts] + [uv]
    _require(all(t.is_cuda for t in tensors), "x, y, ny and uv must be cuda tensors")
    _require(len({t.device for t in tensors}) == 1, "x, y, ny and uv must be on one device")


def hm_aca_block_noalloc(kernel, rho, lam, mu, omega, x, y, ny, eps, cap, uv, stream=None):
    """Allocation-free vector ACA of one block.  x (m, 3), y (n, 3), ny (n, 3) or
    None: contiguous cuda float64; uv: contiguous cuda complex128 of at least
    (3m + 3n) * cap entries (checked here, before the call).
    Returns the rank; U = uv[:3m cap] (3m x cap col-major), V follows."""
    _check_noalloc_args(x, y, ny, cap, uv)
    rank = C.c_int32(-1)
    _check(lib().hm_aca_block_noalloc(kernel, rho, lam, mu, omega, x.data_ptr(), x.shape[0],
                                      y.data_ptr(), ny.data_ptr() if ny is not None else None,
                                      y.shape[0], eps, cap, uv.data_ptr(), C.byref(rank),
                                      _stream_ptr(stream)), "hm_aca_block_noalloc")
    return rank.value


class HMatrix:
    """An H-matrix built (or imported) on the current CUDA device."""

    def __init__(self, handle, n_c):
        self.h = handle
        self.n_c = n_c

    @classmethod
    def build(cls, points, normals=None, rho=1.0, lam=2.0, mu=1.0, omega=4.0, kernel="U",
              eps=1e-4, eta=3.0, leaf_size=32, opts=None, stream=None):
        pts = np.ascontiguousarray(points, dtype=np.float64)
        nrm = np.ascontiguousarray(normals, dtype=np.float64) if normals is not None else None
        k = {"U": HM_KERNEL_U, "T": HM_KERNEL_T}[kernel] if isinstance(kernel, str) else kernel
        h = C.c_void_p()
        st = lib().hm_build(_np_ptr(pts), _np_ptr(nrm) if nrm is not None else None,
                            pts.shape[0], rho, lam, mu, omega, k, eps, eta, leaf_size,
                            C.byref(opts) if opts is not None else None, _stream_ptr(stream),
                            C.byref(h))
        _check(st, "hm_build")
        return cls(h, pts.shape[0])

    @classmethod
    def build_batch(cls, problems, eps=1e-4, opts=None, stream=None):
        """Several problems in one batch build.  problems: list of dicts with
        keys points, normals (or None), rho, lam, mu, omega, kernel ("U"/"T"),
        eta, leaf_size, weights (or None).  Returns a list of HMatrix."""
        keep = []
        arr = (hm_problem * len(problems))()
        for q, P in enumerate(problems):
            pts = np.ascontiguousarray(P["points"], dtype=np.float64)
            nrm = P.get("normals")
            nrm = np.ascontiguousarray(nrm, dtype=np.float64) if nrm is not None else None
            w = P.get("weights")
            w = np.ascontiguousarray(w, dtype=np.float64) if w is not None else None
            keep += [pts, nrm, w]
            k = P.get("kernel", "U")
            a = arr[q]
            a.points = pts.ctypes.data
            a.normals = nrm.ctypes.data if nrm is not None else None
            a.n_c = pts.shape[0]
            a.rho, a.lambda_, a.mu, a.omega = P["rho"], P["lam"], P["mu"], P["omega"]
            a.kernel = {"U": HM_KERNEL_U, "T": HM_KERNEL_T}[k] if isinstance(k, str) else k
            a.pad_ = 0
            a.eta = P.get("eta", 3.0)
            a.leaf_size = P.get("leaf_size", 32)
            a.weights = w.ctypes.data if w is not None else None
        hs = (C.c_void_p * len(problems))()
        st = lib().hm_build_batch(len(problems), arr, eps,
                                  C.byref(opts) if opts is not None else None,
                                  _stream_ptr(stream), hs)
        _check(st, "hm_build_batch")
        return [cls(C.c_void_p(hs[q]), arr[q].n_c) for q in range(len(problems))]

    @classmethod
    def import_(cls, n_c, perm, clusters, blocks, data, opts=None, stream=None):
        perm = np.ascontiguousarray(perm, np.int64)
        clusters = np.ascontiguousarray(clusters, CLUSTER_DTYPE)
        blocks = np.ascontiguousarray(blocks, BLOCK_DTYPE)
        data = np.ascontiguousarray(data, np.complex128)
        h = C.c_void_p()
        st = lib().hm_import(n_c, _np_ptr(perm), len(clusters), _np_ptr(clusters), len(blocks),
                             _np_ptr(blocks), _np_ptr(data),
                             C.byref(opts) if opts is not None else None, _stream_ptr(stream),
                             C.byref(h))
        _check(st, "hm_import")
        return cls(h, n_c)

    def free(self):
        if self.h:
            lib().hm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass

    def matvec(self, x, y=None, stream=None):
        """y = A_H x for cuda complex128 x of shape (3 n_c,) or (3 n_c, nrhs) (column-major)."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        xc = x if x.dim() == 1 else x.t().contiguous()
        yc = y if y.dim() == 1 else torch.empty_like(xc)
        _check(lib().hm_matvec(self.h, nrhs, xc.data_ptr(), yc.data_ptr(), _stream_ptr(stream)),
               "hm_matvec")
        if y.dim() != 1:
            y.copy_(yc.t())
        return y

    def matvec_host(self, x, y=None, stream=None):
        """Same product from host numpy complex128 arrays (copies inside the call)."""
        x = np.asarray(x)
        assert x.dtype == np.complex128 and x.flags.f_contiguous
        if y is None:
            y = np.empty_like(x, order="F")
        nrhs = 1 if x.ndim == 1 else x.shape[1]
        _check(lib().hm_matvec_host(self.h, nrhs, _np_ptr(x), _np_ptr(y), _stream_ptr(stream)),
               "hm_matvec_host")
        return y

    def gmres(self, b, x=None, restart=50, tol=1e-6, maxit=1000, stream=None, check=True):
        import torch
        if x is None:
            x = torch.zeros_like(b)
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        st = lib().hm_gmres(self.h, b.data_ptr(), x.data_ptr(), restart, tol, maxit,
                            C.byref(it), C.byref(rr), _stream_ptr(stream))
        if check and st != HM_ERR_NOCONV:
            _check(st, "hm_gmres")
        return x, it.value, rr.value, st

    @classmethod
    def build2(cls, targets, sources, normals=None, rho=1.0, lam=2.0, mu=1.0, omega=4.0,
               kernel="U", eps=1e-4, eta=3.0, leaf_size=32, opts=None, stream=None):
        """H-matrix between two clouds (hm_build2): rows at the targets, columns at
        the sources (normals and opts weights at the sources)."""
        X = np.ascontiguousarray(targets, dtype=np.float64)
        Y = np.ascontiguousarray(sources, dtype=np.float64)
        N = np.ascontiguousarray(normals, dtype=np.float64) if normals is not None else None
        k = {"U": HM_KERNEL_U, "T": HM_KERNEL_T}[kernel] if isinstance(kernel, str) else kernel
        h = C.c_void_p()
        _check(lib().hm_build2(_np_ptr(X), X.shape[0], _np_ptr(Y), _np_ptr(N) if N is not None else None,
                               Y.shape[0], rho, lam, mu, omega, k, eps, eta, leaf_size,
                               C.byref(opts) if opts is not None else None, _stream_ptr(stream),
                               C.byref(h)), "hm_build2")
        H = cls(h, X.shape[0] + Y.shape[0])
        H.n_targets = X.shape[0]
        return H

    def matvec_sources(self, x, stream=None):
        """A x for a two-cloud handle: x, cuda complex128 (3 n_y,) at the sources;
        returns (3 n_x,) at the targets (the handle's vectors are (targets, sources))."""
        import torch
        nt = 3 * self.n_targets
        xf = torch.zeros(3 * self.n_c, dtype=torch.complex128, device=x.device)
        xf[nt:] = x
        return self.matvec(xf, stream=stream)[:nt]

    @classmethod
    def join(cls, handles, stream=None):
        """The block-diagonal operator of several built handles (hm_batch_join)."""
        arr = (C.c_void_p * len(handles))(*[H.h for H in handles])
        h = C.c_void_p()
        _check(lib().hm_batch_join(len(handles), arr, _stream_ptr(stream), C.byref(h)),
               "hm_batch_join")
        J = cls(h, sum(H.n_c for H in handles))
        J.segments = [H.n_c for H in handles]
        return J

    def gmres_batch(self, b, x=None, restart=50, tol=1e-6, maxit=1000, stream=None, check=True):
        """Lockstep GMRES, one per problem of a joined handle; b: cuda complex128
        concatenated vector.  Returns (x, iters[nprob], relres[nprob], status)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        nprob = len(self.segments)
        it = np.zeros(nprob, np.int32)
        rr = np.zeros(nprob, np.float64)
        st = lib().hm_gmres_batch(self.h, b.data_ptr(), x.data_ptr(), restart, tol, maxit,
                                  _np_ptr(it), _np_ptr(rr), _stream_ptr(stream))
        if check and st != HM_ERR_NOCONV:
            _check(st, "hm_gmres_batch")
        return x, it, rr, st

    def gmres_multi(self, B, X=None, restart=50, tol=1e-6, maxit=1000, stream=None, check=True):
        """Lockstep GMRES for the columns of cuda complex128 B (3 n_c, nrhs).
        Returns (X, iters[nrhs], relres[nrhs], status)."""
        import torch
        nrhs = B.shape[1]
        Bc = B.t().contiguous()
        Xc = torch.zeros_like(Bc)
        it = np.zeros(nrhs, np.int32)
        rr = np.zeros(nrhs, np.float64)
        st = lib().hm_gmres_multi(self.h, nrhs, Bc.data_ptr(), Xc.data_ptr(), restart, tol, maxit,
                                  _np_ptr(it), _np_ptr(rr), _stream_ptr(stream))
        if check and st != HM_ERR_NOCONV:
            _check(st, "hm_gmres_multi")
        if X is None:
            X = torch.empty_like(B)
        X.copy_(Xc.t())
        return X, it, rr, st

    def estimate_error(self, nsample=0, seed=0, stream=None):
        """(||A - A_H||_F, ||A||_F): every point pair (nsample <= 0) or a sample."""
        d = C.c_double(0.0)
        a = C.c_double(0.0)
        _check(lib().hm_estimate_error(self.h, nsample, seed, C.byref(d), C.byref(a),
                                       _stream_ptr(stream)), "hm_estimate_error")
        return d.value, a.value

    def lu_factor(self, eps_lu, stream=None):
        """H-LU factorisation (Sec. 3.2) with truncation tolerance eps_lu."""
        _check(lib().hm_lu_factor(self.h, eps_lu, _stream_ptr(stream)), "hm_lu_factor")

    def lu_solve(self, b, x=None, stream=None):
        """x = (L U)^{-1} b with the H-LU factors; b: 3 n_c (x nrhs) complex128 on the device."""
        import torch
        B = b if b.dim() == 2 else b.reshape(-1, 1)
        Bc = B.t().contiguous()  # column-major
        Xc = torch.empty_like(Bc)
        _check(lib().hm_lu_solve(self.h, Bc.shape[0], Bc.data_ptr(), Xc.data_ptr(),
                                 _stream_ptr(stream)), "hm_lu_solve")
        X = Xc.t()
        if b.dim() == 1:
            X = X.reshape(-1)
        if x is not None:
            x.copy_(X)
            return x
        return X.contiguous()

    def lu_info(self):
        """(seconds, stored complex entries, kernel launches) of the H-LU factorisation."""
        sec = C.c_double(0.0)
        ent = C.c_int64(0)
        lau = C.c_int64(0)
        _check(lib().hm_lu_info(self.h, C.byref(sec), C.byref(ent), C.byref(lau)), "hm_lu_info")
        return sec.value, ent.value, lau.value

    def profile_matvec(self, reps=10, stream=None):
        """Average per-kernel device times (ms) of the product and its algorithmic bytes."""
        ms = (C.c_double * 4)()
        by = (C.c_int64 * 3)()
        _check(lib().hm_profile_matvec(self.h, reps, ms, by, _stream_ptr(stream)),
               "hm_profile_matvec")
        return {"ms": {"gather": ms[0], "phase1": ms[1], "phase2": ms[2], "scatter": ms[3]},
                "bytes": {"phase1": by[0], "phase2": by[1], "matvec": by[2]}}

    def profile_matvec_multi(self, reps=10, stream=None):
        """Per-kernel device times (ms) of one tensor-core block product of
        HM_NRHS_BLOCK right-hand sides (BF16 storage) and its algorithmic bytes."""
        ms = (C.c_double * 4)()
        by = (C.c_int64 * 1)()
        _check(lib().hm_profile_matvec_multi(self.h, reps, ms, by, _stream_ptr(stream)),
               "hm_profile_matvec_multi")
        return {"ms": {"gather": ms[0], "phase1": ms[1], "phase2": ms[2], "scatter": ms[3]},
                "bytes": by[0]}

    def stats(self):
        need = C.c_size_t(0)
        lib().hm_stats(self.h, None, 0, C.byref(need))
        buf = C.create_string_buffer(need.value)
        _check(lib().hm_stats(self.h, buf, need.value, None), "hm_stats")
        return json.loads(buf.value.decode())

    def rank_samples(self):
        """(features n x 6, targets n) of the admissible blocks (float32, host)."""
        n = C.c_int64(0)
        _check(lib().hm_rank_samples(self.h, None, None, C.byref(n)), "hm_rank_samples")
        f = np.zeros((n.value, 6), np.float32)
        t = np.zeros(n.value, np.float32)
        _check(lib().hm_rank_samples(self.h, _np_ptr(f), _np_ptr(t), C.byref(n)), "hm_rank_samples")
        return f, t

    def sizes(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().hm_sizes(self.h, C.byref(a), C.byref(b), C.byref(c)), "hm_sizes")
        return a.value, b.value, c.value

    def tree(self):
        nc, ncl, _ = self.sizes()
        perm = np.zeros(nc, np.int64)
        cl = np.zeros(ncl, CLUSTER_DTYPE)
        _check(lib().hm_get_tree(self.h, _np_ptr(perm), _np_ptr(cl)), "hm_get_tree")
        return perm, cl

    def blocks(self):
        _, _, nb = self.sizes()
        b = np.zeros(nb, BLOCK_DTYPE)
        _check(lib().hm_get_blocks(self.h, _np_ptr(b)), "hm_get_blocks")
        return b

    def block_data(self, b, blocks=None, clusters=None):
        if blocks is None:
            blocks = self.blocks()
        if clusters is None:
            clusters = self.tree()[1]
        B = blocks[b]
        t, s = clusters[B["tau"]], clusters[B["sigma"]]
        m3, n3 = 3 * (t["end"] - t["begin"]), 3 * (s["end"] - s["begin"])
        if not B["admissible"]:
            a = np.zeros((n3, m3), np.complex128)
            _check(lib().hm_get_block_data(self.h, b, _np_ptr(a), None), "hm_get_block_data")
            return a.T.copy()
        r = int(B["rank"])
        u = np.zeros((max(r, 1), m3), np.complex128)
        v = np.zeros((max(r, 1), n3), np.complex128)
        _check(lib().hm_get_block_data(self.h, b, _np_ptr(u), _np_ptr(v)), "hm_get_block_data")
        return u[:r].T.copy(), v[:r].T.copy()
