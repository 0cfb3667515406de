"""ChASE for dense complex Hermitian BSE Hamiltonians on one GB300 GPU.

Thin ctypes binding of the C ABI in include/bsechase.h (libbsechase.so, built
in-tree by paper_2006_08498_gb300.build).  Every step of the solver runs in
the library's CUDA kernels; this module only marshals arguments.  PyTorch
supplies device memory and the stream.

Column-major matrices are represented as torch tensors with strides
(1, ld): ``colmajor_empty(rows, cols)`` allocates one, ``t.T.contiguous().T``
converts any tensor.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libbsechase.so")

BSE_OK, BSE_EINVAL, BSE_ENOMEM, BSE_ENOCONV = 0, -1, -2, -3
BSE_ENONFINITE, BSE_ETIMEOUT, BSE_ECUDA, BSE_EBUSY = -4, -5, -6, -7
CHASE_FP64, CHASE_MIXED_FP32, CHASE_MIXED_BF16X3, CHASE_FP64_DFMA = 0, 1, 2, 3

# Every symbol include/bsechase.h declares.
ABI_SYMBOLS = (
    "bsechase_create", "bsechase_destroy", "bsechase_strerror", "bsechase_last_error",
    "bsechase_set_wait_limit", "bsechase_host_alloc", "bsechase_host_free",
    "bse_dim", "bse_build_hamiltonian", "chase_solve", "chase_solve_host", "chase_solve_bse",
    "chase_lanczos", "chase_filter", "chase_qr", "chase_rayleigh_ritz", "chase_hemm",
    "chase_hemm_slices",
    "chase_gram", "chase_gram_noalloc",
    "chase_server_create", "chase_server_submit", "chase_server_poll", "chase_server_wait",
    "chase_server_evecs", "chase_server_release", "chase_server_info", "chase_server_destroy",
    "chase_server_batching", "chase_server_batch_stats",
)


class BseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_strerror(status), status, msg))
        self.status = status


class Model(ctypes.Structure):
    _fields_ = [("band_gap", ctypes.c_double), ("w0", ctypes.c_double),
                ("x0", ctypes.c_double), ("jitter", ctypes.c_double),
                ("dispersion", ctypes.c_double), ("rank_x", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("deg_init", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("lanczos_steps", ctypes.c_int), ("lanczos_vecs", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("d_V0", ctypes.c_void_p),
                ("ldv0", ctypes.c_int64), ("n_v0", ctypes.c_int),
                ("degree_group", ctypes.c_int), ("nex_damping", ctypes.c_double),
                ("half_storage", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("locked", ctypes.c_int),
                ("matvecs", ctypes.c_int64), ("filter_matvecs", ctypes.c_int64),
                ("ms_lanczos", ctypes.c_double), ("ms_filter", ctypes.c_double),
                ("ms_qr", ctypes.c_double), ("ms_rr", ctypes.c_double),
                ("ms_resid", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("filter_tflops", ctypes.c_double), ("norm_est", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("lower", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("filter_launches", ctypes.c_int64), ("filter_matvecs_low", ctypes.c_int64),
                ("tc_kernel_ms", ctypes.c_double), ("tc_kernel_launches", ctypes.c_int64),
                ("tc_kernel_tflops", ctypes.c_double), ("nex_used", ctypes.c_int),
                ("filter_matvecs_mid", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("ms_h2d", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("Nk", ctypes.c_int), ("Nv", ctypes.c_int),
                ("Nc", ctypes.c_int), ("use_model", ctypes.c_int), ("model", Model),
                ("nev", ctypes.c_int), ("nex", ctypes.c_int), ("tol", ctypes.c_double),
                ("deg_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("warm_ticket", ctypes.c_uint64), ("degree_group", ctypes.c_int),
                ("nex_damping", ctypes.c_double), ("d_H", ctypes.c_void_p),
                ("ldh", ctypes.c_int64), ("half_storage", ctypes.c_int), ("h_free", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("has_evecs", ctypes.c_int), ("N", ctypes.c_int64),
                ("nev", ctypes.c_int), ("evals", ctypes.POINTER(ctypes.c_double)),
                ("resid", ctypes.POINTER(ctypes.c_double)), ("stats", Stats),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double)]

    def as_dict(self):
        n = self.nev
        return dict(status=self.status, N=self.N, nev=n, has_evecs=bool(self.has_evecs),
                    evals=np.array(self.evals[:n]) if self.evals else None,
                    resid=np.array(self.resid[:n]) if self.resid else None,
                    stats=self.stats.as_dict(), t_submit=self.t_submit,
                    t_start=self.t_start, t_end=self.t_end,
                    latency=self.t_end - self.t_submit)


DEFAULT_MODEL = dict(band_gap=2.0, w0=0.3, x0=0.5, jitter=0.01, dispersion=1.0, rank_x=8)

_lib = None


def library_path():
    return _LIBPATH


def load():
    """Load libbsechase.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise RuntimeError("libbsechase.so is not built; run "
                           "`python -m paper_2006_08498_gb300.build` (nvcc, sm_103a)")
    L = ctypes.CDLL(_LIBPATH)
    P, i64, i32, dbl, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                             ctypes.c_double, ctypes.c_uint64)
    DP = ctypes.POINTER(ctypes.c_double)
    L.bsechase_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32, P]
    L.bsechase_create.restype = i32
    L.bsechase_destroy.argtypes = [P]
    L.bsechase_destroy.restype = None
    L.bsechase_strerror.argtypes = [i32]
    L.bsechase_strerror.restype = ctypes.c_char_p
    L.bsechase_last_error.argtypes = [P]
    L.bsechase_last_error.restype = ctypes.c_char_p
    L.bsechase_set_wait_limit.argtypes = [P, dbl]
    L.bsechase_set_wait_limit.restype = i32
    L.bsechase_host_alloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
    L.bsechase_host_alloc.restype = i32
    L.bsechase_host_free.argtypes = [P]
    L.bsechase_host_free.restype = i32
    L.bse_dim.argtypes = [i32, i32, i32]
    L.bse_dim.restype = i64
    L.bse_build_hamiltonian.argtypes = [P, u64, i32, i32, i32, ctypes.POINTER(Model), P, i64]
    L.bse_build_hamiltonian.restype = i32
    L.chase_solve.argtypes = [P, P, i64, i64, i32, i32, dbl, i32, i32, ctypes.POINTER(Opts),
                              DP, P, i64, DP, ctypes.POINTER(Stats)]
    L.chase_solve.restype = i32
    L.chase_solve_host.argtypes = L.chase_solve.argtypes
    L.chase_solve_host.restype = i32
    L.chase_solve_bse.argtypes = [P, u64, i32, i32, i32, ctypes.POINTER(Model), i32, i32, dbl, i32,
                                  i32, ctypes.POINTER(Opts), DP, P, i64, DP, ctypes.POINTER(Stats)]
    L.chase_solve_bse.restype = i32
    L.chase_lanczos.argtypes = [P, P, i64, i64, i32, i32, i32, u64, i32, DP]
    L.chase_lanczos.restype = i32
    L.chase_filter.argtypes = [P, P, i64, i64, P, i64, i32, ctypes.POINTER(ctypes.c_int),
                               dbl, dbl, dbl, i32, ctypes.POINTER(ctypes.c_int64)]
    L.chase_filter.restype = i32
    L.chase_qr.argtypes = [P, P, i64, i32, P, i64, i64, i32]
    L.chase_qr.restype = i32
    L.chase_rayleigh_ritz.argtypes = [P, P, i64, i64, P, i64, i32, i32, DP, P, P, dbl, DP]
    L.chase_rayleigh_ritz.restype = i32
    L.chase_hemm.argtypes = [P, P, i64, i64, P, i64, i32, P, i64, i32]
    L.chase_hemm.restype = i32
    L.chase_hemm_slices.argtypes = L.chase_hemm.argtypes + [i32]
    L.chase_hemm_slices.restype = i32
    L.chase_gram.argtypes = [P, P, i64, P, i64, i64, i32, i32, P, i64]
    L.chase_gram.restype = i32
    L.chase_gram_noalloc.argtypes = [P, i64, P, i64, i64, i32, i32, P, i64, P]
    L.chase_gram_noalloc.restype = i32
    sz = ctypes.c_size_t
    L.chase_server_create.argtypes = [P, sz, i32]
    L.chase_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.chase_server_poll.argtypes = [P, u64, ctypes.POINTER(Result)]
    L.chase_server_wait.argtypes = [P, u64, dbl, ctypes.POINTER(Result)]
    L.chase_server_evecs.argtypes = [P, u64, P, i64]
    L.chase_server_release.argtypes = [P, u64]
    L.chase_server_info.argtypes = [P, ctypes.POINTER(sz), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32)]
    L.chase_server_destroy.argtypes = [P]
    L.chase_server_batching.argtypes = [P, i32, dbl]
    L.chase_server_batch_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                           ctypes.POINTER(i32)]
    for f in ("create", "submit", "poll", "wait", "evecs", "release", "info", "destroy",
              "batching", "batch_stats"):
        getattr(L, "chase_server_" + f).restype = i32
    _lib = L
    return L


def _strerror(status):
    try:
        return load().bsechase_strerror(status).decode()
    except Exception:
        return "status"


def bse_dim(Nk, Nv, Nc):
    return int(load().bse_dim(Nk, Nv, Nc))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ld(t):
    """Leading dimension of a column-major (strides (1, ld)) tensor/array."""
    if hasattr(t, "stride") and callable(t.stride):
        s = t.stride()
        if s[0] != 1:
            raise ValueError("matrix must be column-major (stride (1, ld))")
        return max(s[1], t.shape[0]) if t.dim() == 2 else t.shape[0]
    if not t.flags["F_CONTIGUOUS"]:
        raise ValueError("array must be Fortran-ordered")
    return t.shape[0]


def gram_noalloc(A, B, out, stream=None):
    """G = A^H B through the allocation-free entry point chase_gram_noalloc:
    the caller provides the output `out` (m1 x m2, column-major, on A's
    device); the library allocates nothing.  Runs on `stream` (a
    torch.cuda.Stream; default: the current stream) and returns the status."""
    import torch
    K, m1 = A.shape
    m2 = B.shape[1]
    if B.device != A.device or out.device != A.device:
        raise ValueError("A, B and out must be on one device")
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    # the entry point runs on the current device: make it A's
    with torch.cuda.device(A.device):
        return load().chase_gram_noalloc(ctypes.c_void_p(A.data_ptr()), _ld(A),
                                         ctypes.c_void_p(B.data_ptr()), _ld(B), K, m1, m2,
                                         ctypes.c_void_p(out.data_ptr()), _ld(out),
                                         ctypes.c_void_p(stream.cuda_stream))


def host_empty(shape, dtype=np.complex128, order="F"):
    """Uninitialised numpy array in page-locked host memory from
    bsechase_host_alloc (freed when the array and its views are gone): the
    host buffers of solve_host copy at the host link's full rate."""
    import weakref
    dtype = np.dtype(dtype)
    nbytes = int(np.prod(shape)) * dtype.itemsize
    p = ctypes.c_void_p()
    rc = load().bsechase_host_alloc(ctypes.byref(p), max(nbytes, 1))
    if rc != BSE_OK:
        raise BseError(rc, "host allocation of %d bytes" % nbytes)
    buf = (ctypes.c_char * max(nbytes, 1)).from_address(p.value)
    weakref.finalize(buf, load().bsechase_host_free, p.value)
    return np.frombuffer(buf, dtype=dtype, count=int(np.prod(shape))).reshape(shape, order=order)


def colmajor_empty(rows, cols, device="cuda", dtype=None):
    """Uninitialised column-major (rows x cols) torch tensor."""
    import torch
    dtype = torch.complex128 if dtype is None else dtype
    return torch.empty((cols, rows), dtype=dtype, device=device).T


class Context:
    """A solver context on one device; work runs on torch's current stream
    unless `stream` (a torch.cuda.Stream) is given."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        L = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = L.bsechase_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if rc != BSE_OK:
            raise BseError(rc, "bsechase_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().bsechase_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_wait_limit(self, seconds):
        """Time limit of the bounded waits in the tensor-core kernels."""
        self._check(load().bsechase_set_wait_limit(self._h, float(seconds)))

    def _check(self, rc, allow=(BSE_OK,)):
        if rc not in allow:
            raise BseError(rc, load().bsechase_last_error(self._h).decode())
        return rc

    # ------------------------------------------------------------ generator
    def build_hamiltonian(self, seed, Nk, Nv, Nc, model=None, out=None):
        """Seeded synthetic Eq. (1) Hamiltonian as a column-major N x N
        complex128 device tensor."""
        N = bse_dim(Nk, Nv, Nc)
        if N < 1:
            raise ValueError("bad (Nk, Nv, Nc)")
        if out is None:
            out = colmajor_empty(N, N, device="cuda:%d" % self.device)
        md = dict(DEFAULT_MODEL)
        if model:
            md.update(model)
        m = Model(md["band_gap"], md["w0"], md["x0"], md["jitter"], md["dispersion"],
                  int(md["rank_x"]))
        rc = load().bse_build_hamiltonian(self._h, seed, Nk, Nv, Nc, ctypes.byref(m),
                                          ctypes.c_void_p(out.data_ptr()), _ld(out))
        self._check(rc)
        return out

    # -------------------------------------------------------------- solve
    @staticmethod
    def _opts(deg_init, max_iter, lanczos_steps, lanczos_vecs, seed, V0, degree_group=0,
              nex_damping=0.0, half_storage=False):
        o = Opts(deg_init, max_iter, lanczos_steps, lanczos_vecs, seed, None, 0, 0, degree_group,
                 nex_damping, int(half_storage))
        if V0 is not None:
            o.d_V0 = ctypes.c_void_p(V0.data_ptr())
            o.ldv0 = _ld(V0)
            o.n_v0 = V0.shape[1]
        return o

    def solve(self, H, nev, nex, tol=1e-10, deg_max=36, precision=CHASE_FP64, deg_init=20,
              max_iter=50, lanczos_steps=25, lanczos_vecs=4, seed=0, V0=None,
              evecs=None, allow_noconv=False, degree_group=0, nex_damping=0.0,
              half_storage=False):
        """Lowest nev eigenpairs of the device Hermitian H (column-major).
        Returns (evals ndarray, evecs tensor N x nev, resid ndarray, stats).
        half_storage: the tensor-core slices of H's lower triangle only
        (chase_opts.half_storage)."""
        N = H.shape[0]
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        if evecs is None:
            evecs = colmajor_empty(N, nev, device=H.device)
        st = Stats()
        o = self._opts(deg_init, max_iter, lanczos_steps, lanczos_vecs, seed, V0, degree_group,
                       nex_damping, half_storage)
        rc = load().chase_solve(self._h, ctypes.c_void_p(H.data_ptr()), N, _ld(H), nev, nex,
                                tol, deg_max, precision, ctypes.byref(o), _dp(evals),
                                ctypes.c_void_p(evecs.data_ptr()), _ld(evecs), _dp(resid),
                                ctypes.byref(st))
        self._check(rc, (BSE_OK, BSE_ENOCONV) if allow_noconv else (BSE_OK,))
        d = st.as_dict()
        d["status"] = rc
        return evals, evecs, resid, d

    def solve_bse(self, seed, Nk, Nv, Nc, nev, nex, tol=1e-10, deg_max=36, precision=CHASE_FP64,
                  model=None, deg_init=20, max_iter=50, lanczos_steps=25, lanczos_vecs=4,
                  seed_start=0, evecs=None, degree_group=0, nex_damping=0.0,
                  half_storage=False):
        """Lowest nev eigenpairs of the synthetic Hamiltonian (seed, Nk, Nv,
        Nc, model) without storing it (chase_solve_bse; with half_storage only
        the lower triangle's slices are made).  seed_start seeds the
        Lanczos and start vectors (`seed` of solve()).  Returns (evals, evecs
        tensor N x nev, resid, stats)."""
        torch = self._torch
        N = Nk * Nv * Nc
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        if evecs is None:
            evecs = colmajor_empty(N, nev, device=torch.device("cuda", self.device))
        md = dict(DEFAULT_MODEL)
        if model:
            md.update(model)
        mdl = Model(md["band_gap"], md["w0"], md["x0"], md["jitter"], md["dispersion"],
                    int(md["rank_x"]))
        st = Stats()
        o = self._opts(deg_init, max_iter, lanczos_steps, lanczos_vecs, seed_start, None,
                       degree_group, nex_damping, half_storage)
        rc = load().chase_solve_bse(self._h, seed, Nk, Nv, Nc, ctypes.byref(mdl), nev, nex, tol,
                                    deg_max, precision, ctypes.byref(o), _dp(evals),
                                    ctypes.c_void_p(evecs.data_ptr()), _ld(evecs), _dp(resid),
                                    ctypes.byref(st))
        self._check(rc)
        d = st.as_dict()
        d["status"] = rc
        return evals, evecs, resid, d

    def solve_host(self, H, nev, nex, tol=1e-10, deg_max=36, precision=CHASE_FP64,
                   deg_init=20, max_iter=50, lanczos_steps=25, lanczos_vecs=4, seed=0,
                   evecs=None, degree_group=0, half_storage=False):
        """As solve(), with H and the eigenvectors in host memory (Fortran-
        ordered complex128 numpy arrays, ideally page-locked: host_empty)."""
        N = H.shape[0]
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        if evecs is None:
            evecs = np.zeros((N, nev), dtype=np.complex128, order="F")
        st = Stats()
        o = self._opts(deg_init, max_iter, lanczos_steps, lanczos_vecs, seed, None, degree_group,
                       0.0, half_storage)
        hp = H.data_ptr() if hasattr(H, "data_ptr") else H.ctypes.data
        ep = evecs.data_ptr() if hasattr(evecs, "data_ptr") else evecs.ctypes.data
        rc = load().chase_solve_host(self._h, ctypes.c_void_p(hp), N, _ld(H), nev, nex, tol,
                                     deg_max, precision, ctypes.byref(o), _dp(evals),
                                     ctypes.c_void_p(ep), _ld(evecs), _dp(resid),
                                     ctypes.byref(st))
        self._check(rc)
        d = st.as_dict()
        d["status"] = rc
        return evals, evecs, resid, d

    # ------------------------------------------------------------- phases
    def lanczos(self, H, m, steps=25, runs=4, seed=0, precision=CHASE_FP64):
        out = np.zeros(4)
        rc = load().chase_lanczos(self._h, ctypes.c_void_p(H.data_ptr()), H.shape[0], _ld(H),
                                  m, steps, runs, seed, precision, _dp(out))
        self._check(rc)
        return dict(beta=out[0], mu_1=out[1], mu_m=out[2], norm_est=out[3])

    def filter(self, H, V, degrees, lower, c, e, precision=CHASE_FP64):
        """In-place Chebyshev filter of the columns of V (ld must equal N)."""
        deg = np.ascontiguousarray(degrees, dtype=np.int32)
        mv = ctypes.c_int64(0)
        rc = load().chase_filter(self._h, ctypes.c_void_p(H.data_ptr()), H.shape[0], _ld(H),
                                 ctypes.c_void_p(V.data_ptr()), _ld(V), V.shape[1],
                                 deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), lower, c, e,
                                 precision, ctypes.byref(mv))
        self._check(rc)
        return mv.value

    def qr(self, V, L=None):
        N, m = V.shape
        k = 0 if L is None else L.shape[1]
        rc = load().chase_qr(self._h, ctypes.c_void_p(L.data_ptr() if k else 0),
                             _ld(L) if k else N, k, ctypes.c_void_p(V.data_ptr()), _ld(V), N, m)
        self._check(rc)
        return V

    def hemm(self, H, Y, precision=CHASE_FP64, out=None, slices=None, half_storage=False):
        """C = H Y (the filter's product) as a new column-major tensor; with
        `slices` (4, 5 or 6) or half_storage, the tensor-core product on that
        many slices (default 6) of all of H or of its lower triangle
        (chase_hemm_slices) instead of `precision`'s."""
        N, n = Y.shape
        C = colmajor_empty(N, n, device=Y.device) if out is None else out
        if slices is None and not half_storage:
            fn, last = load().chase_hemm, (precision,)
        else:
            fn, last = load().chase_hemm_slices, (6 if slices is None else slices, int(half_storage))
        rc = fn(self._h, ctypes.c_void_p(H.data_ptr()), N, _ld(H), ctypes.c_void_p(Y.data_ptr()),
                _ld(Y), n, ctypes.c_void_p(C.data_ptr()), _ld(C), *last)
        self._check(rc)
        return C

    def gram(self, A, B, out=None):
        """G = A^H B (m1 x m2, column-major) for tall A (K x m1), B (K x m2)."""
        K, m1 = A.shape
        m2 = B.shape[1]
        G = colmajor_empty(m1, m2, device=A.device) if out is None else out
        rc = load().chase_gram(self._h, ctypes.c_void_p(A.data_ptr()), _ld(A),
                               ctypes.c_void_p(B.data_ptr()), _ld(B), K, m1, m2,
                               ctypes.c_void_p(G.data_ptr()), _ld(G))
        self._check(rc)
        return G

    # ------------------------------------------------------------ serving
    def server_create(self, hbm_budget_bytes, max_slots):
        self._check(load().chase_server_create(self._h, int(hbm_budget_bytes), max_slots))

    def server_destroy(self):
        self._check(load().chase_server_destroy(self._h))

    def submit(self, seed, Nk, Nv, Nc, nev, nex, tol=1e-10, deg_max=36, precision=CHASE_FP64,
               model=None, warm_ticket=0, degree_group=0, nex_damping=0.0, H=None,
               half_storage=False, h_free=False):
        """Queue a solve of the synthetic Hamiltonian (seed, Nk, Nv, Nc), or of
        the caller's device matrix H (N = Nk Nv Nc, column-major; kept alive
        and unchanged by the caller until the request finishes); returns its
        ticket.  half_storage: slices of H's lower triangle only; h_free: the
        synthetic H is not stored (chase_solve_bse)."""
        md = dict(DEFAULT_MODEL)
        if model:
            md.update(model)
        r = Request(seed, Nk, Nv, Nc, 1 if model else 0,
                    Model(md["band_gap"], md["w0"], md["x0"], md["jitter"], md["dispersion"],
                          int(md["rank_x"])),
                    nev, nex, tol, deg_max, precision, warm_ticket, degree_group, nex_damping,
                    None if H is None else ctypes.c_void_p(H.data_ptr()),
                    0 if H is None else _ld(H), int(half_storage), int(h_free))
        t = ctypes.c_uint64(0)
        self._check(load().chase_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """Result dict, or None while pending."""
        out = Result()
        rc = load().chase_server_poll(self._h, ticket, ctypes.byref(out))
        if rc == BSE_EBUSY:
            return None
        self._check(rc)
        return out.as_dict()

    def wait(self, ticket, timeout_s=600.0):
        """Result dict; raises BseError(BSE_ETIMEOUT) if still pending."""
        out = Result()
        self._check(load().chase_server_wait(self._h, ticket, timeout_s, ctypes.byref(out)))
        return out.as_dict()

    def fetch_evecs(self, ticket, N, nev):
        V = colmajor_empty(N, nev, device="cuda:%d" % self.device)
        self._check(load().chase_server_evecs(self._h, ticket, ctypes.c_void_p(V.data_ptr()),
                                              _ld(V)))
        return V

    def release(self, ticket):
        return load().chase_server_release(self._h, ticket)

    def server_info(self):
        held, q, r = ctypes.c_size_t(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(load().chase_server_info(self._h, ctypes.byref(held), ctypes.byref(q),
                                             ctypes.byref(r)))
        return dict(held_bytes=held.value, queued=q.value, running=r.value)

    def server_batching(self, enabled=True, window_s=0.0):
        """Turn the server's product batching on (with this window) or off."""
        self._check(load().chase_server_batching(self._h, 1 if enabled else 0, float(window_s)))

    def server_batch_stats(self):
        n, p, mx = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(0)
        self._check(load().chase_server_batch_stats(self._h, ctypes.byref(n), ctypes.byref(p),
                                                    ctypes.byref(mx)))
        return dict(launches=n.value, products=p.value, max_products=mx.value)

    def rayleigh_ritz(self, H, Q, norm=1.0, precision=CHASE_FP64):
        N, m = Q.shape
        theta = np.zeros(m)
        resid = np.zeros(m)
        V = colmajor_empty(N, m, device=Q.device)
        HV = colmajor_empty(N, m, device=Q.device)
        rc = load().chase_rayleigh_ritz(self._h, ctypes.c_void_p(H.data_ptr()), N, _ld(H),
                                        ctypes.c_void_p(Q.data_ptr()), _ld(Q), m, precision,
                                        _dp(theta),
                                        ctypes.c_void_p(V.data_ptr()),
                                        ctypes.c_void_p(HV.data_ptr()), norm, _dp(resid))
        self._check(rc)
        return theta, V, HV, resid
