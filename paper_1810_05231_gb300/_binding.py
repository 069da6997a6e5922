"""ctypes binding of ``include/proxsdp_gpu.h`` (argument marshalling only).

Every function here converts Python / numpy / torch arguments to the C ABI's
plain pointers and sizes and calls the library; all computation happens in
the library's CUDA kernels.  The library is loaded from this package
directory; if it is missing the import fails loudly (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libproxsdp_gpu.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_BAD_STATE = -4
ERR_UNSUPPORTED = -5
ERR_TIMEOUT = -6

CONVERGED = 0
MAX_ITER = 1
TIME_LIMIT = 2
STALLED_AT_MAX_RANK = 3
NUMERIC_ERROR = 4

OP_EXPLICIT = 0  # settings.operator_form: S^k written to device memory and multiplied
OP_FACTORED = 1  # S^k applied from the factors of X^k and the sparse C + M*(y^k)
OP_AUTO = 2      # factored when the union pattern holds at most n*n/8 entries

EXPORTED = [
    "proxsdp_gpu_settings_default",
    "proxsdp_gpu_create",
    "proxsdp_gpu_set_problem",
    "proxsdp_gpu_solve",
    "proxsdp_gpu_get_primal_dual",
    "proxsdp_gpu_get_saved_pair",
    "proxsdp_gpu_set_iterate",
    "proxsdp_gpu_iterate",
    "proxsdp_gpu_resume",
    "proxsdp_gpu_set_box",
    "proxsdp_gpu_get_box_dual",
    "proxsdp_gpu_destroy",
    "proxsdp_gpu_last_error",
    "proxsdp_gpu_aproj",
    "proxsdp_gpu_block_matvec",
    "proxsdp_gpu_sym_eig",
    "proxsdp_gpu_analyze_problem",
    "proxsdp_gpu_aproj_noalloc",
    "proxsdp_gpu_solve_batch",
]


class Settings(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int64),
        ("time_limit_s", ctypes.c_double),
        ("full_eig", ctypes.c_int),
        ("rank_init", ctypes.c_int),
        ("block_size", ctypes.c_int),
        ("window", ctypes.c_int),
        ("eps_lambda", ctypes.c_double),
        ("alpha_frac", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("normalize_rows", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("max_rank", ctypes.c_int),
        ("lanczos_steps", ctypes.c_int),
        ("lanczos_max_cycles", ctypes.c_int),
        ("lanczos_tol", ctypes.c_double),
        ("guard", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("operator_form", ctypes.c_int),
        ("memory_limit_bytes", ctypes.c_int64),
        ("at_max_rank", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("final_rank", ctypes.c_int),
        ("iters", ctypes.c_int64),
        ("rank_changes", ctypes.c_int),
        ("primal_obj", ctypes.c_double),
        ("dual_obj", ctypes.c_double),
        ("rel_primal_res", ctypes.c_double),
        ("rel_dual_res", ctypes.c_double),
        ("rel_gap", ctypes.c_double),
        ("eps_primal", ctypes.c_double),
        ("eps_dual", ctypes.c_double),
        ("lambda_r", ctypes.c_double),
        ("solve_seconds", ctypes.c_double),
        ("matvecs", ctypes.c_int64),
        ("lanczos_cycles", ctypes.c_int64),
        ("lanczos_unconverged", ctypes.c_int64),
        ("alpha", ctypes.c_double),
        ("norm_M", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib():
    """Load ``libproxsdp_gpu.so`` (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} not found: build it first (python -m paper_1810_05231_gb300.build); "
            "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    L.proxsdp_gpu_settings_default.argtypes = [ctypes.POINTER(Settings)]
    L.proxsdp_gpu_create.argtypes = [ctypes.POINTER(Settings), i32, vp, ctypes.POINTER(vp)]
    L.proxsdp_gpu_set_problem.argtypes = [vp, i64, dp, i64, dp, dp, i64, i64, dp, dp, dp, dp]
    L.proxsdp_gpu_solve.argtypes = [vp, ctypes.POINTER(Info)]
    L.proxsdp_gpu_get_primal_dual.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(i64)]
    L.proxsdp_gpu_get_saved_pair.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.proxsdp_gpu_set_iterate.argtypes = [vp, i32, dp, dp, dp]
    L.proxsdp_gpu_iterate.argtypes = [vp, i64, ctypes.POINTER(Info)]
    L.proxsdp_gpu_resume.argtypes = [vp, i64, ctypes.POINTER(Info)]
    L.proxsdp_gpu_set_box.argtypes = [vp, ctypes.c_double]
    L.proxsdp_gpu_get_box_dual.argtypes = [vp, dp, dp]
    L.proxsdp_gpu_solve_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Info), i32]
    L.proxsdp_gpu_destroy.argtypes = [vp]
    L.proxsdp_gpu_destroy.restype = None
    L.proxsdp_gpu_last_error.argtypes = [vp]
    L.proxsdp_gpu_last_error.restype = ctypes.c_char_p
    L.proxsdp_gpu_aproj.argtypes = [vp, i64, i64, i32, vp, i64, vp, vp, ctypes.POINTER(Settings), vp,
                                    ctypes.POINTER(Info)]
    L.proxsdp_gpu_block_matvec.argtypes = [vp, i64, i64, vp, i64, i32, vp, i64, vp]
    L.proxsdp_gpu_aproj_noalloc.argtypes = [vp, i64, i64, i32, vp, i64, vp, vp, ctypes.POINTER(Settings), vp,
                                            ctypes.POINTER(Info)]
    L.proxsdp_gpu_sym_eig.argtypes = [vp, i32, vp, vp, vp]
    L.proxsdp_gpu_analyze_problem.argtypes = [ctypes.POINTER(Settings), i64, dp, i64, dp, dp, i64, i64, dp, dp, dp,
                                              dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
    for name in EXPORTED:
        if name not in ("proxsdp_gpu_destroy", "proxsdp_gpu_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class ProxSDPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"proxsdp_gpu error {code}: {msg}")
        self.code = code


def _check(code, handle=None):
    if code != OK:
        msg = lib().proxsdp_gpu_last_error(handle)
        raise ProxSDPError(code, msg.decode() if msg else "")


def default_settings(**kw) -> Settings:
    s = Settings()
    lib().proxsdp_gpu_settings_default(ctypes.byref(s))
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    return s


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int64)


class Solver:
    """A ``proxsdp_gpu_t`` handle (create / set_problem / solve / get_primal_dual)."""

    def __init__(self, settings: Settings | None = None, device: int = 0, stream=None, **kw):
        if settings is None:
            settings = default_settings(**kw)
        self.settings = settings
        h = ctypes.c_void_p()
        _check(lib().proxsdp_gpu_create(ctypes.byref(settings), device,
                                        ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.h = h
        self.n = None
        self.m = None

    def close(self):
        if getattr(self, "h", None):
            lib().proxsdp_gpu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_problem(self, n, m_eq, A_rowptr, A_col, A_val, rhs, C_dense=None, C_idx=None, C_val=None):
        rowptr, col, val, b = _i64(A_rowptr), _i64(A_col), _f64(A_val), _f64(rhs)
        Cd = _f64(C_dense)
        ci, cv = _i64(C_idx), _f64(C_val)
        c_nnz = 0 if ci is None else int(ci.shape[0])
        m = int(b.shape[0])
        self._keep = (rowptr, col, val, b, Cd, ci, cv)
        _check(lib().proxsdp_gpu_set_problem(self.h, int(n), _ptr(Cd), c_nnz, _ptr(ci), _ptr(cv), m, int(m_eq),
                                             _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b)), self.h)
        self.n, self.m = int(n), m

    def set_instance(self, p):
        """From an object with the fields of ``sdp_instances.SDPProblem``."""
        self.set_problem(p.n, p.m_eq, p.A_rowptr, p.A_col, p.A_val, p.rhs, C_dense=p.C_dense,
                         C_idx=p.C_idx, C_val=p.C_val)

    def solve(self) -> Info:
        info = Info()
        _check(lib().proxsdp_gpu_solve(self.h, ctypes.byref(info)), self.h)
        return info

    def iterate(self, iters: int) -> Info:
        info = Info()
        _check(lib().proxsdp_gpu_iterate(self.h, int(iters), ctypes.byref(info)), self.h)
        return info

    def resume(self, max_iters: int = -1) -> Info:
        """Continue Alg. 2 from the current iterate until its stop test holds
        (at most ``max_iters`` more iterations; < 0: up to ``max_iter`` in total)."""
        info = Info()
        _check(lib().proxsdp_gpu_resume(self.h, int(max_iters), ctypes.byref(info)), self.h)
        return info

    def set_box(self, u: float = 1.0):
        """Add -u <= X_ij <= u (i != j) as the structured element-wise box rows."""
        _check(lib().proxsdp_gpu_set_box(self.h, float(u)), self.h)

    def get_box_dual(self):
        """Duals (paper's sign, original scaling) of X_ij <= u and -X_ij <= u, n x n each."""
        n = self.n
        Yu, Yl = np.empty((n, n)), np.empty((n, n))
        _check(lib().proxsdp_gpu_get_box_dual(self.h, _ptr(Yu), _ptr(Yl)), self.h)
        return Yu, Yl

    def set_iterate(self, V, lam, y=None):
        V = np.asfortranarray(V, dtype=np.float64)
        lam = _f64(lam)
        y = _f64(y)
        r = int(lam.shape[0])
        _check(lib().proxsdp_gpu_set_iterate(self.h, r, V.ctypes.data_as(ctypes.c_void_p), _ptr(lam), _ptr(y)),
               self.h)

    def get_primal_dual(self, want_X=True):
        n, m = self.n, self.m
        X = np.empty((n, n)) if want_X else None
        y = np.empty(max(m, 1))
        V = np.empty(n * 128)
        lam = np.empty(128)
        r = ctypes.c_int64()
        _check(lib().proxsdp_gpu_get_primal_dual(self.h, _ptr(X), _ptr(y), _ptr(V), _ptr(lam), ctypes.byref(r)),
               self.h)
        rr = int(r.value)
        return dict(X=X, y=y[:m], V=V[: n * rr].reshape(rr, n).T.copy(), lam=lam[:rr].copy(), r=rr)

    def get_saved_pair(self, want_X=True):
        """Alg. 2's saved feasible pair (X_[r], y_[r]) of the last solve (raises if none)."""
        n, m = self.n, self.m
        X = np.empty((n, n)) if want_X else None
        y = np.empty(max(m, 1))
        V = np.empty(n * 128)
        lam = np.empty(128)
        r = ctypes.c_int64()
        it = ctypes.c_int64()
        _check(lib().proxsdp_gpu_get_saved_pair(self.h, _ptr(X), _ptr(y), _ptr(V), _ptr(lam), ctypes.byref(r),
                                                ctypes.byref(it)), self.h)
        rr = int(r.value)
        return dict(X=X, y=y[:m], V=V[: n * rr].reshape(rr, n).T.copy(), lam=lam[:rr].copy(), r=rr,
                    iter=int(it.value))


def solve_batch(solvers, host_threads: int = 0):
    """Solve the problems loaded in ``solvers`` (distinct ``Solver`` objects,
    each on its own stream) concurrently; returns their ``Info`` in order."""
    k = len(solvers)
    hs = (ctypes.c_void_p * max(k, 1))(*[s.h for s in solvers])
    infos = (Info * max(k, 1))()
    code = lib().proxsdp_gpu_solve_batch(hs, k, infos, int(host_threads))
    if code != OK:
        msgs = [lib().proxsdp_gpu_last_error(s.h) for s in solvers if s.h]
        msg = next((m.decode() for m in msgs if m), "")
        if code == ERR_INVALID_ARG and not msg:
            msg = (lib().proxsdp_gpu_last_error(None) or b"").decode()
        raise ProxSDPError(code, msg)
    return [infos[i] for i in range(k)]


def analyze_problem(n, m_eq, A_rowptr, A_col, A_val, rhs, C_dense=None, C_idx=None, C_val=None,
                    settings: Settings | None = None):
    """Host-only validation and preprocessing (no GPU): returns
    dict(norm_M, alpha, n_union, norm_C); raises ProxSDPError on bad input."""
    rowptr, col, val, b = _i64(A_rowptr), _i64(A_col), _f64(A_val), _f64(rhs)
    Cd, ci, cv = _f64(C_dense), _i64(C_idx), _f64(C_val)
    c_nnz = 0 if ci is None else int(ci.shape[0])
    nm, al, nc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    nu = ctypes.c_int64()
    _check(lib().proxsdp_gpu_analyze_problem(ctypes.byref(settings) if settings is not None else None, int(n),
                                             _ptr(Cd), c_nnz, _ptr(ci), _ptr(cv), int(b.shape[0]), int(m_eq),
                                             _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), ctypes.byref(nm),
                                             ctypes.byref(al), ctypes.byref(nu), ctypes.byref(nc)))
    return dict(norm_M=nm.value, alpha=al.value, n_union=nu.value, norm_C=nc.value)


def _torch_stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def aproj(S, r, want_P=True, want_V=True, settings: Settings | None = None, stream=None):
    """Truncated psd projection of a CUDA float32 tensor S (n x n) via the C ABI."""
    import torch

    assert S.is_cuda and S.dtype == torch.float32 and S.dim() == 2
    n = S.shape[0]
    lds = S.stride(0)
    P = torch.empty((n, n), device=S.device, dtype=torch.float32) if want_P else None
    V = torch.empty((r, n), device=S.device, dtype=torch.float32) if want_V else None  # column-major n x r
    lam = torch.empty(r, device=S.device, dtype=torch.float64)
    info = Info()
    code = lib().proxsdp_gpu_aproj(ctypes.c_void_p(S.data_ptr()), n, lds, int(r),
                                   ctypes.c_void_p(P.data_ptr()) if P is not None else None, n,
                                   ctypes.c_void_p(V.data_ptr()) if V is not None else None,
                                   ctypes.c_void_p(lam.data_ptr()),
                                   ctypes.byref(settings) if settings is not None else None,
                                   _torch_stream(stream), ctypes.byref(info))
    _check(code)
    return P, (V.t() if V is not None else None), lam, info


def aproj_noalloc(S, r, P=None, V=None, lam=None, settings: Settings | None = None, stream=None):
    """aproj through proxsdp_gpu_aproj_noalloc (static device scratch, n <= 2048).

    The outputs may be passed in (CUDA tensors: P n x n float32, V r x n
    float32 = column-major n x r, lam r float64) so that the call itself
    allocates nothing; missing ones are created here."""
    import torch

    assert S.is_cuda and S.dtype == torch.float32 and S.dim() == 2
    n = S.shape[0]
    if P is None:
        P = torch.empty((n, n), device=S.device, dtype=torch.float32)
    if V is None:
        V = torch.empty((r, n), device=S.device, dtype=torch.float32)
    if lam is None:
        lam = torch.empty(r, device=S.device, dtype=torch.float64)
    info = Info()
    _check(lib().proxsdp_gpu_aproj_noalloc(ctypes.c_void_p(S.data_ptr()), n, S.stride(0), int(r),
                                           ctypes.c_void_p(P.data_ptr()), P.stride(0),
                                           ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                           ctypes.byref(settings) if settings is not None else None,
                                           _torch_stream(stream), ctypes.byref(info)))
    return P, V.t(), lam, info


def block_matvec(S, Q, stream=None):
    """W = S Q for CUDA float32 tensors; Q given as (k, n) rows = columns of the n x k block."""
    import torch

    n = S.shape[0]
    k = Q.shape[0]
    W = torch.empty((k, n), device=S.device, dtype=torch.float32)
    _check(lib().proxsdp_gpu_block_matvec(ctypes.c_void_p(S.data_ptr()), n, S.stride(0),
                                          ctypes.c_void_p(Q.data_ptr()), Q.stride(0), k,
                                          ctypes.c_void_p(W.data_ptr()), n, _torch_stream(stream)))
    return W


def sym_eig(T, stream=None):
    """Eigendecomposition of a CUDA float64 K x K symmetric tensor (one thread block): (theta desc, Y columns)."""
    import torch

    K = T.shape[0]
    Tc = T.contiguous()
    theta = torch.empty(K, device=T.device, dtype=torch.float64)
    Y = torch.empty((K, K), device=T.device, dtype=torch.float32)  # row t = eigenvector t
    _check(lib().proxsdp_gpu_sym_eig(ctypes.c_void_p(Tc.data_ptr()), K, ctypes.c_void_p(theta.data_ptr()),
                                     ctypes.c_void_p(Y.data_ptr()), _torch_stream(stream)))
    return theta, Y.t()
