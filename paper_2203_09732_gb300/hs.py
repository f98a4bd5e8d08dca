"""ctypes binding of the C ABI in include/hs.h (argument marshalling only).

Every computation runs in libhs.so's CUDA kernels; this module only converts
torch tensors to device pointers and status codes to exceptions. There is no
CPU fallback: if libhs.so is missing, or no GPU is present, the calls raise.

Vectors are torch tensors on the handle's device, in rank order (ascending
Sz = 0 state words; site j is bit j-1, bit = 1 is spin up).
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("HS_LIB_PATH") or os.path.join(_HERE, "_lib", "libhs.so")

HS_OK, HS_BAD_ARG, HS_OOM, HS_CUDA, HS_NOT_CONVERGED, HS_BREAKDOWN, HS_NONFINITE, HS_TIMEOUT = range(8)
STATUS_NAMES = ["HS_OK", "HS_BAD_ARG", "HS_OOM", "HS_CUDA", "HS_NOT_CONVERGED", "HS_BREAKDOWN",
                "HS_NONFINITE", "HS_TIMEOUT"]
F32, F64 = 0, 1
PRECOND = {"id": 0, "jacobi": 1, "row": 2}
FORM_SMEM, FORM_SUPERBLOCK, FORM_PERSISTENT, FORM_GRAPH, FORM_SMEM1 = 1, 2, 3, 4, 5

# every symbol include/hs.h declares
SYMBOLS = ["hs_create", "hs_free", "hs_last_error", "hs_dim", "hs_get_sigma", "hs_set_sigma",
           "hs_extremal", "hs_unrank", "hs_rank", "hs_diag", "hs_matvec", "hs_minres",
           "hs_minres_f32", "hs_lanczos_eigs", "hs_eigs_host", "hs_twist", "hs_tridiag_eig",
           "hs_kernel_launches", "hs_set_sm_budget", "hs_twist_noalloc", "hs_entanglement",
           "hs_level_ratio", "hs_sym_eigvals", "hs_twist_grad", "hs_sweep"]


class MinresInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_longlong), ("sweeps", ctypes.c_int), ("status", ctypes.c_int),
                ("phi", ctypes.c_double), ("resid_minv", ctypes.c_double),
                ("resid_2", ctypes.c_double), ("form", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LanczosInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("converged", ctypes.c_int),
                ("minres_iters", ctypes.c_longlong), ("sweeps", ctypes.c_int),
                ("sigma", ctypes.c_double), ("max_resid", ctypes.c_double),
                ("seconds_solve", ctypes.c_double), ("seconds_total", ctypes.c_double),
                ("seconds_ritz", ctypes.c_double),
                ("unconverged_solves", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SweepInfo(ctypes.Structure):
    _fields_ = [("realisations", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("launches", ctypes.c_int), ("nclass", ctypes.c_int),
                ("pad", ctypes.c_int), ("minres_iters", ctypes.c_longlong),
                ("L", ctypes.c_int * 2), ("S", ctypes.c_int * 2), ("groups", ctypes.c_int * 2),
                ("tuned", ctypes.c_int * 2),
                ("zz_mean", ctypes.c_double * 2), ("zz_std", ctypes.c_double * 2),
                ("max_resid", ctypes.c_double), ("seconds_setup", ctypes.c_double),
                ("seconds_solve", ctypes.c_double), ("seconds_total", ctypes.c_double)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v)[: self.nclass] if isinstance(v, ctypes.Array) else v
        return out


class HSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None

c_dp = ctypes.POINTER(ctypes.c_double)
c_vp = ctypes.c_void_p


def load(path=LIB_PATH):
    """Load libhs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2203_09732_gb300.build.build()")
    lib = ctypes.CDLL(path)
    H = c_vp
    sig = {
        "hs_create": ([ctypes.c_int, c_dp, ctypes.c_double, c_vp, ctypes.POINTER(H)], ctypes.c_int),
        "hs_free": ([H], None),
        "hs_last_error": ([H], ctypes.c_char_p),
        "hs_dim": ([H, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "hs_get_sigma": ([H, c_dp], ctypes.c_int),
        "hs_set_sigma": ([H, ctypes.c_double], ctypes.c_int),
        "hs_extremal": ([H, ctypes.c_int, ctypes.c_double, c_dp, c_dp, c_dp], ctypes.c_int),
        "hs_unrank": ([H, ctypes.c_longlong, ctypes.c_longlong, c_vp], ctypes.c_int),
        "hs_rank": ([H, c_vp, ctypes.c_longlong, c_vp], ctypes.c_int),
        "hs_diag": ([H, c_vp, ctypes.c_int, c_vp], ctypes.c_int),
        "hs_matvec": ([H, c_vp, c_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "hs_minres": ([H, c_vp, c_vp, ctypes.c_double, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                       ctypes.c_double, ctypes.POINTER(MinresInfo)], ctypes.c_int),
        "hs_minres_f32": ([H, c_vp, c_vp, ctypes.c_double, ctypes.c_longlong, ctypes.c_int,
                           ctypes.POINTER(MinresInfo)], ctypes.c_int),
        "hs_lanczos_eigs": ([H, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong, c_vp,
                             ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_longlong, c_dp, c_vp, c_dp, ctypes.POINTER(LanczosInfo)],
                            ctypes.c_int),
        "hs_eigs_host": ([ctypes.c_int, c_dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                          ctypes.c_double, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int,
                          ctypes.c_double, ctypes.c_double, ctypes.c_longlong, ctypes.c_int, c_dp,
                          c_dp, c_dp, c_dp, ctypes.POINTER(LanczosInfo)], ctypes.c_int),
        "hs_twist": ([H, c_vp, ctypes.c_int, c_dp], ctypes.c_int),
        "hs_tridiag_eig": ([ctypes.c_int, c_dp, c_dp, c_dp, c_dp], ctypes.c_int),
        "hs_kernel_launches": ([], ctypes.c_ulonglong),
        "hs_set_sm_budget": ([H, ctypes.c_int], ctypes.c_int),
        "hs_twist_noalloc": ([ctypes.c_int, c_vp, ctypes.c_int, c_vp, c_vp], ctypes.c_int),
        "hs_entanglement": ([H, c_vp, ctypes.c_int, c_dp], ctypes.c_int),
        "hs_twist_grad": ([H, c_vp, c_dp, ctypes.c_int, ctypes.c_double, c_dp, c_dp, c_dp,
                           ctypes.POINTER(MinresInfo)], ctypes.c_int),
        "hs_level_ratio": ([c_dp, ctypes.c_int, c_dp, c_dp], ctypes.c_int),
        "hs_sym_eigvals": ([ctypes.c_int, c_dp, c_dp], ctypes.c_int),
        "hs_sweep": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), c_dp, ctypes.c_int, ctypes.c_int,
                      ctypes.c_double, ctypes.c_ulonglong, ctypes.c_double, ctypes.c_int, c_dp,
                      c_dp, c_dp, c_dp, ctypes.POINTER(SweepInfo)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(c_dp) if a is not None else None


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def twist_noalloc(L, psi, z, stream=None):
    """hs_twist_noalloc: twist overlaps of the K rows of psi (CUDA float64,
    K x n) into z (CUDA float64, 2K), with no device allocation. Returns the
    status code; asynchronous on `stream` (default: the current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    K = psi.shape[0] if psi.dim() == 2 else 1
    return int(load().hs_twist_noalloc(int(L), _ptr(psi), int(K), _ptr(z),
                                       ctypes.c_void_p(s.cuda_stream)))


def kernel_launches():
    """Kernels launched by libhs.so in this process so far."""
    return int(load().hs_kernel_launches())


def level_ratio(evals):
    """hs_level_ratio (host-only): (ratios of the K - 2 interior levels, mean)."""
    e = np.ascontiguousarray(evals, dtype=np.float64)
    r = np.zeros(max(0, len(e) - 2))
    mean = ctypes.c_double()
    st = load().hs_level_ratio(_dp(e), len(e), _dp(r), ctypes.byref(mean))
    if st != HS_OK:
        raise HSError(st, "hs_level_ratio")
    return r, mean.value


def sym_eigvals(a):
    """hs_sym_eigvals (host-only): ascending eigenvalues of a symmetric matrix."""
    A = np.array(a, dtype=np.float64, order="C", copy=True)
    w = np.zeros(A.shape[0])
    st = load().hs_sym_eigvals(A.shape[0], _dp(A), _dp(w))
    if st != HS_OK:
        raise HSError(st, "hs_sym_eigvals")
    return w


def tridiag_eig(alpha, beta, vectors=True):
    """Host-only T_k eigensolver of the library (implicit QL)."""
    lib = load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    k = len(a)
    th = np.zeros(k)
    Y = np.zeros((k, k)) if vectors else None  # column-major == C-order transposed
    st = lib.hs_tridiag_eig(k, _dp(a), _dp(b) if k > 1 else None, _dp(th), _dp(Y))
    if st != HS_OK:
        raise HSError(st, "tridiagonal eigensolver")
    return (th, Y.T.copy()) if vectors else th


class Chain:
    """Handle on one disorder realisation: hs_create(L, h, sigma) ... hs_free."""

    def __init__(self, L, h, sigma=float("nan"), stream=None, device=None):
        import torch
        self.torch = torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required (the library has no CPU path)")
        if device is not None:
            torch.cuda.set_device(device)
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.L = int(L)
        hd = ctypes.c_void_p()
        st = lib.hs_create(self.L, _dp(self.h), float(sigma), ctypes.c_void_p(s.cuda_stream),
                           ctypes.byref(hd))
        if st != HS_OK:
            raise HSError(st, "hs_create failed")
        self._hd = hd
        self._lib = lib
        n = ctypes.c_longlong()
        lib.hs_dim(hd, ctypes.byref(n))
        self.n = n.value

    # -- plumbing ---------------------------------------------------------
    def _check(self, st, what):
        if st != HS_OK:
            msg = self._lib.hs_last_error(self._hd)
            raise HSError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_hd", None):
            self._lib.hs_free(self._hd)
            self._hd = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _vec(self, x, dtype):
        t = self.torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == dtype and x.is_contiguous()
                and x.numel() >= self.n):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor with >= n elements")
        return x

    # -- API --------------------------------------------------------------
    @property
    def sigma(self):
        s = ctypes.c_double()
        self._lib.hs_get_sigma(self._hd, ctypes.byref(s))
        return s.value

    @sigma.setter
    def sigma(self, v):
        self._check(self._lib.hs_set_sigma(self._hd, float(v)), "hs_set_sigma")

    def set_sm_budget(self, nsm):
        """Let persistent solves of this handle use nsm SMs (0 = all)."""
        self._check(self._lib.hs_set_sm_budget(self._hd, int(nsm)), "hs_set_sm_budget")

    def extremal(self, max_steps=600, tol=1e-12):
        lo, hi, mid = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.hs_extremal(self._hd, max_steps, tol, ctypes.byref(lo), ctypes.byref(hi),
                                          ctypes.byref(mid)), "hs_extremal")
        return lo.value, hi.value, mid.value

    def unrank(self, first=0, count=None):
        t = self.torch
        count = self.n - first if count is None else count
        out = t.empty(count, dtype=t.int32, device=self.device)
        self._check(self._lib.hs_unrank(self._hd, first, count, _ptr(out)), "hs_unrank")
        return out

    def rank(self, states):
        t = self.torch
        out = t.empty(states.numel(), dtype=t.int64, device=self.device)
        self._check(self._lib.hs_rank(self._hd, _ptr(states), states.numel(), _ptr(out)), "hs_rank")
        return out

    def diag(self, precond="row"):
        t = self.torch
        d = t.empty(self.n, dtype=t.float64, device=self.device)
        m = t.empty(self.n, dtype=t.float64, device=self.device)
        self._check(self._lib.hs_diag(self._hd, _ptr(d), PRECOND[precond], _ptr(m)), "hs_diag")
        return d, m

    def matvec(self, x, y=None, shifted=False):
        t = self.torch
        dt = F64 if x.dtype == t.float64 else F32
        self._vec(x, x.dtype)
        if y is None:
            y = t.empty_like(x)
        self._vec(y, x.dtype)
        self._check(self._lib.hs_matvec(self._hd, _ptr(x), _ptr(y), dt, int(shifted)), "hs_matvec")
        return y

    def minres(self, b, x=None, tol=1e-12, kmax=0, precond="row", mixed=False, inner_tol=1e-5,
               allow_not_converged=False):
        t = self.torch
        self._vec(b, t.float64)
        if x is None:
            x = t.empty_like(b)
        info = MinresInfo()
        st = self._lib.hs_minres(self._hd, _ptr(b), _ptr(x), tol, kmax, PRECOND[precond], int(mixed),
                                 inner_tol, ctypes.byref(info))
        if not (allow_not_converged and st == HS_NOT_CONVERGED):
            self._check(st, "hs_minres")
        return x, info.as_dict()

    def minres_f32(self, b, x=None, tol=1e-6, kmax=0, precond="row", allow_not_converged=False):
        t = self.torch
        self._vec(b, t.float32)
        if x is None:
            x = t.empty_like(b)
        info = MinresInfo()
        st = self._lib.hs_minres_f32(self._hd, _ptr(b), _ptr(x), tol, kmax, PRECOND[precond],
                                     ctypes.byref(info))
        if not (allow_not_converged and st == HS_NOT_CONVERGED):
            self._check(st, "hs_minres_f32")
        return x, info.as_dict()

    def eigs(self, K, m_max=0, tol=1e-10, seed=0, v0=None, mixed=False, precond="row",
             minres_tol=1e-12, inner_tol=1e-5, minres_kmax=0, vectors=True,
             allow_not_converged=False):
        t = self.torch
        ev = np.zeros(K)
        res = np.zeros(K)
        vecs = t.empty((K, self.n), dtype=t.float64, device=self.device) if vectors else None
        info = LanczosInfo()
        st = self._lib.hs_lanczos_eigs(self._hd, K, m_max, tol, seed, _ptr(v0), int(mixed),
                                       PRECOND[precond], minres_tol, inner_tol, int(minres_kmax),
                                       _dp(ev), _ptr(vecs), _dp(res), ctypes.byref(info))
        if not (allow_not_converged and st == HS_NOT_CONVERGED):
            self._check(st, "hs_lanczos_eigs")
        return ev, vecs, res, info.as_dict()

    def twist_grad(self, psi, evals, tol=1e-10):
        """hs_twist_grad: for the K eigenpairs (rows of psi, evals), returns
        (z [K] complex, d|z|^2/dh [K, L], dE/dh [K, L], MINRES info)."""
        t = self.torch
        psi = psi.reshape(-1, self.n)
        if not (psi.is_cuda and psi.dtype == t.float64 and psi.is_contiguous()):
            raise ValueError("psi must be a contiguous CUDA float64 tensor")
        K = psi.shape[0]
        ev = np.ascontiguousarray(evals, dtype=np.float64)
        if ev.shape != (K,):
            raise ValueError("evals must hold one eigenvalue per row of psi")
        z = np.zeros(2 * K)
        dz2 = np.zeros((K, self.L))
        dE = np.zeros((K, self.L))
        info = MinresInfo()
        self._check(self._lib.hs_twist_grad(self._hd, _ptr(psi), _dp(ev), K, float(tol), _dp(z),
                                            _dp(dz2), _dp(dE), ctypes.byref(info)), "hs_twist_grad")
        return z[0::2] + 1j * z[1::2], dz2, dE, info.as_dict()

    def entanglement(self, psi):
        """Bipartite entanglement entropy of the rows of psi (K x n, FP64), A =
        sites 1..L/2 (hs_entanglement)."""
        t = self.torch
        psi = psi.reshape(-1, self.n)
        if not (psi.is_cuda and psi.dtype == t.float64 and psi.is_contiguous()):
            raise ValueError("psi must be a contiguous CUDA float64 tensor")
        S = np.zeros(psi.shape[0])
        self._check(self._lib.hs_entanglement(self._hd, _ptr(psi), psi.shape[0], _dp(S)),
                    "hs_entanglement")
        return S

    def twist(self, psi):
        t = self.torch
        psi = psi.reshape(-1, self.n)
        if not (psi.is_cuda and psi.dtype == t.float64 and psi.is_contiguous()):
            raise ValueError("psi must be a contiguous CUDA float64 tensor")
        K = psi.shape[0]
        z = np.zeros(2 * K)
        self._check(self._lib.hs_twist(self._hd, _ptr(psi), K, _dp(z)), "hs_twist")
        return z[0::2] + 1j * z[1::2]


def sweep(Ls, hs_list, K, m_max=0, tol=1e-10, seed=0, minres_tol=1e-12, precond="row"):
    """Batched disorder sweep (hs_sweep): realisation r has chain length Ls[r]
    and fields hs_list[r]. Returns (evals (B, K), resid (B, K), z (B, K)
    complex, zz (B,) = mean |z|^2 per realisation, info dict)."""
    lib = load()
    B = len(Ls)
    if len(hs_list) != B:
        raise ValueError("one field array per realisation")
    Larr = (ctypes.c_int * B)(*[int(L) for L in Ls])
    hh = np.ascontiguousarray(np.concatenate([np.asarray(h, dtype=np.float64) for h in hs_list]))
    if any(len(h) != L for h, L in zip(hs_list, Ls)):
        raise ValueError("len(h) must equal L for every realisation")
    ev = np.zeros(B * K)
    res = np.zeros(B * K)
    z = np.zeros(2 * B * K)
    zz = np.zeros(B)
    info = SweepInfo()
    st = lib.hs_sweep(B, Larr, _dp(hh), K, m_max, tol, seed, minres_tol, PRECOND[precond], _dp(ev),
                      _dp(res), _dp(z), _dp(zz), ctypes.byref(info))
    if st not in (HS_OK, HS_NOT_CONVERGED):
        raise HSError(st, "hs_sweep")
    zc = (z[0::2] + 1j * z[1::2]).reshape(B, K)
    return ev.reshape(B, K), res.reshape(B, K), zc, zz, info.as_dict()


def eigs_host(L, h, K, sigma=float("nan"), m_max=0, tol=1e-10, seed=0, mixed=True, precond="row",
              minres_tol=1e-12, inner_tol=1e-5, minres_kmax=0, vectors=True, twist=True,
              sm_budget=0, out=None):
    """End-to-end call with host (numpy) buffers only: hs_eigs_host. `out`
    may supply the (K, n) float64 eigenvector buffer (e.g. pinned memory)."""
    lib = load()
    hh = np.ascontiguousarray(h, dtype=np.float64)
    n = math.comb(L, L // 2)
    ev = np.zeros(K)
    res = np.zeros(K)
    if vectors:
        vec = out if out is not None else np.zeros((K, n))
        if vec.shape != (K, n) or vec.dtype != np.float64 or not vec.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous (K, n) float64 array")
    else:
        vec = None
    z = np.zeros(2 * K) if twist else None
    info = LanczosInfo()
    st = lib.hs_eigs_host(L, _dp(hh), float(sigma), K, m_max, tol, seed, int(mixed), PRECOND[precond],
                          minres_tol, inner_tol, int(minres_kmax), int(sm_budget), _dp(ev), _dp(vec),
                          _dp(res), _dp(z), ctypes.byref(info))
    if st not in (HS_OK, HS_NOT_CONVERGED):
        raise HSError(st, "hs_eigs_host")
    zz = (z[0::2] + 1j * z[1::2]) if twist else None
    return ev, vec, res, zz, info.as_dict()
