"""ctypes binding of libctm (argument marshalling only; every step runs in the
library's CUDA kernels).

Module-level functions carry the C names (``ctm_init_env``, ``ctm_move``, ...)
and return the C status; ``Env`` wraps a context and raises ``CtmError`` on a
non-zero status.  Site tensors are real ``[d, D, D, D, D]`` arrays with legs
(p, u, l, d, r), as numpy arrays (host) or CUDA torch tensors (device).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctm.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NAN, ERR_NOCONV, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
LEFT, UP, RIGHT, DOWN = 0, 1, 2, 3
STANDARD, REDUCED_SEQUENTIAL, REDUCED_ENV = 0, 1, 2
FP64, TF32, BF16 = 0, 1, 2
INIT_NO_GROW = 0x100
PROFILE_SERIAL = 0x100
DIRS = {"left": LEFT, "up": UP, "right": RIGHT, "down": DOWN}
MODES = {"standard": STANDARD, "reduced_sequential": REDUCED_SEQUENTIAL,
         "reduced_env": REDUCED_ENV}
PRECISIONS = {"fp64": FP64, "tf32": TF32, "bf16": BF16}

_lib = None

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)

SIGNATURES = {
    "ctm_init_env": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "ctm_move": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "ctm_converge": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _I, _D]),
    "ctm_expect_bond": (ctypes.c_int, [_P, ctypes.c_int, _D, _D]),
    "ctm_corner_spectrum": (ctypes.c_int, [_P, ctypes.c_int, _D, _I]),
    "ctm_corner_spectra": (ctypes.c_int, [_P, _D, ctypes.c_int, _I]),
    "ctm_correlator": (ctypes.c_int, [_P, _D, _D, ctypes.c_int, _D]),
    "ctm_log_kappa": (ctypes.c_int, [_P, _D]),
    "ctm_get_tensor": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _I]),
    "ctm_set_tensor": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _I]),
    "ctm_kernel_launches": (ctypes.c_longlong, [_P]),
    "ctm_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ctm_profile_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _D, _D]),
    "ctm_singular_values_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "ctm_svd_left_adjoint": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, _P, _P]),
    "ctm_contract_test": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                          ctypes.c_longlong, _D, _D, _D]),
    "ctm_truncated_svd_test": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _D]),
    "ctm_cholqr_test": (ctypes.c_int, [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]),
    "ctm_set_sites": (ctypes.c_int, [_P, _P, _P]),
    "ctm_energy_grad": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _D, _D, _P, _P]),
    "ctm_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int]),
    "ctm_batch_move": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "ctm_batch_last_error": (ctypes.c_char_p, [_P]),
    "ctm_batch_free": (None, [_P]),
    "ctm_last_error": (ctypes.c_char_p, [_P]),
    "ctm_free": (None, [_P]),
}


class CtmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libctm error {code}: {msg}")
        self.code = code


def load(path=None):
    """Load libctm.so (built by ``paper_2306_08212_gb300.build``); raises if missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} is missing: build it with paper_2306_08212_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(_D)


def _ptr_of(t):
    """Host numpy (C-contiguous float64) or CUDA torch tensor -> (void*, keepalive)."""
    if hasattr(t, "data_ptr") and hasattr(t, "is_cuda") and t.is_cuda:
        import torch
        if t.dtype != torch.float64 or not t.is_contiguous():
            t = t.to(torch.float64).contiguous()
        return ctypes.c_void_p(t.data_ptr()), t
    a = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    return ctypes.c_void_p(a.ctypes.data), a


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


# --- thin C-named wrappers -------------------------------------------------
def ctm_init_env(A, B, chi, chi_prime=0, precision=FP64, boundary=None, stream=None):
    """Returns (status, ctx_handle)."""
    lib = load()
    pa, ka = _ptr_of(A)
    pb, kb = _ptr_of(B)
    shape = tuple(A.shape)
    d, D = int(shape[0]), int(shape[1])
    pbnd, kbnd = (_ptr_of(boundary) if boundary is not None else (ctypes.c_void_p(0), None))
    ctx = ctypes.c_void_p()
    st = stream if stream is not None else _current_stream()
    rc = lib.ctm_init_env(ctypes.byref(ctx), pa, pb, d, D, int(chi), int(chi_prime),
                          int(precision), pbnd, st)
    del ka, kb, kbnd
    if rc == OK:
        _site_shape[ctx.value] = (d, D, D, D, D)
    return rc, ctx


def ctm_move(ctx, direction, mode):
    return load().ctm_move(ctx, int(direction), int(mode))


def ctm_converge(ctx, mode, max_iter, tol):
    it = ctypes.c_int(0)
    dl = ctypes.c_double(0.0)
    rc = load().ctm_converge(ctx, int(mode), int(max_iter), float(tol), ctypes.byref(it),
                             ctypes.byref(dl))
    return rc, it.value, dl.value


def ctm_expect_bond(ctx, bond, op):
    op = np.ascontiguousarray(op, dtype=np.float64)
    v = ctypes.c_double(0.0)
    rc = load().ctm_expect_bond(ctx, int(bond), _dptr(op), ctypes.byref(v))
    return rc, v.value


def ctm_corner_spectrum(ctx, corner, maxlen):
    s = np.zeros(maxlen)
    n = ctypes.c_int(0)
    rc = load().ctm_corner_spectrum(ctx, int(corner), _dptr(s), ctypes.byref(n))
    return rc, s[: n.value]


def ctm_corner_spectra(ctx, maxlen):
    s = np.zeros((8, maxlen))
    lens = (ctypes.c_int * 8)()
    rc = load().ctm_corner_spectra(ctx, _dptr(s), int(maxlen), lens)
    return rc, [s[i, : lens[i]] for i in range(8)]


def ctm_correlator(ctx, op1, op2, xmax):
    op1 = np.ascontiguousarray(op1, dtype=np.float64)
    op2 = np.ascontiguousarray(op2, dtype=np.float64)
    out = np.zeros(int(xmax))
    rc = load().ctm_correlator(ctx, _dptr(op1), _dptr(op2), int(xmax), _dptr(out))
    return rc, out


def ctm_log_kappa(ctx):
    v = ctypes.c_double(0.0)
    rc = load().ctm_log_kappa(ctx, ctypes.byref(v))
    return rc, v.value


def ctm_get_tensor(ctx, kind, k, x):
    lib = load()
    dims = (ctypes.c_int * 4)()
    rc = lib.ctm_get_tensor(ctx, kind, k, x, None, dims)
    if rc != OK:
        return rc, None
    shape = [v for v in dims if v > 0]
    out = np.zeros(shape)
    rc = lib.ctm_get_tensor(ctx, kind, k, x, _dptr(out), dims)
    return rc, out


def ctm_set_tensor(ctx, kind, k, x, arr):
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    dims = (ctypes.c_int * 4)(*(list(arr.shape) + [0] * (4 - arr.ndim)))
    return load().ctm_set_tensor(ctx, kind, k, x, _dptr(arr), dims)


def ctm_kernel_launches(ctx):
    return load().ctm_kernel_launches(ctx)


PROFILE_CLASSES = {0: "gemm_f64", 1: "tc_tf32_gemm", 2: "tc_bf16_gemm", 3: "jacobi_f64",
                   4: "cholqr_f64"}


def ctm_profile_enable(ctx, mask=0x1F):
    """Time the kernel classes whose bit (1 << class) is set; 0 stops."""
    return load().ctm_profile_enable(ctx, int(mask))


def ctm_profile_read(ctx, cls):
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    fl = ctypes.c_double(0.0)
    rc = load().ctm_profile_read(ctx, int(cls), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl))
    return rc, n.value, ms.value, fl.value


def ctm_kernel_stats_reset(ctx, mask=0x1F):
    """Clear and start the per-class CUDA-event kernel timing."""
    rc = ctm_profile_enable(ctx, mask)
    if rc != OK:
        raise CtmError(rc, ctm_last_error(ctx))


def ctm_kernel_stats(ctx):
    """[{name, count, ms, flops}] per kernel class since the last reset."""
    out = []
    for cls, name in PROFILE_CLASSES.items():
        rc, n, ms, fl = ctm_profile_read(ctx, cls)
        if rc != OK:
            raise CtmError(rc, ctm_last_error(ctx))
        out.append({"name": name, "count": n, "ms": ms, "flops": fl})
    return out


def ctm_singular_values_noalloc(M_ptr, rows, cols, s_ptr, stream=None):
    """Singular values of a device matrix into a device buffer, allocating nothing.

    M_ptr / s_ptr are device addresses (e.g. ``tensor.data_ptr()``); for callers
    that must not allocate device memory during the call.  Returns the status.
    """
    st = stream if stream is not None else _current_stream()
    return load().ctm_singular_values_noalloc(ctypes.c_void_p(M_ptr), int(rows), int(cols),
                                              ctypes.c_void_p(s_ptr), st)


def ctm_truncated_svd_test(path, M, k):
    """Leading k left singular vectors of the host matrix M in FP64 on the GPU
    (path 0 = library choice, 1 = exact Jacobi, 2 = randomized).  Returns (status, U)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    rows, cols = M.shape
    U = np.zeros((rows, int(k)))
    rc = load().ctm_truncated_svd_test(int(path), _dptr(M), rows, cols, int(k), _dptr(U))
    return rc, U


def ctm_cholqr_test(Y, passes):
    """Orthonormal basis of the columns of the host matrix Y by the library's FP64
    CholeskyQR (first pass shifted).  Returns (status, Q)."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    rows, n = Y.shape
    Q = np.zeros((rows, n))
    rc = load().ctm_cholqr_test(_dptr(Y), rows, n, int(passes), _dptr(Q))
    return rc, Q


def ctm_svd_left_adjoint(U, s, Vt, gU, eps=1e-12, stream=None):
    """gM for M = U diag(s) Vt from the gradient gU of the leading gU.shape[1] columns of U.

    U, s, Vt, gU: CUDA float64 tensors (or host arrays, copied to the current device).
    Returns (status, gM) with gM a CUDA tensor of M's shape."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    t = [torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous() for x in (U, s, Vt, gU)]
    rows, cols, k = t[0].shape[0], t[2].shape[1], t[3].shape[1]
    gM = torch.empty((rows, cols), dtype=torch.float64, device=dev)
    st = stream if stream is not None else _current_stream()
    rc = load().ctm_svd_left_adjoint(*(ctypes.c_void_p(x.data_ptr()) for x in t), int(rows),
                                     int(cols), int(k), float(eps), ctypes.c_void_p(gM.data_ptr()),
                                     st)
    return rc, gM


def ctm_contract_test(precision, A, B):
    """C = A @ B through the library's FP64 or tensor-core contraction kernel."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    C = np.zeros((M, N))
    rc = load().ctm_contract_test(int(precision), M, N, K, _dptr(A), _dptr(B), _dptr(C))
    return rc, C


def ctm_last_error(ctx):
    return load().ctm_last_error(ctx).decode()


def ctm_free(ctx):
    _site_shape.pop(getattr(ctx, "value", ctx), None)
    load().ctm_free(ctx)


def ctm_set_sites(ctx, A, B):
    pa, ka = _ptr_of(A)
    pb, kb = _ptr_of(B)
    rc = load().ctm_set_sites(ctx, pa, pb)
    del ka, kb
    return rc


def ctm_energy_grad(ctx, iters, op, eps=1e-12):
    """(status, E, gA, gB): the mean bond expectation of op after `iters`
    reduced-sequential iterations from the context's environment, and its gradient
    with respect to the site tensors (host arrays of the sites' shape)."""
    op = np.ascontiguousarray(op, dtype=np.float64)
    shape = _site_shape[ctx.value]
    e = ctypes.c_double(0.0)
    gA = np.zeros(shape)
    gB = np.zeros(shape)
    rc = load().ctm_energy_grad(ctx, int(iters), float(eps), _dptr(op), ctypes.byref(e),
                                ctypes.c_void_p(gA.ctypes.data), ctypes.c_void_p(gB.ctypes.data))
    return rc, e.value, gA, gB


_site_shape = {}


# --- convenience wrapper -----------------------------------------------------
class Env:
    """A libctm context: the 16 environment tensors of a 2-site iPEPS on the GPU."""

    def __init__(self, A, B, chi, chi_prime=0, precision="fp64", boundary=None, stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.chi = int(chi)
        self.ctx = None
        rc, ctx = ctm_init_env(A, B, chi, chi_prime, prec, boundary, stream)
        if rc != OK:
            msg = ctm_last_error(ctx) if ctx else "init failed"
            raise CtmError(rc, msg)
        self.ctx = ctx

    def _check(self, rc):
        if rc != OK:
            raise CtmError(rc, ctm_last_error(self.ctx))

    def move(self, direction, mode="reduced_sequential"):
        d = DIRS[direction] if isinstance(direction, str) else int(direction)
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self._check(ctm_move(self.ctx, d, m))

    def converge(self, mode="reduced_sequential", max_iter=50, tol=1e-10, allow_noconv=True):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        rc, it, dl = ctm_converge(self.ctx, m, max_iter, tol)
        if not (rc == OK or (allow_noconv and rc == ERR_NOCONV)):
            self._check(rc)
        return it, dl

    def expect_bond(self, bond, op):
        rc, v = ctm_expect_bond(self.ctx, bond, op)
        self._check(rc)
        return v

    def corner_spectrum(self, corner):
        rc, s = ctm_corner_spectrum(self.ctx, corner, max(self.chi, 1) * 4 + 16)
        self._check(rc)
        return s

    def corner_spectra(self):
        rc, out = ctm_corner_spectra(self.ctx, max(self.chi, 1) * 4 + 16)
        self._check(rc)
        return out

    def correlator(self, op1, op2, xmax):
        rc, out = ctm_correlator(self.ctx, op1, op2, xmax)
        self._check(rc)
        return out

    def log_kappa(self):
        rc, v = ctm_log_kappa(self.ctx)
        self._check(rc)
        return v

    def tensor(self, kind, k, x):
        rc, t = ctm_get_tensor(self.ctx, kind, k, x)
        self._check(rc)
        return t

    def set_tensor(self, kind, k, x, arr):
        self._check(ctm_set_tensor(self.ctx, kind, k, x, arr))

    def set_sites(self, A, B):
        self._check(ctm_set_sites(self.ctx, A, B))

    def energy_grad(self, iters, op, eps=1e-12):
        """(E, dE/dA, dE/dB): see ctm_energy_grad."""
        rc, E, gA, gB = ctm_energy_grad(self.ctx, iters, op, eps)
        self._check(rc)
        return E, gA, gB

    @property
    def launches(self):
        return ctm_kernel_launches(self.ctx)

    def free(self):
        if self.ctx:
            ctm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Independent states advanced together (one CUDA graph per direction once warm).

    Create each Env on its own torch.cuda.Stream for the work to overlap.
    """

    def __init__(self, envs):
        self.envs = list(envs)
        arr = (_P * len(self.envs))(*[e.ctx for e in self.envs])
        self.handle = ctypes.c_void_p()
        rc = load().ctm_batch_create(ctypes.byref(self.handle), arr, len(self.envs))
        if rc != OK:
            raise CtmError(rc, "batch create failed")

    def move(self, direction, mode="reduced_sequential"):
        d = DIRS[direction] if isinstance(direction, str) else int(direction)
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        rc = load().ctm_batch_move(self.handle, d, m)
        if rc != OK:
            raise CtmError(rc, load().ctm_batch_last_error(self.handle).decode())

    def free(self):
        if self.handle:
            load().ctm_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _energy_function():
    import torch

    class CTMEnergy(torch.autograd.Function):
        """E(A, B): the mean bond expectation of op after `iters` checkpointed
        reduced-sequential iterations from the environment held by `env` (a
        constant of the loss).  Forward and reverse pass both run in the library
        (ctm_set_sites, ctm_energy_grad); backward only scales the stored gradient
        by the incoming one."""

        @staticmethod
        def forward(ctx, A, B, env, iters, op, eps):
            env.set_sites(A.detach(), B.detach())
            E, gA, gB = env.energy_grad(iters, op, eps)
            ctx.save_for_backward(torch.as_tensor(gA, dtype=A.dtype, device=A.device),
                                  torch.as_tensor(gB, dtype=B.dtype, device=B.device))
            return torch.tensor(E, dtype=A.dtype, device=A.device)

        @staticmethod
        def backward(ctx, g):
            gA, gB = ctx.saved_tensors
            return g * gA, g * gB, None, None, None, None

    return CTMEnergy


def ctm_energy(A, B, env, iters, op, eps=1e-12):
    """Differentiable E(A, B) (torch tensors, float64) through the library's
    reverse pass; `env` is an Env whose environment is the fixed starting point."""
    return _energy_function().apply(A, B, env, iters, op, eps)
