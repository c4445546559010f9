"""GB300-native preconditioned MINRES for block lower triangular Toeplitz systems (arXiv 2307.07749).

Thin Python binding of libbltt (C ABI in include/bltt.h): argument marshalling only.  Every step of
the solver runs in the library's CUDA kernels; PyTorch supplies device memory and streams.  There
is no CPU fallback: if libbltt.so is missing or cannot load, importing the binding raises.

The functions carry the C names (bltt_create, bltt_matvec, bltt_precond_apply, bltt_minres_solve,
...) and take torch tensors (float64, contiguous, on a CUDA device) where the C calls take device
pointers.  `Solver` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbltt.so")

BLTT_OK = 0
STATUS_NAMES = {
    0: "BLTT_OK", 1: "BLTT_ERR_INVALID_ARG", 2: "BLTT_ERR_ASSUMPTION", 3: "BLTT_ERR_OOM",
    4: "BLTT_ERR_CUDA", 5: "BLTT_ERR_NUMERIC", 6: "BLTT_ERR_NOT_CONVERGED", 7: "BLTT_ERR_TIMEOUT",
    8: "BLTT_ERR_UNSUPPORTED",
}
PREC_F64, PREC_F32, PREC_F32X2 = 64, 32, 96
BASIS_AUTO, BASIS_SPECTRAL, BASIS_PHYSICAL = 0, 1, 2
PRECOND_ABAC, PRECOND_NONE = 0, 1
ARITH_DEFAULT, ARITH_F64, ARITH_F32X2, ARITH_TC = 0, 1, 2, 3


class BlttError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bltt_space(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("m", ctypes.c_int * 3), ("h", ctypes.c_double * 3)]


class bltt_blocks(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("a", ctypes.POINTER(ctypes.c_double)),
                ("b", ctypes.POINTER(ctypes.c_double)), ("space", bltt_space)]


class bltt_solve_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("basis", ctypes.c_int), ("precond", ctypes.c_int),
                ("sync_every", ctypes.c_int), ("rebuild", ctypes.c_int),
                ("matvec_arith", ctypes.c_int), ("no_graph", ctypes.c_int),
                ("single_block", ctypes.c_int), ("defer_window", ctypes.c_int),
                ("refine", ctypes.c_int)]


class bltt_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres_est", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("alpha_used", ctypes.c_double),
                ("alpha_source", ctypes.c_int), ("precision", ctypes.c_int),
                ("basis", ctypes.c_int), ("t_setup_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("status", ctypes.c_int), ("refinements", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bltt_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double), ("active_launches", ctypes.c_longlong),
                ("active_ms", ctypes.c_double)]


# C signatures: name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "bltt_create": (ctypes.c_int, [ctypes.POINTER(bltt_blocks), ctypes.c_int, ctypes.c_longlong,
                                   ctypes.POINTER(_P)]),
    "bltt_destroy": (ctypes.c_int, [_P]),
    "bltt_set_stream": (ctypes.c_int, [_P, _P]),
    "bltt_matvec": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "bltt_set_matvec_arith": (ctypes.c_int, [_P, ctypes.c_int]),
    "bltt_set_variable_coefficient": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                                      ctypes.c_double]),
    "bltt_set_dense_operator": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "bltt_set_block_spectra": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]),
    "bltt_precond_apply": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, ctypes.c_int]),
    "bltt_minres_solve_ex": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(bltt_solve_opts), _P,
                                            ctypes.POINTER(bltt_solve_info)]),
    "bltt_minres_solve": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, _P, ctypes.POINTER(bltt_solve_info)]),
    "bltt_minres_solve_host": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.POINTER(bltt_solve_opts), _P,
                                              ctypes.POINTER(bltt_solve_info)]),
    "bltt_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "bltt_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(bltt_kernel_stat), ctypes.c_int]),
    "bltt_check_guards": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "bltt_guard_poke": (ctypes.c_int, [_P, ctypes.c_int]),
    "bltt_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(bltt_blocks), ctypes.c_int,
                                             ctypes.c_longlong, _P, _P, _P, _P,
                                             ctypes.POINTER(ctypes.c_double)]),
    "bltt_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(bltt_blocks),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_P),
                                          ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(bltt_solve_opts),
                                          ctypes.POINTER(bltt_solve_info)]),
    "bltt_alpha_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
    "bltt_alpha_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_float, _P]),
    "bltt_alpha_predict": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "bltt_last_error": (ctypes.c_char_p, [_P]),
    "bltt_version": (ctypes.c_char_p, []),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbltt.so (raises OSError if it is missing: build it with build.build())."""
    if not os.path.exists(path):
        raise OSError(f"libbltt.so not found at {path}; run paper_2307_07749_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status, handle=None):
    if status != BLTT_OK:
        msg = lib().bltt_last_error(handle)
        raise BlttError(status, msg.decode() if msg else "")


def _ptr(t, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t, name="array"):
    """Address of a contiguous float64 host array (CPU torch tensor or numpy array)."""
    import torch
    if isinstance(t, torch.Tensor):
        if t.dtype != torch.float64 or t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CPU tensor")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags.c_contiguous:
            raise ValueError(f"{name} must be a C-contiguous float64 array")
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(f"{name} must be a CPU torch.Tensor or a numpy array")


# --------------------------------------------------------------------------------------------
# functions with the C names

def bltt_create(a, b, N, ndim, m, h):
    """Create a handle for blocks A_(k) = a[k] I + b[k] L on the grid (ndim, m, h)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = list(m) + [1] * (3 - len(m))
    h = list(h) + [1.0] * (3 - len(h))
    sp = bltt_space(ndim, (ctypes.c_int * 3)(*m), (ctypes.c_double * 3)(*h))
    blk = bltt_blocks(N, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sp)
    M = int(np.prod(m[:ndim]))
    out = ctypes.c_void_p()
    _check(lib().bltt_create(ctypes.byref(blk), N, M, ctypes.byref(out)))
    return out


def bltt_destroy(handle):
    _check(lib().bltt_destroy(handle))


def bltt_set_stream(handle, stream):
    """stream: a torch.cuda.Stream (or an int cudaStream_t)."""
    s = getattr(stream, "cuda_stream", stream)
    _check(lib().bltt_set_stream(handle, ctypes.c_void_p(int(s) if s else 0)), handle)


def bltt_set_matvec_arith(handle, arith):
    _check(lib().bltt_set_matvec_arith(handle, int(arith)), handle)


def bltt_set_variable_coefficient(handle, faces, abar):
    """faces: one array per axis, the coefficient at the faces along that axis (the grid's shape
    with that axis one longer, x fastest); abar: the preconditioner's constant coefficient."""
    arrs = [np.ascontiguousarray(f, dtype=np.float64).reshape(-1) for f in faces]
    ptrs = (ctypes.POINTER(ctypes.c_double) * 3)(
        *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs],
        *[ctypes.POINTER(ctypes.c_double)() for _ in range(3 - len(arrs))])
    _check(lib().bltt_set_variable_coefficient(handle, ptrs, float(abar)), handle)


def bltt_set_dense_operator(handle, K):
    """K: the dense symmetric spatial operator (M x M); the blocks become a_k I + b_k K."""
    k = np.ascontiguousarray(K, dtype=np.float64)
    _check(lib().bltt_set_dense_operator(handle, k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           handle)


def bltt_set_block_spectra(handle, U, lam):
    """General commuting blocks A_(k) = U diag(lam[k]) U^T: U (M x M, columns the eigenvectors),
    lam (N x M, lam[k, i] the eigenvalue of A_(k) on column i)."""
    u = np.ascontiguousarray(U, dtype=np.float64)
    la = np.ascontiguousarray(lam, dtype=np.float64)
    _check(lib().bltt_set_block_spectra(handle, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        la.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), handle)


def bltt_matvec(handle, x, y, flip=1):
    _check(lib().bltt_matvec(handle, _ptr(x, "x"), _ptr(y, "y"), int(flip)), handle)


def bltt_precond_apply(handle, alpha, v, z, precision=PREC_F64):
    _check(lib().bltt_precond_apply(handle, float(alpha), _ptr(v, "v"), _ptr(z, "z"),
                                    int(precision)), handle)


def bltt_minres_solve_ex(handle, f, alpha, tol, maxit, u, precision=PREC_F64, basis=BASIS_AUTO,
                         precond=PRECOND_ABAC, sync_every=0, raise_on_error=True, rebuild=0,
                         matvec_arith=ARITH_DEFAULT, no_graph=0, single_block=0, defer_window=0,
                         refine=0):
    opts = bltt_solve_opts(precision, basis, precond, sync_every, rebuild, matvec_arith, no_graph,
                           int(single_block), int(defer_window), int(refine))
    info = bltt_solve_info()
    st = lib().bltt_minres_solve_ex(handle, _ptr(f, "f"), float(alpha), float(tol), int(maxit),
                                    ctypes.byref(opts), _ptr(u, "u"), ctypes.byref(info))
    if raise_on_error and st not in (BLTT_OK, 6):
        _check(st, handle)
    return st, info.as_dict()


def bltt_minres_solve_host(handle, f_host, alpha, tol, maxit, u_host, precision=PREC_F64,
                           basis=BASIS_AUTO, precond=PRECOND_ABAC, sync_every=0,
                           raise_on_error=True, rebuild=0, matvec_arith=ARITH_DEFAULT, no_graph=0,
                           defer_window=0, refine=0):
    """bltt_minres_solve_ex with f and u in host memory (pinned for asynchronous copies)."""
    if f_host is u_host:
        raise ValueError("u must not alias f")
    opts = bltt_solve_opts(precision, basis, precond, sync_every, rebuild, matvec_arith, no_graph,
                           0, int(defer_window), int(refine))
    info = bltt_solve_info()
    st = lib().bltt_minres_solve_host(handle, _host_ptr(f_host, "f"), float(alpha), float(tol),
                                      int(maxit), ctypes.byref(opts), _host_ptr(u_host, "u"),
                                      ctypes.byref(info))
    if raise_on_error and st not in (BLTT_OK, 6):
        _check(st, handle)
    return st, info.as_dict()


def bltt_minres_solve(handle, f, alpha, tol, maxit, precision, u):
    info = bltt_solve_info()
    st = lib().bltt_minres_solve(handle, _ptr(f, "f"), float(alpha), float(tol), int(maxit),
                                 int(precision), _ptr(u, "u"), ctypes.byref(info))
    return st, info.as_dict()


def bltt_profile_enable(handle, enable=True):
    _check(lib().bltt_profile_enable(handle, 1 if enable else 0), handle)


def bltt_profile_read(handle):
    """{kernel family: (launches, total_ms, active_launches, active_ms)} since profiling began."""
    arr = (bltt_kernel_stat * 64)()
    k = lib().bltt_profile_read(handle, arr, 64)
    if k < 0:
        raise BlttError(1, "null handle")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms, arr[i].active_launches,
                                   arr[i].active_ms) for i in range(min(k, 64))}


def bltt_check_guards(handle):
    """Number of guard bands read; raises BlttError if one was overwritten."""
    n = ctypes.c_int(0)
    _check(lib().bltt_check_guards(handle, ctypes.byref(n)), handle)
    return n.value


def bltt_guard_poke(handle, band):
    _check(lib().bltt_guard_poke(handle, int(band)), handle)


def bltt_residual_noalloc(a, b, N, ndim, m, h, u, f, r=None, stream=None):
    """||f - A u|| / ||f|| (and r = f - A u into `r` if given) with neither a handle nor any
    allocation by the library; returns the relative residual.  See include/bltt.h."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = list(m) + [1] * (3 - len(m))
    h = list(h) + [1.0] * (3 - len(h))
    sp = bltt_space(ndim, (ctypes.c_int * 3)(*m), (ctypes.c_double * 3)(*h))
    blk = bltt_blocks(N, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sp)
    M = int(np.prod(m[:ndim]))
    out = ctypes.c_double()
    s = getattr(stream, "cuda_stream", stream)
    st = lib().bltt_residual_noalloc(ctypes.byref(blk), N, M, _ptr(u, "u"), _ptr(f, "f"),
                                     _ptr(r, "r") if r is not None else None,
                                     ctypes.c_void_p(int(s) if s else 0), ctypes.byref(out))
    if st != BLTT_OK:
        raise BlttError(st, "bltt_residual_noalloc")
    return out.value


def bltt_solve_batched(problems, fs, us, alpha=None, tol=1e-8, maxit=200, precision=PREC_F64,
                       matvec_arith=ARITH_DEFAULT, autotune=True, defer_window=0):
    """Batched solve.  problems: list of objects with N, d, m, h, a, b; fs / us: list (per
    problem) of lists of float64 CUDA tensors.  Returns (status, list of info dicts, system-major)."""
    nsys = len(problems)
    keep = []
    blocks = (bltt_blocks * nsys)()
    for s, p in enumerate(problems):
        a = np.ascontiguousarray(p.a, dtype=np.float64)
        b = np.ascontiguousarray(p.b, dtype=np.float64)
        keep += [a, b]
        m = list(p.m) + [1] * (3 - len(p.m))
        h = list(p.h) + [1.0] * (3 - len(p.h))
        blocks[s] = bltt_blocks(int(p.N), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                bltt_space(int(p.d), (ctypes.c_int * 3)(*m), (ctypes.c_double * 3)(*h)))
    nrhs = (ctypes.c_int * nsys)(*[len(f) for f in fs])
    tot = sum(len(f) for f in fs)
    fp = (_P * tot)(*[_ptr(t, "f").value for f in fs for t in f])
    up = (_P * tot)(*[_ptr(t, "u").value for u in us for t in u])
    al = None if alpha is None else (ctypes.c_double * nsys)(*[float(x) for x in alpha])
    opts = bltt_solve_opts(precision, BASIS_SPECTRAL, PRECOND_ABAC, 0 if autotune else -1, 0,
                           matvec_arith, 0, 0, int(defer_window))
    infos = (bltt_solve_info * tot)()
    st = lib().bltt_solve_batched(nsys, blocks, nrhs, fp, up, al, float(tol), int(maxit),
                                  ctypes.byref(opts), infos)
    return st, [infos[i].as_dict() for i in range(tot)]


ALPHA_MODEL_FLOATS, ALPHA_NPARAM = 1259, 1249


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def bltt_alpha_grad(model, feats, labels):
    """(gradient [1249], loss) of the MSE of the alpha network on (feats [n,4], labels [n])."""
    model, feats, labels = _f32(model), _f32(feats), _f32(labels)
    g = np.zeros(ALPHA_NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    st = lib().bltt_alpha_grad(model.ctypes.data, feats.ctypes.data, labels.ctypes.data,
                               len(labels), g.ctypes.data, loss.ctypes.data)
    if st != BLTT_OK:
        raise BlttError(st, "bltt_alpha_grad")
    return g, float(loss[0])


def bltt_alpha_train(model, feats, labels, epochs, lr=1e-2):
    """Return (trained model copy, loss history)."""
    model, feats, labels = _f32(model).copy(), _f32(feats), _f32(labels)
    hist = np.zeros(max(epochs, 1), np.float32)
    st = lib().bltt_alpha_train(model.ctypes.data, feats.ctypes.data, labels.ctypes.data,
                                len(labels), int(epochs), float(lr), hist.ctypes.data)
    if st != BLTT_OK:
        raise BlttError(st, "bltt_alpha_train")
    return model, hist[:epochs]


def bltt_alpha_predict(model, feats):
    model, feats = _f32(model), _f32(feats)
    out = np.zeros(len(feats), np.float32)
    st = lib().bltt_alpha_predict(model.ctypes.data, feats.ctypes.data, len(feats), out.ctypes.data)
    if st != BLTT_OK:
        raise BlttError(st, "bltt_alpha_predict")
    return out


def bltt_version():
    return lib().bltt_version().decode()


# --------------------------------------------------------------------------------------------
class Solver:
    """A BLTT system on the GPU: wraps one libbltt handle.

    prob: any object with N, d, m, h, a, b (e.g. workloads.Problem).
    """

    def __init__(self, prob, stream=None):
        self.N, self.d = int(prob.N), int(prob.d)
        self.m = tuple(int(v) for v in prob.m)
        self.M = int(np.prod(self.m))
        self.n = self.N * self.M
        meta = getattr(prob, "meta", None) or {}
        spectra = meta.get("U") is not None and meta.get("lam") is not None
        if spectra:
            # general commuting blocks: the handle is created with the identity blocks (a = e_0,
            # b = 0), which the blocks' eigenvalues then replace
            a0 = np.zeros(self.N)
            a0[0] = 1.0
            self.handle = bltt_create(a0, np.zeros(self.N), self.N, self.d, self.m, tuple(prob.h))
        else:
            self.handle = bltt_create(prob.a, prob.b, self.N, self.d, self.m, tuple(prob.h))
        if meta.get("faces") is not None:
            # variable coefficient: L_a in the matvec, the mean coefficient in the preconditioner
            bltt_set_variable_coefficient(self.handle, meta["faces"], meta["abar"])
        if meta.get("K") is not None:
            # commuting dense blocks a_k I + b_k K: the solve runs in K's eigenbasis
            bltt_set_dense_operator(self.handle, meta["K"])
        if spectra:
            bltt_set_block_spectra(self.handle, meta["U"], meta["lam"])
        if stream is not None:
            bltt_set_stream(self.handle, stream)

    def close(self):
        if self.handle:
            bltt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_matvec_arith(self, arith):
        bltt_set_matvec_arith(self.handle, arith)

    def profile(self, enable=True):
        bltt_profile_enable(self.handle, enable)

    def profile_read(self):
        return bltt_profile_read(self.handle)

    def set_stream(self, stream):
        bltt_set_stream(self.handle, stream)

    def matvec(self, x, y=None, flip=True):
        import torch
        y = torch.empty_like(x) if y is None else y
        bltt_matvec(self.handle, x, y, 1 if flip else 0)
        return y

    def precond_apply(self, alpha, v, z=None, precision=PREC_F64):
        import torch
        z = torch.empty_like(v) if z is None else z
        bltt_precond_apply(self.handle, alpha, v, z, precision)
        return z

    def solve(self, f, alpha=1e-8, tol=1e-8, maxit=200, precision=PREC_F64, basis=BASIS_AUTO,
              precond=PRECOND_ABAC, u=None, sync_every=0, raise_on_error=True, rebuild=False,
              matvec_arith=ARITH_DEFAULT, graph=True, single_block=False, defer_window=0,
              refine=0):
        """single_block: the whole solve in one launch of one block (small problems, FP64).
        defer_window: iterations whose (w, x) update is deferred (0: 8, -1: none).
        refine: outer iterative-refinement corrections allowed (0: none)."""
        import torch
        u = torch.empty_like(f) if u is None else u
        st, info = bltt_minres_solve_ex(self.handle, f, alpha, tol, maxit, u, precision, basis,
                                        precond, sync_every, raise_on_error, int(rebuild),
                                        matvec_arith, 0 if graph else 1, int(single_block),
                                        int(defer_window), int(refine))
        info["status_name"] = STATUS_NAMES.get(st, st)
        return u, info

    def solve_host(self, f_host, alpha=1e-8, tol=1e-8, maxit=200, precision=PREC_F64,
                   basis=BASIS_AUTO, precond=PRECOND_ABAC, u_host=None, sync_every=0,
                   raise_on_error=True, rebuild=False, matvec_arith=ARITH_DEFAULT, graph=True,
                   defer_window=0, refine=0):
        """solve() with f and u in host memory; u_host defaults to a pinned tensor."""
        import torch
        if u_host is None:
            u_host = torch.empty(f_host.shape, dtype=torch.float64, pin_memory=True)
        st, info = bltt_minres_solve_host(self.handle, f_host, alpha, tol, maxit, u_host,
                                          precision, basis, precond, sync_every, raise_on_error,
                                          int(rebuild), matvec_arith, 0 if graph else 1,
                                          int(defer_window), int(refine))
        info["status_name"] = STATUS_NAMES.get(st, st)
        return u_host, info
