"""Thin Python binding of the C ABI in include/fcgle.h (argument marshalling only).

Every function of the C ABI is exposed under the same name and takes torch
tensors (device memory, complex128 for FP64 handles / complex64 for BF16X3
handles, shape (n_d, ..., n_1) contiguous = vec order with j_1 fastest) or
plain Python numbers.  All arithmetic happens in libfcgle.so; if the library
is missing this module raises at import time (there is no fallback).

``Solver`` is a convenience wrapper that owns a handle.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcgle.so")

FCGLE_OK = 0
FCGLE_ERR_INVALID_ARG = 1
FCGLE_ERR_NOMEM = 2
FCGLE_ERR_CUDA = 3
FCGLE_ERR_NUMERIC = 4
FCGLE_ERR_TIMEOUT = 5
FCGLE_ERR_UNSUPPORTED = 6

FCGLE_FP64 = 0
FCGLE_TF32 = 1      # not built: fcgle_setup answers FCGLE_ERR_UNSUPPORTED
FCGLE_BF16X3 = 2

FCGLE_EXP_TUCKER = 0
FCGLE_EXP_KRON = 1
EXP_FORMS = {"tucker": FCGLE_EXP_TUCKER, "kron": FCGLE_EXP_KRON}

FCGLE_TUCKER_AUTO = 0
FCGLE_TUCKER_ROTATING = 1
FCGLE_TUCKER_SLAB = 2
TUCKER_FORMS = {"auto": FCGLE_TUCKER_AUTO, "rotating": FCGLE_TUCKER_ROTATING, "slab": FCGLE_TUCKER_SLAB}

FCGLE_F_INV = 0
FCGLE_F_EXP = 1
FCGLE_F_PHI = 2

SCHEMES = {"lie": 0, "lawson_euler": 1, "lawson_rk2": 2, "etd2rk": 3, "krogstad": 4, "lbdf2": 5, "strang": 6}
FUNCS = {"inv": FCGLE_F_INV, "exp": FCGLE_F_EXP, "phi": FCGLE_F_PHI}
PRECISIONS = {"fp64": FCGLE_FP64, "bf16x3": FCGLE_BF16X3}

# exported symbols of include/fcgle.h (checked by the CPU tests)
EXPORTS = ["fcgle_setup", "fcgle_set_stream", "fcgle_set_source", "fcgle_apply_f", "fcgle_step",
           "fcgle_integrate", "fcgle_integrate_host", "fcgle_norm", "fcgle_sync", "fcgle_sizes",
           "fcgle_launch_count", "fcgle_destroy", "fcgle_status_string", "fcgle_last_error",
           "fcgle_internal_elems", "fcgle_mode_product", "fcgle_adjoint", "fcgle_set_coefficients",
           "fcgle_batch_create", "fcgle_batch_instance", "fcgle_batch_integrate", "fcgle_batch_launch_count",
           "fcgle_batch_destroy", "fcgle_norm_static", "fcgle_selftest_bounded_wait", "fcgle_spectral_scalars",
           "fcgle_autotune_report", "fcgle_set_exp_form", "fcgle_set_tucker_form"]


class fcgle_params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int * 3), ("a", ctypes.c_double * 3),
                ("b", ctypes.c_double * 3), ("alpha", ctypes.c_double * 3),
                ("nu", ctypes.c_double), ("eta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kappa", ctypes.c_double), ("zeta", ctypes.c_double),
                ("fd_order", ctypes.c_int), ("precision", ctypes.c_int)]


class FcgleError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2510_21394_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sig = {
        "fcgle_setup": [ctypes.POINTER(fcgle_params), P, ctypes.POINTER(H)],
        "fcgle_set_stream": [H, P],
        "fcgle_set_source": [H, I, ctypes.POINTER(D), ctypes.POINTER(P)],
        "fcgle_apply_f": [H, I, I, D, P, P],
        "fcgle_step": [H, I, D, D, P],
        "fcgle_integrate": [H, I, D, I, D, P, P],
        "fcgle_integrate_host": [H, I, D, I, D, P, P],
        "fcgle_norm": [H, P, ctypes.POINTER(D)],
        "fcgle_sync": [H],
        "fcgle_sizes": [H, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
        "fcgle_launch_count": [H, ctypes.POINTER(ctypes.c_longlong)],
        "fcgle_destroy": [H],
        "fcgle_internal_elems": [H, ctypes.POINTER(ctypes.c_size_t)],
        "fcgle_mode_product": [H, I, I, P, P],
        "fcgle_adjoint": [H, I, D, I, D, P, P, I, P, ctypes.POINTER(D), ctypes.POINTER(D)],
        "fcgle_set_coefficients": [H, D, D, D, D, D],
        "fcgle_batch_create": [I, ctypes.POINTER(fcgle_params), P, I, ctypes.POINTER(H)],
        "fcgle_batch_instance": [H, I, ctypes.POINTER(H)],
        "fcgle_batch_integrate": [H, I, D, I, D, ctypes.POINTER(P), ctypes.POINTER(P), I],
        "fcgle_batch_launch_count": [H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
        "fcgle_batch_destroy": [H],
        "fcgle_norm_static": [ctypes.POINTER(fcgle_params), P, P, ctypes.POINTER(D)],
        "fcgle_selftest_bounded_wait": [P, ctypes.POINTER(I)],
        "fcgle_spectral_scalars": [H, I, I, D, I, ctypes.POINTER(D), ctypes.POINTER(D), I],
        "fcgle_autotune_report": [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
        "fcgle_set_exp_form": [H, I],
        "fcgle_set_tucker_form": [H, I],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fcgle_status_string.argtypes = [ctypes.c_int]
    lib.fcgle_status_string.restype = ctypes.c_char_p
    lib.fcgle_last_error.argtypes = []
    lib.fcgle_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def status_name(s):
    return _lib.fcgle_status_string(int(s)).decode()


def _check(status):
    if status != FCGLE_OK:
        raise FcgleError(status, _lib.fcgle_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------ C ABI mirror
def make_params(ns, boxes, alphas, nu, eta, gamma, kappa, zeta, fd_order=2, precision="fp64"):
    p = fcgle_params()
    p.d = len(ns)
    for mu in range(3):
        p.n[mu] = int(ns[mu]) if mu < p.d else 1
        p.a[mu] = float(boxes[mu][0]) if mu < p.d else 0.0
        p.b[mu] = float(boxes[mu][1]) if mu < p.d else 1.0
        p.alpha[mu] = float(alphas[mu]) if mu < p.d else 1.5
    p.nu, p.eta, p.gamma, p.kappa, p.zeta = map(float, (nu, eta, gamma, kappa, zeta))
    p.fd_order = int(fd_order)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return p


def fcgle_setup(ns, boxes, alphas, nu, eta, gamma, kappa, zeta, fd_order=2, precision="fp64", stream=None):
    p = make_params(ns, boxes, alphas, nu, eta, gamma, kappa, zeta, fd_order, precision)
    h = ctypes.c_void_p()
    _check(_lib.fcgle_setup(ctypes.byref(p), _stream(stream), ctypes.byref(h)))
    return h


def fcgle_batch_create(params_list, stream=None, nstreams=0):
    arr = (fcgle_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(_lib.fcgle_batch_create(len(params_list), arr, _stream(stream), int(nstreams), ctypes.byref(b)))
    return b


def fcgle_batch_instance(b, i):
    h = ctypes.c_void_p()
    _check(_lib.fcgle_batch_instance(b, int(i), ctypes.byref(h)))
    return h


def fcgle_batch_integrate(b, scheme, tau, nsteps, t0, u0_list, uT_list, use_graph=True):
    scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    n = len(u0_list)
    a = (ctypes.c_void_p * n)(*[_ptr(t).value for t in u0_list])
    o = (ctypes.c_void_p * n)(*[_ptr(t).value for t in uT_list])
    _check(_lib.fcgle_batch_integrate(b, scheme, float(tau), int(nsteps), float(t0), a, o, int(use_graph)))


def fcgle_batch_launch_count(b):
    k = ctypes.c_longlong()
    g = ctypes.c_longlong()
    _check(_lib.fcgle_batch_launch_count(b, ctypes.byref(k), ctypes.byref(g)))
    return k.value, g.value


def fcgle_batch_destroy(b):
    _check(_lib.fcgle_batch_destroy(b))


def fcgle_set_stream(h, stream=None):
    _check(_lib.fcgle_set_stream(h, _stream(stream)))


def fcgle_set_source(h, sigmas, tensors):
    n = len(sigmas)
    sig = (ctypes.c_double * max(1, 2 * n))()
    for k, s in enumerate(sigmas):
        s = complex(s)
        sig[2 * k], sig[2 * k + 1] = s.real, s.imag
    ptrs = (ctypes.c_void_p * max(1, n))(*[t.data_ptr() for t in tensors])
    _check(_lib.fcgle_set_source(h, n, sig, ptrs))


def fcgle_set_coefficients(h, nu, eta, gamma, kappa, zeta):
    _check(_lib.fcgle_set_coefficients(h, float(nu), float(eta), float(gamma), float(kappa), float(zeta)))


def fcgle_set_exp_form(h, form):
    form = EXP_FORMS[form] if isinstance(form, str) else int(form)
    _check(_lib.fcgle_set_exp_form(h, form))


def fcgle_set_tucker_form(h, form):
    form = TUCKER_FORMS[form] if isinstance(form, str) else int(form)
    _check(_lib.fcgle_set_tucker_form(h, form))


def fcgle_apply_f(h, func, k, theta, v, out):
    func = FUNCS[func] if isinstance(func, str) else int(func)
    _check(_lib.fcgle_apply_f(h, func, int(k), float(theta), _ptr(v), _ptr(out)))


def fcgle_spectral_scalars(h, func, k, theta, s, flags=0):
    """f(theta (nu + i eta) s_j) for a list of real eigenvalue sums s, evaluated
    on the device by the handle's own arithmetic; returns a list of complex."""
    func = FUNCS[func] if isinstance(func, str) else int(func)
    s = [float(x) for x in s]
    n = len(s)
    sin = (ctypes.c_double * max(1, n))(*s)
    out = (ctypes.c_double * max(1, 2 * n))()
    _check(_lib.fcgle_spectral_scalars(h, func, int(k), float(theta), n, sin, out, int(flags)))
    return [complex(out[2 * j], out[2 * j + 1]) for j in range(n)]


def fcgle_autotune_report():
    """The autotuner's timings and choices so far (one line per tuned shape)."""
    need = ctypes.c_size_t()
    _check(_lib.fcgle_autotune_report(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(max(1, need.value))
    _check(_lib.fcgle_autotune_report(buf, len(buf), None))
    return buf.value.decode()


def fcgle_step(h, scheme, tau, t, u):
    scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(_lib.fcgle_step(h, scheme, float(tau), float(t), _ptr(u)))


def fcgle_integrate(h, scheme, tau, nsteps, t0, u0, uT):
    scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(_lib.fcgle_integrate(h, scheme, float(tau), int(nsteps), float(t0), _ptr(u0), _ptr(uT)))


def fcgle_integrate_host(h, scheme, tau, nsteps, t0, u0, uT):
    scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(_lib.fcgle_integrate_host(h, scheme, float(tau), int(nsteps), float(t0), _ptr(u0), _ptr(uT)))


def fcgle_adjoint(h, scheme, tau, nsteps, t0, u0, u_target, ckpt_every, grad_u0):
    """Returns (loss, [dJ/dnu, dJ/deta, dJ/dgamma, dJ/dkappa, dJ/dzeta]); grad_u0 is written."""
    scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    gp = (ctypes.c_double * 5)()
    loss = ctypes.c_double()
    _check(_lib.fcgle_adjoint(h, scheme, float(tau), int(nsteps), float(t0), _ptr(u0), _ptr(u_target),
                              int(ckpt_every), _ptr(grad_u0), gp, ctypes.byref(loss)))
    return loss.value, list(gp)


def fcgle_norm(h, u):
    out = ctypes.c_double()
    _check(_lib.fcgle_norm(h, _ptr(u), ctypes.byref(out)))
    return out.value


def _check_norm_static_tensor(params, u):
    """A torch tensor given to fcgle_norm_static must hold exactly the tensor
    that params describe: complex128 for FP64, complex64 for BF16X3, prod(n)
    entries, contiguous, on the current CUDA device (the C side trusts these)."""
    want = torch.complex128 if params.precision == FCGLE_FP64 else torch.complex64
    n = 1
    for mu in range(max(0, min(3, params.d))):
        n *= int(params.n[mu])
    bad = None
    if u.dtype != want:
        bad = f"u has dtype {u.dtype}, the precision needs {want}"
    elif u.numel() != n:
        bad = f"u has {u.numel()} entries, params describe {n}"
    elif not u.is_contiguous():
        bad = "u must be contiguous"
    elif not u.is_cuda:
        bad = "u must be a CUDA tensor"
    elif u.device.index != torch.cuda.current_device():
        bad = f"u is on cuda:{u.device.index} but cuda:{torch.cuda.current_device()} is current"
    if bad:
        raise FcgleError(FCGLE_ERR_INVALID_ARG, bad)


def fcgle_norm_static(params, u, stream=None):
    """Discrete L2 norm without a handle or device allocation; u is a device
    tensor (checked against params) or a raw device address (int)."""
    out = ctypes.c_double()
    if not isinstance(u, int):
        _check_norm_static_tensor(params, u)
    ptr = ctypes.c_void_p(u) if isinstance(u, int) else _ptr(u)
    st = ctypes.c_void_p(0) if (stream is None and isinstance(u, int)) else _stream(stream)
    _check(_lib.fcgle_norm_static(ctypes.byref(params), ptr, st, ctypes.byref(out)))
    return out.value


def fcgle_selftest_bounded_wait(stream=None):
    """Runs the bounded-wait self-test; returns (status, code).  The expected
    outcome is (FCGLE_ERR_TIMEOUT, 99): the wait gave up at its limit and
    reported it, and the context still ran the follow-up kernel."""
    code = ctypes.c_int(-1)
    status = _lib.fcgle_selftest_bounded_wait(_stream(stream), ctypes.byref(code))
    return status, code.value


def fcgle_sync(h):
    _check(_lib.fcgle_sync(h))


def fcgle_sizes(h):
    n = ctypes.c_size_t()
    b = ctypes.c_size_t()
    _check(_lib.fcgle_sizes(h, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def fcgle_launch_count(h):
    c = ctypes.c_longlong()
    _check(_lib.fcgle_launch_count(h, ctypes.byref(c)))
    return c.value


def fcgle_internal_elems(h):
    n = ctypes.c_size_t()
    _check(_lib.fcgle_internal_elems(h, ctypes.byref(n)))
    return n.value


def fcgle_mode_product(h, direction, forward, X, Y):
    """X, Y: flat device tensors in the internal layout: 2 P reals (float64 / float32), or with
    bit 1 of `forward` (the C flags) set (BF16X3 handles) 4 P bf16 (hi planes, then lo planes).
    Bit 0 forward (Q^T), bit 2 the precise split-TF32 product (FP32 in and out), bit 3 the
    slab-fused modes 1 + 2 (3D, direction 0), bit 4 the last direction on a natural-order input."""
    _check(_lib.fcgle_mode_product(h, int(direction), int(forward), _ptr(X), _ptr(Y)))


def fcgle_destroy(h):
    _check(_lib.fcgle_destroy(h))


def fcgle_status_string(s):
    return status_name(s)


def fcgle_last_error():
    return _lib.fcgle_last_error().decode()


# ------------------------------------------------------------ convenience
class Solver:
    """Owns one handle; tensors are torch tensors of shape (n_d, ..., n_1)."""

    def __init__(self, ns, boxes, alphas, nu, eta, gamma, kappa, zeta, fd_order=2, precision="fp64",
                 stream=None):
        self.ns = list(ns)
        self.shape = tuple(reversed(self.ns))
        self.precision = precision
        self.dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.h = fcgle_setup(ns, boxes, alphas, nu, eta, gamma, kappa, zeta, fd_order, precision, stream)
        self._src = None

    def close(self):
        if self.h is not None:
            fcgle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t):
        if t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_cuda:
            raise ValueError(f"expected a CUDA {self.dtype} tensor of shape {self.shape}")
        return t

    def set_source(self, sigmas, tensors):
        tensors = [self._check_tensor(t.contiguous()) for t in tensors]
        fcgle_set_source(self.h, sigmas, tensors)

    def set_coefficients(self, nu, eta, gamma, kappa, zeta):
        fcgle_set_coefficients(self.h, nu, eta, gamma, kappa, zeta)

    def set_exp_form(self, form):
        """'tucker' (default for bf16x3) or 'kron' (Kronecker-product form of e^{tau K})."""
        fcgle_set_exp_form(self.h, form)

    def set_tucker_form(self, form):
        """'auto' (default), 'rotating' or 'slab' (3D split-BF16: modes 1 + 2 fused per slab)."""
        fcgle_set_tucker_form(self.h, form)

    def apply_f(self, func, k, theta, v, out=None):
        v = self._check_tensor(v.contiguous())
        out = torch.empty_like(v) if out is None else out
        fcgle_apply_f(self.h, func, k, theta, v, out)
        return out

    def step(self, scheme, tau, t, u):
        fcgle_step(self.h, scheme, tau, t, self._check_tensor(u))
        return u

    def integrate(self, scheme, tau, nsteps, u0, t0=0.0, out=None):
        u0 = self._check_tensor(u0.contiguous())
        out = torch.empty_like(u0) if out is None else out
        fcgle_integrate(self.h, scheme, tau, nsteps, t0, u0, out)
        return out

    def integrate_host(self, scheme, tau, nsteps, u0_host, out_host, t0=0.0):
        fcgle_integrate_host(self.h, scheme, tau, nsteps, t0, u0_host, out_host)
        return out_host

    def adjoint(self, scheme, tau, nsteps, u0, u_target, ckpt_every=25, t0=0.0):
        """(loss, grad_u0, grad_params) of J = 1/2 ||u(T) - u_target||^2."""
        u0 = self._check_tensor(u0.contiguous())
        u_target = self._check_tensor(u_target.contiguous())
        g = torch.empty_like(u0)
        loss, gp = fcgle_adjoint(self.h, scheme, tau, nsteps, t0, u0, u_target, ckpt_every, g)
        return loss, g, gp

    def norm(self, u):
        return fcgle_norm(self.h, self._check_tensor(u))

    def sync(self):
        fcgle_sync(self.h)

    def launches(self):
        return fcgle_launch_count(self.h)


class Batch:
    """Many independent instances advanced together (see fcgle_batch_* in include/fcgle.h).

    specs: list of dicts with keys ns, boxes, alphas, nu, eta, gamma, kappa, zeta
    (and optionally fd_order); all instances share one precision."""

    def __init__(self, specs, precision="bf16x3", stream=None, nstreams=0):
        self.precision = precision
        self.dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.shapes = [tuple(reversed(list(sp["ns"]))) for sp in specs]
        plist = [make_params(sp["ns"], sp["boxes"], sp["alphas"], sp["nu"], sp["eta"], sp["gamma"], sp["kappa"],
                             sp["zeta"], sp.get("fd_order", 2), precision) for sp in specs]
        self.b = fcgle_batch_create(plist, stream, nstreams)

    def instance(self, i):
        return fcgle_batch_instance(self.b, i)

    def integrate(self, scheme, tau, nsteps, u0_list, t0=0.0, out=None, use_graph=True, grouped=False):
        """grouped=True: one persistent launch per phase of a step over all instances."""
        out = [torch.empty_like(u) for u in u0_list] if out is None else out
        mode = 2 if grouped else (1 if use_graph else 0)
        fcgle_batch_integrate(self.b, scheme, tau, nsteps, t0, u0_list, out, mode)
        return out

    def launches(self):
        return fcgle_batch_launch_count(self.b)

    def close(self):
        if self.b is not None:
            fcgle_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
