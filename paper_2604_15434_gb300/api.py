"""Python binding of the ``libpmeft.so`` C ABI (``include/pmeft.h``): argument marshalling only.

Every function takes torch CUDA tensors, checks dtype / device / layout, and passes raw
pointers to the entry point of the same name; all computation happens in the CUDA
library.  There is no CPU fallback: if ``libpmeft.so`` is missing or fails to load, every
call raises.  Build the library with ``python -m paper_2604_15434_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpmeft.so")

PM_OK, PM_ERR_INVALID_ARG, PM_ERR_CUDA, PM_ERR_OOM, PM_ERR_NONFINITE, PM_ERR_NOCONV, PM_ERR_TIMEOUT, \
    PM_ERR_OVERFLOW, PM_ERR_TOO_LARGE = range(9)
_STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_CUDA", 3: "PM_ERR_OOM", 4: "PM_ERR_NONFINITE",
           5: "PM_ERR_NOCONV", 6: "PM_ERR_TIMEOUT", 7: "PM_ERR_OVERFLOW", 8: "PM_ERR_TOO_LARGE"}


class PMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("omega_m0", ctypes.c_double), ("eta", ctypes.c_double), ("npre", ctypes.c_int),
                ("npost", ctypes.c_int), ("max_cycles", ctypes.c_int), ("coarsest_n", ctypes.c_int),
                ("coarse_sweeps", ctypes.c_int), ("precision", ctypes.c_int), ("include_dot_alphaB", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("autotune", ctypes.c_int), ("linear_eft", ctypes.c_int),
                ("smoother", ctypes.c_int), ("coarse_exact", ctypes.c_int), ("grad_order", ctypes.c_int),
                ("batch_persistent", ctypes.c_int), ("zero_start", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("vcycles", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("lam", ctypes.c_double), ("floored_cells", ctypes.c_longlong), ("unstable_nu", ctypes.c_int),
                ("rel_res_hist", ctypes.c_double * 64), ("ms_total", ctypes.c_double),
                ("guess_rel_res", ctypes.c_double), ("guess_rejected", ctypes.c_int)]

    def as_dict(self) -> dict:
        k = min(self.cycles + 1, 64)
        return {"cycles": self.cycles, "vcycles": self.vcycles, "status": self.status, "rel_res": self.rel_res, "lambda": self.lam,
                "floored_cells": self.floored_cells, "unstable_nu": self.unstable_nu,
                "hist": list(self.rel_res_hist[:k]), "ms_total": self.ms_total,
                "guess_rel_res": self.guess_rel_res, "guess_rejected": self.guess_rejected}


class Coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "omega_m_a", "alpha_B", "alpha_M", "geff", "E2", "C2", "C4", "nu", "xi", "kappa", "mu_chi", "mu_psi",
        "src", "poisson_fac")]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_D, _I, _LL, _P = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
SIGNATURES = {
    "pm_default_params": (None, [_P]),
    "pm_coefficients": (_I, [_D, _D, _D, _D, _I, _P]),
    "pm_create": (_I, [_P, _I, _P, _P]),
    "pm_destroy": (None, [_P]),
    "pm_last_error": (ctypes.c_char_p, [_P]),
    "pm_set_params": (_I, [_P, _P]),
    "pm_deposit_cic": (_I, [_P, _P, _LL, _I, _P]),
    "pm_deposit_cic_fixed": (_I, [_P, _P, _LL, _I, _P]),
    "poisson_solve": (_I, [_P, _P, _I, _D, _D, _P]),
    "scalar_mg_solve": (_I, [_P, _P, _I, _D, _D, _D, _D, _P, _P]),
    "force_interp": (_I, [_P, _P, _P, _I, _D, _D, _D, _P, _LL, _P]),
    "pm_step": (_I, [_P, _P, _P, _LL, _I, _D, _D, _D, _D, _D, _P, _P]),
    "pm_mg_sweep": (_I, [_P, _P, _P, _D, _I, _D, _D, _D, _P]),
    "pm_mg_residual": (_I, [_P, _P, _P, _D, _I, _D, _D, _D, _P, _P, _P]),
    "pm_mg_coarse_exact": (_I, [_P, _P, _P, _I, _D, _D, _D, _P, _P]),
    "pm_batch_barrier_test": (_I, [_P, _I, _I, _D]),
    "pm_mg_restrict": (_I, [_P, _P, _I, _P]),
    "pm_mg_prolong_add": (_I, [_P, _P, _I, _P]),
    "pm_trace_enable": (_I, [_P, _I]),
    "pm_trace_select": (_I, [_P, ctypes.c_uint, _I]),
    "pm_trace_get": (_I, [_P, _P]),
    "pm_trace_reset": (_I, [_P]),
    "pm_probe_fma": (_I, [_P, _P, _P]),
    "pm_deposit_cic_static": (_I, [_P, _LL, _I, _P, _P]),
    "lensing_potential": (_I, [_P, _P, _P, _I, _D, _D, _D, _P]),
    "pm_run": (_I, [_P, _P, _P, _LL, _I, _D, _D, _D, _D, _I, _D, _P, _P]),
    "pm_mg_sweep_f32": (_I, [_P, _P, _P, ctypes.c_float, _I, _D, _D, _D, _P, _P, _P, _I]),
    "pm_tune_log": (_I, [_P, _P, _I]),
    "scalar_mg_solve_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _D, _P, _P]),
    "pm_unet_num_params": (_LL, []),
    "pm_unet_create": (_I, [_P, _P]),
    "pm_unet_set_conv_path": (_I, [_P, _I]),
    "pm_unet_destroy": (None, [_P]),
    "pm_unet_set_params": (_I, [_P, _P, _LL]),
    "pm_unet_get_params": (_I, [_P, _P, _LL, _I]),
    "pm_unet_forward": (_I, [_P, _P, _I, _D, _D, _D, _P]),
    "pm_unet_loss_grad": (_I, [_P, _P, _P, _I, _D, _D, _D, _P]),
    "pm_unet_adam_step": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "pm_unet_zero_grad": (_I, [_P]),
    "pm_unet_target": (_I, [_P, _P, _I, _D, _D, _D, _P]),
    "pm_unet_warm_start": (_I, [_P, _P, _I, _D, _D, _D, _P]),
    "pm_linear_start": (_I, [_P, _P, _I, _D, _D, _D, _P]),
}

KERNEL_CLASSES = ("sweep64", "sweep32", "resid64", "resid32", "transfer", "coarsest", "reduce", "pm")


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 8), ("ms", ctypes.c_double * 8), ("cells", ctypes.c_longlong * 8),
                ("fine_launches", ctypes.c_longlong * 8), ("fine_ms", ctypes.c_double * 8)]

    def as_dict(self) -> dict:
        return {k: {"launches": self.launches[i], "ms": self.ms[i], "cells": self.cells[i],
                    "fine_launches": self.fine_launches[i], "fine_ms": self.fine_ms[i]}
                for i, k in enumerate(KERNEL_CLASSES)}


def load():
    """Load libpmeft.so and declare the C signatures; raises if the library is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2604_15434_gb300.build`")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def default_params(**overrides) -> Params:
    p = Params()
    load().pm_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def coefficients(alpha_B0, alpha_M0, a, omega_m0=0.3, include_dot_alphaB=True) -> dict:
    c = Coeffs()
    st = load().pm_coefficients(alpha_B0, alpha_M0, a, omega_m0, int(bool(include_dot_alphaB)), ctypes.byref(c))
    if st != PM_OK:
        raise PMError(st, "pm_coefficients: invalid argument")
    return {n: getattr(c, n) for n, _ in Coeffs._fields_}


class Context:
    """Owns a ``pm_ctx``: device scratch (multigrid levels, FFT plans) and the stream it enqueues on."""

    def __init__(self, device=None, stream=None, **params):
        lib = load()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.params = default_params(**params)
        h = ctypes.c_void_p()
        st = lib.pm_create(ctypes.byref(h), dev.index, ctypes.c_void_p(self.stream.cuda_stream),
                           ctypes.byref(self.params))
        if st != PM_OK:
            raise PMError(st, "pm_create failed")
        self._h = h

    def set_params(self, **params):
        for k, v in params.items():
            setattr(self.params, k, v)
        self._check(load().pm_set_params(self._h, ctypes.byref(self.params)))

    def _check(self, st):
        if st != PM_OK:
            msg = load().pm_last_error(self._h)
            raise PMError(st, msg.decode() if msg else "")

    def batch_barrier_test(self, block: int, barrier: int = 0, wait_s: float = 0.0):
        """Make block `block` of the batched solve's persistent kernel leave before barrier
        `barrier`, so that the others' bounded waits (wait_s seconds) run out; block < 0 undoes it
        (see pm_batch_barrier_test)."""
        self._check(load().pm_batch_barrier_test(self._h, int(block), int(barrier), float(wait_s)))

    def trace(self, on: bool = True):
        """Per-launch CUDA-event tracing of the library's kernels (see pm_trace_enable)."""
        self._check(load().pm_trace_enable(self._h, int(bool(on))))

    def trace_select(self, classes, fine_only: bool = False):
        """Trace only the launches of the given PM_K_* class indices (see pm_trace_select)."""
        mask = 0
        for c in classes:
            mask |= 1 << int(c)
        self._check(load().pm_trace_select(self._h, mask, int(bool(fine_only))))

    def trace_get(self) -> dict:
        p = Profile()
        self._check(load().pm_trace_get(self._h, ctypes.byref(p)))
        return p.as_dict()

    def trace_reset(self):
        self._check(load().pm_trace_reset(self._h))

    def tune_log(self) -> str:
        full = load().pm_tune_log(self._h, None, 0)
        buf = ctypes.create_string_buffer(full + 1)
        load().pm_tune_log(self._h, buf, full + 1)
        return buf.value.decode()

    def probe_fma(self):
        """(FP64, FP32) FMA throughput of this device in GFLOP/s."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(load().pm_probe_fma(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            load().pm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context() -> Context:
    dev = torch.cuda.current_device()
    s = torch.cuda.current_stream(dev)
    key = (dev, s.cuda_stream)
    if key not in _default_ctx:
        _default_ctx[key] = Context(dev, s)
    return _default_ctx[key]


def _ptr(t: torch.Tensor | None, dtype=torch.float64, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def pm_deposit_cic(pos, n, delta=None, ctx=None):
    """delta (n,n,n) float64 from particle positions pos (3, np) float64 in [0,1)."""
    ctx = ctx or default_context()
    npart = pos.shape[1]
    if delta is None:
        delta = torch.empty((n, n, n), dtype=torch.float64, device=pos.device)
    ctx._check(load().pm_deposit_cic(ctx._h, _ptr(pos, name="pos"), npart, n, _ptr(delta, shape=(n, n, n))))
    return delta


def pm_deposit_cic_fixed(pos, n, acc=None, ctx=None):
    ctx = ctx or default_context()
    if acc is None:
        acc = torch.empty((n, n, n), dtype=torch.int64, device=pos.device)
    ctx._check(load().pm_deposit_cic_fixed(ctx._h, _ptr(pos, name="pos"), pos.shape[1], n,
                                           _ptr(acc, torch.int64, (n, n, n), "acc")))
    return acc


def poisson_solve(delta, a, alpha_M0, psi=None, ctx=None):
    ctx = ctx or default_context()
    n = delta.shape[0]
    if psi is None:
        psi = torch.empty_like(delta)
    ctx._check(load().poisson_solve(ctx._h, _ptr(delta, shape=(n, n, n)), n, a, alpha_M0, _ptr(psi, shape=(n, n, n))))
    return psi


def scalar_mg_solve(delta, alpha_B0, alpha_M0, a, tol, phi=None, ctx=None, raise_on_noconv=True):
    """chi for the density contrast delta; phi (in/out) is the initial guess.  Returns (phi, info)."""
    ctx = ctx or default_context()
    n = delta.shape[0]
    if phi is None:
        phi = torch.zeros_like(delta)
    info = SolveInfo()
    st = load().scalar_mg_solve(ctx._h, _ptr(delta, shape=(n, n, n), name="delta"), n, alpha_B0, alpha_M0, a, tol,
                                _ptr(phi, shape=(n, n, n), name="phi"), ctypes.byref(info))
    if st != PM_OK and (raise_on_noconv or st != PM_ERR_NOCONV):
        ctx._check(st)
    return phi, info.as_dict()


def scalar_mg_solve_batched(deltas, alpha_B0, alpha_M0, a, tol, phis=None, ctx=None, raise_on_noconv=True):
    """Solve many boxes at once (see scalar_mg_solve_batched in pmeft.h).  deltas: list of
    (n_b, n_b, n_b) float64 CUDA tensors; alpha_B0, alpha_M0, a: sequences.  Returns (phis, infos)."""
    ctx = ctx or default_context()
    nb = len(deltas)
    if phis is None:
        phis = [torch.zeros_like(d) for d in deltas]
    ns = (ctypes.c_int * nb)(*[d.shape[0] for d in deltas])
    dp = (ctypes.c_void_p * nb)(*[_ptr(d, shape=(d.shape[0],) * 3, name="delta").value for d in deltas])
    pp = (ctypes.c_void_p * nb)(*[_ptr(p, shape=(d.shape[0],) * 3, name="phi").value for p, d in zip(phis, deltas)])
    aB = (ctypes.c_double * nb)(*alpha_B0)
    aM = (ctypes.c_double * nb)(*alpha_M0)
    aa = (ctypes.c_double * nb)(*a)
    infos = (SolveInfo * nb)()
    st = load().scalar_mg_solve_batched(ctx._h, nb, ns, dp, aB, aM, aa, tol, pp, infos)
    if st != PM_OK and (raise_on_noconv or st != PM_ERR_NOCONV):
        ctx._check(st)
    return phis, [i.as_dict() for i in infos]


def force_interp(psi_N, phi, alpha_B0, alpha_M0, a, pos, acc=None, ctx=None):
    ctx = ctx or default_context()
    n = psi_N.shape[0]
    if acc is None:
        acc = torch.empty_like(pos)
    ctx._check(load().force_interp(ctx._h, _ptr(psi_N, shape=(n, n, n)), _ptr(phi, shape=(n, n, n)), n, alpha_B0,
                                   alpha_M0, a, _ptr(pos, name="pos"), pos.shape[1], _ptr(acc, shape=pos.shape)))
    return acc


def lensing_potential(psi_N, chi, alpha_B0, alpha_M0, a, Phi=None, ctx=None):
    """Phi = Psi_N + alpha_B(a) chi on the device (see lensing_potential in pmeft.h)."""
    ctx = ctx or default_context()
    n = psi_N.shape[0]
    if Phi is None:
        Phi = torch.empty_like(psi_N)
    ctx._check(load().lensing_potential(ctx._h, _ptr(psi_N, shape=(n, n, n)), _ptr(chi, shape=(n, n, n)), n, alpha_B0,
                                        alpha_M0, a, _ptr(Phi, shape=(n, n, n))))
    return Phi


def pm_step(pos, vel, n, alpha_B0, alpha_M0, a, dt, tol, phi_state, ctx=None):
    """One PM step in place on pos/vel (3, np); phi_state (n,n,n) warm start in, chi out.  Returns info."""
    ctx = ctx or default_context()
    info = SolveInfo()
    ctx._check(load().pm_step(ctx._h, _ptr(pos, name="pos"), _ptr(vel, shape=pos.shape, name="vel"), pos.shape[1], n,
                              alpha_B0, alpha_M0, a, dt, tol, _ptr(phi_state, shape=(n, n, n)), ctypes.byref(info)))
    return info.as_dict()


def pm_run(pos, vel, n, alpha_B0, alpha_M0, a_start, a_end, nsteps, tol, phi_state, ctx=None):
    """nsteps PM steps in place on pos/vel (3, np) from a_start to a_end (see pm_run in pmeft.h);
    phi_state (n,n,n): warm start in, last chi out.  Returns the last step's info."""
    ctx = ctx or default_context()
    info = SolveInfo()
    ctx._check(load().pm_run(ctx._h, _ptr(pos, name="pos"), _ptr(vel, shape=pos.shape, name="vel"), pos.shape[1], n,
                             alpha_B0, alpha_M0, a_start, a_end, nsteps, tol, _ptr(phi_state, shape=(n, n, n)),
                             ctypes.byref(info)))
    return info.as_dict()


def pm_mg_sweep(u, f, lam, nu, kappa, eta, kmask=None, ctx=None):
    """One red-black sweep of u in place (periodic n^3)."""
    ctx = ctx or default_context()
    n = u.shape[0]
    ctx._check(load().pm_mg_sweep(ctx._h, _ptr(u, shape=(n, n, n)), _ptr(f, shape=(n, n, n)), lam, n, nu, kappa, eta,
                                  _ptr(kmask, torch.uint8, (n, n, n), "kmask")))
    return u


def pm_mg_coarse_exact(u, f, nu, kappa, eta, kmask=None, ctx=None):
    """The exact coarsest-level solve alone (n = 2 or 4): u solved in place; returns (u, lambda)."""
    ctx = ctx or default_context()
    n = u.shape[0]
    lam = ctypes.c_double(0.0)
    ctx._check(load().pm_mg_coarse_exact(ctx._h, _ptr(u, shape=(n, n, n)), _ptr(f, shape=(n, n, n)), n, nu, kappa,
                                         eta, _ptr(kmask, torch.uint8, (n, n, n), "kmask"), ctypes.byref(lam)))
    return u, lam.value


def pm_mg_sweep_f32(u, f, lam, nu, kappa, eta, kmask=None, mode=1, bg=None, gap=None, ctx=None):
    """One red-black sweep of an FP32 grid in place; mode 0: two half-sweep launches, k >= 1: the
    single-pass kernel with tile variant k-1, 100 + k the same through the background's BF16
    coefficients, 200 the zero-start kernel (u taken as zero).  bg / gap: the correction form
    (see pmeft.h)."""
    ctx = ctx or default_context()
    n = u.shape[0]
    ctx._check(load().pm_mg_sweep_f32(ctx._h, _ptr(u, torch.float32, (n, n, n)), _ptr(f, torch.float32, (n, n, n)),
                                      lam, n, nu, kappa, eta, _ptr(kmask, torch.uint8, (n, n, n), "kmask"),
                                      _ptr(bg, torch.float32, (n, n, n), "bg"), _ptr(gap, torch.float32, (n, n, n), "gap"),
                                      mode))
    return u


def pm_mg_residual(u, f, lam, nu, kappa, eta, kmask=None, ctx=None):
    ctx = ctx or default_context()
    n = u.shape[0]
    r = torch.empty_like(u)
    fl = torch.empty((n, n, n), dtype=torch.uint8, device=u.device)
    ctx._check(load().pm_mg_residual(ctx._h, _ptr(u, shape=(n, n, n)), _ptr(f, shape=(n, n, n)), lam, n, nu, kappa,
                                     eta, _ptr(kmask, torch.uint8, (n, n, n), "kmask"), _ptr(r), _ptr(fl, torch.uint8)))
    return r, fl


def pm_mg_restrict(fine, ctx=None):
    ctx = ctx or default_context()
    n = fine.shape[0]
    out = torch.empty((n // 2,) * 3, dtype=torch.float64, device=fine.device)
    ctx._check(load().pm_mg_restrict(ctx._h, _ptr(fine, shape=(n, n, n)), n, _ptr(out)))
    return out


def pm_mg_prolong_add(coarse, fine, ctx=None):
    ctx = ctx or default_context()
    n = fine.shape[0]
    ctx._check(load().pm_mg_prolong_add(ctx._h, _ptr(coarse, shape=(n // 2,) * 3), n, _ptr(fine, shape=(n, n, n))))
    return fine


def pm_deposit_cic_static(pos, n, delta=None, stream=None):
    """Allocation-free deposit (see pm_deposit_cic_static in pmeft.h): n <= 128, no context.

    Returns (delta, status) without raising, so callers can handle PM_ERR_TOO_LARGE."""
    if delta is None:
        delta = torch.empty((n, n, n), dtype=torch.float64, device=pos.device)
    if delta.device != pos.device:
        raise ValueError(f"delta is on {delta.device}, pos on {pos.device}: both must be on the same GPU")
    # the entry point works on the current device: make it the one holding the buffers
    with torch.cuda.device(pos.device):
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        st = load().pm_deposit_cic_static(_ptr(pos, name="pos"), pos.shape[1], n, _ptr(delta, shape=(n, n, n)),
                                          ctypes.c_void_p(s.cuda_stream))
    return delta, st


class UNet:
    """The warm-start network (pm_unet): FP32 master parameters on the device, BF16 kernels."""

    def __init__(self, ctx=None):
        self.ctx = ctx or default_context()
        h = ctypes.c_void_p()
        self.ctx._check(load().pm_unet_create(self.ctx._h, ctypes.byref(h)))
        self._h = h
        self.num_params = int(load().pm_unet_num_params())

    def set_conv_path(self, path: int):
        """0: mma.sync convolutions, 1 (default): tcgen05 tensor-core convolutions (see pm_unet_set_conv_path)."""
        self.ctx._check(load().pm_unet_set_conv_path(self._h, int(path)))

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {p.size}")
        self.ctx._check(load().pm_unet_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size))

    def get_params(self, grads=False):
        import numpy as np

        out = np.empty(self.num_params, dtype=np.float32)
        self.ctx._check(load().pm_unet_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p), out.size,
                                                  1 if grads else 0))
        return out

    def forward(self, delta, alpha_B0, alpha_M0, a):
        n = delta.shape[0]
        out = torch.empty_like(delta)
        self.ctx._check(load().pm_unet_forward(self._h, _ptr(delta, shape=(n, n, n)), n, alpha_B0, alpha_M0, a,
                                               _ptr(out)))
        return out

    def loss_grad(self, delta, target, alpha_B0, alpha_M0, a):
        n = delta.shape[0]
        loss = ctypes.c_double()
        self.ctx._check(load().pm_unet_loss_grad(self._h, _ptr(delta, shape=(n, n, n)),
                                                 _ptr(target, torch.float32, (n, n, n), "target"), n, alpha_B0,
                                                 alpha_M0, a, ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.ctx._check(load().pm_unet_adam_step(self._h, lr, beta1, beta2, eps))

    def zero_grad(self):
        self.ctx._check(load().pm_unet_zero_grad(self._h))

    def warm_start(self, delta, alpha_B0, alpha_M0, a, phi=None):
        n = delta.shape[0]
        if phi is None:
            phi = torch.empty_like(delta)
        self.ctx._check(load().pm_unet_warm_start(self._h, _ptr(delta, shape=(n, n, n)), n, alpha_B0, alpha_M0, a,
                                                  _ptr(phi, shape=(n, n, n))))
        return phi

    def close(self):
        if getattr(self, "_h", None):
            load().pm_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unet_target(chi, alpha_B0, alpha_M0, a, ctx=None):
    """Training target T = nu L(chi) / src of a solved chi (float32 n^3)."""
    ctx = ctx or default_context()
    n = chi.shape[0]
    out = torch.empty((n, n, n), dtype=torch.float32, device=chi.device)
    ctx._check(load().pm_unet_target(ctx._h, _ptr(chi, shape=(n, n, n)), n, alpha_B0, alpha_M0, a,
                                     _ptr(out, torch.float32)))
    return out


def linear_start(delta, alpha_B0, alpha_M0, a, phi=None, ctx=None):
    """The linearised solution the paper's PySCo-EFT starts from (Sec. 3.5.1)."""
    ctx = ctx or default_context()
    n = delta.shape[0]
    if phi is None:
        phi = torch.empty_like(delta)
    ctx._check(load().pm_linear_start(ctx._h, _ptr(delta, shape=(n, n, n)), n, alpha_B0, alpha_M0, a,
                                      _ptr(phi, shape=(n, n, n))))
    return phi
