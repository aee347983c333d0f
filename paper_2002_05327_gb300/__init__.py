"""Python binding of libhelm (include/helm.h): argument marshalling only.

Every step of the diagonal sweeping DDM runs in the CUDA library; this module
loads ``libhelm.so`` with ctypes and exposes the C entry points under the same
names.  Host data are numpy arrays (complex128 ``[nrhs, *grid]``, float64
grids); device data are CUDA torch tensors of the same dtypes and shapes.
There is no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhelm.so")

HELM_OK = 0
HELM_ERR_ARG = -1
HELM_ERR_OOM = -2
HELM_ERR_NOT_FACTORED = -3
HELM_ERR_NO_CONVERGENCE = -4
HELM_ERR_TIMEOUT = -5
HELM_ERR_CUDA = -6
HELM_ERR_NUMERIC = -7
HELM_PREC_F64 = 0
HELM_PREC_MIXED = 1
HELM_PREC_TF32 = 2
HELM_PREC_F16 = 3
HELM_PML_LITERAL = 0
HELM_PML_OMEGA = 1
HELM_MEM_HOST = 0
HELM_MEM_DEVICE = 1


class helm_pml(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("power", ctypes.c_int32),
                ("sigma0", ctypes.c_double), ("form", ctypes.c_int32)]


class helm_partition(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int32 * 3), ("cuts", ctypes.POINTER(ctypes.c_int64) * 3),
                ("overlap", ctypes.c_int32), ("sub_pml", ctypes.c_int32)]


class helm_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rhs_panel", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("verbose", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("tc_kernel", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("sweep_order", ctypes.c_int32), ("max_device_bytes", ctypes.c_int64),
                ("algorithm", ctypes.c_int32)]


KERNEL_CLASSES = ("factor", "solve", "gather", "assemble", "krylov")


class helm_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8),
                ("bytes", ctypes.c_double * 8), ("flops", ctypes.c_double * 8)]

    def as_dict(self):
        return {name: {"launches": int(self.launches[i]), "ms": float(self.ms[i]),
                       "bytes": float(self.bytes[i]), "flops": float(self.flops[i])}
                for i, name in enumerate(KERNEL_CLASSES)}


class helm_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("applications", ctypes.c_int32),
                ("resid", ctypes.c_double), ("t_factor_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("levels", ctypes.c_int32),
                ("solves", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_SIGS = {
    "helm_setup": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.c_double, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.POINTER(helm_pml),
                                  ctypes.POINTER(helm_partition), ctypes.POINTER(helm_config)]),
    "helm_factor": (ctypes.c_int, [ctypes.c_void_p]),
    "helm_apply_ddm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int]),
    "helm_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(helm_stats)]),
    "helm_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(helm_stats)]),
    "helm_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(helm_stats)]),
    "helm_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "helm_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "helm_subdomain_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "helm_subdomain_solve_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_void_p]),
    "helm_window_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "helm_problem_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64)]),
    "helm_device_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "helm_release": (ctypes.c_int, [ctypes.c_void_p]),
    "helm_profile_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "helm_profile_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(helm_profile)]),
    "helm_destroy": (None, [ctypes.c_void_p]),
    "helm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "helm_last_error": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libhelm.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhelm.so not built at {LIB_PATH}: run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HelmError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        msg = L.helm_last_error().decode()
        super().__init__(f"{where}: {L.helm_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def _check(code, where):
    if code != HELM_OK:
        raise HelmError(code, where)


# ----------------------------------------------------------------------------- data marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_mem(x, dtype):
    """(pointer, mem flag, keepalive) for a numpy array or CUDA torch tensor."""
    if _is_torch(x):
        import torch
        want = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        if not x.is_cuda or x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous CUDA tensor of {want}")
        torch.cuda.current_stream(x.device).synchronize()
        return ctypes.c_void_p(x.data_ptr()), HELM_MEM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), HELM_MEM_HOST, a


def _empty_like(x, shape, dtype):
    if _is_torch(x):
        import torch
        want = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=want, device=x.device)
    return np.empty(shape, dtype=dtype)


@dataclass
class Context:
    """Owns a helm_ctx; destroyed with the object."""
    ptr: ctypes.c_void_p
    ndim: int
    N: tuple
    nsub: int

    @property
    def grid_shape(self):
        return tuple(reversed(self.N))

    def close(self):
        if self.ptr:
            lib().helm_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- entry points
def helm_setup(ndim, n, h, omega, m, pml_width, sigma0, nb, overlap, power=2,
               form=HELM_PML_LITERAL, cuts=None, sub_pml=0, precision=HELM_PREC_MIXED,
               rhs_panel=0, restart=30, verbose=0, stream=None, profile=0,
               tc_kernel=0, wait_limit=0, sweep_order=0, max_device_bytes=0, algorithm=0) -> Context:
    L = lib()
    nn = (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    m = np.ascontiguousarray(m, dtype=np.float64)
    pml = helm_pml(int(pml_width), int(power), float(sigma0), int(form))
    part = helm_partition()
    keep = []
    for a in range(3):
        part.nb[a] = int(nb[a]) if a < len(nb) else 1
        if cuts is not None and a < len(cuts) and cuts[a] is not None:
            arr = np.ascontiguousarray(cuts[a], dtype=np.int64)
            keep.append(arr)
            part.cuts[a] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        else:
            part.cuts[a] = ctypes.POINTER(ctypes.c_int64)()
    part.overlap = int(overlap)
    part.sub_pml = int(sub_pml)
    cfg = helm_config(int(precision), int(rhs_panel), int(restart), int(verbose),
                      ctypes.c_void_p(stream) if stream else None, int(profile), int(tc_kernel),
                      int(wait_limit), int(sweep_order), int(max_device_bytes), int(algorithm))
    out = ctypes.c_void_p()
    _check(L.helm_setup(ctypes.byref(out), int(ndim), nn, float(h), float(omega),
                        m.ctypes.data_as(ctypes.c_void_p), ctypes.byref(pml), ctypes.byref(part),
                        ctypes.byref(cfg)), "helm_setup")
    nsub = ctypes.c_int64()
    N = (ctypes.c_int64 * 3)()
    _check(L.helm_problem_info(out, ctypes.byref(nsub), N), "helm_problem_info")
    return Context(out, int(ndim), tuple(int(N[a]) for a in range(ndim)), int(nsub.value))


def helm_setup_workload(wl, **cfg) -> Context:
    """helm_setup from any object with the attributes of a workload description
    (ndim, n, h, omega, pml, sigma0, power, nb, cuts, overlap, sub_pml, m)."""
    return helm_setup(wl.ndim, wl.n, wl.h, wl.omega, wl.m, wl.pml, wl.sigma0, wl.nb,
                      wl.overlap, power=wl.power, cuts=wl.cuts, sub_pml=wl.sub_pml, **cfg)


def helm_factor(ctx: Context):
    _check(lib().helm_factor(ctx.ptr), "helm_factor")


def _nrhs(F, ctx):
    shp = tuple(F.shape)
    if shp[1:] != ctx.grid_shape:
        raise ValueError(f"expected [nrhs, {ctx.grid_shape}], got {shp}")
    return shp[0]


def helm_apply_ddm(ctx: Context, F):
    nr = _nrhs(F, ctx)
    fp, mem, kf = _ptr_mem(F, np.complex128)
    U = _empty_like(F, tuple(F.shape), np.complex128)
    up, mem2, ku = _ptr_mem(U, np.complex128)
    _check(lib().helm_apply_ddm(ctx.ptr, nr, fp, up, mem), "helm_apply_ddm")
    return U


def helm_solve(ctx: Context, F, rtol=1e-8, maxit=100, allow_noconv=False):
    nr = _nrhs(F, ctx)
    fp, mem, kf = _ptr_mem(F, np.complex128)
    U = _empty_like(F, tuple(F.shape), np.complex128)
    up, _, ku = _ptr_mem(U, np.complex128)
    st = helm_stats()
    rc = lib().helm_solve(ctx.ptr, nr, fp, up, mem, float(rtol), int(maxit), ctypes.byref(st))
    if not (allow_noconv and rc == HELM_ERR_NO_CONVERGENCE):
        _check(rc, "helm_solve")
    return U, st.as_dict()


def helm_iterate(ctx: Context, F, rtol=1e-8, maxit=100, allow_noconv=False):
    """The DDM as a stationary iteration (helm_iterate): returns U and the stats."""
    nr = _nrhs(F, ctx)
    fp, mem, kf = _ptr_mem(F, np.complex128)
    U = _empty_like(F, tuple(F.shape), np.complex128)
    up, _, ku = _ptr_mem(U, np.complex128)
    st = helm_stats()
    rc = lib().helm_iterate(ctx.ptr, nr, fp, up, mem, float(rtol), int(maxit), ctypes.byref(st))
    if not (allow_noconv and rc == HELM_ERR_NO_CONVERGENCE):
        _check(rc, "helm_iterate")
    return U, st.as_dict()


def helm_adjoint(ctx: Context, G, rtol=1e-8, maxit=100):
    nr = _nrhs(G, ctx)
    gp, mem, kg = _ptr_mem(G, np.complex128)
    Lm = _empty_like(G, tuple(G.shape), np.complex128)
    lp, _, kl = _ptr_mem(Lm, np.complex128)
    st = helm_stats()
    _check(lib().helm_adjoint(ctx.ptr, nr, gp, lp, mem, float(rtol), int(maxit),
                              ctypes.byref(st)), "helm_adjoint")
    return Lm, st.as_dict()


def helm_gradient(ctx: Context, U, Lam):
    nr = _nrhs(U, ctx)
    up, mem, ku = _ptr_mem(U, np.complex128)
    lp, _, kl = _ptr_mem(Lam, np.complex128)
    g = _empty_like(U, ctx.grid_shape, np.float64)
    gp, _, kg = _ptr_mem(g, np.float64)
    _check(lib().helm_gradient(ctx.ptr, nr, up, lp, gp, mem), "helm_gradient")
    return g


def helm_residual(ctx: Context, F, U):
    nr = _nrhs(F, ctx)
    fp, mem, kf = _ptr_mem(F, np.complex128)
    up, _, ku = _ptr_mem(U, np.complex128)
    R = _empty_like(F, tuple(F.shape), np.complex128)
    rp, _, kr = _ptr_mem(R, np.complex128)
    _check(lib().helm_residual(ctx.ptr, nr, fp, up, rp, mem), "helm_residual")
    return R


def helm_window_info(ctx: Context, s):
    lo = (ctypes.c_int64 * 3)()
    hi = (ctypes.c_int64 * 3)()
    _check(lib().helm_window_info(ctx.ptr, int(s), lo, hi), "helm_window_info")
    return [int(lo[a]) for a in range(ctx.ndim)], [int(hi[a]) for a in range(ctx.ndim)]


def helm_subdomain_solve(ctx: Context, s, R):
    lo, hi = helm_window_info(ctx, s)
    shape = tuple(reversed([h - l for l, h in zip(lo, hi)]))
    if tuple(R.shape[1:]) != shape:
        raise ValueError(f"expected [nrhs, {shape}]")
    rp, mem, kr = _ptr_mem(R, np.complex128)
    U = _empty_like(R, tuple(R.shape), np.complex128)
    up, _, ku = _ptr_mem(U, np.complex128)
    _check(lib().helm_subdomain_solve(ctx.ptr, int(s), R.shape[0], rp, up, mem),
           "helm_subdomain_solve")
    return U


def helm_subdomain_solve_noalloc(ctx: Context, s, R):
    """Subdomain solve that allocates no device memory (see include/helm.h):
    R is a CUDA complex128 tensor [nrhs, *window]; returns U of the same shape
    (the output tensor is allocated here, by torch, before the call)."""
    if not _is_torch(R):
        raise TypeError("helm_subdomain_solve_noalloc takes CUDA tensors")
    lo, hi = helm_window_info(ctx, s)
    shape = tuple(reversed([h - l for l, h in zip(lo, hi)]))
    if tuple(R.shape[1:]) != shape:
        raise ValueError(f"expected [nrhs, {shape}], got {tuple(R.shape)}")
    rp, _, kr = _ptr_mem(R, np.complex128)
    U = _empty_like(R, tuple(R.shape), np.complex128)
    up, _, ku = _ptr_mem(U, np.complex128)
    _check(lib().helm_subdomain_solve_noalloc(ctx.ptr, int(s), R.shape[0], rp, up),
           "helm_subdomain_solve_noalloc")
    return U


def helm_device_bytes(ctx: Context) -> int:
    return int(lib().helm_device_bytes(ctx.ptr))


def helm_release(ctx: Context) -> None:
    _check(lib().helm_release(ctx.ptr), "helm_release")


def helm_profile_reset(ctx: Context):
    _check(lib().helm_profile_reset(ctx.ptr), "helm_profile_reset")


def helm_profile_get(ctx: Context) -> dict:
    out = helm_profile()
    _check(lib().helm_profile_get(ctx.ptr, ctypes.byref(out)), "helm_profile_get")
    return out.as_dict()


# ----------------------------------------------------------------------------- autograd
def _make_helm_solve():
    import torch

    class HelmSolve(torch.autograd.Function):
        """U = A(m)^{-1} J F for a squared slowness m on the full grid, with the
        gradient of any real loss of U with respect to m (Remark 2: the
        adjoint-state gradient that full waveform inversion uses).

        forward(m, F, spec, rtol, maxit, keep_bytes): m is a float64 tensor of
        the full grid (copied to the host for helm_setup); F a CUDA complex128
        tensor [nrhs, *grid]; spec the keyword arguments of helm_setup other
        than m (ndim, n, h, omega, pml_width, sigma0, nb, overlap, ...).  It
        sets up and factors a context for this m, solves with helm_solve and
        keeps the context for the backward pass.  When keep_bytes is given and
        the context holds more device memory than that after the solve, its
        factors and work buffers are released (helm_release) and backward
        recomputes them (helm_factor): the same factors, so the same gradient,
        for one more factorization instead of the memory between the passes.

        backward(gU), with gU = dL/dRe U + i dL/dIm U (torch's convention for
        complex tensors): lam = A^{-H} gU by helm_adjoint on the same factors,
        then dL/dm = -omega^2 sum_s Re(conj(lam_s) J u_s) by helm_gradient.
        F is not differentiated (its gradient is None)."""

        @staticmethod
        def forward(actx, m, F, spec, rtol=1e-8, maxit=100, keep_bytes=None):
            mh = m.detach().to("cpu", torch.float64).numpy()
            helm = helm_setup(m=mh, **spec)
            helm_factor(helm)
            U, _ = helm_solve(helm, F.detach().contiguous(), rtol, maxit)
            actx.released = keep_bytes is not None and helm_device_bytes(helm) > keep_bytes
            if actx.released:
                helm_release(helm)
            actx.helm, actx.rtol, actx.maxit = helm, rtol, maxit
            actx.m_meta = (m.device, m.dtype)
            actx.save_for_backward(U)
            return U

        @staticmethod
        def backward(actx, gU):
            (U,) = actx.saved_tensors
            if actx.released:
                helm_factor(actx.helm)
            lam, _ = helm_adjoint(actx.helm, gU.contiguous(), actx.rtol, actx.maxit)
            g = helm_gradient(actx.helm, U, lam)
            dev, dt = actx.m_meta
            return g.to(dev, dt), None, None, None, None, None

    return HelmSolve


_helm_solve_cls = None


def __getattr__(name):
    """``HelmSolve`` (a torch.autograd.Function) is built on first access so that
    importing this module does not import torch:
    ``U = paper_2002_05327_gb300.HelmSolve.apply(m, F, spec, rtol, maxit)``."""
    global _helm_solve_cls
    if name == "HelmSolve":
        if _helm_solve_cls is None:
            _helm_solve_cls = _make_helm_solve()
        return _helm_solve_cls
    raise AttributeError(name)


__all__ = [n for n in dir() if n.startswith("helm_") or n.startswith("HELM_")] + [
    "Context", "HelmError", "HelmSolve", "lib", "LIB_PATH"]
