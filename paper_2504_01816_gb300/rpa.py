"""ctypes binding of librpa (include/rpa.h).

Argument marshalling only: every computation runs in the CUDA library.  Tensors are torch
tensors on the current CUDA device; torch is used for device memory and streams.  The
module raises at import time if librpa.so is missing (build it with
``python paper_2504_01816_gb300/_build.py`` or ``__graft_entry__.build()``): there is no
fallback path.

Layouts follow the C interface.  A block of K grid functions (the N_d x K column-major
matrix of the C interface) is a contiguous float64 tensor of shape (K, N_d).  Complex
solutions are complex128 tensors of shape (K, N_d).
"""
from __future__ import annotations

import ctypes
import os
import dataclasses
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpa.so")

RPA_OK, RPA_ERR_INVALID, RPA_ERR_CUDA, RPA_ERR_OOM = 0, 1, 2, 3
RPA_ERR_NOT_CONVERGED, RPA_ERR_BREAKDOWN, RPA_ERR_NOT_SPD = 4, 5, 6
RPA_FP64, RPA_MIXED = 0, 1

STATUS_NAMES = {0: "RPA_OK", 1: "RPA_ERR_INVALID", 2: "RPA_ERR_CUDA", 3: "RPA_ERR_OOM",
                4: "RPA_ERR_NOT_CONVERGED", 5: "RPA_ERR_BREAKDOWN", 6: "RPA_ERR_NOT_SPD"}

EXPORTED = ("rpa_default_options", "rpa_setup", "rpa_set_options", "rpa_coulomb_apply", "rpa_coulomb_apply_noalloc",
            "rpa_sternheimer_solve", "rpa_apply_nuchi0", "rpa_ec", "rpa_ec_gradient", "rpa_autotune", "rpa_destroy",
            "rpa_last_error", "rpa_version", "rpa_apply_nuchi0_batch", "rpa_ec_batch")


class rpa_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("inner_tol", ctypes.c_double), ("eps_c", ctypes.c_double),
                ("n_omega", ctypes.c_int), ("omega0", ctypes.c_double), ("max_subspace_iters", ctypes.c_int),
                ("fixed_subspace_iters", ctypes.c_int), ("n_atoms", ctypes.c_int),
                ("batch_systems", ctypes.c_int), ("profile", ctypes.c_int), ("project_solution", ctypes.c_int),
                ("z_chunks", ctypes.c_int), ("stencil_shape", ctypes.c_int),
                ("independent_frequencies", ctypes.c_int), ("sq_order", ctypes.c_int),
                ("contractions", ctypes.c_int), ("omega_first", ctypes.c_int), ("omega_count", ctypes.c_int),
                ("periodic", ctypes.c_int), ("precondition", ctypes.c_int),
                ("block_cocg", ctypes.c_int)]


PROF_SLOTS = 8


class rpa_stats(ctypes.Structure):
    _fields_ = [("sternheimer_solves", ctypes.c_longlong), ("cocg_iterations", ctypes.c_longlong),
                ("refinement_steps", ctypes.c_longlong), ("stencil_points", ctypes.c_longlong),
                ("subspace_iterations", ctypes.c_int * 64), ("omegas", ctypes.c_double * 64),
                ("weights", ctypes.c_double * 64), ("ms_coulomb", ctypes.c_double),
                ("ms_projection", ctypes.c_double), ("ms_cocg", ctypes.c_double), ("ms_density", ctypes.c_double),
                ("ms_subspace", ctypes.c_double), ("ms_total", ctypes.c_double), ("worst_status", ctypes.c_int),
                ("prof_count", ctypes.c_int), ("prof_name", (ctypes.c_char * 32) * PROF_SLOTS),
                ("prof_launches", ctypes.c_longlong * PROF_SLOTS), ("prof_ms", ctypes.c_double * PROF_SLOTS),
                ("prof_points", ctypes.c_double * PROF_SLOTS), ("prof_bytes", ctypes.c_double * PROF_SLOTS),
                ("launches", ctypes.c_longlong), ("near_breakdowns", ctypes.c_longlong),
                ("host_syncs", ctypes.c_longlong)]


def stats_dict(stats: "rpa_stats", n_omega: int) -> dict:
    sd = {f[0]: getattr(stats, f[0]) for f in rpa_stats._fields_ if not f[0].startswith("prof_")}
    sd["subspace_iterations"] = list(stats.subspace_iterations)[:n_omega]
    sd["omegas"] = list(stats.omegas)[:n_omega]
    sd["weights"] = list(stats.weights)[:n_omega]
    sd["kernels"] = [{"name": stats.prof_name[i].value.decode(), "launches": stats.prof_launches[i],
                      "ms": stats.prof_ms[i], "points": stats.prof_points[i], "bytes": stats.prof_bytes[i]}
                     for i in range(stats.prof_count)]
    return sd


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librpa.so not found at {LIB_PATH}; build it with "
                          "`python paper_2504_01816_gb300/_build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, i, d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.rpa_default_options.argtypes = [ctypes.POINTER(rpa_options)]
    lib.rpa_default_options.restype = None
    lib.rpa_setup.argtypes = [ctypes.POINTER(vp), i, i, i, d, i, dp, dp, ctypes.POINTER(ctypes.c_double), i,
                              ctypes.POINTER(rpa_options), vp]
    lib.rpa_setup.restype = i
    lib.rpa_set_options.argtypes = [vp, ctypes.POINTER(rpa_options)]
    lib.rpa_set_options.restype = i
    lib.rpa_coulomb_apply.argtypes = [vp, d, dp, dp, i, vp]
    lib.rpa_coulomb_apply.restype = i
    lib.rpa_coulomb_apply_noalloc.argtypes = [vp, d, dp, dp, i, vp]
    lib.rpa_coulomb_apply_noalloc.restype = i
    lib.rpa_sternheimer_solve.argtypes = [vp, d, ctypes.POINTER(ctypes.c_int), i, dp, i, dp, ip, ip, vp]
    lib.rpa_sternheimer_solve.restype = i
    lib.rpa_apply_nuchi0.argtypes = [vp, d, dp, dp, i, i, vp]
    lib.rpa_apply_nuchi0.restype = i
    lib.rpa_ec.argtypes = [vp, i, dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(rpa_stats), vp]
    lib.rpa_ec.restype = i
    lib.rpa_ec_gradient.argtypes = [vp, i, dp, dp, dp, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(rpa_stats), vp]
    lib.rpa_ec_gradient.restype = i
    lib.rpa_apply_nuchi0_batch.argtypes = [ctypes.POINTER(vp), i, d, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(ctypes.c_int), i, vp]
    lib.rpa_apply_nuchi0_batch.restype = i
    lib.rpa_ec_batch.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp),
                                 ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp),
                                 ctypes.POINTER(rpa_stats), vp]
    lib.rpa_ec_batch.restype = i
    lib.rpa_autotune.argtypes = [vp, d, dp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp]
    lib.rpa_autotune.restype = i
    lib.rpa_destroy.argtypes = [vp]
    lib.rpa_destroy.restype = None
    lib.rpa_last_error.restype = ctypes.c_char_p
    lib.rpa_version.restype = ctypes.c_char_p
    return lib


_lib = _load()


def library():
    return _lib


class RpaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def last_error() -> str:
    return _lib.rpa_last_error().decode()


def _check(st: int, allow=(RPA_OK,)):
    if st not in allow:
        raise RpaError(st, last_error())
    return st


def _ptr(t) -> int:
    return t.data_ptr() if t is not None else None


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev64(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


@dataclass
class Options:
    prec: int = RPA_FP64
    tol: float = 1e-8
    maxit: int = 20000
    max_refine: int = 20
    inner_tol: float = 1e-4
    eps_c: float = 1e-5
    n_omega: int = 8
    omega0: float = 1.0
    max_subspace_iters: int = 100
    fixed_subspace_iters: int = 0
    n_atoms: int = 1
    batch_systems: int = 0
    profile: int = 0
    project_solution: int = 0
    z_chunks: int = 0
    stencil_shape: int = 0
    independent_frequencies: int = 0
    sq_order: int = 0
    contractions: int = 0
    omega_first: int = 0
    omega_count: int = 0
    periodic: int = 0
    precondition: int = 0
    block_cocg: int = 0

    def to_c(self) -> rpa_options:
        o = rpa_options()
        for f in rpa_options._fields_:
            setattr(o, f[0], getattr(self, f[0]))
        return o


def default_options() -> Options:
    o = rpa_options()
    _lib.rpa_default_options(ctypes.byref(o))
    return Options(**{f[0]: getattr(o, f[0]) for f in rpa_options._fields_})


@dataclass
class EcResult:
    e_c: float
    e_c_per_atom: float
    e_c_per_omega: np.ndarray
    lambdas: np.ndarray
    status: int
    stats: dict = field(default_factory=dict)


class Context:
    """One model system on the GPU (rpa_setup ... rpa_destroy)."""

    def __init__(self, nx: int, ny: int, nz: int, h: float, vloc, psi, eps: Sequence[float],
                 options: Optional[Options] = None, stream=None):
        n_d = nx * ny * nz
        eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        n_s = eps.shape[0]
        _dev64(vloc, (n_d,))
        _dev64(psi, (n_s, n_d))
        self.nx, self.ny, self.nz, self.h, self.n_d, self.n_s = nx, ny, nz, h, n_d, n_s
        self.options = options or default_options()
        handle = ctypes.c_void_p()
        opt = self.options.to_c()
        _check(_lib.rpa_setup(ctypes.byref(handle), nx, ny, nz, float(h), 12, _ptr(vloc), _ptr(psi),
                              eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_s, ctypes.byref(opt),
                              _stream(stream)))
        self._h = handle

    @classmethod
    def from_system(cls, system, options: Optional[Options] = None, device="cuda"):
        import torch
        vloc = torch.as_tensor(system.vloc, dtype=torch.float64, device=device).contiguous()
        psi = torch.as_tensor(system.psi, dtype=torch.float64, device=device).contiguous()
        if getattr(system, "periodic", False):      # the system's boundary conditions
            options = dataclasses.replace(options if options is not None else default_options(), periodic=1)
        return cls(system.nx, system.ny, system.nz, system.h, vloc, psi, system.eps, options)

    def close(self):
        if getattr(self, "_h", None):
            _lib.rpa_destroy(self._h)
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

    def set_options(self, options: Options):
        opt = options.to_c()
        _check(_lib.rpa_set_options(self._h, ctypes.byref(opt)))
        self.options = options

    def coulomb_apply(self, power: float, X, out=None, stream=None):
        import torch
        k = X.shape[0]
        _dev64(X, (k, self.n_d))
        out = torch.empty_like(X) if out is None else _dev64(out, (k, self.n_d))
        _check(_lib.rpa_coulomb_apply(self._h, float(power), _ptr(X), _ptr(out), k, _stream(stream)))
        return out

    def sternheimer_solve(self, omega: float, orbitals: Sequence[int], rhs, project: bool = True, stream=None):
        import torch
        orb = np.ascontiguousarray(np.asarray(orbitals, dtype=np.int32))
        k = orb.shape[0]
        _dev64(rhs, (k, self.n_d))
        x = torch.empty((k, self.n_d), dtype=torch.complex128, device=rhs.device)
        iters = torch.zeros(k, dtype=torch.int32, device=rhs.device)
        status = torch.zeros(k, dtype=torch.int32, device=rhs.device)
        st = _lib.rpa_sternheimer_solve(self._h, float(omega), orb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), k,
                                        _ptr(rhs), int(bool(project)), x.data_ptr(), iters.data_ptr(),
                                        status.data_ptr(), _stream(stream))
        _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED, RPA_ERR_BREAKDOWN))
        return x, iters, status, st

    def apply_nuchi0(self, omega: float, V, symmetric: bool = True, out=None, stream=None):
        import torch
        k = V.shape[0]
        _dev64(V, (k, self.n_d))
        R = torch.empty_like(V) if out is None else _dev64(out, (k, self.n_d))
        st = _lib.rpa_apply_nuchi0(self._h, float(omega), _ptr(V), _ptr(R), k, int(bool(symmetric)), _stream(stream))
        _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED))
        return R, st

    def ec(self, V0, stream=None) -> EcResult:
        n_r = V0.shape[0]
        _dev64(V0, (n_r, self.n_d))
        nw = self.options.n_omega
        lam = np.zeros((nw, n_r))
        ec = np.zeros(2)
        ecm = np.zeros(nw)
        stats = rpa_stats()
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        st = _lib.rpa_ec(self._h, n_r, _ptr(V0), dptr(lam), dptr(ec), dptr(ecm), ctypes.byref(stats),
                         _stream(stream))
        _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED))
        return EcResult(float(ec[0]), float(ec[1]), ecm, lam, st, stats_dict(stats, nw))

    AUTOTUNE_CANDIDATES = [f"split kernels, {shape}, {z} z chunk(s)"
                           for shape in ("1 column/thread <= 640 threads", "1 column/thread <= 320 threads x 2 blocks",
                                         "2 columns/thread <= 384 threads") for z in (1, 2)] + \
                          ["fused single-pass kernel, whole planes in a shared-memory ring",
                           "fused single-pass kernel, warp-specialised (producer / consumer threads)",
                           "fused single-pass kernel, cluster form (bands of the plane, two blocks per SM)"]

    def autotune(self, omega: float, V, stream=None):
        """rpa_autotune: time the COCG kernel configurations on this workload, keep the fastest.
        Returns (chosen index, candidate descriptions, times in ms; -1 = not applicable)."""
        n_r = V.shape[0]
        _dev64(V, (n_r, self.n_d))
        chosen = ctypes.c_int(0)
        times = (ctypes.c_double * len(self.AUTOTUNE_CANDIDATES))()
        _check(_lib.rpa_autotune(self._h, float(omega), _ptr(V), n_r, ctypes.byref(chosen), times, _stream(stream)))
        # the autotuner sets stencil_shape and z_chunks; keep the Python-side options in step
        i = chosen.value
        self.options.stencil_shape = i - 2 if i >= 6 else i // 2 + 1
        self.options.z_chunks = 1 if i >= 6 else i % 2 + 1
        return i, self.AUTOTUNE_CANDIDATES, list(times)

    def ec_gradient(self, V0, want_subspace: bool = False, stream=None):
        """E_c and dE_c/dV_loc (N_d, float64 CUDA tensor) at fixed orbitals (rpa_ec_gradient);
        with want_subspace also the final subspace (n_r x N_d)."""
        import torch
        n_r = V0.shape[0]
        _dev64(V0, (n_r, self.n_d))
        nw = self.options.n_omega
        lam = np.zeros((nw, n_r))
        ec = np.zeros(2)
        ecm = np.zeros(nw)
        stats = rpa_stats()
        grad = torch.empty(self.n_d, dtype=torch.float64, device=V0.device)
        vout = torch.empty_like(V0) if want_subspace else None
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        st = _lib.rpa_ec_gradient(self._h, n_r, _ptr(V0), grad.data_ptr(), _ptr(vout), dptr(lam), dptr(ec),
                                  dptr(ecm), ctypes.byref(stats), _stream(stream))
        _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED))
        res = EcResult(float(ec[0]), float(ec[1]), ecm, lam, st, stats_dict(stats, nw))
        return (res, grad, vout) if want_subspace else (res, grad)


# ----------------------------------------------------------------------------------------
# The C entry points under their own names (raw marshalling, returning the status code).
# ----------------------------------------------------------------------------------------
def rpa_default_options() -> Options:
    return default_options()


def rpa_setup(nx, ny, nz, h, vloc, psi, eps, options: Optional[Options] = None, stream=None) -> Context:
    return Context(nx, ny, nz, h, vloc, psi, eps, options, stream)


def rpa_set_options(ctx: Context, options: Options):
    ctx.set_options(options)


def rpa_coulomb_apply(ctx: Context, power, X, out=None, stream=None):
    return ctx.coulomb_apply(power, X, out, stream)


def rpa_coulomb_apply_noalloc(ctx: Context, power, X, out=None, stream=None):
    """Same result as rpa_coulomb_apply, with the scratch in the library's fixed device array
    (the call itself allocates no device memory; ``out`` must then be given by the caller)."""
    import torch
    k = X.shape[0]
    _dev64(X, (k, ctx.n_d))
    out = torch.empty_like(X) if out is None else _dev64(out, (k, ctx.n_d))
    _check(_lib.rpa_coulomb_apply_noalloc(ctx._h, float(power), _ptr(X), _ptr(out), k, _stream(stream)))
    return out


def rpa_sternheimer_solve(ctx: Context, omega, orbitals, rhs, project=True, stream=None):
    return ctx.sternheimer_solve(omega, orbitals, rhs, project, stream)


def rpa_apply_nuchi0(ctx: Context, omega, V, symmetric=True, out=None, stream=None):
    return ctx.apply_nuchi0(omega, V, symmetric, out, stream)


def rpa_ec(ctx: Context, V0, stream=None) -> EcResult:
    return ctx.ec(V0, stream)


def rpa_ec_gradient(ctx: Context, V0, stream=None):
    return ctx.ec_gradient(V0, stream=stream)


def _autograd_function():
    import torch

    class EcFunction(torch.autograd.Function):
        """E_c as a differentiable function of V_loc at fixed occupied orbitals and eigenvalues.

        forward(vloc, psi, eps, V0, nx, ny, nz, h, options) -> E_c (Ha, 0-d tensor); backward gives
        dE_c/dV_loc from rpa_ec_gradient (the hand-written adjoint; no graph is recorded through
        the library)."""

        @staticmethod
        def forward(ctx, vloc, psi, eps, V0, nx, ny, nz, h, options):
            with Context(nx, ny, nz, h, vloc.detach().contiguous(), psi.detach().contiguous(),
                         np.asarray(eps, dtype=np.float64), options) as c:
                res, grad = c.ec_gradient(V0.detach().contiguous())
            ctx.save_for_backward(grad)
            return torch.tensor(res.e_c, dtype=torch.float64, device=vloc.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad, None, None, None, None, None, None, None, None

    return EcFunction


def apply_nuchi0_batch(contexts: Sequence[Context], omega: float, Vs, symmetric: bool = True, stream=None):
    """rpa_apply_nuchi0_batch: nu^1/2 chi0 nu^1/2 V (or nu chi0 V) for every context with its own
    block of columns Vs[k] ((n_k, N_d_k) float64 CUDA tensors), all Sternheimer systems in one set
    of launches.  Returns ([R_k], status)."""
    import torch
    n = len(contexts)
    for c, V in zip(contexts, Vs):
        _dev64(V, (V.shape[0], c.n_d))
    Rs = [torch.empty_like(V) for V in Vs]
    hs = (ctypes.c_void_p * n)(*[c._h for c in contexts])
    vp = (ctypes.c_void_p * n)(*[V.data_ptr() for V in Vs])
    rp = (ctypes.c_void_p * n)(*[R.data_ptr() for R in Rs])
    nc = (ctypes.c_int * n)(*[V.shape[0] for V in Vs])
    st = _lib.rpa_apply_nuchi0_batch(hs, n, float(omega), vp, rp, nc, int(bool(symmetric)), _stream(stream))
    _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED))
    return Rs, st


def ec_batch(contexts: Sequence[Context], V0s, stream=None):
    """rpa_ec_batch: E_c of every context from its own trial vectors V0s[k] ((n_r_k, N_d_k) float64
    CUDA tensors), the contexts' chi0 applications batched into one set of launches.  Returns a
    list of EcResult and the call's status."""
    n = len(contexts)
    for c, V in zip(contexts, V0s):
        _dev64(V, (V.shape[0], c.n_d))
    lams = [np.zeros((c.options.n_omega, V.shape[0])) for c, V in zip(contexts, V0s)]
    ecms = [np.zeros(c.options.n_omega) for c in contexts]
    ec = np.zeros(2 * n)
    stats = (rpa_stats * n)()
    hs = (ctypes.c_void_p * n)(*[c._h for c in contexts])
    vp = (ctypes.c_void_p * n)(*[V.data_ptr() for V in V0s])
    lp = (ctypes.c_void_p * n)(*[lam.ctypes.data for lam in lams])
    ep = (ctypes.c_void_p * n)(*[e.ctypes.data for e in ecms])
    nr = (ctypes.c_int * n)(*[V.shape[0] for V in V0s])
    st = _lib.rpa_ec_batch(hs, n, nr, vp, lp, ec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ep, stats,
                           _stream(stream))
    _check(st, allow=(RPA_OK, RPA_ERR_NOT_CONVERGED))
    out = []
    for k, c in enumerate(contexts):
        nw = c.options.n_omega
        sd = stats_dict(stats[k], nw)
        out.append(EcResult(float(ec[2 * k]), float(ec[2 * k + 1]), ecms[k], lams[k], st, sd))
    return out, st


def ec_autograd(vloc, psi, eps, V0, nx, ny, nz, h, options: Optional[Options] = None):
    """Differentiable E_c(V_loc): torch.autograd sees dE_c/dV_loc from the library's adjoint."""
    opts = options or default_options()
    return _autograd_function().apply(vloc, psi, eps, V0, nx, ny, nz, h, opts)


def rpa_destroy(ctx: Context):
    ctx.close()


def rpa_last_error() -> str:
    return last_error()


def rpa_version() -> str:
    return _lib.rpa_version().decode()
