"""Thin ctypes binding of libvie (include/vie.h).

Argument marshalling only: every step of the operator, setup and solver runs
in the CUDA library.  Tensors are PyTorch CUDA tensors (used for device memory
and streams); host arrays are NumPy.  If the library is missing this module
raises at first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VIE_OK = 0
VIE_C64 = 1
VIE_C128 = 2
VIE_PLAN_DEFAULT = 0
VIE_PLAN_CIRC_2N = 1
VIE_PLAN_AUTOTUNE = 2

_STATUS = {0: "VIE_OK", 1: "VIE_ERR_INVALID", 2: "VIE_ERR_OOM", 3: "VIE_ERR_CUDA",
           4: "VIE_ERR_NOT_CONVERGED", 5: "VIE_ERR_TIMEOUT", 6: "VIE_ERR_NONFINITE"}


class VieError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class vie_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("m", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("k0", ctypes.c_double), ("eps_bg", ctypes.c_double), ("kappa", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("setup_ms", ctypes.c_double), ("tune_ms", ctypes.c_double),
                ("tune_candidates", ctypes.c_int), ("x_lines_per_block", ctypes.c_int),
                ("x_lines_per_block_inverse", ctypes.c_int)]


class vie_absorber(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("length", ctypes.c_double), ("degree", ctypes.c_int),
                ("direction", ctypes.c_int), ("eps2_max", ctypes.c_double)]


class vie_solve_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("x0_given", ctypes.c_int),
                ("use_preconditioner", ctypes.c_int), ("check_every", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("host_buffers", ctypes.c_int), ("resident", ctypes.c_int)]


class vie_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("matvecs64", ctypes.c_int),
                ("matvecs32", ctypes.c_int), ("converged", ctypes.c_int), ("fallback", ctypes.c_int),
                ("residual", ctypes.c_double), ("time_ms", ctypes.c_double), ("history_len", ctypes.c_int),
                ("history", ctypes.c_double * 64), ("graph_cycles", ctypes.c_int), ("reorth_steps", ctypes.c_int)]


VIE_SOLVE_FP64 = 0
VIE_SOLVE_MIXED = 1

_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGNATURES = {
    "vie_plan_create": ([ctypes.POINTER(_P), ctypes.POINTER(_I), _D, _D, _D, _I], _I),
    "vie_plan_destroy": ([_P], _I),
    "vie_plan_get_info": ([_P, ctypes.POINTER(vie_plan_info)], _I),
    "vie_set_permittivity": ([_P, _P, ctypes.POINTER(vie_absorber), _I], _I),
    "vie_set_contrast": ([_P, _P], _I),
    "vie_matvec": ([_P, _P, _P, _I, _P], _I),
    "vie_rhs_from_source": ([_P, _P, _P, _I, _P], _I),
    "vie_get_toeplitz": ([_P, _P], _I),
    "vie_eps2_from_round_trip": ([_D, _I, _D, _D, _D, _D, _D, ctypes.POINTER(_D)], _I),
    "vie_matvec_static_scratch": ([_P, _P, _P, _I, _P], _I),
    "vie_axis_field": ([_P, _P, _I, _P, _P], _I),
    "vie_net_param_count": ([], ctypes.c_size_t),
    "vie_net_create": ([ctypes.POINTER(_P), _P, ctypes.c_size_t, ctypes.c_ulonglong], _I),
    "vie_net_destroy": ([_P], _I),
    "vie_net_get_params": ([_P, _P], _I),
    "vie_net_get_grads": ([_P, _P], _I),
    "vie_net_apply": ([_P, _P, _P, _P, _I, _P], _I),
    "vie_net_accumulate": ([_P, _P, _P, _P, ctypes.POINTER(_D), _P], _I),
    "vie_net_zero_grad": ([_P], _I),
    "vie_net_set_training": ([_P, _I], _I),
    "vie_net_adam_step": ([_P, ctypes.c_float, ctypes.c_float, _P], _I),
    "vie_net_status": ([_P, ctypes.POINTER(_I), _I], _I),
    "vie_circulant_create": ([_P, _I, ctypes.POINTER(_P), _P], _I),
    "vie_circulant_apply": ([_P, _P, _P, _I, _P], _I),
    "vie_circulant_info": ([_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_size_t)], _I),
    "vie_circulant_destroy": ([_P], _I),
    "vie_set_circulant_preconditioner": ([_P, _P], _I),
    "vie_set_preconditioner": ([_P, _P, ctypes.c_size_t], _I),
    "vie_set_preconditioner_net": ([_P, _P], _I),
    "vie_plan_clone": ([_P, ctypes.POINTER(_P)], _I),
    "vie_matvec_batch": ([ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P], _I),
    "vie_solve_batch": ([ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D,
                         ctypes.POINTER(vie_solve_opts), ctypes.POINTER(vie_solve_info), _P], _I),
    "vie_reflection": ([_P, _P, _I, ctypes.POINTER(_D), _P], _I),
    "vie_solve": ([_P, _P, _P, _D, ctypes.POINTER(vie_solve_opts), ctypes.POINTER(vie_solve_info), _P], _I),
    "vie_probe_fma_tflops": ([_I, ctypes.POINTER(_D), _P], _I),
    "vie_probe_grid_barrier": ([_I, _D, ctypes.POINTER(_I)], _I),
    "vie_set_permeability": ([_P, _P], _I),
    "vie_slice_power": ([_P, _P, _I, ctypes.POINTER(_D), _P], _I),
    "vie_jm_matvec": ([_P, _P, _P, _I, _P], _I),
    "vie_jm_rhs_from_source": ([_P, _P, _P, _I, _P], _I),
    "vie_jm_solve": ([_P, _P, _P, _D, ctypes.POINTER(vie_solve_opts), ctypes.POINTER(vie_solve_info), _P], _I),
    "vie_last_error": ([], ctypes.c_char_p),
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libvie.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libvie.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != VIE_OK:
        msg = load().vie_last_error()
        raise VieError(status, where, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return VIE_C64
    if t.dtype == torch.complex128:
        return VIE_C128
    raise TypeError(f"unsupported dtype {t.dtype}; use complex64 or complex128")


class Plan:
    """Owns a vie_plan*; destroyed with the object or by close()."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = tuple(int(v) for v in n)

    @property
    def n_vox(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def close(self):
        if self.handle:
            load().vie_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = vie_plan_info()
        _check(load().vie_plan_get_info(self.handle, ctypes.byref(inf)), "vie_plan_get_info")
        return {"n": tuple(inf.n), "m": tuple(inf.m), "h": inf.h, "k0": inf.k0, "eps_bg": inf.eps_bg,
                "kappa": inf.kappa, "device_bytes": inf.device_bytes, "setup_ms": inf.setup_ms,
                "tune_ms": inf.tune_ms, "tune_candidates": inf.tune_candidates,
                "x_lines_per_block": inf.x_lines_per_block,
                "x_lines_per_block_inverse": inf.x_lines_per_block_inverse}


# ----------------------------------------------------------------------------
# entry points (same names as include/vie.h)
# ----------------------------------------------------------------------------
def vie_plan_create(n, h: float, k0: float, eps_bg: float, flags: int = VIE_PLAN_DEFAULT) -> Plan:
    lib = load()
    arr = (ctypes.c_int * 3)(*[int(v) for v in n])
    h_out = ctypes.c_void_p()
    _check(lib.vie_plan_create(ctypes.byref(h_out), arr, float(h), float(k0), float(eps_bg), int(flags)),
           "vie_plan_create")
    return Plan(h_out, n)


def vie_plan_destroy(plan: Plan):
    plan.close()


def vie_plan_get_info(plan: Plan) -> dict:
    return plan.info()


def _host_c128(a, count: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).ravel())
    if a.size != count:
        raise ValueError(f"expected {count} complex values, got {a.size}")
    return a


def vie_set_permittivity(plan: Plan, eps, absorbers=()):
    """eps: (nz, ny, nx) complex relative permittivity; absorbers: sequence of
    dicts with keys x0, length, degree, eps2_max and optional direction."""
    e = _host_c128(eps, plan.n_vox)
    arr = (vie_absorber * max(1, len(absorbers)))()
    for i, ab in enumerate(absorbers):
        arr[i] = vie_absorber(float(ab["x0"]), float(ab["length"]), int(ab["degree"]),
                              int(ab.get("direction", 1)), float(ab["eps2_max"]))
    _check(load().vie_set_permittivity(plan.handle, e.ctypes.data_as(ctypes.c_void_p), arr, len(absorbers)),
           "vie_set_permittivity")


def vie_set_contrast(plan: Plan, chi):
    c = _host_c128(chi, plan.n_vox)
    _check(load().vie_set_contrast(plan.handle, c.ctypes.data_as(ctypes.c_void_p)), "vie_set_contrast")


def _vec_call(fn_name, plan: Plan, x, y, stream):
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous CUDA tensors")
    if x.dtype != y.dtype or x.numel() != 3 * plan.n_vox or y.numel() != 3 * plan.n_vox:
        raise ValueError("x and y must be complex vectors of 3*nx*ny*nz elements and equal dtype")
    fn = getattr(load(), fn_name)
    _check(fn(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), _dtype_code(x),
              _stream_handle(stream)), fn_name)
    return y


def vie_matvec(plan: Plan, x, y, stream=None):
    """y = x - M (N x) on the device (stream: torch stream or None = current)."""
    return _vec_call("vie_matvec", plan, x, y, stream)


def vie_matvec_static_scratch(plan: Plan, x, y, stream=None):
    """y = x - M (N x) using the library's static workspace (allocates nothing)."""
    return _vec_call("vie_matvec_static_scratch", plan, x, y, stream)


def vie_rhs_from_source(plan: Plan, src, b, stream=None):
    """b = M ((N - I) src) on the device."""
    return _vec_call("vie_rhs_from_source", plan, src, b, stream)


def vie_get_toeplitz(plan: Plan) -> np.ndarray:
    """FP64 octant (6, nz, ny, nx) complex128."""
    nx, ny, nz = plan.n
    out = np.empty((6, nz, ny, nx), dtype=np.complex128)
    _check(load().vie_get_toeplitz(plan.handle, out.ctypes.data_as(ctypes.c_void_p)), "vie_get_toeplitz")
    return out


def vie_eps2_from_round_trip(r_rt, degree, length, k0, eps_r, D=2.0, eta=1.0) -> float:
    out = ctypes.c_double()
    _check(load().vie_eps2_from_round_trip(float(r_rt), int(degree), float(length), float(k0), float(eps_r),
                                           float(D), float(eta), ctypes.byref(out)), "vie_eps2_from_round_trip")
    return out.value


def vie_solve(plan: Plan, b, x, tol: float, mode: int = VIE_SOLVE_MIXED, restart: int = 100,
              max_iters: int = 5000, inner_tol: float = 1e-4, max_outer: int = 200, x0_given: bool = False,
              use_preconditioner: bool = False, check_every: int = 4, timeout_s: float = 600.0,
              stream=None, raise_on_not_converged: bool = True, resident: bool = False) -> dict:
    """Solve (I - M N) x = b on the device.  b, x: complex128 CUDA tensors, or
    (both) C-contiguous complex128 NumPy arrays on the host, which the library
    stages through device buffers (opts.host_buffers = 1); x is written in
    place either way.  With raise_on_not_converged=False a solve that stopped
    at a cap (VIE_ERR_NOT_CONVERGED) or at the time limit (VIE_ERR_TIMEOUT)
    returns its report (x holds the last iterate) instead of raising."""
    host = _vectors_kind([(b, x)], [plan])
    opts = vie_solve_opts(int(mode), int(restart), int(max_iters), float(inner_tol), int(max_outer),
                          int(bool(x0_given)), int(bool(use_preconditioner)), int(check_every), float(timeout_s),
                          int(host), int(bool(resident)))
    info = vie_solve_info()
    st = load().vie_solve(plan.handle, _vec_ptr(b), _vec_ptr(x), float(tol),
                          ctypes.byref(opts), ctypes.byref(info), _stream_handle(stream))
    out = {"status": st, "iterations": info.iterations, "outer": info.outer, "matvecs64": info.matvecs64,
           "matvecs32": info.matvecs32, "converged": bool(info.converged), "fallback": bool(info.fallback),
           "residual": info.residual, "time_ms": info.time_ms,
           "history": [info.history[i] for i in range(min(info.history_len, 64))],
           "graph_cycles": info.graph_cycles, "reorth_steps": info.reorth_steps}
    if st != VIE_OK and not (st in (4, 5) and not raise_on_not_converged):
        _check(st, "vie_solve")
    return out


def _vectors_kind(pairs, plans) -> bool:
    """True for host NumPy vectors, False for CUDA tensors; checks type, size
    and contiguity of every (b, x) pair."""
    import torch
    host = isinstance(pairs[0][0], np.ndarray)
    for (b, x), p in zip(pairs, plans):
        for t in (b, x):
            if host:
                ok = (isinstance(t, np.ndarray) and t.dtype == np.complex128 and t.flags.c_contiguous
                      and t.size == 3 * p.n_vox)
                if t is x and not t.flags.writeable:
                    ok = False
            else:
                ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
                      and t.dtype == torch.complex128 and t.numel() == 3 * p.n_vox)
            if not ok:
                raise ValueError("b and x must both be contiguous complex128 vectors of 3*nx*ny*nz entries: "
                                 "CUDA tensors, or writable NumPy arrays on the host")
    return host


def _vec_ptr(t):
    return ctypes.c_void_p(t.ctypes.data if isinstance(t, np.ndarray) else t.data_ptr())


def vie_plan_clone(base: Plan) -> Plan:
    """A plan sharing base's entries and spectra, with its own (zero) contrast."""
    h_out = ctypes.c_void_p()
    _check(load().vie_plan_clone(base.handle, ctypes.byref(h_out)), "vie_plan_clone")
    return Plan(h_out, base.n)


def _ptr_array(vals):
    return (ctypes.c_void_p * len(vals))(*[ctypes.c_void_p(v) for v in vals])


def vie_matvec_batch(plans, xs, ys, stream=None):
    """y_i = x_i - M_i (N_i x_i) for every plan (CUDA tensors of one dtype)."""
    if not (len(plans) == len(xs) == len(ys)) or not plans:
        raise ValueError("plans, xs and ys must have the same non-zero length")
    code = _dtype_code(xs[0])
    for p, x, y in zip(plans, xs, ys):
        if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous() and x.dtype == y.dtype
                and x.dtype == xs[0].dtype and x.numel() == 3 * p.n_vox and y.numel() == 3 * p.n_vox):
            raise ValueError("every x_i, y_i must be a contiguous CUDA vector of 3*nx*ny*nz entries of one dtype")
    _check(load().vie_matvec_batch(_ptr_array([p.handle.value for p in plans]), len(plans),
                                   _ptr_array([x.data_ptr() for x in xs]), _ptr_array([y.data_ptr() for y in ys]),
                                   code, _stream_handle(stream)), "vie_matvec_batch")


def vie_solve_batch(plans, bs, xs, tol: float, mode: int = VIE_SOLVE_MIXED, restart: int = 100,
                    max_iters: int = 5000, inner_tol: float = 1e-4, max_outer: int = 200, x0_given: bool = False,
                    use_preconditioner: bool = False, check_every: int = 4, timeout_s: float = 600.0,
                    stream=None, raise_on_not_converged: bool = True, resident: bool = False):
    """Solve every (plan, b, x) together (CUDA tensors, or host NumPy arrays
    as in vie_solve); returns (status, [info dict per problem])."""
    n = len(plans)
    if not (n == len(bs) == len(xs)) or n == 0:
        raise ValueError("plans, bs and xs must have the same non-zero length")
    host = _vectors_kind(list(zip(bs, xs)), plans)
    if any(isinstance(t, np.ndarray) != host for t in list(bs) + list(xs)):
        raise ValueError("every b and x must be of one kind: all CUDA tensors or all host arrays")
    opts = vie_solve_opts(int(mode), int(restart), int(max_iters), float(inner_tol), int(max_outer),
                          int(bool(x0_given)), int(bool(use_preconditioner)), int(check_every), float(timeout_s),
                          int(host), int(bool(resident)))
    infos = (vie_solve_info * n)()
    st = load().vie_solve_batch(_ptr_array([p.handle.value for p in plans]), n,
                                _ptr_array([_vec_ptr(b).value for b in bs]), _ptr_array([_vec_ptr(x).value for x in xs]),
                                float(tol), ctypes.byref(opts), infos, _stream_handle(stream))
    out = []
    for info in infos:
        out.append({"iterations": info.iterations, "outer": info.outer, "matvecs64": info.matvecs64,
                    "matvecs32": info.matvecs32, "converged": bool(info.converged), "fallback": bool(info.fallback),
                    "residual": info.residual, "time_ms": info.time_ms,
                    "history": [info.history[i] for i in range(min(info.history_len, 64))],
                    "graph_cycles": info.graph_cycles, "reorth_steps": info.reorth_steps})
    if st != VIE_OK and not (st in (4, 5) and not raise_on_not_converged):
        _check(st, "vie_solve_batch")
    return st, out


class Net:
    """Owns a vie_net* (learned preconditioner)."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            load().vie_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Circulant:
    """Owns a vie_circulant* (block-circulant preconditioner of a plan)."""

    def __init__(self, handle, plan):
        self.handle = handle
        self.plan = plan          # keeps the plan alive while the factors exist

    def close(self):
        if self.handle:
            load().vie_circulant_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


VIE_CIRC_DEFAULT = 0
VIE_CIRC_FP16_FACTORS = 1


def vie_circulant_create(plan: Plan, flags: int = VIE_CIRC_DEFAULT, stream=None) -> Circulant:
    h = ctypes.c_void_p()
    _check(load().vie_circulant_create(plan.handle, int(flags), ctypes.byref(h), _stream_handle(stream)),
           "vie_circulant_create")
    return Circulant(h, plan)


def vie_circulant_apply(c: Circulant, v, z, stream=None):
    if not (v.is_cuda and z.is_cuda and v.dtype == z.dtype and v.numel() == 3 * c.plan.n_vox == z.numel()):
        raise ValueError("v and z must be CUDA vectors of 3*nx*ny*nz entries of one dtype")
    _check(load().vie_circulant_apply(c.handle, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                      _dtype_code(v), _stream_handle(stream)), "vie_circulant_apply")
    return z


def vie_circulant_info(c: Circulant) -> dict:
    ms = ctypes.c_double()
    nbytes = ctypes.c_size_t()
    _check(load().vie_circulant_info(c.handle, ctypes.byref(ms), ctypes.byref(nbytes)), "vie_circulant_info")
    return {"build_ms": ms.value, "device_bytes": nbytes.value}


def vie_circulant_destroy(c: Circulant):
    c.close()


def vie_set_circulant_preconditioner(plan: Plan, c: Circulant | None):
    _check(load().vie_set_circulant_preconditioner(plan.handle, c.handle if c is not None else None),
           "vie_set_circulant_preconditioner")
    plan._net = c        # keep the preconditioner alive while it is set


def vie_net_param_count() -> int:
    return int(load().vie_net_param_count())


def vie_net_create(params=None, seed: int = 0) -> Net:
    h = ctypes.c_void_p()
    if params is None:
        _check(load().vie_net_create(ctypes.byref(h), None, 0, int(seed)), "vie_net_create")
    else:
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        _check(load().vie_net_create(ctypes.byref(h), a.ctypes.data_as(ctypes.c_void_p), a.size, int(seed)),
               "vie_net_create")
    return Net(h)


def vie_net_destroy(net: Net):
    net.close()


def vie_net_get_params(net: Net) -> np.ndarray:
    out = np.empty(vie_net_param_count(), dtype=np.float32)
    _check(load().vie_net_get_params(net.handle, out.ctypes.data_as(ctypes.c_void_p)), "vie_net_get_params")
    return out


def vie_net_get_grads(net: Net) -> np.ndarray:
    out = np.empty(vie_net_param_count(), dtype=np.float32)
    _check(load().vie_net_get_grads(net.handle, out.ctypes.data_as(ctypes.c_void_p)), "vie_net_get_grads")
    return out


def vie_net_apply(net: Net, plan: Plan, v, z, stream=None):
    if not (v.is_cuda and z.is_cuda and v.dtype == z.dtype and v.numel() == 3 * plan.n_vox == z.numel()):
        raise ValueError("v and z must be CUDA vectors of 3*nx*ny*nz entries of one dtype")
    _check(load().vie_net_apply(net.handle, plan.handle, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                _dtype_code(v), _stream_handle(stream)), "vie_net_apply")
    return z


def vie_net_status(net: Net, clear: bool = False) -> int:
    """0 fine, 1 a non-finite output was replaced by v, 2 a tensor-core wait
    timed out (synchronises the device)."""
    flag = ctypes.c_int()
    _check(load().vie_net_status(net.handle, ctypes.byref(flag), int(bool(clear))), "vie_net_status")
    return flag.value


def vie_net_accumulate(net: Net, plan: Plan, r, e, stream=None) -> float:
    import torch
    for t in (r, e):
        if not (t.is_cuda and t.dtype == torch.complex64 and t.numel() == 3 * plan.n_vox and t.is_contiguous()):
            raise ValueError("r and e must be contiguous complex64 CUDA vectors of 3*nx*ny*nz entries")
    loss = ctypes.c_double()
    _check(load().vie_net_accumulate(net.handle, plan.handle, ctypes.c_void_p(r.data_ptr()),
                                     ctypes.c_void_p(e.data_ptr()), ctypes.byref(loss), _stream_handle(stream)),
           "vie_net_accumulate")
    return loss.value


VIE_TRAIN_TENSOR_BF16 = 0
VIE_TRAIN_FP32 = 1


def vie_net_set_training(net: Net, mode: int):
    _check(load().vie_net_set_training(net.handle, int(mode)), "vie_net_set_training")


def vie_net_zero_grad(net: Net):
    _check(load().vie_net_zero_grad(net.handle), "vie_net_zero_grad")


def vie_net_adam_step(net: Net, lr: float, grad_scale: float = 1.0, stream=None):
    _check(load().vie_net_adam_step(net.handle, float(lr), float(grad_scale), _stream_handle(stream)),
           "vie_net_adam_step")


def vie_set_preconditioner(plan: Plan, weights):
    """Learned right preconditioner from FP32 parameters (host array of
    vie_net_param_count() floats); None removes any preconditioner.  The plan
    keeps its own copy."""
    if weights is None:
        _check(load().vie_set_preconditioner(plan.handle, None, 0), "vie_set_preconditioner")
    else:
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(load().vie_set_preconditioner(plan.handle, ctypes.c_void_p(w.ctypes.data), w.nbytes),
               "vie_set_preconditioner")
    plan._net = None


def vie_set_preconditioner_net(plan: Plan, net):
    """A network object (kept by the caller) as the right preconditioner."""
    _check(load().vie_set_preconditioner_net(plan.handle, net.handle if net is not None else None),
           "vie_set_preconditioner_net")
    plan._net = net      # keep the network alive while it is set


def vie_axis_field(plan: Plan, w, n_keep: int, stream=None):
    """E = w / chi on the centre axis for ix < n_keep: complex128 tensor (3, n_keep)."""
    import torch
    if not (w.is_cuda and w.dtype == torch.complex128 and w.numel() == 3 * plan.n_vox and w.is_contiguous()):
        raise ValueError("w must be a contiguous complex128 CUDA vector of 3*nx*ny*nz entries")
    e = torch.empty((3, int(n_keep)), dtype=torch.complex128, device=w.device)
    _check(load().vie_axis_field(plan.handle, ctypes.c_void_p(w.data_ptr()), int(n_keep),
                                 ctypes.c_void_p(e.data_ptr()), _stream_handle(stream)), "vie_axis_field")
    return e


def vie_reflection(e_ref, e, stream=None) -> float:
    """R = sum |e_ref - e|^2 / sum |e_ref|^2 on the device (complex128 tensors)."""
    import torch
    for t in (e_ref, e):
        if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
            raise ValueError("fields must be contiguous complex128 CUDA tensors")
    if e_ref.numel() != e.numel():
        raise ValueError("fields differ in size")
    out = ctypes.c_double()
    _check(load().vie_reflection(ctypes.c_void_p(e_ref.data_ptr()), ctypes.c_void_p(e.data_ptr()), e.numel(),
                                 ctypes.byref(out), _stream_handle(stream)), "vie_reflection")
    return out.value


def vie_set_permeability(plan: Plan, mu=None):
    """mu: (nz, ny, nx) complex relative permeability, or None for the
    impedance-matched permeability of the plan's current permittivity."""
    if mu is None:
        _check(load().vie_set_permeability(plan.handle, None), "vie_set_permeability")
    else:
        m = _host_c128(mu, plan.n_vox)
        _check(load().vie_set_permeability(plan.handle, m.ctypes.data_as(ctypes.c_void_p)), "vie_set_permeability")


def _jm_vec_call(fn_name, plan: Plan, x, y, stream):
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous CUDA tensors")
    if x.dtype != y.dtype or x.numel() != 6 * plan.n_vox or y.numel() != 6 * plan.n_vox:
        raise ValueError("x and y must be complex vectors of 6*nx*ny*nz elements and equal dtype")
    _check(getattr(load(), fn_name)(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    _dtype_code(x), _stream_handle(stream)), fn_name)


def vie_jm_matvec(plan: Plan, x, y, stream=None):
    """y = u - M (T u) for the JM-VIE (6N vectors)."""
    _jm_vec_call("vie_jm_matvec", plan, x, y, stream)


def vie_jm_rhs_from_source(plan: Plan, src, b, stream=None):
    """b for impressed currents (w_e, w_m) (6N vectors)."""
    _jm_vec_call("vie_jm_rhs_from_source", plan, src, b, stream)


def vie_jm_solve(plan: Plan, b, x, tol: float, mode: int = VIE_SOLVE_MIXED, restart: int = 100,
                 max_iters: int = 5000, inner_tol: float = 1e-4, max_outer: int = 200, x0_given: bool = False,
                 check_every: int = 4, timeout_s: float = 600.0, stream=None,
                 raise_on_not_converged: bool = True) -> dict:
    """Solve the JM-VIE; b, x: 6N complex128 CUDA tensors or host NumPy arrays."""
    import torch
    host = isinstance(b, np.ndarray)
    for t in (b, x):
        ok = (isinstance(t, np.ndarray) and t.dtype == np.complex128 and t.flags.c_contiguous) if host else \
             (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == torch.complex128)
        if not ok or (t.size if host else t.numel()) != 6 * plan.n_vox:
            raise ValueError("b and x must be contiguous complex128 vectors of 6*nx*ny*nz entries")
    opts = vie_solve_opts(int(mode), int(restart), int(max_iters), float(inner_tol), int(max_outer),
                          int(bool(x0_given)), 0, int(check_every), float(timeout_s), int(host), 0)
    info = vie_solve_info()
    st = load().vie_jm_solve(plan.handle, _vec_ptr(b), _vec_ptr(x), float(tol), ctypes.byref(opts),
                             ctypes.byref(info), _stream_handle(stream))
    out = {"status": st, "iterations": info.iterations, "outer": info.outer, "matvecs64": info.matvecs64,
           "matvecs32": info.matvecs32, "converged": bool(info.converged), "residual": info.residual,
           "time_ms": info.time_ms}
    if st != VIE_OK and not (st in (4, 5) and not raise_on_not_converged):
        _check(st, "vie_jm_solve")
    return out


def vie_probe_grid_barrier(absent_block: int, wait_ms: float) -> bool:
    """One grid barrier with block absent_block (-1: none) missing; True if
    the other blocks gave up after wait_ms (the solver's barrier timeout)."""
    out = _I()
    _check(load().vie_probe_grid_barrier(int(absent_block), float(wait_ms), ctypes.byref(out)),
           "vie_probe_grid_barrier")
    return bool(out.value)


def vie_probe_fma_tflops(dtype_code: int, stream=None) -> float:
    """Measured FP32 (VIE_C64) or FP64 (VIE_C128) FMA throughput, TFLOP/s."""
    out = ctypes.c_double()
    _check(load().vie_probe_fma_tflops(int(dtype_code), ctypes.byref(out), _stream_handle(stream)),
           "vie_probe_fma_tflops")
    return out.value


def vie_slice_power(plan: Plan, w, ix: int, stream=None) -> float:
    """T = sum |w / chi|^2 over the voxels of plane ix with chi != 0."""
    import torch
    if not (w.is_cuda and w.dtype == torch.complex128 and w.numel() == 3 * plan.n_vox and w.is_contiguous()):
        raise ValueError("w must be a contiguous complex128 CUDA vector of 3*nx*ny*nz entries")
    out = ctypes.c_double()
    _check(load().vie_slice_power(plan.handle, ctypes.c_void_p(w.data_ptr()), int(ix), ctypes.byref(out),
                                  _stream_handle(stream)), "vie_slice_power")
    return out.value


def vie_last_error() -> str:
    m = load().vie_last_error()
    return m.decode() if m else ""
