"""Thin ctypes binding of libcrkfr (include/crkfr.h).

Only argument marshalling lives here: every step of the method runs in the
library's CUDA kernels.  Device memory and streams come from PyTorch: state
and coefficient arrays are contiguous float64 CUDA tensors in the library's
nodal layout, and calls go to ``torch.cuda.current_stream()``.

The functions of the C ABI are reachable under their own names through
``lib()``; ``Solver`` wraps one context.
"""
import ctypes
import os

import numpy as np

from .build import library_path

CRKFR_OK = 0
STATUS = {0: "CRKFR_OK", -1: "CRKFR_ERR_ARG", -2: "CRKFR_ERR_UNSUPPORTED", -3: "CRKFR_ERR_CUDA",
          -4: "CRKFR_ERR_NONPHYSICAL", -6: "CRKFR_ERR_STATE", -7: "CRKFR_ERR_ALLOC"}
# the *_wb systems are the well-balanced shallow-water forms (pressure in the
# non-conservative product, free-surface dissipation)
SYSTEMS = {"varadv1d": 0, "swe1d": 1, "swe2d": 2, "swe1d_wb": 3, "swe2d_wb": 4}
NODES = {"gl": 0, "gll": 1}
# source terms (crkfr_source): None, linear damping -K v (advection), Chezy
# friction -C_f |v| v on the momentum (shallow water)
SOURCES = {None: 0, "linear": 1, "chezy": 2}
NVARS = {"varadv1d": 1, "swe1d": 2, "swe2d": 3, "swe1d_wb": 2, "swe2d_wb": 3}
DIM = {"varadv1d": 1, "swe1d": 1, "swe2d": 2, "swe1d_wb": 1, "swe2d_wb": 2}


class CrkfrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("nodes", ctypes.c_int32), ("source", ctypes.c_int32),
                ("gravity", ctypes.c_double), ("cfl_safety", ctypes.c_double),
                ("cfl_number", ctypes.c_double), ("source_coef", ctypes.c_double),
                ("rk", ctypes.c_int32), ("nc_face_mode", ctypes.c_int32),
                ("coef_dissipation", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# face non-conservative terms (crkfr_nc_face): only "frozen" is built
NC_FACE = {"frozen": 0, "literal": 1, "stagewise": 2}


def make_config(system, degree, nodes, gravity, cfl_safety, cfl_number, source, source_coef,
                rk=0, nc_face="frozen", coef_dissipation=False):
    return Config(SYSTEMS[system], degree, NODES[nodes], SOURCES[source], gravity, cfl_safety,
                  cfl_number, float(source_coef), int(rk), NC_FACE[nc_face],
                  1 if coef_dissipation else 0, 0)


_P = ctypes.c_void_p
_D = ctypes.c_double
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); mirrors include/crkfr.h
SIGNATURES = {
    "crkfr_create": (_I32, [ctypes.POINTER(_P), ctypes.POINTER(Config)]),
    "crkfr_destroy": (None, [_P]),
    "crkfr_set_mesh": (_I32, [_P, _I32, _PI64, _PD, _PD, _I32]),
    "crkfr_sizes": (_I32, [_P, _PI64, _PI64]),
    "crkfr_get_nodes": (_I32, [_P, _PD, _PD]),
    "crkfr_get_cfl": (_I32, [_P, _PD]),
    "crkfr_set_coefficients": (_I32, [_P, _P, _P]),
    "crkfr_compute_dt": (_I32, [_P, _P, _PD, _P]),
    "crkfr_residual": (_I32, [_P, _P, _D, _P, _P]),
    "crkfr_step": (_I32, [_P, _P, _D, _I64, _P]),
    "crkfr_advance": (_I32, [_P, _P, _D, _I64, _PI64, _P]),
    "crkfr_step_host": (_I32, [_P, _P, _P, _D, _I64, _P]),
    "crkfr_set_subdomain": (_I32, [_P, _I32]),
    "crkfr_halo_buffers": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                  ctypes.POINTER(_P), _PI64]),
    "crkfr_step_local": (_I32, [_P, _P, _D, _P]),
    "crkfr_step_indicator": (_I32, [_P, _P, _P]),
    "crkfr_limiter_halo_buffers": (_I32, [_P, _I32, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                          ctypes.POINTER(_P), ctypes.POINTER(_P), _PI64]),
    "crkfr_step_faces": (_I32, [_P, _P, _P]),
    "crkfr_step_adjoint": (_I32, [_P, _P, _P, _P, _P, _D, _P]),
    "crkfr_adjoint_local": (_I32, [_P, _P, _P, _D, _P]),
    "crkfr_adjoint_halo_buffers": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                          ctypes.POINTER(_P), ctypes.POINTER(_P), _PI64]),
    "crkfr_adjoint_faces": (_I32, [_P, _P, _P, _P, _P, _D, _P]),
    "crkfr_record_size": (_I32, [_P, _PI64]),
    "crkfr_step_record": (_I32, [_P, _P, _D, _P, _I32, _P]),
    "crkfr_step_adjoint_recorded": (_I32, [_P, _P, _P, _P, _P, _P, _D, _P]),
    "crkfr_step_local_record": (_I32, [_P, _P, _D, _P, _I32, _P]),
    "crkfr_record_halo_buffers": (_I32, [_P, _P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), ctypes.POINTER(_P), _PI64]),
    "crkfr_step_faces_record": (_I32, [_P, _P, _P, _P]),
    "crkfr_adjoint_sums": (_I32, [_P, _P, _P]),
    "crkfr_adjoint_faces_recorded": (_I32, [_P, _P, _P, _P, _P, _P, _D, _P]),
    "crkfr_get_time": (_I32, [_P, _PD, _PD, _P]),
    "crkfr_set_time": (_I32, [_P, _D, _P]),
    "crkfr_get_status": (_I32, [_P, _P]),
    "crkfr_launch_count": (_I64, [_P]),
    "crkfr_profile_enable": (_I32, [_P, _I32]),
    "crkfr_set_limiter": (_I32, [_P, _I32, _D]),
    "crkfr_set_tile_1d": (_I32, [_P, _I32]),
    "crkfr_batch_set_tuning": (_I32, [_P, _I32, _I32, _I32]),
    "crkfr_batch_get_tuning": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                      ctypes.POINTER(_I32), _PD]),
    "crkfr_batch_autotune": (_I32, [_P, _P, _I32, _P]),
    "crkfr_limiter_alpha": (_I32, [_P, _P, _P]),
    "crkfr_profile_read": (_I32, [_P, _I32, _PI64, _PD]),
    "crkfr_math_check": (_I32, [_P, _P, _I64, _I32, _P]),
    "crkfr_fp64_probe": (_I32, [_I32, _I32, _I32, _P, _PD, _P]),
    "crkfr_step_1d_noalloc": (_I32, [ctypes.POINTER(Config), _I64, _D, _D, _P, _P, _P, _D, _I64,
                                     _P]),
    "crkfr_batch_create": (_I32, [ctypes.POINTER(_P), ctypes.POINTER(Config), _I32,
                                  ctypes.POINTER(ctypes.c_int32), _PI64, _PD, _PD]),
    "crkfr_batch_destroy": (None, [_P]),
    "crkfr_batch_layout": (_I32, [_P, _PI64, _PI64]),
    "crkfr_batch_set_coefficients": (_I32, [_P, _P, _P]),
    "crkfr_batch_step": (_I32, [_P, _P, _D, _I64, _I32, _P]),
    "crkfr_batch_get_times": (_I32, [_P, _PD, _P]),
    "crkfr_batch_get_status": (_I32, [_P, _P]),
    "crkfr_batch_launch_count": (_I64, [_P]),
    "crkfr_batch_profile_enable": (_I32, [_P, _I32]),
    "crkfr_batch_profile_read": (_I32, [_P, _PI64, _PD]),
    "crkfr_batch_last_error": (ctypes.c_char_p, [_P]),
    "crkfr_error_string": (ctypes.c_char_p, [_I32]),
    "crkfr_last_error": (ctypes.c_char_p, [_P]),
}

_LIB = None


def lib():
    """The loaded library (loaded on first use; raises if it was not built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_2512_08611_gb300.build`")
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def _stream():
    import torch
    if not torch.cuda.is_available():
        return ctypes.c_void_p(0)   # calls that reach CUDA report the error themselves
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _DeviceBlock:
    """A library-owned device array exposed to torch without a copy."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3}


def math_check(x, op):
    """out = 1/x (op 'rcp'), sqrt(x) (op 'sqrt') or 1/sqrt(x) (op 'rsqrt') by
    the kernels' own FP64 routines; x a contiguous float64 CUDA tensor."""
    import torch
    if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    out = torch.empty_like(x)
    st = lib().crkfr_math_check(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                x.numel(), {"rcp": 0, "sqrt": 1, "rsqrt": 2}[op], _stream())
    if st != CRKFR_OK:
        raise CrkfrError(st, lib().crkfr_error_string(st).decode())
    return out


def fp64_probe(mode, blocks=None, iters=4096, repeats=5):
    """FP64 throughput of this GPU in TFLOP/s (crkfr_fp64_probe): 'fma' (the
    FP64 pipe of the CUDA cores), 'mma' (mma.sync m8n8k4 on the tensor
    cores) or 'both' interleaved.  Best of `repeats` launches timed with CUDA
    events on the current stream, after one warm-up launch."""
    import torch
    m = {"fma": 0, "mma": 1, "both": 2}[mode]
    if blocks is None:
        blocks = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8
    sink = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    flops = ctypes.c_double(0.0)
    stream = torch.cuda.current_stream()
    best = None
    for r in range(repeats + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = lib().crkfr_fp64_probe(m, int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()),
                                    ctypes.byref(flops), _stream())
        e1.record(stream)
        if st != CRKFR_OK:
            raise CrkfrError(st, lib().crkfr_error_string(st).decode())
        e1.synchronize()
        if r > 0:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    if not torch.isfinite(sink).all():
        raise RuntimeError("probe produced non-finite values")
    return flops.value / (best * 1e-3) / 1e12


def step_1d_noalloc(system, degree, n_elem, lo, hi, c, u_in, u_out, dt=0.0, nsteps=1,
                    nodes="gl", gravity=9.81, cfl_safety=0.5, cfl_number=0.0, source=None,
                    source_coef=0.0, rk=0, nc_face="frozen", coef_dissipation=False):
    """crkfr_step_1d_noalloc: 1D steps whose scratch lives in the library's
    static device array, for callers that cannot allocate device memory."""
    import torch
    if system not in NVARS or DIM[system] != 1:
        raise ValueError(f"step_1d_noalloc takes a 1D system, got {system!r}")
    n_elem, n = int(n_elem), int(degree) + 1
    shapes = {"c": (n_elem, n), "u_in": (NVARS[system], n_elem, n),
              "u_out": (NVARS[system], n_elem, n)}
    for name, t in (("c", c), ("u_in", u_in), ("u_out", u_out)):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"{name}: expected a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != shapes[name]:
            raise ValueError(f"{name}: expected contiguous float64 of shape {shapes[name]}, got "
                             f"{t.dtype} {tuple(t.shape)}")
    cfg = make_config(system, degree, nodes, gravity, cfl_safety, cfl_number, source, source_coef,
                      rk, nc_face, coef_dissipation)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib().crkfr_step_1d_noalloc(ctypes.byref(cfg), int(n_elem), float(lo), float(hi), ptr(c),
                                     ptr(u_in), ptr(u_out), float(dt), int(nsteps), _stream())
    if st != CRKFR_OK:
        raise CrkfrError(st, lib().crkfr_last_error(None).decode() or
                         lib().crkfr_error_string(st).decode())
    return u_out


class Solver:
    """One library context: a system, degree and node family on one mesh.

    ``system``: 'varadv1d', 'swe1d', 'swe2d', or the well-balanced
    shallow-water forms 'swe1d_wb', 'swe2d_wb'; ``nodes``: 'gl' (Radau
    correction) or 'gll' (g_2 correction).  ``cfl_number`` <= 0 takes the
    library's own von Neumann CFL(N).  ``source``: None, 'linear' (s = -K v,
    advection) or 'chezy' (s = -C_f |v| v on the momentum, shallow water),
    with ``source_coef`` K or C_f; a source switches the stages to
    SSP3-IMEX(4,3,3)."""

    def __init__(self, system, degree, nodes="gl", gravity=9.81, cfl_safety=0.5, cfl_number=0.0,
                 source=None, source_coef=0.0, rk=0, nc_face="frozen", coef_dissipation=False):
        self.system, self.degree, self.family = system, degree, nodes
        self.source, self.source_coef = source, source_coef
        self.limiter = (None, 0.0)
        self.M = NVARS[system]
        self.dim = DIM[system]
        self.n = degree + 1
        cfg = make_config(system, degree, nodes, gravity, cfl_safety, cfl_number, source,
                          source_coef, rk, nc_face, coef_dissipation)
        h = ctypes.c_void_p()
        self._check(lib().crkfr_create(ctypes.byref(h), ctypes.byref(cfg)), None)
        self.h = h
        self.shape = None

    def _check(self, status, h="self"):
        if status != CRKFR_OK:
            handle = self.h if h == "self" else h
            msg = lib().crkfr_last_error(handle).decode()   # NULL: this thread's last error
            raise CrkfrError(status, msg or lib().crkfr_error_string(status).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().crkfr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up ----------------------------------------------------------------
    def set_mesh(self, n_elem, lo, hi, periodic=True):
        n_elem = [int(v) for v in np.atleast_1d(n_elem)]
        lo = [float(v) for v in np.atleast_1d(lo)]
        hi = [float(v) for v in np.atleast_1d(hi)]
        d = len(n_elem)
        arr = (ctypes.c_int64 * d)(*n_elem)
        self._check(lib().crkfr_set_mesh(self.h, d, arr, (ctypes.c_double * d)(*lo),
                                         (ctypes.c_double * d)(*hi),
                                         (1 << d) - 1 if periodic else 0))
        self.n_elem, self.lo, self.hi = n_elem, lo, hi
        self.limiter = (None, 0.0)   # a new mesh switches the limiter off
        n = self.n
        if self.dim == 1:
            self.shape = (self.M, n_elem[0], n)
            self.coef_shape = (n_elem[0], n)
        else:
            self.shape = (self.M, n_elem[1], n_elem[0], n, n)
            self.coef_shape = (n_elem[1], n_elem[0], n, n)
        return self

    def set_subdomain(self, enable=True):
        """Make the context one part of a larger mesh: in 2D a horizontal slab
        whose coefficient field carries one halo row below and one above, in
        1D a range of elements whose coefficient field carries the element
        left of it and the element right of it."""
        self._check(lib().crkfr_set_subdomain(self.h, 1 if enable else 0))
        self.subdomain = bool(enable)
        if self.shape is not None and self.dim == 2:
            n, (Ex, Ey) = self.n, self.n_elem
            self.coef_shape = (Ey + 2 if enable else Ey, Ex, n, n)
        elif self.shape is not None:
            self.coef_shape = (self.n_elem[0] + 2 if enable else self.n_elem[0], self.n)

    def halo_buffers(self):
        """(send_bottom, send_top, recv_bottom, recv_top) as float64 CUDA
        tensors viewing the context's trace buffer (no copy)."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        cnt = ctypes.c_int64()
        self._check(lib().crkfr_halo_buffers(self.h, *[ctypes.byref(p) for p in ptrs],
                                             ctypes.byref(cnt)))
        return tuple(torch.as_tensor(_DeviceBlock(p.value, cnt.value), device="cuda")
                     for p in ptrs)

    def limiter_halo_buffers(self, kind):
        """Limited 2D slab: (send_bottom, send_top, recv_bottom, recv_top) of
        the raw indicator rows (kind 0) or of the limiter's y-face data
        (kind 1), float64 CUDA tensors viewing the context's buffers."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        cnt = ctypes.c_int64()
        self._check(lib().crkfr_limiter_halo_buffers(self.h, int(kind),
                                                     *[ctypes.byref(p) for p in ptrs],
                                                     ctypes.byref(cnt)))
        return tuple(torch.as_tensor(_DeviceBlock(p.value, cnt.value), device="cuda")
                     for p in ptrs)

    def step_indicator(self, u):
        """Limited 2D slab: the raw indicator of the slab's own rows."""
        self._check(lib().crkfr_step_indicator(self.h, self._dev(u, self.shape), _stream()))

    def step_local(self, u, dt):
        self._check(lib().crkfr_step_local(self.h, self._dev(u, self.shape), float(dt), _stream()))

    def step_faces(self, u):
        self._check(lib().crkfr_step_faces(self.h, self._dev(u, self.shape), _stream()))

    def nodes(self):
        n = self.n
        xi, w = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        self._check(lib().crkfr_get_nodes(self.h, xi, w))
        return np.array(xi[:]), np.array(w[:])

    def cfl(self):
        v = ctypes.c_double()
        self._check(lib().crkfr_get_cfl(self.h, ctypes.byref(v)))
        return v.value

    def positions(self):
        """Coordinates of the solution points in the library's layout:
        1D x[elem, p]; 2D (x, y) each [ey, ex, q, p]."""
        xi, _ = self.nodes()
        if self.dim == 1:
            dx = (self.hi[0] - self.lo[0]) / self.n_elem[0]
            return self.lo[0] + (np.arange(self.n_elem[0])[:, None] + xi[None, :]) * dx
        Ex, Ey = self.n_elem
        dx = (self.hi[0] - self.lo[0]) / Ex
        dy = (self.hi[1] - self.lo[1]) / Ey
        x = self.lo[0] + (np.arange(Ex)[None, :, None, None] + xi[None, None, None, :]) * dx
        y = self.lo[1] + (np.arange(Ey)[:, None, None, None] + xi[None, None, :, None]) * dy
        return np.broadcast_arrays(x, y)

    def _dev(self, t, shape):
        import torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError("expected a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected contiguous float64 of shape {shape}, got "
                             f"{t.dtype} {tuple(t.shape)}")
        return ctypes.c_void_p(t.data_ptr())

    def set_coefficients(self, c):
        self._check(lib().crkfr_set_coefficients(self.h, self._dev(c, self.coef_shape), _stream()))

    # -- compute -----------------------------------------------------------------
    def compute_dt(self, u):
        v = ctypes.c_double()
        self._check(lib().crkfr_compute_dt(self.h, self._dev(u, self.shape), ctypes.byref(v),
                                           _stream()))
        return v.value

    def residual(self, u, dt, out=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        self._check(lib().crkfr_residual(self.h, self._dev(u, self.shape), float(dt),
                                         self._dev(out, self.shape), _stream()))
        return out

    def step(self, u, dt=0.0, nsteps=1):
        self._check(lib().crkfr_step(self.h, self._dev(u, self.shape), float(dt), int(nsteps),
                                     _stream()))
        return u

    def advance(self, u, t_end, max_steps=10 ** 7):
        k = ctypes.c_int64()
        self._check(lib().crkfr_advance(self.h, self._dev(u, self.shape), float(t_end),
                                        int(max_steps), ctypes.byref(k), _stream()))
        return k.value

    def step_host(self, u_in, u_out=None, dt=0.0, nsteps=1):
        """Steps a host (numpy float64, C-contiguous) state; the copies to and
        from the device happen inside the library call."""
        if u_in.dtype != np.float64 or not u_in.flags["C_CONTIGUOUS"] or u_in.shape != self.shape:
            raise ValueError("expected C-contiguous float64 host array of the state shape")
        if u_out is None:
            u_out = np.empty_like(u_in)
        self._check(lib().crkfr_step_host(self.h, u_in.ctypes.data_as(ctypes.c_void_p),
                                          u_out.ctypes.data_as(ctypes.c_void_p), float(dt),
                                          int(nsteps), _stream()))
        return u_out

    def adjoint_local(self, u, ubar1, dt):
        """2D slab, first phase of the adjoint step: forward traces of u and
        the correction sums of ubar1 the neighbouring slabs need."""
        self._check(lib().crkfr_adjoint_local(self.h, self._dev(u, self.shape),
                                              self._dev(ubar1, self.shape), float(dt), _stream()))

    def adjoint_halo_buffers(self):
        """2D slab: (send_bottom, send_top, recv_bottom, recv_top) of the
        adjoint's correction sums (after the first adjoint_local)."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        cnt = ctypes.c_int64()
        self._check(lib().crkfr_adjoint_halo_buffers(self.h, *[ctypes.byref(p) for p in ptrs],
                                                     ctypes.byref(cnt)))
        return tuple(torch.as_tensor(_DeviceBlock(p.value, cnt.value), device="cuda")
                     for p in ptrs)

    def adjoint_faces(self, u, ubar1, dt, ubar0=None, bbar=None):
        """2D slab, second phase (after both exchanges): ubar0 of the slab
        and its bathymetry gradient added to bbar.  Returns (ubar0, bbar)."""
        import torch
        if ubar0 is None:
            ubar0 = torch.empty_like(ubar1)
        if bbar is None:
            bbar = torch.zeros((self.n_elem[1], self.n_elem[0], self.n, self.n),
                               dtype=torch.float64, device=u.device)
        self._check(lib().crkfr_adjoint_faces(self.h, self._dev(u, self.shape),
                                              self._dev(ubar1, self.shape),
                                              self._dev(ubar0, self.shape),
                                              self._dev(bbar, (self.n_elem[1], self.n_elem[0],
                                                               self.n, self.n)),
                                              float(dt), _stream()))
        return ubar0, bbar

    def step_adjoint(self, u, ubar1, dt, ubar0=None, bbar=None):
        """ubar0 = (dS/du)^T ubar1; bbar += (dS/db)^T ubar1 for one 2D step of
        size dt from state u (crkfr_step_adjoint).  Returns (ubar0, bbar)."""
        import torch
        if ubar0 is None:
            ubar0 = torch.empty_like(ubar1)
        if bbar is None:
            bbar = torch.zeros(self.coef_shape, dtype=torch.float64, device=u.device)
        self._check(lib().crkfr_step_adjoint(self.h, self._dev(u, self.shape),
                                             self._dev(ubar1, self.shape),
                                             self._dev(ubar0, self.shape),
                                             self._dev(bbar, self.coef_shape), float(dt),
                                             _stream()))
        return ubar0, bbar

    def record_size(self):
        """Doubles of one step record (crkfr_record_size)."""
        n = ctypes.c_int64()
        self._check(lib().crkfr_record_size(self.h, ctypes.byref(n)))
        return n.value

    def new_records(self, count):
        """``count`` step records, one per row of a zeroed device array (a
        record leaves the two unused sides of the y-trace halo rows
        unwritten)."""
        import torch
        return torch.zeros((count, self.record_size()), dtype=torch.float64, device="cuda")

    def step_record(self, u, dt, record, advance=True):
        """One fixed step of u in place (advance) or none, writing the record
        of the step from the input state (crkfr_step_record)."""
        self._check(lib().crkfr_step_record(self.h, self._dev(u, self.shape), float(dt),
                                            self._dev(record, (self.record_size(),)),
                                            1 if advance else 0, _stream()))

    def step_adjoint_recorded(self, u, record, ubar1, dt, ubar0=None, bbar=None):
        """step_adjoint of the step from u whose record crkfr_step_record
        wrote (crkfr_step_adjoint_recorded).  Returns (ubar0, bbar)."""
        import torch
        if ubar0 is None:
            ubar0 = torch.empty_like(ubar1)
        if bbar is None:
            bbar = torch.zeros(self.coef_shape, dtype=torch.float64, device=u.device)
        self._check(lib().crkfr_step_adjoint_recorded(
            self.h, self._dev(u, self.shape), self._dev(record, (self.record_size(),)),
            self._dev(ubar1, self.shape), self._dev(ubar0, self.shape),
            self._dev(bbar, self.coef_shape), float(dt), _stream()))
        return ubar0, bbar

    def step_local_record(self, u, dt, record, advance=True):
        """2D slab: local phase of a recorded step (crkfr_step_local_record)."""
        self._check(lib().crkfr_step_local_record(self.h, self._dev(u, self.shape), float(dt),
                                                  self._dev(record, (self.record_size(),)),
                                                  1 if advance else 0, _stream()))

    def record_halo_buffers(self, record):
        """2D slab: the boundary blocks of a record's y traces to exchange,
        (send_bottom, send_top, recv_bottom, recv_top) viewing the record."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        cnt = ctypes.c_int64()
        self._check(lib().crkfr_record_halo_buffers(
            self.h, self._dev(record, (self.record_size(),)), *[ctypes.byref(p) for p in ptrs],
            ctypes.byref(cnt)))
        return tuple(torch.as_tensor(_DeviceBlock(p.value, cnt.value), device="cuda")
                     for p in ptrs)

    def step_faces_record(self, u, record):
        """2D slab: face phase of a recorded step (crkfr_step_faces_record)."""
        self._check(lib().crkfr_step_faces_record(self.h, self._dev(u, self.shape),
                                                  self._dev(record, (self.record_size(),)),
                                                  _stream()))

    def adjoint_sums(self, ubar1):
        """2D slab: the correction sums of ubar1 of a recorded adjoint step."""
        self._check(lib().crkfr_adjoint_sums(self.h, self._dev(ubar1, self.shape), _stream()))

    def adjoint_faces_recorded(self, u, record, ubar1, dt, ubar0=None, bbar=None):
        """2D slab: the recorded adjoint step after the exchange of the sums.
        Returns (ubar0, bbar)."""
        import torch
        if ubar0 is None:
            ubar0 = torch.empty_like(ubar1)
        bshape = (self.n_elem[1], self.n_elem[0], self.n, self.n)
        if bbar is None:
            bbar = torch.zeros(bshape, dtype=torch.float64, device=u.device)
        self._check(lib().crkfr_adjoint_faces_recorded(
            self.h, self._dev(u, self.shape), self._dev(record, (self.record_size(),)),
            self._dev(ubar1, self.shape), self._dev(ubar0, self.shape), self._dev(bbar, bshape),
            float(dt), _stream()))
        return ubar0, bbar

    def time(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        self._check(lib().crkfr_get_time(self.h, ctypes.byref(t), ctypes.byref(dt), _stream()))
        return t.value, dt.value

    def set_time(self, t):
        self._check(lib().crkfr_set_time(self.h, float(t), _stream()))

    def state_dict(self, u):
        """Checkpoint of a run: the state (a copy), the simulated time and
        the configuration it belongs to (including the limiter setting).  The
        CFL step and the limiter's coefficients are recomputed from the state
        at every call, so resuming from a checkpoint repeats the run."""
        t, dt_last = self.time()
        return {"u": u.detach().clone(), "t": t, "dt_last": dt_last, "system": self.system,
                "degree": self.degree, "nodes": self.family, "n_elem": list(self.n_elem),
                "lo": list(self.lo), "hi": list(self.hi), "source": self.source,
                "source_coef": self.source_coef, "limiter": list(self.limiter)}

    def load_state_dict(self, sd, u):
        """Restore a checkpoint into the device tensor u and the context's
        time; the context must hold the same system, degree, nodes and mesh
        (and coefficients)."""
        for k in ("system", "degree", "nodes"):
            want = {"system": self.system, "degree": self.degree, "nodes": self.family}[k]
            if sd[k] != want:
                raise ValueError(f"checkpoint {k} {sd[k]!r} differs from {want!r}")
        if list(sd["n_elem"]) != list(self.n_elem):
            raise ValueError("checkpoint mesh differs")
        mode, alpha = sd.get("limiter", (None, 0.0))
        if (mode, float(alpha)) != self.limiter:
            self.set_limiter(mode, alpha)
        u.copy_(sd["u"])
        self.set_time(sd["t"])
        return u

    def status(self):
        """Raises CrkfrError(CRKFR_ERR_NONPHYSICAL) if a non-physical state was
        produced since the last call."""
        self._check(lib().crkfr_get_status(self.h, _stream()))

    def launch_count(self):
        return lib().crkfr_launch_count(self.h)

    KERNELS = {"step_1d": 0, "local_2d": 1, "face_2d": 2, "rate": 3, "coef": 4, "adjoint_2d": 5,
               "indicator": 6}
    LIMITERS = {None: 0, "blend": 1, "fixed": 2}

    def set_limiter(self, mode="blend", alpha=0.0):
        """Subcell blending limiter of the step (1D, or 2D on a whole periodic
        mesh): 'blend' (smoothness indicator), 'fixed' (alpha for every
        element) or None (off)."""
        self._check(lib().crkfr_set_limiter(self.h, self.LIMITERS[mode], float(alpha)))
        self.limiter = (mode, float(alpha))

    def set_tile_1d(self, threads=0):
        """Threads per block of the 1D step: 0 chooses per mesh, 64, 96 or 128
        fixes it (the results do not change)."""
        self._check(lib().crkfr_set_tile_1d(self.h, int(threads)))

    def limiter_alpha(self):
        """alpha_e of the last limited step (cuda float64 tensor: (E,) in 1D,
        (Ey, Ex) in 2D)."""
        import torch
        shape = tuple(reversed(self.n_elem))
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        self._check(lib().crkfr_limiter_alpha(self.h, ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def profile(self, enable=True):
        """Start (clearing earlier values) or stop per-kernel event timing."""
        self._check(lib().crkfr_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel: (launches, total ms)} since profiling was enabled."""
        out = {}
        for name, k in self.KERNELS.items():
            n, ms = ctypes.c_int64(), ctypes.c_double()
            self._check(lib().crkfr_profile_read(self.h, k, ctypes.byref(n), ctypes.byref(ms)))
            if n.value:
                out[name] = (n.value, ms.value)
        return out


class Batch:
    """Ragged ensemble of independent 1D meshes advanced together
    (crkfr_batch_*).  ``members``: list of (degree, n_elem, lo, hi)."""

    def __init__(self, system, members, nodes="gl", gravity=9.81, cfl_safety=0.5, cfl_number=0.0,
                 source=None, source_coef=0.0, rk=0, nc_face="frozen", coef_dissipation=False):
        self.system = system
        self.M = NVARS[system]
        self.members = [(int(d), int(e), float(a), float(b)) for d, e, a, b in members]
        n = len(self.members)
        cfg = make_config(system, 0, nodes, gravity, cfl_safety, cfl_number, source, source_coef,
                          rk, nc_face, coef_dissipation)
        deg = (ctypes.c_int32 * n)(*[m[0] for m in self.members])
        ne = (ctypes.c_int64 * n)(*[m[1] for m in self.members])
        lo = (ctypes.c_double * n)(*[m[2] for m in self.members])
        hi = (ctypes.c_double * n)(*[m[3] for m in self.members])
        h = ctypes.c_void_p()
        st = lib().crkfr_batch_create(ctypes.byref(h), ctypes.byref(cfg), n, deg, ne, lo, hi)
        if st != CRKFR_OK:
            raise CrkfrError(st, lib().crkfr_last_error(None).decode() or
                             lib().crkfr_error_string(st).decode())
        self.h = h
        so, co = (ctypes.c_int64 * (n + 1))(), (ctypes.c_int64 * (n + 1))()
        self._check(lib().crkfr_batch_layout(self.h, so, co))
        self.state_offsets, self.coef_offsets = list(so), list(co)

    def _check(self, st):
        if st != CRKFR_OK:
            raise CrkfrError(st, lib().crkfr_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().crkfr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state_view(self, u, i):
        """Instance i's state (var, elem, node) as a view of the packed u."""
        d, E, _, _ = self.members[i]
        a, b = self.state_offsets[i], self.state_offsets[i + 1]
        return u[a:b].view(self.M, E, d + 1)

    def coef_view(self, c, i):
        d, E, _, _ = self.members[i]
        a, b = self.coef_offsets[i], self.coef_offsets[i + 1]
        return c[a:b].view(E, d + 1)

    def set_coefficients(self, c):
        self._check(lib().crkfr_batch_set_coefficients(self.h, ctypes.c_void_p(c.data_ptr()),
                                                       _stream()))

    def step(self, u, dt=0.0, nsteps=1, graph=True):
        self._check(lib().crkfr_batch_step(self.h, ctypes.c_void_p(u.data_ptr()), float(dt),
                                           int(nsteps), 1 if graph else 0, _stream()))
        return u

    def set_tuning(self, tiles_per_block=1, order=0, parallel=False):
        """Launch shape of a step (never changes the result)."""
        self._check(lib().crkfr_batch_set_tuning(self.h, int(tiles_per_block), int(order),
                                                 1 if parallel else 0))

    def tuning(self):
        """(tiles_per_block, order, parallel, ms per step of the tuned shape)."""
        t, o, p, ms = _I32(), _I32(), _I32(), ctypes.c_double()
        self._check(lib().crkfr_batch_get_tuning(self.h, ctypes.byref(t), ctypes.byref(o),
                                                 ctypes.byref(p), ctypes.byref(ms)))
        return t.value, o.value, bool(p.value), ms.value

    def autotune(self, u, steps=3):
        """Time the launch shapes on a scratch copy of u and keep the fastest."""
        self._check(lib().crkfr_batch_autotune(self.h, ctypes.c_void_p(u.data_ptr()), int(steps),
                                               _stream()))
        return self.tuning()

    def times(self):
        t = (ctypes.c_double * len(self.members))()
        self._check(lib().crkfr_batch_get_times(self.h, t, _stream()))
        return np.array(t[:])

    def status(self):
        self._check(lib().crkfr_batch_get_status(self.h, _stream()))

    def launch_count(self):
        return lib().crkfr_batch_launch_count(self.h)

    def profile(self, enable=True):
        """Time every step kernel of calls without a graph (crkfr_batch_profile_*)."""
        self._check(lib().crkfr_batch_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """(timed launches, summed kernel ms) since profiling was enabled."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(lib().crkfr_batch_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value
