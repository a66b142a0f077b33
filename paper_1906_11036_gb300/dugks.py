"""Thin Python binding of the C ABI in ``include/dugks.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library.  PyTorch provides device memory (phi and state tensors) and the
stream.  If the library is missing the import fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs
from .build import LIB

OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid configuration", 3: "CUDA error",
          4: "non-finite value in phi", 5: "unsupported", 6: "out of memory", 7: "device wait timed out"}
KERNELS = {"auto": 0, "fused": 1, "naive": 2}


class DugksError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("xf", ctypes.POINTER(ctypes.c_double)), ("yf", ctypes.POINTER(ctypes.c_double)),
                ("bc", ctypes.c_int * 4), ("bc_value", ctypes.c_double * 4)]


class VSet(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c", ctypes.c_double)]


class Coef(ctypes.Structure):
    _fields_ = [("u", ctypes.c_double * 2), ("nb", ctypes.c_int), ("b", ctypes.c_double * 8),
                ("alpha", ctypes.c_double), ("nd", ctypes.c_int), ("d", ctypes.c_double * 8),
                ("c_zero", ctypes.c_int), ("d_tensor", ctypes.c_int), ("ndt", ctypes.c_int),
                ("dxx", ctypes.c_double * 8), ("dxy", ctypes.c_double * 8), ("dyy", ctypes.c_double * 8)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("kernel", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("pitch", ctypes.c_longlong), ("steps_done", ctypes.c_longlong), ("dt", ctypes.c_double),
                ("lam", ctypes.c_double), ("cfl", ctypes.c_double), ("block_threads", ctypes.c_int),
                ("grid_blocks", ctypes.c_int), ("state_bytes", ctypes.c_longlong), ("time", ctypes.c_double),
                ("nsrc", ctypes.c_int)]


class Mesh3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("xf", ctypes.POINTER(ctypes.c_double)), ("yf", ctypes.POINTER(ctypes.c_double)),
                ("zf", ctypes.POINTER(ctypes.c_double)), ("bc", ctypes.c_int * 6), ("bc_value", ctypes.c_double * 6)]


class VSet3(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("c", ctypes.c_double)]


class Coef3(ctypes.Structure):
    _fields_ = [("u", ctypes.c_double * 3), ("nb", ctypes.c_int), ("b", ctypes.c_double * 8),
                ("alpha", ctypes.c_double), ("nd", ctypes.c_int), ("d", ctypes.c_double * 8), ("c_zero", ctypes.c_int)]


class Info3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("q", ctypes.c_int),
                ("precision", ctypes.c_int), ("steps_done", ctypes.c_longlong), ("dt", ctypes.c_double),
                ("lam", ctypes.c_double), ("cfl", ctypes.c_double), ("block_threads", ctypes.c_int),
                ("grid", ctypes.c_int * 3), ("zseg", ctypes.c_int), ("state_bytes", ctypes.c_longlong)]


_lib = None


def library():
    """Load ``libdugks.so`` (build it with ``paper_1906_11036_gb300.build.build()`` first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"CUDA library not built: {LIB} (run paper_1906_11036_gb300.build.build())")
        L = ctypes.CDLL(LIB)
        vp, P = ctypes.c_void_p, ctypes.POINTER
        L.dugks_check_config.argtypes = [P(Mesh), P(VSet), P(Coef), ctypes.c_double]
        L.dugks_check_feq.argtypes = [P(VSet), P(Coef), ctypes.c_double, ctypes.c_double, P(ctypes.c_double)]
        L.dugks_create.argtypes = [P(Mesh), P(VSet), P(Coef), ctypes.c_double, P(Options), P(vp)]
        L.dugks_destroy.argtypes = [vp]
        L.dugks_init_phi.argtypes = [vp, vp]
        L.dugks_init_phi_host.argtypes = [vp, P(ctypes.c_double)]
        L.dugks_step.argtypes = [vp, ctypes.c_longlong]
        L.dugks_get_phi.argtypes = [vp, vp, P(ctypes.c_double)]
        L.dugks_get_phi_host.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double)]
        L.dugks_save_state.argtypes = [vp, vp]
        L.dugks_load_state.argtypes = [vp, vp]
        L.dugks_set_stream.argtypes = [vp, vp]
        L.dugks_sync.argtypes = [vp]
        L.dugks_wait_timeout_check.argtypes = [vp, ctypes.c_int]
        L.dugks_set_adjoint_kernel.argtypes = [vp, ctypes.c_int]
        L.dugks_set_feq_check.argtypes = [vp, ctypes.c_int]
        L.dugks_info.argtypes = [vp, P(Info)]
        L.dugks_adjoint_step.argtypes = [vp, vp, vp, vp, vp, vp]
        L.dugks_set_source.argtypes = [vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int), vp, ctypes.c_double]
        L.dugks_adjoint.argtypes = [vp, vp, ctypes.c_longlong, ctypes.c_int, vp, vp, P(ctypes.c_double),
                                    P(ctypes.c_double)]
        L.dugks_phi_mass_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
        L.dugks_batch_create.argtypes = [ctypes.c_int, P(Mesh), P(VSet), P(Coef), P(ctypes.c_double), P(Options),
                                         P(vp)]
        L.dugks_batch_destroy.argtypes = [vp]
        L.dugks_batch_init_phi.argtypes = [vp, ctypes.c_int, vp]
        L.dugks_batch_step.argtypes = [vp, ctypes.c_longlong]
        L.dugks_batch_get_phi.argtypes = [vp, ctypes.c_int, vp, P(ctypes.c_double)]
        L.dugks_batch_save_state.argtypes = [vp, ctypes.c_int, vp]
        L.dugks_batch_sync.argtypes = [vp]
        L.dugks_batch_autotune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_float)]
        L.dugks_batch_last_error.argtypes = [vp]
        L.dugks_batch_last_error.restype = ctypes.c_char_p
        P3 = P
        L.dugks_3d_check_config.argtypes = [P3(Mesh3), P3(VSet3), P3(Coef3), ctypes.c_double]
        L.dugks_3d_create.argtypes = [P3(Mesh3), P3(VSet3), P3(Coef3), ctypes.c_double, P(Options), P(vp)]
        L.dugks_3d_destroy.argtypes = [vp]
        L.dugks_3d_init_phi.argtypes = [vp, vp]
        L.dugks_3d_step.argtypes = [vp, ctypes.c_longlong]
        L.dugks_3d_get_phi.argtypes = [vp, vp, P(ctypes.c_double)]
        L.dugks_3d_save_state.argtypes = [vp, vp]
        L.dugks_3d_load_state.argtypes = [vp, vp]
        L.dugks_3d_sync.argtypes = [vp]
        L.dugks_3d_info.argtypes = [vp, P(Info3)]
        L.dugks_3d_last_error.argtypes = [vp]
        L.dugks_3d_last_error.restype = ctypes.c_char_p
        for name in ("dugks_3d_check_config", "dugks_3d_create", "dugks_3d_destroy", "dugks_3d_init_phi",
                     "dugks_3d_step", "dugks_3d_get_phi", "dugks_3d_save_state", "dugks_3d_load_state",
                     "dugks_3d_sync", "dugks_3d_info"):
            getattr(L, name).restype = ctypes.c_int
        L.dugks_status_string.argtypes = [ctypes.c_int]
        L.dugks_status_string.restype = ctypes.c_char_p
        L.dugks_last_error.argtypes = [vp]
        L.dugks_last_error.restype = ctypes.c_char_p
        for name in ("dugks_check_config", "dugks_create", "dugks_destroy", "dugks_init_phi", "dugks_init_phi_host",
                     "dugks_step", "dugks_get_phi", "dugks_get_phi_host", "dugks_save_state", "dugks_load_state",
                     "dugks_set_stream", "dugks_sync", "dugks_wait_timeout_check", "dugks_info",
                     "dugks_adjoint_step", "dugks_adjoint",
                     "dugks_set_source",
                     "dugks_phi_mass_noalloc", "dugks_batch_create", "dugks_batch_destroy", "dugks_batch_init_phi",
                     "dugks_batch_step", "dugks_batch_get_phi", "dugks_batch_save_state", "dugks_batch_sync",
                     "dugks_batch_autotune"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def marshal(problem: inputs.Problem):
    """Problem -> (Mesh, VSet, Coef, keepalive arrays)."""
    xf = np.ascontiguousarray(problem.xf, dtype=np.float64)
    yf = np.ascontiguousarray(problem.yf, dtype=np.float64)
    m = Mesh()
    m.nx, m.ny = len(xf) - 1, len(yf) - 1
    m.xf, m.yf = _dptr(xf), _dptr(yf)
    for i in range(4):
        m.bc[i] = int(problem.bc[i])
        m.bc_value[i] = float(problem.bc_value[i])
    v = VSet()
    v.kind, v.c = 9, float(problem.c)
    c = Coef()
    c.u[0], c.u[1] = float(problem.u[0]), float(problem.u[1])
    if len(problem.b) > 8 or len(problem.d) > 8:
        raise ValueError("at most 8 polynomial coefficients")
    c.nb = len(problem.b)
    for k, x in enumerate(problem.b):
        c.b[k] = float(x)
    c.alpha = float(problem.alpha)
    c.nd = len(problem.d)
    for k, x in enumerate(problem.d):
        c.d[k] = float(x)
    c.c_zero = int(bool(problem.c_zero))
    if problem.d_tensor is not None:
        dt3 = [tuple(map(float, x)) for x in problem.d_tensor]
        if len(dt3) != 3 or max(len(x) for x in dt3) > 8:
            raise ValueError("d_tensor = (dxx, dxy, dyy), at most 8 coefficients each")
        c.d_tensor, c.ndt = 1, max(len(x) for x in dt3)
        for arr, x in zip((c.dxx, c.dxy, c.dyy), dt3):
            for k, val in enumerate(x):
                arr[k] = val
    return m, v, c, (xf, yf)


def check_config(problem: inputs.Problem) -> int:
    """Host-only validation (no CUDA call); returns the status code."""
    m, v, c, keep = marshal(problem)
    return int(library().dugks_check_config(ctypes.byref(m), ctypes.byref(v), ctypes.byref(c), float(problem.dt)))


def check_feq(problem: inputs.Problem, phi_min: float, phi_max: float) -> tuple[int, float]:
    """Host-only positivity test of the equilibrium over [phi_min, phi_max]:
    (status, smallest f^eq)."""
    m, v, c, keep = marshal(problem)
    out = ctypes.c_double(0.0)
    st = library().dugks_check_feq(ctypes.byref(v), ctypes.byref(c), float(phi_min), float(phi_max), ctypes.byref(out))
    return int(st), float(out.value)


class Solver:
    """One NCDE instance advanced by the CUDA DUGKS step."""

    def __init__(self, problem: inputs.Problem, precision: int = 32, kernel: str = "auto", stream=None,
                 device: int | None = None):
        import torch

        self.torch = torch
        self.problem = problem
        self.precision = int(precision)
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        L = library()
        m, v, c, keep = marshal(problem)
        o = Options()
        o.precision = self.precision
        o.kernel = KERNELS[kernel]
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        o.device = self.device.index
        h = ctypes.c_void_p()
        st = L.dugks_create(ctypes.byref(m), ctypes.byref(v), ctypes.byref(c), float(problem.dt), ctypes.byref(o),
                            ctypes.byref(h))
        if st != OK:
            raise DugksError(st, "dugks_create")
        self.h = h
        self.L = L
        self.nx, self.ny = m.nx, m.ny
        if problem.source:
            self.set_source(problem.source, problem.t0)

    # -- helpers --------------------------------------------------------------
    def _check(self, st, where):
        if st != OK:
            raise DugksError(st, where, self.L.dugks_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.dugks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API ------------------------------------------------------------------
    def init_phi(self, phi0):
        """phi0: CUDA tensor [ny, nx] (converted to the solver's dtype) or a numpy array (host path)."""
        if isinstance(phi0, np.ndarray):
            a = np.ascontiguousarray(phi0, dtype=np.float64)
            assert a.shape == (self.ny, self.nx)
            self._check(self.L.dugks_init_phi_host(self.h, _dptr(a)), "dugks_init_phi_host")
            return
        t = phi0.to(device=self.device, dtype=self.dtype).contiguous()
        assert tuple(t.shape) == (self.ny, self.nx)
        self._keep = t
        self._check(self.L.dugks_init_phi(self.h, ctypes.c_void_p(t.data_ptr())), "dugks_init_phi")

    def step(self, n: int = 1):
        self._check(self.L.dugks_step(self.h, int(n)), "dugks_step")

    def set_source(self, terms, t0: float = 0.0):
        """Source F = sum_k exp(rate_k t) phi^power_k S_k(x) (inputs.SourceTerm list; empty removes it)."""
        terms = tuple(terms)
        n = len(terms)
        rate = (ctypes.c_double * max(n, 1))(*[float(t.rate) for t in terms])
        power = (ctypes.c_int * max(n, 1))(*[int(t.power) for t in terms])
        fields = None
        if n:
            fields = self.torch.tensor(np.stack([np.asarray(t.field, dtype=np.float64) for t in terms]),
                                       dtype=self.dtype, device=self.device).contiguous()
            assert tuple(fields.shape) == (n, self.ny, self.nx)
            self.torch.cuda.current_stream(self.device).synchronize()  # the fields are on the device before the copy
        self._check(self.L.dugks_set_source(self.h, n, rate, power,
                                            ctypes.c_void_p(fields.data_ptr()) if n else None, float(t0)),
                    "dugks_set_source")
        self._src_keep = fields  # the library copies on its stream; keep until that copy ran

    def get_phi(self, out=None, mass: bool = False):
        """phi as a CUDA tensor [ny, nx]; with mass=True also returns M (synchronises)."""
        if out is None:
            out = self.torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        m = ctypes.c_double(0.0)
        self._check(self.L.dugks_get_phi(self.h, ctypes.c_void_p(out.data_ptr()), ctypes.byref(m) if mass else None),
                    "dugks_get_phi")
        return (out, m.value) if mass else out

    def get_phi_host(self, out: np.ndarray | None = None):
        """(phi as float64 numpy [ny, nx], mass); synchronises."""
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=np.float64)
        m = ctypes.c_double(0.0)
        self._check(self.L.dugks_get_phi_host(self.h, _dptr(out), ctypes.byref(m)), "dugks_get_phi_host")
        return out, m.value

    def mass(self) -> float:
        m = ctypes.c_double(0.0)
        self._check(self.L.dugks_get_phi(self.h, None, ctypes.byref(m)), "dugks_get_phi")
        return m.value

    def save_state(self, out=None):
        if out is None:
            out = self.torch.empty((9, self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(self.L.dugks_save_state(self.h, ctypes.c_void_p(out.data_ptr())), "dugks_save_state")
        return out

    def load_state(self, f):
        t = f.to(device=self.device, dtype=self.dtype).contiguous()
        assert tuple(t.shape) == (9, self.ny, self.nx)
        self._keep_state = t
        self._check(self.L.dugks_load_state(self.h, ctypes.c_void_p(t.data_ptr())), "dugks_load_state")

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.L.dugks_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "dugks_set_stream")

    def sync(self):
        self._check(self.L.dugks_sync(self.h), "dugks_sync")

    def wait_timeout_check(self, limit_us: int = 2000):
        """Let one bounded device wait expire on purpose (no fault): the next sync raises DUGKS_ERR_TIMEOUT."""
        self._check(self.L.dugks_wait_timeout_check(self.h, int(limit_us)), "dugks_wait_timeout_check")

    def set_feq_check(self, on: bool = True):
        """Later initialisations reject a negative equilibrium of phi0 (see dugks_check_feq)."""
        self._check(self.L.dugks_set_feq_check(self.h, 1 if on else 0), "dugks_set_feq_check")

    ADJ_KERNELS = {"auto": 0, "tiled": 1, "rows": 2}

    def set_adjoint_kernel(self, kind: str):
        """Which kernel runs an FP32 adjoint step: "auto", "tiled" or "rows" (cross-check hook)."""
        self._check(self.L.dugks_set_adjoint_kernel(self.h, self.ADJ_KERNELS[kind]), "dugks_set_adjoint_kernel")

    def adjoint_step(self, f, mu, dj_dalpha=None, dj_du=None, with_u=False, with_alpha=True):
        """lam = (d f^{n+1}/d f^n)^T mu at state f (CUDA tensors [9, ny, nx]); the
        explicit alpha-derivative is accumulated into dj_dalpha (a CUDA float64
        tensor of one element, created if None).  Returns (lam, dj_dalpha); with
        with_u (or dj_du given: a CUDA float64 tensor of two elements) the explicit
        u-derivative is accumulated too and (lam, dj_dalpha, dj_du) is returned.
        with_alpha=False: lam only (returned as (lam, None))."""
        t = self.torch
        f = f.to(device=self.device, dtype=self.dtype).contiguous()
        mu = mu.to(device=self.device, dtype=self.dtype).contiguous()
        lam = t.empty_like(f)
        if not with_alpha:
            self._check(self.L.dugks_adjoint_step(self.h, ctypes.c_void_p(f.data_ptr()),
                                                  ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                                  None, None), "dugks_adjoint_step")
            return lam, None
        if dj_dalpha is None:
            dj_dalpha = t.zeros(1, dtype=t.float64, device=self.device)
        with_u = with_u or dj_du is not None
        if with_u and dj_du is None:
            dj_du = t.zeros(2, dtype=t.float64, device=self.device)
        du_ptr = ctypes.c_void_p(dj_du.data_ptr()) if with_u else None
        self._check(self.L.dugks_adjoint_step(self.h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(mu.data_ptr()),
                                              ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(dj_dalpha.data_ptr()),
                                              du_ptr), "dugks_adjoint_step")
        return (lam, dj_dalpha, dj_du) if with_u else (lam, dj_dalpha)

    def gradient(self, phi0, nsteps: int, grad_phiN, checkpoint_every: int = 20, with_u: bool = False):
        """(dJ/dphi0, dJ/dalpha) through nsteps steps, given dJ/dphi^N (checkpointed
        reverse sweep in the library); with_u: (dJ/dphi0, dJ/dalpha, (dJ/du_x,
        dJ/du_y)).  Leaves the solver's state at an intermediate step."""
        t = self.torch
        phi0 = phi0.to(device=self.device, dtype=self.dtype).contiguous()
        g = grad_phiN.to(device=self.device, dtype=self.dtype).contiguous()
        out = t.empty_like(phi0)
        da = ctypes.c_double(0.0)
        du = (ctypes.c_double * 2)(0.0, 0.0)
        self._check(self.L.dugks_adjoint(self.h, ctypes.c_void_p(phi0.data_ptr()), int(nsteps), int(checkpoint_every),
                                         ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.byref(da),
                                         ctypes.cast(du, ctypes.POINTER(ctypes.c_double)) if with_u else None),
                    "dugks_adjoint")
        return (out, da.value, (du[0], du[1])) if with_u else (out, da.value)

    def info(self) -> dict:
        i = Info()
        self._check(self.L.dugks_info(self.h, ctypes.byref(i)), "dugks_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}


class BatchSolver:
    """Many independent instances (list of inputs.Problem) advanced together in
    single precision by the batched persistent step."""

    def __init__(self, problems, stream=None, device: int | None = None):
        import torch

        self.torch = torch
        self.problems = list(problems)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        n = len(self.problems)
        L = library()
        meshes, vsets, coefs = (Mesh * n)(), (VSet * n)(), (Coef * n)()
        self._keep = []
        for i, p in enumerate(self.problems):
            m, v, c, keep = marshal(p)
            meshes[i], vsets[i], coefs[i] = m, v, c
            self._keep.append(keep)
        dts = (ctypes.c_double * n)(*[float(p.dt) for p in self.problems])
        o = Options()
        o.precision, o.kernel = 32, KERNELS["fused"]
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        o.device = self.device.index
        h = ctypes.c_void_p()
        st = L.dugks_batch_create(n, meshes, vsets, coefs, dts, ctypes.byref(o), ctypes.byref(h))
        if st != OK:
            raise DugksError(st, "dugks_batch_create")
        self.h, self.L, self.n = h, L, n

    def _check(self, st, where):
        if st != OK:
            raise DugksError(st, where, self.L.dugks_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.dugks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_phi(self, i: int, phi0):
        p = self.problems[i]
        t = self.torch.as_tensor(phi0).to(device=self.device, dtype=self.torch.float32).contiguous()
        assert tuple(t.shape) == (p.ny, p.nx)
        self._check(self.L.dugks_batch_init_phi(self.h, int(i), ctypes.c_void_p(t.data_ptr())), "dugks_batch_init_phi")
        self.sync()

    def step(self, n: int = 1):
        self._check(self.L.dugks_batch_step(self.h, int(n)), "dugks_batch_step")

    def get_phi(self, i: int, mass: bool = False):
        p = self.problems[i]
        out = self.torch.empty((p.ny, p.nx), dtype=self.torch.float32, device=self.device)
        m = ctypes.c_double(0.0)
        self._check(self.L.dugks_batch_get_phi(self.h, int(i), ctypes.c_void_p(out.data_ptr()),
                                               ctypes.byref(m) if mass else None), "dugks_batch_get_phi")
        return (out, m.value) if mass else out

    def save_state(self, i: int):
        p = self.problems[i]
        out = self.torch.empty((9, p.ny, p.nx), dtype=self.torch.float32, device=self.device)
        self._check(self.L.dugks_batch_save_state(self.h, int(i), ctypes.c_void_p(out.data_ptr())),
                    "dugks_batch_save_state")
        return out

    def sync(self):
        self._check(self.L.dugks_batch_sync(self.h), "dugks_batch_sync")

    def autotune(self, steps_per_trial: int = 20):
        rows, ms = ctypes.c_int(0), ctypes.c_float(0.0)
        self._check(self.L.dugks_batch_autotune(self.h, int(steps_per_trial), ctypes.byref(rows), ctypes.byref(ms)),
                    "dugks_batch_autotune")
        return rows.value, ms.value


def run_fn():
    """A torch.autograd.Function over the whole run: phiN = run(phi0, alpha).

    forward(phi0, alpha, solver, nsteps, checkpoint_every) advances the solver
    (created with that alpha) from phi0; backward runs the library's
    checkpointed adjoint and returns dJ/dphi0 and dJ/dalpha.  alpha is a
    one-element tensor that must equal the solver's diffusion coefficient;
    it is an input only so that its gradient can be returned.
    """
    import torch

    class DugksRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi0, alpha, solver, nsteps, checkpoint_every):
            if abs(float(alpha) - float(solver.problem.alpha)) > 1e-12 * abs(float(solver.problem.alpha)):
                raise ValueError("alpha does not match the solver's diffusion coefficient")
            solver.init_phi(phi0.detach())
            solver.step(nsteps)
            ctx.solver, ctx.nsteps, ctx.k = solver, int(nsteps), int(checkpoint_every)
            ctx.save_for_backward(phi0.detach())
            return solver.get_phi().to(phi0.dtype)

        @staticmethod
        def backward(ctx, grad_phiN):
            (phi0,) = ctx.saved_tensors
            gphi0, galpha = ctx.solver.gradient(phi0, ctx.nsteps, grad_phiN, ctx.k)
            return (gphi0.to(phi0.dtype), torch.tensor([galpha], dtype=torch.float64, device=phi0.device),
                    None, None, None)

    return DugksRun



def marshal3(problem):
    """inputs.Problem3 -> (Mesh3, VSet3, Coef3, keepalive arrays)."""
    f = [np.ascontiguousarray(a, dtype=np.float64) for a in (problem.xf, problem.yf, problem.zf)]
    m = Mesh3()
    m.nx, m.ny, m.nz = (len(a) - 1 for a in f)
    m.xf, m.yf, m.zf = (_dptr(a) for a in f)
    for i in range(6):
        m.bc[i] = int(problem.bc[i])
        m.bc_value[i] = float(problem.bc_value[i])
    v = VSet3()
    v.kind, v.c = int(problem.lattice), float(problem.c)
    c = Coef3()
    for a in range(3):
        c.u[a] = float(problem.u[a])
    if len(problem.b) > 8 or len(problem.d) > 8:
        raise ValueError("at most 8 polynomial coefficients")
    c.nb = len(problem.b)
    for k, x in enumerate(problem.b):
        c.b[k] = float(x)
    c.alpha = float(problem.alpha)
    c.nd = len(problem.d)
    for k, x in enumerate(problem.d):
        c.d[k] = float(x)
    c.c_zero = int(bool(problem.c_zero))
    return m, v, c, f


class Solver3:
    """One 3-D NCDE instance (inputs.Problem3, D3Q15 or D3Q19) advanced by the CUDA step."""

    def __init__(self, problem, precision: int = 32, stream=None, device: int | None = None):
        import torch

        self.torch = torch
        self.problem = problem
        self.precision = int(precision)
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        L = library()
        m, v, c, keep = marshal3(problem)
        o = Options()
        o.precision, o.kernel = self.precision, KERNELS["fused"]
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        o.device = self.device.index
        h = ctypes.c_void_p()
        st = L.dugks_3d_create(ctypes.byref(m), ctypes.byref(v), ctypes.byref(c), float(problem.dt), ctypes.byref(o),
                               ctypes.byref(h))
        if st != OK:
            raise DugksError(st, "dugks_3d_create")
        self.h, self.L = h, L
        self.nx, self.ny, self.nz, self.Q = m.nx, m.ny, m.nz, v.kind

    def _check(self, st, where):
        if st != OK:
            raise DugksError(st, where, self.L.dugks_3d_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.dugks_3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_phi(self, phi0):
        """phi0: tensor or array [nz, ny, nx]."""
        t = self.torch.as_tensor(phi0).to(device=self.device, dtype=self.dtype).contiguous()
        assert tuple(t.shape) == (self.nz, self.ny, self.nx)
        self._keep = t
        self._check(self.L.dugks_3d_init_phi(self.h, ctypes.c_void_p(t.data_ptr())), "dugks_3d_init_phi")

    def step(self, n: int = 1):
        self._check(self.L.dugks_3d_step(self.h, int(n)), "dugks_3d_step")

    def get_phi(self, mass: bool = False):
        out = self.torch.empty((self.nz, self.ny, self.nx), dtype=self.dtype, device=self.device)
        m = ctypes.c_double(0.0)
        self._check(self.L.dugks_3d_get_phi(self.h, ctypes.c_void_p(out.data_ptr()), ctypes.byref(m) if mass else None),
                    "dugks_3d_get_phi")
        return (out, m.value) if mass else out

    def save_state(self):
        out = self.torch.empty((self.Q, self.nz, self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(self.L.dugks_3d_save_state(self.h, ctypes.c_void_p(out.data_ptr())), "dugks_3d_save_state")
        return out

    def load_state(self, f):
        t = f.to(device=self.device, dtype=self.dtype).contiguous()
        assert tuple(t.shape) == (self.Q, self.nz, self.ny, self.nx)
        self._keep_state = t
        self._check(self.L.dugks_3d_load_state(self.h, ctypes.c_void_p(t.data_ptr())), "dugks_3d_load_state")

    def sync(self):
        self._check(self.L.dugks_3d_sync(self.h), "dugks_3d_sync")

    def info(self) -> dict:
        i = Info3()
        self._check(self.L.dugks_3d_info(self.h, ctypes.byref(i)), "dugks_3d_info")
        out = {f: getattr(i, f) for f, _ in Info3._fields_}
        out["grid"] = tuple(i.grid)
        return out
