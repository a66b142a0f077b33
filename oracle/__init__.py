"""FP64 CPU oracle of the DUGKS step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``dugks_oracle.c`` (plain C,
built with gcc, ``-O2 -ffp-contract=off``, OpenMP over rows) through ctypes
and shares no code with the CUDA library.

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):
  equilibrium           moment identities of Eq. 2.7 (quadrature for C)
  cell_transforms       Eqs. 2.11, 2.13, 2.15, 2.17 composed independently
  face_original         Eq. 2.22 derived from Eqs. 2.15 / 2.11
  step / run            exact rational stepper on tiny grids, Gaussian-hill
                        and Cole-Hopf closed forms with second-order
                        convergence, plane-wave decay, conservation,
                        Dirichlet steady states, symmetry
  sources (step_src)    exact rational stepper with F and R, discrete mass
                        balance, uniform growth, Examples 4.1 / 4.5 closed forms
  tensor D              second-moment identity of Eq. 2.7, Example 4.4
                        anisotropic Gaussian hills
  Oracle3 (3-D)         exact rational 3-D stepper, D3Q15 / D3Q19 moments,
                        3-D kinetic dispersion root, conservation, symmetry
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dugks_oracle.c")
_SRC3 = os.path.join(_HERE, "dugks3d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

Q = 9


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, _SRC3, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("xf", ctypes.POINTER(ctypes.c_double)), ("yf", ctypes.POINTER(ctypes.c_double)),
        ("bc", ctypes.c_int * 4), ("bc_value", ctypes.c_double * 4),
        ("c", ctypes.c_double), ("u", ctypes.c_double * 2),
        ("nb", ctypes.c_int), ("b", ctypes.c_double * 8),
        ("alpha", ctypes.c_double),
        ("nd", ctypes.c_int), ("d", ctypes.c_double * 8),
        ("c_zero", ctypes.c_int), ("dt", ctypes.c_double),
        ("d_tensor", ctypes.c_int), ("ndt", ctypes.c_int),
        ("dxx", ctypes.c_double * 8), ("dxy", ctypes.c_double * 8), ("dyy", ctypes.c_double * 8),
        ("t0", ctypes.c_double),
        ("nsrc", ctypes.c_int), ("src_rate", ctypes.c_double * 8), ("src_pow", ctypes.c_int * 8),
        ("src_field", ctypes.POINTER(ctypes.c_double)),
    ]


class _Problem3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("xf", ctypes.POINTER(ctypes.c_double)), ("yf", ctypes.POINTER(ctypes.c_double)),
        ("zf", ctypes.POINTER(ctypes.c_double)),
        ("bc", ctypes.c_int * 6), ("bc_value", ctypes.c_double * 6),
        ("lattice", ctypes.c_int), ("c", ctypes.c_double), ("u", ctypes.c_double * 3),
        ("nb", ctypes.c_int), ("b", ctypes.c_double * 8),
        ("alpha", ctypes.c_double),
        ("nd", ctypes.c_int), ("d", ctypes.c_double * 8),
        ("c_zero", ctypes.c_int), ("dt", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_equilibrium.argtypes = [P, ctypes.c_double, dp]
        L.oracle_cell_transforms.argtypes = [P, dp, dp, dp, dp]
        L.oracle_face_original.argtypes = [P, dp, dp]
        L.oracle_face_original.restype = ctypes.c_double
        L.oracle_init.argtypes = [P, dp, dp]
        L.oracle_phi.argtypes = [P, dp, dp]
        L.oracle_mass.argtypes = [P, dp]
        L.oracle_mass.restype = ctypes.c_double
        L.oracle_step.argtypes = [P, dp, dp, ctypes.c_int]
        L.oracle_run.argtypes = [P, dp, ctypes.c_long, ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_equilibrium_deriv.argtypes = [P, ctypes.c_double, dp]
        L.oracle_adjoint_step.argtypes = [P, dp, dp, dp, dp, dp]
        L.oracle_equilibrium_du.argtypes = [P, ctypes.c_double, dp, dp]
        L.oracle_step_src.argtypes = [P, dp, dp, ctypes.c_double, dp, dp, dp, dp, ctypes.c_int]
        P3 = ctypes.POINTER(_Problem3)
        L.oracle3_equilibrium.argtypes = [P3, ctypes.c_double, dp]
        L.oracle3_init.argtypes = [P3, dp, dp]
        L.oracle3_phi.argtypes = [P3, dp, dp]
        L.oracle3_mass.argtypes = [P3, dp]
        L.oracle3_mass.restype = ctypes.c_double
        L.oracle3_step.argtypes = [P3, dp, dp, ctypes.c_int]
        L.oracle3_run.argtypes = [P3, dp, ctypes.c_long, ctypes.c_int]
        L.oracle_source.argtypes = [P, ctypes.c_long, ctypes.c_double, ctypes.c_double]
        L.oracle_source.restype = ctypes.c_double
        L.oracle_source_distributions.argtypes = [P, ctypes.c_double, ctypes.c_double, dp, dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """Holds a problem (see ``paper_1906_11036_gb300.inputs.Problem``) in the
    C struct layout; arrays are [Q][ny][nx] float64."""

    def __init__(self, problem):
        self.p = problem
        self._xf = np.ascontiguousarray(problem.xf, dtype=np.float64)
        self._yf = np.ascontiguousarray(problem.yf, dtype=np.float64)
        s = _Problem()
        s.nx, s.ny = len(self._xf) - 1, len(self._yf) - 1
        s.xf, s.yf = _ptr(self._xf), _ptr(self._yf)
        for i in range(4):
            s.bc[i] = int(problem.bc[i])
            s.bc_value[i] = float(problem.bc_value[i])
        s.c = float(problem.c)
        s.u[0], s.u[1] = float(problem.u[0]), float(problem.u[1])
        if len(problem.b) > 8 or len(problem.d) > 8:
            raise ValueError("at most 8 polynomial coefficients")
        s.nb = len(problem.b)
        for k, v in enumerate(problem.b):
            s.b[k] = float(v)
        s.alpha = float(problem.alpha)
        s.nd = len(problem.d)
        for k, v in enumerate(problem.d):
            s.d[k] = float(v)
        s.c_zero = int(bool(problem.c_zero))
        s.dt = float(problem.dt)
        if problem.d_tensor is not None:
            dt3 = [tuple(map(float, x)) for x in problem.d_tensor]
            ndt = max(len(x) for x in dt3)
            if len(dt3) != 3 or ndt > 8:
                raise ValueError("d_tensor = (dxx, dxy, dyy), at most 8 coefficients each")
            s.d_tensor, s.ndt = 1, ndt
            for arr, x in zip((s.dxx, s.dxy, s.dyy), dt3):
                for k, v in enumerate(x):
                    arr[k] = v
        s.t0 = float(problem.t0)
        src = tuple(problem.source)
        if len(src) > 8:
            raise ValueError("at most 8 source terms")
        self._src = None
        if src:
            self._src = np.ascontiguousarray(np.stack([np.asarray(t.field, dtype=np.float64) for t in src]))
            if self._src.shape[1:] != (s.ny, s.nx):
                raise ValueError("source fields must be [ny][nx]")
            s.nsrc = len(src)
            for k, t in enumerate(src):
                s.src_rate[k] = float(t.rate)
                s.src_pow[k] = int(t.power)
            s.src_field = _ptr(self._src)
        self.s = s
        self.L = lib()
        self.nx, self.ny = s.nx, s.ny

    # pointwise helpers --------------------------------------------------
    def equilibrium(self, phi: float) -> np.ndarray:
        out = np.zeros(Q)
        self.L.oracle_equilibrium(ctypes.byref(self.s), float(phi), _ptr(out))
        return out

    def equilibrium_deriv(self, phi: float) -> np.ndarray:
        out = np.zeros(Q)
        self.L.oracle_equilibrium_deriv(ctypes.byref(self.s), float(phi), _ptr(out))
        return out

    def equilibrium_du(self, phi: float) -> np.ndarray:
        """d feq_i / d u_a as a [2, 9] array (B = u b(phi), C = u u int b'^2)."""
        dx, dy = np.zeros(Q), np.zeros(Q)
        self.L.oracle_equilibrium_du(ctypes.byref(self.s), float(phi), _ptr(dx), _ptr(dy))
        return np.stack([dx, dy])

    def cell_transforms(self, ft, feq):
        ft = np.ascontiguousarray(ft, dtype=np.float64)
        feq = np.ascontiguousarray(feq, dtype=np.float64)
        fbp, ftp = np.zeros(Q), np.zeros(Q)
        self.L.oracle_cell_transforms(ctypes.byref(self.s), _ptr(ft), _ptr(feq), _ptr(fbp), _ptr(ftp))
        return fbp, ftp

    def face_original(self, fbar):
        fbar = np.ascontiguousarray(fbar, dtype=np.float64)
        f = np.zeros(Q)
        phib = self.L.oracle_face_original(ctypes.byref(self.s), _ptr(fbar), _ptr(f))
        return phib, f

    # fields --------------------------------------------------------------
    def init(self, phi0: np.ndarray) -> np.ndarray:
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == (self.ny, self.nx)
        f = np.zeros((Q, self.ny, self.nx))
        self.L.oracle_init(ctypes.byref(self.s), _ptr(phi0), _ptr(f))
        return f

    def step(self, f: np.ndarray, threads: int = 0) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        rc = self.L.oracle_step(ctypes.byref(self.s), _ptr(f), _ptr(out), int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle_step failed ({rc})")
        return out

    def run(self, f: np.ndarray, nsteps: int, threads: int = 0) -> np.ndarray:
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        rc = self.L.oracle_run(ctypes.byref(self.s), _ptr(f), int(nsteps), int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle_run failed ({rc})")
        return f

    def step_src(self, f: np.ndarray, t: float, R_prev=None, F_prev=None, threads: int = 0):
        """One step with sources at time t given R_i^{n-1}, F_i^{n-1} (None on the
        first step); returns (f^{n+1}, R_i^n, F_i^n), all [Q][ny][nx]."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        out, R, F = np.empty_like(f), np.empty_like(f), np.empty_like(f)
        null = ctypes.POINTER(ctypes.c_double)()
        rp = _ptr(np.ascontiguousarray(R_prev, dtype=np.float64)) if R_prev is not None else null
        fp = _ptr(np.ascontiguousarray(F_prev, dtype=np.float64)) if F_prev is not None else null
        keep = (R_prev, F_prev)  # noqa: F841
        rc = self.L.oracle_step_src(ctypes.byref(self.s), _ptr(f), _ptr(out), float(t), rp, fp, _ptr(R), _ptr(F),
                                    int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle_step_src failed ({rc})")
        return out, R, F

    def source(self, phi: np.ndarray, t: float) -> np.ndarray:
        """F(x_c, t, phi) at every cell (Eq. 2.1 source)."""
        phi = np.asarray(phi, dtype=np.float64)
        out = np.empty((self.ny, self.nx))
        for c in range(self.nx * self.ny):
            out.flat[c] = self.L.oracle_source(ctypes.byref(self.s), c, float(t), float(phi.flat[c]))
        return out

    def source_distributions(self, phi: float, F: float):
        R, Fi = np.zeros(Q), np.zeros(Q)
        self.L.oracle_source_distributions(ctypes.byref(self.s), float(phi), float(F), _ptr(R), _ptr(Fi))
        return R, Fi

    def adjoint_step(self, f: np.ndarray, mu: np.ndarray):
        """(lam, dJ/dalpha) for one step at state f given mu = dJ/d f^{n+1}."""
        lam, da, _ = self.adjoint_step_full(f, mu)
        return lam, da

    def adjoint_step_full(self, f: np.ndarray, mu: np.ndarray):
        """(lam, dJ/dalpha, dJ/du) for one step at state f given mu = dJ/d f^{n+1};
        dJ/du is the explicit dependence of the step on u of B = u b(phi)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        lam = np.empty_like(f)
        da = ctypes.c_double(0.0)
        du = np.zeros(2)
        rc = self.L.oracle_adjoint_step(ctypes.byref(self.s), _ptr(f), _ptr(mu), _ptr(lam),
                                        ctypes.cast(ctypes.pointer(da), ctypes.POINTER(ctypes.c_double)), _ptr(du))
        if rc != 0:
            raise RuntimeError(f"oracle_adjoint_step failed ({rc})")
        return lam, da.value, du

    def gradient(self, phi0: np.ndarray, nsteps: int, dj_dphiN, threads: int = 0, checkpoint_every: int = 0,
                 with_u: bool = False):
        """Reverse-mode gradient of J(phi^N) with respect to phi0 and alpha.
        dj_dphiN(phi^N) returns dJ/dphi^N.  With checkpoint_every = K > 0 only
        every K-th state is kept and each segment is recomputed.  Returns
        (dJ/dphi0, dJ/dalpha, phi^N), or with with_u (dJ/dphi0, dJ/dalpha,
        dJ/du, phi^N) where u is the velocity of B = u b(phi)."""
        K = nsteps if checkpoint_every <= 0 else checkpoint_every
        K = max(1, min(K, max(nsteps, 1)))
        ckpt = [self.init(phi0)]
        for s in range(0, nsteps, K):
            f = ckpt[-1]
            f = self.run(f, min(K, nsteps - s), threads)
            ckpt.append(f)
        phiN = self.phi(ckpt[-1])
        g = np.asarray(dj_dphiN(phiN), dtype=np.float64)
        lam = np.broadcast_to(g, (Q,) + g.shape).copy()   # phi = sum_i f_i
        dalpha = 0.0
        du = np.zeros(2)
        for si in range(len(ckpt) - 2, -1, -1):
            ns = min(K, nsteps - si * K)
            states = [ckpt[si]]
            for _ in range(ns - 1):
                states.append(self.step(states[-1], threads))
            for n in range(ns - 1, -1, -1):
                lam, da, d = self.adjoint_step_full(states[n], lam)
                dalpha += da
                du += d
        # f^0 = feq(phi0): dJ/dphi0 = sum_i feq_i'(phi0) lam_i, and f^0 depends on u too
        gphi = np.zeros(phi0.shape, dtype=np.float64)
        for k in range(self.ny):
            for j in range(self.nx):
                gphi[k, j] = float(self.equilibrium_deriv(phi0[k, j]) @ lam[:, k, j])
                if with_u:
                    du += self.equilibrium_du(phi0[k, j]) @ lam[:, k, j]
        if with_u:
            return gphi, dalpha, du, phiN
        return gphi, dalpha, phiN

    def phi(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((self.ny, self.nx))
        self.L.oracle_phi(ctypes.byref(self.s), _ptr(f), _ptr(out))
        return out

    def mass(self, f: np.ndarray) -> float:
        f = np.ascontiguousarray(f, dtype=np.float64)
        return float(self.L.oracle_mass(ctypes.byref(self.s), _ptr(f)))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


class Oracle3:
    """The 3-D oracle (D3Q15 / D3Q19) for a ``paper_1906_11036_gb300.inputs.Problem3``;
    arrays are [Q][nz][ny][nx] float64, phi [nz][ny][nx]."""

    def __init__(self, problem):
        self.p = problem
        self._f = [np.ascontiguousarray(a, dtype=np.float64) for a in (problem.xf, problem.yf, problem.zf)]
        s = _Problem3()
        s.nx, s.ny, s.nz = (len(a) - 1 for a in self._f)
        s.xf, s.yf, s.zf = (_ptr(a) for a in self._f)
        for i in range(6):
            s.bc[i] = int(problem.bc[i])
            s.bc_value[i] = float(problem.bc_value[i])
        s.lattice = int(problem.lattice)
        s.c = float(problem.c)
        for a in range(3):
            s.u[a] = float(problem.u[a])
        if len(problem.b) > 8 or len(problem.d) > 8:
            raise ValueError("at most 8 polynomial coefficients")
        s.nb = len(problem.b)
        for k, v in enumerate(problem.b):
            s.b[k] = float(v)
        s.alpha = float(problem.alpha)
        s.nd = len(problem.d)
        for k, v in enumerate(problem.d):
            s.d[k] = float(v)
        s.c_zero = int(bool(problem.c_zero))
        s.dt = float(problem.dt)
        self.s = s
        self.L = lib()
        self.nx, self.ny, self.nz = s.nx, s.ny, s.nz
        self.Q = int(problem.lattice)

    def equilibrium(self, phi: float) -> np.ndarray:
        out = np.zeros(self.Q)
        self.L.oracle3_equilibrium(ctypes.byref(self.s), float(phi), _ptr(out))
        return out

    def init(self, phi0: np.ndarray) -> np.ndarray:
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == (self.nz, self.ny, self.nx)
        f = np.zeros((self.Q, self.nz, self.ny, self.nx))
        self.L.oracle3_init(ctypes.byref(self.s), _ptr(phi0), _ptr(f))
        return f

    def step(self, f: np.ndarray, threads: int = 0) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        rc = self.L.oracle3_step(ctypes.byref(self.s), _ptr(f), _ptr(out), int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle3_step failed ({rc})")
        return out

    def run(self, f: np.ndarray, nsteps: int, threads: int = 0) -> np.ndarray:
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        rc = self.L.oracle3_run(ctypes.byref(self.s), _ptr(f), int(nsteps), int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle3_run failed ({rc})")
        return f

    def phi(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty((self.nz, self.ny, self.nx))
        self.L.oracle3_phi(ctypes.byref(self.s), _ptr(f), _ptr(out))
        return out

    def mass(self, f: np.ndarray) -> float:
        f = np.ascontiguousarray(f, dtype=np.float64)
        return float(self.L.oracle3_mass(ctypes.byref(self.s), _ptr(f)))
