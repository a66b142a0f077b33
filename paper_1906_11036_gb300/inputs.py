"""Seeded synthetic inputs for the DUGKS step: meshes, initial fields and
problem presets.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle.  It holds no arithmetic of the method itself (no equilibrium, no
transform, no flux): only face coordinates, initial phi fields drawn from
numpy's ``default_rng`` and the coefficient presets of the workloads.

Workloads (all 2-D, D2Q9):

* ``gaussian_hill``  -- linear convection-diffusion of a Gaussian hill on a
  periodic uniform mesh over [0,2]^2, B = phi u, u = (0.1, 0.1), D = phi I,
  alpha = 0.01, c = 1, CFL 0.5 (Section 4, Example 4.4 setting, moved to the
  smaller box and faster flow of the 64^2 parity case).
* ``burgers``        -- nonlinear Burgers-type NCDE, B = (phi^2/2)(1, 1),
  D = phi I, alpha = 0.005, periodic [0,1]^2, c = 10, CFL 0.4,
  phi0 = 1 + 0.2 sin(2 pi x) sin(2 pi y) + 0.01 * band-limited noise.
* ``nonuniform``     -- nonlinear diffusion on a tanh-stretched mesh
  (k = 2, clustered toward both walls of [0,1]^2), Dirichlet phi = 1 on the
  west wall and 0.5 elsewhere, D = phi^2 I, alpha = 0.01, B = phi (0.05, 0),
  c = 10 (the lattice speed of the paper's non-uniform-mesh example, Section 4,
  Example 4.3), CFL 0.4, smooth phi0 in (0.5, 1.5).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC = 0
DIRICHLET = 1
WALLS = ("W", "E", "S", "N")


@dataclass
class Problem:
    """A complete description of one NCDE instance (pure data).

    B(phi) = u * b(phi), D(phi) = d(phi) I with b, d polynomials given by
    their coefficients (lowest order first); C = u u * int_0^phi b'(s)^2 ds
    unless ``c_zero``.  ``bc`` and ``bc_value`` are ordered W, E, S, N.
    """

    xf: np.ndarray
    yf: np.ndarray
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    bc_value: tuple = (0.0, 0.0, 0.0, 0.0)
    c: float = 1.0
    u: tuple = (0.0, 0.0)
    b: tuple = (0.0, 1.0)
    alpha: float = 0.01
    d: tuple = (0.0, 1.0)
    c_zero: bool = False
    dt: float = 0.0
    steps: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return len(self.xf) - 1

    @property
    def ny(self) -> int:
        return len(self.yf) - 1

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def centres(self):
        xc = 0.5 * (self.xf[1:] + self.xf[:-1])
        yc = 0.5 * (self.yf[1:] + self.yf[:-1])
        return xc, yc

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

def uniform_faces(n: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    return np.linspace(a, b, n + 1, dtype=np.float64)


def tanh_faces(n: int, k: float = 2.0, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """Faces clustered toward both ends: x = (1 + tanh(k(2s-1))/tanh(k))/2,
    s = j/n (the stretching of Section 4, Example 4.3, mirrored so that it
    clusters toward both walls)."""
    s = np.arange(n + 1, dtype=np.float64) / n
    x = 0.5 * (1.0 + np.tanh(k * (2.0 * s - 1.0)) / np.tanh(k))
    x[0], x[-1] = 0.0, 1.0
    return a + (b - a) * x


def cfl_dt(xf: np.ndarray, yf: np.ndarray, c: float, cfl: float) -> float:
    """Time step from the CFL number (Remark 1): dt = CFL * min(dx, dy) / c."""
    return float(cfl * min(np.diff(xf).min(), np.diff(yf).min()) / c)


# ---------------------------------------------------------------------------
# initial fields (point values at cell centres)
# ---------------------------------------------------------------------------

def _fourier_noise(xc, yc, kmax, rng, lx=1.0, ly=1.0):
    """Sum of random cos/sin plane waves with |kx|, |ky| <= kmax, normalised to
    unit RMS on the grid; evaluated separably."""
    ks = np.arange(-kmax, kmax + 1)
    A = rng.standard_normal((len(ks), len(ks)))  # [ky, kx]
    Bc = rng.standard_normal((len(ks), len(ks)))
    c0 = kmax  # index of k = 0
    A[c0, c0] = 0.0
    Bc[c0, c0] = 0.0
    ax = 2.0 * np.pi * np.outer(xc / lx, ks)  # [nx, K]
    ay = 2.0 * np.pi * np.outer(yc / ly, ks)  # [ny, K]
    cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
    # cos(a+b) = ca cb - sa sb ; sin(a+b) = sa cb + ca sb
    noise = cy @ A @ cx.T - sy @ A @ sx.T + cy @ Bc @ sx.T + sy @ Bc @ cx.T
    noise /= np.sqrt(np.mean(noise * noise))
    return noise  # [ny, nx]


def gaussian_hill_phi0(xc, yc, x0=1.0, y0=1.0, s2=0.01):
    X, Y = np.meshgrid(xc, yc)
    return np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * s2))


def burgers_phi0(xc, yc, seed=2):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(xc, yc)
    base = 1.0 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    return base + 0.01 * _fourier_noise(xc, yc, 8, rng)


def smooth_phi0(xc, yc, seed=3):
    """Smooth field in (0.5, 1.5): 1 + 0.5 tanh(sum of low modes)."""
    rng = np.random.default_rng(seed)
    return 1.0 + 0.5 * np.tanh(_fourier_noise(xc, yc, 2, rng))


# ---------------------------------------------------------------------------
# presets
# ---------------------------------------------------------------------------

def gaussian_hill(n: int = 64, steps: int = 200, cfl: float = 0.5) -> tuple[Problem, np.ndarray]:
    xf = uniform_faces(n, 0.0, 2.0)
    p = Problem(xf=xf, yf=xf.copy(), c=1.0, u=(0.1, 0.1), b=(0.0, 1.0), alpha=0.01,
                d=(0.0, 1.0), dt=cfl_dt(xf, xf, 1.0, cfl), steps=steps,
                name=f"gaussian_hill_{n}x{n}", meta={"cfl": cfl})
    xc, yc = p.centres()
    return p, gaussian_hill_phi0(xc, yc)


def burgers(nx: int = 1024, ny: int | None = None, steps: int = 2000, seed: int = 2,
            cfl: float = 0.4) -> tuple[Problem, np.ndarray]:
    ny = nx if ny is None else ny
    xf, yf = uniform_faces(nx), uniform_faces(ny)
    p = Problem(xf=xf, yf=yf, c=10.0, u=(1.0, 1.0), b=(0.0, 0.0, 0.5), alpha=0.005,
                d=(0.0, 1.0), dt=cfl_dt(xf, yf, 10.0, cfl), steps=steps,
                name=f"burgers_{nx}x{ny}", meta={"cfl": cfl, "seed": seed})
    xc, yc = p.centres()
    return p, burgers_phi0(xc, yc, seed)


def nonuniform(nx: int = 2048, ny: int | None = None, steps: int = 5000, seed: int = 3,
               k: float = 2.0, cfl: float = 0.4) -> tuple[Problem, np.ndarray]:
    ny = nx if ny is None else ny
    xf, yf = tanh_faces(nx, k), tanh_faces(ny, k)
    p = Problem(xf=xf, yf=yf, bc=(DIRICHLET,) * 4, bc_value=(1.0, 0.5, 0.5, 0.5), c=10.0,
                u=(0.05, 0.0), b=(0.0, 1.0), alpha=0.01, d=(0.0, 0.0, 1.0),
                dt=cfl_dt(xf, yf, 10.0, cfl), steps=steps,
                name=f"nonuniform_{nx}x{ny}", meta={"cfl": cfl, "seed": seed, "k": k})
    xc, yc = p.centres()
    return p, smooth_phi0(xc, yc, seed)


def batched(n: int = 256, seed: int = 7, steps: int = 1000, sides=(64, 128, 256, 512),
            cfl: float = 0.4) -> list[tuple[Problem, np.ndarray]]:
    """Independent periodic Burgers-type instances: square sides drawn uniformly
    from `sides`, B = a phi^2/2 (1, 1) with a ~ U[0.5, 2], D = D0 (1 + phi^2) I
    read as alpha = D0 ~ U[0.002, 0.02] and d = 1 + phi^2; c = 10, CFL 0.4 per
    instance; phi0 of the Burgers form with a per-instance seed."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=n)
    a = rng.uniform(0.5, 2.0, size=n)
    d0 = rng.uniform(0.002, 0.02, size=n)
    out = []
    for i in range(n):
        m = int(side[i])
        xf = uniform_faces(m)
        p = Problem(xf=xf, yf=xf.copy(), c=10.0, u=(1.0, 1.0), b=(0.0, 0.0, 0.5 * float(a[i])),
                    alpha=float(d0[i]), d=(1.0, 0.0, 1.0), dt=cfl_dt(xf, xf, 10.0, cfl), steps=steps,
                    name=f"batched_{i}_{m}x{m}", meta={"a": float(a[i]), "D0": float(d0[i]), "seed": seed + 1 + i})
        xc, yc = p.centres()
        out.append((p, burgers_phi0(xc, yc, seed + 1 + i)))
    return out


PRESETS = {
    "gaussian_hill": gaussian_hill,
    "burgers": burgers,
    "nonuniform": nonuniform,
}
