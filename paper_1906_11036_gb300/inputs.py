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


@dataclass(frozen=True)
class SourceTerm:
    """One term exp(rate t) phi^power S(x) of the source F (S: [ny][nx] array)."""

    rate: float
    power: int
    field: np.ndarray


@dataclass
class Problem:
    """A complete description of one NCDE instance (pure data).

    B(phi) = u * b(phi), D(phi) = d(phi) I with b, d polynomials given by
    their coefficients (lowest order first); C = u u * int_0^phi b'(s)^2 ds
    unless ``c_zero``.  ``bc`` and ``bc_value`` are ordered W, E, S, N.

    ``d_tensor`` = (dxx, dxy, dyy), each a coefficient tuple, replaces d(phi) I
    by the symmetric tensor [[dxx, dxy], [dxy, dyy]](phi).  ``source`` is a
    tuple of SourceTerm: F(x, t, phi) = sum_k exp(rate_k t) phi^power_k S_k(x)
    with S_k an [ny][nx] array sampled at the cell centres (Eq. 2.1); ``t0``
    is the time of the initial state.
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
    d_tensor: tuple | None = None
    source: tuple = ()
    t0: float = 0.0
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


def gaussian_hill_exact(xc, yc, t, u, alpha, s2=0.01, L=2.0, x0=1.0, y0=1.0, images=3):
    """Closed form of the linear CDE for the Gaussian hill (Eq. 4.4.3 with K = alpha I,
    sigma0^2 = s2, peak 1 at t = 0), summed over periodic images of the box of side L."""
    X, Y = np.meshgrid(xc, yc)
    s = s2 + 2 * alpha * t
    out = np.zeros_like(X)
    for m in range(-images, images + 1):
        for n in range(-images, images + 1):
            dx = X - x0 - u[0] * t - m * L
            dy = Y - y0 - u[1] * t - n * L
            out += s2 / s * np.exp(-(dx * dx + dy * dy) / (2 * s))
    return out


def gre(num, exact):
    """Global relative error, Eq. 4.1.1."""
    return float(np.abs(num - exact).sum() / np.abs(exact).sum())


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


def cde_source(n: int = 200, pe: float = 100.0, t_end: float = 3.0, cfl: float = 0.5,
               c: float = 1.0) -> tuple[Problem, np.ndarray]:
    """Section 4, Example 4.1: isotropic CDE with constant u = (0.1, 0.1) and the
    source of Eq. 4.1.3 on the periodic box [0, 2]^2; alpha = L u_x / Pe with
    L = 2; B = phi u, C = phi u u, D = phi I; phi0 = sin(pi (x + y)).  The exact
    solution (Eq. 4.1.5) is in meta["exact"](t)."""
    ux = uy = 0.1
    alpha = 2.0 * ux / pe
    xf = uniform_faces(n, 0.0, 2.0)
    xc = 0.5 * (xf[1:] + xf[:-1])
    X, Y = np.meshgrid(xc, xc)
    rate = 1.0 - 2.0 * np.pi ** 2 * alpha
    S = np.sin(np.pi * (X + Y)) + np.pi * (ux + uy) * np.cos(np.pi * (X + Y))
    dt = cfl_dt(xf, xf, c, cfl)
    p = Problem(xf=xf, yf=xf.copy(), c=c, u=(ux, uy), b=(0.0, 1.0), alpha=alpha, d=(0.0, 1.0), dt=dt,
                source=(SourceTerm(rate, 0, S),), steps=int(round(t_end / dt)),
                name=f"cde_source_{n}x{n}_pe{pe:g}",
                meta={"pe": pe, "cfl": cfl, "exact": lambda t: np.exp(rate * t) * np.sin(np.pi * (X + Y))})
    return p, np.sin(np.pi * (X + Y))


def nonlinear_source(n: int = 400, pe: float = 100.0, t_end: float = 3.0, cfl: float = 0.5, c: float = 1.0,
                     u=(0.1, 0.1), m: int = 2, nx_: int = 2, ny_: int = 3, A: float = 1.0,
                     kappa: float = 1.1) -> tuple[Problem, np.ndarray]:
    """Section 4, Example 4.5: B = phi^m u, D = diag(phi^nx, phi^ny), the source of
    Eq. 4.5.3, periodic [0, 1]^2, exact solution kappa - exp(-A t) cos(2 pi x)
    cos(2 pi y) (Eq. 4.5.4, meta["exact"]).  The example does not state u; it is
    read as (0.1, 0.1) as in Example 4.1, with alpha = L u_x / Pe, L = 1.
    C = m^2 phi^(2m-1)/(2m-1) u u is the Remark 3 choice.  The source is
    expanded into terms exp(rate t) phi^p S(x)."""
    ux, uy = float(u[0]), float(u[1])
    alpha = 1.0 * ux / pe
    xf = uniform_faces(n)
    xc = 0.5 * (xf[1:] + xf[:-1])
    X, Y = np.meshgrid(xc, xc)
    sx, cx, sy, cy = np.sin(2 * np.pi * X), np.cos(2 * np.pi * X), np.sin(2 * np.pi * Y), np.cos(2 * np.pi * Y)
    cc = cx * cy
    pi2 = np.pi ** 2
    src = (SourceTerm(-A, 0, A * cc),
           SourceTerm(-2 * A, nx_ - 2, -4 * nx_ * (nx_ - 1) * pi2 * alpha * sx ** 2 * cy ** 2),
           SourceTerm(-A, nx_ - 1, -4 * nx_ * pi2 * alpha * cc),
           SourceTerm(-2 * A, ny_ - 2, -4 * ny_ * (ny_ - 1) * pi2 * alpha * sy ** 2 * cx ** 2),
           SourceTerm(-A, ny_ - 1, -4 * ny_ * pi2 * alpha * cc),
           SourceTerm(-A, m - 1, 2 * np.pi * m * (ux * sx * cy + uy * cx * sy)))
    dt = cfl_dt(xf, xf, c, cfl)
    p = Problem(xf=xf, yf=xf.copy(), c=c, u=(ux, uy), b=tuple([0.0] * m + [1.0]), alpha=alpha, d=(0.0,),
                d_tensor=(tuple([0.0] * nx_ + [1.0]), (0.0,), tuple([0.0] * ny_ + [1.0])), dt=dt, source=src,
                steps=int(round(t_end / dt)), name=f"nonlinear_source_{n}x{n}_pe{pe:g}",
                meta={"pe": pe, "cfl": cfl, "exact": lambda t: kappa - np.exp(-A * t) * cc})
    return p, kappa - cc


ANISO_K = {"isotropic": ((1.0, 0.0), (0.0, 1.0)), "diagonal": ((1.0, 0.0), (0.0, 2.0)),
           "full": ((1.0, 1.0), (1.0, 2.0))}


def gaussian_hill_aniso(n: int = 400, kind: str = "full", t_end: float = 10.0, cfl: float = 0.5,
                        c: float = 1.0) -> tuple[Problem, np.ndarray]:
    """Section 4, Example 4.4: Gaussian hill on the periodic box [-1, 1]^2 with
    u = (0.01, 0.01), kappa = alpha = 1e-3 and D = K phi / kappa for the three
    tensors K of Eq. 4.4.5 (times 1e-3); sigma0^2 = 0.01, peak 1 at the origin."""
    K = ANISO_K[kind]
    xf = uniform_faces(n, -1.0, 1.0)
    dt = cfl_dt(xf, xf, c, cfl)
    p = Problem(xf=xf, yf=xf.copy(), c=c, u=(0.01, 0.01), b=(0.0, 1.0), alpha=1e-3, d=(0.0,),
                d_tensor=((0.0, K[0][0]), (0.0, K[0][1]), (0.0, K[1][1])), dt=dt,
                steps=int(round(t_end / dt)), name=f"gaussian_hill_{kind}_{n}x{n}",
                meta={"cfl": cfl, "K": K, "sigma0_sq": 0.01})
    xc, yc = p.centres()
    X, Y = np.meshgrid(xc, yc)
    return p, np.exp(-(X ** 2 + Y ** 2) / (2 * 0.01))


# ---------------------------------------------------------------------------
# three dimensions (D3Q15 / D3Q19)
# ---------------------------------------------------------------------------

@dataclass
class Problem3:
    """One 3-D NCDE instance: B = u b(phi) with u in R^3, D = d(phi) I,
    C = u u int_0^phi b'(s)^2 ds unless c_zero; ``lattice`` 15 (D3Q15, Eq. 2.28)
    or 19 (D3Q19, Eq. 2.6).  ``bc`` / ``bc_value`` ordered W, E, S, N, B, T
    (x low/high, y low/high, z low/high)."""

    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray
    bc: tuple = (PERIODIC,) * 6
    bc_value: tuple = (0.0,) * 6
    lattice: int = 19
    c: float = 1.0
    u: tuple = (0.0, 0.0, 0.0)
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
    def nz(self) -> int:
        return len(self.zf) - 1

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def centres(self):
        return tuple(0.5 * (f[1:] + f[:-1]) for f in (self.xf, self.yf, self.zf))

    def with_(self, **kw) -> "Problem3":
        return replace(self, **kw)


def cfl_dt3(xf, yf, zf, c: float, cfl: float) -> float:
    """dt = CFL * min cell width / c (Remark 1)."""
    return float(cfl * min(np.diff(xf).min(), np.diff(yf).min(), np.diff(zf).min()) / c)


def burgers3d_phi0(xc, yc, zc, seed=2):
    """1 + 0.2 sin 2pi x sin 2pi y sin 2pi z + 0.01 x (24 random low plane waves,
    unit RMS); array [nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    base = 1.0 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z)
    noise = np.zeros_like(X)
    for _ in range(24):
        k = rng.integers(-4, 5, size=3)
        noise += rng.standard_normal() * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 2 * np.pi))
    noise /= np.sqrt(np.mean(noise * noise))
    return base + 0.01 * noise


def burgers3d(n: int = 256, ny: int | None = None, nz: int | None = None, lattice: int = 19, steps: int = 500,
              seed: int = 2, cfl: float = 0.4) -> tuple[Problem3, np.ndarray]:
    """3-D periodic Burgers-type NCDE on [0,1]^3: B = (1,1,1) phi^2/2, D = phi I,
    alpha = 0.005, c = 10, CFL 0.4 (the 2-D Burgers workload lifted to 3-D)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    xf, yf, zf = uniform_faces(n), uniform_faces(ny), uniform_faces(nz)
    p = Problem3(xf=xf, yf=yf, zf=zf, lattice=lattice, c=10.0, u=(1.0, 1.0, 1.0), b=(0.0, 0.0, 0.5),
                 alpha=0.005, d=(0.0, 1.0), dt=cfl_dt3(xf, yf, zf, 10.0, cfl), steps=steps,
                 name=f"burgers3d_d3q{lattice}_{n}x{ny}x{nz}", meta={"cfl": cfl, "seed": seed})
    xc, yc, zc = p.centres()
    return p, burgers3d_phi0(xc, yc, zc, seed)


def adjoint_workload(n: int = 512, steps: int = 400):
    """The adjoint workload: the Burgers-type NCDE on n^2 periodic cells, `steps`
    steps, misfit J = 1/2 sum_cells |V| (phi^N - phi_target)^2 to a seeded target of
    the same form as phi0 (seed 5).  Returns (problem, phi0, target, cell areas)."""
    p, phi0 = burgers(n, steps=steps)
    xc, yc = p.centres()
    return p, phi0, burgers_phi0(xc, yc, seed=5), np.outer(np.diff(p.yf), np.diff(p.xf))


def unit_directions(shape, count: int, seed: int = 5):
    """`count` seeded random directions of unit 2-norm (standard normal entries)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = rng.standard_normal(shape)
        out.append(d / np.linalg.norm(d))
    return out


def batched_sample(count: int = 16, seed: int = 17, n: int = 256):
    """Indices of `count` instances of the batched workload, drawn without repetition."""
    return sorted(int(i) for i in np.random.default_rng(seed).choice(n, size=count, replace=False))


PRESETS = {
    "gaussian_hill": gaussian_hill,
    "burgers": burgers,
    "nonuniform": nonuniform,
    "cde_source": cde_source,
    "nonlinear_source": nonlinear_source,
    "gaussian_hill_aniso": gaussian_hill_aniso,
}
