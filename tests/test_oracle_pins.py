"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code.

Each test names the passage it follows.  Together they are chosen so that a
plausible slip anywhere in the oracle (a dropped term, a wrong sign, a wrong
index or weight, a transposed operand, a wrong relaxation time) fails at
least one of them:

* equilibrium moments (Eq. 2.7), with C from numerical quadrature;
* the composite transforms (Eqs. 2.21-2.23) against the basic ones
  (Eqs. 2.11, 2.13, 2.15, 2.17);
* an exact rational stepper on tiny grids, periodic and Dirichlet,
  uniform and non-uniform;
* the slow-mode dispersion root of the discrete-velocity BGK equation
  (Eq. 2.2) approached at second order (Section 4 convergence claims);
* closed-form solutions: Gaussian hill (Eq. 4.4.3) and viscous Burgers
  (Cole-Hopf), second order in space;
* conservation, fixed points, symmetry, Dirichlet steady states;
* the paper's printed GRE of Example 4.4 as a soft pin.
"""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy.integrate import fixed_quad
from scipy.optimize import fsolve

from oracle import Oracle
from paper_1906_11036_gb300 import inputs as I
from rational_stepper import RationalDUGKS

CV = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _problem(**kw):
    xf = kw.pop("xf", I.uniform_faces(4))
    return I.Problem(xf=xf, yf=kw.pop("yf", xf.copy()), **kw)


# ---------------------------------------------------------------------------
# Eq. 2.3 / Eq. 2.7: moments of the equilibrium
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("c,u,b,d,czero", [
    (1.0, (0.1, 0.1), (0.0, 1.0), (0.0, 1.0), False),          # linear CDE
    (10.0, (1.0, 1.0), (0.0, 0.0, 0.5), (0.0, 1.0), False),    # Burgers-type
    (1.0, (0.05, 0.0), (0.0, 1.0), (0.0, 0.0, 1.0), False),    # nonlinear diffusion
    (3.0, (0.7, -0.4), (0.2, -0.3, 0.5, 0.25), (1.0, 0.0, 1.0), False),
    (2.0, (0.3, 0.6), (0.0, 0.0, 0.5), (0.0, 1.0), True),      # C = 0
])
def test_equilibrium_moments(c, u, b, d, czero):
    p = _problem(c=c, u=u, b=b, d=d, c_zero=czero, alpha=0.01, dt=1e-3)
    o = Oracle(p)
    cs2 = c * c / 3.0
    bp = np.polynomial.Polynomial(b).deriv()
    for phi in np.random.default_rng(1).uniform(0.3, 1.7, 7):
        feq = o.equilibrium(phi)
        ci = CV * c
        B = np.array(u) * np.polynomial.Polynomial(b)(phi)
        D = np.polynomial.Polynomial(d)(phi) * np.eye(2)
        # Gauss-Legendre with 16 nodes integrates the polynomial b'^2 exactly
        Cint = 0.0 if czero else fixed_quad(lambda s: bp(s) ** 2, 0.0, phi, n=16)[0]
        C = Cint * np.outer(u, u)
        assert abs(feq.sum() - phi) <= 1e-14 * max(1.0, abs(phi))
        np.testing.assert_allclose(ci.T @ feq, B, rtol=1e-13, atol=1e-14)
        second = np.einsum("ia,ib,i->ab", ci, ci, feq)
        np.testing.assert_allclose(second, cs2 * D + C, rtol=1e-13, atol=1e-13)


def test_equilibrium_weights_at_rest():
    """With B = 0, D = phi I the equilibrium is w_i phi: the D2Q9 weights 4/9, 1/9, 1/36 (Eq. 2.5)."""
    p = _problem(c=2.0, u=(0.0, 0.0), b=(0.0, 1.0), d=(0.0, 1.0), alpha=0.01, dt=1e-3)
    feq = Oracle(p).equilibrium(1.0)
    np.testing.assert_allclose(feq, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


# ---------------------------------------------------------------------------
# Eqs. 2.11-2.23: transforms
# ---------------------------------------------------------------------------

def test_composite_transforms_match_basic_definitions():
    c, alpha, dt = 2.0, 0.013, 0.0037
    p = _problem(c=c, u=(0.3, -0.2), b=(0.0, 0.0, 0.5), d=(0.0, 1.0), alpha=alpha, dt=dt)
    o = Oracle(p)
    lam, h = alpha / (c * c / 3.0), dt / 2.0
    rng = np.random.default_rng(4)
    ft = rng.uniform(0.0, 0.3, 9)
    feq = o.equilibrium(ft.sum())
    fbp, ftp = o.cell_transforms(ft, feq)
    f = (2 * lam * ft + dt * feq) / (2 * lam + dt)                  # Eq. 2.11 solved for f
    fbar = (2 * lam + h) / (2 * lam) * f - h / (2 * lam) * feq      # Eq. 2.15 (f_i restored)
    fbp_ref = (2 * lam - h) / (2 * lam + h) * fbar + 2 * h / (2 * lam + h) * feq   # Eq. 2.17
    ftilde_again = f + dt / (2 * lam) * (f - feq)                   # Eq. 2.11: ft = f - dt/2 Omega
    ftp_ref = ftilde_again + dt * (-(f - feq) / lam)                # ft^+ = f + dt/2 Omega (Eq. 2.13 origin)
    np.testing.assert_allclose(fbp, fbp_ref, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(ftp, ftp_ref, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(ftp, 4.0 / 3.0 * fbp - ft / 3.0, rtol=1e-13, atol=1e-16)  # Eq. 2.23
    assert abs(ftp.sum() - ft.sum()) < 1e-15


def test_face_original_inverts_eq_2_15():
    c, alpha, dt = 1.0, 0.02, 0.01
    p = _problem(c=c, u=(0.1, 0.1), b=(0.0, 1.0), d=(0.0, 1.0), alpha=alpha, dt=dt)
    o = Oracle(p)
    lam, h = alpha / (c * c / 3.0), dt / 2.0
    fbar = np.random.default_rng(5).uniform(0.0, 0.2, 9)
    phib, f = o.face_original(fbar)
    assert phib == pytest.approx(fbar.sum(), rel=1e-15)
    feqb = o.equilibrium(fbar.sum())
    np.testing.assert_allclose((2 * lam + h) / (2 * lam) * f - h / (2 * lam) * feqb, fbar, rtol=1e-14)


# ---------------------------------------------------------------------------
# exact rational arithmetic on tiny grids
# ---------------------------------------------------------------------------

def _rational_case(nx, ny, bc, bcv, b, d, u, c, alpha, dt, nsteps, nonuni, czero, seed):
    rng = np.random.default_rng(seed)
    if nonuni:
        xf = [Fr(0)] + sorted(Fr(int(v), 64) for v in rng.choice(np.arange(1, 64), nx - 1, replace=False)) + [Fr(1)]
        yf = [Fr(0)] + sorted(Fr(int(v), 64) for v in rng.choice(np.arange(1, 64), ny - 1, replace=False)) + [Fr(1)]
    else:
        xf = [Fr(j, nx) for j in range(nx + 1)]
        yf = [Fr(k, ny) for k in range(ny + 1)]
    phi0 = [[Fr(int(rng.integers(50, 150)), 100) for _ in range(nx)] for _ in range(ny)]
    R = RationalDUGKS(xf, yf, bc, bcv, c, u, b, alpha, d, czero, dt)
    st = R.init(phi0)
    for _ in range(nsteps):
        st = R.step(st)
    exact = R.to_array(st)
    p = I.Problem(xf=np.array([float(v) for v in xf]), yf=np.array([float(v) for v in yf]), bc=bc,
                  bc_value=tuple(float(v) for v in bcv), c=float(c), u=tuple(float(v) for v in u),
                  b=tuple(float(v) for v in b), alpha=float(alpha), d=tuple(float(v) for v in d),
                  c_zero=czero, dt=float(dt))
    o = Oracle(p)
    f = o.run(o.init(np.array([[float(v) for v in r] for r in phi0])), nsteps)
    return f, exact


RATIONAL_CASES = [
    # nx, ny, bc, bc values, b, d, u, c, alpha, dt, steps, non-uniform, C=0
    (4, 4, (0, 0, 0, 0), (0, 0, 0, 0), (0, 1), (0, 1), (Fr(1, 10), Fr(1, 20)), 1, Fr(1, 100), Fr(1, 16), 3, False, False),
    (5, 3, (0, 0, 0, 0), (0, 0, 0, 0), (0, 0, Fr(1, 2)), (0, 1), (1, 1), 10, Fr(1, 200), Fr(1, 400), 2, False, False),
    (5, 3, (0, 0, 0, 0), (0, 0, 0, 0), (0, 0, Fr(1, 2)), (0, 1), (1, Fr(1, 3)), 10, Fr(1, 200), Fr(1, 400), 2, True, True),
    (4, 4, (1, 1, 1, 1), (1, Fr(1, 2), Fr(1, 2), Fr(1, 2)), (0, 1), (0, 0, 1), (Fr(1, 20), 0), 1, Fr(1, 100), Fr(1, 64), 2, True, False),
    (4, 3, (1, 1, 0, 0), (1, Fr(1, 2), 0, 0), (0, 1), (0, 1), (Fr(1, 20), Fr(1, 10)), 1, Fr(1, 100), Fr(1, 64), 2, True, False),
    (3, 4, (0, 0, 1, 1), (0, 0, Fr(3, 4), Fr(1, 4)), (0, 0, Fr(1, 2)), (1, 0, 1), (1, Fr(-1, 2)), 10, Fr(1, 100), Fr(1, 640), 2, True, False),
    (1, 3, (0, 0, 0, 0), (0, 0, 0, 0), (0, 1), (0, 1), (Fr(1, 10), Fr(1, 10)), 1, Fr(1, 50), Fr(1, 32), 2, False, False),
]


@pytest.mark.parametrize("case", RATIONAL_CASES, ids=[f"case{i}" for i in range(len(RATIONAL_CASES))])
def test_oracle_matches_exact_rational_stepper(case):
    f, exact = _rational_case(*case, seed=RATIONAL_CASES.index(case))
    assert np.abs(f - exact).max() <= 1e-14 * np.abs(exact).max()


# ---------------------------------------------------------------------------
# kinetic dispersion root, approached at second order
# ---------------------------------------------------------------------------

def _dbe_root(kvec, u, alpha, c):
    """Slow-mode root s of the linearised discrete-velocity BGK equation (Eq. 2.2,
    no source) for f_eq linear in phi (b = phi, d = phi, C = uu phi):
    sum_i w_i g_i / (1 + lam s + i lam k.c_i) = 1."""
    cs2 = c * c / 3.0
    lam = alpha / cs2
    ci = CV * c
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    cu = ci @ np.asarray(u)
    g = 1 + cu / cs2 + (cu ** 2 - cs2 * np.dot(u, u)) / (2 * cs2 * cs2)
    kc = ci @ np.asarray(kvec)

    def F(z):
        r = np.sum(w * g / (1 + lam * (z[0] + 1j * z[1]) + 1j * lam * kc)) - 1
        return [r.real, r.imag]

    z = fsolve(F, [-alpha * np.dot(kvec, kvec), -np.dot(kvec, u)], xtol=1e-14)
    return z[0] + 1j * z[1]


@pytest.mark.parametrize("kv,u", [((2 * np.pi, 2 * np.pi), (0.1, 0.05)), ((2 * np.pi, 0.0), (0.2, 0.0)),
                                  ((0.0, 4 * np.pi), (0.0, -0.1))])
def test_plane_wave_rate_converges_to_kinetic_dispersion(kv, u, nthreads):
    c, alpha = 1.0, 0.01
    s_ex = _dbe_root(np.array(kv), u, alpha, c)
    errs = []
    for n in (32, 64, 128):
        xf = I.uniform_faces(n)
        p = I.Problem(xf=xf, yf=xf.copy(), c=c, u=u, b=(0, 1), alpha=alpha, d=(0, 1),
                      dt=I.cfl_dt(xf, xf, c, 0.5))
        xc, yc = p.centres()
        X, Y = np.meshgrid(xc, yc)
        ph = kv[0] * X + kv[1] * Y
        o = Oracle(p)
        s1 = int(round(1.0 / p.dt))
        f = o.run(o.init(1 + 0.1 * np.cos(ph)), s1, nthreads)
        A1 = np.mean((o.phi(f) - 1) * np.exp(-1j * ph))
        f = o.run(f, s1, nthreads)
        A2 = np.mean((o.phi(f) - 1) * np.exp(-1j * ph))
        s = np.log(A2 / A1) / (s1 * p.dt)
        errs.append(abs(s - s_ex) / abs(s_ex))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 3e-3, errs
    assert np.all(orders > 1.85), (errs, orders)


# ---------------------------------------------------------------------------
# closed-form solutions of the PDE (Eq. 2.1)
# ---------------------------------------------------------------------------

gaussian_hill_exact = I.gaussian_hill_exact  # Eq. 4.4.3 summed over periodic images
gre = I.gre  # Eq. 4.1.1


def test_gaussian_hill_second_order(nthreads):
    """Linear CDE of the 64^2 Gaussian-hill workload; c = 10 so that the
    kinetic (finite relaxation time) error stays below the discretisation error."""
    errs = []
    for n in (32, 64, 128):
        p, phi0 = I.gaussian_hill(n)
        p = p.with_(c=10.0, dt=p.dt / 10.0)
        steps = int(round(3.125 / p.dt))
        o = Oracle(p)
        f = o.run(o.init(phi0), steps, nthreads)
        xc, yc = p.centres()
        errs.append(gre(o.phi(f), gaussian_hill_exact(xc, yc, steps * p.dt, p.u, p.alpha)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3 and orders[0] > 1.9 and orders[1] > 1.7, (errs, orders)


def test_gaussian_hill_workload_closed_form(nthreads):
    """The 64^2, c = 1 parity workload itself: GRE against the closed form and
    exact conservation over its 200 steps."""
    p, phi0 = I.gaussian_hill(64)
    o = Oracle(p)
    f0 = o.init(phi0)
    f = o.run(f0, p.steps, nthreads)
    xc, yc = p.centres()
    e = gre(o.phi(f), gaussian_hill_exact(xc, yc, p.steps * p.dt, p.u, p.alpha))
    assert 5e-3 < e < 3e-2, e   # dominated by the c = 1 kinetic error (see dispersion test)
    assert abs(o.mass(f) - o.mass(f0)) <= 1e-13 * o.mass(f0)


def cole_hopf(x, t, nu, U=1.0, a=2.0, bb=1.0, k=2 * np.pi):
    """Periodic viscous-Burgers solution phi_t + (phi^2/2)_x = nu phi_xx via the
    Cole-Hopf transform of theta = a + bb exp(-nu k^2 t) cos(k (x - U t))."""
    e = bb * np.exp(-nu * k * k * t)
    z = k * (x - U * t)
    return U + 2 * nu * k * e * np.sin(z) / (a + e * np.cos(z))


def test_burgers_cole_hopf_second_order(nthreads):
    errs = []
    nu, c = 0.05, 50.0
    for n in (32, 64, 128):
        xf, yf = I.uniform_faces(n), I.uniform_faces(2)
        p = I.Problem(xf=xf, yf=yf, c=c, u=(1.0, 0.0), b=(0, 0, 0.5), alpha=nu, d=(0, 1),
                      dt=I.cfl_dt(xf, xf, c, 0.5))
        xc, yc = p.centres()
        X, _ = np.meshgrid(xc, yc)
        steps = int(round(0.5 / p.dt))
        o = Oracle(p)
        f = o.run(o.init(cole_hopf(X, 0.0, nu)), steps, nthreads)
        errs.append(gre(o.phi(f), cole_hopf(X, steps * p.dt, nu)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-4 and np.all(orders > 1.8), (errs, orders)


# ---------------------------------------------------------------------------
# structure: conservation, fixed points, symmetry
# ---------------------------------------------------------------------------

def test_mass_conservation_periodic_nonlinear(nthreads):
    p, phi0 = I.burgers(48, 40, steps=100)
    o = Oracle(p)
    f0 = o.init(phi0)
    f = o.run(f0, p.steps, nthreads)
    m0 = o.mass(f0)
    assert abs(o.mass(f) - m0) <= 1e-13 * m0


@pytest.mark.parametrize("preset", ["burgers", "nonuniform"])
def test_uniform_state_is_fixed_point(preset):
    p, _ = I.PRESETS[preset](12, 10, steps=5)
    if preset == "nonuniform":
        p = p.with_(bc_value=(0.8,) * 4)
    o = Oracle(p)
    f0 = o.init(np.full((p.ny, p.nx), 0.8))
    f = o.run(f0, 5)
    np.testing.assert_allclose(f, f0, rtol=1e-14, atol=1e-16)


def test_periodic_shift_equivariance():
    # 16 x 8 cells on [0,1]^2: every coordinate and spacing is exact in binary,
    # so a shifted input gives a bitwise-shifted output
    p, phi0 = I.burgers(16, 8, steps=3)
    o = Oracle(p)
    f = o.run(o.init(phi0), 3)
    g = o.run(o.init(np.roll(np.roll(phi0, 3, axis=1), -2, axis=0)), 3)
    np.testing.assert_array_equal(np.roll(np.roll(f, 3, axis=2), -2, axis=1), g)


def test_xy_mirror_symmetry():
    """u = (a, a) and phi0 = phi0^T: the solution stays symmetric under x <-> y,
    velocities mapped by the mirror (1<->2, 3<->4, 6<->8)."""
    p, phi0 = I.burgers(16, 16, steps=4)
    phi0 = 0.5 * (phi0 + phi0.T)
    o = Oracle(p)
    f = o.run(o.init(phi0), 4)
    perm = [0, 2, 1, 4, 3, 5, 8, 7, 6]
    g = np.transpose(f[perm], (0, 2, 1))
    np.testing.assert_allclose(f, g, rtol=1e-14, atol=1e-15)


def test_nonuniform_with_uniform_coordinates_matches_uniform():
    """The same grid given as an explicit face list: identical arithmetic path."""
    p, phi0 = I.burgers(10, 8, steps=3)
    q = p.with_(xf=np.array(list(p.xf)), yf=np.array(list(p.yf)))
    f1 = Oracle(p).run(Oracle(p).init(phi0), 3)
    f2 = Oracle(q).run(Oracle(q).init(phi0), 3)
    np.testing.assert_array_equal(f1, f2)


def test_dirichlet_linear_steady_state():
    """B = 0, D = phi I, Dirichlet 1 / 0.5 on x-walls of a tanh mesh, periodic in
    y: the steady state is the linear profile (exact for the linear
    reconstruction and the mirrored ghost)."""
    xf = I.tanh_faces(16, 2.0)
    yf = I.uniform_faces(2)
    p = I.Problem(xf=xf, yf=yf, bc=(I.DIRICHLET, I.DIRICHLET, I.PERIODIC, I.PERIODIC),
                  bc_value=(1.0, 0.5, 0.0, 0.0), c=1.0, u=(0.0, 0.0), b=(0, 1), alpha=0.1,
                  d=(0, 1), dt=I.cfl_dt(xf, yf, 1.0, 0.5))
    o = Oracle(p)
    xc, _ = p.centres()
    f = o.run(o.init(np.full((2, 16), 0.75)), int(60.0 / p.dt))
    np.testing.assert_allclose(o.phi(f)[0], 1.0 - 0.5 * xc, rtol=0, atol=1e-12)


def test_dirichlet_nonlinear_diffusion_steady_state():
    """D = phi^2 I (the non-uniform workload's diffusion), B = 0: the steady
    state of phi_t = alpha (phi^2)_xx between phi = 1 and 0.5 is
    phi = sqrt(1 - 0.75 x); the discrete one approaches it at second order."""
    errs = []
    for n in (8, 16, 32):
        xf = I.tanh_faces(n, 2.0)
        yf = I.uniform_faces(2)
        p = I.Problem(xf=xf, yf=yf, bc=(I.DIRICHLET, I.DIRICHLET, I.PERIODIC, I.PERIODIC),
                      bc_value=(1.0, 0.5, 0.0, 0.0), c=1.0, u=(0.0, 0.0), b=(0, 1), alpha=0.1,
                      d=(0, 0, 1), dt=I.cfl_dt(xf, yf, 1.0, 0.5))
        o = Oracle(p)
        xc, _ = p.centres()
        f = o.run(o.init(np.full((2, n), 0.75)), int(60.0 / p.dt))
        errs.append(np.abs(o.phi(f)[0] - np.sqrt(1.0 - 0.75 * xc)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.7), (errs, orders)


# ---------------------------------------------------------------------------
# the paper's printed number (soft pin)
# ---------------------------------------------------------------------------

def test_example_4_4_isotropic_gre_same_decade(nthreads):
    g = json.load(open(GOLDEN))["ex44_isotropic_gre"]
    s = g["setting"]
    n = s["n"]
    xf = I.uniform_faces(n, *s["domain"])
    p = I.Problem(xf=xf, yf=xf.copy(), c=s["c"], u=tuple(s["u"]), b=(0, 1), alpha=s["kappa"],
                  d=(0, 1), dt=I.cfl_dt(xf, xf, s["c"], s["cfl"]))
    xc, yc = p.centres()
    X, Y = np.meshgrid(xc, yc)
    phi0 = np.exp(-(X ** 2 + Y ** 2) / (2 * s["sigma0_sq"]))
    o = Oracle(p)
    steps = int(round(s["t_end"] / p.dt))
    f = o.run(o.init(phi0), steps, nthreads)
    ex = gaussian_hill_exact(xc, yc, steps * p.dt, p.u, p.alpha, s2=s["sigma0_sq"], L=2.0, x0=0.0, y0=0.0)
    e = gre(o.phi(f), ex)
    assert g["value"] / 10 < e < g["value"] * 10, e
