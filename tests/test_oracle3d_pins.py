"""Pins of the FP64 3-D oracle (D3Q15, Eq. 2.28; D3Q19, Eq. 2.6).

* Eq. 2.3 / Eq. 2.7 moments of the 3-D equilibria, with the lattice tables
  typed here from the paper (they fix directions and weights: the second
  moment needs the fourth-order isotropy of the lattice);
* the exact rational 3-D stepper (``rational_stepper3d.py``) on tiny grids,
  periodic, Dirichlet and non-uniform;
* the plane-wave rate against the slow root of the D3Q19 / D3Q15 BGK
  dispersion relation (Eq. 2.2), approached at second order;
* mass conservation, the uniform fixed point, axis-permutation symmetry and
  a Dirichlet linear steady state.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy.optimize import fsolve

from oracle import Oracle3
from paper_1906_11036_gb300 import inputs as I
from rational_stepper3d import D3Q15, D3Q19, RationalDUGKS3D


def _lattice(q):
    vecs, w = D3Q15 if q == 15 else D3Q19
    return np.array(vecs, float), np.array([float(x) for x in w])


def _p3(n=(4, 4, 4), **kw):
    f = [I.uniform_faces(m) for m in n]
    return I.Problem3(xf=f[0], yf=f[1], zf=f[2], **kw)


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("c,u,b,d", [(1.0, (0.1, 0.05, -0.07), (0.0, 1.0), (0.0, 1.0)),
                                     (10.0, (1.0, 1.0, 1.0), (0.0, 0.0, 0.5), (0.0, 1.0)),
                                     (3.0, (0.4, -0.3, 0.2), (0.2, -0.3, 0.5, 0.25), (1.0, 0.0, 1.0))])
def test_equilibrium_moments_3d(q, c, u, b, d):
    p = _p3(lattice=q, c=c, u=u, b=b, d=d, alpha=0.01, dt=1e-3)
    o = Oracle3(p)
    cv, w = _lattice(q)
    assert abs(w.sum() - 1) < 1e-15
    ci = cv * c
    cs2 = c * c / 3
    bpol = np.polynomial.Polynomial(b)
    cint = (bpol.deriv() ** 2).integ()
    for phi in np.random.default_rng(q).uniform(0.3, 1.7, 5):
        feq = o.equilibrium(phi)
        assert abs(feq.sum() - phi) <= 1e-14
        assert np.allclose(ci.T @ feq, np.array(u) * bpol(phi), atol=1e-13)
        M2 = np.einsum("i,ia,ib->ab", feq, ci, ci)
        expect = cs2 * np.polynomial.Polynomial(d)(phi) * np.eye(3) + np.outer(u, u) * cint(phi)
        assert np.allclose(M2, expect, rtol=1e-13, atol=1e-13)
    # at rest (u = 0, d = phi) the equilibrium is w_i phi: the oracle's weights
    p0 = _p3(lattice=q, c=c, u=(0, 0, 0), b=(0.0, 1.0), d=(0.0, 1.0), alpha=0.01, dt=1e-3)
    assert np.allclose(Oracle3(p0).equilibrium(1.0), w, rtol=1e-15)


# ---------------------------------------------------------------------------
# exact rational arithmetic
# ---------------------------------------------------------------------------

def _rational3(n, bc, bcv, q, c, u, b, alpha, d, dt, nsteps, nonuni, seed):
    rng = np.random.default_rng(seed)
    faces = []
    for m in n:
        if nonuni and m > 1:
            inner = sorted(Fr(int(v), 64) for v in rng.choice(np.arange(1, 64), m - 1, replace=False))
            faces.append([Fr(0)] + inner + [Fr(1)])
        else:
            faces.append([Fr(j, m) for j in range(m + 1)])
    phi0 = [[[Fr(int(rng.integers(50, 150)), 100) for _ in range(n[0])] for _ in range(n[1])] for _ in range(n[2])]
    R = RationalDUGKS3D(faces, bc, bcv, q, c, u, b, alpha, d, dt)
    st = R.init(phi0)
    for _ in range(nsteps):
        st = R.step(st)
    exact = R.to_array(st)
    p = I.Problem3(xf=np.array([float(v) for v in faces[0]]), yf=np.array([float(v) for v in faces[1]]),
                   zf=np.array([float(v) for v in faces[2]]), bc=bc, bc_value=tuple(float(v) for v in bcv),
                   lattice=q, c=float(c), u=tuple(float(v) for v in u), b=tuple(float(v) for v in b),
                   alpha=float(alpha), d=tuple(float(v) for v in d), dt=float(dt))
    o = Oracle3(p)
    f = o.run(o.init(np.array([[[float(v) for v in r] for r in pl] for pl in phi0])), nsteps)
    return f, exact


RATIONAL3 = [
    # n, bc, bc values, lattice, c, u, b, alpha, d, dt, steps, non-uniform
    ((3, 3, 3), (0,) * 6, (0,) * 6, 19, 1, (Fr(1, 10), Fr(1, 20), Fr(-1, 20)), (0, 1), Fr(1, 100), (0, 1),
     Fr(1, 16), 2, False),
    ((3, 2, 3), (0,) * 6, (0,) * 6, 15, 10, (1, Fr(1, 2), Fr(1, 3)), (0, 0, Fr(1, 2)), Fr(1, 200), (0, 1),
     Fr(1, 400), 2, True),
    ((3, 3, 2), (1, 1, 0, 0, 0, 0), (1, Fr(1, 2), 0, 0, 0, 0), 19, 1, (Fr(1, 20), 0, Fr(1, 10)), (0, 1),
     Fr(1, 100), (0, 0, 1), Fr(1, 64), 2, True),
    ((2, 3, 3), (1, 1, 1, 1, 0, 0), (Fr(3, 4), Fr(1, 2), 1, Fr(1, 4), 0, 0), 15, 1, (0, Fr(1, 20), Fr(1, 10)),
     (0, 1), Fr(1, 100), (0, 1), Fr(1, 64), 2, False),
    ((2, 2, 3), (1, 1, 1, 1, 1, 1), (1, Fr(1, 2), Fr(3, 4), Fr(1, 4), Fr(9, 10), Fr(3, 5)), 19, 1,
     (Fr(1, 20), Fr(-1, 20), Fr(1, 30)), (0, 1), Fr(1, 100), (0, 1), Fr(1, 64), 2, True),
]


@pytest.mark.parametrize("case", RATIONAL3, ids=[f"case{i}" for i in range(len(RATIONAL3))])
def test_oracle3_matches_exact_rational_stepper(case):
    f, exact = _rational3(*case, seed=20 + RATIONAL3.index(case))
    assert np.abs(f - exact).max() <= 2e-14 * np.abs(exact).max()


# ---------------------------------------------------------------------------
# kinetic dispersion root, second-order approach
# ---------------------------------------------------------------------------

def _dbe_root3(kvec, u, alpha, c, q):
    """Slow root s of the linearised 3-D discrete-velocity BGK equation for
    B = u phi, C = u u phi, D = phi I: sum_i w_i g_i / (1 + lam s + i lam k.c_i) = 1."""
    cv, w = _lattice(q)
    cs2 = c * c / 3.0
    lam = alpha / cs2
    ci = cv * c
    u = np.asarray(u, float)
    cu = ci @ u
    g = 1 + cu / cs2 + (cu ** 2 - cs2 * (u @ u)) / (2 * cs2 * cs2)
    kc = ci @ np.asarray(kvec)

    def F(z):
        r = np.sum(w * g / (1 + lam * (z[0] + 1j * z[1]) + 1j * lam * kc)) - 1
        return [r.real, r.imag]

    z = fsolve(F, [-alpha * np.dot(kvec, kvec), -np.dot(kvec, u)], xtol=1e-13)
    return z[0] + 1j * z[1]


def _plane_wave_errors(q, ns, nthreads):
    c, alpha, u = 1.0, 0.01, (0.1, 0.05, -0.08)
    kv = np.array([2 * np.pi, 2 * np.pi, 2 * np.pi])
    s_ex = _dbe_root3(kv, u, alpha, c, q)
    errs = []
    for n in ns:
        f = I.uniform_faces(n)
        p = I.Problem3(xf=f, yf=f.copy(), zf=f.copy(), lattice=q, c=c, u=u, b=(0, 1), alpha=alpha, d=(0, 1),
                       dt=I.cfl_dt3(f, f, f, c, 0.5))
        xc, yc, zc = p.centres()
        Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
        ph = kv[0] * X + kv[1] * Y + kv[2] * Z
        o = Oracle3(p)
        s1 = int(round(0.5 / p.dt))
        fs = o.run(o.init(1 + 0.1 * np.cos(ph)), s1, nthreads)
        A1 = np.mean((o.phi(fs) - 1) * np.exp(-1j * ph))
        fs = o.run(fs, s1, nthreads)
        A2 = np.mean((o.phi(fs) - 1) * np.exp(-1j * ph))
        s = np.log(A2 / A1) / (s1 * p.dt)
        errs.append(abs(s - s_ex) / abs(s_ex))
    return np.array(errs)


@pytest.mark.parametrize("q", [19, 15])
def test_plane_wave_rate_converges_to_kinetic_dispersion_3d(q, nthreads):
    errs = _plane_wave_errors(q, (16, 32, 64), nthreads)
    orders = np.log2(errs[:-1] / errs[1:])
    # measured: D3Q19 orders 1.74, 1.87; D3Q15 1.73, 1.86 (rising toward 2)
    assert errs[-1] < 2e-3, errs
    assert orders[-1] > 1.8 and np.all(orders > 1.6), (errs, orders)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q", [15, 19])
def test_mass_conservation_and_fixed_point_3d(q):
    p, phi0 = I.burgers3d(10, 8, 9, lattice=q)
    p = p.with_(xf=I.tanh_faces(10, 1.2))  # non-uniform, still periodic
    o = Oracle3(p)
    f = o.init(phi0)
    m0 = o.mass(f)
    f = o.run(f, 6)
    assert abs(o.mass(f) - m0) <= 1e-13 * abs(m0)
    g = o.init(np.full((9, 8, 10), 0.9))
    assert np.abs(o.run(g, 3) - g).max() <= 1e-15


def test_axis_permutation_symmetry_3d():
    """D3Q19 is closed under the cyclic permutation of the axes; so is the step."""
    p, phi0 = I.burgers3d(6, 5, 4, lattice=19)
    p = p.with_(u=(0.7, -0.4, 0.2))
    q = p.with_(xf=p.zf, yf=p.xf, zf=p.yf, u=(p.u[2], p.u[0], p.u[1]))
    a = Oracle3(p)
    b = Oracle3(q)
    pa = a.phi(a.run(a.init(phi0), 3))
    # new axes x' = z, y' = x, z' = y; arrays are [z][y][x], so new[z'][y'][x'] = old[y][x][z]
    pb = b.phi(b.run(b.init(np.transpose(phi0, (1, 2, 0))), 3))
    assert np.allclose(np.transpose(pa, (1, 2, 0)), pb, rtol=1e-13, atol=1e-14)


def test_dirichlet_linear_steady_state_3d():
    """Linear diffusion (b = 0, d = phi) between Dirichlet walls in x, periodic in y
    and z, on a stretched mesh: the linear profile between the wall values is a
    steady state of the step."""
    n = 12
    xf = I.tanh_faces(n, 1.3)
    f4 = I.uniform_faces(4)
    p = I.Problem3(xf=xf, yf=f4, zf=f4.copy(), bc=(1, 1, 0, 0, 0, 0), bc_value=(1.0, 0.4, 0, 0, 0, 0),
                   lattice=19, c=1.0, u=(0, 0, 0), b=(0.0,), alpha=0.05, d=(0.0, 1.0),
                   dt=I.cfl_dt3(xf, f4, f4, 1.0, 0.5))
    o = Oracle3(p)
    xc = 0.5 * (xf[1:] + xf[:-1])
    lin = 1.0 + (0.4 - 1.0) * xc
    f = o.init(np.broadcast_to(lin, (4, 4, n)).copy())
    f = o.run(f, 50)
    assert np.abs(o.phi(f) - lin[None, None, :]).max() <= 1e-12
