"""Pins of the oracle's hand-written adjoint (reverse mode of one DUGKS step)
against central finite differences of the oracle's own forward step.

The adjoint is what the GPU adjoint kernel is compared with, so it is pinned
here independently of its code:
  * d feq / d phi against central differences of Eq. 2.3;
  * the dot-product identity <J v, w> = <v, J^T w> for random v, w, with J v
    by central differences, on periodic, Dirichlet and mixed grids, uniform
    and stretched, with C = 0 and with higher-degree B, D;
  * the explicit alpha-derivative against central differences in alpha;
  * the gradient of J = 1/2 sum |V| (phi^N - phi_t)^2 over many steps with
    respect to phi0 (random directions) and alpha, against central
    differences of J (eps = 1e-4, FP64);
  * d feq / d u and the explicit u-derivative of the step (u of B = u b(phi):
    the B coefficients of Eq. 2.3), and dJ/du over many steps, the same way.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1906_11036_gb300 import inputs as I


def _mixed(xwall, ywall, nx=6, ny=5):
    xf = I.tanh_faces(nx, 1.5) if xwall else I.uniform_faces(nx)
    yf = I.tanh_faces(ny, 1.5) if ywall else I.uniform_faces(ny)
    bc = ((I.DIRICHLET,) * 2 if xwall else (I.PERIODIC,) * 2) + ((I.DIRICHLET,) * 2 if ywall else (I.PERIODIC,) * 2)
    return I.Problem(xf=xf, yf=yf, bc=bc, bc_value=(1.2, 0.6, 0.9, 0.7), c=2.0, u=(0.3, -0.2),
                     b=(0.0, 0.0, 0.5), alpha=0.02, d=(0.0, 1.0, 0.5), dt=I.cfl_dt(xf, yf, 2.0, 0.4))


CASES = {
    "burgers_periodic": lambda: I.burgers(7, 5)[0],
    "nonuniform_walls": lambda: I.nonuniform(6, 7)[0],
    "xwall": lambda: _mixed(True, False),
    "ywall": lambda: _mixed(False, True),
    "czero": lambda: I.burgers(6, 6)[0].with_(c_zero=True),
    "poly": lambda: I.burgers(5, 6)[0].with_(b=(0.05, 0.3, 0.2, 0.1), d=(0.1, 0.6, 0.2, 0.05)),
    "gaussian_hill": lambda: I.gaussian_hill(8)[0],
}


def test_equilibrium_derivative_matches_central_differences():
    for name in ("burgers_periodic", "nonuniform_walls", "poly"):
        o = Oracle(CASES[name]())
        for phi in (0.4, 1.0, 1.7):
            fd = (o.equilibrium(phi + 1e-6) - o.equilibrium(phi - 1e-6)) / 2e-6
            np.testing.assert_allclose(o.equilibrium_deriv(phi), fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_step_dot_product_and_alpha(name):
    p = CASES[name]()
    o = Oracle(p)
    rng = np.random.default_rng(abs(hash(name)) % 2 ** 32)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    v = rng.standard_normal(f.shape)
    w = rng.standard_normal(f.shape)
    eps = 1e-6
    jv = (o.step(f + eps * v) - o.step(f - eps * v)) / (2 * eps)
    lam, dalpha = o.adjoint_step(f, w)
    lhs, rhs = float((jv * w).sum()), float((v * lam).sum())
    assert abs(lhs - rhs) <= 1e-8 * max(abs(lhs), 1.0)
    ea = 1e-6 * p.alpha
    fa = Oracle(p.with_(alpha=p.alpha + ea)).step(f)
    fb = Oracle(p.with_(alpha=p.alpha - ea)).step(f)
    ja = float((((fa - fb) / (2 * ea)) * w).sum())
    assert abs(ja - dalpha) <= 1e-6 * max(abs(ja), 1.0)


def test_multi_step_gradient_against_central_differences():
    """The reduced adjoint workload: Burgers-type NCDE, misfit to a seeded target,
    gradient with respect to phi0 (random directions) and alpha."""
    p, phi0 = I.burgers(16, 12, steps=30)
    xc, yc = p.centres()
    area = np.outer(np.diff(p.yf), np.diff(p.xf))
    target = I.burgers_phi0(xc, yc, seed=5)

    def J(phi0_, alpha_):
        o_ = Oracle(p.with_(alpha=alpha_))
        phiN = o_.phi(o_.run(o_.init(phi0_), p.steps))
        return 0.5 * float((area * (phiN - target) ** 2).sum())

    o = Oracle(p)
    gphi, galpha, _ = o.gradient(phi0, p.steps, lambda phiN: area * (phiN - target))
    rng = np.random.default_rng(5)
    eps = 1e-4
    for _ in range(4):
        d = rng.standard_normal(phi0.shape)
        d /= np.linalg.norm(d)
        fd = (J(phi0 + eps * d, p.alpha) - J(phi0 - eps * d, p.alpha)) / (2 * eps)
        assert abs(fd - float((gphi * d).sum())) <= 1e-6 * max(abs(fd), 1e-12)
    ea = eps * p.alpha
    fda = (J(phi0, p.alpha + ea) - J(phi0, p.alpha - ea)) / (2 * ea)
    assert abs(fda - galpha) <= 1e-6 * abs(fda)


def test_equilibrium_u_derivative_matches_central_differences():
    """d feq / d u (B = u b(phi), C = u u int b'^2) against central differences of Eq. 2.3 in u."""
    for name in ("burgers_periodic", "nonuniform_walls", "poly", "xwall", "czero"):
        p = CASES[name]()
        o = Oracle(p)
        for phi in (0.4, 1.0, 1.7):
            got = o.equilibrium_du(phi)
            for a in range(2):
                up, um = list(p.u), list(p.u)
                up[a] += 1e-6
                um[a] -= 1e-6
                fd = (Oracle(p.with_(u=tuple(up))).equilibrium(phi) - Oracle(p.with_(u=tuple(um))).equilibrium(phi)) / 2e-6
                np.testing.assert_allclose(got[a], fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_step_u_derivative(name):
    """The explicit u-derivative of one step, contracted with w, against central
    differences of the forward step in u (cells, faces and ghosts all depend on u)."""
    p = CASES[name]()
    o = Oracle(p)
    rng = np.random.default_rng(abs(hash(name + "u")) % 2 ** 32)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    w = rng.standard_normal(f.shape)
    _, _, du = o.adjoint_step_full(f, w)
    for a in range(2):
        up, um = list(p.u), list(p.u)
        up[a] += 1e-6
        um[a] -= 1e-6
        fa = Oracle(p.with_(u=tuple(up))).step(f)
        fb = Oracle(p.with_(u=tuple(um))).step(f)
        ju = float((((fa - fb) / 2e-6) * w).sum())
        assert abs(ju - du[a]) <= 1e-6 * max(abs(ju), 1.0), (a, ju, du[a])


def test_multi_step_u_gradient_against_central_differences():
    """dJ/du of the reduced adjoint workload (the initial f^0 = feq(phi0) depends on u
    as well as every step) against central differences of J in u_x and u_y."""
    p, phi0 = I.burgers(16, 12, steps=30)
    xc, yc = p.centres()
    area = np.outer(np.diff(p.yf), np.diff(p.xf))
    target = I.burgers_phi0(xc, yc, seed=5)

    def J(q):
        o_ = Oracle(q)
        phiN = o_.phi(o_.run(o_.init(phi0), q.steps))
        return 0.5 * float((area * (phiN - target) ** 2).sum())

    _, _, du, _ = Oracle(p).gradient(phi0, p.steps, lambda phiN: area * (phiN - target), with_u=True)
    for a in range(2):
        up, um = list(p.u), list(p.u)
        up[a] += 1e-4
        um[a] -= 1e-4
        fd = (J(p.with_(u=tuple(up))) - J(p.with_(u=tuple(um)))) / 2e-4
        assert abs(fd - du[a]) <= 1e-6 * abs(fd), (a, fd, du[a])
