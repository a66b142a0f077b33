"""The 3-D step (dugks_3d_*, D3Q15 / D3Q19, through the C ABI) against the
FP64 3-D oracle, which test_oracle3d_pins.py pins to an exact rational
stepper and to the 3-D kinetic dispersion root.

Tolerances as in 2-D: FP64 rel-L2 1e-12, FP32 rel-L2 2e-5 (phi and ftilde)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle3  # noqa: E402
from paper_1906_11036_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _walls(n, q, bc, stretched=True):
    faces = [I.tanh_faces(m, 1.4) if stretched else I.uniform_faces(m) for m in n]
    p = I.Problem3(xf=faces[0], yf=faces[1], zf=faces[2], bc=bc, bc_value=(1.2, 0.6, 0.9, 0.7, 1.1, 0.8),
                   lattice=q, c=4.0, u=(0.3, -0.2, 0.15), b=(0.0, 1.0), alpha=0.02, d=(0.0, 0.0, 1.0),
                   dt=I.cfl_dt3(*faces, 4.0, 0.4))
    xc, yc, zc = p.centres()
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return p, 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y) * np.cos(3 * Z)


CASES = {
    "d3q19_periodic_20x17x23": lambda: I.burgers3d(20, 17, 23, lattice=19),
    "d3q15_periodic_33x29x12": lambda: I.burgers3d(33, 29, 12, lattice=15),
    "d3q19_walls_35x18x16": lambda: _walls((35, 18, 16), 19, (1,) * 6),
    "d3q15_mixed_31x16x9": lambda: _walls((31, 16, 9), 15, (1, 1, 0, 0, 1, 1)),
    "d3q19_mixed_uniform_64x15x10": lambda: _walls((64, 15, 10), 19, (0, 0, 1, 1, 0, 0), stretched=False),
    "d3q19_degree5_24x20x10": lambda: (lambda pp: (pp[0].with_(b=(0.0, 0.2, 0.1, 0.3)), pp[1]))(I.burgers3d(24, 20, 10)),
    "tiny_3x2x2_walls": lambda: _walls((3, 2, 2), 19, (1,) * 6, stretched=False),
    "tiny_1x3x2_periodic": lambda: I.burgers3d(1, 3, 2, lattice=15),
    # nx a multiple of 4: the FP32 step runs the face-halves kernel (TMA-staged)
    "d3q15_periodic_32x29x12": lambda: I.burgers3d(32, 29, 12, lattice=15),
    "d3q19_walls_36x18x16": lambda: _walls((36, 18, 16), 19, (1,) * 6),
    "d3q15_walls_28x16x9": lambda: _walls((28, 16, 9), 15, (1,) * 6),
    "d3q15_mixed_uniform_40x23x11": lambda: _walls((40, 23, 11), 15, (0, 0, 1, 1, 1, 1), stretched=False),
    "d3q19_mixed_60x21x13": lambda: _walls((60, 21, 13), 19, (1, 1, 0, 0, 1, 1)),
    "d3q15_periodic_72x64x40": lambda: I.burgers3d(72, 64, 40, lattice=15),
    "tiny_4x2x2_walls": lambda: _walls((4, 2, 2), 19, (1,) * 6, stretched=False),
    "tiny_4x1x3_periodic": lambda: I.burgers3d(4, 1, 3, lattice=15),
    "d3q15_degree5_32x20x10": lambda: (lambda pp: (pp[0].with_(b=(0.0, 0.2, 0.1, 0.3)), pp[1]))(
        I.burgers3d(32, 20, 10, lattice=15)),
}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run3(p, phi0, prec, steps):
    from paper_1906_11036_gb300.dugks import Solver3

    s = Solver3(p, precision=prec)
    s.init_phi(phi0)
    s.step(steps)
    phi, mass = s.get_phi(mass=True)
    f = s.save_state()
    s.sync()
    out = (phi.double().cpu().numpy(), f.double().cpu().numpy(), mass, s.info())
    s.close()
    return out


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_3d_matches_oracle(name, prec):
    p, phi0 = CASES[name]()
    steps = 10
    o = Oracle3(p)
    fr = o.run(o.init(phi0), steps)
    phi, f, mass, _ = _run3(p, phi0, prec, steps)
    tol = 1e-12 if prec == 64 else 2e-5
    assert _rel(phi, o.phi(fr)) <= tol, _rel(phi, o.phi(fr))
    assert _rel(f, fr) <= tol, _rel(f, fr)
    assert abs(mass - o.mass(fr)) <= 1e2 * tol * abs(o.mass(fr))


def test_3d_128_cubed_fp32_against_oracle_and_mass(nthreads):
    """A 128^3 D3Q19 periodic Burgers-type run (several CTAs per axis, many z
    segments), 6 FP32 steps, against the oracle; mass conserved to FP32 rounding."""
    p, phi0 = I.burgers3d(128, lattice=19)
    o = Oracle3(p)
    fr = o.run(o.init(phi0), 6, nthreads)
    phi, _, mass, info = _run3(p, phi0, 32, 6)
    print(f"3-D 128^3 FP32: rel-L2(phi) {_rel(phi, o.phi(fr)):.2e}, grid {info['grid']}, zseg {info['zseg']}")
    assert _rel(phi, o.phi(fr)) <= 2e-5
    m0 = o.mass(o.init(phi0))
    assert abs(mass - m0) <= 1e-5 * abs(m0)


def test_3d_save_load_restart_is_exact():
    from paper_1906_11036_gb300.dugks import Solver3

    p, phi0 = I.burgers3d(24, 20, 16, lattice=19)
    s = Solver3(p, precision=32)
    s.init_phi(phi0)
    s.step(7)
    ref = s.get_phi().clone()
    s.init_phi(phi0)
    s.step(3)
    f3 = s.save_state().clone()
    s.step(2)
    s.load_state(f3)
    s.step(4)
    got = s.get_phi()
    s.sync()
    assert torch.equal(got, ref)
    s.close()
