"""GPU parity: the CUDA DUGKS step (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (relative L2 of phi, and of the full ftilde state where noted):
  FP64 GPU mode : 1e-12  (only FMA contraction and summation order differ)
  FP32 mode     : 2e-5   (after the configured steps)
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle  # noqa: E402
from paper_1906_11036_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {64: 1e-12, 32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _solver(p, prec, kernel="auto"):
    from paper_1906_11036_gb300.dugks import Solver

    return Solver(p, precision=prec, kernel=kernel)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _mixed(nx, ny, xwall, ywall, steps, nonuni=True):
    xf = I.tanh_faces(nx, 1.5) if nonuni else I.uniform_faces(nx)
    yf = I.tanh_faces(ny, 1.5) if nonuni else I.uniform_faces(ny)
    bc = ((I.DIRICHLET,) * 2 if xwall else (I.PERIODIC,) * 2) + ((I.DIRICHLET,) * 2 if ywall else (I.PERIODIC,) * 2)
    p = I.Problem(xf=xf, yf=yf, bc=bc, bc_value=(1.2, 0.6, 0.9, 0.7), c=2.0, u=(0.3, -0.2), b=(0.0, 0.0, 0.5),
                  alpha=0.02, d=(0.0, 1.0, 0.5), dt=I.cfl_dt(xf, yf, 2.0, 0.45), steps=steps,
                  name=f"mixed_{nx}x{ny}_{int(xwall)}{int(ywall)}")
    xc, yc = p.centres()
    return p, I.smooth_phi0(xc, yc, seed=nx * 31 + ny)


def _poly(nx, ny, steps):
    """Higher-degree B and D polynomials (the generic equilibrium path)."""
    xf, yf = I.uniform_faces(nx), I.uniform_faces(ny)
    p = I.Problem(xf=xf, yf=yf, c=8.0, u=(0.4, 0.25), b=(0.05, 0.3, 0.2, 0.1, 0.02), alpha=0.01,
                  d=(0.1, 0.6, 0.2, 0.05, 0.01), dt=I.cfl_dt(xf, yf, 8.0, 0.4), steps=steps, name=f"poly_{nx}x{ny}")
    xc, yc = p.centres()
    return p, I.smooth_phi0(xc, yc, seed=5)


CASES = {
    "burgers_70x45": lambda: I.burgers(70, 45, steps=30),
    "nonuniform_77x61": lambda: I.nonuniform(77, 61, steps=30),
    "gaussian_hill_64": lambda: I.gaussian_hill(64, steps=200),
    "mixed_xwall_33x17": lambda: _mixed(33, 17, True, False, 25),
    "mixed_ywall_29x40": lambda: _mixed(29, 40, False, True, 25),
    "burgers_czero_37x23": lambda: (lambda pp: (pp[0].with_(c_zero=True), pp[1]))(I.burgers(37, 23, steps=20)),
    "poly_41x19": lambda: _poly(41, 19, 20),
    "wide_400x9": lambda: I.burgers(400, 9, steps=12),
    "tall_9x300": lambda: I.nonuniform(9, 300, steps=12),
    "strips_330x70": lambda: _mixed(330, 70, True, True, 10),
    "tiny_1x1": lambda: I.burgers(1, 1, steps=5),
    "tiny_1x7": lambda: I.burgers(1, 7, steps=5),
    "tiny_5x3": lambda: I.burgers(5, 3, steps=5),
    "tiny_2x2_walls": lambda: I.nonuniform(2, 2, steps=5),
    "tiny_3x1_walls": lambda: _mixed(3, 1, True, False, 5),
}


@pytest.fixture(scope="module")
def oracle_results():
    cache = {}

    def get(name):
        if name not in cache:
            p, phi0 = CASES[name]()
            o = Oracle(p)
            f = o.run(o.init(phi0), p.steps, 8)
            cache[name] = (p, phi0, f, o.phi(f), o)
        return cache[name]

    return get


@pytest.mark.parametrize("kernel", ["fused", "naive"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_parity_vs_oracle(name, prec, kernel, oracle_results):
    p, phi0, fref, phiref, o = oracle_results(name)
    s = _solver(p, prec, kernel)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(p.steps)
    phi = s.get_phi().double().cpu().numpy()
    f = s.save_state().double().cpu().numpy()
    s.sync()
    s.close()
    assert rel_l2(phi, phiref) <= TOL[prec], rel_l2(phi, phiref)
    assert rel_l2(f, fref) <= TOL[prec] * 5, rel_l2(f, fref)
    if prec == 64:
        assert np.abs(f - fref).max() <= 1e-12 * np.abs(fref).max()


def test_fused_equals_naive_fp64_each_step(oracle_results):
    """One step at a time from the oracle's own state: the kernels and the oracle
    agree per step (no error accumulation hides a one-step bug)."""
    p, phi0, _, _, o = oracle_results("nonuniform_77x61")
    f = o.init(phi0)
    for _ in range(3):
        ref = o.step(f)
        for kernel in ("fused", "naive"):
            s = _solver(p, 64, kernel)
            s.load_state(torch.tensor(f, device="cuda"))
            s.step(1)
            got = s.save_state().cpu().numpy()
            s.close()
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        f = ref


def test_gaussian_hill_fp64_mass_and_closed_form(oracle_results):
    from test_oracle_pins import gaussian_hill_exact, gre

    p, phi0, _, phiref, o = oracle_results("gaussian_hill_64")
    s = _solver(p, 64)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    m0 = s.mass()
    s.step(p.steps)
    phi, m = s.get_phi(mass=True)
    s.close()
    assert abs(m - m0) <= 1e-13 * m0
    xc, yc = p.centres()
    e = gre(phi.cpu().numpy(), gaussian_hill_exact(xc, yc, p.steps * p.dt, p.u, p.alpha))
    e_or = gre(phiref, gaussian_hill_exact(xc, yc, p.steps * p.dt, p.u, p.alpha))
    assert abs(e - e_or) <= 1e-10


def test_fp32_mass_conservation_periodic():
    p, phi0 = I.burgers(256, 192, steps=500)
    s = _solver(p, 32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    m0 = s.mass()
    s.step(p.steps)
    m = s.mass()
    s.close()
    assert abs(m - m0) <= 2e-6 * m0


def test_uniform_state_fixed_point_fp32():
    p, _ = I.burgers(130, 70, steps=50)
    s = _solver(p, 32)
    s.init_phi(torch.full((70, 130), 1.1, device="cuda"))
    s.step(50)
    phi = s.get_phi().double().cpu().numpy()
    s.close()
    assert np.abs(phi - 1.1).max() <= 1e-5


def test_determinism_and_checkpoint_resume():
    p, phi0 = I.nonuniform(190, 150, steps=20)
    s = _solver(p, 32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(20)
    a = s.save_state().clone()
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(8)
    ck = s.save_state().clone()
    s2 = _solver(p, 32)
    s2.load_state(ck)
    s2.step(12)
    b = s2.save_state()
    s.step(12)
    c = s.save_state()
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    s.close()
    s2.close()


def test_host_paths_match_device_paths():
    p, phi0 = I.burgers(96, 80, steps=10)
    s = _solver(p, 32)
    s.init_phi(phi0)  # host path
    s.step(10)
    ph, mh = s.get_phi_host()
    pd, md = s.get_phi(mass=True)
    s.close()
    np.testing.assert_array_equal(ph, pd.double().cpu().numpy())
    assert mh == md


def test_nonfinite_detected():
    from paper_1906_11036_gb300.dugks import DugksError

    p, phi0 = I.burgers(64, 64, steps=3)
    phi0 = phi0.copy()
    phi0[10, 20] = np.nan
    s = _solver(p, 32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(3)
    with pytest.raises(DugksError) as e:
        s.mass()
    assert e.value.status == 4
    s.close()


def test_config_errors():
    from paper_1906_11036_gb300.dugks import DugksError

    p, _ = I.burgers(32, 32)
    with pytest.raises(DugksError) as e:
        _solver(p.with_(dt=p.dt * 10), 32)  # CFL 4
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# full-size workloads, full length, against stored oracle samples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["burgers", "nonuniform"])
def test_full_size_fp32_vs_stored_oracle(name):
    path = os.path.join(GOLDEN, f"oracle_{name}.npz")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    g = np.load(path)
    p, phi0 = I.PRESETS[name]()
    assert (p.nx, p.ny, p.steps) == (int(g["nx"]), int(g["ny"]), int(g["steps"]))
    s = _solver(p, 32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(p.steps)
    phi, m = s.get_phi(mass=True)
    s.close()
    got = phi.double().cpu().numpy().reshape(-1)[g["sample"]]
    err = rel_l2(got, g["phi"])
    print(f"{name}: FP32 rel-L2 vs FP64 oracle over {len(got)} samples after {p.steps} steps: {err:.3e}")
    assert err <= 2e-5
    assert abs(m - float(g["mass"])) <= 2e-5 * abs(float(g["mass"]))


def test_expired_bounded_wait_is_reported_without_a_fault():
    """Failure detection without a GPU fault: a bounded device wait that nothing
    completes expires after ~2 ms, sets the error word, and dugks_sync reports
    DUGKS_ERR_TIMEOUT; the context and the device stay usable."""
    from paper_1906_11036_gb300.dugks import DugksError, Solver

    p, phi0 = I.burgers(40, 30, steps=5)
    s = Solver(p, precision=32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(2)
    s.sync()
    s.wait_timeout_check(2000)
    with pytest.raises(DugksError) as ei:
        s.sync()
    assert ei.value.status == 7  # DUGKS_ERR_TIMEOUT
    s.close()
    t = Solver(p, precision=32)  # a fresh context runs normally afterwards
    t.init_phi(torch.tensor(phi0, device="cuda"))
    t.step(3)
    t.sync()
    t.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_negative_initial_equilibrium_refused_when_checked(prec):
    """With the equilibrium check on, the Burgers form at c = 1 (f^eq down to -0.24)
    is refused: on the host path before any device work, on the device path by the
    next sync.  The same state at c = 10 passes, and with the check off (the default)
    nothing is tested."""
    from paper_1906_11036_gb300.dugks import DugksError, Solver

    p, phi0 = I.burgers(40, 33)
    bad = p.with_(c=1.0, dt=p.dt * 10.0)
    s = Solver(bad, precision=prec)
    s.set_feq_check(True)
    with pytest.raises(DugksError) as ei:
        s.init_phi(phi0)                                   # host path
    assert ei.value.status == 2
    s.init_phi(torch.tensor(phi0, device="cuda"))         # device path
    with pytest.raises(DugksError) as ei:
        s.sync()
    assert ei.value.status == 2
    s.close()
    s = Solver(bad, precision=prec)                        # check off: no test
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.sync()
    s.close()
    s = Solver(p, precision=prec)
    s.set_feq_check(True)
    s.init_phi(phi0)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(3)
    s.sync()
    s.close()
