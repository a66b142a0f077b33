"""Batched persistent step (dugks_batch_*, through the C ABI): every instance
must equal the single-instance fused step bit for bit (same arithmetic, any
tile shape), the single-instance step being parity-tested against the FP64
oracle; small instances are also checked against the oracle directly."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle  # noqa: E402
from paper_1906_11036_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN_BATCHED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_batched16.npz")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _mixed_set():
    xf = I.tanh_faces(45, 1.5)
    yf = I.uniform_faces(50)
    wall_x = I.Problem(xf=xf, yf=yf, bc=(I.DIRICHLET, I.DIRICHLET, I.PERIODIC, I.PERIODIC),
                       bc_value=(1.2, 0.6, 0.0, 0.0), c=10.0, u=(0.3, -0.2), b=(0.0, 0.0, 0.5), alpha=0.01,
                       d=(0.0, 1.0), dt=I.cfl_dt(xf, yf, 10.0, 0.4))
    xc, yc = wall_x.centres()
    return [I.burgers(64, 64), I.burgers(37, 29), I.burgers(100, 64), I.burgers(130, 33),
            I.nonuniform(45, 50), (wall_x, I.smooth_phi0(xc, yc, seed=4)), I.gaussian_hill(64)]


def _single(p, phi0, steps):
    from paper_1906_11036_gb300.dugks import Solver

    s = Solver(p, precision=32)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(steps)
    f = s.save_state()
    s.sync()
    s.close()
    return f


def _batch(items, steps, autotune=False):
    from paper_1906_11036_gb300.dugks import BatchSolver

    b = BatchSolver([p for p, _ in items])
    for i, (_, phi0) in enumerate(items):
        b.init_phi(i, phi0)
    if autotune:
        b.autotune(8)
    b.step(steps)
    b.sync()
    out = [b.save_state(i) for i in range(len(items))]
    b.sync()
    b.close()
    return out


@pytest.mark.parametrize("steps", [1, 7, 61])
def test_batch_equals_single_instance_bitwise(steps):
    items = _mixed_set()
    got = _batch(items, steps)
    for (p, phi0), f in zip(items, got):
        assert torch.equal(f, _single(p, phi0, steps)), p.name


def test_autotune_restores_state_and_keeps_results():
    items = _mixed_set()[:4]
    a = _batch(items, 20)
    b = _batch(items, 20, autotune=True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_batch_small_instances_vs_oracle():
    items = [I.burgers(24, 24, steps=40), I.burgers(40, 32, steps=40), I.nonuniform(33, 30, steps=40)]
    got = _batch(items, 40)
    for (p, phi0), f in zip(items, got):
        o = Oracle(p)
        ref = o.phi(o.run(o.init(phi0), 40))
        phi = f.double().sum(0).cpu().numpy()
        assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) <= 2e-5


def test_batched_workload_256_instances():
    """The batched workload: 256 periodic instances with sides from {64..512}
    (seed 7), 1000 steps.  16 sampled instances equal their single-instance
    runs bit for bit; every instance conserves mass to FP32 rounding; 16
    instances drawn by inputs.batched_sample() match stored FP64 oracle runs
    (relative L2 over 2048 sample cells <= 2e-5, mass to 2e-5)."""
    from paper_1906_11036_gb300.dugks import BatchSolver

    items = I.batched()
    b = BatchSolver([p for p, _ in items])
    m0 = []
    for i, (_, phi0) in enumerate(items):
        b.init_phi(i, phi0)
    for i in range(len(items)):
        m0.append(b.get_phi(i, mass=True)[1])
    rows, ms = b.autotune(20)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    b.step(1000)
    b.sync()
    t1.record()
    t1.synchronize()
    cells = sum(p.nx * p.ny for p, _ in items)
    print(f"batched 256 instances x 1000 steps: {t0.elapsed_time(t1):.1f} ms, "
          f"{cells * 9 * 1000 / (t0.elapsed_time(t1) / 1e3) / 1e9:.1f} G CVU/s, tile rows {rows}")
    for i in range(len(items)):
        m = b.get_phi(i, mass=True)[1]
        assert abs(m - m0[i]) <= 1e-5 * abs(m0[i])
    # 16 sampled instances against the FP64 oracle's runs (stored by make_batched_oracle.py)
    z = np.load(GOLDEN_BATCHED)
    assert int(z["steps"]) == 1000
    errs = {}
    for i in (int(v) for v in z["ids"]):
        phi, m = b.get_phi(i, mass=True)
        got = phi.double().cpu().numpy().reshape(-1)[z[f"sample_{i}"]]
        ref = z[f"phi_{i}"]
        errs[i] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert abs(m - float(z[f"mass_{i}"])) <= 2e-5 * abs(float(z[f"mass_{i}"]))
    print("batched vs FP64 oracle, rel-L2 per sampled instance:",
          ", ".join(f"{i}:{e:.2e}" for i, e in errs.items()))
    assert max(errs.values()) <= 2e-5
    sample = np.random.default_rng(7).choice(len(items), 16, replace=False)
    states = {int(i): b.save_state(int(i)) for i in sample}
    b.sync()
    b.close()
    for i, f in states.items():
        p, phi0 = items[i]
        assert torch.equal(f, _single(p, phi0, 1000)), p.name
