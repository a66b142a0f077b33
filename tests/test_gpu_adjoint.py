"""GPU adjoint (dugks_adjoint_step / dugks_adjoint, through the C ABI) against
the FP64 oracle's adjoint, which test_oracle_adjoint.py pins to central
finite differences.

Tolerances: FP64 GPU 1e-11 relative (rounding order only); FP32 GPU 1e-4
relative on the gradient (the FP64 accumulation of dJ/dalpha and dJ/du keeps
their error at FP32 rounding of the summands).  The adjoint workload (512^2,
400 steps) is checked against stored FP64 central differences of the oracle
(tests/golden/oracle_adjoint_fd.npz, written by make_adjoint_fd.py there).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle  # noqa: E402
from paper_1906_11036_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _solver(p, prec, adj="auto"):
    from paper_1906_11036_gb300.dugks import Solver

    s = Solver(p, precision=prec)
    s.set_adjoint_kernel(adj)
    return s


def _mixed(xwall, ywall, nx, ny):
    xf = I.tanh_faces(nx, 1.5) if xwall else I.uniform_faces(nx)
    yf = I.tanh_faces(ny, 1.5) if ywall else I.uniform_faces(ny)
    bc = ((I.DIRICHLET,) * 2 if xwall else (I.PERIODIC,) * 2) + ((I.DIRICHLET,) * 2 if ywall else (I.PERIODIC,) * 2)
    return I.Problem(xf=xf, yf=yf, bc=bc, bc_value=(1.2, 0.6, 0.9, 0.7), c=2.0, u=(0.3, -0.2),
                     b=(0.0, 0.0, 0.5), alpha=0.02, d=(0.0, 1.0, 0.5), dt=I.cfl_dt(xf, yf, 2.0, 0.4))


CASES = {
    "burgers_37x23": lambda: I.burgers(37, 23)[0],
    "nonuniform_33x29": lambda: I.nonuniform(33, 29)[0],
    "xwall_21x17": lambda: _mixed(True, False, 21, 17),
    "ywall_19x22": lambda: _mixed(False, True, 19, 22),
    "czero_16x16": lambda: I.burgers(16, 16)[0].with_(c_zero=True),
    "poly_20x13": lambda: I.burgers(20, 13)[0].with_(b=(0.05, 0.3, 0.2, 0.1), d=(0.1, 0.6, 0.2, 0.05)),
    "tiny_3x2": lambda: I.burgers(3, 2)[0],
    "tiny_walls_2x3": lambda: I.nonuniform(2, 3)[0],
    # periodic grids with nx a multiple of 4: FP32 runs the row-marching adjoint
    "periodic_rows_64x37": lambda: I.burgers(64, 37)[0],
    "periodic_rows_124x50": lambda: I.burgers(124, 50)[0],
    "periodic_mixed_40x33": lambda: _mixed(False, False, 40, 33),
    "periodic_rows_8x5": lambda: I.burgers(8, 5)[0],
    # Dirichlet walls with nx a multiple of 4: FP32 runs the row-marching adjoint with ghost folds
    "wallrows_both_64x37": lambda: I.nonuniform(64, 37)[0],
    "wallrows_x_40x33": lambda: _mixed(True, False, 40, 33),
    "wallrows_y_44x30": lambda: _mixed(False, True, 44, 30),
    "wallrows_both_8x5": lambda: I.nonuniform(8, 5)[0],
    "wallrows_both_124x50": lambda: I.nonuniform(124, 50)[0],
    "wallrows_both_poly_36x20": lambda: I.nonuniform(36, 20)[0].with_(b=(0.0, 0.6, 0.3, 0.1)),
}


def _kind(name):
    """The adjoint kernel a case asks for: the row-marching one wherever it applies."""
    return "rows" if name.startswith(("periodic_", "wallrows_")) else "auto"


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_step_matches_oracle(name, prec):
    # periodic and wallrows cases: the row-marching FP32 adjoint, whatever the size
    adj = _kind(name)
    p = CASES[name]()
    rng = np.random.default_rng(len(name))
    o = Oracle(p)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    mu = rng.standard_normal(f.shape)
    lam_ref, da_ref = o.adjoint_step(f, mu)
    s = _solver(p, prec, adj)
    dt = s.dtype
    lam, da = s.adjoint_step(torch.tensor(f, dtype=dt, device="cuda"), torch.tensor(mu, dtype=dt, device="cuda"))
    lam = lam.double().cpu().numpy()
    da = float(da.item())
    s.close()
    tol = 1e-11 if prec == 64 else 2e-5
    assert _rel(lam, lam_ref) <= tol, _rel(lam, lam_ref)
    assert abs(da - da_ref) <= tol * 10 * max(abs(da_ref), 1e-12)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_step_u_derivative_matches_oracle(name, prec):
    """The explicit u-derivative of one step (u of B = u b(phi)): cells, faces,
    ghosts; lam and dJ/dalpha are unchanged by asking for it."""
    adj = _kind(name)
    p = CASES[name]()
    rng = np.random.default_rng(len(name) + 100)
    o = Oracle(p)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    mu = rng.standard_normal(f.shape)
    lam_ref, da_ref, du_ref = o.adjoint_step_full(f, mu)
    s = _solver(p, prec, adj)
    dt = s.dtype
    lam, da, du = s.adjoint_step(torch.tensor(f, dtype=dt, device="cuda"), torch.tensor(mu, dtype=dt, device="cuda"),
                                 with_u=True)
    lam = lam.double().cpu().numpy()
    da, du = float(da.item()), du.cpu().numpy()
    s.close()
    tol = 1e-11 if prec == 64 else 2e-5
    assert _rel(lam, lam_ref) <= tol, _rel(lam, lam_ref)
    assert abs(da - da_ref) <= tol * 10 * max(abs(da_ref), 1e-12)
    scale = max(float(np.abs(du_ref).max()), 1e-12)
    assert np.abs(du - du_ref).max() <= tol * 10 * scale, (du, du_ref)


def test_adjoint_step_without_alpha_returns_the_same_lambda():
    """dj_dalpha = NULL: only lam is formed (no sum); it equals lam of the full call."""
    for name in ("periodic_rows_64x37", "nonuniform_33x29"):
        p = CASES[name]()
        rng = np.random.default_rng(7)
        o = Oracle(p)
        f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
        mu = rng.standard_normal(f.shape)
        s = _solver(p, 32, "rows" if name.startswith("periodic_") else "auto")
        ft = torch.tensor(f, dtype=torch.float32, device="cuda")
        mt = torch.tensor(mu, dtype=torch.float32, device="cuda")
        lam1, _ = s.adjoint_step(ft, mt)
        lam2, none = s.adjoint_step(ft, mt, with_alpha=False)
        s.close()
        assert none is None and torch.equal(lam1, lam2)


def test_u_derivative_with_zero_velocity():
    """u = 0: the step's equilibrium has no b terms, but d feq / d u does (b and
    int b'^2 of higher degree than the step's own polynomial)."""
    p = I.burgers(24, 20)[0].with_(u=(0.0, 0.0), b=(0.0, 0.2, 0.3, 0.1))
    rng = np.random.default_rng(11)
    o = Oracle(p)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    mu = rng.standard_normal(f.shape)
    _, _, du_ref = o.adjoint_step_full(f, mu)
    for prec in (64, 32):
        s = _solver(p, prec)
        _, _, du = s.adjoint_step(torch.tensor(f, dtype=s.dtype, device="cuda"),
                                  torch.tensor(mu, dtype=s.dtype, device="cuda"), with_u=True)
        du = du.cpu().numpy()
        s.close()
        tol = 1e-10 if prec == 64 else 2e-4
        assert np.abs(du - du_ref).max() <= tol * float(np.abs(du_ref).max()), (prec, du, du_ref)


def test_row_marching_and_tiled_fp32_adjoints_agree():
    """On a periodic grid the FP32 adjoint step runs as a row march; the tiled
    kernel computes the same quantities: they agree to FP32 rounding, and both
    match the FP64 oracle."""
    p = I.burgers(256, 200)[0]
    rng = np.random.default_rng(3)
    o = Oracle(p)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    mu = rng.standard_normal(f.shape)
    lam_ref, da_ref = o.adjoint_step(f, mu)
    out = []
    for kind in ("rows", "tiled"):
        s = _solver(p, 32, kind)
        lam, da = s.adjoint_step(torch.tensor(f, dtype=torch.float32, device="cuda"),
                                 torch.tensor(mu, dtype=torch.float32, device="cuda"))
        out.append((lam.double().cpu().numpy(), float(da.item())))
        s.close()
    (lr, dr), (lt, dtl) = out
    assert _rel(lr, lt) <= 1e-5 and abs(dr - dtl) <= 1e-4 * abs(dtl)
    assert _rel(lr, lam_ref) <= 2e-5 and abs(dr - da_ref) <= 2e-4 * abs(da_ref)


def test_row_marching_and_tiled_fp32_adjoints_agree_with_walls():
    """The same cross-check on a tanh mesh with Dirichlet walls on both axes (ghost folds)."""
    p = I.nonuniform(256, 200)[0]
    rng = np.random.default_rng(4)
    o = Oracle(p)
    f = o.init(1.0 + 0.2 * rng.standard_normal((p.ny, p.nx))) + 0.01 * rng.standard_normal((9, p.ny, p.nx))
    mu = rng.standard_normal(f.shape)
    lam_ref, da_ref, du_ref = o.adjoint_step_full(f, mu)
    out = []
    for kind in ("rows", "tiled"):
        s = _solver(p, 32, kind)
        lam, da, du = s.adjoint_step(torch.tensor(f, dtype=torch.float32, device="cuda"),
                                     torch.tensor(mu, dtype=torch.float32, device="cuda"), with_u=True)
        out.append((lam.double().cpu().numpy(), float(da.item()), du.cpu().numpy()))
        s.close()
    (lr, dr, ur), (lt, dtl, ut) = out
    assert _rel(lr, lt) <= 1e-5 and abs(dr - dtl) <= 1e-4 * abs(dtl)
    assert _rel(lr, lam_ref) <= 2e-5 and abs(dr - da_ref) <= 2e-4 * abs(da_ref)
    assert np.abs(ur - du_ref).max() <= 2e-4 * float(np.abs(du_ref).max())


@pytest.mark.parametrize("kind", ["tiled", "rows"])
def test_checkpointed_gradient_with_walls_matches_oracle(kind):
    """The checkpointed FP32 gradient (phi0, alpha, u) on the non-uniform mesh with walls."""
    p, phi0 = I.nonuniform(48, 40, steps=40)
    xc, yc = p.centres()
    area = np.outer(np.diff(p.yf), np.diff(p.xf))
    target = I.smooth_phi0(xc, yc, seed=9)
    gref, daref, duref, _ = Oracle(p).gradient(phi0, p.steps, lambda ph: area * (ph - target), threads=8,
                                               checkpoint_every=10, with_u=True)
    s = _solver(p, 32, kind)
    x0 = torch.tensor(phi0, dtype=torch.float32, device="cuda")
    s.init_phi(x0)
    s.step(p.steps)
    gN = torch.tensor(area * (s.get_phi().double().cpu().numpy() - target), dtype=torch.float32, device="cuda")
    g0, da, du = s.gradient(x0, p.steps, gN, checkpoint_every=10, with_u=True)
    s.close()
    assert _rel(g0.double().cpu().numpy(), gref) <= 1e-4
    assert abs(da - daref) <= 1e-4 * abs(daref)
    assert np.abs(np.asarray(du) - duref).max() <= 1e-4 * float(np.abs(duref).max())


@pytest.mark.parametrize("prec,kind", [(64, "tiled"), (32, "tiled"), (32, "rows")])
def test_checkpointed_gradient_matches_oracle(prec, kind):
    # FP32: the tiled and the row-marching adjoint
    p, phi0 = I.burgers(48, 40, steps=60)
    xc, yc = p.centres()
    area = np.outer(np.diff(p.yf), np.diff(p.xf))
    target = I.burgers_phi0(xc, yc, seed=5)
    gref, daref, phiN_ref = Oracle(p).gradient(phi0, p.steps, lambda phiN: area * (phiN - target), threads=8,
                                               checkpoint_every=20)
    s = _solver(p, prec, kind)
    dt = s.dtype
    s.init_phi(torch.tensor(phi0, dtype=dt, device="cuda"))
    s.step(p.steps)
    phiN = s.get_phi().double().cpu().numpy()
    gN = torch.tensor(area * (phiN - target), dtype=dt, device="cuda")
    g0, da = s.gradient(torch.tensor(phi0, dtype=dt, device="cuda"), p.steps, gN, checkpoint_every=20)
    tol = 1e-10 if prec == 64 else 1e-4
    assert _rel(g0.double().cpu().numpy(), gref) <= tol
    assert abs(da - daref) <= tol * abs(daref)
    # with dJ/du: the same phi0 and alpha gradients, and dJ/du against the oracle's
    g1, da1, du = s.gradient(torch.tensor(phi0, dtype=dt, device="cuda"), p.steps, gN, checkpoint_every=20,
                             with_u=True)
    s.close()
    _, _, duref, _ = Oracle(p).gradient(phi0, p.steps, lambda phiN: area * (phiN - target), threads=8,
                                        checkpoint_every=20, with_u=True)
    assert _rel(g1.double().cpu().numpy(), gref) <= tol and abs(da1 - daref) <= tol * abs(daref)
    assert np.abs(np.asarray(du) - duref).max() <= tol * float(np.abs(duref).max()), (du, duref)


def test_gradient_workspace_reuse_and_growth():
    """dugks_adjoint keeps its workspace in the context: a second call gives the
    same gradient bit for bit, and a longer run (a larger workspace) after a
    shorter one still matches the oracle."""
    p, phi0 = I.burgers(40, 32, steps=30)
    xc, yc = p.centres()
    area = np.outer(np.diff(p.yf), np.diff(p.xf))
    target = I.burgers_phi0(xc, yc, seed=5)
    s = _solver(p, 64)
    x0 = torch.tensor(phi0, dtype=torch.float64, device="cuda")

    def grad(n, k):
        s.init_phi(x0)
        s.step(n)
        gN = torch.tensor(area * (s.get_phi().cpu().numpy() - target), device="cuda")
        return s.gradient(x0, n, gN, checkpoint_every=k, with_u=True)

    a = grad(10, 5)
    b = grad(10, 5)
    assert torch.equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]
    g, da, du = grad(30, 4)
    s.close()
    gref, daref, duref, _ = Oracle(p).gradient(phi0, 30, lambda ph: area * (ph - target), checkpoint_every=4,
                                               with_u=True)
    assert _rel(g.cpu().numpy(), gref) <= 1e-10 and abs(da - daref) <= 1e-10 * abs(daref)
    assert np.abs(np.asarray(du) - duref).max() <= 1e-10 * float(np.abs(duref).max())


def test_autograd_function_and_checkpoint_length_invariance():
    """torch.autograd through the run; the gradient does not depend on the
    checkpoint spacing (recomputation is exact)."""
    from paper_1906_11036_gb300.dugks import Solver, run_fn

    p, phi0 = I.nonuniform(40, 36, steps=25)
    xc, yc = p.centres()
    target = torch.tensor(I.smooth_phi0(xc, yc, seed=9), dtype=torch.float64, device="cuda")
    area = torch.tensor(np.outer(np.diff(p.yf), np.diff(p.xf)), device="cuda")
    s = Solver(p, precision=64)
    Run = run_fn()
    grads = []
    for k in (1, 7, 25):
        x = torch.tensor(phi0, dtype=torch.float64, device="cuda", requires_grad=True)
        al = torch.tensor([p.alpha], dtype=torch.float64, device="cuda", requires_grad=True)
        phiN = Run.apply(x, al, s, p.steps, k)
        J = 0.5 * (area * (phiN - target) ** 2).sum()
        J.backward()
        grads.append((x.grad.cpu().numpy(), float(al.grad.item())))
    s.close()
    gref, daref, _ = Oracle(p).gradient(phi0, p.steps,
                                        lambda phiN: area.cpu().numpy() * (phiN - target.cpu().numpy()))
    for g, da in grads:
        assert _rel(g, gref) <= 1e-10 and abs(da - daref) <= 1e-10 * abs(daref)


GOLDEN_FD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_adjoint_fd.npz")


def test_adjoint_workload_512_fp32_against_stored_fd():
    """The adjoint workload at full size: 512^2 periodic Burgers-type NCDE, 400
    FP32 steps checkpointed every 20; gradient of the L2 misfit to a seeded
    target w.r.t. phi0, alpha and u, against stored FP64 central differences of
    the oracle (eps = 1e-4) along 32 seeded unit directions, in alpha and in
    u_x, u_y, and against the oracle's own adjoint on a fixed sample of cells."""
    if not os.path.exists(GOLDEN_FD):
        pytest.skip(f"{GOLDEN_FD} not generated")
    z = np.load(GOLDEN_FD)
    n, steps = int(z["n"]), int(z["steps"])
    p, phi0, target, area = I.adjoint_workload(n, steps)
    s = _solver(p, 32)
    s.init_phi(torch.tensor(phi0, dtype=torch.float32, device="cuda"))
    s.step(p.steps)
    phiN = s.get_phi().double().cpu().numpy()
    J = 0.5 * float((area * (phiN - target) ** 2).sum())
    gN = torch.tensor(area * (phiN - target), dtype=torch.float32, device="cuda")
    g0, da, du = s.gradient(torch.tensor(phi0, dtype=torch.float32, device="cuda"), p.steps, gN,
                            checkpoint_every=20, with_u=True)
    s.close()
    g0 = g0.double().cpu().numpy()
    dirs = I.unit_directions(phi0.shape, int(z["ndir"]), seed=5)
    gd = np.array([float((g0 * d).sum()) for d in dirs])
    rel_dirs = np.abs(gd - z["fd_dirs"]) / np.abs(z["fd_dirs"])
    rel_alpha = abs(da - float(z["fd_alpha"])) / abs(float(z["fd_alpha"]))
    rel_u = np.abs(np.asarray(du) - z["fd_u"]) / np.abs(z["fd_u"])
    samp = g0.reshape(-1)[z["grad_sample_idx"]]
    rel_samp = _rel(samp, z["grad_sample"])
    print(f"adjoint {n}^2 x {steps} FP32 vs FP64 FD: max rel over {len(dirs)} directions {rel_dirs.max():.2e}, "
          f"dJ/dalpha {rel_alpha:.2e}, dJ/du {rel_u.max():.2e}; vs oracle adjoint on {samp.size} cells "
          f"{rel_samp:.2e}; J {J:.6e} (oracle {float(z['J']):.6e})")
    assert abs(J - float(z["J"])) <= 1e-5 * abs(float(z["J"]))
    assert rel_dirs.max() <= 1e-3
    assert rel_alpha <= 1e-3
    assert rel_u.max() <= 1e-3
    assert rel_samp <= 1e-4
