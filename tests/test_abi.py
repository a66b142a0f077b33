"""The C ABI library loads, exports every symbol the header declares, and its
host-only validation behaves as documented (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1906_11036_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1906_11036_gb300 import build
    from paper_1906_11036_gb300 import dugks

    build.build()
    return dugks.library()


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(dugks_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("dugks_create", "dugks_step", "dugks_get_phi", "dugks_init_phi", "dugks_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code in range(8):
        assert lib.dugks_status_string(code)
    assert lib.dugks_status_string(99) == b"unknown status"


def _status(p):
    from paper_1906_11036_gb300 import dugks

    return dugks.check_config(p)


def test_check_config_accepts_the_workloads(lib):
    for name in ("gaussian_hill", "burgers", "nonuniform"):
        p, _ = I.PRESETS[name](16, 12) if name != "gaussian_hill" else I.PRESETS[name](16)
        assert _status(p) == 0, name


def test_check_config_rejects(lib):
    p, _ = I.burgers(16, 12)
    assert _status(p.with_(dt=p.dt * 3)) == 2              # CFL >= 1
    assert _status(p.with_(alpha=0.0)) == 2                # lambda <= 0
    assert _status(p.with_(alpha=float("nan"))) == 2
    assert _status(p.with_(c=-1.0)) == 2
    xf = p.xf.copy()
    xf[3] = xf[2]
    assert _status(p.with_(xf=xf)) == 2                    # zero-width cell
    assert _status(p.with_(bc=(I.PERIODIC, I.DIRICHLET, I.PERIODIC, I.PERIODIC))) == 1
    with pytest.raises(ValueError):
        _status(p.with_(b=tuple(range(9))))                # more than 8 coefficients
    assert _status(p.with_(xf=np.array([0.0]))) == 1       # nx = 0


def test_check_feq_rejects_a_negative_equilibrium(lib):
    """Eq. 2.3 turns negative for large |B|/c: the Burgers workload's form at c = 1
    (f^eq down to -0.24 for phi in its range) is refused, at c = 10 accepted."""
    from paper_1906_11036_gb300.dugks import check_feq

    p, phi0 = I.burgers(32, 24)
    lo, hi = float(phi0.min()), float(phi0.max())
    st, fmin = check_feq(p, lo, hi)
    assert st == 0 and fmin > 0.0
    st, fmin = check_feq(p.with_(c=1.0), lo, hi)
    assert st == 2 and fmin < -0.1
    # the rest velocity's equilibrium with b = phi, d = phi: w0 phi (1 - 3|u|^2/(2c^2)), written out
    q = I.gaussian_hill(16)[0]
    st, fmin = check_feq(q, 0.0, 1.0)
    assert st == 0 and abs(fmin) < 1e-12          # f^eq(0) = 0 is the minimum
    st, fmin = check_feq(q, -1.0, 1.0)
    assert st == 2 and fmin < 0.0                  # negative phi: negative equilibrium
    assert check_feq(q, 1.0, 0.0)[0] == 1          # phi_min > phi_max


def test_check_feq_accepts_marginal_negativity_of_the_nonuniform_workload(lib):
    """With D = phi^2 the diagonal equilibria vanish at phi = 1/2 up to the advective
    term, so the non-uniform workload's f^eq dips to about -2e-4: within the 1e-3
    relative margin of the rule."""
    from paper_1906_11036_gb300.dugks import check_feq

    p, phi0 = I.nonuniform(32)
    st, fmin = check_feq(p, 0.5, 1.5)
    assert st == 0 and -5e-4 < fmin < 0.0
    # the value at phi = 1/2 written out: w_diag [3 (e.u)/c phi + (9 (e.u)^2 - 3|u|^2)/(2c^2) phi] for e.u = -u_x
    ux, c = p.u[0], p.c
    expect = (1.0 / 36.0) * (3.0 * (-ux) / c * 0.5 + (9.0 * ux * ux - 3.0 * ux * ux) / (2.0 * c * c) * 0.5)
    assert abs(fmin - expect) < 1e-12
