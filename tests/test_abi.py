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
