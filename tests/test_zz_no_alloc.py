"""The allocation-free phi / mass entry point (dugks_phi_mass_noalloc) against
the context-based one (dugks_get_phi), through the C ABI.

The entry point serves callers that cannot allocate device memory, e.g. an
application whose memory pool already holds the GPU's free memory, or code
that must avoid the implicit synchronisation of cudaMalloc/cudaFree.  Its
partial sums live in a fixed array inside the library, shared by all calls,
so two calls in a row on different grids must each match the reference.

The file name sorts after every other test file, so pytest collects it last:
a run with -x that stops at a failure here has already run all other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1906_11036_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1906_11036_gb300 import dugks

    L = dugks.library()
    L.dugks_phi_mass_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.dugks_phi_mass_noalloc.restype = ctypes.c_int
    torch.cuda.set_device(0)
    return L


def _reference_and_state(p, phi0, precision, steps):
    """phi and mass from the context path, plus the state and cell widths the
    allocation-free call needs."""
    from paper_1906_11036_gb300.dugks import Solver

    s = Solver(p, precision=precision)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    s.step(steps)
    phi, mass = s.get_phi(mass=True)
    f = s.save_state()
    s.sync()
    s.close()
    dx = torch.tensor(np.diff(p.xf), dtype=torch.float64, device="cuda")
    dy = torch.tensor(np.diff(p.yf), dtype=torch.float64, device="cuda")
    return phi, mass, f, dx, dy


def _noalloc(L, f, precision, nx, ny, dx, dy, want_phi=True):
    phi = torch.full((ny, nx), float("nan"), dtype=f.dtype, device="cuda") if want_phi else None
    mass = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = L.dugks_phi_mass_noalloc(f.data_ptr(), precision, nx, ny, dx.data_ptr(), dy.data_ptr(),
                                  phi.data_ptr() if want_phi else None, mass.data_ptr(), stream)
    torch.cuda.synchronize()
    return st, phi, float(mass.item())


@pytest.mark.parametrize("precision", [32, 64])
def test_noalloc_matches_context_path_two_calls_in_a_row(lib, precision):
    cases = [I.burgers(300, 200, steps=7), I.nonuniform(77, 61, steps=5)]
    for p, phi0 in cases:  # the second call reuses the shared scratch left by the first
        ref_phi, ref_mass, f, dx, dy = _reference_and_state(p, phi0, precision, p.steps)
        st, phi, mass = _noalloc(lib, f, precision, p.nx, p.ny, dx, dy)
        assert st == 0
        assert torch.equal(phi, ref_phi)
        assert abs(mass - ref_mass) <= 1e-12 * abs(ref_mass)
    # a mass-only call (phi output omitted)
    st, _, mass = _noalloc(lib, f, precision, p.nx, p.ny, dx, dy, want_phi=False)
    assert st == 0 and abs(mass - ref_mass) <= 1e-12 * abs(ref_mass)


def test_noalloc_rejects_bad_requests(lib):
    big = 1 << 13  # 8192 x 8192 cells exceeds the fixed scratch (4096 x 4096)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = dummy.data_ptr()
    assert lib.dugks_phi_mass_noalloc(p, 32, big, big, p, p, None, p, stream) == 5   # too large
    assert lib.dugks_phi_mass_noalloc(None, 32, 4, 4, p, p, None, p, stream) == 1    # null state
    assert lib.dugks_phi_mass_noalloc(p, 16, 4, 4, p, p, None, p, stream) == 1       # bad precision
    assert lib.dugks_phi_mass_noalloc(p, 32, 0, 4, p, p, None, p, stream) == 1       # empty grid
