"""The stored oracle results under tests/golden, checked on the CPU.

Each file is written by a committed script there that calls only the oracle.
These tests check that the cheap ones still match the oracle as it stands
(re-running it), and that the expensive adjoint file is consistent with
itself: its stored FP64 central differences of the misfit (eps = 1e-4, 32
seeded directions, alpha and u) agree with the oracle's adjoint gradient
stored beside them, which pins the oracle's adjoint on the full adjoint
workload (512^2, 400 steps).
"""
import os

import numpy as np

from oracle import Oracle
from paper_1906_11036_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_gaussian_hill_run_matches_oracle():
    z = np.load(os.path.join(GOLDEN, "oracle_gaussian_hill.npz"))
    p, phi0 = I.gaussian_hill()
    o = Oracle(p)
    phi = o.phi(o.run(o.init(phi0), p.steps)).reshape(-1)[z["sample"]]
    np.testing.assert_allclose(phi, z["phi"], rtol=1e-13, atol=1e-15)


def test_batched_sample_small_instances_match_oracle():
    z = np.load(os.path.join(GOLDEN, "oracle_batched16.npz"))
    assert list(z["ids"]) == I.batched_sample()
    items = I.batched(steps=int(z["steps"]))
    small = [int(i) for i in z["ids"] if int(z[f"side_{int(i)}"]) == 64]
    assert small
    for i in small:
        p, phi0 = items[i]
        o = Oracle(p)
        f = o.run(o.init(phi0), int(z["steps"]), 4)
        np.testing.assert_allclose(o.phi(f).reshape(-1)[z[f"sample_{i}"]], z[f"phi_{i}"], rtol=1e-12, atol=1e-14)
        assert abs(o.mass(f) - float(z[f"mass_{i}"])) <= 1e-12 * abs(float(z[f"mass_{i}"]))


def test_adjoint_fd_file_is_consistent():
    z = np.load(os.path.join(GOLDEN, "oracle_adjoint_fd.npz"))
    assert (int(z["n"]), int(z["steps"]), int(z["ndir"]), float(z["eps"])) == (512, 400, 32, 1e-4)
    rel = np.abs(z["fd_dirs"] - z["adjoint_dirs"]) / np.abs(z["fd_dirs"])
    assert rel.max() <= 1e-6
    assert abs(float(z["fd_alpha"]) - float(z["adjoint_alpha"])) <= 1e-6 * abs(float(z["fd_alpha"]))
    np.testing.assert_allclose(z["adjoint_u"], z["fd_u"], rtol=1e-6)
