"""Write stored central differences of the adjoint workload's misfit.

The adjoint workload (512^2 periodic Burgers-type NCDE, 400 steps, misfit
J = 1/2 sum |V| (phi^N - phi_target)^2) is checked against FP64 central
differences (eps = 1e-4) of J along 32 seeded unit directions in phi0, and with
respect to alpha and the velocity u of B = u b(phi).  Each difference takes two
full oracle runs, too slow for a test, so this script computes them once with
the FP64 CPU oracle and stores them in ``tests/golden/oracle_adjoint_fd.npz``,
together with the oracle's own adjoint gradient along the same directions.  It
calls only ``oracle/`` and the seeded input generators.

    python tests/golden/make_adjoint_fd.py --threads 8
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from paper_1906_11036_gb300 import inputs as I  # noqa: E402

EPS = 1e-4
NDIR = 32


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--steps", type=int, default=400)
    a = ap.parse_args()
    t0 = time.time()
    p, phi0, target, area = I.adjoint_workload(a.n, a.steps)

    def J(q, ph0):
        o = Oracle(q)
        ph = o.phi(o.run(o.init(ph0), q.steps, a.threads))
        return 0.5 * float((area * (ph - target) ** 2).sum())

    o = Oracle(p)
    g, dalpha, du, phiN = o.gradient(phi0, p.steps, lambda ph: area * (ph - target), threads=a.threads,
                                     checkpoint_every=20, with_u=True)
    j0 = 0.5 * float((area * (phiN - target) ** 2).sum())
    dirs = I.unit_directions(phi0.shape, NDIR, seed=5)
    fd = np.array([(J(p, phi0 + EPS * d) - J(p, phi0 - EPS * d)) / (2 * EPS) for d in dirs])
    adj = np.array([float((g * d).sum()) for d in dirs])
    ea = EPS * p.alpha
    fd_alpha = (J(p.with_(alpha=p.alpha + ea), phi0) - J(p.with_(alpha=p.alpha - ea), phi0)) / (2 * ea)
    fd_u = []
    for k in range(2):
        up, um = list(p.u), list(p.u)
        up[k] += EPS
        um[k] -= EPS
        fd_u.append((J(p.with_(u=tuple(up)), phi0) - J(p.with_(u=tuple(um)), phi0)) / (2 * EPS))
    out = os.path.join(HERE, "oracle_adjoint_fd.npz")
    np.savez_compressed(out, n=a.n, steps=a.steps, eps=EPS, ndir=NDIR, J=j0, fd_dirs=fd, adjoint_dirs=adj,
                        fd_alpha=fd_alpha, adjoint_alpha=dalpha, fd_u=np.array(fd_u), adjoint_u=np.asarray(du),
                        grad_sample_idx=np.arange(0, phi0.size, 97), grad_sample=g.reshape(-1)[::97],
                        seconds=time.time() - t0, threads=a.threads)
    rel = np.abs(fd - adj) / np.abs(fd)
    print(f"{out}: J = {j0:.6e}, max rel |FD - adjoint| over {NDIR} directions {rel.max():.2e}, "
          f"dJ/dalpha FD {fd_alpha:.6e} adjoint {dalpha:.6e}, dJ/du FD {fd_u} adjoint {list(du)}, "
          f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
