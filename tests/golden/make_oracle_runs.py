"""Write stored oracle results for the full-size, full-length workloads.

The FP64 CPU oracle is too slow to run 2048^2 x 5000 steps inside a test, so
this script runs it once and stores phi at seeded sample cells (plus the
mass) in ``tests/golden/oracle_<workload>.npz``.  It calls only ``oracle/``
and the seeded input generators; no value comes from the CUDA path.

    python tests/golden/make_oracle_runs.py burgers nonuniform --threads 8
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

NSAMPLE = 16384


def sample_cells(ny: int, nx: int, seed: int = 11):
    rng = np.random.default_rng(seed)
    flat = rng.choice(ny * nx, size=min(NSAMPLE, ny * nx), replace=False)
    return np.sort(flat)


def run(name: str, threads: int) -> str:
    p, phi0 = I.PRESETS[name]()
    o = Oracle(p)
    t0 = time.time()
    f0 = o.init(phi0)
    m0 = o.mass(f0)
    f = o.run(f0, p.steps, threads)
    el = time.time() - t0
    phi = o.phi(f)
    idx = sample_cells(p.ny, p.nx)
    out = os.path.join(HERE, f"oracle_{name}.npz")
    np.savez_compressed(out, name=name, nx=p.nx, ny=p.ny, steps=p.steps, sample=idx,
                        phi=phi.reshape(-1)[idx], mass0=m0, mass=o.mass(f),
                        phi_l2=float(np.sqrt(np.sum(phi * phi))), seconds=el, threads=threads)
    return f"{out}: {p.nx}x{p.ny}, {p.steps} steps, {el:.0f} s"


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+", choices=sorted(I.PRESETS))
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    a = ap.parse_args()
    for n in a.names:
        print(run(n, a.threads), flush=True)
