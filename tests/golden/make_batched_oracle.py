"""Write stored oracle results for 16 sampled instances of the batched workload.

The batched workload is 256 periodic Burgers-type instances with sides from
{64, 128, 256, 512} (seed 7) advanced 1000 steps.  Running the FP64 CPU oracle
on all of them inside a test is too slow, so this script runs it once on 16
instances drawn by ``inputs.batched_sample()`` and stores, per instance, phi at
seeded sample cells and the mass in ``tests/golden/oracle_batched16.npz``.  It
calls only ``oracle/`` and the seeded input generators.

    python tests/golden/make_batched_oracle.py --threads 8
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

NSAMPLE = 2048


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--steps", type=int, default=1000)
    a = ap.parse_args()
    t0 = time.time()
    items = I.batched(steps=a.steps)
    ids = I.batched_sample()
    rng = np.random.default_rng(11)
    out = {"ids": np.asarray(ids), "steps": a.steps}
    for i in ids:
        p, phi0 = items[i]
        o = Oracle(p)
        f0 = o.init(phi0)
        f = o.run(f0, a.steps, a.threads)
        phi = o.phi(f).reshape(-1)
        idx = np.sort(rng.choice(phi.size, size=min(NSAMPLE, phi.size), replace=False))
        out[f"sample_{i}"] = idx
        out[f"phi_{i}"] = phi[idx]
        out[f"mass0_{i}"] = o.mass(f0)
        out[f"mass_{i}"] = o.mass(f)
        out[f"side_{i}"] = p.nx
        print(f"instance {i} ({p.nx}^2): {time.time() - t0:.0f} s", flush=True)
    out["seconds"] = time.time() - t0
    out["threads"] = a.threads
    path = os.path.join(HERE, "oracle_batched16.npz")
    np.savez_compressed(path, **out)
    print(f"{path}: {len(ids)} instances, {a.steps} steps, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
