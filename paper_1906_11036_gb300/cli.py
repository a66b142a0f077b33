"""Command line: advance one of the preset workloads on the GPU.

    python -m paper_1906_11036_gb300.cli --workload nonuniform --n 2048 --steps 5 [--precision 32]
    python -m paper_1906_11036_gb300.cli --workload burgers --n 512 --steps 40 --adjoint 20
    python -m paper_1906_11036_gb300.cli --workload burgers3d --n 128 --steps 5 [--lattice 15]

Builds the library if needed, initialises ftilde = feq(phi0) and runs the
requested number of DUGKS time steps through the C ABI, then prints the
mass and the range of phi.  With --adjoint K it then takes the gradient of
J = 1/2 sum_cells |cell| (phi^N)^2 with respect to phi^0 and alpha by the
checkpointed reverse sweep (a checkpoint every K steps).  Also the command
used for kernel profiles.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1906_11036_gb300.cli")
    from . import inputs as _inputs

    ap.add_argument("--workload", default="nonuniform", choices=sorted(_inputs.PRESETS) + ["burgers3d"])
    ap.add_argument("--lattice", type=int, default=19, choices=[15, 19], help="3-D velocity set")
    ap.add_argument("--n", type=int, default=None, help="cells per side (default: the preset's)")
    ap.add_argument("--steps", type=int, default=None, help="time steps (default: the preset's)")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "naive"])
    ap.add_argument("--adjoint", type=int, default=0, metavar="K",
                    help="also run the reverse sweep, a checkpoint every K steps")
    a = ap.parse_args(argv)

    import torch

    from . import build, inputs
    from .dugks import Solver

    build.build()
    if a.workload == "burgers3d":  # the 3-D step (D3Q15 / D3Q19)
        from .dugks import Solver3

        p, phi0 = inputs.burgers3d(256 if a.n is None else a.n, lattice=a.lattice)
        steps = p.steps if a.steps is None else a.steps
        s = Solver3(p, precision=a.precision)
        s.init_phi(phi0)
        _, m0 = s.get_phi(mass=True)
        t0 = time.perf_counter()
        s.step(steps)
        phi, m = s.get_phi(mass=True)
        info = s.info()
        s.close()
        print(json.dumps({"workload": p.name, "steps": steps, "precision": a.precision, "mass0": m0, "mass": m,
                          "phi_min": float(phi.min()), "phi_max": float(phi.max()),
                          "seconds": time.perf_counter() - t0, "block": info["block_threads"],
                          "grid": list(info["grid"]), "zseg": info["zseg"]}))
        return 0
    maker = inputs.PRESETS[a.workload]
    p, phi0 = maker() if a.n is None else maker(a.n)
    steps = p.steps if a.steps is None else a.steps
    s = Solver(p, precision=a.precision, kernel=a.kernel)
    s.init_phi(torch.tensor(phi0, device="cuda"))
    m0 = s.mass()
    t0 = time.perf_counter()
    s.step(steps)
    phi, m = s.get_phi(mass=True)
    el = time.perf_counter() - t0
    info = s.info()
    out = {"workload": p.name, "steps": steps, "precision": a.precision, "mass0": m0, "mass": m,
           "phi_min": float(phi.min()), "phi_max": float(phi.max()), "seconds": el,
           "block": info["block_threads"], "grid": info["grid_blocks"]}
    if a.adjoint > 0:
        area = torch.tensor(np.outer(np.diff(p.yf), np.diff(p.xf)), device="cuda", dtype=s.dtype)
        t0 = time.perf_counter()
        g0, da = s.gradient(torch.tensor(phi0, device="cuda"), steps, area * phi, checkpoint_every=a.adjoint)
        s.sync()
        out.update({"adjoint_seconds": time.perf_counter() - t0, "grad_phi0_norm": float(g0.double().norm()),
                    "dJ_dalpha": da})
    s.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
