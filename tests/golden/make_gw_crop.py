"""Writes gw_crop_128_order4_100steps.json (classic RK4) or, with the
argument ssprk3, gw_crop_128_order4_100steps_ssprk3.json (low-storage SSPRK3,
integrator type 10): the CPU oracle's 16-field state (Sec. 5 tensor u_ij,
v_ij with the scalar field of Sec. 3.1) after 100 steps of the 128^3
periodic crop of the largest single-GPU workload -- Gaussian psi (k_max = pi/(4 dx), seed 3), Pi = u = v = 0,
4th-order Laplacian and gradients, dx = 1/8, dt = dx/4, eta from 0.1 --
at 64 seeded cells plus four corners, and every field's sum of squares.
Calls only oracle/ and the seeded input generator; the oracle takes about
10 minutes here, which is why the GPU test reads the stored values instead
of recomputing them.

    python tests/golden/make_gw_crop.py [rk4|ssprk3]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gw as ogw  # noqa: E402
from oracle import ssprk3 as ossp  # noqa: E402
from oracle.eom import EOMParams  # noqa: E402
from paper_2404_02950_gb300 import inputs  # noqa: E402

N, DX, ETA0, STEPS, ORDER, SEED = 128, 0.125, 0.1, 100, 4, 3


def sample_cells():
    rng = np.random.default_rng(11)
    idx = [tuple(int(v) for v in rng.integers(0, N, size=3)) for _ in range(64)]
    return idx + [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 7), (N - 1, 5, 0)]


def main(integrator="rk4"):
    dt = DX / 4
    p1, p2, z, _ = inputs.gaussian_field(N, N / 8.0, SEED)
    y = tuple([p1, p2, z, z.copy()] + [np.zeros_like(p1) for _ in range(12)])
    eta = ETA0
    for _ in range(STEPS):
        if integrator == "ssprk3":
            y = ossp.ssprk3_step_periodic(y, eta, dt, DX, EOMParams(order=ORDER), f=ogw.f_periodic)
        else:
            y = ogw.rk4_step_periodic(y, eta, dt, DX, EOMParams(order=ORDER))
        eta += dt
    cells = sample_cells()
    out = {
        "source": ("oracle/ssprk3.py ssprk3_step_periodic with oracle/gw.py f_periodic (SSPRK3, "
                   if integrator == "ssprk3" else "oracle/gw.py rk4_step_periodic (classic RK4, ")
                  + "Sec. 5 tensor source in conformal time), written by tests/golden/make_gw_crop.py",
        "integrator": integrator,
        "n": N, "dx": DX, "eta0": ETA0, "steps": STEPS, "order": ORDER, "seed": SEED,
        "init": "inputs.gaussian_field(n, n/8, seed) for psi1, psi2; Pi = u = v = 0",
        "cells_zyx": [list(c) for c in cells],
        "values": [[float(y[c][cz, cy, cx]) for c in range(16)] for cz, cy, cx in cells],
        "sumsq": [float(np.sum(np.asarray(y[c], dtype=np.float64) ** 2)) for c in range(16)],
    }
    name = "gw_crop_128_order4_100steps" + ("_ssprk3" if integrator == "ssprk3" else "") + ".json"
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), name), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "rk4")
