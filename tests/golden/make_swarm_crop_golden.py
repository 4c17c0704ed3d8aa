"""Write the FP64 oracle's result for the dispersed-swarm crop (tests/golden).

Workload: the 64x64x128 crop of the 384x384x768 swarm (Sec. 4 bubble column,
shaped as a dispersed swarm): omega 1.7, half-way bounce-back on all six faces,
g = 1e-5, 463 bubbles (100,000 scaled by volume) with lognormal diameters of
mean 1.5 and standard deviation 0.3, centres uniform in the bottom 20 %,
released at rest, seed 1234.  The oracle runs Algorithm 1 for 3000 steps.

Stored (``swarm_crop_64x64x128.npz``):

* ``u1000``, ``u3000``: bare Eq. 10 velocity [3, 64, 32, 32] on the even
  sublattice (every other node along each axis, 65,536 nodes), float32;
* ``drho3000``: rho - 1 on the same sublattice, float32;
* ``pos1000``, ``pos3000``, ``vel3000``: bubble centres and velocities,
  float64 [463, 3]; ``active3000``: whether each bubble is still coupled;
* ``ubz_last200``: mean u_b,z over all bubbles after each of steps
  2801..3000, float64 (its mean is the terminal rise velocity).

float32 keeps 6e-8 of each value, far below the tolerances the tests use.
Only ``oracle`` and the seeded input generators are imported.

Run from the repository root:  python tests/golden/make_swarm_crop_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import bubble as obub          # noqa: E402
from oracle.step import OracleSim          # noqa: E402
from paper_1710_07073_gb300 import workloads as wl   # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "swarm_crop_64x64x128.npz")
DIMS = wl.SWARM_CROP
OMEGA = 1.7
STEPS = 3000
WINDOW = 200


def main():
    count = wl.swarm_count_for_crop(wl.SWARM_FULL, 100_000, DIMS)
    pos, vel, diam = wl.swarm(DIMS, count, seed=1234)
    sim = OracleSim(DIMS, OMEGA, 0x3F, obub.BubbleParams(OMEGA, g=1e-5))
    sim.set_bubbles(pos, vel, diam)
    out = {}
    ubz = []
    t0 = time.time()
    for step in range(1, STEPS + 1):
        sim.step()
        if step > STEPS - WINDOW:
            ubz.append(float(sim.u[:, 2].mean()))
        if step == 1000:
            _, u = sim.fields()
            out["u1000"] = u[:, ::2, ::2, ::2].astype(np.float32)
            out["pos1000"] = sim.x.copy()
        if step % 100 == 0:
            print("step %d  %.0f s" % (step, time.time() - t0), flush=True)
    rho, u = sim.fields()
    out["u3000"] = u[:, ::2, ::2, ::2].astype(np.float32)
    out["drho3000"] = (rho[::2, ::2, ::2] - 1.0).astype(np.float32)
    out["pos3000"] = sim.x.copy()
    out["vel3000"] = sim.u.copy()
    out["active3000"] = sim.active.copy()
    out["ubz_last200"] = np.array(ubz)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
