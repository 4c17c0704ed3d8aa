"""GPU: the dispersed swarm at its full size (384x384x768, 100,000 bubbles), in
the launch configuration bench.py times, against the FP64 oracle on what the
oracle can compute at that size.

* Binning: after two steps the tile lists (221,184 tiles, the count-scan-fill-
  sort path) equal the oracle's lists of the GPU's own centres, bit for bit.
* Light cone: in one step a node's value depends on its neighbours and on the
  bubbles whose windows cover it, whose reaction depends on the field over
  their own windows: everything within 2 (n_max + 1) = 14 cells (n_max = 6,
  d <= 4).  So an oracle run on an 80^3 periodic crop inside the swarm
  reproduces, after 2 steps, the velocity field of the crop's inner 24^3
  (28 cells from every face) and the bubbles whose windows lie 14 cells
  inside: velocity 1e-5 relative L-inf, positions 1e-6, velocities 1e-5.
* Mass: the FP64 total over the box is conserved to 1e-12 relative.
"""
import numpy as np
import pytest

from oracle import binning as obin
from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

STEPS = 2
CROP = 80
CONE = 14 * STEPS
LO = np.array([152, 152, 40])          # crop origin (x, y, z), inside the swarm


@pytest.fixture(scope="module")
def swarm_run():
    dims = workloads.SWARM_FULL
    pos, vel, diam = workloads.swarm(dims, 100_000, seed=1234)
    p = lbm.lbm_default_params()
    col = lbm.Column(dims, 1.7, lbm.LBM_WALL_ALL, params=p)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    mass0 = lbm.lbm_get_totals(col.ctx)[0]
    lbm.lbm_step(col.ctx, STEPS)
    out = {"dims": dims, "pos0": pos, "vel0": vel, "diam": diam, "params": p,
           "mass0": mass0, "mass1": lbm.lbm_get_totals(col.ctx)[0],
           "bins": lbm.lbm_get_bins(col.ctx), "bub": lbm.lbm_get_bubbles(col.ctx),
           "sweep": lbm.lbm_sweep_kernel(col.ctx)}
    _, u = lbm.lbm_get_fields(col.ctx, rho=False)
    nx, ny, nz = dims
    u = u.reshape(3, nz, ny, nx)
    out["u_crop"] = u[:, LO[2]:LO[2] + CROP, LO[1]:LO[1] + CROP, LO[0]:LO[0] + CROP].copy()
    del u
    col.close()
    return out


def test_full_swarm_takes_the_bench_path(swarm_run):
    assert swarm_run["sweep"] == "k_collide_stream_pair<0,1>"


def test_full_swarm_binning_bit_exact(swarm_run):
    r = swarm_run
    b = r["bub"]
    bins = r["bins"]
    off, items = obin.tile_lists(b["pos"], 1.5 * r["diam"], b["active"], r["dims"],
                                 olat.ALL_WALLS, bins["tile"])
    assert np.array_equal(bins["offsets"], np.array(off, dtype=np.int32))
    assert np.array_equal(bins["items"], np.array(items, dtype=np.int32))


def test_full_swarm_mass_conserved(swarm_run):
    assert abs(swarm_run["mass1"] / swarm_run["mass0"] - 1.0) < 1e-12


def test_full_swarm_inner_crop_against_oracle(swarm_run):
    r = swarm_run
    pos0, vel0, diam = r["pos0"], r["vel0"], r["diam"]
    inside = np.all((pos0 >= LO) & (pos0 < LO + CROP), axis=1)
    idx = np.flatnonzero(inside)
    sim = OracleSim((CROP, CROP, CROP), 1.7, 0, params_for_oracle(r["params"], 1.7))
    sim.set_bubbles(pos0[idx] - LO, vel0[idx], diam[idx])
    sim.run(STEPS)
    _, u_or = sim.fields()
    a, e = CONE, CROP - CONE
    sub_gpu = r["u_crop"][:, a:e, a:e, a:e]
    sub_or = u_or[:, a:e, a:e, a:e]
    assert np.abs(sub_or).max() > 0.0
    assert rel_linf(sub_gpu, sub_or) < 1e-5
    # Bubbles whose windows lie 14 cells inside the crop at the start.
    n = 1.5 * diam[idx]
    rel = pos0[idx] - LO
    deep = np.all((rel - n[:, None] >= CONE // 2) & (rel + n[:, None] <= CROP - CONE // 2), axis=1)
    assert deep.sum() > 50
    b = r["bub"]
    gpos = b["pos"][idx][deep] - LO
    gvel = b["vel"][idx][deep]
    assert np.abs(gpos - sim.x[deep]).max() < 1e-6 * 768
    assert rel_linf(gvel, sim.u[deep]) < 1e-5
