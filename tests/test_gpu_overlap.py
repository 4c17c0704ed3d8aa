"""GPU: the bubble update overlapped with the sweep gives the same bits as plain
stream order.

A single column runs each step's bubble update (Algorithm 1 steps 2-6; one
launch for few bubbles, and one persistent launch of covered-tile
velocities, update and binning for many) and the collide-stream sweep
(Eq. 12-16, 21) as overlapping launches: sweep CTAs whose z tile layer the
previous update cleared (no bubble support, widened by 4 cells, reaches it)
do not wait for the update, and run first.
With wall-bounded z (and, for few bubbles, a column of 2^24 sites or more)
the step is split once the z range of the bubbles' reach has been read back
(two steps on): the update and the sweep of the z blocks it can reach run on
one stream, the sweep of the other blocks without force on another.  With kernel timing on, the library keeps plain stream
order instead, so the two runs below differ only in that scheduling; every
population and bubble value must agree bit for bit.  A bubble faster than 4 cells per step is
reported as an instability.
"""
import os

import numpy as np
import pytest

from oracle import binning as obin
from oracle import lattice as olat
from paper_1710_07073_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    assert os.path.exists(lbm.LIB_PATH), "liblbm.so must be built (run __graft_entry__.build())"
    torch.cuda.init()


def _run(dims, walls, pos, vel, diam, steps, plain, storage=lbm.LBM_STORE_F32, scale=1.0,
         g=1e-2, chunks=1):
    p = lbm.lbm_default_params()
    p.g = g
    col = lbm.Column(dims, 1.6, walls, storage, scale, params=p)
    lbm.lbm_set_bubbles(col.ctx, np.asarray(pos, float).reshape(-1),
                        np.asarray(vel, float).reshape(-1), np.asarray(diam, float))
    lbm.lbm_set_kernel_timing(col.ctx, plain)
    for _ in range(chunks):
        lbm.lbm_step(col.ctx, steps // chunks)
    f = lbm.lbm_get_populations(col.ctx)
    b = lbm.lbm_get_bubbles(col.ctx)
    b["bins"] = lbm.lbm_get_bins(col.ctx)
    b["sweep"] = lbm.lbm_sweep_kernel(col.ctx)
    col.close()
    return f, b


def _assert_same(a, b):
    fa, ba = a
    fb, bb = b
    assert np.array_equal(fa, fb)
    for k in ("pos", "vel", "active"):
        assert np.array_equal(ba[k], bb[k]), k


# Bubbles rising at ~0.02-0.05 cells per step cross tile layers (4 cells).
CASES = {
    "walls, one bubble": ((32, 16, 40), olat.ALL_WALLS, [[16.0, 8.0, 7.7]], [[0, 0, 0.05]],
                          [2.0]),
    "periodic z, wraps through the top": (
        (32, 16, 24), olat.WALL_XM | olat.WALL_XP | olat.WALL_YM | olat.WALL_YP,
        [[12.0, 8.0, 21.5]], [[0, 0, 0.05]], [1.5]),
    "three bubbles": ((64, 16, 48), olat.ALL_WALLS,
                      [[10.0, 8.0, 6.0], [40.0, 6.0, 20.2], [52.5, 9.5, 33.9]],
                      [[0, 0, 0.04], [0.01, 0, 0.03], [0, -0.01, 0.05]], [2.0, 1.6, 2.4]),
    "window split over CTAs": ((48, 32, 48), olat.ALL_WALLS, [[24.0, 16.0, 11.9]],
                               [[0, 0, 0.05]], [4.0]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_overlapped_steps_match_plain_order(case):
    dims, walls, pos, vel, diam = CASES[case]
    plain = _run(dims, walls, pos, vel, diam, 240, plain=True)
    over = _run(dims, walls, pos, vel, diam, 240, plain=False, chunks=3)
    _assert_same(plain, over)
    # the bubbles did move across at least one tile layer boundary
    z0 = np.asarray(pos, float)[:, 2]
    z1 = over[1]["pos"][:, 2]
    assert np.any(np.floor(z0 / 4) != np.floor(z1 / 4))


@pytest.mark.parametrize("storage,scale", [(lbm.LBM_STORE_F16, 256.0),
                                           (lbm.LBM_STORE_BF16, 1.0)])
def test_overlapped_steps_match_plain_order_16bit(storage, scale):
    dims, walls, pos, vel, diam = CASES["three bubbles"]
    plain = _run(dims, walls, pos, vel, diam, 120, plain=True, storage=storage, scale=scale)
    over = _run(dims, walls, pos, vel, diam, 120, plain=False, storage=storage, scale=scale)
    _assert_same(plain, over)


def test_bubble_faster_than_guard_is_unstable():
    # u_b = 20 cells per step: the drag slows it to ~9 over the step's
    # sub-steps, so it moves ~14 cells, past the 4-cell bound.
    dims = (32, 32, 64)
    walls = olat.WALL_XM | olat.WALL_XP | olat.WALL_YM | olat.WALL_YP
    col = lbm.Column(dims, 1.6, walls)
    lbm.lbm_set_bubbles(col.ctx, [16.0, 16.0, 20.0], [0.0, 0.0, 20.0], [2.0])
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(col.ctx, 1)
    assert e.value.code == lbm.LBM_ERR_UNSTABLE


def _swarm_case(dims, walls, count, seed, bottom_fraction=0.4):
    pos, _, diam = workloads.swarm(dims, count, seed=seed, bottom_fraction=bottom_fraction)
    rng = np.random.default_rng(seed)
    vel = np.zeros((count, 3))
    vel[:, 2] = rng.uniform(0.02, 0.06, count)
    return dims, walls, pos, vel, diam


# Enough bubbles that their (tile, bubble) pairs may exceed 4096: the
# many-bubble path.
MANY = {
    "swarm, walls": _swarm_case((64, 32, 96), olat.ALL_WALLS, 320, 9),
    "swarm, periodic z": _swarm_case((64, 32, 64), olat.WALL_XM | olat.WALL_XP | olat.WALL_YM
                                     | olat.WALL_YP, 300, 10),
    # bubbles over the whole height: every z block is guarded
    "swarm, walls, full height": _swarm_case((64, 32, 64), olat.ALL_WALLS, 400, 11, 1.0),
}


@pytest.mark.parametrize("case", sorted(MANY))
@pytest.mark.parametrize("storage,scale", [(lbm.LBM_STORE_F32, 1.0), (lbm.LBM_STORE_F16, 256.0)])
def test_many_bubbles_overlapped_match_plain_order(case, storage, scale):
    dims, walls, pos, vel, diam = MANY[case]
    plain = _run(dims, walls, pos, vel, diam, 120, plain=True, storage=storage, scale=scale)
    over = _run(dims, walls, pos, vel, diam, 120, plain=False, storage=storage, scale=scale,
                chunks=3)
    _assert_same(plain, over)
    z0 = np.asarray(pos, float)[:, 2]
    z1 = over[1]["pos"][:, 2]
    assert np.count_nonzero(np.floor(z0 / 4) != np.floor(z1 / 4)) > 10
    assert over[1]["sweep"].endswith(",1>")   # the many-bubble path ran
    if not over[1]["active"].all():
        # Bubbles stopped at the top (the full-height case): which of them
        # the last binning still held is not visible from outside.
        assert case.endswith("full height")
        return
    # The binning left by the last update is the oracle's brute-force binning
    # of the same centres (Algorithm 1 step 2).
    bins = over[1]["bins"]
    hw = lbm.lbm_default_params().width_factor * np.asarray(diam)
    off, items = obin.tile_lists(list(over[1]["pos"]), list(hw), np.ones(len(hw), bool), dims,
                                 walls, bins["tile"])
    assert np.array_equal(bins["offsets"], np.array(off))
    assert np.array_equal(bins["items"], np.array(items))


def test_many_bubbles_split_sweep_runs():
    # Wall-bounded z, default order: after the first steps (whose z ranges
    # are not yet read back) a step is five launches -- interpolation, update,
    # binning, the sweep of the z blocks bubbles can reach, and that of the
    # others on a second stream.
    dims, walls, pos, vel, diam = MANY["swarm, walls"]
    p = lbm.lbm_default_params()
    col = lbm.Column(dims, 1.6, walls, params=p)
    lbm.lbm_set_bubbles(col.ctx, np.asarray(pos, float).reshape(-1),
                        np.asarray(vel, float).reshape(-1), np.asarray(diam, float))
    lbm.lbm_step(col.ctx, 4)
    n0 = lbm.lbm_launch_count(col.ctx)
    lbm.lbm_step(col.ctx, 10)
    assert lbm.lbm_launch_count(col.ctx) - n0 == 50
    lbm.lbm_set_kernel_timing(col.ctx, True)      # plain order: one sweep per step
    n0 = lbm.lbm_launch_count(col.ctx)
    lbm.lbm_step(col.ctx, 10)
    assert lbm.lbm_launch_count(col.ctx) - n0 == 40
    col.close()


def test_few_bubbles_split_sweep_matches_plain_order():
    # A column of 2^24 sites or more with wall-bounded z: after the first
    # steps a step is three launches -- the update, the sweep of the z blocks
    # its bubble can reach, and that of the others (without force) on a second
    # stream -- and gives the bits of plain stream order.  Smaller columns
    # and periodic z keep the overlapped update and sweep: two launches.
    dims = (256, 256, 256)
    pos, vel, diam = [[128.0, 128.0, 60.3]], [[0.0, 0.0, 0.05]], [2.0]
    runs = []
    for plain in (True, False):
        col = lbm.Column(dims, 1.6, olat.ALL_WALLS, params=lbm.lbm_default_params())
        lbm.lbm_set_bubbles(col.ctx, np.asarray(pos, float).reshape(-1),
                            np.asarray(vel, float).reshape(-1), np.asarray(diam, float))
        lbm.lbm_set_kernel_timing(col.ctx, plain)
        lbm.lbm_step(col.ctx, 4)
        n0 = lbm.lbm_launch_count(col.ctx)
        lbm.lbm_step(col.ctx, 10)
        assert lbm.lbm_launch_count(col.ctx) - n0 == (20 if plain else 30)
        rho, u = lbm.lbm_get_fields(col.ctx)
        b = lbm.lbm_get_bubbles(col.ctx)
        runs.append((rho, u, b))
        col.close()
    (r0, u0, b0), (r1, u1, b1) = runs
    assert np.array_equal(r0, r1) and np.array_equal(u0, u1)
    for k in ("pos", "vel", "active"):
        assert np.array_equal(b0[k], b1[k]), k
    for case in ("walls, one bubble", "periodic z, wraps through the top"):
        dims, walls, pos, vel, diam = CASES[case]
        col = lbm.Column(dims, 1.6, walls, params=lbm.lbm_default_params())
        lbm.lbm_set_bubbles(col.ctx, np.asarray(pos, float).reshape(-1),
                            np.asarray(vel, float).reshape(-1), np.asarray(diam, float))
        lbm.lbm_step(col.ctx, 4)
        n0 = lbm.lbm_launch_count(col.ctx)
        lbm.lbm_step(col.ctx, 10)
        assert lbm.lbm_launch_count(col.ctx) - n0 == 20, case
        col.close()
