"""Batched columns (one persistent launch per step under a CUDA graph, autotuned
launch shape) against the single-column path and the FP64 oracle."""
import numpy as np
import pytest

from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

COLS = [((32, 32, 64), 1.3, olat.ALL_WALLS), ((48, 48, 96), 1.8, olat.ALL_WALLS),
        ((16, 24, 40), 1.0, olat.WALL_ZM | olat.WALL_ZP), ((64, 12, 24), 1.6, 0),
        ((2, 4, 6), 1.9, olat.ALL_WALLS)]


def _bubbles():
    counts, pos, diam = [], [], []
    rng = np.random.default_rng(3)
    for dims, _, _ in COLS:
        if min(dims) < 8:
            counts.append(0)
            continue
        k = 2 if dims[2] >= 40 else 1
        counts.append(k)
        for _ in range(k):
            d = rng.uniform(1.5, 2.2)
            pos.append([dims[0] / 2 + rng.uniform(-2, 2), dims[1] / 2 + rng.uniform(-1, 1),
                        rng.uniform(d, dims[2] / 3)])
            diam.append(d)
    return counts, np.array(pos), np.array(diam)


def _params():
    p = lbm.lbm_default_params()
    p.g = 2e-4
    return p


def _single_runs(steps, storage=lbm.LBM_STORE_F32, scale=1.0):
    counts, pos, diam = _bubbles()
    out, k = [], 0
    for (dims, om, walls), n in zip(COLS, counts):
        col = lbm.Column(dims, om, walls, storage, scale, params=_params())
        if n:
            lbm.lbm_set_bubbles(col.ctx, pos[k:k + n].reshape(-1), np.zeros(3 * n), diam[k:k + n])
        k += n
        lbm.lbm_step(col.ctx, steps)
        out.append((col.fields(), lbm.lbm_get_bubbles(col.ctx)))
        col.close()
    return out


def _batch(storage=lbm.LBM_STORE_F32, scale=1.0):
    counts, pos, diam = _bubbles()
    b = lbm.Batch([c[0] for c in COLS], [c[1] for c in COLS], [c[2] for c in COLS], storage,
                  scale, params=_params())
    lbm.lbm_batch_set_bubbles(b.h, counts, pos.reshape(-1), np.zeros(pos.size), diam)
    return b, counts


def _compare_exact(b, counts, singles):
    allb = lbm.lbm_batch_get_bubbles(b.h)
    k = 0
    for c, ((rho_s, u_s), bub_s) in enumerate(singles):
        rho_b, u_b = b.fields(c)
        assert np.array_equal(rho_b, rho_s), c
        assert np.array_equal(u_b, u_s), c
        n = counts[c]
        for key in ("pos", "vel", "ul", "psi"):
            assert np.array_equal(allb[key][k:k + n], bub_s[key]), (c, key)
        k += n


@pytest.mark.parametrize("steps", [1, 2, 37])
def test_batch_equals_single_columns(steps):
    # Uneven sizes, omegas and walls; odd step counts end on a single step
    # after the two-step graph replays.
    b, counts = _batch()
    lbm.lbm_batch_step(b.h, steps)
    _compare_exact(b, counts, _single_runs(steps))


def test_batch_fp16_equals_single_columns():
    b, counts = _batch(lbm.LBM_STORE_F16, 256.0)
    lbm.lbm_batch_step(b.h, 20)
    _compare_exact(b, counts, _single_runs(20, lbm.LBM_STORE_F16, 256.0))


def test_tuning_restores_state_and_keeps_results():
    b, counts = _batch()
    lbm.lbm_batch_step(b.h, 6)
    depth, grid = lbm.lbm_batch_tune(b.h, 4)
    assert depth in (1, 2, 4, 8) and grid > 0
    planes, depth2, grid2 = lbm.lbm_batch_launch_shape(b.h)
    assert planes in (1, 2, 4) and (depth2, grid2) == (depth, grid)
    lbm.lbm_batch_step(b.h, 14)
    _compare_exact(b, counts, _single_runs(20))


@pytest.mark.parametrize("storage,scale", [(lbm.LBM_STORE_F32, 1.0), (lbm.LBM_STORE_F16, 256.0)])
def test_every_tile_shape_equals_single_columns(storage, scale):
    # The tuner's candidates -- 32 x 4 x {1, 2, 4} node tiles, any depth and
    # grid -- give the same bits: the shape changes only who computes a node.
    ref = _single_runs(12, storage, scale)
    for planes in (1, 2, 4):
        b, counts = _batch(storage, scale)
        lbm.lbm_batch_set_launch_shape(b.h, planes, 3, 152 * planes)
        assert lbm.lbm_batch_launch_shape(b.h) == (planes, 3, 152 * planes)
        lbm.lbm_batch_step(b.h, 12)
        _compare_exact(b, counts, ref)


def test_batch_column_against_oracle():
    b, counts = _batch()
    lbm.lbm_batch_step(b.h, 60)
    dims, om, walls = COLS[0]
    _, pos, diam = _bubbles()
    sim = OracleSim(dims, om, walls, params_for_oracle(_params(), om))
    sim.set_bubbles(pos[:counts[0]], np.zeros((counts[0], 3)), diam[:counts[0]])
    sim.run(60)
    _, u_b = b.fields(0)
    assert rel_linf(u_b, sim.fields()[1]) < 1e-5
    allb = lbm.lbm_batch_get_bubbles(b.h)
    assert np.abs(allb["pos"][:counts[0]] - sim.x).max() < 1e-6 * 64


def test_batch_rejects_odd_nx_and_too_many_pairs():
    with pytest.raises(lbm.LbmError):
        lbm.Batch([(31, 8, 8)], [1.6])
    b = lbm.Batch([(64, 64, 64)], [1.6])
    n = 200
    pos = np.tile([32.0, 32.0, 32.0], (n, 1))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_set_bubbles(b.h, [n], pos.reshape(-1), None, np.full(n, 3.0))
