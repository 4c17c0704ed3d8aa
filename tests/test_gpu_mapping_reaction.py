"""GPU: point-sampled mapping and the -sum F reaction (Sec. 3.2) against the FP64 oracle.

lbm_params.mapping = LBM_MAP_POINT weights the nodes by Z sampled at the node
instead of its cell integral (Eq. 19), renormalised over the in-box nodes;
lbm_params.reaction = LBM_REACTION_ALL spreads psi_b = -(F_D + F_L + F_S +
F_VM) instead of Algorithm 1's -(F_D + F_L).  Bars as for the plain method:
velocity field 1e-5 relative L-inf, bubble positions 1e-6, velocities 1e-5.
"""
import numpy as np
import pytest

from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

SWITCHES = [(lbm.LBM_MAP_POINT, lbm.LBM_REACTION_DRAG_LIFT),
            (lbm.LBM_MAP_CELL, lbm.LBM_REACTION_ALL),
            (lbm.LBM_MAP_POINT, lbm.LBM_REACTION_ALL)]
IDS = ["point", "react_all", "point_react_all"]


def _pair(dims, walls, pos, vel, diam, mapping, reaction, forces=0, g=1e-5, omega=1.6,
          storage=lbm.LBM_STORE_F32):
    p = lbm.lbm_default_params()
    p.g = g
    p.forces = forces
    p.mapping = mapping
    p.reaction = reaction
    col = lbm.Column(dims, omega, walls, params=p, storage=storage)
    sim = OracleSim(dims, omega, walls, params_for_oracle(p, omega))
    rho, u = workloads.random_fields(dims, seed=17, amp=1e-4, rho_amp=1e-4)
    lbm.lbm_set_fields(col.ctx, rho.reshape(-1), u.reshape(-1))
    sim.set_fields(rho, u)
    pos, vel, diam = (np.asarray(v, float) for v in (pos, vel, diam))
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    sim.set_bubbles(pos.reshape(-1, 3), vel.reshape(-1, 3), diam)
    return col, sim


def _compare(col, sim):
    b = lbm.lbm_get_bubbles(col.ctx)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < 1e-5
    assert np.abs(b["pos"] - sim.x).max() < 1e-6 * np.abs(sim.x).max()
    assert rel_linf(b["vel"], sim.u) < 1e-5
    assert rel_linf(b["psi"], sim.psi) < 1e-5
    return b


@pytest.mark.parametrize("mapping,reaction", SWITCHES, ids=IDS)
@pytest.mark.parametrize("walls", [olat.ALL_WALLS, olat.ALL_WALLS | olat.TOP_FREE_SLIP,
                                   olat.WALL_ZM | olat.WALL_ZP])
def test_single_bubble_matches_oracle(mapping, reaction, walls):
    # Near the -x face (x = 1.6) the window is clipped on a wall axis and
    # wraps on a periodic one; the bubble accelerates from rest, so F_VM
    # is large in the -sum F reaction.
    dims = (16, 16, 32)
    col, sim = _pair(dims, walls, [[1.6, 8.3, 9.0]], [[0.0, 0.0, 0.0]], [2.0], mapping, reaction,
                     g=1e-4)
    for _ in range(4):
        lbm.lbm_step(col.ctx, 15)
        sim.run(15)
        _compare(col, sim)


@pytest.mark.parametrize("mapping,reaction", SWITCHES, ids=IDS)
def test_many_bubbles_path_matches_oracle(mapping, reaction):
    dims = (32, 32, 64)
    pos, vel, diam = workloads.swarm(dims, 200, seed=33)
    col, sim = _pair(dims, olat.ALL_WALLS, pos, vel, diam, mapping, reaction, g=1e-4)
    assert lbm.lbm_sweep_kernel(col.ctx).endswith(",1>")
    for _ in range(2):
        lbm.lbm_step(col.ctx, 15)
        sim.run(15)
        _compare(col, sim)


def test_point_mapping_with_lift_matches_oracle():
    # The vorticity's difference weights come from the point samples too.
    dims = (16, 16, 32)
    both = lbm.LBM_FORCE_LIFT | lbm.LBM_FORCE_STRESS
    col, sim = _pair(dims, olat.ALL_WALLS, [[3.0, 8.0, 10.0]], [[0.0, 0.0, 0.0]], [2.0],
                     lbm.LBM_MAP_POINT, lbm.LBM_REACTION_ALL, forces=both, g=1e-4)
    for _ in range(3):
        lbm.lbm_step(col.ctx, 20)
        sim.run(20)
        _compare(col, sim)


def test_point_mapping_fp16_storage_tracks_oracle():
    # The switches sit in the bubble path, not in the population storage.
    dims = (16, 16, 32)
    col, sim = _pair(dims, olat.ALL_WALLS, [[8.0, 8.0, 8.0]], [[0.0, 0.0, 0.0]], [2.0],
                     lbm.LBM_MAP_POINT, lbm.LBM_REACTION_ALL, g=1e-4,
                     storage=lbm.LBM_STORE_F16)
    lbm.lbm_step(col.ctx, 60)
    sim.run(60)
    b = lbm.lbm_get_bubbles(col.ctx)
    assert rel_linf(b["vel"], sim.u) < 1e-3


def test_reaction_all_mixture_momentum_on_gpu():
    # Fully periodic box: the liquid's momentum (FP64 totals of the stored
    # populations) plus sum m_b u_b grows by sum F_B per step.
    dims = (16, 16, 32)
    p = lbm.lbm_default_params()
    p.g = 1e-3
    p.rho_ratio = 0.05
    p.reaction = lbm.LBM_REACTION_ALL
    col = lbm.Column(dims, 1.6, 0, params=p)
    diam = np.array([2.0, 1.5])
    lbm.lbm_set_bubbles(col.ctx, [6.0, 6.2, 5.0, 3.1, 9.0, 20.5], [0, 0, 0, 1e-4, 0, 0], diam)
    vol = np.pi * diam ** 3 / 6.0
    mb = p.rho_ratio * p.rho_l * vol
    fb = ((p.rho_l - p.rho_ratio * p.rho_l) * vol * p.g).sum()

    def total():
        t = lbm.lbm_get_totals(col.ctx)
        v = lbm.lbm_get_bubbles(col.ctx)["vel"]
        return t[1:] + (mb[:, None] * v).sum(axis=0)

    p0 = total()
    for k in range(1, 6):
        lbm.lbm_step(col.ctx, 1)
        gain = total() - p0
        np.testing.assert_allclose(gain, [0.0, 0.0, k * fb], atol=2e-3 * k * fb, rtol=0)


def test_mapping_switch_needs_no_bubbles_and_adjoint_refuses():
    col = lbm.Column((16, 16, 32), 1.6, lbm.LBM_WALL_ALL)
    lbm.lbm_set_bubbles(col.ctx, [8.0, 8.0, 6.0], [0.0, 0.0, 0.0], [2.0])
    p = lbm.lbm_get_params(col.ctx)
    p.mapping = lbm.LBM_MAP_POINT
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_params(col.ctx, p)
    assert e.value.code == lbm.LBM_ERR_STATE
    p.mapping = lbm.LBM_MAP_CELL
    p.reaction = lbm.LBM_REACTION_ALL            # the reaction may change at any time
    lbm.lbm_set_params(col.ctx, p)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adj_forward(col.ctx, 10, 5, 5, 0.0)
    assert e.value.code == lbm.LBM_ERR_STATE
    lbm.lbm_set_bubbles(col.ctx, [], [], [])
    p.reaction = lbm.LBM_REACTION_DRAG_LIFT
    p.mapping = lbm.LBM_MAP_POINT
    lbm.lbm_set_params(col.ctx, p)
    lbm.lbm_set_bubbles(col.ctx, [8.0, 8.0, 6.0], [0.0, 0.0, 0.0], [2.0])
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adj_forward(col.ctx, 10, 5, 5, 0.0)
    assert e.value.code == lbm.LBM_ERR_STATE


def test_switches_batch_column_equals_single_column():
    dims = (32, 16, 32)
    p = lbm.lbm_default_params()
    p.mapping = lbm.LBM_MAP_POINT
    p.reaction = lbm.LBM_REACTION_ALL
    p.g = 1e-4
    b = lbm.Batch([dims, (48, 16, 32)], [1.6, 1.3], params=p)
    lbm.lbm_batch_set_bubbles(b.h, [1, 1], np.array([10.0, 8.0, 12.0, 24.0, 8.0, 10.0]),
                              np.zeros(6), np.array([2.0, 2.5]))
    lbm.lbm_batch_step(b.h, 30)
    _, u_batch = b.fields(0)
    col = lbm.Column(dims, 1.6, lbm.LBM_WALL_ALL, params=p)
    lbm.lbm_set_bubbles(col.ctx, [10.0, 8.0, 12.0], [0.0, 0.0, 0.0], [2.0])
    lbm.lbm_step(col.ctx, 30)
    _, u_single = col.fields()
    assert np.array_equal(u_batch, u_single)
