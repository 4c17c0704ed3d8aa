"""GPU: the free-slip top (Sec. 3.3) against the FP64 oracle, through the C ABI.

With LBM_TOP_FREE_SLIP the +z face reflects populations specularly (c_z
reversed, tangential components kept).  One-step parity from random
populations is in test_gpu_parity (its wall cases include the free-slip top);
here: 16-bit storage, a coupled run in which the bubble rises to the free-slip
top and stops there (Algorithm 1), a batch column with a free-slip top, and
the adjoint's refusal of it.
"""
import numpy as np
import pytest

from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import lib_pops_to_oracle, oracle_pops_to_lib, params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

FREE_TOP = olat.ALL_WALLS | olat.TOP_FREE_SLIP


@pytest.mark.parametrize("storage,scale,tol", [(lbm.LBM_STORE_F16, 256.0, 2.0 ** -11),
                                               (lbm.LBM_STORE_BF16, 1.0, 2.0 ** -8)])
@pytest.mark.parametrize("dims", [(37, 9, 11), (40, 9, 11)])
def test_one_step_16bit_free_slip(storage, scale, tol, dims):
    rho, u = workloads.random_fields(dims, seed=8, amp=1e-3, rho_amp=1e-3)
    f = olat.equilibrium(rho, u)
    col = lbm.Column(dims, 1.7, FREE_TOP, storage, scale)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    f_exact = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    lbm.lbm_step(col.ctx, 1)
    got = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    want = olat.lb_step(f_exact, 1.7, FREE_TOP)
    dev = np.abs(want - olat.W[:, None, None, None])
    assert (np.abs(got - want) <= tol * dev + 1e-10).all()


@pytest.mark.parametrize("walls", [FREE_TOP, olat.WALL_ZM | olat.WALL_ZP | olat.TOP_FREE_SLIP])
def test_bubble_rises_to_free_slip_top_and_stops(walls):
    dims = (16, 16, 24)
    p = lbm.lbm_default_params()
    p.g = 1e-2
    pos = np.array([[8.0, 8.0, 17.5]])
    vel = np.array([[0.0, 0.0, 0.04]])
    diam = np.array([2.0])
    col = lbm.Column(dims, 1.6, walls, params=p)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    sim = OracleSim(dims, 1.6, walls, params_for_oracle(p, 1.6))
    sim.set_bubbles(pos, vel, diam)
    stopped = None
    for step in range(300):
        lbm.lbm_step(col.ctx, 1)
        sim.step()
        b = lbm.lbm_get_bubbles(col.ctx)
        assert bool(b["active"][0]) == bool(sim.active[0]), step
        assert np.abs(b["pos"] - sim.x).max() < 1e-6 * np.abs(sim.x).max()
        if not sim.active[0]:
            stopped = step
            break
    assert stopped is not None
    lbm.lbm_step(col.ctx, 20)
    sim.run(20)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < 1e-5


def test_batch_column_with_free_slip_top_equals_single_column():
    cols = [((32, 16, 24), 1.6), ((48, 16, 32), 1.3)]
    walls = [FREE_TOP, olat.ALL_WALLS]
    pos = np.array([[16.0, 8.0, 6.0], [24.0, 8.0, 8.0]])
    diam = np.array([2.0, 2.5])
    p = lbm.lbm_default_params()
    p.g = 1e-3
    b = lbm.Batch([c[0] for c in cols], [c[1] for c in cols], walls, params=p)
    lbm.lbm_batch_set_bubbles(b.h, [1, 1], pos.reshape(-1), np.zeros(6), diam)
    lbm.lbm_batch_step(b.h, 40)
    _, u_batch = b.fields(0)
    col = lbm.Column(cols[0][0], cols[0][1], FREE_TOP, params=p)
    lbm.lbm_set_bubbles(col.ctx, pos[0], np.zeros(3), diam[:1])
    lbm.lbm_step(col.ctx, 40)
    _, u_single = col.fields()
    assert np.array_equal(u_batch, u_single)


def test_adjoint_refuses_free_slip_top():
    col = lbm.Column((16, 16, 32), 1.6, FREE_TOP)
    lbm.lbm_set_bubbles(col.ctx, [8.0, 8.0, 6.0], [0.0, 0.0, 0.0], [2.0])
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adj_forward(col.ctx, 10, 5, 5, 0.0)
    assert e.value.code == lbm.LBM_ERR_STATE
