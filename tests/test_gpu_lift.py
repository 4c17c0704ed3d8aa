"""GPU: lift and stress-gradient forces (Table 1) against the FP64 oracle.

With lbm_params.forces = LBM_FORCE_LIFT | LBM_FORCE_STRESS the bubble update
adds F_L = -C_L rho_l V_b (u_b - u_l) x (curl u_l) and F_S = rho_l V_b D_t u_l.
The oracle forms the vorticity by central differences at the nodes and
interpolates it (Sec. 3.2); the GPU sums the velocities with difference
weights (summation by parts), so the two agree only if both are right.
Bars as for the plain method: velocity field 1e-5 relative L-inf, bubble
positions 1e-6, bubble velocities 1e-5.
"""
import numpy as np
import pytest

from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

BOTH = lbm.LBM_FORCE_LIFT | lbm.LBM_FORCE_STRESS


def _shear_field(dims, gamma=2e-4):
    """u_x = gamma (z - nz/2): uniform vorticity gamma along +y."""
    nx, ny, nz = dims
    z = np.arange(nz) + 0.5
    u = np.zeros((3, nz, ny, nx))
    u[0] = gamma * (z - nz / 2.0)[:, None, None]
    return np.ones((nz, ny, nx)), u


def _pair(dims, walls, pos, vel, diam, forces, g=1e-5, field=True, omega=1.6):
    p = lbm.lbm_default_params()
    p.g = g
    p.forces = forces
    col = lbm.Column(dims, omega, walls, params=p)
    op = params_for_oracle(p, omega)
    op.lift = bool(forces & lbm.LBM_FORCE_LIFT)
    op.stress_gradient = bool(forces & lbm.LBM_FORCE_STRESS)
    sim = OracleSim(dims, omega, walls, op)
    if field:
        rho, u = _shear_field(dims)
        lbm.lbm_set_fields(col.ctx, rho.reshape(-1), u.reshape(-1))
        sim.set_fields(rho, u)
    lbm.lbm_set_bubbles(col.ctx, np.asarray(pos, float).reshape(-1),
                        np.asarray(vel, float).reshape(-1), np.asarray(diam, float))
    sim.set_bubbles(np.asarray(pos, float), np.asarray(vel, float), np.asarray(diam, float))
    return col, sim


def _compare(col, sim):
    b = lbm.lbm_get_bubbles(col.ctx)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < 1e-5
    assert np.abs(b["pos"] - sim.x).max() < 1e-6 * np.abs(sim.x).max()
    assert rel_linf(b["vel"], sim.u) < 1e-5
    return b


@pytest.mark.parametrize("walls", [olat.ALL_WALLS, olat.ALL_WALLS | olat.TOP_FREE_SLIP,
                                   olat.WALL_ZM | olat.WALL_ZP])
def test_lift_and_stress_single_bubble_in_shear(walls):
    # A bubble released in a uniform shear: the slip across the vorticity
    # gives a lift at right angles to both.  Near a wall (x = 3) the window's
    # halo is clipped; on the periodic case it wraps.
    dims = (16, 16, 32)
    col, sim = _pair(dims, walls, [[3.0, 8.0, 12.0]], [[0.0, 0.0, 0.0]], [2.0], BOTH)
    for _ in range(4):
        lbm.lbm_step(col.ctx, 25)
        sim.run(25)
        b = _compare(col, sim)
    # the lift did act: the oracle without it ends elsewhere
    col0, sim0 = _pair(dims, walls, [[3.0, 8.0, 12.0]], [[0.0, 0.0, 0.0]], [2.0], 0)
    sim0.run(100)
    assert np.abs(sim0.x - sim.x).max() > 1e-6


def test_lift_many_bubbles_path():
    # Enough bubbles for the many-bubble path (interpolation summed per tile):
    # the parts of the vorticity sums are added per tile.
    dims = (32, 32, 64)
    pos, vel, diam = workloads.swarm(dims, 200, seed=31)
    col, sim = _pair(dims, olat.ALL_WALLS, pos, vel, diam, BOTH, g=1e-4)
    assert lbm.lbm_sweep_kernel(col.ctx).endswith(",1>")
    for _ in range(2):
        lbm.lbm_step(col.ctx, 20)
        sim.run(20)
        _compare(col, sim)


def test_lift_batch_column_equals_single_column():
    dims = (32, 16, 32)
    rho, u = _shear_field(dims)
    p = lbm.lbm_default_params()
    p.forces = BOTH
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


def test_adjoint_refuses_optional_forces():
    p = lbm.lbm_default_params()
    p.forces = lbm.LBM_FORCE_LIFT
    col = lbm.Column((16, 16, 32), 1.6, lbm.LBM_WALL_ALL, params=p)
    lbm.lbm_set_bubbles(col.ctx, [8.0, 8.0, 6.0], [0.0, 0.0, 0.0], [2.0])
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adj_forward(col.ctx, 10, 5, 5, 0.0)
    assert e.value.code == lbm.LBM_ERR_STATE
