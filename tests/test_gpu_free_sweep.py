"""The sweep of blocks without tile lists (k_collide_stream_free) against the
listed sweep (k_collide_stream_pair): the same Eq. 13-16 arithmetic, so after
one step from the same populations every node the bubble's force cannot reach
has the same bits with and without the bubble; the nodes it reaches differ."""
import numpy as np
import pytest

from oracle import lattice as olat
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import oracle_pops_to_lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,scale", [(lbm.LBM_STORE_F32, 1.0), (lbm.LBM_STORE_F16, 256.0),
                                           (lbm.LBM_STORE_BF16, 1.0)])
@pytest.mark.parametrize("walls", [olat.ALL_WALLS, 0])
def test_force_free_sweep_matches_listed_sweep(storage, scale, walls):
    dims = (64, 16, 40)
    nx, ny, nz = dims
    rho, u = workloads.random_fields(dims, seed=21, amp=1e-3, rho_amp=1e-3)
    f = oracle_pops_to_lib(olat.equilibrium(rho, u))
    zb, d = 20.0, 2.0
    runs = {}
    for with_bubble in (False, True):
        p = lbm.lbm_default_params()
        p.g = 1e-4
        col = lbm.Column(dims, 1.6, walls, storage, scale, params=p)
        lbm.lbm_set_populations(col.ctx, f)
        if with_bubble:
            # Rising at 0.02: a drag, and so a reaction, well above a 16-bit ulp.
            lbm.lbm_set_bubbles(col.ctx, np.array([32.0, 8.0, zb]), np.array([0.0, 0.0, 0.02]),
                                np.array([d]))
        runs[with_bubble] = lbm.lbm_sweep_kernel(col.ctx)
        lbm.lbm_step(col.ctx, 1)
        runs[(with_bubble, "f")] = lbm.lbm_get_populations(col.ctx).reshape(19, nz, ny, nx)
        col.close()
    assert runs[False].startswith("k_collide_stream_free<")
    assert runs[True].startswith("k_collide_stream_pair<")
    a, b = runs[(False, "f")], runs[(True, "f")]
    # The window reaches n = 1.5 d cells around the centre; the step moves the
    # bubble by far less than a cell.
    reach = 1.5 * d + 2
    far = (np.arange(nz) < zb - reach) | (np.arange(nz) > zb + reach)
    assert np.array_equal(a[:, far], b[:, far])
    assert not np.array_equal(a[:, ~far], b[:, ~far])
