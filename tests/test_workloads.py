"""The seeded input generators follow their stated recipe (CPU only).

The generators draw the inputs that both the oracle and the CUDA path see; they
hold none of the method's arithmetic.  These checks fix the shapes, placements
and distributions the workloads state (lattice units).
"""
import numpy as np
import pytest

from paper_1710_07073_gb300 import workloads as wl


def test_single_bubble_placement():
    for dims in (wl.SINGLE_SMALL, wl.SINGLE_LARGE):
        pos, vel, d = wl.single_bubble(dims)
        nx, ny, nz = dims
        assert pos.shape == (1, 3) and vel.shape == (1, 3) and d.shape == (1,)
        assert np.array_equal(pos[0], [nx / 2, ny / 2, nz / 8])
        assert not vel.any() and d[0] == 2.0


def test_lognormal_diameters_have_the_stated_moments():
    d = wl.lognormal_diameters(np.random.default_rng(0), 400_000)
    assert abs(d.mean() - 1.5) < 0.005 and abs(d.std() - 0.3) < 0.005
    assert d.min() > 0.0


@pytest.mark.parametrize("dims,count", [(wl.SWARM_CROP, 463), ((32, 32, 64), 58),
                                        ((96, 80, 200), 1000)])
def test_swarm_inside_walls_and_bottom_fraction(dims, count):
    pos, vel, d = wl.swarm(dims, count, seed=1234)
    nx, ny, nz = dims
    r = 0.5 * d
    assert pos.shape == (count, 3) and not vel.any()
    assert d.max() <= 4.0
    for a, L in enumerate((nx, ny)):
        assert np.all(pos[:, a] >= r) and np.all(pos[:, a] <= L - r)
    assert np.all(pos[:, 2] >= r) and np.all(pos[:, 2] <= 0.2 * nz - r)
    # seeded: the same draw again, another seed differs
    pos2, _, d2 = wl.swarm(dims, count, seed=1234)
    assert np.array_equal(pos, pos2) and np.array_equal(d, d2)
    pos3, _, _ = wl.swarm(dims, count, seed=1235)
    assert not np.array_equal(pos, pos3)


def test_swarm_crop_counts_scale_with_volume():
    full = 100_000
    assert wl.swarm_count_for_crop(wl.SWARM_FULL, full, (32, 32, 64)) == 58
    assert wl.swarm_count_for_crop(wl.SWARM_FULL, full, wl.SWARM_CROP) == 463
    assert wl.swarm_count_for_crop(wl.SWARM_FULL, full, wl.SWARM_FULL) == full
    assert wl.swarm_count_for_crop(wl.SWARM_FULL, full, (1, 1, 1)) == 1


def test_batch_columns_recipe():
    cols = wl.batch_columns(64, seed=1234)
    assert len(cols) == 64
    sites = 0
    for dims, omega, pos, vel, d in cols:
        assert dims in wl.COLUMN_SIZES
        assert 1.0 <= omega <= 1.9 and 1.5 <= d[0] <= 3.0
        assert np.array_equal(pos[0], [dims[0] / 2, dims[1] / 2, dims[2] / 8])
        assert not vel.any()
        sites += dims[0] * dims[1] * dims[2]
    assert abs(sites / 1e6 - 106.8) < 0.05
    again = wl.batch_columns(64, seed=1234)
    assert [c[0] for c in cols] == [c[0] for c in again]
    assert [c[1] for c in cols] == [c[1] for c in again]


def test_field_generators_shapes_and_seeds():
    dims = (6, 5, 4)
    rho, u = wl.random_fields(dims, seed=3, amp=1e-2, rho_amp=2e-2)
    assert rho.shape == (4, 5, 6) and u.shape == (3, 4, 5, 6)
    assert abs(rho.mean() - 1.0) < 0.02 and np.abs(u).max() < 0.1
    rho2, u2 = wl.random_fields(dims, seed=3, amp=1e-2, rho_amp=2e-2)
    assert np.array_equal(rho, rho2) and np.array_equal(u, u2)
    p = wl.gaussian_velocity_perturbation(dims, seed=4, amp=1e-4)
    assert p.shape == (3, 4, 5, 6) and np.array_equal(p, wl.gaussian_velocity_perturbation(dims))
