"""GPU (sm_103a) parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances:
* populations after one step: 2e-8 absolute (f ~ 0.05; FP32 arithmetic on
  populations shifted by w_j rho0 keeps ~1e-9);
* velocity field: 1e-5 relative L-inf (max |u_gpu - u_oracle| / max |u_oracle|)
  after up to 1000 steps; bubble positions 1e-6 relative;
* binning (cell ids, per-tile lists): bit-exact.
"""
import os

import numpy as np
import pytest

from oracle import binning as obin
from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import (lib_pops_to_oracle, oracle_pops_to_lib, params_for_oracle,
                            rel_linf)

pytestmark = pytest.mark.gpu

POP_ATOL = 2e-8
U_RTOL = 1e-5
X_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    assert os.path.exists(lbm.LIB_PATH), "liblbm.so must be built (run __graft_entry__.build())"
    torch.cuda.init()


def _random_pops(dims, seed, amp=1e-2):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    rho, u = workloads.random_fields(dims, seed=seed, amp=amp, rho_amp=amp)
    f = olat.equilibrium(rho, u)
    return f * (1.0 + 0.1 * amp * rng.standard_normal(f.shape))


WALL_CASES = [olat.ALL_WALLS, 0, olat.WALL_ZM | olat.WALL_ZP, olat.WALL_XM | olat.WALL_XP,
              olat.ALL_WALLS | olat.TOP_FREE_SLIP,
              olat.WALL_ZM | olat.WALL_ZP | olat.TOP_FREE_SLIP]


@pytest.mark.parametrize("dims", [(37, 9, 11), (1, 1, 12), (64, 4, 4)])
@pytest.mark.parametrize("walls", WALL_CASES)
def test_population_roundtrip(dims, walls):
    f = _random_pops(dims, 11)
    col = lbm.Column(dims, 1.6, walls)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    back = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    # Stored as FP32 deviations from w_j rho0: exact up to FP32 rounding of ~1e-3.
    assert np.abs(back - f).max() < 1e-9


@pytest.mark.parametrize("dims", [(37, 9, 11), (38, 9, 11), (2, 3, 5), (96, 6, 7)])
@pytest.mark.parametrize("omega", [1.0, 1.6, 1.9])
@pytest.mark.parametrize("walls", WALL_CASES)
def test_one_step_random_populations(omega, walls, dims):
    # Odd nx runs the one-node-per-thread sweep, even nx the two-node one.
    # Ragged tails in every axis: x tiles of 32, y tiles of 4, z pairs.
    f = _random_pops(dims, 5)
    col = lbm.Column(dims, omega, walls)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    lbm.lbm_step(col.ctx, 1)
    got = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    want = olat.lb_step(f, omega, walls)
    assert np.abs(got - want).max() < POP_ATOL


@pytest.mark.parametrize("storage,scale,tol", [(lbm.LBM_STORE_F16, 256.0, 2.0 ** -11),
                                               (lbm.LBM_STORE_BF16, 1.0, 2.0 ** -8)])
@pytest.mark.parametrize("dims", [(37, 9, 11), (38, 9, 11), (40, 9, 11), (32, 8, 8), (64, 12, 9)])
def test_one_step_16bit_from_representable_input(storage, scale, tol, dims):
    # nx odd: one node per thread; nx even: two nodes per thread (ragged tiles
    # in x, y and z included).
    # Both sweeps in 16-bit storage: from populations the format holds exactly,
    # one step differs from the FP64 step by FP32 arithmetic plus one rounding
    # of each stored value (half an ulp, relative to f - w rho0).
    rho, u = workloads.random_fields(dims, seed=8, amp=1e-3, rho_amp=1e-3)
    f = olat.equilibrium(rho, u)
    col = lbm.Column(dims, 1.7, olat.ALL_WALLS, storage, scale)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    f_exact = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    lbm.lbm_step(col.ctx, 1)
    got = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    want = olat.lb_step(f_exact, 1.7, olat.ALL_WALLS)
    dev = np.abs(want - olat.W[:, None, None, None])
    assert (np.abs(got - want) <= tol * dev + 1e-10).all()


def test_fifty_steps_fields():
    dims = (37, 9, 11)
    rho, u = workloads.random_fields(dims, seed=3, amp=1e-3, rho_amp=1e-3)
    col = lbm.Column(dims, 1.7, olat.ALL_WALLS)
    lbm.lbm_set_fields(col.ctx, rho.reshape(-1), u.reshape(-1))
    sim = OracleSim(dims, 1.7, olat.ALL_WALLS)
    sim.set_fields(rho, u)
    lbm.lbm_step(col.ctx, 50)
    sim.run(50)
    r_gpu, u_gpu = col.fields()
    r_or, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < U_RTOL
    assert np.abs(r_gpu - r_or).max() < 1e-9


def _coupled_pair(dims, omega, walls, pos, vel, diam, params=None):
    col = lbm.Column(dims, omega, walls)
    p = params if params is not None else lbm.lbm_default_params()
    lbm.lbm_set_params(col.ctx, p)
    lbm.lbm_set_bubbles(col.ctx, np.asarray(pos).reshape(-1), np.asarray(vel).reshape(-1), diam)
    sim = OracleSim(dims, omega, walls, params_for_oracle(p, omega))
    sim.set_bubbles(pos, vel, diam)
    return col, sim


@pytest.mark.parametrize("walls", [olat.ALL_WALLS, 0])
def test_one_coupled_step_populations(walls):
    # Eq. 19-21 interpolation and spreading, Table 1 update, Guo forcing: one
    # step compared population by population.  One bubble sits by the -x face
    # (clipped window, or wrapping on the periodic box), one inside.
    dims = (40, 12, 20)
    pos = [[1.2, 6.3, 9.7], [21.6, 5.0, 12.2]]
    vel = [[0.0, 1e-3, 2e-3], [-1e-3, 0.0, 5e-3]]
    diam = [2.0, 1.6]
    p = lbm.lbm_default_params()
    p.g = 1e-3                      # a strong force so the coupling terms matter
    col, sim = _coupled_pair(dims, 1.6, walls, pos, vel, diam, p)
    f0 = _random_pops(dims, 9, amp=1e-3)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f0))
    sim.f = f0.copy()
    lbm.lbm_step(col.ctx, 1)
    sim.step()
    got = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    assert np.abs(got - sim.f).max() < POP_ATOL
    b = lbm.lbm_get_bubbles(col.ctx)
    assert rel_linf(b["ul"], sim.ul) < 1e-6
    assert rel_linf(b["psi"], sim.psi) < 1e-6
    assert np.abs(b["pos"] - sim.x).max() < X_RTOL * np.abs(sim.x).max()


def test_single_bubble_1000_steps():
    # Single bubble rising in stagnant liquid, 32x32x64, omega 1.6, bounce-back
    # on all six walls, d = 2 released at rest at (16, 16, 8).
    dims = workloads.SINGLE_SMALL
    pos, vel, diam = workloads.single_bubble(dims)
    col, sim = _coupled_pair(dims, 1.6, olat.ALL_WALLS, pos, vel, diam)
    lbm.lbm_step(col.ctx, 1000)
    sim.run(1000)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < U_RTOL
    b = lbm.lbm_get_bubbles(col.ctx)
    assert np.abs(b["pos"] - sim.x).max() < X_RTOL * np.abs(sim.x).max()
    assert rel_linf(b["vel"], sim.u) < U_RTOL


@pytest.mark.parametrize("count", [None, 200])
def test_swarm_crop_100_steps(count):
    # Dispersed swarm: lognormal diameters (mean 1.5, sd 0.3), uniform in the
    # bottom 20 %, count scaled by volume from 100 000 bubbles in 384x384x768
    # (58 bubbles: single-launch binning), or 200 bubbles (count-scan-fill-sort
    # binning).
    dims = (32, 32, 64)
    if count is None:
        count = workloads.swarm_count_for_crop(workloads.SWARM_FULL, 100_000, dims)
    pos, vel, diam = workloads.swarm(dims, count, seed=1234)
    p = lbm.lbm_default_params()
    p.g = 1e-4
    col, sim = _coupled_pair(dims, 1.7, olat.ALL_WALLS, pos, vel, diam, p)
    lbm.lbm_step(col.ctx, 100)
    sim.run(100)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < U_RTOL
    b = lbm.lbm_get_bubbles(col.ctx)
    assert np.abs(b["pos"] - sim.x).max() < X_RTOL * np.abs(sim.x).max()
    assert (b["active"] == sim.active).all()


@pytest.mark.parametrize("storage,scale,u_tol", [(lbm.LBM_STORE_F16, 256.0, 3e-3),
                                                 (lbm.LBM_STORE_BF16, 1.0, 3e-2)])
def test_swarm_crop_16bit_storage(storage, scale, u_tol):
    # 200 bubbles in 32x32x64 take the many-bubble kernels and the sweep's
    # tabulated force gather; with 16-bit storage the bars are those of the
    # storage rounding (about 6e-4 and 8e-3 on a single bubble after 1000
    # steps, here with a margin), positions to 1e-5.
    dims = (32, 32, 64)
    pos, vel, diam = workloads.swarm(dims, 200, seed=1234)
    p = lbm.lbm_default_params()
    p.g = 1e-4
    col = lbm.Column(dims, 1.7, olat.ALL_WALLS, storage, scale)
    lbm.lbm_set_params(col.ctx, p)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    sim = OracleSim(dims, 1.7, olat.ALL_WALLS, params_for_oracle(p, 1.7))
    sim.set_bubbles(pos, vel, diam)
    lbm.lbm_step(col.ctx, 100)
    sim.run(100)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < u_tol
    b = lbm.lbm_get_bubbles(col.ctx)
    assert np.abs(b["pos"] - sim.x).max() < 1e-5 * np.abs(sim.x).max()
    assert (b["active"] == sim.active).all()


@pytest.mark.parametrize("count", [None, 40])
@pytest.mark.parametrize("walls", [olat.ALL_WALLS, olat.WALL_ZM | olat.WALL_ZP])
def test_binning_bit_exact(walls, count):
    # 463 bubbles (volume-scaled swarm) use the count-scan-fill-sort binning,
    # 40 bubbles the single-launch path; both must give the same lists.
    dims = workloads.SWARM_CROP
    if count is None:
        count = workloads.swarm_count_for_crop(workloads.SWARM_FULL, 100_000, dims)
    pos, vel, diam = workloads.swarm(dims, count, seed=99)
    col = lbm.Column(dims, 1.7, walls)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    lbm.lbm_step(col.ctx, 3)
    bins = lbm.lbm_get_bins(col.ctx)
    b = lbm.lbm_get_bubbles(col.ctx)
    n = 1.5 * diam
    # Same input positions on both sides: the GPU's updated centres.
    off, items = obin.tile_lists(b["pos"], n, np.ones(count, bool), dims, walls, bins["tile"])
    assert np.array_equal(bins["offsets"], np.array(off, dtype=np.int32))
    assert np.array_equal(bins["items"], np.array(items, dtype=np.int32))
    cells = [obin.containing_cell(x, dims) for x in b["pos"]]
    assert np.array_equal(bins["cell"], np.array(cells, dtype=np.int32))


def test_bubble_reaches_top_and_stops():
    dims = (8, 8, 12)
    p = lbm.lbm_default_params()
    p.g = 1e-2
    col, sim = _coupled_pair(dims, 1.6, olat.ALL_WALLS, [[4.0, 4.0, 10.5]], [[0, 0, 0.05]],
                             [1.0], p)
    for step in range(400):
        lbm.lbm_step(col.ctx, 1)
        sim.step()
        b = lbm.lbm_get_bubbles(col.ctx)
        assert bool(b["active"][0]) == bool(sim.active[0]), step
        if not sim.active[0]:
            break
    assert not sim.active[0]
    lbm.lbm_step(col.ctx, 5)
    sim.run(5)
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < U_RTOL


def test_periodic_bubble_crosses_face():
    dims = (16, 16, 24)
    walls = olat.WALL_XM | olat.WALL_XP | olat.WALL_YM | olat.WALL_YP
    p = lbm.lbm_default_params()
    p.g = 1e-2                         # terminal velocity ~0.02 per step
    col, sim = _coupled_pair(dims, 1.5, walls, [[8.0, 8.0, 23.3]], [[0, 0, 0.02]], [1.5], p)
    lbm.lbm_step(col.ctx, 60)
    sim.run(60)
    b = lbm.lbm_get_bubbles(col.ctx)
    assert sim.x[0, 2] < 20.0          # wrapped through the top face
    assert np.abs(b["pos"] - sim.x).max() < X_RTOL * 24.0
    _, u_gpu = col.fields()
    _, u_or = sim.fields()
    assert rel_linf(u_gpu, u_or) < U_RTOL


def test_one_way_coupling_leaves_liquid_at_rest():
    dims = (16, 16, 32)
    p = lbm.lbm_default_params()
    p.two_way = 0
    col = lbm.Column(dims, 1.6, olat.ALL_WALLS, params=p)
    lbm.lbm_set_bubbles(col.ctx, [8.0, 8.0, 8.0], [0, 0, 0], [2.0])
    lbm.lbm_step(col.ctx, 20)
    _, u = col.fields()
    assert np.abs(u).max() == 0.0
    b = lbm.lbm_get_bubbles(col.ctx)
    assert b["vel"][0, 2] > 0.0


def test_mass_conserved_and_totals():
    dims = (24, 20, 40)
    pos, vel, diam = workloads.swarm(dims, 12, seed=5)
    p = lbm.lbm_default_params()
    p.g = 1e-3
    col = lbm.Column(dims, 1.8, olat.ALL_WALLS, params=p)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    m0 = lbm.lbm_get_totals(col.ctx)
    assert abs(m0[0] - np.prod(dims)) < 1e-9 and np.abs(m0[1:]).max() == 0.0
    lbm.lbm_step(col.ctx, 200)
    t = lbm.lbm_get_totals(col.ctx)
    rho, u = col.fields()
    assert abs(t[0] - m0[0]) < 1e-9 * m0[0]
    assert abs(t[0] - rho.sum()) < 1e-9 * m0[0]
    assert np.allclose(t[1:], (rho[None] * u).sum(axis=(1, 2, 3)), rtol=1e-9, atol=1e-15)


def test_instability_is_reported_and_sticky():
    # Beyond the stable range (the paper finds omega = 1.98 unstable) a fast
    # shear flow blows up; the step reports it instead of faulting or hanging.
    dims = (16, 16, 16)
    col = lbm.Column(dims, 1.999, 0)
    z = np.arange(16) + 0.5
    u = np.zeros((3, 16, 16, 16))
    u[0] = 0.28 * np.sign(np.sin(2 * np.pi * z / 16))[:, None, None]
    lbm.lbm_set_fields(col.ctx, None, u.reshape(-1))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(col.ctx, 2000)
    assert e.value.code == lbm.LBM_ERR_UNSTABLE
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(col.ctx, 1)
    assert e.value.code == lbm.LBM_ERR_UNSTABLE
    lbm.lbm_set_fields(col.ctx)          # reset to rest clears the flag
    lbm.lbm_step(col.ctx, 5)


def test_torch_allocator_and_stream():
    import torch
    dims = workloads.SINGLE_SMALL
    pos, vel, diam = workloads.single_bubble(dims)
    before = torch.cuda.memory_allocated()
    col = lbm.Column(dims, 1.6, olat.ALL_WALLS, torch_plumbing=True)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    assert torch.cuda.memory_allocated() - before >= 2 * 19 * 4 * np.prod(dims)
    lbm.lbm_step(col.ctx, 10)
    ref = lbm.Column(dims, 1.6, olat.ALL_WALLS)
    lbm.lbm_set_bubbles(ref.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    lbm.lbm_step(ref.ctx, 10)
    assert np.array_equal(col.fields()[1], ref.fields()[1])       # deterministic
    col.close()
    assert torch.cuda.memory_allocated() == before


@pytest.mark.parametrize("omega", [1.0, 1.6, 1.9])
def test_large_column_sampled_against_oracle(omega):
    # Full 256x256x512 column in the benchmark's launch configuration.  After k
    # steps the disturbance of a bubble released at rest has moved at most one
    # node per step from its window, so an oracle run on a periodic crop around
    # the bubble (wider than window + k on every side) must give the same field
    # there.  Checked after 12 steps on the 40^3 crop.
    dims = workloads.SINGLE_LARGE
    pos, vel, diam = workloads.single_bubble(dims)      # (128, 128, 64)
    k = 12
    crop = 40
    col = lbm.Column(dims, omega, olat.ALL_WALLS)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)
    lbm.lbm_step(col.ctx, k)
    _, u_gpu = col.fields()
    nx, ny, nz = dims
    u_gpu = u_gpu.reshape(3, nz, ny, nx)
    lo = [int(pos[0, a]) - crop // 2 for a in range(3)]
    sub = u_gpu[:, lo[2]:lo[2] + crop, lo[1]:lo[1] + crop, lo[0]:lo[0] + crop]
    outside = u_gpu.copy()
    outside[:, lo[2]:lo[2] + crop, lo[1]:lo[1] + crop, lo[0]:lo[0] + crop] = 0.0
    assert np.abs(outside).max() == 0.0
    sim = OracleSim((crop, crop, crop), omega, 0)
    sim.set_bubbles(pos - np.array(lo, dtype=np.float64), vel, diam)
    sim.run(k)
    _, u_or = sim.fields()
    assert rel_linf(sub, u_or) < U_RTOL
    b = lbm.lbm_get_bubbles(col.ctx)
    assert np.abs(b["pos"] - (sim.x + np.array(lo))).max() < X_RTOL * 512
