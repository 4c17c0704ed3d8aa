"""Shifted 16-bit population storage (FP16 / BF16) against the FP64 oracle.

Populations are stored as (f_j - w_j rho0) * scale / w_j in 16 bits; all
collision arithmetic stays FP32.  The error is stated per field and for the
bubble's terminal velocity (mean u_b,z over the last 200 of 1000 steps) of the
single-bubble column (32x32x64, omega 1.6, d = 2, bounce-back walls).

Bars: FP32 storage matches the oracle to 1e-5 (relative L-inf, velocity);
FP16 storage keeps the terminal velocity within 1 % of the oracle; BF16's
8-bit mantissa is measured and held to 5 %.
"""
import os

import numpy as np
import pytest

from oracle.step import OracleSim
from oracle import lattice as olat
from paper_1710_07073_gb300 import lbm, workloads
from tests.gpu_util import lib_pops_to_oracle, oracle_pops_to_lib, params_for_oracle, rel_linf

pytestmark = pytest.mark.gpu

STEPS = 1000
TAIL = 200


@pytest.fixture(scope="module")
def oracle_run():
    dims = workloads.SINGLE_SMALL
    pos, vel, diam = workloads.single_bubble(dims)
    p = lbm.lbm_default_params()
    sim = OracleSim(dims, 1.6, olat.ALL_WALLS, params_for_oracle(p, 1.6))
    sim.set_bubbles(pos, vel, diam)
    uz = []
    for _ in range(STEPS):
        sim.step()
        uz.append(sim.u[0, 2])
    rho, u = sim.fields()
    return dict(dims=dims, pos=pos, vel=vel, diam=diam, rho=rho, u=u,
                vt=float(np.mean(uz[-TAIL:])), x=sim.x.copy())


def _gpu_run(storage, scale, o):
    assert os.path.exists(lbm.LIB_PATH)
    col = lbm.Column(o["dims"], 1.6, olat.ALL_WALLS, storage, scale)
    lbm.lbm_set_bubbles(col.ctx, o["pos"].reshape(-1), o["vel"].reshape(-1), o["diam"])
    uz = []
    for _ in range(STEPS):
        lbm.lbm_step(col.ctx, 1)
        uz.append(lbm.lbm_get_bubbles(col.ctx)["vel"][0, 2])
    rho, u = col.fields()
    b = lbm.lbm_get_bubbles(col.ctx)
    return dict(rho=rho, u=u, vt=float(np.mean(uz[-TAIL:])), x=b["pos"])


def _report(name, g, o):
    err = {
        "u_rel_linf": rel_linf(g["u"], o["u"]),
        "uz_rel_linf": rel_linf(g["u"][2], o["u"][2]),
        "rho_abs_linf": float(np.abs(g["rho"] - o["rho"]).max()),
        "vt_rel": abs(g["vt"] / o["vt"] - 1.0),
        "x_rel": float(np.abs(g["x"] - o["x"]).max() / np.abs(o["x"]).max()),
    }
    print("%s storage vs FP64 oracle: %s" % (name, err))
    return err


def test_fp32_storage(oracle_run):
    e = _report("FP32", _gpu_run(lbm.LBM_STORE_F32, 1.0, oracle_run), oracle_run)
    assert e["u_rel_linf"] < 1e-5 and e["vt_rel"] < 1e-5 and e["x_rel"] < 1e-6


def test_fp16_storage(oracle_run):
    e = _report("FP16", _gpu_run(lbm.LBM_STORE_F16, 256.0, oracle_run), oracle_run)
    assert e["vt_rel"] < 0.01
    assert e["u_rel_linf"] < 0.02
    assert e["rho_abs_linf"] < 1e-6


def test_bf16_storage(oracle_run):
    e = _report("BF16", _gpu_run(lbm.LBM_STORE_BF16, 1.0, oracle_run), oracle_run)
    assert e["vt_rel"] < 0.05


@pytest.mark.parametrize("storage,scale,tol", [(lbm.LBM_STORE_F16, 256.0, 2.0 ** -11),
                                               (lbm.LBM_STORE_BF16, 1.0, 2.0 ** -8)])
def test_16bit_roundtrip_within_format_rounding(storage, scale, tol):
    # Each stored value is (f - w rho0) scale / w rounded once to nearest even:
    # the round trip error is at most half an ulp of that value, back in f units.
    dims = (37, 9, 11)
    rng = np.random.default_rng(2)
    rho, u = workloads.random_fields(dims, seed=2, amp=1e-3, rho_amp=1e-3)
    f = olat.equilibrium(rho, u) * (1.0 + 1e-4 * rng.standard_normal((19,) + rho.shape))
    col = lbm.Column(dims, 1.6, olat.ALL_WALLS, storage, scale)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    back = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    dev = f - olat.W[:, None, None, None]
    # Below FP16's normal range the spacing is fixed: half of 2^-24, in f units.
    atol = 2.0 ** -25 * (1.0 / 3.0) / scale
    assert (np.abs(back - f) <= tol * np.abs(dev) + atol).all()


def test_fp16_step_matches_oracle_on_rounded_input():
    # One step from populations that FP16 represents exactly: the only error is
    # the FP32 arithmetic plus one FP16 rounding of the result.
    dims = (37, 9, 11)
    rho, u = workloads.random_fields(dims, seed=8, amp=1e-3, rho_amp=1e-3)
    f = olat.equilibrium(rho, u)
    col = lbm.Column(dims, 1.7, olat.ALL_WALLS, lbm.LBM_STORE_F16, 256.0)
    lbm.lbm_set_populations(col.ctx, oracle_pops_to_lib(f))
    f_exact = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    lbm.lbm_step(col.ctx, 1)
    got = lib_pops_to_oracle(lbm.lbm_get_populations(col.ctx), dims)
    want = olat.lb_step(f_exact, 1.7, olat.ALL_WALLS)
    dev = np.abs(want - olat.W[:, None, None, None])
    assert (np.abs(got - want) <= 2.0 ** -11 * dev + 1e-10).all()
