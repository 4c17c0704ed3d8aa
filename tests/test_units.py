"""Appendix A unit conversion (lbm_units_from_physical) against Table 5 and the
appendix's worked 4 mm case; the replay set-ups built from it (host only)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table5_unit_conversion.txt")


def _table5():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [float(x) for x in line.split()]
            rows.append(dict(zip(("aspect", "lcf", "mcf", "tcf", "dx", "w", "depth", "h", "d_mm",
                                  "d_lu"), v)))
    return rows


def test_appendix_a_worked_case(libpath):
    # Appendix A: dx = 1.25 * 4 mm = 0.005 m, dt = 1e-4 s, rho 1000 -> 1:
    # LCF = 200, TCF = 10000, MCF = 8000; h, w, d = 90, 30, 30; d_b = 0.8.
    from paper_1710_07073_gb300 import lbm, replay
    u, p, omega = lbm.lbm_units_from_physical(0.005, 1e-4)
    assert (u.lcf, u.tcf, u.mcf) == pytest.approx((200.0, 10000.0, 8000.0), rel=1e-14)
    su = replay.setup(4, 1.25)
    assert su["dims"] == (30, 30, 90)
    assert su["d_lu"] == pytest.approx(0.8, rel=1e-14)
    # Table 3 in lattice units: g = 9.81 LCF/TCF^2, sigma = 0.073 MCF/TCF^2
    # (the library's default sigma), nu = 1e-6 LCF^2/TCF = 4e-6 (Eq. 9).
    assert p.g == pytest.approx(1.962e-5, rel=1e-12)
    assert p.sigma == pytest.approx(5.84e-6, rel=1e-12)
    assert p.sigma == pytest.approx(lbm.lbm_default_params().sigma, rel=1e-12)
    assert p.rho_l == 1.0 and p.rho_ratio == pytest.approx(1e-3, rel=1e-14)
    assert omega == pytest.approx(1.0 / (3.0 * 4e-6 + 0.5), rel=1e-14)


def test_table5_rows(libpath):
    from paper_1710_07073_gb300 import lbm, replay
    misprints = []
    for r in _table5():
        u, _, _ = lbm.lbm_units_from_physical(r["dx"], 1e-4)
        assert u.lcf == pytest.approx(r["lcf"], rel=1e-12)
        assert u.tcf == pytest.approx(r["tcf"], rel=1e-12)
        if abs(u.mcf - r["mcf"]) > 1e-9 * r["mcf"]:
            misprints.append((r["aspect"], r["d_mm"], r["mcf"], u.mcf))
        assert r["dx"] == pytest.approx(r["aspect"] * r["d_mm"] * 1e-3, rel=1e-12)
        su = replay.setup(r["d_mm"], r["aspect"])
        assert su["dims"] == (r["w"], r["depth"], r["h"])
        assert su["d_lu"] == pytest.approx(r["d_lu"], rel=1e-12)
    # Only the sixth row's MCF (printed 640000 for LCF = 400) disagrees.
    assert misprints == [(0.3125, 8.0, 640000.0, pytest.approx(64000.0, rel=1e-12))]


def test_conversion_scales_by_dimension(libpath):
    # A quantity of dimension m^a s^b kg^c scales by LCF^a TCF^b MCF^c:
    # doubling dx halves LCF, divides MCF by 8 and g_lu by 2, nu_lu by 4.
    from paper_1710_07073_gb300 import lbm
    u1, p1, o1 = lbm.lbm_units_from_physical(0.004, 2e-4, mu_l=3e-3, sigma=0.05, g=7.0)
    u2, p2, o2 = lbm.lbm_units_from_physical(0.008, 2e-4, mu_l=3e-3, sigma=0.05, g=7.0)
    assert u1.lcf == pytest.approx(2 * u2.lcf) and u1.mcf == pytest.approx(8 * u2.mcf)
    assert p1.g == pytest.approx(2 * p2.g) and p1.sigma == pytest.approx(8 * p2.sigma)
    nu1, nu2 = (1.0 / o1 - 0.5) / 3.0, (1.0 / o2 - 0.5) / 3.0
    assert nu1 == pytest.approx(4 * nu2, rel=1e-9)
    assert nu1 == pytest.approx(3e-3 / 1000.0 * 250.0 ** 2 / 5000.0, rel=1e-9)


@pytest.mark.parametrize("bad", [dict(dx=0.0), dict(dt=-1.0), dict(rho_b=1000.0),
                                 dict(mu_l=0.0), dict(sigma=float("nan")), dict(g=-9.81)])
def test_conversion_rejects_bad_input(libpath, bad):
    from paper_1710_07073_gb300 import lbm
    args = dict(dx=0.005, dt=1e-4)
    args.update(bad)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_units_from_physical(**args)
    assert e.value.code == lbm.LBM_ERR_ARG


def test_replay_setups_fit_the_library(libpath):
    # Every replay case passes the library's argument checks on the host:
    # diameters within LBM_MAX_DIAMETER, the bubble inside its column.
    from paper_1710_07073_gb300 import lbm, replay
    cases = [(d, 1.25) for d in replay.E2_DIAMETERS_MM] + replay.E4_CASES
    for d_mm, a in cases:
        su = replay.setup(d_mm, a)
        assert 0.0 < su["d_lu"] <= lbm.LBM_MAX_DIAMETER
        nx, ny, nz = su["dims"]
        x, y, z = su["pos"]
        assert 0.0 < x < nx and 0.0 < y < ny and su["d_lu"] / 2 < z < nz
        assert 0.0 < su["omega"] < 2.0
        assert math.isclose(su["units"].tcf, 1e4)
