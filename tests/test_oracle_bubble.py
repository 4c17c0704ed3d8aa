"""Pins for the oracle's bubble closures and update (Table 1, Eq. 1-4, Eq. 22-25)."""
import math

import numpy as np
import pytest

from oracle import bubble as bub
from oracle import lattice as lat
from oracle import validation as val

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                    "table4_terminal_velocity.txt")


def _table4():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            d, fb, me = line.split()
            rows.append((float(d) * 1e-3, float(fb), float(me)))
    return rows


def test_table4_force_balance_column():
    # Table 4 "Force balance eq." with Table 3 properties: Eq. 23 with the
    # Table 1 drag law, Eo = d^2-form (Eq. 3) and rho_l restored in Eq. 24.
    for d, fb, _ in _table4():
        v = val.terminal_velocity_force_balance(d, 1000.0, 1.0, 1e-3, 0.073, 9.81)
        assert abs(v - fb) <= 1e-4 + 1e-12, (d, v, fb)


def test_table4_force_balance_rejects_printed_eo():
    # With Eo printed without d_b^2 (Eq. 3 as typeset) the column is missed.
    misses = 0
    for d, fb, _ in _table4():
        sigma_eff = 0.073 * d          # turns d^2/sigma into d/sigma
        v = val.terminal_velocity_force_balance(d, 1000.0, 1.0, 1e-3, sigma_eff, 9.81)
        misses += abs(v - fb) > 1e-3
    assert misses == 9


def test_table4_mendelson_column():
    # Table 4 "Mendelson eq.": Eq. 25.
    for d, _, me in _table4():
        v = val.terminal_velocity_mendelson(d, 1000.0, 0.073, 9.81)
        assert abs(v - me) <= 5e-5 + 1e-12, (d, v, me)


def test_drag_coefficient_branches():
    # Table 1 C_D: Stokes-like branch at small Re, 48/Re cap, Eo plateau.
    assert val.drag_cd(1e-3, 0.0) == pytest.approx(24.0 / 1e-3 * (1 + 0.15 * 1e-3 ** 0.687))
    # At Re = 1000 the 48/Re cap is below the Schiller-Naumann value.
    assert val.drag_cd(1000.0, 0.0) == pytest.approx(0.048)
    assert val.drag_cd(1e5, 2.0) == pytest.approx(8.0 / 3.0 * 2.0 / 6.0)
    p = bub.BubbleParams(1.6)
    v = np.array([0.0, 0.0, 2e-4])
    d = 2.0
    re = bub.reynolds(v, d, p)
    cd = bub.drag_coefficient(re, bub.eotvos(d, p), p)
    assert bub.drag_cd_times_speed(v, d, p) == pytest.approx(cd * 2e-4, rel=1e-13)
    # Finite at rest: C_D |v| -> 24 nu / d.
    assert bub.drag_cd_times_speed(np.zeros(3), d, p) == pytest.approx(24.0 * p.nu / d)


def test_linear_drag_update_has_closed_form():
    # With a = 0 in the drag law and Eo -> 0, F_D = -3 pi mu d v (Stokes).  The
    # explicit update of Eq. 4 with m_eff then is the geometric sequence
    # v_k = v_T (1 - (1 - K dt/m)^k), v_T = F_B / K, K = 3 pi rho_l nu d.
    p = bub.BubbleParams(1.6, sn_coeff=0.0, sigma=1e30)
    d = 2.0
    dims = (32, 32, 64)
    x = np.array([16.0, 16.0, 8.0])
    u = np.zeros(3)
    kdrag = 3.0 * math.pi * p.rho_l * p.nu * d
    vt = bub.buoyancy_force(d, p)[2] / kdrag
    q = 1.0 - kdrag * p.dt_b / bub.effective_mass(d, p)
    z = x[2]
    for step in range(1, 21):
        x, u, psi = bub.advance(x, u, d, np.zeros(3), np.zeros(3), dims, lat.ALL_WALLS, p)
        k = step * p.substeps
        assert u[2] == pytest.approx(vt * (1.0 - q ** k), rel=1e-12)
        # Position: sum of v_k dt_b over the sub-steps.
        z += sum(vt * (1.0 - q ** i) for i in range(k - p.substeps + 1, k + 1)) * p.dt_b
        assert x[2] == pytest.approx(z, rel=1e-13)
    # The reaction is minus the mean drag over the sub-steps: equal and opposite impulse.
    assert psi[2] > 0.0


def test_terminal_velocity_in_lattice_units():
    # Config "single bubble" closures in lattice units (omega 1.6, g 1e-5,
    # d = 2): the bubble in still liquid settles at the Eq. 23 root.
    p = bub.BubbleParams(1.6)
    d = 2.0
    x, u = np.array([16.0, 16.0, 8.0]), np.zeros(3)
    for _ in range(400):
        x, u, psi = bub.advance(x, u, d, np.zeros(3), np.zeros(3), (32, 32, 64),
                                lat.ALL_WALLS, p)
    vt = val.terminal_velocity_force_balance(d, p.rho_l, p.rho_b, p.rho_l * p.nu, p.sigma, p.g)
    assert u[2] == pytest.approx(vt, rel=1e-10)
    # Force balance: the reaction equals the net buoyancy at terminal velocity.
    assert psi[2] == pytest.approx(bub.buoyancy_force(d, p)[2], rel=1e-9)


def test_eq22_history_matches_update():
    # Eq. 22 integrated with the bubble's sub-step and m_eff reproduces the
    # velocity history of the Newton update in still liquid.
    p = bub.BubbleParams(1.9)
    d = 1.5
    hist = val.relative_velocity_history(d, p.rho_l, p.rho_b, p.rho_l * p.nu, p.sigma, p.g,
                                         bub.effective_mass(d, p), p.dt_b, 300)
    x, u = np.array([8.0, 8.0, 8.0]), np.zeros(3)
    for step in range(30):
        x, u, _ = bub.advance(x, u, d, np.zeros(3), np.zeros(3), (16, 16, 64), lat.ALL_WALLS, p)
        assert u[2] == pytest.approx(hist[(step + 1) * p.substeps - 1], rel=1e-12)


def test_wall_clamp_and_periodic_wrap():
    p = bub.BubbleParams(1.6, g=1e-3)
    d = 2.0
    # Pushed against the top wall: held at nz - r with no velocity into it.
    x, u, _ = bub.advance([4.0, 4.0, 14.95], [0.0, 0.0, 0.1], d, np.zeros(3), np.zeros(3),
                          (8, 8, 16), lat.ALL_WALLS, p)
    assert x[2] == 15.0 and u[2] == 0.0
    # Periodic z: wraps around.
    x, u, _ = bub.advance([4.0, 4.0, 15.99], [0.0, 0.0, 0.1], d, np.zeros(3), np.zeros(3),
                          (8, 8, 16), lat.WALL_XM | lat.WALL_XP | lat.WALL_YM | lat.WALL_YP, p)
    assert 0.0 <= x[2] < 1.0


def test_added_mass_liquid_acceleration_closed_form():
    # Table 1's virtual-mass force carries C_A rho_l V_b D_t u_l.  With linear
    # (Stokes) drag F_D = -K (u - u_l), K = 3 pi rho_l nu d, a constant u_l and
    # a constant D_t u_l, the explicit update of Eq. 4 with m_eff is the
    # geometric sequence u_k = v_inf (1 - q^k) from rest, with
    # v_inf = u_l + (F_B + C_A rho_l V_b D_t u_l) / K and q = 1 - K dt_b / m_eff.
    # Position: x_k = x_0 + sum_{i <= k} u_i dt_b; reaction: minus the mean drag
    # of a liquid step's sub-steps, psi = K/N sum (u_i - u_l).
    p = bub.BubbleParams(1.7, sn_coeff=0.0, sigma=1e30)
    d = 1.8
    dims = (64, 64, 64)
    ul = np.array([1e-4, -2e-4, 3e-4])
    dul = np.array([2e-6, 1e-6, -3e-6])
    kdrag = 3.0 * math.pi * p.rho_l * p.nu * d
    meff = bub.effective_mass(d, p)
    force = bub.buoyancy_force(d, p) + p.c_added_mass * p.rho_l * bub.volume(d) * dul
    vinf = ul + force / kdrag
    q = 1.0 - kdrag * p.dt_b / meff
    x0 = np.array([32.0, 32.0, 20.0])
    x, u = x0.copy(), np.zeros(3)
    xs = x0.copy()
    for step in range(1, 11):
        k0 = (step - 1) * p.substeps
        x, u, psi = bub.advance(x, u, d, ul, dul, dims, lat.ALL_WALLS, p)
        k = step * p.substeps
        np.testing.assert_allclose(u, vinf * (1.0 - q ** k), rtol=1e-11, atol=0)
        xs = xs + sum(vinf * (1.0 - q ** i) for i in range(k0 + 1, k + 1)) * p.dt_b
        np.testing.assert_allclose(x, xs, rtol=1e-14, atol=0)
        start = [vinf * (1.0 - q ** i) for i in range(k0, k)]   # velocity at each sub-step's start
        psi_exp = kdrag / p.substeps * sum(s - ul for s in start)
        np.testing.assert_allclose(psi, psi_exp, rtol=1e-10, atol=0)
