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


# ---- lift and stress-gradient forces (Table 1) --------------------------------

def test_deformed_eotvos_number():
    # Eo_d = Eo / E^(2/3), E = 1 / (1 + 0.163 Eo^0.757): E -> 1 for a small
    # bubble; Eo = 1 by hand: E = 1/1.163, Eo_d = 1.163^(2/3).
    assert bub.eotvos_deformed(1e-12) == pytest.approx(1e-12, rel=1e-6)
    assert bub.eotvos_deformed(1.0) == pytest.approx(1.163 ** (2.0 / 3.0), rel=1e-14)


def test_lift_coefficient_branches_join():
    # With the published constant 0.474 in f(Eo_d), the three branches of
    # Table 1 join: at Eo_d = 4 the min() branch equals f (large Re), and at
    # Eo_d = 10 f(10) = -0.27 meets the -0.29 plateau within 0.02.  Small,
    # nearly round bubbles take the tanh branch: C_L -> 0.288 at large Re,
    # 0.288 * 0.121 Re at small Re.  As printed (no constant) f(10) = -0.744:
    # a jump of 0.45 to -0.29.
    f4, f10 = bub.lift_f(4.0), bub.lift_f(10.0)
    assert f4 == pytest.approx(0.2052, abs=1e-4)
    assert f10 == pytest.approx(-0.270, abs=1e-3)
    assert abs(f10 - (-0.29)) < 0.025
    printed = lambda e: 0.00105 * e ** 3 - 0.0159 * e ** 2 - 0.0204 * e
    assert abs(printed(10.0) - (-0.29)) > 0.4
    # Eo chosen so that Eo_d sits just below / above 4 and 10.
    def eo_for(eo_d):
        lo, hi = 1e-9, 1e3
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if bub.eotvos_deformed(mid) < eo_d else (lo, mid)
        return 0.5 * (lo + hi)
    assert bub.lift_coefficient(1e4, eo_for(4.0 - 1e-9)) == pytest.approx(f4, abs=1e-6)
    assert bub.lift_coefficient(1e4, eo_for(4.0 + 1e-9)) == pytest.approx(f4, abs=1e-6)
    assert bub.lift_coefficient(1e4, eo_for(10.0 + 1e-6)) == -0.29
    assert bub.lift_coefficient(1e4, 1e-6) == pytest.approx(0.288, rel=1e-12)
    assert bub.lift_coefficient(1e-3, 1e-6) == pytest.approx(0.288 * 0.121e-3, rel=1e-6)


def test_lift_rotates_the_slip_velocity():
    # Lift without drag in a uniform vorticity Omega z: with the horizontal
    # slip w = u_b - u_l = (w_x, w_y) as z = w_x + i w_y, F_L = -C_L rho_l V_b
    # (w x Omega z) = i C_L rho_l V_b Omega z, so each explicit sub-step of
    # Eq. 4 multiplies z by (1 + i c), c = C_L rho_l V_b Omega dt_b / m_eff,
    # while buoyancy alone accelerates u_z.  A large Eo puts C_L on its -0.29
    # plateau.  This fixes the order of the cross product, the sign and the
    # coefficient of Table 1's lift.
    p = bub.BubbleParams(1.6, sigma=1e-9, drag_scale=0.0, lift=True)
    d = 2.0
    omega_l = np.array([0.0, 0.0, 3e-3])
    assert bub.lift_coefficient(1.0, bub.eotvos(d, p)) == -0.29
    c = -0.29 * p.rho_l * bub.volume(d) * omega_l[2] * p.dt_b / bub.effective_mass(d, p)
    x, u = np.array([32.0, 32.0, 32.0]), np.array([1e-3, 0.0, 0.0])
    z = complex(u[0], u[1])
    xs = x.copy()
    for step in range(1, 6):
        zs = [z * (1 + 1j * c) ** k for k in range(p.substeps + 1)]
        x, u, psi = bub.advance(x, u, d, np.zeros(3), np.zeros(3), (64, 64, 64),
                                lat.ALL_WALLS, p, omega_l=omega_l)
        assert complex(u[0], u[1]) == pytest.approx(zs[-1], rel=1e-12)
        kb = bub.buoyancy_force(d, p)[2] * p.dt_b / bub.effective_mass(d, p)
        assert u[2] == pytest.approx(kb * step * p.substeps, rel=1e-12)
        xs[:2] = xs[:2] + p.dt_b * np.array([sum(zz.real for zz in zs[1:]),
                                            sum(zz.imag for zz in zs[1:])])
        np.testing.assert_allclose(x[:2], xs[:2], rtol=1e-15, atol=0)
        # Reaction: minus the mean lift over the sub-steps.
        fl = [1j * -0.29 * p.rho_l * bub.volume(d) * omega_l[2] * zz for zz in zs[:-1]]
        mean = sum(fl) / p.substeps
        assert complex(psi[0], psi[1]) == pytest.approx(-mean, rel=1e-12)
        z = zs[-1]


def test_stress_gradient_adds_rho_l_v_b_dtul():
    # Table 1: F_S = rho_l V_b D_t u_l, on top of the virtual mass's
    # C_A rho_l V_b D_t u_l: with Stokes drag the update tends to
    # u_l + (F_B + (1 + C_A) rho_l V_b D_t u_l) / K.
    p = bub.BubbleParams(1.7, sn_coeff=0.0, sigma=1e30, stress_gradient=True)
    d = 1.8
    ul = np.array([1e-4, -2e-4, 3e-4])
    dul = np.array([2e-6, 1e-6, -3e-6])
    kdrag = 3.0 * math.pi * p.rho_l * p.nu * d
    force = bub.buoyancy_force(d, p) + (1.0 + p.c_added_mass) * p.rho_l * bub.volume(d) * dul
    vinf = ul + force / kdrag
    q = 1.0 - kdrag * p.dt_b / bub.effective_mass(d, p)
    x, u = np.array([32.0, 32.0, 20.0]), np.zeros(3)
    for step in range(1, 6):
        x, u, _ = bub.advance(x, u, d, ul, dul, (64, 64, 64), lat.ALL_WALLS, p)
        np.testing.assert_allclose(u, vinf * (1.0 - q ** (step * p.substeps)), rtol=1e-11, atol=0)


@pytest.mark.parametrize("lift,stress", [(False, False), (True, True)])
def test_reaction_all_interphase_forces_closed_form(lift, stress):
    # Sec. 3.2's psi_b = -sum F over the interphase forces F_D + F_L + F_S +
    # F_VM, with F_VM = C_A rho_l V_b (D_t u_l - a_k): since m_eff a_k =
    # F_B + F_D + F_L + F_S + C_A rho_l V_b D_t u_l, the sum is m_b a_k - F_B,
    # and its mean over the sub-steps is m_b (u_new - u_old)/dt_l - F_B.  So
    # psi = F_B - m_b (u_new - u_old)/dt_l whatever the closures (no clamp).
    rng = np.random.default_rng(41)
    for _ in range(20):
        p = bub.BubbleParams(1.6, g=1e-4, lift=lift, stress_gradient=stress, reaction="all",
                             rho_ratio=rng.uniform(1e-3, 0.5))
        d = rng.uniform(1.0, 3.0)
        x = np.array([20.0, 20.0, 20.0])
        u = rng.normal(scale=1e-3, size=3)
        ul = rng.normal(scale=1e-3, size=3)
        dul = rng.normal(scale=1e-5, size=3)
        om = rng.normal(scale=1e-3, size=3)
        x1, u1, psi = bub.advance(x, u, d, ul, dul, (40, 40, 40), lat.ALL_WALLS, p, omega_l=om)
        mb = p.rho_b * bub.volume(d)
        expect = bub.buoyancy_force(d, p) - mb * (u1 - u) / p.dt_l
        np.testing.assert_allclose(psi, expect, rtol=1e-9, atol=1e-12 * np.abs(expect).max())
        # and it differs from Algorithm 1's -(F_D + F_L) while the bubble accelerates
        p0 = bub.BubbleParams(1.6, g=1e-4, lift=lift, stress_gradient=stress,
                              rho_ratio=p.rho_b / p.rho_l)
        _, _, psi0 = bub.advance(x, u, d, ul, dul, (40, 40, 40), lat.ALL_WALLS, p0, omega_l=om)
        assert np.abs(psi0 - psi).max() > 1e-3 * np.abs(psi).max()


def test_reaction_all_of_massless_bubble_is_buoyancy():
    # m_b = 0: the liquid takes the whole buoyancy at every step, however far
    # from terminal the bubble is.
    p = bub.BubbleParams(1.6, rho_ratio=0.0, reaction="all")
    x, u = np.array([8.0, 8.0, 8.0]), np.zeros(3)
    for _ in range(3):
        x, u, psi = bub.advance(x, u, 2.0, np.zeros(3), np.array([1e-6, 0.0, 2e-6]),
                                (16, 16, 32), lat.ALL_WALLS, p)
        np.testing.assert_allclose(psi, bub.buoyancy_force(2.0, p), rtol=1e-12, atol=1e-20)


def test_mapping_and_reaction_switches_validated():
    with pytest.raises(ValueError):
        bub.BubbleParams(1.6, mapping="nodal")
    with pytest.raises(ValueError):
        bub.BubbleParams(1.6, reaction="drag")
