"""Pins for the oracle's coupled loop (Algorithm 1)."""
import numpy as np
import pytest

from oracle import bubble as bub
from oracle import lattice as lat
from oracle import validation as val
from oracle.step import OracleSim


def test_two_way_exchange_is_equal_and_opposite():
    # Algorithm 1 step 6 + Eq. 21 + Eq. 13-15: on a periodic box the liquid
    # gains exactly the reaction psi_b = -mean F_D of every bubble per step.
    sim = OracleSim((12, 12, 16), 1.6, 0)
    sim.set_bubbles([[6.0, 6.2, 5.0], [3.1, 9.0, 11.5]], [[0, 0, 0], [1e-4, 0, 0]], [2.0, 1.5])
    for _ in range(5):
        p0 = lat.momentum(sim.f).sum(axis=(1, 2, 3))
        sim.step()
        p1 = lat.momentum(sim.f).sum(axis=(1, 2, 3))
        assert np.allclose(p1 - p0, sim.psi.sum(axis=0), rtol=1e-9, atol=1e-14)
        assert np.allclose(sim.last_force.sum(axis=(1, 2, 3)), sim.psi.sum(axis=0),
                           rtol=1e-12, atol=0)


def test_mass_conserved_with_walls_and_bubbles():
    sim = OracleSim((10, 10, 20), 1.3, lat.ALL_WALLS)
    sim.set_bubbles([[5.0, 5.0, 5.0]], [[0, 0, 0]], [2.0])
    m0 = lat.density(sim.f).sum()
    sim.run(10)
    assert abs(lat.density(sim.f).sum() - m0) < 1e-11


def test_slip_velocity_reaches_force_balance_terminal_velocity():
    # Single bubble rising in stagnant liquid: the slip |u_b - u_l(x_b)| tends
    # to the Eq. 23 terminal velocity (drag balances net buoyancy; the added
    # mass term vanishes once the liquid's Lagrangian acceleration is small).
    omega = 1.6
    sim = OracleSim((16, 16, 32), omega, lat.ALL_WALLS)
    sim.set_bubbles([[8.0, 8.0, 8.0]], [[0, 0, 0]], [2.0])
    sim.run(120)
    p = sim.p
    vt = val.terminal_velocity_force_balance(2.0, p.rho_l, p.rho_b, p.rho_l * p.nu, p.sigma, p.g)
    slip = sim.u[0] - sim.ul[0]
    assert abs(slip[2] / vt - 1.0) < 0.01
    assert abs(slip[0]) < 1e-3 * vt and abs(slip[1]) < 1e-3 * vt
    # The liquid has been dragged upward around the bubble.
    assert sim.ul[0, 2] > 0.0


def test_bubble_deactivated_at_top_wall():
    p = bub.BubbleParams(1.6, g=1e-2)
    sim = OracleSim((8, 8, 12), 1.6, lat.ALL_WALLS, p)
    sim.set_bubbles([[4.0, 4.0, 10.5]], [[0, 0, 0.05]], [1.0])
    for _ in range(400):
        sim.step()
        if not sim.active[0]:
            break
    assert not sim.active[0]
    x_stop = sim.x[0].copy()
    sim.run(3)
    assert np.array_equal(sim.x[0], x_stop)
    assert sim.last_force is None


@pytest.mark.parametrize("point", [False, True])
def test_reaction_all_conserves_mixture_momentum(point):
    # With psi_b = -sum F (Sec. 3.2) Newton's third law holds for the mixture:
    # on a periodic box the liquid's momentum sum c_j f_j plus the bubbles'
    # own momentum m_b u_b grows by exactly the buoyancy sum F_B per step
    # (liquid: + sum psi, Eq. 12-15; bubble: m_b (u_new - u_old) = F_B - psi).
    # With Algorithm 1's -(F_D + F_L) the added-mass exchange is missing.
    def run(reaction):
        p = bub.BubbleParams(1.6, g=1e-4, rho_ratio=0.05, reaction=reaction,
                             mapping="point" if point else "cell")
        sim = OracleSim((12, 12, 16), 1.6, 0, p)
        sim.set_bubbles([[6.0, 6.2, 5.0], [3.1, 9.0, 11.5]], [[0, 0, 0], [1e-4, 0, 0]],
                        [2.0, 1.5])
        mb = p.rho_b * bub.volume(sim.d)
        fb = sum(bub.buoyancy_force(d, p) for d in sim.d)
        gaps = []
        for _ in range(6):
            p0 = lat.momentum(sim.f).sum(axis=(1, 2, 3)) + (mb[:, None] * sim.u).sum(axis=0)
            sim.step()
            p1 = lat.momentum(sim.f).sum(axis=(1, 2, 3)) + (mb[:, None] * sim.u).sum(axis=0)
            gaps.append(np.abs(p1 - p0 - fb).max() / np.abs(fb).max())
        return max(gaps)
    assert run("all") < 1e-9
    assert run("drag_lift") > 1e-4


def test_point_mapping_two_way_exchange_is_equal_and_opposite():
    p = bub.BubbleParams(1.6, mapping="point")
    sim = OracleSim((12, 12, 16), 1.6, lat.ALL_WALLS, p)
    sim.set_bubbles([[1.3, 6.2, 5.0], [3.1, 9.0, 14.5]], [[0, 0, 0], [1e-4, 0, 0]], [2.0, 1.5])
    for _ in range(4):
        sim.step()
        assert np.allclose(sim.last_force.sum(axis=(1, 2, 3)), sim.psi.sum(axis=0),
                           rtol=1e-12, atol=1e-18)
