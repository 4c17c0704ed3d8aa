"""Pins for the oracle's liquid solver (D3Q19 BGK with Guo forcing, Eq. 5-16).

Each check is fixed by mathematics the paper's equations imply, not by the
oracle itself: lattice isotropy of the velocity set, moments of the
equilibrium, the fixed point of collision, exact mass/momentum budgets,
shear-wave decay at the viscosity of Eq. 9, and plane Poiseuille flow.
"""
import numpy as np
import pytest

from oracle import lattice as lat


def _delta(a, b):
    return 1.0 if a == b else 0.0


def test_velocity_set_isotropy():
    # Eq. 7-8: zeroth..fourth lattice moments of a D3Q19 set with c_s^2 = 1/3.
    c = lat.C.astype(np.float64)
    w = lat.W
    assert len(set(map(tuple, lat.C))) == 19
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    for a in range(3):
        assert abs((w * c[:, a]).sum()) < 1e-16
        for b in range(3):
            assert np.isclose((w * c[:, a] * c[:, b]).sum(), _delta(a, b) / 3.0, atol=1e-15)
            for g in range(3):
                assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-16
                for e in range(3):
                    m4 = (w * c[:, a] * c[:, b] * c[:, g] * c[:, e]).sum()
                    iso = (_delta(a, b) * _delta(g, e) + _delta(a, g) * _delta(b, e)
                           + _delta(a, e) * _delta(b, g)) / 9.0
                    assert np.isclose(m4, iso, atol=1e-15)
    for j in range(19):
        assert (lat.C[lat.OPP[j]] == -lat.C[j]).all()


def test_equilibrium_moments():
    # Eq. 10: sum f^eq = rho, sum c f^eq = rho u; second moment rho/3 I + rho u u.
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.1 * rng.standard_normal((3, 4, 5))
    u = 0.05 * rng.standard_normal((3, 3, 4, 5))
    feq = lat.equilibrium(rho, u)
    assert np.allclose(lat.density(feq), rho, rtol=0, atol=1e-14)
    assert np.allclose(lat.momentum(feq), rho * u, rtol=0, atol=1e-14)
    c = lat.C.astype(np.float64)
    for a in range(3):
        for b in range(3):
            pi = np.tensordot(c[:, a] * c[:, b], feq, axes=(0, 0))
            assert np.allclose(pi, rho * _delta(a, b) / 3.0 + rho * u[a] * u[b], atol=1e-14)


def test_equilibrium_is_fixed_point_of_collision():
    # Eq. 14 with F = 0: f = f^eq(rho, u) is left unchanged for any omega.
    rng = np.random.default_rng(2)
    rho = 1.0 + 0.05 * rng.standard_normal((4, 4, 4))
    u = 0.03 * rng.standard_normal((3, 4, 4, 4))
    feq = lat.equilibrium(rho, u)
    for omega in (0.7, 1.0, 1.6, 1.95):
        assert np.allclose(lat.collide(feq, omega), feq, rtol=0, atol=1e-15)


def test_guo_term_moments():
    # Eq. 12: sum_j F_j = 0 and sum_j c_j F_j = (1 - omega/2) F.
    rng = np.random.default_rng(3)
    u = 0.05 * rng.standard_normal((3, 2, 3, 4))
    force = 1e-3 * rng.standard_normal((3, 2, 3, 4))
    for omega in (0.8, 1.6):
        fj = lat.guo_term(u, force, omega)
        assert np.allclose(fj.sum(axis=0), 0.0, atol=1e-18)
        assert np.allclose(lat.momentum(fj), (1.0 - omega / 2.0) * force, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("walls", [0, lat.ALL_WALLS, lat.WALL_ZM | lat.WALL_ZP])
def test_mass_conserved_momentum_budget(walls):
    # Collision conserves mass; with forcing the momentum grows by exactly
    # F dt per step (Eq. 13-15).  Streaming conserves mass; on a periodic box
    # it also conserves momentum.
    rng = np.random.default_rng(4)
    nx, ny, nz = 5, 4, 6
    f = lat.equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    f = f * (1.0 + 0.01 * rng.standard_normal(f.shape))
    force = 1e-4 * rng.standard_normal((3, nz, ny, nx))
    m0 = lat.density(f).sum()
    p0 = lat.momentum(f).sum(axis=(1, 2, 3))
    fc = lat.collide(f, 1.3, force)
    assert np.isclose(lat.density(fc).sum(), m0, rtol=0, atol=1e-12)
    p1 = lat.momentum(fc).sum(axis=(1, 2, 3))
    assert np.allclose(p1 - p0, force.sum(axis=(1, 2, 3)), rtol=0, atol=1e-13)
    fs = lat.stream(fc, walls)
    assert np.isclose(lat.density(fs).sum(), m0, rtol=0, atol=1e-12)
    if walls == 0:
        assert np.allclose(lat.momentum(fs).sum(axis=(1, 2, 3)), p1, rtol=0, atol=1e-13)


def test_stream_moves_single_population():
    # Eq. 16: a population at x with velocity c_j arrives at x + c_j (periodic box).
    nx, ny, nz = 4, 4, 8
    for j in range(19):
        f = np.zeros((19, nz, ny, nx))
        f[j, 3, 2, 1] = 1.0
        out = lat.stream(f, 0)
        x, y, z = 1 + lat.C[j, 0], 2 + lat.C[j, 1], 3 + lat.C[j, 2]
        assert out[j, z % nz, y % ny, x % nx] == 1.0
        assert out.sum() == 1.0


def test_bounce_back_returns_to_same_node():
    # Sec. 3.3 half-way bounce-back: a population leaving through a wall comes
    # back to the same node as the opposite direction.
    nx, ny, nz = 4, 4, 8
    for j in range(18):
        f = np.zeros((19, nz, ny, nx))
        # Node at the low corner: every direction with a negative component
        # crosses a wall there.
        f[j, 0, 0, 0] = 1.0
        out = lat.stream(f, lat.ALL_WALLS)
        if (lat.C[j] < 0).any():
            assert out[lat.OPP[j], 0, 0, 0] == 1.0
        else:
            x, y, z = lat.C[j]
            assert out[j, z, y, x] == 1.0
        assert out.sum() == 1.0


@pytest.mark.parametrize("walls", [0, lat.ALL_WALLS, lat.WALL_XM | lat.WALL_XP])
def test_stream_reversal_is_identity(walls):
    # Streaming with half-way bounce-back is time-reversible: stream, reverse
    # every velocity, stream again and reverse back recovers the field exactly.
    rng = np.random.default_rng(5)
    f = rng.random((19, 6, 5, 4))
    g = lat.stream(f, walls)[lat.OPP]
    back = lat.stream(g, walls)[lat.OPP]
    assert np.array_equal(back, f)


@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_shear_wave_decay_matches_eq9_viscosity(omega):
    # A periodic shear wave u_x = A sin(k z) decays as exp(-nu k^2 t) with
    # nu = (1/omega - 1/2)/3 (Eq. 9).
    nz = 32
    k = 2.0 * np.pi / nz
    z = np.arange(nz) + 0.5
    amp = 1e-4
    u = np.zeros((3, nz, 1, 1))
    u[0, :, 0, 0] = amp * np.sin(k * z)
    f = lat.equilibrium(np.ones((nz, 1, 1)), u)
    nsteps = 300
    amps = []
    for t in range(nsteps + 1):
        ux = lat.velocity(f)[0, :, 0, 0]
        amps.append(2.0 / nz * (ux * np.sin(k * z)).sum())
        f = lat.lb_step(f, omega, 0)
    # Fit the decay rate after the initial non-equilibrium transient.
    t = np.arange(50, nsteps + 1)
    rate = -np.polyfit(t, np.log(np.array(amps)[50:]), 1)[0]
    nu = (1.0 / omega - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 5e-3


def _poiseuille(omega, height, nsteps):
    f = lat.equilibrium(np.ones((height, 1, 1)), np.zeros((3, height, 1, 1)))
    force = np.zeros((3, height, 1, 1))
    gx = 1e-6
    force[0] = gx
    walls = lat.WALL_ZM | lat.WALL_ZP
    for _ in range(nsteps):
        f = lat.lb_step(f, omega, walls, force)
    u = lat.velocity(f, force)[0, :, 0, 0]
    z = np.arange(height) + 0.5
    exact = gx / (2.0 * lat.viscosity(omega)) * z * (height - z)
    return np.abs(u - exact).max() / exact.max()


@pytest.mark.slow
def test_poiseuille_exact_at_magic_relaxation():
    # Body-force driven plane Poiseuille between half-way bounce-back walls at
    # z = 0 and z = H: u = F z (H - z) / (2 rho nu).  BGK with half-way
    # bounce-back puts the wall exactly half-way when (tau - 1/2)^2 = 3/16.
    omega_magic = 1.0 / (0.5 + np.sqrt(3.0) / 4.0)
    assert _poiseuille(omega_magic, 12, 6000) < 1e-9


def test_poiseuille_second_order_in_height():
    # Away from the magic value the wall slip is O(1/H^2): halving the error
    # scale when H doubles by about 4.
    e8 = _poiseuille(1.0, 8, 1500)
    e16 = _poiseuille(1.0, 16, 3000)
    assert e16 < 5e-3
    assert 3.5 < e8 / e16 < 4.5


# ---- free-slip top (Sec. 3.3) --------------------------------------------------

def _mirror_z(f):
    """Populations of the column reflected in z: f'_j(z) = f_{mirz(j)}(nz - 1 - z)."""
    return f[lat.MIRZ][:, ::-1]


@pytest.mark.parametrize("side_walls", [lat.WALL_XM | lat.WALL_XP, 0])
def test_free_slip_top_is_a_mirror_plane(side_walls):
    # A specular (free-slip) plane half-way above the top layer is a plane of
    # symmetry: a column of height H with a free-slip top evolves exactly like
    # the lower half of a column of height 2H with no-slip walls at both ends,
    # started from the mirror image of itself (populations with c_z reversed,
    # the force with F_z reversed).  This fixes the reflected direction, the
    # tangential shift, and the height of the plane.
    rng = np.random.default_rng(11)
    nx, ny, H = 6, 5, 7
    rho = 1.0 + 1e-3 * rng.standard_normal((H, ny, nx))
    u = 1e-2 * rng.standard_normal((3, H, ny, nx))
    f = lat.equilibrium(rho, u) * (1.0 + 1e-3 * rng.standard_normal((lat.Q, H, ny, nx)))
    force = 1e-4 * rng.standard_normal((3, H, ny, nx))
    full = np.concatenate([f, _mirror_z(f)], axis=1)
    fmir = force[:, ::-1].copy()
    fmir[2] *= -1.0
    force_full = np.concatenate([force, fmir], axis=1)
    w_half = side_walls | lat.WALL_ZM | lat.WALL_ZP | lat.TOP_FREE_SLIP
    w_full = side_walls | lat.WALL_ZM | lat.WALL_ZP
    for _ in range(4):
        f = lat.lb_step(f, 1.3, w_half, force)
        full = lat.lb_step(full, 1.3, w_full, force_full)
        assert np.abs(full[:, :H] - f).max() < 1e-15
        assert np.abs(full[:, H:] - _mirror_z(f)).max() < 1e-15


def test_free_slip_top_reflects_a_single_population():
    # A population leaving the top layer through the free-slip plane comes
    # back into the top layer with c_z reversed, one tangential step along
    # (c_x, c_y) (periodic sides), and nothing is lost.
    nx, ny, nz = 5, 4, 6
    walls = lat.WALL_ZM | lat.WALL_ZP | lat.TOP_FREE_SLIP
    for j in range(lat.Q):
        f = np.zeros((lat.Q, nz, ny, nx))
        f[j, nz - 1, 2, 1] = 1.0
        out = lat.stream(f, walls)
        cx, cy, cz = lat.C[j]
        if cz == 1:
            assert out[lat.MIRZ[j], nz - 1, (2 + cy) % ny, (1 + cx) % nx] == 1.0
        else:
            assert out[j, nz - 1 + cz, (2 + cy) % ny, (1 + cx) % nx] == 1.0
        assert out.sum() == 1.0
    # Also through an edge where the top meets a no-slip side wall: the
    # link crosses the wall, so it bounces back to the same node.
    walls_x = walls | lat.WALL_XM | lat.WALL_XP
    for j in range(lat.Q):
        if lat.C[j, 2] != 1 or lat.C[j, 0] != 1:
            continue
        f = np.zeros((lat.Q, nz, ny, nx))
        f[j, nz - 1, 2, nx - 1] = 1.0
        out = lat.stream(f, walls_x)
        assert out[lat.OPP[j], nz - 1, 2, nx - 1] == 1.0


def test_free_slip_top_half_poiseuille_exact():
    # Body-force driven flow between a no-slip wall at z = 0 and a free-slip
    # plane at z = H: u = F z (2H - z) / (2 rho nu), zero shear at z = H (half
    # of the Poiseuille profile of height 2H).  Exact at (tau - 1/2)^2 = 3/16,
    # where half-way bounce-back puts the wall at z = 0.
    omega = 1.0 / (0.5 + np.sqrt(3.0) / 4.0)
    H = 6
    f = lat.equilibrium(np.ones((H, 1, 1)), np.zeros((3, H, 1, 1)))
    force = np.zeros((3, H, 1, 1))
    gx = 1e-6
    force[0] = gx
    walls = lat.WALL_ZM | lat.WALL_ZP | lat.TOP_FREE_SLIP
    for _ in range(3000):
        f = lat.lb_step(f, omega, walls, force)
    u = lat.velocity(f, force)[0, :, 0, 0]
    z = np.arange(H) + 0.5
    exact = gx / (2.0 * lat.viscosity(omega)) * z * (2.0 * H - z)
    assert np.abs(u - exact).max() / exact.max() < 1e-9


# ---- vorticity at the nodes (lift) ----------------------------------------------

def test_vorticity_exact_for_quadratic_fields():
    # Central differences are exact for polynomials of degree two: away from
    # the faces the node curl equals the analytic curl of
    # u = (a y^2 + b z, c x z, e x y + h x^2).
    nx, ny, nz = 7, 8, 9
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    a, b, c, e, h = 0.3, -0.7, 1.1, 0.4, -0.2
    u = np.stack([a * yy ** 2 + b * zz, c * xx * zz, e * xx * yy + h * xx ** 2])
    w = lat.vorticity(u, lat.ALL_WALLS)
    exact = np.stack([e * xx - c * xx,            # d(u_z)/dy - d(u_y)/dz
                      b - (e * yy + 2 * h * xx),  # d(u_x)/dz - d(u_z)/dx
                      c * zz - 2 * a * yy])       # d(u_y)/dx - d(u_x)/dy
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(w[inner] - exact[inner]).max() < 1e-12


def test_vorticity_ghost_nodes_at_faces():
    # A single u_x = 1 on the bottom layer: the no-slip ghost below is -1, so
    # d(u_x)/dz there is (0 - (-1))/2 = 1/2; one layer up it is (0 - 1)/2.
    # Under a free-slip top the tangential ghost is +u: a u_x = 1 on the top
    # layer gives d(u_x)/dz = (1 - 0)/2 there.  Periodic axes wrap.
    nx, ny, nz = 4, 5, 6
    u = np.zeros((3, nz, ny, nx))
    u[0, 0, 2, 1] = 1.0
    w = lat.vorticity(u, lat.ALL_WALLS)
    assert w[1, 0, 2, 1] == 0.5 and w[1, 1, 2, 1] == -0.5
    u = np.zeros((3, nz, ny, nx))
    u[0, nz - 1, 2, 1] = 1.0
    w = lat.vorticity(u, lat.ALL_WALLS | lat.TOP_FREE_SLIP)
    assert w[1, nz - 1, 2, 1] == 0.5 and w[1, nz - 2, 2, 1] == 0.5
    w = lat.vorticity(u, lat.ALL_WALLS)
    assert w[1, nz - 1, 2, 1] == -0.5
    w = lat.vorticity(u, lat.WALL_XM | lat.WALL_XP | lat.WALL_YM | lat.WALL_YP)
    assert w[1, 0, 2, 1] == -0.5 and w[1, nz - 2, 2, 1] == 0.5


def test_vorticity_of_a_gradient_field_vanishes():
    # Central differences along different axes commute, so the node curl of
    # a discrete gradient field vanishes on a periodic box.
    rng = np.random.default_rng(9)
    phi = rng.standard_normal((6, 5, 7))
    grad = np.stack([0.5 * (np.roll(phi, -1, 2) - np.roll(phi, 1, 2)),
                     0.5 * (np.roll(phi, -1, 1) - np.roll(phi, 1, 1)),
                     0.5 * (np.roll(phi, -1, 0) - np.roll(phi, 1, 0))])
    assert np.abs(lat.vorticity(grad, 0)).max() < 1e-14
