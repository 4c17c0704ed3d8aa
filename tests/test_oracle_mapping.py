"""Pins for the oracle's coupling maps (Sec. 3.2, Eq. 18-21) and binning (Algorithm 1 step 2)."""
import numpy as np
import pytest

from oracle import binning, lattice as lat, mapping


@pytest.mark.parametrize("n", [0.75, 1.5, 3.0, 4.5])
def test_mapping_function_criteria(n):
    # The four criteria listed before Eq. 18: smooth (continuous first
    # derivative, zero at the window edge), maximum at the bubble, zero at the
    # boundary of a finite window, unit integral.
    nodes, wts = np.polynomial.legendre.leggauss(8)
    integral = (mapping.kernel_z(n * nodes, n) * wts).sum() * n
    assert abs(integral - 1.0) < 1e-14
    assert mapping.kernel_z(n, n) == pytest.approx(0.0, abs=1e-15)
    assert mapping.kernel_z(-n, n) == pytest.approx(0.0, abs=1e-15)
    assert mapping.kernel_z(n * 1.0001, n) == 0.0
    h = 1e-6 * n
    for edge in (-n, n):
        inside = edge - np.sign(edge) * h
        slope = (mapping.kernel_z(edge, n) - mapping.kernel_z(inside, n)) / h
        assert abs(slope) < 1e-5 / n ** 2
    r = np.linspace(-n, n, 2001)
    assert np.argmax(mapping.kernel_z(r, n)) == 1000
    assert mapping.kernel_z(0.0, n) == pytest.approx(15.0 / (16.0 * n))


def test_cell_integral_matches_quadrature():
    # Eq. 19 one factor: G(b) - G(a) equals Gauss-Legendre quadrature of Z over
    # [a, b] clipped to the window (a quartic is integrated exactly with 3+ points).
    rng = np.random.default_rng(7)
    nodes, wts = np.polynomial.legendre.leggauss(5)
    for _ in range(200):
        n = rng.uniform(0.5, 5.0)
        a = rng.uniform(-1.5 * n, 1.2 * n)
        b = a + rng.uniform(0.0, 2.0)
        lo, hi = max(a, -n), min(b, n)
        quad = 0.0
        if hi > lo:
            xs = 0.5 * (hi - lo) * nodes + 0.5 * (hi + lo)
            quad = 0.5 * (hi - lo) * (mapping.kernel_z(xs, n) * wts).sum()
        exact = mapping.kernel_g(b, n) - mapping.kernel_g(a, n)
        assert abs(exact - quad) < 1e-14


@pytest.mark.parametrize("walls", [0, lat.ALL_WALLS])
def test_weights_partition_of_unity(walls):
    # Sum over nodes of int_{Omega_j} Z is one, also for a window cut by a wall
    # (renormalised) or wrapping a periodic face.
    rng = np.random.default_rng(8)
    dims = (12, 10, 14)
    for _ in range(20):
        d = rng.uniform(0.8, 2.5)
        n = 1.5 * d
        xb = [rng.uniform(0.0, L) for L in dims]
        w = mapping.node_weights(xb, n, dims, walls)
        assert abs(w.sum() - 1.0) < 1e-13
        assert (w >= 0.0).all()


@pytest.mark.parametrize("walls", [0, lat.ALL_WALLS, lat.WALL_ZM | lat.WALL_ZP])
def test_window_weights_equal_full_grid_weights(walls):
    # The window restriction drops only zero weights (Eq. 18 vanishes outside
    # [-n, n]); periodic windows must not overlap themselves (2n + 2 <= L).
    rng = np.random.default_rng(10)
    dims = (14, 12, 16)
    for _ in range(20):
        n = 1.5 * rng.uniform(0.7, 2.6)
        xb = [rng.uniform(0.0, L) for L in dims]
        full = mapping.node_weights(xb, n, dims, walls)
        cz, cy, cx, w = mapping.window_weights(xb, n, dims, walls)
        assert len(set(cx)) == len(cx) and len(set(cy)) == len(cy) and len(set(cz)) == len(cz)
        sub = full[cz[:, None, None], cy[None, :, None], cx[None, None, :]]
        assert np.allclose(sub, w, rtol=1e-12, atol=1e-15)
        assert abs(full.sum() - w.sum()) < 1e-13


def test_unclipped_weights_need_no_renormalisation():
    # Away from walls the raw tensor-product cell integrals already sum to one.
    dims = (16, 16, 16)
    per = [False, False, False]
    xb = (7.3, 8.1, 8.9)
    n = 3.0
    w = [mapping.axis_weights(xb[a], n, dims[a], per[a]) for a in range(3)]
    assert abs(w[0].sum() * w[1].sum() * w[2].sum() - 1.0) < 1e-14


def test_spreading_equal_and_opposite():
    # Eq. 21: the spread field carries exactly the bubbles' total reaction.
    rng = np.random.default_rng(9)
    dims = (10, 9, 12)
    psis = [1e-5 * rng.standard_normal(3) for _ in range(4)]
    xbs = [[rng.uniform(0.5, L - 0.5) for L in dims] for _ in range(4)]
    ns = [1.5 * rng.uniform(1.0, 2.0) for _ in range(4)]
    phi = mapping.spread(psis, xbs, ns, dims, lat.ALL_WALLS)
    assert np.allclose(phi.sum(axis=(1, 2, 3)), np.sum(psis, axis=0), rtol=1e-13, atol=0)


def test_interpolation_of_constant_field():
    # Eq. 20 reproduces a uniform field exactly (follows from the partition of unity).
    dims = (8, 8, 10)
    sigma = np.empty((3,) + dims[::-1])
    sigma[0], sigma[1], sigma[2] = 1.5e-4, -2e-5, 3e-4
    out = mapping.interpolate(sigma, (0.9, 4.4, 9.6), 2.25, lat.ALL_WALLS)
    assert np.allclose(out, [1.5e-4, -2e-5, 3e-4], rtol=1e-13, atol=0)


def test_window_support_by_hand():
    # Bubble at x = 16.3 with d = 2 (n = 3): the window (13.3, 19.3) overlaps
    # cells 13..19; at x = 1.0 it is cut by the wall to cells 0..3; on a
    # periodic axis of length 8 it wraps to 6, 7, 0, 1, 2, 3.
    assert binning.support_cells(16.3, 3.0, 64, False) == list(range(13, 20))
    assert binning.support_cells(1.0, 3.0, 64, False) == [0, 1, 2, 3]
    assert binning.support_cells(1.0, 3.0, 8, True) == [6, 7, 0, 1, 2, 3]
    # Integer window ends: (14, 20) overlaps cells 14..19 exactly.
    assert binning.support_cells(17.0, 3.0, 64, False) == list(range(14, 20))
    assert binning.containing_cell((16.3, 16.7, 8.2), (32, 32, 64)) == (8 * 32 + 16) * 32 + 16


def test_tile_lists_by_hand():
    # 64 x 8 x 8 box, tiles 32 x 4 x 4.  Bubble 0 at (31.5, 1.5, 6.5), n = 1.5:
    # x cells 30..32 -> x tiles 0, 1; y cells 0..2 -> tile 0; z cells 5..7 -> tile 1.
    # Bubble 1 (inactive) is ignored; bubble 2 at (5, 5, 1), n = 0.75: x 4..5,
    # y 4..5, z 0..1 -> tile (0, 1, 0).
    dims, tile = (64, 8, 8), (32, 4, 4)
    xs = [(31.5, 1.5, 6.5), (10.0, 2.0, 2.0), (5.0, 5.0, 1.0)]
    ns = [1.5, 1.5, 0.75]
    off, items = binning.tile_lists(xs, ns, [True, False, True], dims, lat.ALL_WALLS, tile)
    # tiles per axis (2, 2, 2): id = (tz * 2 + ty) * 2 + tx
    expect = {4: [0], 5: [0], 2: [2]}
    for t in range(8):
        assert items[off[t]:off[t + 1]] == expect.get(t, [])


def test_interpolation_hand_computed_two_cells():
    # Eq. 18-20 by hand: half-width n = 1/2 around x_b = 5.25 touches cells 4
    # ([4, 5], node 4.5) and 5 ([5, 6], node 5.5).  With s = r/n the cell
    # integral of Z is 15/16 [s^5/5 - 2 s^3/3 + s] between the cell's ends:
    # cell 4 spans s in [-1, -1/2], giving 15/16 (-203/480 + 256/480) = 53/512,
    # and cell 5 the remaining 459/512.  A linear field sampled at the nodes
    # interpolates to 4.5 * 53/512 + 5.5 * 459/512 = 2763/512.
    cells, w = mapping.axis_window(5.25, 0.5, 12, False)
    assert list(cells) == [4, 5]
    assert w[0] == pytest.approx(53.0 / 512.0, abs=1e-15)
    assert w[1] == pytest.approx(459.0 / 512.0, abs=1e-15)
    dims = (12, 12, 12)
    x_nodes = np.arange(dims[0]) + 0.5
    sigma = np.broadcast_to(x_nodes[None, None, None, :], (1, 12, 12, 12)).copy()
    out = mapping.interpolate(sigma, (5.25, 6.0, 6.0), 0.5, lat.ALL_WALLS)
    assert out[0] == pytest.approx(2763.0 / 512.0, abs=1e-13)


@pytest.mark.parametrize("n,tol", [(1.5, 3e-3), (3.0, 2e-4)])
def test_interpolation_reproduces_linear_field(n, tol):
    # The weights are the cell integrals of a symmetric Z, so their first
    # moment over the node centres i + 1/2 lies within a small fraction of a
    # cell of x_b (the sawtooth floor(x) + 1/2 - x integrated against Z): a
    # linear field u = a x + b interpolates to a x_b + b.  Nodes placed half a
    # cell off (at i or i + 1) would miss by |a| / 2.
    rng = np.random.default_rng(3)
    dims = (32, 32, 32)
    c = np.arange(32) + 0.5
    a = np.array([0.3, -0.7, 1.1])
    b = 0.25
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")   # [z, y, x] node centres
    sigma = np.stack([a[0] * xx + b, a[1] * yy + b, a[2] * zz + b])
    for _ in range(60):
        xb = rng.uniform(n + 1.0, 31.0 - n, 3)
        out = mapping.interpolate(sigma, xb, n, lat.ALL_WALLS)
        assert np.all(np.abs(out - (a * xb + b)) <= tol * np.abs(a)), (xb, out)


# ---- point-sampled variant of Eq. 19 (node values of Z, renormalised) -------

def test_point_sampled_weights_node_centred_by_hand():
    # n = 3 with the centre on node 6 (x = 6.5): the node samples of
    # (1 - (r/n)^2)^2 at r = 0, +-1, +-2 are 1, 64/81, 25/81 (r = +-3 sits on
    # the window edge, Z = 0), so the renormalised factors are
    # (25, 64, 81, 64, 25) / 259 on nodes 4..8.
    cells, w = mapping.axis_window(6.5, 3.0, 16, False, point=True)
    keep = w > 0
    assert list(cells[keep]) == [4, 5, 6, 7, 8]
    np.testing.assert_allclose(w[keep] / w.sum(), np.array([25, 64, 81, 64, 25]) / 259.0,
                               rtol=1e-15, atol=0)
    cz, cy, cx, w3 = mapping.window_weights([6.5, 6.5, 6.5], 3.0, (16, 16, 16), lat.ALL_WALLS,
                                            point=True)
    ax = np.array([0, 25, 64, 81, 64, 25, 0]) / 259.0
    np.testing.assert_allclose(w3, ax[:, None, None] * ax[None, :, None] * ax[None, None, :],
                               rtol=1e-14, atol=1e-18)


def test_point_samples_sum_to_one_up_to_midpoint_error():
    # The node samples of Z are a midpoint rule for its unit integral; Z and Z'
    # vanish at +-n and Z'' jumps there by J = 15/(2 n^3), so by Poisson
    # summation the error is at most 2 J sum_{k != 0} |2 pi k|^-3 + O(n^-4)
    # = 2 J 2 zeta(3) / (2 pi)^3 + ... = 0.145 n^-3 + ...
    rng = np.random.default_rng(21)
    for _ in range(300):
        n = rng.uniform(1.0, 12.0)
        xb = 40.0 + rng.uniform(0.0, 1.0)
        raw = mapping.cell_factor(np.arange(0, 80), xb, n, point=True).sum()
        assert abs(raw - 1.0) < 0.16 / n ** 3


def test_point_and_cell_weights_converge_second_order():
    # The midpoint value of a cell differs from its mean by h^2 Z''/24: the
    # two maps agree to O(n^-2) relative to the O(1/n) weights.  A sample off
    # the node centre (x = i instead of i + 1/2) would differ at O(1/n).
    rng = np.random.default_rng(22)
    for n in (1.5, 3.0, 6.0, 12.0):
        worst = 0.0
        for _ in range(50):
            xb = 30.0 + rng.uniform(0.0, 1.0)
            cells = np.arange(0, 60)
            wp = mapping.cell_factor(cells, xb, n, point=True)
            wc = mapping.cell_factor(cells, xb, n, point=False)
            worst = max(worst, n * np.abs(wp / wp.sum() - wc).max())
        assert worst < 0.35 / n ** 2


@pytest.mark.parametrize("walls", [0, lat.ALL_WALLS])
def test_point_spreading_equal_and_opposite(walls):
    # Eq. 21 with point-sampled weights: after renormalisation the spread
    # force sums to psi also for windows cut by a wall or wrapping.
    rng = np.random.default_rng(23)
    dims = (12, 10, 14)
    psis = [rng.normal(size=3) for _ in range(4)]
    xs = [[rng.uniform(0.0, L) for L in dims] for _ in range(4)]
    ns = [1.5 * rng.uniform(0.6, 2.0) for _ in range(4)]
    phi = mapping.spread(psis, xs, ns, dims, walls, point=True)
    np.testing.assert_allclose(phi.sum(axis=(1, 2, 3)), np.sum(psis, axis=0), rtol=1e-12,
                               atol=1e-14)
    for xb, n in zip(xs, ns):
        w = mapping.node_weights(xb, n, dims, walls, point=True)
        assert abs(w.sum() - 1.0) < 1e-13 and (w >= 0.0).all()
        cz, cy, cx, ww = mapping.window_weights(xb, n, dims, walls, point=True)
        np.testing.assert_allclose(w[np.ix_(cz, cy, cx)], ww, rtol=1e-12, atol=1e-16)
