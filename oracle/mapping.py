"""Clipped fourth-order polynomial mapping (Sec. 3.2), FP64 (test infrastructure only).

Node j of the lattice sits at the centre (i + 1/2) of cell Omega_j = [i, i+1]
along each axis; the box is [0, nx] x [0, ny] x [0, nz].

Readings of the printed formulas:

* Eq. 18 prints the polynomial as (r)/n^5 - 2 (r)/n^3 + 1/n.  Only the form
  Z(r) = 15/16 [r^4/n^5 - 2 r^2/n^3 + 1/n] on |r| <= n meets the stated
  criteria (maximum at the bubble, zero at the window edge, unit integral), so
  that is the one used.
* n = 1.5 d_b is the half-width: the support is [-n, n].
* Eq. 19 integrates Z over the cell.  The integral is exact through the
  antiderivative G(s) = 15/16 [s^5/(5 n^5) - 2 s^3/(3 n^3) + s/n], held at
  +-1/2 beyond +-n.
* Near a wall part of the window lies outside the liquid.  The weights are
  renormalised so that they sum to one over the nodes inside the box
  ("clipped"), both for interpolation (Eq. 20) and spreading (Eq. 21).
  On a periodic axis the window wraps around instead (needs 2n + 2 <= L).
* Point sampling (``point=True``) is the variant that takes Z at the node
  itself instead of its cell integral: the factor of node i along an axis is
  Z(i + 1/2 - x_b) Delta x, with the same renormalisation over the in-box
  nodes (the node values of Z sum to one only up to the midpoint rule's
  error, so the renormalisation is needed even far from walls).
"""
import numpy as np


def kernel_z(r, n):
    """Eq. 18 (read with r^4 and r^2): the mapping function Z(r) for half-width n."""
    r = np.asarray(r, dtype=np.float64)
    z = 15.0 / 16.0 * (r ** 4 / n ** 5 - 2.0 * r ** 2 / n ** 3 + 1.0 / n)
    return np.where(np.abs(r) <= n, z, 0.0)


def kernel_g(s, n):
    """Antiderivative of Z with G(0) = 0, constant (+-1/2) outside [-n, n]."""
    s = np.clip(np.asarray(s, dtype=np.float64), -n, n)
    return 15.0 / 16.0 * (s ** 5 / (5.0 * n ** 5) - 2.0 * s ** 3 / (3.0 * n ** 3) + s / n)


def cell_factor(cells, xb, n, point=False):
    """One axis factor of Eq. 19 for the cells [i, i+1] of ``cells``: the cell
    integral of Z(x - xb), or with ``point`` the node sample Z(i + 1/2 - xb)
    times the cell width."""
    cells = np.asarray(cells, dtype=np.float64)
    if point:
        return kernel_z(cells + 0.5 - xb, n)
    return kernel_g(cells + 1.0 - xb, n) - kernel_g(cells - xb, n)


def axis_weights(xb, n, length, periodic, point=False):
    """Per-axis factors of Eq. 19 for every cell i = 0..length-1.

    Returns the raw integrals int_{i}^{i+1} Z(x - xb) dx (or the point
    samples), with periodic images summed on a periodic axis.
    """
    i = np.arange(length, dtype=np.float64)
    w = cell_factor(i, xb, n, point)
    if periodic:
        for shift in (-length, length):
            w = w + cell_factor(i + shift, xb, n, point)
    return w


def node_weights(xb, n, dims, walls, point=False):
    """Eq. 19: tensor-product weights int_{Omega_j} Z dOmega for all nodes, renormalised.

    xb: (x, y, z) bubble centre; dims: (nx, ny, nz); returns [nz, ny, nx] that
    sums to one (the clipped reading).
    """
    per = [not bool(walls & (1 << (2 * d))) for d in range(3)]
    wx = axis_weights(xb[0], n, dims[0], per[0], point)
    wy = axis_weights(xb[1], n, dims[1], per[1], point)
    wz = axis_weights(xb[2], n, dims[2], per[2], point)
    w3 = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    return w3 / w3.sum()


def axis_window(xb, n, length, periodic, point=False):
    """Cells of one axis whose interval overlaps the window (xb - n, xb + n) and
    their cell integrals of Z (Eq. 19, one factor; node samples with
    ``point``).  On a periodic axis the cells are wrapped into [0, length); on
    a wall axis cells outside the box are dropped (the weights of the in-box
    cells are the only non-zero ones)."""
    lo = int(np.floor(xb - n))
    hi = int(np.ceil(xb + n)) - 1
    cells = np.arange(lo, hi + 1)
    w = cell_factor(cells, xb, n, point)
    if periodic:
        cells = np.mod(cells, length)
    else:
        keep = (cells >= 0) & (cells < length)
        cells, w = cells[keep], w[keep]
    return cells, w


def window_weights(xb, n, dims, walls, point=False):
    """Eq. 19 weights on the window's nodes, renormalised to sum to one.

    Returns (cz, cy, cx, w3) with w3[k, j, i] the weight of node (cx[i], cy[j], cz[k]).
    Equal to ``node_weights`` restricted to its non-zero entries.
    """
    per = [not bool(walls & (1 << (2 * d))) for d in range(3)]
    cx, wx = axis_window(xb[0], n, dims[0], per[0], point)
    cy, wy = axis_window(xb[1], n, dims[1], per[1], point)
    cz, wz = axis_window(xb[2], n, dims[2], per[2], point)
    w3 = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    return cz, cy, cx, w3 / w3.sum()


def interpolate(sigma, xb, n, walls, point=False):
    """Eq. 20: Psi = sum_j sigma(j) int_{Omega_j} Z.  sigma: [C, nz, ny, nx] -> [C]."""
    nz, ny, nx = sigma.shape[1:]
    cz, cy, cx, w = window_weights(xb, n, (nx, ny, nz), walls, point)
    sub = sigma[:, cz[:, None, None], cy[None, :, None], cx[None, None, :]]
    return np.array([(sub[c] * w).sum() for c in range(sigma.shape[0])])


def spread(psi_list, xb_list, n_list, dims, walls, point=False):
    """Eq. 21: Phi(j) = sum_b psi_b int_{Omega_j} Z, summed over bubbles -> [3, nz, ny, nx]."""
    nx, ny, nz = dims
    phi = np.zeros((3, nz, ny, nx), dtype=np.float64)
    for psi, xb, n in zip(psi_list, xb_list, n_list):
        cz, cy, cx, w = window_weights(xb, n, dims, walls, point)
        idx = (cz[:, None, None], cy[None, :, None], cx[None, None, :])
        for d in range(3):
            phi[d][idx] += psi[d] * w
    return phi
