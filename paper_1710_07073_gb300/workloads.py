"""Seeded synthetic workloads shaped like the paper's bubble-column runs.

This module only draws inputs (lattice sizes, bubble positions, diameters,
initial velocity perturbations).  It holds none of the method's arithmetic and
is shared by the tests, the benchmark and the oracle runs so that both sides
see identical inputs.

Workloads (lattice units, dx = dt_l = 1):

* ``single_bubble``: one bubble of diameter 2 released at rest at
  (nx/2, ny/2, nz/8) in a wall-bounded column (the 4 mm validation case of
  Sec. 4.1 scaled to lattice units).  32x32x64 is the small case,
  256x256x512 the large single column.
* ``swarm``: N bubbles with lognormal diameters of mean 1.5 and standard
  deviation 0.3, centres uniform in the bottom 20 % of the column, released at
  rest (a dispersed swarm).
* ``batch_columns``: independent columns with sizes drawn from the grid
  independence study's family of aspect ratios and omega uniform in
  [1.0, 1.9] (Sec. 4.2-4.3).
"""
import math

import numpy as np

ALL_WALLS = 0x3F

SINGLE_SMALL = (32, 32, 64)
SINGLE_LARGE = (256, 256, 512)
SWARM_FULL = (384, 384, 768)
SWARM_CROP = (64, 64, 128)
COLUMN_SIZES = ((32, 32, 64), (48, 48, 96), (64, 64, 128), (96, 96, 192), (128, 128, 256))


def single_bubble(dims, diameter=2.0):
    """One bubble at rest at (nx/2, ny/2, nz/8): (pos[1,3], vel[1,3], diam[1])."""
    nx, ny, nz = dims
    pos = np.array([[nx / 2.0, ny / 2.0, nz / 8.0]], dtype=np.float64)
    return pos, np.zeros((1, 3)), np.array([float(diameter)])


def lognormal_diameters(rng, count, mean=1.5, std=0.3):
    """Diameters whose own mean and standard deviation are ``mean`` and ``std``."""
    s2 = math.log(1.0 + (std / mean) ** 2)
    mu = math.log(mean) - 0.5 * s2
    return rng.lognormal(mu, math.sqrt(s2), size=count)


def swarm(dims, count, seed=1234, bottom_fraction=0.2, max_diameter=4.0):
    """``count`` bubbles, lognormal diameters (clipped to ``max_diameter``),
    centres uniform in the bottom ``bottom_fraction`` of the column, inside
    the walls by one radius."""
    rng = np.random.default_rng(seed)
    d = np.minimum(lognormal_diameters(rng, count), max_diameter)
    r = 0.5 * d
    nx, ny, nz = dims
    pos = np.empty((count, 3))
    pos[:, 0] = r + rng.random(count) * (nx - 2 * r)
    pos[:, 1] = r + rng.random(count) * (ny - 2 * r)
    pos[:, 2] = r + rng.random(count) * (bottom_fraction * nz - 2 * r)
    return pos, np.zeros((count, 3)), d


def swarm_count_for_crop(full_dims, full_count, crop_dims):
    """Bubble count scaled by volume from the full swarm to a crop."""
    vf = full_dims[0] * full_dims[1] * full_dims[2]
    vc = crop_dims[0] * crop_dims[1] * crop_dims[2]
    return max(1, int(round(full_count * vc / vf)))


def batch_columns(count, seed=1234):
    """Independent columns: list of (dims, omega, pos[1,3], vel[1,3], diam[1])."""
    rng = np.random.default_rng(seed)
    cols = []
    for _ in range(count):
        dims = COLUMN_SIZES[int(rng.integers(len(COLUMN_SIZES)))]
        omega = float(rng.uniform(1.0, 1.9))
        diam = float(rng.uniform(1.5, 3.0))
        pos = np.array([[dims[0] / 2.0, dims[1] / 2.0, dims[2] / 8.0]])
        cols.append((dims, omega, pos, np.zeros((1, 3)), np.array([diam])))
    return cols


def random_fields(dims, seed=7, amp=1e-3, rho_amp=1e-3):
    """Smooth-ish random (rho, u) fields: rho [nz,ny,nx], u [3,nz,ny,nx]."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    rho = 1.0 + rho_amp * rng.standard_normal((nz, ny, nx))
    u = amp * rng.standard_normal((3, nz, ny, nx))
    return rho, u


def gaussian_velocity_perturbation(dims, seed=4, amp=1e-4):
    """Seeded Gaussian perturbation of the initial velocity field, u [3,nz,ny,nx]."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    return amp * rng.standard_normal((3, nz, ny, nx))
