"""D3Q19 BGK liquid solver, FP64 (test infrastructure only; see package docstring).

Fields are numpy arrays indexed ``[q, z, y, x]`` for populations and
``[z, y, x]`` for scalars; vectors carry a leading component axis
``[3, z, y, x]`` ordered (x, y, z).  Lattice units: dx = dt_l = e = 1.

Direction numbering follows the paper's grouping (Eq. 7): the six axis
directions first, then the twelve edge diagonals, the rest velocity last.
"""
import numpy as np

# --- Eq. 7: discrete velocities c_j (e = 1).  j = 0..5 axis, 6..17 edges, 18 rest.
C = np.array(
    [
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
        (0, 0, 0),
    ],
    dtype=np.int64,
)
Q = 19

# --- Eq. 8: weights w_j.
W = np.array([1.0 / 18.0] * 6 + [1.0 / 36.0] * 12 + [1.0 / 3.0], dtype=np.float64)

# Opposite direction of each c_j (the direction with velocity -c_j).
OPP = np.array([int(np.flatnonzero((C == -C[j]).all(axis=1))[0]) for j in range(Q)])

# Wall bit for each face, in the order (-x, +x, -y, +y, -z, +z).
WALL_XM, WALL_XP, WALL_YM, WALL_YP, WALL_ZM, WALL_ZP = (1 << k for k in range(6))
ALL_WALLS = 0x3F
# With the +z face bounded (WALL_ZP), this bit makes it free-slip instead of
# no-slip (Sec. 3.3: free-slip top).
TOP_FREE_SLIP = 0x40

# The direction with c_z reversed (same tangential components) of each c_j.
MIRZ = np.array([int(np.flatnonzero((C == C[j] * np.array([1, 1, -1])).all(axis=1))[0])
                 for j in range(Q)])


def viscosity(omega):
    """Eq. 9 with dx = dt_l = 1: nu = (2 tau - 1)/6, tau = 1/omega."""
    tau = 1.0 / omega
    return (2.0 * tau - 1.0) / 6.0


def equilibrium(rho, u):
    """Eq. 6 (e = 1): f_j^eq = w_j rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u].

    rho: [...]; u: [3, ...]  ->  [Q, ...].
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    usq = (u * u).sum(axis=0)
    feq = np.empty((Q,) + rho.shape, dtype=np.float64)
    for j in range(Q):
        cu = C[j, 0] * u[0] + C[j, 1] * u[1] + C[j, 2] * u[2]
        feq[j] = W[j] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
    return feq


def density(f):
    """Eq. 10: rho = sum_j f_j."""
    return f.sum(axis=0)


def momentum(f):
    """Eq. 10: rho u = sum_j c_j f_j  -> [3, ...]."""
    m = np.zeros((3,) + f.shape[1:], dtype=np.float64)
    for j in range(Q):
        for d in range(3):
            if C[j, d] != 0:
                m[d] += C[j, d] * f[j]
    return m


def velocity(f, force=None):
    """Macroscopic velocity.

    With ``force=None`` this is the bare moment of Eq. 10, u = sum c f / rho
    (the quantity Algorithm 1 step 3 interpolates to the bubble).  With a force
    field it is the first-forcing velocity of Eq. 13,
    u = (sum c f + F dt_l / 2) / rho.  The sum in Eq. 13 is printed over
    j = 1..9, a D2Q9 leftover; it runs over all 19 directions here.
    """
    m = momentum(f)
    if force is not None:
        m = m + 0.5 * force
    return m / density(f)


def guo_term(u, force, omega):
    """Eq. 12: F_j = (1 - 1/(2 tau)) w_j [3 (c_j - u) + 9 (c_j . u) c_j] . F."""
    pref = 1.0 - 0.5 * omega
    out = np.empty((Q,) + u.shape[1:], dtype=np.float64)
    for j in range(Q):
        cu = C[j, 0] * u[0] + C[j, 1] * u[1] + C[j, 2] * u[2]
        acc = np.zeros(u.shape[1:], dtype=np.float64)
        for d in range(3):
            acc += (3.0 * (C[j, d] - u[d]) + 9.0 * cu * C[j, d]) * force[d]
        out[j] = pref * W[j] * acc
    return out


def collide(f, omega, force=None):
    """One local forced BGK update, Eq. 13 -> 14 -> 15 (dt_l = 1).

    First forcing (Eq. 13) gives rho and the velocity u; the collision (Eq. 14)
    relaxes towards f^eq(rho, u) of Eq. 6 with rate 1/tau = omega; the second
    forcing (Eq. 15) adds the Guo term of Eq. 12 built from the same u.
    Returns the post-collision populations f''.
    """
    rho = density(f)
    u = velocity(f, force)
    feq = equilibrium(rho, u)
    fpost = f - omega * (f - feq)
    if force is not None:
        fpost = fpost + guo_term(u, force, omega)
    return fpost


def stream(fpost, walls):
    """Eq. 16, f_j(x + c_j, t + 1) = f''_j(x, t), with walls on the box faces.

    ``walls`` has one bit per face (-x, +x, -y, +y, -z, +z).  A clear bit makes
    that axis periodic (both faces of an axis must agree).  A set bit is a
    stationary no-slip wall half-way between the boundary node and the next
    (outside) node (Sec. 3.3, read as plain half-way bounce-back): a population
    whose link x -> x + c_j crosses a wall returns to x as the opposite
    population, f_{opp(j)}(x, t + 1) = f''_j(x, t).

    With ``TOP_FREE_SLIP`` set the +z face is a free-slip plane half-way above
    the top layer (Sec. 3.3): a population leaving through it is reflected
    specularly, its z component reversed and its tangential ones kept, so it
    arrives one tangential step further in the top layer,
    f_{mirz(j)}(x + (c_x, c_y, 0), t + 1) = f''_j(x, t).  A link that also
    crosses a no-slip face bounces back instead.
    """
    _check_walls(walls)
    nz, ny, nx = fpost.shape[1:]
    shape = (nx, ny, nz)
    wall_axis = [bool(walls & (1 << (2 * d))) for d in range(3)]
    free_top = bool(walls & TOP_FREE_SLIP)
    out = np.empty_like(fpost)
    # Coordinates of every node, per axis, broadcast to the field shape.
    coord = [np.arange(shape[0])[None, None, :], np.arange(shape[1])[None, :, None],
             np.arange(shape[2])[:, None, None]]
    for j in range(Q):
        moved = fpost[j]
        for d in range(3):
            if C[j, d] != 0:
                moved = np.roll(moved, C[j, d], axis=2 - d)
        out[j] = moved
    # Half-way bounce-back: a node x receives population j from x - c_j.  If
    # that link crosses a wall, the value is instead f''_{opp(j)}(x).
    for j in range(Q):
        crosses = np.zeros(fpost.shape[1:], dtype=bool)
        through_top = np.zeros(fpost.shape[1:], dtype=bool)
        for d in range(3):
            if C[j, d] == 0 or not wall_axis[d]:
                continue
            src = coord[d] - C[j, d]
            out_lo = np.broadcast_to(src < 0, crosses.shape)
            out_hi = np.broadcast_to(src >= shape[d], crosses.shape)
            if d == 2 and free_top:
                crosses = crosses | out_lo
                through_top = out_hi
            else:
                crosses = crosses | out_lo | out_hi
        out[j][crosses] = fpost[OPP[j]][crosses]
        if free_top and C[j, 2] == -1:
            # Specular reflection at the free-slip top: the population c_j
            # arrives from the mirrored one, mirz(j), that left the top layer
            # one tangential step back (wrapped on periodic axes).
            mirrored = fpost[MIRZ[j]]
            for d in range(2):
                if C[j, d] != 0:
                    mirrored = np.roll(mirrored, C[j, d], axis=2 - d)
            specular = through_top & ~crosses
            out[j][specular] = mirrored[specular]
    return out


def _check_walls(walls):
    for d in range(3):
        lo = bool(walls & (1 << (2 * d)))
        hi = bool(walls & (1 << (2 * d + 1)))
        if lo != hi:
            raise ValueError("both faces of an axis must be walls, or both periodic")
    if (walls & TOP_FREE_SLIP) and not (walls & WALL_ZP):
        raise ValueError("a free-slip top needs a bounded z axis")


def lb_step(f, omega, walls, force=None):
    """Collide (Eq. 13-15) then stream (Eq. 16) once."""
    return stream(collide(f, omega, force), walls)


def vorticity(u, walls):
    """curl u at the nodes by central differences, [3, nz, ny, nx].

    The paper interpolates the liquid vorticity to the bubble (Sec. 3.2,
    Algorithm 1 step 3) without saying how it is formed; it is read as the
    central difference (u(i+1) - u(i-1)) / 2 of the bare Eq. 10 velocity.  A
    neighbour beyond a face is a ghost node: periodic faces wrap; the no-slip
    wall half-way beyond the boundary node gives the ghost -u (velocity zero
    at the wall); the free-slip top gives the tangential components +u (zero
    shear at the plane).  Only tangential components are differentiated
    across a face in the curl.
    """
    u = np.asarray(u, dtype=np.float64)
    free_top = bool(walls & TOP_FREE_SLIP)

    def diff(comp, d):
        # d/dx_d of u[comp]; array axis of x_d is 2 - d
        f = u[comp]
        ax = 2 - d
        if not (walls & (1 << (2 * d))):
            return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))
        lo = np.take(f, [0], axis=ax)
        hi = np.take(f, [f.shape[ax] - 1], axis=ax)
        s_hi = 1.0 if (d == 2 and free_top) else -1.0
        padded = np.concatenate([-lo, f, s_hi * hi], axis=ax)
        n = f.shape[ax]
        return 0.5 * (np.take(padded, np.arange(2, n + 2), axis=ax)
                      - np.take(padded, np.arange(0, n), axis=ax))

    return np.stack([diff(2, 1) - diff(1, 2),     # d u_z/dy - d u_y/dz
                     diff(0, 2) - diff(2, 0),     # d u_x/dz - d u_z/dx
                     diff(1, 0) - diff(0, 1)])    # d u_y/dx - d u_x/dy
