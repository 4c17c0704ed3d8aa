"""The coupled LBGK-LPT time loop (Algorithm 1), FP64 (test infrastructure only).

One call of ``OracleSim.step`` is one pass of Algorithm 1's loop body:

  step 2   locate the active bubbles (the binning itself is in ``binning``);
  step 3   forward coupling: the bare Eq. 10 velocity of the current
           populations, interpolated to each bubble centre (Eq. 19-20), and
           with lift on its vorticity (central differences, the same map);
  step 4-5 forces (Table 1) and the explicit Newton update with sub-steps
           (Eq. 4, Table 2);
  step 6   backward coupling: psi_b = -(F_D + F_L) (or the sum of the
           interphase forces, Sec. 3.2) spread with Eq. 21 at the updated
           bubble position;
  step 7-9 first forcing, collision, second forcing (Eq. 12-15) with the
           spread force, then streaming (Eq. 16) with half-way bounce-back;
  step 10  a bubble that reaches the top wall stops (it is deactivated after
           this step's spreading and is not coupled again).

Initialisation sets f = f^eq(rho_l, u = 0) (Algorithm 1, initialisation).
"""
import numpy as np

from . import bubble as bub
from . import lattice as lat
from . import mapping


class OracleSim:
    def __init__(self, dims, omega, walls, params=None):
        self.dims = tuple(int(v) for v in dims)          # (nx, ny, nz)
        self.omega = float(omega)
        self.walls = int(walls)
        self.p = params if params is not None else bub.BubbleParams(omega)
        nx, ny, nz = self.dims
        rho = np.full((nz, ny, nx), self.p.rho_l)
        self.f = lat.equilibrium(rho, np.zeros((3, nz, ny, nx)))
        self.set_bubbles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
        self.last_force = None

    # ---- state ---------------------------------------------------------------
    def set_fields(self, rho, u):
        """f = f^eq(rho, u) (Algorithm 1 initialisation with a given field)."""
        self.f = lat.equilibrium(np.asarray(rho, dtype=np.float64),
                                 np.asarray(u, dtype=np.float64))

    def set_bubbles(self, pos, vel, diam):
        pos = np.array(pos, dtype=np.float64).reshape(-1, 3)
        self.x = pos.copy()
        self.u = np.array(vel, dtype=np.float64).reshape(-1, 3).copy()
        self.d = np.array(diam, dtype=np.float64).reshape(-1).copy()
        nb = len(self.d)
        self.n = self.p.width_factor * self.d
        self.active = np.ones(nb, dtype=bool)
        self.has_prev = np.zeros(nb, dtype=bool)
        self.ul_prev = np.zeros((nb, 3))
        self.ul = np.zeros((nb, 3))
        self.psi = np.zeros((nb, 3))

    def fields(self):
        """rho and the bare Eq. 10 velocity of the current populations."""
        return lat.density(self.f), lat.velocity(self.f)

    # ---- one step of Algorithm 1 ---------------------------------------------
    def step(self):
        p = self.p
        nb = len(self.d)
        force = None
        point = p.mapping == "point"
        if nb and self.active.any():
            rho = lat.density(self.f)
            u_nodes = lat.momentum(self.f) / rho                 # Eq. 10, bare moment
            w_nodes = lat.vorticity(u_nodes, self.walls) if p.lift else None
            xs_new, psis, ns = [], [], []
            for b in range(nb):
                if not self.active[b]:
                    continue
                ul = mapping.interpolate(u_nodes, self.x[b], self.n[b], self.walls,
                                         point)                                    # Eq. 20
                wl = (mapping.interpolate(w_nodes, self.x[b], self.n[b], self.walls, point)
                      if p.lift else None)
                dul = (ul - self.ul_prev[b]) / p.dt_l if self.has_prev[b] else np.zeros(3)
                x_new, u_new, psi = bub.advance(self.x[b], self.u[b], self.d[b], ul, dul,
                                                self.dims, self.walls, p, omega_l=wl)
                self.ul[b] = ul
                self.ul_prev[b] = ul
                self.has_prev[b] = True
                self.x[b] = x_new
                self.u[b] = u_new
                self.psi[b] = psi
                xs_new.append(x_new)
                psis.append(psi)
                ns.append(self.n[b])
            force = mapping.spread(psis, xs_new, ns, self.dims, self.walls, point)   # Eq. 21
            if self.walls & lat.WALL_ZP:
                nz = self.dims[2]
                for b in range(nb):
                    if self.active[b] and self.x[b, 2] >= nz - 0.5 * self.d[b]:
                        self.active[b] = False
        self.last_force = force
        self.f = lat.lb_step(self.f, self.omega, self.walls, force)

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
