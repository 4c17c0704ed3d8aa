"""Theoretical bubble velocities used to validate the method (Sec. 4.1), FP64.

Test infrastructure only.

* Eq. 23-24: force-balance terminal velocity.  Eq. 24 as printed drops rho_l
  from the drag side of Eq. 23; it is restored here (Table 4 pins this).  The
  drag coefficient follows Table 1 and depends on v_T through Re, so the
  balance is solved for its root by bisection.
* Eq. 25: Mendelson's terminal velocity, a closed form.
* Eq. 22: the relative-velocity ODE dv_r/dt = (F_B + F_D)/m, integrated with
  the same explicit step as the bubble update.  The paper writes m_b; the mass
  is an argument here (the bubble update uses m_b + C_A rho_l V_b).
"""
import math


def drag_cd(re, eo, sn_coeff=0.15, sn_exp=0.687):
    """Table 1 drag coefficient C_D(Re, Eo)."""
    visc = min(24.0 / re * (1.0 + sn_coeff * re ** sn_exp), 48.0 / re)
    return max(visc, 8.0 / 3.0 * eo / (eo + 4.0))


def terminal_velocity_force_balance(d, rho_l, rho_b, mu_l, sigma, g,
                                    sn_coeff=0.15, sn_exp=0.687, drag_scale=1.0):
    """Eq. 23: (rho_l - rho_b) V_b g = 1/2 C_D rho_l pi r_b^2 v_T^2, solved for v_T."""
    r = 0.5 * d
    vol = math.pi * d ** 3 / 6.0
    eo = (rho_l - rho_b) * g * d * d / sigma
    fb = (rho_l - rho_b) * vol * g

    def residual(v):
        re = rho_l * v * d / mu_l
        return 0.5 * drag_scale * drag_cd(re, eo, sn_coeff, sn_exp) * rho_l * math.pi * r * r * v * v - fb

    lo, hi = 0.0, 1.0
    while residual(hi) < 0.0:
        hi *= 2.0
    lo = hi * 1e-30
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if residual(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def terminal_velocity_mendelson(d, rho_l, sigma, g):
    """Eq. 25: v_TM = sqrt(2 sigma / (rho_l d_b) + g d_b / 2)."""
    return math.sqrt(2.0 * sigma / (rho_l * d) + g * d / 2.0)


def relative_velocity_history(d, rho_l, rho_b, mu_l, sigma, g, mass, dt, nsteps,
                              sn_coeff=0.15, sn_exp=0.687, drag_scale=1.0):
    """Eq. 22 along the vertical: dv_r/dt = (F_B + F_D)/mass, explicit Euler from rest."""
    r = 0.5 * d
    vol = math.pi * d ** 3 / 6.0
    eo = (rho_l - rho_b) * g * d * d / sigma
    fb = (rho_l - rho_b) * vol * g
    v = 0.0
    out = []
    for _ in range(nsteps):
        speed = abs(v)
        re = rho_l * speed * d / mu_l
        nu = mu_l / rho_l
        cdv = max(min(24.0 * nu / d * (1.0 + sn_coeff * re ** sn_exp), 48.0 * nu / d),
                  8.0 / 3.0 * eo / (eo + 4.0) * speed)
        fd = -0.5 * drag_scale * cdv * rho_l * math.pi * r * r * v
        v = v + (fb + fd) / mass * dt
        out.append(v)
    return out
