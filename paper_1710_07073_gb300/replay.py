"""Physical-unit replay of the paper's validation runs (Sec. 4, Appendix A).

Every run goes through the library (include/lbm.h): the set-up is converted
to lattice units by ``lbm_units_from_physical`` (Appendix A) and stepped by
``lbm_step``; this module only chooses the set-ups and converts the bubble
state back to SI units.

Set-up (Sec. 3.1, Table 2, Table 3, Table 5):

* a 0.15 m x 0.15 m column filled with water to 0.45 m; no-slip walls and a
  free-slip top (Sec. 3.3); a bubble leaves the coupling when it reaches the
  free surface (Algorithm 1, stop at the top);
* cell size dx = a_r d_b with the aspect ratio a_r = 1.25 (Eq. 17), or 0.625
  and 0.3125 for the grid study (Table 5); liquid step 1e-4 s and bubble
  sub-step 1e-5 s (Table 2: 10 sub-steps);
* Table 3 properties: water 1000 kg/m^3 and 1e-3 kg/(m s), air 1 kg/m^3,
  surface tension 0.073 N/m, g = 9.81 m/s^2;
* one bubble released at rest at the column axis, its lowest point 5 mm
  above the floor (the paper gives no release height; with the 4 mm bubble
  this reproduces its quoted rise time of about 1.86 s to the surface).

Lattice sizes are the physical sizes times LCF rounded to whole cells (the
7 mm and 9 mm cases of Table 4 do not divide the column evenly).

Runs:

* E1 (Sec. 4.1, Fig. 2a): 4 mm, a_r = 1.25: the relative velocity
  u_b - u_l(x_b) against time, and the time to reach the surface;
* E2 (Table 4, Fig. 2b): 2-10 mm at a_r = 1.25: the terminal velocity;
* E4 (Table 6, Fig. 4): 4, 8 and 10 mm at the three aspect ratios.

The terminal velocity is the mean vertical bubble velocity between 0.5 s and
0.2 s before the bubble reaches the surface.

Run from the repository root (needs a GPU):  python -m paper_1710_07073_gb300.replay
"""
import json
import sys

import numpy as np

from . import lbm

WIDTH = 0.15           # m, column width and depth (Sec. 3.1)
HEIGHT = 0.45          # m, water level (Sec. 3.1)
DT = 1e-4              # s, liquid time step (Table 2)
RELEASE_GAP = 0.005    # m, from the floor to the bubble's lowest point
WATER_AIR = dict(rho_l=1000.0, rho_b=1.0, mu_l=1e-3, sigma=0.073, g=9.81)   # Table 3

E2_DIAMETERS_MM = (2, 3, 4, 5, 6, 7, 8, 9, 10)        # Table 4
E4_CASES = [(d, a) for d in (4, 8, 10) for a in (1.25, 0.625, 0.3125)]   # Table 5-6


def setup(d_mm, aspect=1.25, dt=DT, props=None):
    """Lattice set-up of one run: dims, omega, params, bubble (lattice units), units."""
    d = d_mm * 1e-3
    dx = aspect * d
    ph = dict(WATER_AIR if props is None else props)
    units, params, omega = lbm.lbm_units_from_physical(dx, dt, **ph)
    lcf = units.lcf
    n_w = int(round(WIDTH * lcf))
    n_h = int(round(HEIGHT * lcf))
    d_lu = d * lcf
    pos = np.array([0.5 * n_w, 0.5 * n_w, (RELEASE_GAP + 0.5 * d) * lcf])
    return {"d_mm": d_mm, "aspect": aspect, "dims": (n_w, n_w, n_h), "omega": omega,
            "params": params, "units": units, "d_lu": d_lu, "pos": pos}


def run(su, seconds=2.0, record_every=10, early_steps=300, storage=lbm.LBM_STORE_F32):
    """Step one set-up until the bubble leaves the coupling (or ``seconds``).

    Returns a history in SI units: t (s, after each recorded step), z (m),
    u_b and u_l (m/s, vertical), active, every step for the first
    ``early_steps`` and every ``record_every`` steps after, plus the time the
    bubble reached the surface (None if it did not) and whether the liquid
    solver flagged an instability.
    """
    u = su["units"]
    vel_scale = u.tcf / u.lcf
    col = lbm.Column(su["dims"], su["omega"], lbm.LBM_WALL_ALL_FREE_TOP, storage=storage,
                     params=su["params"])
    lbm.lbm_set_bubbles(col.ctx, su["pos"], [0.0, 0.0, 0.0], [su["d_lu"]])
    total = int(round(seconds * u.tcf))
    t, z, ub, ul, act = [], [], [], [], []
    step, t_top, unstable = 0, None, False
    try:
        while step < total:
            k = 1 if step < early_steps else min(record_every, total - step)
            try:
                lbm.lbm_step(col.ctx, k)
            except lbm.LbmError as e:
                if e.code != lbm.LBM_ERR_UNSTABLE:
                    raise
                unstable = True
                break
            step += k
            b = lbm.lbm_get_bubbles(col.ctx)
            t.append(step / u.tcf)
            z.append(b["pos"][0, 2] / u.lcf)
            ub.append(b["vel"][0, 2] * vel_scale)
            ul.append(b["ul"][0, 2] * vel_scale)
            act.append(bool(b["active"][0]))
            if not act[-1]:
                t_top = step / u.tcf
                break
    finally:
        col.close()
    return {"t": np.array(t), "z": np.array(z), "u_b": np.array(ub), "u_l": np.array(ul),
            "active": np.array(act), "t_top": t_top, "unstable": unstable, "steps": step}


def terminal_velocity(hist, start=0.5, end_gap=0.2):
    """Mean vertical bubble velocity (and slip) between ``start`` and
    ``end_gap`` before the bubble reached the surface (or the run ended)."""
    t = hist["t"]
    stop = (hist["t_top"] if hist["t_top"] is not None else t[-1]) - end_gap
    sel = (t >= start) & (t <= stop) & hist["active"]
    if not sel.any():
        return float("nan"), float("nan")
    return float(hist["u_b"][sel].mean()), float((hist["u_b"] - hist["u_l"])[sel].mean())


def replay(cases, seconds=2.0):
    """Run each (d_mm, aspect) case; one result dict per case."""
    out = []
    for d_mm, aspect in cases:
        su = setup(d_mm, aspect)
        h = run(su, seconds)
        vt, slip = terminal_velocity(h)
        out.append({"d_mm": d_mm, "aspect": aspect, "dims": list(su["dims"]),
                    "omega": su["omega"], "d_lu": su["d_lu"], "lcf": su["units"].lcf,
                    "mcf": su["units"].mcf, "tcf": su["units"].tcf, "g_lu": su["params"].g,
                    "sigma_lu": su["params"].sigma, "v_terminal": vt, "slip_terminal": slip,
                    "t_top": h["t_top"], "unstable": h["unstable"], "steps": h["steps"]})
    return out


def main(argv=None):
    cases = sorted(set([(d, 1.25) for d in E2_DIAMETERS_MM] + E4_CASES))
    res = replay(cases)
    for r in res:
        print(json.dumps(r))
    return 0 if not any(r["unstable"] for r in res) else 1


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
