"""Helpers for the GPU parity tests: marshal between the library and the oracle.

Only index bookkeeping lives here (direction order, array shapes); no
arithmetic of the method.
"""
import numpy as np

from oracle import lattice as olat
from paper_1710_07073_gb300 import lbm


def library_to_oracle_order():
    """perm such that f_oracle[j] = f_library[perm[j]] (matched by velocity vector)."""
    c_lib, _ = lbm.lbm_velocity_set()
    perm = []
    for j in range(19):
        k = int(np.flatnonzero((c_lib == olat.C[j]).all(axis=1))[0])
        perm.append(k)
    return np.array(perm)


def lib_pops_to_oracle(flat, dims):
    nx, ny, nz = dims
    f = flat.reshape(19, nz, ny, nx)
    return f[library_to_oracle_order()]


def oracle_pops_to_lib(f):
    perm = library_to_oracle_order()
    out = np.empty_like(f)
    out[perm] = f
    return out.reshape(-1)


def params_for_oracle(col_params, omega):
    from oracle import bubble as obub
    p = col_params
    return obub.BubbleParams(omega, g=p.g, rho_l=p.rho_l, rho_ratio=p.rho_ratio, sigma=p.sigma,
                             c_added_mass=p.c_added_mass, drag_scale=p.drag_scale,
                             sn_coeff=p.sn_coeff, sn_exp=p.sn_exp, width_factor=p.width_factor,
                             substeps=p.substeps,
                             lift=bool(p.forces & lbm.LBM_FORCE_LIFT),
                             stress_gradient=bool(p.forces & lbm.LBM_FORCE_STRESS),
                             mapping="point" if p.mapping == lbm.LBM_MAP_POINT else "cell",
                             reaction="all" if p.reaction == lbm.LBM_REACTION_ALL else "drag_lift")


def rel_linf(a, b):
    """max |a - b| / max |b|."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())
