"""Test helpers: set a CPU oracle problem up from a workload ``Case``."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

_FACE = {"xmin": O.XMIN, "xmax": O.XMAX, "ymin": O.YMIN, "ymax": O.YMAX, "zmin": O.ZMIN, "zmax": O.ZMAX}
_BC = {"zero_flux": O.ZERO_FLUX, "dirichlet": O.DIRICHLET, "flux": O.FLUX,
       "free_drainage": O.FREE_DRAINAGE, "seepage": O.SEEPAGE}
_MODEL = {"vg": O.VG, "gardner": O.GARDNER, "brooks_corey": O.BROOKS_COREY}


def oracle_soil(s: dict) -> dict:
    d = dict(s)
    d["model"] = _MODEL[s.get("model", "vg")]
    return d


def oracle_from_case(case, openmp=False, **param_overrides) -> O.Oracle:
    o = O.Oracle(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz, case.z_bottom, case.active, openmp=openmp)
    o.set_soils([oracle_soil(s) for s in case.soils], case.zone_of_cell, case.Ks_cell)
    for bc in case.bcs:
        o.set_bc(_FACE[bc.face], _BC[bc.type], bc.t, bc.v)
    p = dict(case.params)
    if tuple(case.gravity) != (0.0, 0.0, 1.0):
        p.update(grav_x=case.gravity[0], grav_y=case.gravity[1], grav_z=case.gravity[2])
    p.update(param_overrides)
    o.set_params(**p)
    o.set_state(case.h0, case.t0)
    return o


def steps_table(steps):
    return np.array([[s.dt, s.t, s.picard, s.cg, s.rejected, s.max_dh] for s in steps])
