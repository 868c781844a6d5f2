"""Writes appendix_a_gardner.json: the steady Gardner column of Appendix A
(Orgogozo et al., arXiv:1809.10895) solved by the CPU oracle, with the
closed-form profile of Eq. A8 beside it.  Calls only oracle/ (and the input
recipe below); run from the repository root:

    python tests/golden/make_appendix_a.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

# Appendix A as printed: a homogeneous 1 m column, water table at the bottom
# (h = 0), imposed top flux q, Ks = 1e-6 m/s, alpha = 0.06 1/m, 100 cells of
# 1 cm, PCG precision 1e-10, Picard precision 1e-8 m, initial time step 1 s,
# maximum time step 3600 s.  theta_r, theta_s and S do not enter the steady
# state; the values below are this recipe's.
CONFIG = dict(L=1.0, nz=100, Ks=1e-6, alpha=0.06, theta_r=0.05, theta_s=0.40, S=1e-5, tol_cg=1e-10,
              tol_picard=1e-8, dt0=1.0, dt_max=3600.0, t_end=3.0e6)
FLUXES = [-4e-6, -1e-6, 5e-7, 9e-7]     # evaporation (< 0) and infiltration (> 0)


def oracle_column(q, cfg=CONFIG, picard_form=0):
    nz = cfg["nz"]
    dz = cfg["L"] / nz
    o = O.Oracle(1, 1, nz, 1.0, 1.0, dz, 0.0, None)
    o.set_soils([dict(model=O.GARDNER, theta_r=cfg["theta_r"], theta_s=cfg["theta_s"], alpha=cfg["alpha"],
                      n=2.0, Ks=cfg["Ks"], S=cfg["S"])], None, None)
    o.set_bc(O.ZMIN, O.DIRICHLET, np.array([0.0]), np.array([0.0]))
    o.set_bc(O.ZMAX, O.FLUX, np.array([0.0]), np.array([q]))
    o.set_params(tol_cg=cfg["tol_cg"], tol_picard=cfg["tol_picard"], dt0=cfg["dt0"], dt_max=cfg["dt_max"],
                 cg_max_it=10000, dt_min=1e-3, f_grow=1.3, f_shrink=1.3, n_inc=10, n_small=3, n_max=8,
                 eps_chord=1e-10, picard_form=picard_form)
    zc = (np.arange(nz) + 0.5) * dz
    o.set_state(-zc, 0.0)
    o.run(cfg["t_end"])
    return zc, o.get_state()[0]


def main():
    out = {"citation": "Appendix A (steady Gardner column, Eq. A8) of arXiv:1809.10895: configuration as printed; "
                       "h_oracle from the CPU oracle at t_end, h_exact from Eq. A8",
           "config": CONFIG, "cases": []}
    for q in FLUXES:
        zc, h = oracle_column(q)
        out["cases"].append({"q": q, "z": zc.tolist(), "h_oracle": h.tolist(),
                             "h_exact": O.gardner_steady_profile(zc, q, CONFIG["Ks"], CONFIG["alpha"]).tolist()})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "appendix_a_gardner.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
