"""Closed-form pins of the oracle's boundary readings.

Saturated homogeneous flow is linear in total head, and a two-point flux
scheme with half-cell Dirichlet distances reproduces linear heads exactly:
a ponded column draining through a seepage face (R13: Dirichlet h = 0 while
the bottom cell is saturated) must settle on h(z) = H0 (z / L) above the
bottom face; flow between two Dirichlet x-faces of a one-cell-thick strip
(no vertical flow) must settle on a linear h(x)."""
import numpy as np

from oracle import oracle as O

SAT = dict(model=O.VG, theta_r=0.05, theta_s=0.40, alpha=2.0, n=1.8, Ks=1e-5, S=1e-4)


def test_seepage_column_settles_on_the_linear_profile():
    nz, dz, H0 = 20, 0.05, 0.3
    L = nz * dz
    o = O.Oracle(1, 1, nz, 1.0, 1.0, dz, 0.0, None)
    o.set_soils([SAT], None, None)
    o.set_bc(O.ZMAX, O.DIRICHLET, np.array([0.0]), np.array([H0]))
    o.set_bc(O.ZMIN, O.SEEPAGE)
    o.set_params(dt_max=1e5, tol_cg=1e-14)
    o.set_state(np.full(nz, 0.2), 0.0)              # saturated throughout
    o.run(1e7)
    zc = (np.arange(nz) + 0.5) * dz
    # total head H = h + z linear from 0 (bottom face, h = 0) to H0 + L (top face)
    exact = (H0 + L) * zc / L - zc
    np.testing.assert_allclose(o.get_state()[0], exact, rtol=0, atol=1e-9)
    mb = o.mass_balance()
    assert mb["outflow_cum"] > 0.0 and mb["closure_rel"] <= 1e-9


def test_lateral_dirichlet_flow_is_linear_in_x():
    nx, nz, dx, dz = 16, 1, 0.5, 0.2
    o = O.Oracle(nx, 1, nz, dx, 1.0, dz, 0.0, None)
    o.set_soils([SAT], None, None)
    o.set_bc(O.XMIN, O.DIRICHLET, np.array([0.0]), np.array([1.2]))
    o.set_bc(O.XMAX, O.DIRICHLET, np.array([0.0]), np.array([0.4]))
    o.set_params(dt_max=1e5, tol_cg=1e-14)
    o.set_state(np.full(nx * nz, 0.8), 0.0)
    o.run(1e7)
    h = o.get_state()[0].reshape(nz, nx)
    xc = (np.arange(nx) + 0.5) * dx
    # one cell thick, zero flux above and below: h (and total head) linear in x
    exact = 1.2 + (0.4 - 1.2) * xc / (nx * dx)
    np.testing.assert_allclose(h[0], exact, rtol=0, atol=1e-9)
