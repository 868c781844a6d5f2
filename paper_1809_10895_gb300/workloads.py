"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Each builder returns a :class:`Case`: mesh, soils, per-cell fields, boundary
series, solver parameters and the initial state.  The same ``Case`` feeds the
CUDA solver (through its binding) and the CPU oracle (through the tests'
helper), so both sides see identical inputs.  Faces and boundary types are
named by strings here so that neither side's enumerations leak into the other.

The paper's own cases and data sets are not available; these recipes stand in
for them with the shapes, sizes and value distributions of the paper's
workloads (Sec. 3.1 loam column, Appendix A/B soil blocks) and of the
benchmark configurations (1-D infiltration column, 3-D heterogeneous box,
synthetic watershed, uneven ensemble).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

FACES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")
BC_TYPES = ("zero_flux", "dirichlet", "flux", "free_drainage", "seepage")

# Sec. 3.1 loam (code-to-code case): Ks, alpha, n, theta_s, theta_r.
LOAM = dict(model="vg", theta_r=0.078, theta_s=0.43, alpha=3.6, n=1.56, Ks=2.89e-6, S=1e-5)
# Eq. 5 layers of the field case (Sec. 3.2).
FIELD_LAYERS = (
    dict(model="vg", theta_r=0.08, theta_s=0.45, alpha=2.3, n=1.2, Ks=1e-3, S=1e-5),
    dict(model="vg", theta_r=0.20, theta_s=0.50, alpha=2.1, n=2.4, Ks=1e-5, S=1e-5),
    dict(model="vg", theta_r=0.15, theta_s=0.55, alpha=1.7, n=1.9, Ks=1e-6, S=1e-5),
)


@dataclass
class BC:
    face: str
    type: str
    t: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    z_bottom: float = 0.0
    active: Optional[np.ndarray] = None          # uint8 [N] or None (all active)
    soils: list = field(default_factory=list)    # list of dicts
    zone_of_cell: Optional[np.ndarray] = None    # uint8 [N] or None
    Ks_cell: Optional[np.ndarray] = None         # float64 [N] or None
    bcs: list = field(default_factory=list)      # list of BC
    params: dict = field(default_factory=dict)
    h0: Optional[np.ndarray] = None              # float64 [N]
    t0: float = 0.0
    t_end: float = 0.0
    gravity: tuple = (0.0, 0.0, 1.0)             # elevation gradient in the grid's axes (z up)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def z_centres(self) -> np.ndarray:
        """Cell-centre elevation per cell (x fastest, z slowest)."""
        k = np.arange(self.nz)
        z = self.z_bottom + (k + 0.5) * self.dz
        return np.repeat(z, self.nx * self.ny)

    def n_active(self) -> int:
        return self.N if self.active is None else int(np.count_nonzero(self.active))


def default_params(**kw) -> dict:
    """Solver parameters (readings: Picard 1e-6 m, CG 1e-10 relative, EBATS
    thresholds 10 / 3 / 8 and factor 1.3, chord threshold 1e-10 m)."""
    p = dict(tol_picard=1e-6, tol_cg=1e-10, cg_max_it=10000, dt0=1.0, dt_max=600.0, dt_min=1e-3,
             f_grow=1.3, f_shrink=1.3, n_inc=10, n_small=3, n_max=8, eps_chord=1e-10)
    p.update(kw)
    return p


# --------------------------------------------------------------------------
# 1-D vertical infiltration column
# --------------------------------------------------------------------------
def infiltration_column(nz: int = 200, dz: float = 0.005, t_end: float = 86400.0,
                        h_init: float = -1.0, h_top: float = 0.0, soil: Optional[dict] = None,
                        **param_overrides) -> Case:
    """1x1xnz column, homogeneous loam, uniform initial head, ponded top
    (Dirichlet), free-draining bottom.  Per unit area (dx = dy = 1 m).
    Defaults: 200 cells of 0.5 cm, h0 = -1 m, top h = 0, dt 1 s growing by
    1.2 up to 600 s, one simulated day, CG tolerance 1e-12."""
    soil = dict(LOAM if soil is None else soil)
    params = default_params(tol_cg=1e-12, f_grow=1.2, f_shrink=1.2)
    params.update(param_overrides)
    return Case(name=f"infiltration_column_1x1x{nz}", nx=1, ny=1, nz=nz, dx=1.0, dy=1.0, dz=dz,
                soils=[soil],
                bcs=[BC("zmax", "dirichlet", np.array([0.0]), np.array([h_top])),
                     BC("zmin", "free_drainage")],
                params=params, h0=np.full(nz, h_init), t_end=t_end)


# --------------------------------------------------------------------------
# Gaussian random field with exponential covariance (circulant embedding)
# --------------------------------------------------------------------------
def gaussian_random_field(shape, corr_len_cells: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance stationary Gaussian field on a grid of
    ``shape`` (nx, ny, nz) with covariance exp(-r / corr_len) (r in cells),
    synthesised spectrally on a periodic grid padded to twice the size.
    Negative embedding eigenvalues (if any) are clipped, and the result is
    rescaled to unit sample variance.  Returned in x-fastest order."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    px, py, pz = 2 * nx, 2 * ny, 2 * nz
    ix = np.minimum(np.arange(px), px - np.arange(px)).astype(np.float64)
    iy = np.minimum(np.arange(py), py - np.arange(py)).astype(np.float64)
    iz = np.minimum(np.arange(pz), pz - np.arange(pz)).astype(np.float64)
    r = np.sqrt(ix[:, None, None] ** 2 + iy[None, :, None] ** 2 + iz[None, None, :] ** 2)
    cov = np.exp(-r / corr_len_cells)
    lam = np.fft.fftn(cov).real
    lam = np.clip(lam, 0.0, None)
    noise = rng.standard_normal((px, py, pz)) + 1j * rng.standard_normal((px, py, pz))
    f = np.fft.ifftn(np.sqrt(lam) * noise) * np.sqrt(px * py * pz)
    g = f.real[:nx, :ny, :nz]
    g = (g - g.mean()) / g.std()
    # (nx, ny, nz) array indexed [i, j, k] -> x-fastest flat order
    return np.ascontiguousarray(g.transpose(2, 1, 0)).ravel()


# --------------------------------------------------------------------------
# 3-D heterogeneous box
# --------------------------------------------------------------------------
def stiff_block(nx: int = 256, ny: int = 256, nz: int = 64, seed: int = 12, sigma_lnK: float = 1.5) -> Case:
    """A stiff linear system for comparing preconditioners: saturated soil
    (hydrostatic head above a Dirichlet bottom), log-normal Ks (geometric mean
    1e-4 m/s, uncorrelated, sigma_lnK), 10:1 anisotropic cells (1 x 1 x 0.1 m),
    a specific storage of 1e-6 1/m so that the capacity term is far below the
    face conductances, and a top flux of 5e-5 m/s."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    Ks = np.exp(np.log(1e-4) + sigma_lnK * rng.standard_normal(N))
    c = Case(name=f"stiff_block_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=1.0, dy=1.0, dz=0.1,
             soils=[dict(model="vg", theta_r=0.05, theta_s=0.4, alpha=2.0, n=1.8, Ks=1e-4, S=1e-6)],
             Ks_cell=Ks, params=default_params(tol_cg=1e-10))
    c.h0 = (nz * 0.1 + 2.0) - c.z_centres()
    c.bcs = [BC("zmin", "dirichlet", np.array([0.0]), np.array([nz * 0.1 + 1.5])),
             BC("zmax", "flux", np.array([0.0]), np.array([5e-5]))]
    return c


def heterogeneous_box(nx: int = 128, ny: int = 128, nz: int = 64, d: float = 0.25, seed: int = 0,
                      t_end: float = 48 * 3600.0, rain: float = 1e-6, rain_hours: float = 6.0,
                      water_table_depth: float = 10.0, sigma_lnK: float = 1.0,
                      corr_len_cells: float = 8.0, Kg: float = 1e-5, **param_overrides) -> Case:
    """nx*ny*nz cubes of side d.  ln Ks = ln Kg + sigma * g, g a seeded
    Gaussian random field with exponential covariance (correlation length in
    cells).  One van Genuchten soil otherwise (alpha 2 1/m, n 1.8, theta_r
    0.05, theta_s 0.40).  Hydrostatic initial head with the water table at
    ``water_table_depth`` below the top; bottom face held at that hydrostatic
    head; top flux ``rain`` (m/s) for ``rain_hours`` then 0; lateral faces
    zero-flux."""
    g = gaussian_random_field((nx, ny, nz), corr_len_cells, seed)
    Ks = np.exp(np.log(Kg) + sigma_lnK * g)
    soil = dict(model="vg", theta_r=0.05, theta_s=0.40, alpha=2.0, n=1.8, Ks=Kg, S=1e-5)
    case = Case(name=f"heterogeneous_box_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=d, dy=d, dz=d,
                soils=[soil], Ks_cell=Ks, params=default_params(**param_overrides), t_end=t_end)
    z_top = nz * d
    z_wt = z_top - water_table_depth
    case.h0 = z_wt - case.z_centres()
    case.bcs = [BC("zmax", "flux", np.array([0.0, rain_hours * 3600.0]), np.array([rain, 0.0])),
                BC("zmin", "dirichlet", np.array([0.0]), np.array([z_wt - 0.0]))]
    return case


# --------------------------------------------------------------------------
# Synthetic watershed: diamond-square terrain, masked columns, layers, rain
# --------------------------------------------------------------------------
def diamond_square(n_pow2: int, roughness: float, seed: int) -> np.ndarray:
    """Fractal height map on a (2^k+1)^2 grid by the diamond-square
    algorithm; amplitude halves by 2^-roughness per level.  Values in [0,1]."""
    rng = np.random.default_rng(seed)
    size = n_pow2 + 1
    a = np.zeros((size, size))
    a[0, 0], a[0, -1], a[-1, 0], a[-1, -1] = rng.uniform(-1, 1, 4)
    step, scale = n_pow2, 1.0
    while step > 1:
        half = step // 2
        # diamond step: centres of squares
        for y in range(half, size, step):
            for x in range(half, size, step):
                avg = (a[y - half, x - half] + a[y - half, x + half] + a[y + half, x - half]
                       + a[y + half, x + half]) / 4.0
                a[y, x] = avg + rng.uniform(-scale, scale)
        # square step: edge midpoints
        for y in range(0, size, half):
            for x in range((y + half) % step, size, step):
                s, c = 0.0, 0
                for dy_, dx_ in ((-half, 0), (half, 0), (0, -half), (0, half)):
                    yy, xx = y + dy_, x + dx_
                    if 0 <= yy < size and 0 <= xx < size:
                        s += a[yy, xx]
                        c += 1
                a[y, x] = s / c + rng.uniform(-scale, scale)
        step = half
        scale *= 2.0 ** (-roughness)
    a -= a.min()
    a /= max(a.max(), 1e-300)
    return a


def poisson_rain_series(hours: int, mean_gap_h: float, mean_dur_h: float, mean_int_mm_h: float,
                        seed: int) -> tuple:
    """Hourly rainfall (m/s) with Poisson storm arrivals (exponential gaps),
    exponential durations (rounded up to whole hours) and exponential
    intensities constant within a storm.  Returns (t breakpoints [s], v)."""
    rng = np.random.default_rng(seed)
    r = np.zeros(hours)
    t = rng.exponential(mean_gap_h)
    while t < hours:
        dur = int(np.ceil(rng.exponential(mean_dur_h)))
        inten = rng.exponential(mean_int_mm_h) * 1e-3 / 3600.0
        i0 = int(t)
        r[i0:min(hours, i0 + max(dur, 1))] = inten
        t += dur + rng.exponential(mean_gap_h)
    return np.arange(hours) * 3600.0, r


def watershed(nx: int = 512, ny: int = 512, nz: int = 64, dx: float = 10.0, dz: float = 0.5,
              seed: int = 0, hours: int = 720, water_table: float = 0.0, **param_overrides) -> Case:
    """Masked structured watershed: diamond-square terrain (roughness 0.8)
    scaled to 16-32 m above the bottom, cells above the surface inactive, four
    soil layers of nz/4 cells with uniformly sampled van Genuchten parameters,
    hydrostatic initial head with the water table at ``water_table`` metres
    above the bottom (default: at the bottom, so the seepage face starts
    inactive), hourly Poisson rain on the surface, seepage bottom, lateral
    zero flux."""
    rng = np.random.default_rng(seed + 7)
    k = int(np.ceil(np.log2(max(nx, ny))))
    hm = diamond_square(2 ** k, 0.8, seed)[:ny, :nx]
    top = 16.0 + 16.0 * hm                                   # surface elevation [m]
    zc = (np.arange(nz) + 0.5) * dz
    active = (zc[:, None, None] < top[None, :, :]).astype(np.uint8).ravel()
    soils = []
    for _ in range(4):
        soils.append(dict(model="vg", theta_r=0.05, theta_s=0.40, alpha=float(rng.uniform(0.5, 5.0)),
                          n=float(rng.uniform(1.2, 2.5)), Ks=float(10 ** rng.uniform(-7, -4)), S=1e-5))
    band = max(nz // 4, 1)
    zone = np.minimum(np.arange(nz) // band, 3).astype(np.uint8)
    zone_of_cell = np.repeat(zone, nx * ny)
    t, v = poisson_rain_series(hours, 48.0, 6.0, 3.0, seed + 11)
    case = Case(name=f"watershed_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dz,
                active=active, soils=soils, zone_of_cell=zone_of_cell,
                params=default_params(**param_overrides), t_end=hours * 3600.0)
    case.h0 = water_table - case.z_centres()
    case.bcs = [BC("zmax", "flux", t, v), BC("zmin", "seepage")]
    return case


# --------------------------------------------------------------------------
# Tilted slope (Sec. 4.2)
# --------------------------------------------------------------------------
def tilted_slope(nx: int = 850, ny: int = 850, nz: int = 50, dx: float = 2.0, dy: float = 2.0, dz: float = 0.2,
                 slope_deg: float = 20.0, river_deg: float = 3.0, h_init: float = -10.0, rain: float = 2e-7,
                 days: float = 10.0, **param_overrides) -> Case:
    """The strong-scaling slope of Sec. 4.2 on a grid aligned with the slab:
    a homogeneous layer of the Sec. 3.1 loam, nz dz thick (10 m), its plane
    rising at slope_deg along x away from the river and at river_deg along y
    (the river's own slope); x = 0 is the river (Dirichlet h = 0 over that
    face), rain on the top face, zero flux elsewhere; dry initial head
    h_init.  Gravity is the elevation gradient in the grid's axes,
    (sin a, cos a sin b, cos a cos b).  Defaults: 2 m x 2 m x 0.2 m cells over
    1.7 km x 1.7 km (36 M cells), 10 days, Picard 1 mm, dt 0.1 s .. 30 min as
    printed; the rain rate is not printed -- 2e-7 m/s keeps the slope
    unsaturated, as the paper's smooth regime requires."""
    a, b = np.radians(slope_deg), np.radians(river_deg)
    params = default_params(tol_picard=1e-3, dt0=0.1, dt_max=1800.0)
    params.update(param_overrides)
    case = Case(name=f"tilted_slope_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, soils=[dict(LOAM)],
                params=params, t_end=days * 86400.0,
                gravity=(float(np.sin(a)), float(np.cos(a) * np.sin(b)), float(np.cos(a) * np.cos(b))))
    case.h0 = np.full(case.N, float(h_init))
    case.bcs = [BC("xmin", "dirichlet", np.array([0.0]), np.array([0.0])),
                BC("zmax", "flux", np.array([0.0]), np.array([float(rain)]))]
    return case


# --------------------------------------------------------------------------
# Uneven ensemble
# --------------------------------------------------------------------------
def ensemble(n: int = 256, seed: int = 0, t_end: float = 2 * 86400.0, max_side: int = 16,
             nz_range=(50, 400), dz: float = 0.01, top_head: float = -0.01, **param_overrides) -> list:
    """Independent instances of uneven size: footprint nx, ny ~ U{1..max_side},
    depth nz ~ U{nz_range}, 1 cm cells, uniformly sampled van Genuchten
    parameters, uniform initial head in [-3, -0.1] m, top held at
    ``top_head`` (default -1 cm: water at the surface without positive
    pressure; a head of exactly 0 drives soils with n < 2 to the h = 0 state in
    which classical Picard cannot contract), free-draining bottom, lateral
    zero flux."""
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(n):
        nx, ny = (int(v) for v in rng.integers(1, max_side + 1, 2))
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        soil = dict(model="vg", theta_r=0.05, theta_s=0.40, alpha=float(rng.uniform(0.5, 5.0)),
                    n=float(rng.uniform(1.2, 2.5)), Ks=float(10 ** rng.uniform(-7, -4)), S=1e-5)
        h_init = float(rng.uniform(-3.0, -0.1))
        c = Case(name=f"ensemble_{i}_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dz, dy=dz, dz=dz,
                 soils=[soil], params=default_params(**param_overrides), t_end=t_end)
        c.h0 = np.full(c.N, h_init)
        c.bcs = [BC("zmax", "dirichlet", np.array([0.0]), np.array([top_head])), BC("zmin", "free_drainage")]
        cases.append(c)
    return cases


# Layer shapes (cin, cout) of the warm-start network: input convolution,
# two per residual block (four blocks), output convolution.
NN_LAYERS = [(4, 32)] + [(32, 32)] * 8 + [(32, 1)]


def nn_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the warm-start network, flat FP64.

    Layer by layer: W[cout, 3, 3, 3, cin] then b[cout].  Weights are normal
    with std sqrt(2 / fan_in) (He et al. 2015), scaled by 0.1 for the second
    convolution of each residual block and for the output convolution so
    the network starts close to the identity map plus a small output;
    biases are zero.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co) in enumerate(NN_LAYERS):
        std = np.sqrt(2.0 / (27 * ci))
        if li == len(NN_LAYERS) - 1 or (li >= 1 and li % 2 == 0):
            std *= 0.1
        parts.append(rng.normal(0.0, std, size=27 * ci * co))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
