"""Seeded synthetic basins and request streams.

The paper's North Atlantic run (Section 6) uses Mercator bathymetry and ERA15 winds, which are
not available here. The generators below stand in for that workload with seeded synthetic basins
that keep its shapes and scales: a thin layered (sigma-coordinate) domain, depths of hundreds of
metres to 5 km over thousands of kilometres, the viscosity and time step of Section 6, artificial
slip boundaries on the south ("Equator") and north ("70 N") edges, a zonal wind stress and a
beta-plane Coriolis parameter.

Every array here is input data. Nothing in this module evaluates the finite element method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Lateral walls that are artificial slip boundaries (Gamma_1 in Section 2): bit flags.
WALL_WEST = 1   # x = 0
WALL_EAST = 2   # x = (nx-1) dx
WALL_SOUTH = 4  # y = 0
WALL_NORTH = 8  # y = (ny-1) dy
WALL_ALL = WALL_WEST | WALL_EAST | WALL_SOUTH | WALL_NORTH

OMEGA_EARTH = 7.2921e-5   # rad/s
RHO0 = 1025.0             # kg/m^3, converts a wind stress (N/m^2) to a kinematic tension


@dataclass
class Basin:
    """A layered basin on a structured nx x ny x nz node grid.

    Arrays are indexed [j, i] (j along y, i along x). A node column (i, j) is ocean where
    mask[j, i] == 1; its nz nodes sit at z_k = -depth[j, i] * (1 - k/(nz-1)).
    """
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    mask: np.ndarray            # (ny, nx) uint8
    depth: np.ndarray           # (ny, nx) float64, > 0 on ocean columns
    slip_walls: int             # WALL_* bits: outer walls that are Gamma_1
    nu: tuple                   # (nu1, nu2, nu3)
    dt: float
    coriolis: Optional[np.ndarray] = None   # (ny, nx) float64 f = 2 omega_3, or None (f = 0)
    theta: Optional[np.ndarray] = None      # (2, ny, nx) float64 kinematic wind tension, or None
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def Lx(self) -> float:
        return (self.nx - 1) * self.dx

    @property
    def Ly(self) -> float:
        return (self.ny - 1) * self.dy


def box_basin(nh: int = 16, nz: int = 8, eps: float = 0.01, nu=(1.0, 1.0, 1e-4), dt: float = 0.01,
              nhy: Optional[int] = None, slip_walls: int = WALL_ALL, seed: int = 1207) -> Basin:
    """Unit-square box of constant depth eps (aspect ratio eps), nh x nh x nz nodes.

    Defaults: 16 x 16 x 8 nodes, eps = 0.01, nu = (1, 1, 1e-4) = (lambda_1, lambda_2,
    eps^2 lambda_3) as in Section 2's scaling, all four lateral walls slip.
    """
    ny = nh if nhy is None else nhy
    mask = np.ones((ny, nh), dtype=np.uint8)
    depth = np.full((ny, nh), float(eps))
    return Basin(name=f"box{nh}x{ny}x{nz}", nx=nh, ny=ny, nz=nz, dx=1.0 / (nh - 1), dy=1.0 / (ny - 1),
                 mask=mask, depth=depth, slip_walls=slip_walls, nu=tuple(nu), dt=dt, seed=seed)


def _periodic_gaussian_smooth(field_: np.ndarray, sigma: float) -> np.ndarray:
    ny, nx = field_.shape
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    kern = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (kx ** 2 + ky ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(field_) * kern))


def _keep_largest_cell_component(node_mask: np.ndarray) -> np.ndarray:
    """Keep the largest 8-connected component of active hex columns (cells).

    A cell is active when its four corner columns are ocean; two cells that share a corner
    column share nodes, hence 8-connectivity. Returns the node mask of the kept cells.
    """
    from scipy import ndimage
    m = node_mask.astype(bool)
    cell = m[:-1, :-1] & m[1:, :-1] & m[:-1, 1:] & m[1:, 1:]
    lab, nlab = ndimage.label(cell, structure=np.ones((3, 3), dtype=int))
    if nlab == 0:
        raise ValueError("basin has no ocean cell")
    sizes = np.bincount(lab.ravel())
    sizes[0] = 0
    keep = lab == int(np.argmax(sizes))
    out = np.zeros_like(m)
    out[:-1, :-1] |= keep
    out[1:, :-1] |= keep
    out[:-1, 1:] |= keep
    out[1:, 1:] |= keep
    return out.astype(np.uint8)


def ocean_basin(seed: int = 1207, nx: int = 512, ny: int = 512, nz: int = 32, dx: float = 1.0e4,
                ocean_fraction: float = 0.6, smooth_sigma: float = 16.0, n_gauss: int = 40,
                hmin: float = 200.0, hmax: float = 5000.0, nu=(1.0e8, 1.0e8, 1.0e2),
                dt: float = 2.592e6, tau0: float = 0.1, lat_north_deg: float = 70.0) -> Basin:
    """Synthetic ocean basin: 512 x 512 columns of 10 km, 32 sigma layers (about 5M nodes).

    Land mask: seeded white noise, periodic Gaussian smoothing (sigma = 16 cells), thresholded and the
    largest connected component kept, with the threshold chosen so that the kept component covers
    about 60% of the columns. Bathymetry: 200 m plus
    4800 m times a [0, 1]-normalised sum of 40 seeded Gaussians. Wind stress
    tau = tau0 (-cos(pi y / Ly), 0) N/m^2, applied as the kinematic tension theta = tau / rho0.
    Coriolis: beta plane f = 2 Omega sin(latitude), latitude from 0 (y = 0, the Equator) to 70 N
    (y = Ly). Viscosity nu_h = 1e8 m^2/s and the one-month time step follow Section 6; the
    vertical viscosity is nu_h / 1e6. South and north edges are artificial slip walls.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((ny, nx))
    smooth = _periodic_gaussian_smooth(noise, smooth_sigma)
    # Raise the threshold's ocean share until the kept component itself covers ~ocean_fraction.
    frac = ocean_fraction
    while True:
        thr = np.quantile(smooth, 1.0 - frac)
        mask = _keep_largest_cell_component((smooth > thr).astype(np.uint8))
        if mask.mean() >= ocean_fraction or frac >= 0.95:
            break
        frac += 0.01

    Lx, Ly = (nx - 1) * dx, (ny - 1) * dx
    X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dx)
    cx = rng.uniform(0.0, Lx, n_gauss)
    cy = rng.uniform(0.0, Ly, n_gauss)
    w = rng.uniform(0.02, 0.15, n_gauss) * Lx
    a = rng.uniform(0.2, 1.0, n_gauss)
    g = np.zeros((ny, nx))
    for q in range(n_gauss):
        g += a[q] * np.exp(-((X - cx[q]) ** 2 + (Y - cy[q]) ** 2) / (2.0 * w[q] ** 2))
    g = (g - g.min()) / (g.max() - g.min())
    depth = hmin + (hmax - hmin) * g

    theta = np.zeros((2, ny, nx))
    theta[0] = tau0 * (-np.cos(math.pi * Y / Ly)) / RHO0
    lat = np.deg2rad(lat_north_deg) * Y / Ly
    coriolis = 2.0 * OMEGA_EARTH * np.sin(lat)
    return Basin(name=f"ocean{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, mask=mask,
                 depth=depth, slip_walls=WALL_SOUTH | WALL_NORTH, nu=tuple(nu), dt=dt,
                 coriolis=coriolis, theta=theta, seed=seed)


def batch_basins(seed: int = 1207, count: int = 64, smin: int = 48, smax: int = 384,
                 nzmin: int = 8, nzmax: int = 48) -> List[Basin]:
    """Independent box basins (as the 16x16x8 box) of uneven size for batched solves.

    Basin b draws, from seed + b, a side s = round(exp(U[ln smin, ln smax])) and nz in
    U{nzmin..nzmax}: about 18k to 7M nodes.
    """
    out = []
    for b in range(count):
        rng = np.random.default_rng(seed + b)
        s = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        nz = int(rng.integers(nzmin, nzmax + 1))
        bas = box_basin(nh=s, nz=nz, seed=seed + b)
        bas.name = f"batch{b}_{s}x{s}x{nz}"
        out.append(bas)
    return out


@dataclass
class Request:
    t_arrival: float
    session: int
    step: int
    nrhs: int
    rhs_seed: int


@dataclass
class Session:
    side: int
    nz: int
    seed: int


def request_stream(seed: int = 1207, rate: float = 200.0, n_requests: int = 2000,
                   concurrent_sessions: int = 8, steps_per_session: int = 100,
                   median_nodes: float = 1.5e5, sigma: float = 1.0, max_nodes: float = 8e6,
                   max_rhs: int = 4):
    """Poisson arrivals of solve requests (rate per second) over basins with lognormal node counts.

    Each session is one box basin that issues `steps_per_session` consecutive requests; requests
    are dealt round-robin to `concurrent_sessions` open sessions, and a finished session is
    replaced by a new basin. A basin draws n ~ lognormal(median, sigma) clipped to max_nodes,
    nz in U{8..48} and side sqrt(n / nz). Each request carries 1..max_rhs right-hand sides (4: the
    systems of a step with the lumped correction; 7 with the consistent-mass one).
    Returns (sessions, requests).
    """
    rng = np.random.default_rng(seed)
    sessions: List[Session] = []

    def new_session() -> int:
        n = min(float(np.exp(rng.normal(math.log(median_nodes), sigma))), max_nodes)
        nz = int(rng.integers(8, 49))
        side = max(4, int(round(math.sqrt(n / nz))))
        sessions.append(Session(side=side, nz=nz, seed=int(rng.integers(0, 2 ** 31 - 1))))
        return len(sessions) - 1

    open_s = [new_session() for _ in range(concurrent_sessions)]
    used = {s: 0 for s in open_s}
    t = 0.0
    reqs: List[Request] = []
    for q in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        slot = q % concurrent_sessions
        s = open_s[slot]
        reqs.append(Request(t_arrival=t, session=s, step=used[s], nrhs=int(rng.integers(1, max_rhs + 1)),
                            rhs_seed=int(rng.integers(0, 2 ** 31 - 1))))
        used[s] += 1
        if used[s] >= steps_per_session:
            ns = new_session()
            open_s[slot] = ns
            used[ns] = 0
    return sessions, reqs


def mms_modes(seed: int = 1207, count: int = 4):
    """Seeded modes for a manufactured solution: (amplitude ~ N(0,1), m, l in {1,2,3})."""
    rng = np.random.default_rng(seed)
    amps = rng.standard_normal(count)
    ms = rng.integers(1, 4, count)
    ls = rng.integers(1, 4, count)
    return [(float(amps[q]), int(ms[q]), int(ls[q])) for q in range(count)]


def manufactured_field(basin: Basin, col_i: np.ndarray, col_j: np.ndarray, modes) -> np.ndarray:
    """A smooth field sampled at the nodes of the given columns (node = column * nz + k, the
    library's and the oracle's order), for manufactured right-hand sides b = A u*:
        u*(x, y, z) = sum_q a_q sin(m_q pi x / Lx) sin(l_q pi y / Ly) cos(pi s / 2),
    s = -z / h in [0, 1] the depth fraction (1 at the sea floor, 0 at the surface), with the
    modes (a_q, m_q, l_q) of mms_modes. Grid geometry only: x = i dx, y = j dy,
    z_k = -h (1 - k / (nz - 1))."""
    col_i = np.asarray(col_i)
    col_j = np.asarray(col_j)
    x = col_i * basin.dx / max(basin.Lx, 1e-300)
    y = col_j * basin.dy / max(basin.Ly, 1e-300)
    s = 1.0 - np.arange(basin.nz) / (basin.nz - 1)
    horiz = np.zeros(len(col_i))
    for a, m, l in modes:
        horiz += a * np.sin(m * math.pi * x) * np.sin(l * math.pi * y)
    return (horiz[:, None] * np.cos(0.5 * math.pi * s)[None, :]).ravel()


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded N(0, 1) float64 vector of length n."""
    return np.random.default_rng(seed).standard_normal(n)
