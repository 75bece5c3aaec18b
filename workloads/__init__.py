"""Seeded synthetic inputs for the shallow-water step: bathymetry, initial
states and solver settings.

This module is shared by the oracle side and the CUDA side and holds none of
the method's arithmetic: it only builds inputs (beds, still-water depths,
initial waves) as float64 host arrays of shape (ny, nx), row-major, x fastest.

The workloads stand in for the paper's data that is not available here:
  * the Crescent City DEM of "Real-world scenario" (4 m NOAA grid) is replaced
    by a seeded synthetic shelf-and-coast DEM (``coastal_dem``);
  * the ISEC planar-beach benchmark of "Validation for tsunami simulations"
    is replaced by a solitary-wave runup on a 1:20 slope (``planar_beach``);
  * the hill layouts of the Lunghino et al. comparison are replaced by seeded
    Gaussian coastal hills behind a seeded shoreline (``mitigation_ensemble``).
The initial wave of the ensemble is the Carrier N-wave of the paper's
Eq. (20), with the minus sign of the second exponent restored.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

WALL, INFLOW, PERIODIC = 0, 1, 2
G = 9.81


@dataclasses.dataclass
class Scenario:
    """One solve: grid, bed, initial state and settings."""

    name: str
    dx: float
    dy: float
    b: np.ndarray
    h: np.ndarray
    hu: np.ndarray
    hv: np.ndarray
    g: float = G
    manning_n: float = 0.0
    h_dry: float = 1e-5
    h_wet: float = 1e-3
    h_film: float = 1e-3  # film depth of the velocity desingularisation
    weno_eps: float = 1e-6
    fixed_dt: float = 0.0
    cfl: float = 0.4
    t_end: float = 0.0
    bc: Tuple[int, int, int, int] = (WALL, WALL, WALL, WALL)
    b_jump_x: float = 0.0
    b_jump_y: float = 0.0
    inflow_amp: float = 0.0
    inflow_period: float = 0.0
    inflow_depth: float = 0.0
    z_ref: float = 0.0  # still-water level; still-water depth d = max(z_ref - b, 0)
    alpha_margin: float = 0.0  # > 0: the fused-step variant (one splitting speed per step); 0: per stage
    shore: int = 0  # 1: the shoreline variant (hydrostatic-reconstruction faces at dry and land cells)
    t0: float = 0.0
    steps: int = 0  # suggested number of RK3 steps for this workload

    @property
    def ny(self) -> int:
        return int(self.b.shape[0])

    @property
    def nx(self) -> int:
        return int(self.b.shape[1])

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def copy(self, **changes) -> "Scenario":
        s = dataclasses.replace(self, **changes)
        for f in ("b", "h", "hu", "hv"):
            if f not in changes:
                setattr(s, f, getattr(self, f).copy())
        return s

    def eta(self) -> np.ndarray:
        return self.h + self.b


def _centres(n: int, d: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * d


def _fractal_field_2d(ny: int, nx: int, seed: int, rms: float, slope: float = -2.0) -> np.ndarray:
    """Gaussian random field with isotropic power spectrum |k|^slope, zero
    mean, scaled to the given rms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((ny, nx))
    spec = np.fft.rfft2(white)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = 1.0
    amp = k ** (slope / 2.0)
    amp[0, 0] = 0.0
    f = np.fft.irfft2(spec * amp, s=(ny, nx))
    f -= f.mean()
    return f * (rms / f.std())


def _fractal_field_1d(n: int, seed: int, rms: float, slope: float = -2.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal(n)
    spec = np.fft.rfft(white)
    k = np.fft.rfftfreq(n)
    k[0] = 1.0
    amp = k ** (slope / 2.0)
    amp[0] = 0.0
    f = np.fft.irfft(spec * amp, n=n)
    f -= f.mean()
    return f * (rms / f.std())


def _still(b: np.ndarray, eta: np.ndarray | float = 0.0):
    h = np.maximum(np.asarray(eta) - b, 0.0) * np.ones_like(b)
    z = np.zeros_like(b)
    return h, z, z.copy()


# --------------------------------------------------------------- configs
def gaussian_hump(n: int = 128, dx: float = 1.0, depth: float = 1.0, amp: float = 0.1,
                  sigma_cells: float = 8.0, steps: int = 200) -> Scenario:
    """Flat bottom, reflective walls, centred Gaussian hump at rest (FP64 case)."""
    c = (n - 1) / 2.0
    i = np.arange(n, dtype=np.float64)
    r2 = (i[None, :] - c) ** 2 + (i[:, None] - c) ** 2
    eta = amp * np.exp(-r2 / (2.0 * sigma_cells ** 2))
    b = np.full((n, n), -depth)
    h = eta - b
    z = np.zeros_like(b)
    return Scenario("gaussian_hump_%d" % n, dx, dx, b, h, z, z.copy(), steps=steps)


def planar_beach(nx: int = 2048, ny: int = 64, dx: float = 0.5, depth: float = 10.0,
                 slope: float = 1.0 / 20.0, land: float = 5.0, H_over_d: float = 0.02,
                 manning_n: float = 0.025, steps: int = 5000) -> Scenario:
    """Solitary wave running up a plane beach: flat bed at -depth, then a
    1:20 slope from -depth to +land over the last (depth+land)/slope metres.
    The crest starts arccosh(sqrt(20))/k seaward of the toe (the standard
    Synolakis placement), with u = eta sqrt(g/d) toward the shore."""
    x = _centres(nx, dx)
    L = nx * dx
    x_toe = L - (depth + land) / slope
    bx = np.where(x < x_toe, -depth, -depth + (x - x_toe) * slope)
    H = H_over_d * depth
    k = math.sqrt(3.0 * H / (4.0 * depth ** 3))
    x0 = x_toe - math.acosh(math.sqrt(20.0)) / k
    eta = H / np.cosh(k * (x - x0)) ** 2
    h1 = np.maximum(eta - bx, 0.0)
    u1 = eta * math.sqrt(G / depth)
    hu1 = np.where(h1 > 0.0, h1 * u1, 0.0)
    b = np.repeat(bx[None, :], ny, axis=0)
    h = np.repeat(h1[None, :], ny, axis=0)
    hu = np.repeat(hu1[None, :], ny, axis=0)
    return Scenario("planar_beach_%dx%d" % (nx, ny), dx, dx, b, h, hu, np.zeros_like(b),
                    manning_n=manning_n, steps=steps)


def carrier_nwave(X: np.ndarray, A: float, lam: float) -> np.ndarray:
    """Carrier N-wave of Eq. (20) as a function of the seaward distance X from
    the shoreline (the paper's 1000 m / 6000 m shifts are its code's own
    origin offsets and are dropped here)."""
    a1, a2 = A, A / 3.0
    k1, k2 = 28.416 / lam ** 2, 256.0 / lam ** 2
    x1, x2 = 0.5151125 * lam, 0.2048 * lam
    return 2.0 * (a1 * np.exp(-k1 * (X - x1) ** 2) - a2 * np.exp(-k2 * (X - x2) ** 2))


def coastal_dem(n: int = 4096, dx: float = 5.0, seed: int = 3, shelf_depth: float = 200.0,
                land_height: float = 20.0, noise_rms: float = 3.0, amp: float = 4.0,
                period: float = 600.0, t0: float = 600.0, steps: int = 200) -> Scenario:
    """Synthetic coastal DEM: a continental-shelf ramp from -200 m at x=0 to 0
    at x=0.8 L, land rising to +20 m at x=L, plus a seeded Gaussian random
    field with power-spectrum slope -2 and 3 m rms.  An N-wave enters through
    the x- edge (amplitude = peak elevation, period T).  The state at t0 holds
    the part of the wave that entered before t0 as a right-going long wave."""
    x = _centres(n, dx)
    L = n * dx
    base = np.where(x < 0.8 * L, -shelf_depth + shelf_depth * x / (0.8 * L),
                    land_height * (x - 0.8 * L) / (0.2 * L))
    b = base[None, :] + _fractal_field_2d(n, n, seed, noise_rms)
    c0 = math.sqrt(G * shelf_depth)
    lam = period * c0
    # wave already inside: eta(x, t0) = eta_in(t0 - x/c0), eta_in from Eq. (20)
    s = 1.3 * lam - c0 * (t0 - x / c0)
    eta1 = carrier_nwave(s, amp / 2.0, lam)
    eta1 = np.where(x < 0.5 * L, eta1, 0.0)
    eta = np.repeat(eta1[None, :], n, axis=0)
    h = np.maximum(eta - b, 0.0)
    u = eta * math.sqrt(G / shelf_depth)
    hu = np.where(h > 1e-3, h * u, 0.0)
    return Scenario("coastal_dem_%d" % n, dx, dx, b, h, hu, np.zeros_like(b), bc=(INFLOW, WALL, WALL, WALL),
                    inflow_amp=amp, inflow_period=period, inflow_depth=shelf_depth, t0=t0,
                    manning_n=0.025, steps=steps)


def _shoreline_offsets(ny_max_cells: int, dy: float, seed: int, rms: float = 5.0) -> np.ndarray:
    return _fractal_field_1d(ny_max_cells, seed, rms)


def mitigation_scenario(nx: int, ny: int, rng: np.random.Generator, shore: np.ndarray,
                        dx: float = 2.0, land_width: float = 400.0, beach_slope: float = 1.0 / 50.0,
                        deep: float = 20.0, high: float = 10.0, A: float = 2.0,
                        name: str = "mitigation") -> Scenario:
    """Coast with a 1:50 beach from -20 m to +10 m whose shoreline sits
    land_width seaward of the x+ edge, displaced along y by the shared seeded
    offsets; 1-12 Gaussian hills (2-8 m high, 10-30 m radius) behind it; a
    Carrier N-wave of Eq. (20) at rest offshore with lambda = half the
    offshore width."""
    x = _centres(nx, dx)
    y = _centres(ny, dx)
    X = nx * dx
    xs = (X - land_width) + shore[:ny][:, None]
    b = np.clip((x[None, :] - xs) * beach_slope, -deep, high)
    nh = int(rng.integers(1, 13))
    for _ in range(nh):
        H = rng.uniform(2.0, 8.0)
        R = rng.uniform(10.0, 30.0)
        hx = (X - land_width) + rng.uniform(20.0, land_width - 60.0)
        hy = rng.uniform(0.0, ny * dx)
        b = b + H * np.exp(-(((x[None, :] - hx) ** 2 + (y[:, None] - hy) ** 2) / R ** 2))
    offshore = X - land_width
    lam = 0.5 * offshore
    eta = carrier_nwave(xs - x[None, :], A, lam)
    h = np.maximum(eta - b, 0.0)
    z = np.zeros_like(b)
    return Scenario(name, dx, dx, b, h, z, z.copy(), manning_n=0.025)


def mitigation_ensemble(count: int = 64, seed: int = 4, dx: float = 2.0, t_end: float = 1200.0,
                        nx_range=(512, 1024), ny_range=(256, 1024), land_width: float = 400.0) -> List[Scenario]:
    """Seeded ensemble of uneven grids (multiples of 32) sharing one seeded
    shoreline, each with its own hill layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shore = _shoreline_offsets(ny_range[1], dx, seed + 1000)
    out = []
    for s in range(count):
        nx = int(rng.integers(nx_range[0] // 32, nx_range[1] // 32 + 1)) * 32
        ny = int(rng.integers(ny_range[0] // 32, ny_range[1] // 32 + 1)) * 32
        sc = mitigation_scenario(nx, ny, rng, shore, dx=dx, land_width=land_width, name="ensemble_%02d" % s)
        sc.t_end = t_end
        out.append(sc)
    return out


@dataclasses.dataclass
class Request:
    arrival: float
    scenario: Scenario
    deadline: Optional[float] = None   # s after arrival by which the result is wanted (None: none)
    cancel_at: Optional[float] = None  # s after arrival at which the client withdraws (None: never)


def serving_requests(rate: float, count: int, seed: int = 5, dx: float = 2.0,
                     horizon: float = 600.0, n_range=(256, 2048)) -> List[Request]:
    """Poisson arrivals at the given rate; square grids with N log-uniform in
    n_range rounded to 32; coast and hills as in the ensemble."""
    rng = np.random.Generator(np.random.PCG64(seed * 1000003 + int(rate * 1000)))
    shore = _shoreline_offsets(n_range[1], dx, seed + 2000)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        n = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        n = int(max(n_range[0], min(n_range[1], round(n / 32.0) * 32)))
        sc = mitigation_scenario(n, n, rng, shore, dx=dx, name="req_%04d" % k)
        sc.t_end = horizon
        out.append(Request(t, sc))
    return out


# ----------------------------------------------------- verification cases
def standing_wave_slope(nx_sea: int = 200, nx_land: int = 40, ny: int = 4, dx: float = 5.0,
                        slope: float = 0.05, amp: float = 0.002) -> Scenario:
    """Small-amplitude standing wave on a plane beach (the linear limit of the
    Carrier-Greenspan problem): offshore wall at x = 0, shoreline at
    x = L = nx_sea dx, bed b = -slope (L - x) everywhere (land rising beyond
    the shoreline), at rest with eta = amp J0(j11 sqrt(r / L)) on the wet side,
    r = L - x the distance from the shoreline and j11 the first zero of J1
    (the mode whose velocity vanishes at the offshore wall)."""
    from scipy.special import j0, jn_zeros
    nx = nx_sea + nx_land
    L = nx_sea * dx
    x = _centres(nx, dx)
    r = L - x
    bx = -slope * r
    j11 = float(jn_zeros(1, 1)[0])
    eta = np.where(r > 0.0, amp * j0(j11 * np.sqrt(np.maximum(r, 0.0) / L)), amp)
    h1 = np.maximum(eta - bx, 0.0)
    b = np.repeat(bx[None, :], ny, axis=0)
    h = np.repeat(h1[None, :], ny, axis=0)
    return Scenario("standing_wave_slope_%dx%d" % (nx, ny), dx, dx, b, h, np.zeros_like(b), np.zeros_like(b))


# ------------------------------------------------------------ real DEMs
def read_esri_ascii(path: str):
    """Read an ESRI ASCII grid (header keys ncols, nrows, xllcorner|xllcenter,
    yllcorner|yllcenter, cellsize or dx and dy, optional NODATA_value; then
    nrows rows of ncols values, northernmost row first).

    Returns (z, dx, dy, x0, y0, nodata): z float64 (ny, nx) with row j at
    y = y0 + (j + 0.5) dy, i.e. flipped so that y grows with the row index as
    in every array of this module; (x0, y0) the lower-left corner; nodata a
    bool mask of the cells that held the NODATA value."""
    with open(path) as f:
        tokens = f.read().split()
    head, k = {}, 0
    while k + 1 < len(tokens) and not _is_number(tokens[k]):
        head[tokens[k].lower()] = float(tokens[k + 1])
        k += 2
    nx, ny = int(head["ncols"]), int(head["nrows"])
    if "cellsize" in head:
        dx = dy = head["cellsize"]
    else:
        dx, dy = head["dx"], head["dy"]
    if "xllcorner" in head:
        x0 = head["xllcorner"]
    else:
        x0 = head["xllcenter"] - 0.5 * dx
    if "yllcorner" in head:
        y0 = head["yllcorner"]
    else:
        y0 = head["yllcenter"] - 0.5 * dy
    vals = np.array([float(t) for t in tokens[k:k + nx * ny]], dtype=np.float64)
    if vals.size != nx * ny or not (dx > 0 and dy > 0):
        raise ValueError("%s: expected %d x %d values and positive cell sizes" % (path, ny, nx))
    z = vals.reshape(ny, nx)[::-1].copy()
    nodata = np.zeros(z.shape, dtype=bool)
    if "nodata_value" in head:
        nodata = z == head["nodata_value"]
    return z, float(dx), float(dy), float(x0), float(y0), nodata


def _is_number(t: str) -> bool:
    try:
        float(t)
        return True
    except ValueError:
        return False


def read_dem(path: str):
    """An elevation grid from a GeoTIFF (recognised by the TIFF header) or an
    ESRI ASCII file, as (z, dx, dy, x0, y0, nodata) of read_esri_ascii."""
    with open(path, "rb") as f:
        head = f.read(4)
    if head in (b"II*\0", b"MM\0*", b"II+\0", b"MM\0+"):
        from workloads.geotiff import read_geotiff
        return read_geotiff(path)
    return read_esri_ascii(path)


def dem_scenario(path: str, sea_level: float = 0.0, nodata_elevation: Optional[float] = None,
                 crop: Optional[Tuple[int, int, int, int]] = None, stride: int = 1, **settings) -> Scenario:
    """Still water at sea_level over the bed of an elevation grid (m, positive
    up): a GeoTIFF or an ESRI ASCII file (read_dem).  NODATA cells take nodata_elevation (default:
    the highest valid elevation, i.e. dry land behind walls).  crop =
    (j0, j1, i0, i1) selects rows j0..j1-1 and columns i0..i1-1 (after the
    flip to y-up order) and stride keeps every stride-th cell.  Further keyword
    arguments set Scenario fields (boundary types, inflow wave, friction ...);
    z_ref defaults to sea_level."""
    z, dx, dy, _, _, nodata = read_dem(path)
    if nodata.any():
        if nodata.all():
            raise ValueError("%s holds no valid elevation" % path)
        fill = float(z[~nodata].max()) if nodata_elevation is None else float(nodata_elevation)
        z = np.where(nodata, fill, z)
    if crop is not None:
        j0, j1, i0, i1 = crop
        z = z[j0:j1, i0:i1]
    if stride > 1:
        z = z[::stride, ::stride]
        dx, dy = dx * stride, dy * stride
    b = np.ascontiguousarray(z)
    h, hu, hv = _still(b, sea_level)
    settings.setdefault("z_ref", sea_level)
    name = settings.pop("name", "dem_%dx%d" % (b.shape[1], b.shape[0]))
    return Scenario(name, dx, dy, b, h, hu, hv, **settings)


def lake_at_rest(nx: int = 32, ny: int = 32, dx: float = 1.0, eta0: float = 0.5, depth: float = 10.0,
                 rms: float = 3.0, seed: int = 11, islands: bool = False) -> Scenario:
    """Still water over a seeded rough bed (slope -2 spectrum).  With islands,
    parts of the bed stick out of the water."""
    b = -depth + _fractal_field_2d(ny, nx, seed, rms)
    if islands:
        b = b + 14.0 * np.exp(-(((np.arange(nx)[None, :] - nx / 3) ** 2 +
                                (np.arange(ny)[:, None] - ny / 2) ** 2) / (0.02 * nx * ny)))
    h, hu, hv = _still(b, eta0)
    return Scenario("lake_at_rest", dx, dx, b, h, hu, hv, z_ref=eta0)


def dam_break(nx: int = 1000, ny: int = 4, length: float = 100.0, x0: float = 50.0,
              h_l: float = 2.0, h_r: float = 1.0) -> Scenario:
    """Wet dam break of Section 2.1 (flat bed b = 0, walls, 1-D in 2-D)."""
    dx = length / nx
    x = _centres(nx, dx)
    h1 = np.where(x <= x0, h_l, h_r)
    b = np.zeros((ny, nx))
    h = np.repeat(h1[None, :], ny, axis=0)
    z = np.zeros_like(b)
    return Scenario("dam_break", dx, dx, b, h, z, z.copy())


def parabolic_bowl(nx: int = 400, ny: int = 4, dx: float = 1.0, h0: float = 1.0, a: float = 100.0) -> Scenario:
    """Planar parabolic bowl of Section 2.2: b = h0((x-L/2)^2/a^2 - 1), the
    Eq. (17) initial surface, at rest."""
    L = nx * dx
    x = _centres(nx, dx)
    bx = h0 * ((x - L / 2.0) ** 2 / a ** 2 - 1.0)
    h1 = np.maximum(-h0 * (((2.0 * x - L + 1.0) / (2.0 * a)) ** 2 - 1.0), 0.0)
    b = np.repeat(bx[None, :], ny, axis=0)
    h = np.repeat(h1[None, :], ny, axis=0)
    z = np.zeros_like(b)
    return Scenario("parabolic_bowl", dx, dx, b, h, z, z.copy())


def manning_slope(nx: int = 32, ny: int = 4, dx: float = 1.0, slope: float = 1.0 / 20.0, depth: float = 0.5,
                  n: float = 0.033, q: Optional[float] = None) -> Scenario:
    """Flow down a 1:20 slope with Manning n = 0.033 (Section 2.3): periodic in
    x with the bed offset of one period, walls in y.  q is the initial
    discharge hu (default: the Eq. (19) normal-flow value is supplied by the
    caller)."""
    x = _centres(nx, dx)
    bx = -slope * x
    b = np.repeat(bx[None, :], ny, axis=0)
    h = np.full((ny, nx), depth)
    hu = np.full((ny, nx), 0.0 if q is None else q)
    return Scenario("manning_slope", dx, dx, b, h, hu, np.zeros_like(b), manning_n=n,
                    bc=(PERIODIC, PERIODIC, WALL, WALL), b_jump_x=-slope * nx * dx, z_ref=10.0)
