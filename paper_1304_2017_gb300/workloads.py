"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only builds inputs: the measurement geometry of a spherical-aperture
scanner (Sec. III.A), voxelised phantoms (Eq. coeffint: point samples of A(r) at the
grid nodes) and random data vectors.  It contains none of the operator arithmetic
(no lattice, no interpolation, no D), so that the oracle and the GPU path can both
draw their inputs from it without sharing any code of the method.

Units: millimetres, microseconds, MHz.  Volumes are numpy arrays of shape
(nz, ny, nx) (x fastest); data are (Q, K) (time fastest), transducer index
q = ring * n_views + view (Sec. III.A, the data layout of Alg. 4).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Geometry", "arc_positions", "centred_origin", "enclosing_radius", "centred_tmin",
    "make_geometry", "spheres_phantom", "ellipsoids_phantom", "supersampled_sphere",
    "config", "CONFIGS", "random_data",
]


@dataclasses.dataclass
class Geometry:
    """Scanner + grid description (Sec. III.A).  All fields are plain inputs."""
    nx: int
    ny: int
    nz: int
    spacing_mm: float
    origin_mm: tuple            # position of node (0, 0, 0)
    positions_mm: np.ndarray    # (Q, 3) float64, measurement sphere centred at the origin
    n_samples: int              # K
    fs_mhz: float               # sampling rate; Delta_t = 1 / fs
    t_min_us: float             # time of sample 0
    c_mm_per_us: float          # speed of sound
    support_radius_mm: float    # R: sphere (centred at the origin) that contains the object
    gruneisen: float = 1.0      # Gamma = beta c^2 / C_p, scales D
    lattice_weights: int = 0    # 0: Delta_s^2 per shell-lattice point; 1: exact ring-strip area

    @property
    def n_transducers(self) -> int:
        return int(self.positions_mm.shape[0])

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def data_shape(self):
        return (self.n_transducers, self.n_samples)

    def node_coords_mm(self):
        """1-D node coordinates along x, y, z."""
        o = self.origin_mm
        d = self.spacing_mm
        return (o[0] + d * np.arange(self.nx), o[1] + d * np.arange(self.ny),
                o[2] + d * np.arange(self.nz))

    def subset(self, qs) -> "Geometry":
        """Same scanner restricted to transducers `qs` (used to time the oracle on a sample)."""
        g = dataclasses.replace(self)
        g.positions_mm = np.ascontiguousarray(self.positions_mm[np.asarray(qs)])
        return g


def arc_positions(n_rings: int, n_views: int, radius_mm: float, theta_min: float | None = None):
    """Transducers on a sphere: N_r rings at polar angles theta_min + n * pi / N_r, N_v views
    at azimuth 2 pi v / N_v (Sec. III.A).  Default theta_min = pi / (2 N_r) makes the rings
    cover the full polar range symmetrically (Sec. IV.A uses pi/256 for 128 rings)."""
    if theta_min is None:
        theta_min = math.pi / (2 * n_rings)
    pos = np.empty((n_rings * n_views, 3), dtype=np.float64)
    for r in range(n_rings):
        th = theta_min + r * math.pi / n_rings
        for v in range(n_views):
            ph = 2.0 * math.pi * v / n_views
            pos[r * n_views + v] = (radius_mm * math.sin(th) * math.cos(ph),
                                    radius_mm * math.sin(th) * math.sin(ph),
                                    radius_mm * math.cos(th))
    return pos


def centred_origin(nx, ny, nz, spacing_mm):
    """Origin that centres the node cuboid on (0, 0, 0)."""
    return (-spacing_mm * (nx - 1) / 2.0, -spacing_mm * (ny - 1) / 2.0, -spacing_mm * (nz - 1) / 2.0)


def enclosing_radius(nx, ny, nz, spacing_mm, origin_mm):
    """Radius of the origin-centred sphere that contains the node cuboid grown by one
    spacing on every side (the support of the trilinear expansion functions)."""
    best = 0.0
    for cx in (origin_mm[0] - spacing_mm, origin_mm[0] + spacing_mm * nx):
        for cy in (origin_mm[1] - spacing_mm, origin_mm[1] + spacing_mm * ny):
            for cz in (origin_mm[2] - spacing_mm, origin_mm[2] + spacing_mm * nz):
                best = max(best, math.sqrt(cx * cx + cy * cy + cz * cz))
    return best


def centred_tmin(radius_mm, n_samples, fs_mhz, c):
    """Time window centred on the arrival from the origin: t_min = max(0, R_s/c - K dt / 2)."""
    return max(0.0, radius_mm / c - n_samples / fs_mhz / 2.0)


def make_geometry(n, spacing_mm, rings, views, radius_mm, n_samples, fs_mhz=20.0, c=1.5,
                  t_min_us=None, support_radius_mm=None, gruneisen=1.0, theta_min=None,
                  positions_mm=None, origin_mm=None, lattice_weights=0):
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(n)
    origin = centred_origin(nx, ny, nz, spacing_mm) if origin_mm is None else tuple(origin_mm)
    pos = arc_positions(rings, views, radius_mm, theta_min) if positions_mm is None else \
        np.ascontiguousarray(positions_mm, dtype=np.float64)
    if support_radius_mm is None:
        support_radius_mm = enclosing_radius(nx, ny, nz, spacing_mm, origin)
    if t_min_us is None:
        t_min_us = centred_tmin(radius_mm, n_samples, fs_mhz, c)
    return Geometry(nx, ny, nz, float(spacing_mm), origin, pos, int(n_samples), float(fs_mhz),
                    float(t_min_us), float(c), float(support_radius_mm), float(gruneisen), int(lattice_weights))


# ----------------------------------------------------------------------------- phantoms

def _central_box(geom: Geometry, frac=0.7):
    xs, ys, zs = geom.node_coords_mm()
    lo = np.array([xs[0], ys[0], zs[0]])
    hi = np.array([xs[-1], ys[-1], zs[-1]])
    mid = (lo + hi) / 2
    half = (hi - lo) / 2 * frac
    return mid - half, mid + half


def spheres_phantom(geom: Geometry, n_spheres=8, seed=1304, r_range=(0.5, 2.0), a_range=(0.5, 1.0)):
    """Sum of uniform spheres, point-sampled at the nodes (Eq. coeffint).  Centres are
    uniform in the central 70 % of the grid."""
    rng = np.random.default_rng(seed)
    lo, hi = _central_box(geom)
    xs, ys, zs = geom.node_coords_mm()
    vol = np.zeros(geom.vol_shape, dtype=np.float64)
    for _ in range(n_spheres):
        c = rng.uniform(lo, hi)
        r = rng.uniform(*r_range)
        a = rng.uniform(*a_range)
        _add_ellipsoid(vol, xs, ys, zs, c, np.eye(3), np.array([r, r, r]), a, geom.spacing_mm)
    return vol.astype(np.float32)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _add_ellipsoid(vol, xs, ys, zs, centre, rot, semi, amp, spacing):
    ext = semi.max() + spacing
    ix = np.nonzero((xs >= centre[0] - ext) & (xs <= centre[0] + ext))[0]
    iy = np.nonzero((ys >= centre[1] - ext) & (ys <= centre[1] + ext))[0]
    iz = np.nonzero((zs >= centre[2] - ext) & (zs <= centre[2] + ext))[0]
    if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
        return
    Z, Y, X = np.meshgrid(zs[iz] - centre[2], ys[iy] - centre[1], xs[ix] - centre[0], indexing="ij")
    p = np.stack([X, Y, Z], axis=-1) @ rot  # coordinates in the ellipsoid frame
    inside = ((p / semi) ** 2).sum(axis=-1) <= 1.0
    vol[np.ix_(iz, iy, ix)] += amp * inside


def ellipsoids_phantom(geom: Geometry, n=200, seed=1304, semi_range=(0.2, 3.0), a_range=(0.2, 1.0)):
    """Random ellipsoids (vascular / tumour-like mix): semi-axes U(0.2, 3) mm, amplitude
    U(0.2, 1), uniformly random orientation, centres in the central 70 %."""
    rng = np.random.default_rng(seed)
    lo, hi = _central_box(geom)
    xs, ys, zs = geom.node_coords_mm()
    vol = np.zeros(geom.vol_shape, dtype=np.float64)
    for _ in range(n):
        c = rng.uniform(lo, hi)
        semi = rng.uniform(*semi_range, size=3)
        a = rng.uniform(*a_range)
        _add_ellipsoid(vol, xs, ys, zs, c, _random_rotation(rng), semi, a, geom.spacing_mm)
    return vol.astype(np.float32)


def supersampled_sphere(geom: Geometry, centre, radius, amp=1.0, ss=4):
    """Partial-volume voxelisation of one uniform sphere: each node gets the fraction of an
    ss^3 sub-sample cloud (spanning one spacing around the node) that lies inside."""
    xs, ys, zs = geom.node_coords_mm()
    d = geom.spacing_mm
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    vol = np.zeros(geom.vol_shape, dtype=np.float64)
    ext = radius + d
    ix = np.nonzero(np.abs(xs - centre[0]) <= ext)[0]
    iy = np.nonzero(np.abs(ys - centre[1]) <= ext)[0]
    iz = np.nonzero(np.abs(zs - centre[2]) <= ext)[0]
    Z, Y, X = np.meshgrid(zs[iz] - centre[2], ys[iy] - centre[1], xs[ix] - centre[0], indexing="ij")
    acc = np.zeros(X.shape)
    for ox in offs:
        for oy in offs:
            for oz in offs:
                acc += ((X + ox * d) ** 2 + (Y + oy * d) ** 2 + (Z + oz * d) ** 2) <= radius * radius
    vol[np.ix_(iz, iy, ix)] = amp * acc / ss ** 3
    return vol


def random_data(geom: Geometry, seed=7, dtype=np.float32):
    """Seeded N(0, 1) data vector (adjoint tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(geom.data_shape).astype(dtype)


def random_volume(geom: Geometry, seed=11, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(geom.vol_shape).astype(dtype)


def eir_taps(fs_mhz=20.0, kind="gaussian", fwhm_us=0.5, centre_mhz=2.25, cycles=1.5):
    """Synthetic transducer-response taps h_m = dt h^e(m dt) and their first index m0.

    kind="gaussian": the temporal blur of the simulation studies (a Gaussian of FWHM `fwhm_us`,
    unit area), centred (no delay: its peak at m = -1, where the model's one-sample offset
    cancels).  kind="bandpass": a causal band-pass pulse, a Gaussian-windowed cosine of centre
    frequency `centre_mhz` with `cycles` cycles per standard deviation, zero mean, starting at
    m = 0 (a stand-in for a measured EIR)."""
    dt = 1.0 / fs_mhz
    if kind == "gaussian":
        sig = fwhm_us / (2.0 * np.sqrt(2.0 * np.log(2.0))) / dt       # samples
        half = int(np.ceil(4.0 * sig))
        m = np.arange(-half, half + 1)
        h = np.exp(-0.5 * (m / sig) ** 2)
        return h / h.sum(), -1 - half
    if kind == "bandpass":
        sig = cycles / centre_mhz / dt
        n = int(np.ceil(8.0 * sig)) + 1
        t = np.arange(n) - 4.0 * sig
        h = np.exp(-0.5 * (t / sig) ** 2) * np.cos(2.0 * np.pi * centre_mhz * dt * t)
        h -= h.mean() * np.exp(-0.5 * (t / sig) ** 2) / np.exp(-0.5 * (t / sig) ** 2).mean()
        return dt * h / np.abs(dt * h).sum(), 0
    raise ValueError(kind)


# ----------------------------------------------------------------------------- configurations

def _c1():
    return make_geometry(64, 0.2, 16, 16, 20.0, 256)


def _c2():
    return make_geometry(256, 0.2, 128, 180, 65.0, 1536)


def _c3():
    return make_geometry(160, 0.25, 96, 90, 50.0, 1024)


def _c3_grad():
    return make_geometry(32, 0.25, 8, 8, 50.0, 128)


def _c4():
    return make_geometry(128, 0.25, 32, 45, 50.0, 1024)


def _c5():
    return make_geometry(256, 0.2, 128, 60, 65.0, 1536)


def _tiny():
    # dense brute-force case: 6^3 nodes, 4 transducers, 24 samples
    return make_geometry(6, 0.5, 2, 2, 6.0, 24, fs_mhz=10.0, c=1.5)


def _small():
    # non-cubic, ragged sizes (not multiples of any tile), several radius-equal transducers
    return make_geometry((21, 18, 27), 0.3, 3, 5, 12.0, 120, fs_mhz=20.0, c=1.5)


CONFIGS = {
    "c1": _c1, "c2": _c2, "c3": _c3, "c3_grad": _c3_grad, "c4": _c4, "c5": _c5,
    "tiny": _tiny, "small": _small,
}

DESCRIPTIONS = {
    "c1": "64^3 @ 0.2 mm, 8 spheres, 16 rings x 16 views on 20 mm, K=256 @ 20 MHz, c=1.5",
    "c2": "256^3 @ 0.2 mm, 200 ellipsoids, 128 rings x 180 views on 65 mm, K=1536 @ 20 MHz, c=1.5",
    "c3": "160^3 @ 0.25 mm, 96 rings x 90 views on 50 mm, K=1024",
    "c3_grad": "32^3 @ 0.25 mm, 8 x 8 transducers on 50 mm, K=128",
    "c4": "128^3 @ 0.25 mm, 32 rings x 45 views on 50 mm, K=1024",
    "c5": "256^3 @ 0.2 mm, 128 rings x 60 views on 65 mm, K=1536, FP16/BF16 data",
}


def config(name: str) -> Geometry:
    return CONFIGS[name]()


SPH_DESCRIPTION = ("210 x 210 x 440 @ 0.14 mm, 9 spheres, 64 rings x 90 views on 65 mm, "
                   "511 frequencies in (0, 5] MHz, c=1.54")


def sph_config() -> Geometry:
    """The spherical-voxel workload: the grid of the paper's simulation studies (210 x 210 x 440
    nodes at 0.14 mm, Sec. IV), the 64 rings x 90 views subset of its spherical scan on 65 mm, and
    its speed of sound 1.54 mm/us.  The time-sampling fields are unused by that model."""
    return make_geometry((210, 210, 440), 0.14, 64, 90, 65.0, 16, c=1.54)


def phantom_sph(geom: Geometry, seed=1304):
    """Nine uniform spheres (the paper's simulation object has nine; their sizes and places are
    not given), point-sampled at the nodes."""
    return spheres_phantom(geom, n_spheres=9, seed=seed)


def phantom(name: str, geom: Geometry | None = None, seed=1304):
    """Phantom for a named configuration."""
    geom = geom or config(name)
    if name in ("c1", "tiny", "small", "c3_grad"):
        n = 8 if name != "tiny" else 2
        if name == "tiny":
            return spheres_phantom(geom, n_spheres=2, seed=seed, r_range=(0.4, 0.9))
        return spheres_phantom(geom, n_spheres=n, seed=seed)
    if name in ("c2", "c5"):
        return ellipsoids_phantom(geom, n=200, seed=seed)
    if name == "c3":
        return ellipsoids_phantom(geom, n=120, seed=seed)
    if name == "c4":
        return ellipsoids_phantom(geom, n=60, seed=seed)
    raise KeyError(name)
