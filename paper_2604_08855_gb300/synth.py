"""Seeded synthetic catalogues (numpy PCG64); no estimator arithmetic here.

These stand in for the paper's galaxy catalogues and simulation maps (its
"Features" section lists CFITSIO / HEALPix / GADGET-2 / ASCII readers for
data that is not available here).  Both the CUDA path and the FP64 oracle
consume exactly these arrays; this module holds only point generation, so
neither side borrows the other's arithmetic through it.

Workloads (sizes as the configurations name them):
  uniform      N points uniform in a periodic cube of side L.
  thomas       Thomas process: n_par parents uniform in the cube, each child
               picks a parent uniformly (multinomial, so N is exact) and adds
               an isotropic Gaussian offset of width sigma; wrapped
               periodically.
  sector       cut-sky shell sector (RA in [0, 60) deg, Dec in [-30, 30] deg,
               radius in [500, 1500]): clustered data plus uniform randoms.
  mock batch   many independent Thomas catalogues of log-uniform sizes.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# fixed-point grids
#
# Every generated coordinate is snapped onto a fine grid: the L / 2^32 grid of
# a periodic cube (L = 1000 and 2000 have short mantissas, so grid points are
# exact float64 values and x / L * 2^32 is an exact integer), or a dyadic grid
# for open space.  A bin decision then depends only on an exact squared
# separation, identical for every exact evaluation; the statistics are
# unchanged (the grid step is ~1e-7 of the box).


def snap_periodic(xyz, box: float):
    """Wrap into [0, box) and snap onto the box / 2^32 grid (exact for box = 1000, 2000)."""
    k = np.floor(np.mod(np.asarray(xyz, dtype=np.float64), box) / box * 4294967296.0)
    k = np.clip(k, 0.0, 4294967295.0)
    return k * (box / 4294967296.0)


def snap_dyadic(xyz, step: float = 2.0 ** -20):
    """Snap onto the grid of multiples of a power of two (open space)."""
    return np.round(np.asarray(xyz, dtype=np.float64) / step) * step


# ---------------------------------------------------------------------------
# primitive generators


def uniform(n: int, box: float, seed: int, weights: str = "unit", snap: bool = True):
    """N uniform points in a periodic cube; snap=False keeps the raw float64
    draws (off the fixed-point grid)."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, box, size=(n, 3))
    xyz = snap_periodic(xyz, box) if snap else xyz
    w = _weights(rng, n, weights)
    return xyz, w


def thomas(n: int, box: float, n_par: int, sigma: float, seed: int, weights: str = "unit", snap: bool = True):
    """Thomas process in a periodic cube, exactly n points; snap=False keeps
    the raw float64 values wrapped into [0, box) (off the fixed-point grid)."""
    rng = np.random.default_rng(seed)
    parents = rng.uniform(0.0, box, size=(n_par, 3))
    owner = rng.integers(0, n_par, size=n)
    xyz = parents[owner] + rng.normal(0.0, sigma, size=(n, 3))
    xyz = snap_periodic(xyz, box) if snap else np.mod(xyz, box)
    w = _weights(rng, n, weights)
    return xyz, w


def _weights(rng, n, kind):
    if kind == "unit":
        return np.ones(n)
    if kind == "u0.5-1.5":
        return rng.uniform(0.5, 1.5, size=n)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# cut-sky sector

SECTOR_RA = (0.0, np.deg2rad(60.0))
SECTOR_DEC = (np.deg2rad(-30.0), np.deg2rad(30.0))
SECTOR_R = (500.0, 1500.0)


def in_sector(xyz):
    r = np.sqrt(np.sum(xyz * xyz, axis=1))
    ra = np.arctan2(xyz[:, 1], xyz[:, 0])
    dec = np.arcsin(np.clip(xyz[:, 2] / np.maximum(r, 1e-300), -1.0, 1.0))
    return ((r >= SECTOR_R[0]) & (r <= SECTOR_R[1]) & (ra >= SECTOR_RA[0]) & (ra < SECTOR_RA[1])
            & (dec >= SECTOR_DEC[0]) & (dec <= SECTOR_DEC[1]))


def sector_randoms(n: int, seed: int, snap: bool = True):
    """Uniform in the sector volume: RA uniform, sin(Dec) uniform, r^3 uniform
    (snap=False: raw float64, off the dyadic grid)."""
    rng = np.random.default_rng(seed)
    ra = rng.uniform(SECTOR_RA[0], SECTOR_RA[1], size=n)
    sdec = rng.uniform(np.sin(SECTOR_DEC[0]), np.sin(SECTOR_DEC[1]), size=n)
    r3 = rng.uniform(SECTOR_R[0] ** 3, SECTOR_R[1] ** 3, size=n)
    r = np.cbrt(r3)
    cdec = np.sqrt(1.0 - sdec * sdec)
    xyz = np.stack([r * cdec * np.cos(ra), r * cdec * np.sin(ra), r * sdec], axis=1)
    return snap_dyadic(xyz) if snap else xyz


def sector_data(n: int, seed: int, sigma: float = 5.0, per_parent: float = 100.0, snap: bool = True):
    """Thomas process in the sector's bounding box (5 sigma margin), clipped to
    the sector, then exactly n points drawn without replacement."""
    rng = np.random.default_rng(seed)
    lo = np.array([SECTOR_R[0] * np.cos(SECTOR_DEC[1]) * np.cos(SECTOR_RA[1]), 0.0,
                   SECTOR_R[1] * np.sin(SECTOR_DEC[0])]) - 5 * sigma
    hi = np.array([SECTOR_R[1], SECTOR_R[1] * np.sin(SECTOR_RA[1]),
                   SECTOR_R[1] * np.sin(SECTOR_DEC[1])]) + 5 * sigma
    vol_box = float(np.prod(hi - lo))
    vol_sector = (SECTOR_RA[1] - SECTOR_RA[0]) * (np.sin(SECTOR_DEC[1]) - np.sin(SECTOR_DEC[0])) \
        * (SECTOR_R[1] ** 3 - SECTOR_R[0] ** 3) / 3.0
    total = int(np.ceil(1.15 * n * vol_box / vol_sector))
    while True:
        n_par = max(1, int(round(total / per_parent)))
        parents = rng.uniform(lo, hi, size=(n_par, 3))
        owner = rng.integers(0, n_par, size=total)
        xyz = parents[owner] + rng.normal(0.0, sigma, size=(total, 3))
        xyz = xyz[in_sector(xyz)]
        if xyz.shape[0] >= n:
            break
        total = int(total * 1.2)
    pick = rng.choice(xyz.shape[0], size=n, replace=False)
    xyz = xyz[np.sort(pick)]
    return snap_dyadic(xyz) if snap else xyz


# ---------------------------------------------------------------------------
# the named workloads


def config_params(k: int) -> dict:
    """Estimator parameters of workload k (1..5)."""
    return {
        1: dict(box=1000.0, rmin=10.0, rmax=100.0, nbins=10, lmax=10),
        2: dict(box=1000.0, rmin=5.0, rmax=200.0, nbins=20, lmax=10),
        3: dict(box=2000.0, rmin=10.0, rmax=200.0, nbins=32, lmax=20),
        4: dict(box=1000.0, rmin=10.0, rmax=150.0, nbins=20, lmax=10),
        5: dict(box=0.0, rmin=20.0, rmax=200.0, nbins=36, lmax=10),
    }[k]


def uniform_20k():
    """20,000 uniform points, L = 1000, unit weights, seed 0."""
    return uniform(20_000, 1000.0, seed=0)


def thomas_1m():
    """1,000,000 Thomas points, L = 1000, 10,000 parents (density 1e-5),
    sigma = 5, weights U[0.5, 1.5], seed 1."""
    return thomas(1_000_000, 1000.0, 10_000, 5.0, seed=1, weights="u0.5-1.5")


def thomas_4m():
    """4,000,000 Thomas points, L = 2000, 40,000 parents (about 100 children
    each), sigma = 5, weights U[0.5, 1.5], seed 2."""
    return thomas(4_000_000, 2000.0, 40_000, 5.0, seed=2, weights="u0.5-1.5")


def thomas_4m_subset(n: int = 200_000):
    """The seeded 200k subset of the 4M catalogue (rng(102), no replacement)."""
    xyz, w = thomas_4m()
    pick = np.sort(np.random.default_rng(102).choice(xyz.shape[0], size=n, replace=False))
    return xyz[pick], w[pick]


def mock_sizes(k: int = 256, seed: int = 4000):
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(5e4), np.log(2e6), size=k))).astype(np.int64)


def mock_catalogue(i: int, n: int):
    """Catalogue i of the mock batch: Thomas, L = 1000, n/100 parents, w = 1."""
    return thomas(int(n), 1000.0, max(1, int(round(n / 100))), 5.0, seed=4001 + i)


def cut_sky(n_data: int = 8_000_000, n_rand: int = 24_000_000):
    """Sector data (w = +1, seed 5) followed by randoms (w = -n_data/n_rand, seed 6)."""
    d = sector_data(n_data, seed=5)
    r = sector_randoms(n_rand, seed=6)
    xyz = np.concatenate([d, r], axis=0)
    w = np.concatenate([np.ones(n_data), np.full(n_rand, -n_data / n_rand)])
    return xyz, w


def sample_primaries(n: int, k: int, seed: int = 7):
    """k distinct primary indices out of n, seeded, sorted."""
    k = min(k, n)
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False)).astype(np.int64)


# ---------------------------------------------------------------------------
# the unit sphere (projected fields)


def fibonacci_sphere(n: int) -> np.ndarray:
    """n directions on the golden-angle spiral: equal-area and near-uniform,
    standing in for the pixel centres of a HEALPix map with n pixels.
    Snapped to the 2^-20 dyadic grid (so not exactly unit length)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = k * (np.pi * (3.0 - np.sqrt(5.0)))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return snap_dyadic(np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1))


def sphere_cap(n: int, seed: int, theta_cap: float = 0.3, centre=(0.2, -0.3, 0.93), snap: bool = True) -> np.ndarray:
    """n random directions uniform in a spherical cap (snapped to 2^-20, or
    exact unit vectors with snap=False)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, dtype=np.float64)
    c /= np.linalg.norm(c)
    mu = rng.uniform(np.cos(theta_cap), 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(1.0 - mu * mu)
    local = np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, c)
    sn, cs = np.linalg.norm(v), float(z @ c)
    if sn > 1e-12:
        k = v / sn
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        local = local @ (np.eye(3) + sn * K + (1 - cs) * K @ K).T
    return snap_dyadic(local) if snap else local / np.linalg.norm(local, axis=1, keepdims=True)


def sphere_field(xyz: np.ndarray, seed: int, nblobs: int = 64, width: float = 0.05, noise: float = 0.1):
    """A smooth random scalar field at the given directions (a stand-in for a
    convergence map): von Mises blobs of random sign and amplitude plus white
    noise.  These are the weights of the projected estimator."""
    rng = np.random.default_rng(seed)
    cen = rng.normal(size=(nblobs, 3))
    cen /= np.linalg.norm(cen, axis=1)[:, None]
    amp = rng.normal(size=nblobs)
    kappa = 1.0 / (width * width)
    f = np.zeros(xyz.shape[0])
    for i0 in range(0, xyz.shape[0], 1 << 20):
        x = xyz[i0:i0 + (1 << 20)]
        f[i0:i0 + x.shape[0]] = np.exp(kappa * (x @ cen.T - 1.0)) @ amp
    return f + noise * rng.normal(size=xyz.shape[0])


def sphere_map(nside: int, seed: int = 11):
    """A full-sky map with 12 nside^2 pixels (Fibonacci directions) and a
    smooth random field as pixel values."""
    xyz = fibonacci_sphere(12 * nside * nside)
    return xyz, sphere_field(xyz, seed)
