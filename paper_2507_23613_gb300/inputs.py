"""Seeded synthetic workloads for MFWH: grids, frequencies and Gaussian sources.

This module only draws inputs; it holds none of the method's arithmetic and is
shared by the tests, the benchmark and the oracle comparisons.  Sources follow
the paper's Gaussian form f = A exp(-b ||x - x0||^2) (eq. gaussianSource, with
b standing for b_g^2), centres drawn uniformly in [0.2, 0.8]^d, frequencies
drawn uniformly in a band, sorted, with adjacent gaps of at least `min_gap`.
Random numbers come from numpy's PCG64 seeded with `seed`.
"""

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n: tuple                 # cells per axis, x first
    length: tuple            # domain extent per axis, x first
    omega: np.ndarray        # (N_f,) increasing
    forcing: np.ndarray      # (N_f, *shape), float64, x fastest
    c2: object = 1.0         # scalar c^2, or a grid array for a layered medium
    cfl: float = 0.5
    n_p: int = 1
    layer: dict = field(default_factory=dict)   # two-layer description, if any

    @property
    def shape(self):
        return tuple(k + 1 for k in reversed(self.n))

    @property
    def nf(self):
        return int(self.omega.size)

    @property
    def points(self):
        return int(np.prod(self.shape))

    @property
    def interior_points(self):
        return int(np.prod([k - 1 for k in self.n]))


def coordinates(n, length):
    """Coordinate arrays x, y[, z] at the grid points, each shaped like the grid (x fastest)."""
    axes = [np.arange(k + 1) * (L / k) for k, L in zip(n, length)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return tuple(reversed(mesh))


def gaussian(coords, centre, amplitude, b):
    r2 = np.zeros_like(coords[0])
    for x, x0 in zip(coords, centre):
        r2 += (x - x0) ** 2
    return amplitude * np.exp(-b * r2)


def draw_frequencies(rng, nf, lo, hi, min_gap=1.0, max_tries=10000):
    for _ in range(max_tries):
        om = np.sort(rng.uniform(lo, hi, size=nf))
        if nf == 1 or np.min(np.diff(om)) >= min_gap:
            return om
    raise RuntimeError("could not draw separated frequencies")


def gaussian_workload(name, n, nf, omega, b, seed, amplitude=1.0, sources_per_freq=1,
                      length=None, c2=1.0, cfl=0.5, n_p=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    length = tuple(length or (1.0,) * len(n))
    coords = coordinates(n, length)
    shape = tuple(k + 1 for k in reversed(n))
    if callable(omega):
        omega = omega(rng)
    omega = np.asarray(omega, dtype=np.float64)
    forcing = np.zeros((omega.size,) + shape)
    for m in range(omega.size):
        for _ in range(sources_per_freq):
            centre = rng.uniform(0.2, 0.8, size=len(n)) * np.asarray(length)
            forcing[m] += gaussian(coords, centre, amplitude, b)
    return Workload(name, tuple(n), length, omega, forcing, c2, cfl, n_p)


def random_filter_params(seed, nf):
    """Seeded filter parameters (a, c, s) near the traditional (-1/4, 1, 0): inputs for
    runs that prescribe the filter instead of optimising it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.array([-0.25, 1.0, 0.0])
    return base + rng.uniform(-0.2, 0.2, size=(nf, 3))


def square_small(seed=1000):
    """65^2 unit square, c = 1, N_f = 2 (omega = 5.5, 9.3), Gaussians A = 1, b = 200, CFL 0.5."""
    return gaussian_workload("square65_nf2", (64, 64), 2, [5.5, 9.3], 200.0, seed)


def square_large(seed=2000, n=1024, nf=8, n_p=2):
    """1025^2 unit square, c = 1, N_f = 8 frequencies uniform in [10, 60], Gaussians b = 400,
    CFL 0.5, N_p = 2 (integration over two periods of the longest period)."""
    return gaussian_workload(f"square{n + 1}_nf{nf}", (n, n), nf,
                             lambda r: draw_frequencies(r, nf, 10.0, 60.0), 400.0, seed, n_p=n_p)


def two_layer_c2(n, length, c_lo, c_hi, z_interface):
    """c^2 on the grid: c_lo below the plane z = z_interface, c_hi at and above it (z the last axis)."""
    coords = coordinates(n, length)
    z = coords[-1]
    return np.where(z < z_interface, c_lo * c_lo, c_hi * c_hi)


def random_c2(n, seed, c_lo=1.0, c_hi=1.5):
    """Seeded c^2 field on the grid of n cells per axis: c drawn uniformly in [c_lo, c_hi]
    independently at every grid point (a rough medium for the MFWH_C_FIELD mode)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(k + 1 for k in reversed(n))
    c = rng.uniform(c_lo, c_hi, size=shape)
    return c * c


def cube_layered(seed=3000, n=256, nf=4):
    """257^3 unit cube, c = 1.0 / 1.5 split at z = 0.5, N_f = 4 in [8, 30], Gaussians b = 300, CFL 0.5."""
    dims = (n, n, n)
    c2 = two_layer_c2(dims, (1.0, 1.0, 1.0), 1.0, 1.5, 0.5)
    wl = gaussian_workload(f"cube{n + 1}_nf{nf}", dims, nf,
                           lambda r: draw_frequencies(r, nf, 8.0, 30.0), 300.0, seed, c2=c2)
    wl.layer = {"c_lo": 1.0, "c_hi": 1.5, "interface": 0.5, "axis": 2}
    return wl


BATCH_SIZES = (256, 512, 1024, 2048)


def batch_workload(seed):
    """One problem of the batched workload: a 2D unit square with a size drawn from
    {257^2, 513^2, 1025^2, 2049^2}, N_f drawn in 1..16, frequencies uniform in [5, 80]
    (adjacent gaps >= 1.5), 1-4 Gaussian sources per frequency with b uniform in
    [200, 400], c = 1, CFL 0.5, N_p = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.choice(BATCH_SIZES))
    nf = int(rng.integers(1, 17))
    omega = draw_frequencies(rng, nf, 5.0, 80.0, min_gap=1.5)
    b = float(rng.uniform(200.0, 400.0))
    k = int(rng.integers(1, 5))
    return gaussian_workload(f"batch{seed}_n{n + 1}_nf{nf}", (n, n), nf, omega, b,
                             int(rng.integers(0, 2**31)), sources_per_freq=k)


def paper_three_frequency(n=128):
    """The paper's explicit three-frequency example (eq. Nf3parameters): unit square with
    n x n cells, omega = {5.1, 10.1, 15.1}, Gaussians f_m = a_m exp(-b_m^2 ||x - x0_m||^2)
    with a = {25, 100, 225}, b = 15 and centres (0.6, 0.45), (0.4, 0.5), (0.55, 0.5)
    (eq. gaussianSource), N_p = 2."""
    dims = (n, n)
    coords = coordinates(dims, (1.0, 1.0))
    omega = np.array([5.1, 10.1, 15.1])
    amps = (25.0, 100.0, 225.0)
    centres = ((0.6, 0.45), (0.4, 0.5), (0.55, 0.5))
    forcing = np.stack([gaussian(coords, c, a, 15.0 ** 2) for a, c in zip(amps, centres)])
    return Workload(f"paper3freq_square{n}", dims, (1.0, 1.0), omega, forcing, 1.0, 0.5, 2)


def paper_three_frequency_cube(n=64):
    """A 3D analogue of the paper's three-frequency example: unit cube with n^3 cells, the same
    omega, amplitudes, width b = 15 and N_p = 2, the centres of eq. Nf3parameters extended by
    z = 0.5."""
    dims = (n, n, n)
    coords = coordinates(dims, (1.0, 1.0, 1.0))
    omega = np.array([5.1, 10.1, 15.1])
    amps = (25.0, 100.0, 225.0)
    centres = ((0.6, 0.45, 0.5), (0.4, 0.5, 0.5), (0.55, 0.5, 0.5))
    forcing = np.stack([gaussian(coords, c, a, 15.0 ** 2) for a, c in zip(amps, centres)])
    return Workload(f"paper3freq_cube{n}", dims, (1.0, 1.0, 1.0), omega, forcing, 1.0, 0.5, 2)


def warm_start_workload(seed, n=128, nf=6):
    """One problem of the learned-warm-start workload: unit square with n x n cells, N_f
    frequencies uniform in [15, 45] (adjacent gaps >= 1.5), 1-4 Gaussian sources per frequency
    with b uniform in [200, 400], c = 1, CFL 0.5, N_p = 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    omega = draw_frequencies(rng, nf, 15.0, 45.0, min_gap=1.5)
    b = float(rng.uniform(200.0, 400.0))
    k = int(rng.integers(1, 5))
    wl = gaussian_workload(f"ws{seed}_n{n + 1}_nf{nf}", (n, n), nf, omega, b,
                           int(rng.integers(0, 2**31)), sources_per_freq=k)
    wl.n_p = 2
    return wl
