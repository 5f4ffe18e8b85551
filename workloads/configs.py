"""The synthetic workloads: unit-cell mesh, lattice, wavenumbers and incident
directions of the five benchmark configurations.

Sizes, spacings and frequencies are the ones of the paper's kinds of workload
(sphere arrays of the scattering study, a cylinder sonic-crystal barrier, a
3-D lattice of cubes, a mixed request stream).  Speed of sound c = 343 m/s as
in the numerical examples of the paper.
"""
from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np

from .meshes import icosphere, capped_cylinder, cube, open_cylinder, quad9_sphere

SPEED_OF_SOUND = 343.0


@dataclass
class Workload:
    name: str
    make_mesh: Callable[[], Tuple[np.ndarray, np.ndarray]]
    counts: Tuple[int, int, int]           # cells along the lattice vectors
    lattice: np.ndarray                    # 3x3, row i = lattice vector i (metres)
    wavenumbers: List[float]               # k = 2 pi f / c
    directions: np.ndarray                 # R x 3 unit incidence directions
    rhs_seed: int                          # PCG32 seed of the random test vectors
    pbem_form: bool = False                # every offset dense (cells too tall for the FMM)
    n_t: int = 0                           # truncation number (0 = not an FMM workload)
    notes: str = ""
    plane: tuple = None                    # (axis, offset, R_p) of a half-space workload
    monopoles: tuple = ()                  # ((x, y, z), amplitude at 1 m) incident monopoles

    @property
    def dim(self) -> int:
        return sum(1 for m in self.counts if m > 1) or 1

    def mesh(self):
        return self.make_mesh()


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors spread uniformly over the sphere (spherical Fibonacci
    lattice: z_i = 1 - (2 i + 1)/n, golden-angle longitude)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    ga = np.pi * (3.0 - np.sqrt(5.0))
    rho = np.sqrt(1.0 - z * z)
    return np.stack([rho * np.cos(ga * i), rho * np.sin(ga * i), z], axis=1)


def _freqs_to_k(freqs):
    return [2.0 * np.pi * f / SPEED_OF_SOUND for f in freqs]


_SEED = 220112050

WORKLOADS = {
    "sphere_row_4": Workload(
        name="sphere_row_4",
        make_mesh=lambda: icosphere(2, 0.2),
        counts=(4, 1, 1),
        lattice=np.diag([1.0, 1.0, 1.0]),
        wavenumbers=[2.0],
        directions=np.array([[1.0, 0.0, 0.0]]),
        rhs_seed=_SEED + 0,
        n_t=6,
        notes="1-D row of 4 rigid spheres r=0.2 m, lattice 1.0 m, 320 triangles per cell, N=1,280, k=2",
    ),
    "sonic_crystal_3x20": Workload(
        name="sonic_crystal_3x20",
        make_mesh=lambda: capped_cylinder(0.15, 3.0, 20, 29),
        counts=(3, 20, 1),
        lattice=np.diag([0.4, 0.4, 3.0]),
        wavenumbers=_freqs_to_k([100.0 * i for i in range(1, 11)]),
        directions=np.array([[np.cos(np.pi / 6), np.sin(np.pi / 6), 0.0]]),
        rhs_seed=_SEED + 1,
        pbem_form=True,
        notes="3x20 rigid capped cylinders r=0.15 m h=3.0 m, square lattice 0.4 m, 1,200 triangles per cell, N=72,000",
    ),
    "sphere_array_32x32": Workload(
        name="sphere_array_32x32",
        make_mesh=lambda: icosphere(2, 0.2),
        counts=(32, 32, 1),
        lattice=np.diag([0.6, 0.6, 1.0]),
        wavenumbers=[4.0],
        directions=np.array([[1.0, 0.0, 0.0]]),
        rhs_seed=_SEED + 2,
        n_t=8,
        notes="32x32 rigid spheres r=0.2 m, lattice 0.6 m, 320 triangles per cell, N=327,680, k=4",
    ),
    "cube_lattice_16x16x4": Workload(
        name="cube_lattice_16x16x4",
        make_mesh=lambda: cube(0.3, 6),
        counts=(16, 16, 4),
        lattice=np.diag([0.5, 0.5, 0.5]),
        wavenumbers=_freqs_to_k([200.0 * i for i in range(1, 9)]),
        directions=fibonacci_directions(64),
        rhs_seed=_SEED + 3,
        n_t=12,
        notes="16x16x4 rigid cubes edge 0.3 m in 0.5 m cells, 432 triangles per cell, N=442,368",
    ),
    # large unit cells (the h-refinement study of the sphere array): 5 x 10
    # spheres of 5,120 triangles each, for the multilevel near field (FMPBEM2)
    "sphere_array_5x10_fine": Workload(
        name="sphere_array_5x10_fine",
        make_mesh=lambda: icosphere(4, 0.2),
        counts=(5, 10, 1),
        lattice=np.diag([0.6, 0.6, 1.0]),
        wavenumbers=[4.0],
        directions=np.array([[1.0, 0.0, 0.0]]),
        rhs_seed=_SEED + 6,
        n_t=8,
        notes="5x10 rigid spheres r=0.2 m, lattice 0.6 m, 5,120 triangles per cell, N=256,000, k=4",
    ),
    # the paper's first scattering example on its own element family: 5 x 5
    # rigid spheres r = 0.1 m at 0.35 m, each of 600 nine-node quadratic
    # quadrilaterals (40 over the circumference), N = 15,000, 500 Hz, plane
    # wave along x
    "sphere_array_5x5_q9": Workload(
        name="sphere_array_5x5_q9",
        make_mesh=lambda: quad9_sphere(10, 0.1),
        counts=(5, 5, 1),
        lattice=np.diag([0.35, 0.35, 1.0]),
        wavenumbers=_freqs_to_k([100.0, 500.0]),
        directions=np.array([[1.0, 0.0, 0.0]]),
        rhs_seed=_SEED + 7,
        pbem_form=True,
        notes="5x5 rigid spheres r=0.1 m, lattice 0.35 m, 600 nine-node quadrilaterals per cell, N=15,000",
    ),
    # the cylinder sound barrier of the paper's barrier study: 3 x 25 rigid
    # cylinders r = 0.1 m, 2 m high, on a sound-hard ground, as cells of
    # 0.4 m stacked 5 high (the z axis is perpendicular to the ground: block
    # Hankel image part); two monopoles 1 m above the ground
    "barrier_cylinders_3x25x5": Workload(
        name="barrier_cylinders_3x25x5",
        make_mesh=lambda: open_cylinder(0.1, 0.4, 12, 14),
        counts=(3, 25, 5),
        lattice=np.diag([0.4, 0.4, 0.4]),
        wavenumbers=_freqs_to_k([100.0, 200.0, 300.0, 428.75, 500.0]),
        directions=np.array([[1.0, 0.0, 0.0]]),
        rhs_seed=_SEED + 5,
        n_t=10,
        notes="3x25x5 cells of open cylinder segments r=0.1 m h=0.4 m, lattice 0.4 m, ground z=0 (R_p=1), "
              "336 triangles per cell, N=126,000",
        plane=(2, -0.2, 1.0),
        monopoles=(((-4.0, 6.5, 0.8), 2.0), ((-4.0, 3.5, 0.8), 1.0)),
    ),
}


def serving_stream(n_requests: int, seed: int = _SEED + 4, rate_hz: float = 50.0):
    """Seeded request stream of the serving workload: Poisson arrivals at
    rate_hz, cell grids uniform from 4x4 to 64x8 of the capped-cylinder cell
    or the sphere cell, frequencies uniform in 100-2000 Hz, 1-16 incident
    plane waves with directions uniform on the sphere.  Returns a list of dicts
    (arrival time s, cell name, counts, lattice, k, directions)."""
    from .rng import PCG32
    g = PCG32(seed)
    u = lambda: g.uniform(1)[0]
    out, t = [], 0.0
    for _ in range(n_requests):
        t += -np.log(1.0 - u()) / rate_hz
        cell = "cylinder" if u() < 0.5 else "sphere"
        mx = 4 + int(u() * 61)
        my = 4 + int(u() * 5)
        f = 100.0 + 1900.0 * u()
        R = 1 + int(u() * 16)
        z = 2.0 * g.uniform(R) - 1.0
        ph = 2.0 * np.pi * g.uniform(R)
        rho = np.sqrt(1.0 - z * z)
        dirs = np.stack([rho * np.cos(ph), rho * np.sin(ph), z], axis=1)
        lattice = np.diag([0.4, 0.4, 3.0]) if cell == "cylinder" else np.diag([1.0, 1.0, 1.0])
        out.append({"t": t, "cell": cell, "counts": (mx, my, 1), "lattice": lattice,
                    "k": 2.0 * np.pi * f / SPEED_OF_SOUND, "freq_hz": f, "dirs": dirs})
    return out
