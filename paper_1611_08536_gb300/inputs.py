"""Seeded synthetic inputs for the DRTS time step.

This module holds no arithmetic of the method: it only writes down problem
descriptions (grid, media table, medium map, boundary mode, detector patch
grid) and source terms (state indices, weights, time profiles).  Both the CUDA
path and the FP64 oracle consume what it returns.

State indexing (Eq. 22): voxel v = (z*ny + y)*nx + x, lattice direction d
enumerates {-1,0,1}^3 minus the origin with dz slowest and dx fastest, and
state s = v*26 + d.

Workloads (all synthetic; the paper publishes no dataset):
  * ``fresnel_cube``   homogeneous cube, Fresnel boundary to vacuum, delta
                       pulse at the centre of the z=0 face along +z.
  * ``three_layers``   three planar layers along z (1/2/9 thickness ratio)
                       with refraction at the interfaces, Gaussian pulse.
  * ``inclusions``     homogeneous cube with seed-placed spherical
                       absorbing inclusions, many surface pulse sources.
  * ``ellipsoids``     voxelised medium with seed-placed ellipsoidal
                       inclusions of differing optical properties.
  * ``served_request`` one request of a served stream (side, medium, steps,
                       sources drawn from a seeded generator).
  * ``load_config``    one of the JSON problem files in ``configs/`` (the five
                       benchmark configurations: generator, arguments, seeds,
                       precision, steps).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

import numpy as np

OPEN, MIRROR, FRESNEL = 0, 1, 2
FP64, FP32, FP16_ROWSCALE = 0, 1, 2
FACE_MX, FACE_PX, FACE_MY, FACE_PY, FACE_MZ, FACE_PZ = range(6)
NDIR = 26


def direction_index(dx: int, dy: int, dz: int) -> int:
    """Index of the lattice direction (dx, dy, dz) in the state enumeration."""
    if (dx, dy, dz) == (0, 0, 0) or max(abs(dx), abs(dy), abs(dz)) > 1:
        raise ValueError("not a lattice direction")
    q = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    return q if q < 13 else q - 1


def direction_vector(d: int):
    q = d if d < 13 else d + 1
    return (q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1)


# weights of the outgoing directions in the discrete Henyey-Greenstein
# kernel: every lattice direction alike, or each by its quadrature weight
HG_EQUAL, HG_QUADRATURE = 0, 1

# interface treatment (Section 4.2): per-contribution first-order folding, or
# the two-step crossing of planar interfaces (layered media only)
INTERFACE_FIRST_ORDER, INTERFACE_TWO_STEP = 0, 1


@dataclasses.dataclass
class Problem:
    shape: tuple                   # (nx, ny, nz)
    voxel_mm: float
    media: list                    # [(mu_s 1/mm, mu_a 1/mm, g, n)]
    medium_of_voxel: np.ndarray    # uint8, [nz][ny][nx] (x fastest)
    n_outside: float = 1.0
    boundary: int = FRESNEL
    precision: int = FP32
    n_rhs: int = 1
    det_face: int = FACE_PZ
    det_nu: int = 16
    det_nv: int = 16
    name: str = ""
    batched_kernel: int = 0        # 0 CUDA cores, 1 tensor cores (n_rhs > 1)
    interface: int = 0             # INTERFACE_FIRST_ORDER or INTERFACE_TWO_STEP (layered media)
    direction_weights: int = 0     # HG_EQUAL or HG_QUADRATURE (weights of the HG kernel's directions)

    @property
    def n_voxels(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def n_states(self) -> int:
        return self.n_voxels * NDIR

    def state(self, x: int, y: int, z: int, d: int) -> int:
        nx, ny, _ = self.shape
        return ((z * ny + y) * nx + x) * NDIR + d


@dataclasses.dataclass
class Source:
    """s(t) = sum_e weight[e] * profile[t - t0] * e_{state[e]} (Eq. 26)."""
    state: np.ndarray              # int64 canonical state indices
    weight: np.ndarray             # float64
    t0: int
    profile: np.ndarray            # float64, P(t0 .. t0+len-1)

    def as_tuple(self):
        return (self.state, self.weight, self.t0, self.profile)


def delta_profile() -> np.ndarray:
    return np.ones(1, np.float64)


def gaussian_profile(fwhm_steps: float) -> tuple:
    """Gaussian pulse centred at 2*FWHM, truncated at +-3*FWHM, sum 1.
    Returns (t0, profile)."""
    centre = 2.0 * fwhm_steps
    half = int(math.floor(3.0 * fwhm_steps))
    t = np.arange(int(round(centre)) - half, int(round(centre)) + half + 1)
    t = t[t >= 0]
    p = np.exp(-4.0 * math.log(2.0) * (t - centre) ** 2 / fwhm_steps ** 2)
    return int(t[0]), p / p.sum()


def homogeneous(n: int, voxel_mm: float, medium, boundary=FRESNEL,
                n_outside=1.0, precision=FP32, det=(FACE_PZ, 16, 16), name=""):
    shape = (n, n, n)
    mov = np.zeros((n, n, n), np.uint8)
    return Problem(shape, voxel_mm, [tuple(medium)], mov, n_outside, boundary,
                   precision, 1, det[0], min(det[1], n), min(det[2], n), name)


def fresnel_cube(n: int = 16, precision=FP64):
    """Homogeneous cube, voxel 0.1 mm, mu_s=10, mu_a=0.01 /mm, g=0.9, n=1.4 in
    vacuum; delta pulse at the centre of the z=0 face along +z."""
    prob = homogeneous(n, 0.1, (10.0, 0.01, 0.9, 1.4), FRESNEL, 1.0, precision,
                       name=f"fresnel_cube_{n}")
    src = Source(np.array([prob.state(n // 2, n // 2, 0, direction_index(0, 0, 1))],
                          np.int64), np.ones(1), 0, delta_profile())
    return prob, src


def three_layers(n: int = 128, precision=FP32, fwhm_steps=3.0):
    """Three planar layers along z (thickness 1:2:9 over 12 mm), mu_s 20/10/5,
    mu_a 0.02/0.005/0.01 /mm, g 0.9/0.85/0.9, n 1.45/1.44/1.37, Fresnel to
    vacuum, Gaussian pulse (FWHM 3 steps) at the centre of z=0 along +z,
    16x16 detector patches on the z=n-1 face."""
    media = [(20.0, 0.02, 0.90, 1.45), (10.0, 0.005, 0.85, 1.44),
             (5.0, 0.01, 0.90, 1.37)]
    z1 = int(round(n * 1.0 / 12.0))
    z2 = int(round(n * 3.0 / 12.0))
    mov = np.empty((n, n, n), np.uint8)
    mov[:z1] = 0
    mov[z1:z2] = 1
    mov[z2:] = 2
    prob = Problem((n, n, n), 12.0 / n, media, mov, 1.0, FRESNEL, precision, 1,
                   FACE_PZ, min(16, n), min(16, n), f"three_layers_{n}")
    t0, prof = gaussian_profile(fwhm_steps)
    src = Source(np.array([prob.state(n // 2, n // 2, 0, direction_index(0, 0, 1))],
                          np.int64), np.ones(1), t0, prof)
    return prob, src


def _inward_directions(face):
    axis, high = face // 2, face % 2
    out = []
    for d in range(NDIR):
        v = direction_vector(d)
        if (v[axis] < 0) if high else (v[axis] > 0):
            out.append(d)
    return out


def surface_sources(prob: Problem, n_sources: int, seed: int, t0=0, profile=None):
    """One pulse source per right-hand side at a seed-random surface voxel and
    a seed-random lattice direction pointing into the medium."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = prob.shape
    N = (nx, ny, nz)
    srcs = []
    for _ in range(n_sources):
        face = int(rng.integers(0, 6))
        axis, high = face // 2, face % 2
        c = [int(rng.integers(0, N[a])) for a in range(3)]
        c[axis] = N[axis] - 1 if high else 0
        dirs = _inward_directions(face)
        d = dirs[int(rng.integers(0, len(dirs)))]
        srcs.append(Source(np.array([prob.state(c[0], c[1], c[2], d)], np.int64),
                           np.ones(1), t0,
                           delta_profile() if profile is None else profile))
    return srcs


def inclusions(n: int = 96, n_rhs: int = 64, seed: int = 3, precision=FP32,
               n_spheres: int = 4):
    """Homogeneous cube (mu_s=10, mu_a=0.01 /mm, g=0.9, n=1.4, voxel 0.1 mm)
    with seed-placed spheres of radius 4-10 voxels whose mu_a is 10x; one
    delta source per right-hand side at seed-random surface positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    media = [(10.0, 0.01, 0.9, 1.4), (10.0, 0.1, 0.9, 1.4)]
    mov = np.zeros((n, n, n), np.uint8)
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    rmax = max(1, min(10, n // 4))
    rmin = max(1, min(4, rmax))
    for _ in range(n_spheres):
        r = int(rng.integers(rmin, rmax + 1))
        c = [int(rng.integers(r, max(r + 1, n - r))) for _ in range(3)]
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        mov[inside] = 1
    prob = Problem((n, n, n), 0.1, media, mov, 1.0, FRESNEL, precision, n_rhs,
                   FACE_PZ, min(16, n), min(16, n), f"inclusions_{n}_r{n_rhs}")
    srcs = surface_sources(prob, n_rhs, seed + 1000)
    return prob, srcs


def ellipsoids(n: int = 192, n_ell: int = 12, seed: int = 5, precision=FP32,
               fwhm_steps=3.0):
    """Voxelised medium (background mu_s=10, mu_a=0.01, g=0.9, n=1.4, voxel
    0.1 mm) with seed-placed axis-aligned ellipsoids of differing mu_s, mu_a,
    g and n; Gaussian pulse at the centre of z=0; full exit-face readout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    media = [(10.0, 0.01, 0.9, 1.4)]
    mov = np.zeros((n, n, n), np.uint8)
    ax = np.arange(n)
    for e in range(n_ell):
        mu_s = float(rng.uniform(5.0, 30.0))
        mu_a = float(10 ** rng.uniform(math.log10(0.002), math.log10(0.05)))
        g = float(rng.uniform(0.7, 0.95))
        nr = float(np.round(rng.uniform(1.33, 1.5), 3))
        media.append((mu_s, mu_a, g, nr))
        semi = [max(1, int(rng.integers(max(1, n // 24), max(2, n // 6) + 1)))
                for _ in range(3)]
        c = [int(rng.integers(0, n)) for _ in range(3)]
        dz = ((ax - c[2]) / semi[2]) ** 2
        dy = ((ax - c[1]) / semi[1]) ** 2
        dx = ((ax - c[0]) / semi[0]) ** 2
        inside = dz[:, None, None] + dy[None, :, None] + dx[None, None, :] <= 1.0
        mov[inside] = e + 1
    prob = Problem((n, n, n), 0.1, media, mov, 1.0, FRESNEL, precision, 1,
                   FACE_PZ, n, n, f"ellipsoids_{n}")
    t0, prof = gaussian_profile(fwhm_steps)
    src = Source(np.array([prob.state(n // 2, n // 2, 0, direction_index(0, 0, 1))],
                          np.int64), np.ones(1), t0, prof)
    return prob, src


SERVED_SIDES = (32, 48, 64, 80, 96)


@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: Problem
    sources: list
    n_steps: int


def served_request(seed: int, index: int, sides=SERVED_SIDES,
                   steps=(500, 3000), max_sources=16) -> Request:
    """One simulation request: cube side from ``sides``, layered or inclusion
    medium (mu_s U[1,30], mu_a logU[0.001,0.1], g U[0.7,0.95], n U[1.33,1.5]),
    steps U[steps], 1..max_sources pulse sources as right-hand sides."""
    rng = np.random.Generator(np.random.PCG64([seed, index]))
    n = int(sides[int(rng.integers(0, len(sides)))])

    def rand_medium():
        return (float(rng.uniform(1.0, 30.0)),
                float(10 ** rng.uniform(-3.0, -1.0)),
                float(rng.uniform(0.7, 0.95)),
                float(np.round(rng.uniform(1.33, 1.5), 3)))

    mov = np.zeros((n, n, n), np.uint8)
    if rng.uniform() < 0.5:
        n_layers = int(rng.integers(2, 4))
        media = [rand_medium() for _ in range(n_layers)]
        cuts = np.sort(rng.choice(np.arange(1, n), n_layers - 1, replace=False))
        for li, c in enumerate(cuts):
            mov[c:] = li + 1
    else:
        media = [rand_medium(), rand_medium()]
        ax = np.arange(n)
        for _ in range(int(rng.integers(1, 4))):
            r = int(rng.integers(max(2, n // 16), max(3, n // 5) + 1))
            c = [int(rng.integers(0, n)) for _ in range(3)]
            d2 = ((ax - c[2]) ** 2)[:, None, None] + ((ax - c[1]) ** 2)[None, :, None] \
                + ((ax - c[0]) ** 2)[None, None, :]
            mov[d2 <= r * r] = 1
    n_src = int(rng.integers(1, max_sources + 1))
    prob = Problem((n, n, n), 0.1, media, mov, 1.0, FRESNEL, FP32, n_src,
                   FACE_PZ, min(16, n), min(16, n), f"request_{index}_n{n}")
    srcs = surface_sources(prob, n_src, int(rng.integers(0, 2 ** 31)))
    n_steps = int(rng.integers(steps[0], steps[1] + 1))
    return Request(0.0, prob, srcs, n_steps)


def served_stream(n_requests: int = 1000, rate_per_s: float = 50.0, seed: int = 4,
                  **kw):
    """Poisson arrivals at ``rate_per_s``; request i from ``served_request``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    arrivals = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        r = served_request(seed, i, **kw)
        r.arrival_s = float(arrivals[i])
        out.append(r)
    return out


# ---------------------------------------------------------------------------
# JSON problem files (paper_1611_08536_gb300/configs/*.json): a named
# workload = one of the seeded generators above, its arguments, the
# precision and the step count.  The generators are the only place a
# workload is built, so a config file and the generator call give the same
# problem.

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
_PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP16_ROWSCALE}


@dataclasses.dataclass
class Config:
    name: str
    spec: dict                     # the file's content
    problem: Problem = None        # None for a served stream
    sources: list = None           # Source per right-hand side
    requests: list = None          # served stream: Request list
    steps: int = 0


def config_names():
    """Names of the JSON problem files shipped with the package."""
    return sorted(f[:-5] for f in os.listdir(CONFIG_DIR) if f.endswith(".json"))


def load_config(name_or_path: str, precision: str = None) -> Config:
    """Build the workload a JSON problem file names (a path, or the name of a
    file in ``CONFIG_DIR``).  ``precision`` overrides the file's ("fp64",
    "fp32" or "fp16")."""
    path = name_or_path if name_or_path.endswith(".json") else os.path.join(CONFIG_DIR, name_or_path + ".json")
    with open(path) as f:
        spec = json.load(f)
    prec_name = precision or spec["precision"]
    if prec_name not in _PRECISIONS:
        raise ValueError(f"unknown precision {prec_name!r}")
    gen, args = spec["generator"], dict(spec.get("args", {}))
    if gen == "served_stream":
        return Config(spec["name"], spec, requests=served_stream(**args), steps=0)
    makers = {"fresnel_cube": fresnel_cube, "three_layers": three_layers,
              "inclusions": inclusions, "ellipsoids": ellipsoids}
    if gen not in makers:
        raise ValueError(f"unknown generator {gen!r}")
    prob, src = makers[gen](precision=_PRECISIONS[prec_name], **args)
    srcs = src if isinstance(src, list) else [src]
    return Config(spec["name"], spec, problem=prob, sources=srcs, steps=int(spec.get("steps", 0)))
