"""Seeded synthetic inputs for the phase-field twin step.

This module only shapes inputs: grids, twin nuclei, Voronoi grains, grain
orientations, the synthetic plastic-strain field that stands in for the
crystal-plasticity finite-element side, and the mean-strain loading history.
It holds none of the method's arithmetic (no stiffness, no eigenstrain, no
Fourier solve, no driving force); both the FP64 CPU oracle and the CUDA
library consume what it returns.

Array layout: every field is indexed ``[..., z, y, x]`` (C order, x fastest),
i.e. flat voxel index ``x + nx * (y + ny * z)``, with unit grid spacing and
voxel centres at integer coordinates.  Symmetric tensors are stored as six
Voigt components ``xx, yy, zz, yz, xz, xy`` holding *tensor* (not engineering)
shear components.

The paper's workloads (Sec. 4.2: a 64x64x128 pillar grid loaded along
[10-10]; Sec. 5: a 64x64x16 polycrystal; Sec. 6.1: 16x16x32 .. 64x64x128
meshes) use experimental or finite-element data that is not available, so
every input here is drawn from ``numpy.random.Generator(PCG64(seed))`` with
the shapes and structure of those runs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Lattice ratio of the HCP cell (Sec. 2.1) and the six {10-12}<-1011>
# tension-twin variants as (plane hkil, direction uvtw) Miller-Bravais indices.
C_OVER_A = 1.633
TWIN_VARIANTS_MB = (
    ((1, 0, -1, 2), (-1, 0, 1, 1)),
    ((0, 1, -1, 2), (0, -1, 1, 1)),
    ((-1, 1, 0, 2), (1, -1, 0, 1)),
    ((-1, 0, 1, 2), (1, 0, -1, 1)),
    ((0, -1, 1, 2), (0, 1, -1, 1)),
    ((1, -1, 0, 2), (-1, 1, 0, 1)),
)
# Loading axis of the pillar, [10-10] in the crystal frame (Sec. 4.1).
D_10M10 = np.array([math.sqrt(3.0) / 2.0, 0.5, 0.0])

# Phase-field parameters shared by every workload: c1 = 31.25 MPa (Table 5)
# in GPa, an interface width of W = 3 voxels giving c2 = c1 (W/4)^2, unit
# mobility and dt = 0.05.
C1_GPA = 0.03125
INTERFACE_W = 3.0
C2 = C1_GPA * (INTERFACE_W / 4.0) ** 2
C3 = 1.0
DT = 0.05
GAMMA_TW = 0.129
C_HEX_GPA = (59.4, 25.6, 21.4, 61.6, 16.4)  # C11, C12, C13, C33, C44 (Table 1)


def _nucleus_axes(variant: int, c_a: float = C_OVER_A):
    """Unit shear direction s, t = n x s and plane normal n of a twin variant,
    crystal frame, used only to orient ellipsoidal nuclei."""
    (h, k, _i, l), (u, v, t, w) = TWIN_VARIANTS_MB[variant]
    a1 = np.array([1.0, 0.0, 0.0])
    a2 = np.array([-0.5, math.sqrt(3.0) / 2.0, 0.0])
    a3 = np.array([-0.5, -math.sqrt(3.0) / 2.0, 0.0])
    s = u * a1 + v * a2 + t * a3 + w * np.array([0.0, 0.0, c_a])
    n = np.array([h, (h + 2 * k) / math.sqrt(3.0), l / c_a])
    s /= np.linalg.norm(s)
    n /= np.linalg.norm(n)
    tt = np.cross(n, s)
    return s, tt / np.linalg.norm(tt), n


def _periodic_offsets(shape, centre):
    """Minimum-image offsets (dx, dy, dz) of every voxel centre from `centre`."""
    nz, ny, nx = shape
    out = []
    for n, c in ((nx, centre[0]), (ny, centre[1]), (nz, centre[2])):
        d = np.arange(n, dtype=np.float64) - c
        d = (d + n / 2.0) % n - n / 2.0
        out.append(d)
    dx = out[0][None, None, :]
    dy = out[1][None, :, None]
    dz = out[2][:, None, None]
    return dx, dy, dz


def ellipsoid_mask(shape, centre, axes, semi):
    """Voxels whose centres lie inside a periodic ellipsoid.

    axes: three orthonormal rows (sample frame); semi: the three semi-axes."""
    dx, dy, dz = _periodic_offsets(shape, centre)
    q = np.zeros(shape)
    for a, r in zip(axes, semi):
        p = dx * a[0] + dy * a[1] + dz * a[2]
        q = q + (p / r) ** 2
    return q <= 1.0


def shoemake_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """k uniformly random rotation matrices (Shoemake unit quaternions);
    each maps crystal-frame vectors to the sample frame."""
    u = rng.random((k, 3))
    q = np.stack([
        np.sqrt(u[:, 0]) * np.cos(2 * np.pi * u[:, 2]),        # w
        np.sqrt(1 - u[:, 0]) * np.sin(2 * np.pi * u[:, 1]),    # x
        np.sqrt(1 - u[:, 0]) * np.cos(2 * np.pi * u[:, 1]),    # y
        np.sqrt(u[:, 0]) * np.sin(2 * np.pi * u[:, 2]),        # z
    ], axis=1)
    w, x, y, z = q.T
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def voronoi_grains(rng: np.random.Generator, shape, n_grains: int) -> np.ndarray:
    """Periodic Voronoi tessellation: seeds uniform in the box, each voxel takes
    the nearest seed (minimum image), ties go to the lowest seed index."""
    nz, ny, nx = shape
    seeds = rng.random((n_grains, 3)) * np.array([nx, ny, nz])
    best = np.full(shape, np.inf, dtype=np.float64)
    grain = np.zeros(shape, dtype=np.uint16)
    for g in range(n_grains):
        dx, dy, dz = _periodic_offsets(shape, seeds[g])
        d2 = dx * dx + dy * dy + dz * dz
        upd = d2 < best
        best = np.where(upd, d2, best)
        grain[upd] = g
    return grain


def gaussian_plastic_strain(rng: np.random.Generator, shape, corr: float,
                            rms: float) -> np.ndarray:
    """Smooth traceless Gaussian random field standing in for the plastic strain.

    Five amplitudes a_m (white noise convolved with a periodic Gaussian of
    standard deviation `corr` voxels, mean removed) multiply an orthonormal
    deviatoric basis B_m; the sum is scaled to the RMS Frobenius norm `rms`.
    Returns six Voigt components with tensor shears."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * 2 * np.pi
    ky = np.fft.fftfreq(ny) * 2 * np.pi
    kx = np.fft.rfftfreq(nx) * 2 * np.pi
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    kernel = np.exp(-0.5 * corr * corr * k2)
    kernel[0, 0, 0] = 0.0  # mean removed
    a = np.empty((5,) + tuple(shape))
    for m in range(5):
        w = rng.standard_normal(shape)
        a[m] = np.fft.irfftn(np.fft.rfftn(w) * kernel, s=shape, axes=(0, 1, 2))
    r2 = 1.0 / math.sqrt(2.0)
    r6 = 1.0 / math.sqrt(6.0)
    eps = np.zeros((6,) + tuple(shape))
    eps[0] = r2 * a[0] - r6 * a[1]
    eps[1] = -r2 * a[0] - r6 * a[1]
    eps[2] = 2 * r6 * a[1]
    eps[3] = r2 * a[2]
    eps[4] = r2 * a[3]
    eps[5] = r2 * a[4]
    scale = rms / math.sqrt(np.mean(np.sum(a * a, axis=0)))
    return eps * scale


def uniaxial_strain(strain: float, d) -> np.ndarray:
    """Voigt (tensor-shear) components of strain * d (x) d for a unit vector d."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return strain * np.array([d[0] * d[0], d[1] * d[1], d[2] * d[2],
                              d[1] * d[2], d[0] * d[2], d[0] * d[1]])


@dataclass
class Workload:
    """One phase-field instance: fields, parameters and loading history."""
    name: str
    shape: tuple                   # (nz, ny, nx)
    variant_ids: list              # which of the six twin variants are evolved
    f: np.ndarray                  # [V, nz, ny, nx] twin fractions
    eps_p: np.ndarray | None       # [6, nz, ny, nx] plastic strain, or None
    grain: np.ndarray | None       # [nz, ny, nx] uint16 grain ids, or None
    grain_R: np.ndarray            # [G, 3, 3] crystal -> sample rotations
    E: np.ndarray                  # [steps, 6] mean strain of each step
    twin_stiffness: int = 1        # 1: rotated twin stiffness; 0: C_twin := C_matrix
    c1: float = C1_GPA
    c2: float = C2
    c3: float = C3
    dt: float = DT
    gamma_tw: float = GAMMA_TW
    c_over_a: float = C_OVER_A
    C_hex: tuple = C_HEX_GPA
    ms_tol: float = 1e-6
    ms_max_it: int = 100
    precision: str = "fp32"
    mobility: np.ndarray | None = None  # [nz, ny, nx] mobility factor in [0, 1] (pad layer), or None
    extra: dict = field(default_factory=dict)

    @property
    def nvox(self) -> int:
        return int(np.prod(self.shape))

    @property
    def V(self) -> int:
        return len(self.variant_ids)


def _place_nuclei(rng, shape, variant_ids, grain, grain_R, n_nuclei,
                  semi_s=(2.0, 6.0), semi_tn=(1.0, 3.0)):
    """Random ellipsoidal nuclei (f = 1 inside, later nuclei overwrite earlier
    ones), axes along the chosen variant's s, t, n in the host grain's frame."""
    nz, ny, nx = shape
    V = len(variant_ids)
    f = np.zeros((V,) + tuple(shape))
    for _ in range(n_nuclei):
        c = rng.random(3) * np.array([nx, ny, nz])
        a_s = rng.uniform(*semi_s)
        a_t = rng.uniform(*semi_tn)
        a_n = rng.uniform(*semi_tn)
        v = int(rng.integers(V))
        g = 0
        if grain is not None:
            g = int(grain[int(c[2]) % nz, int(c[1]) % ny, int(c[0]) % nx])
        s, t, n = _nucleus_axes(variant_ids[v])
        R = grain_R[g]
        m = ellipsoid_mask(shape, c, (R @ s, R @ t, R @ n), (a_s, a_t, a_n))
        f[:, m] = 0.0
        f[v, m] = 1.0
    return f


def config1(steps: int = 100, n: int = 32) -> Workload:
    """32^3 single crystal, one variant (10-12)[-1011], homogeneous stiffness,
    no plastic strain, one 4/2/2 ellipsoidal nucleus at the centre, constant
    mean strain -0.5% along [10-10], FP64."""
    shape = (n, n, n)
    s, t, nn = _nucleus_axes(0)
    c = np.array([n / 2.0] * 3)
    f = ellipsoid_mask(shape, c, (s, t, nn), (4.0, 2.0, 2.0)).astype(np.float64)[None]
    E = np.tile(uniaxial_strain(-0.005, D_10M10), (steps, 1))
    return Workload("cfg1_32c_fp64", shape, [0], f, None, None, np.eye(3)[None],
                    E, twin_stiffness=0, ms_tol=1e-12, precision="fp64")


def config2(steps: int = 500, n: int = 128, seed: int = 1002,
            total_steps: int = 500) -> Workload:
    """128^3 single-crystal pillar, the two Schmid-factor-0.499 variants under
    [10-10] compression, rotated twin stiffness, 8 random nuclei, smooth
    plastic strain (correlation 8 voxels, RMS 0.2%), mean strain ramped
    linearly to -4% over `total_steps` steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    vids = [0, 3]
    R = np.eye(3)[None]
    f = _place_nuclei(rng, shape, vids, None, R, 8)
    eps_p = gaussian_plastic_strain(rng, shape, 8.0, 0.002)
    E = np.stack([uniaxial_strain(-0.04 * (k + 1) / total_steps, D_10M10)
                  for k in range(steps)])
    return Workload(f"cfg2_{n}c", shape, vids, f, eps_p, None, R, E)


def pad_mobility(shape, widths, low):
    """Mobility factor 1 inside a box-shaped sample and `low` in a pad layer of
    widths (wz, wy, wx) voxels on every side of the periodic cell."""
    nz, ny, nx = shape
    wz, wy, wx = widths
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    pad = (z < wz) | (z >= nz - wz) | (y < wy) | (y >= ny - wy) | (x < wx) | (x >= nx - wx)
    return np.where(pad, low, 1.0)


def pillar_pad(steps: int = 100, seed: int = 1006, low: float = 1e-3,
               total_steps: int = 500) -> Workload:
    """The micro-pillar cell of Sec. 4: 64 x 64 x 128 FFT cells (x, y, z) whose
    outer 5 voxels (about 0.5 um of a 6.6 um wide cell) form the low-mobility
    pad, the config-2 crystal (two variants, [10-10] compression ramped to -4%,
    smooth plastic strain) inside."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (128, 64, 64)
    vids = [0, 3]
    R = np.eye(3)[None]
    f = _place_nuclei(rng, shape, vids, None, R, 8)
    mob = pad_mobility(shape, (5, 5, 5), low)
    f = f * (mob == 1.0)  # nuclei inside the sample only
    eps_p = gaussian_plastic_strain(rng, shape, 8.0, 0.002)
    E = np.stack([uniaxial_strain(-0.04 * (k + 1) / total_steps, D_10M10)
                  for k in range(steps)])
    return Workload("pillar_pad", shape, vids, f, eps_p, None, R, E, mobility=mob)


def mesh_study(level: int, steps: int = 20, seed: int = 1007) -> Workload:
    """The discretisation study of Sec. 6: FFT grids 16 x 16 x 32 (mesh1),
    32 x 32 x 64 (mesh2) and 64 x 64 x 128 (mesh3) cells (x, y, z) of the
    pillar crystal (two variants, [10-10] compression ramped to -4% over 500
    steps, smooth plastic strain), nuclei scaled with the grid."""
    rng = np.random.Generator(np.random.PCG64(seed + level))
    n = 16 * 2 ** (level - 1)
    shape = (2 * n, n, n)
    vids = [0, 3]
    R = np.eye(3)[None]
    s = n / 16.0
    f = _place_nuclei(rng, shape, vids, None, R, 4, semi_s=(2.0 * s, 4.0 * s), semi_tn=(1.0 * s, 2.0 * s))
    eps_p = gaussian_plastic_strain(rng, shape, 0.5 * n, 0.002)
    E = np.stack([uniaxial_strain(-0.04 * (k + 1) / 500, D_10M10) for k in range(steps)])
    return Workload(f"mesh{level}", shape, vids, f, eps_p, None, R, E)


def config3(steps: int = 200, n: int = 256, seed: int = 1003,
            n_grains: int = 64) -> Workload:
    """256^3 polycrystal: 64 periodic Voronoi grains with uniformly random
    orientations, all six variants, 8 random nuclei, no plastic strain,
    constant mean strain -2% along the sample z axis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    grain = voronoi_grains(rng, shape, n_grains)
    R = shoemake_rotations(rng, n_grains)
    vids = [0, 1, 2, 3, 4, 5]
    f = _place_nuclei(rng, shape, vids, grain, R, 8)
    E = np.tile(uniaxial_strain(-0.02, (0.0, 0.0, 1.0)), (steps, 1))
    return Workload(f"cfg3_{n}c_poly{n_grains}", shape, vids, f, None, grain, R, E)


BATCH_SIZES = (64, 80, 96, 120, 128, 160)


def config4_instance(i: int, steps: int = 100) -> Workload:
    """Instance i of the batched workload: each grid size drawn from
    {64, 80, 96, 120, 128, 160}, 1-3 variants, 1-4 nuclei, rotated twin
    stiffness, mean strain -1% along a random direction."""
    rng = np.random.Generator(np.random.PCG64(2000 + i))
    nx, ny, nz = (int(rng.choice(BATCH_SIZES)) for _ in range(3))
    shape = (nz, ny, nx)
    V = int(rng.integers(1, 4))
    vids = sorted(int(v) for v in rng.choice(6, size=V, replace=False))
    R = np.eye(3)[None]
    f = _place_nuclei(rng, shape, vids, None, R, int(rng.integers(1, 5)))
    d = rng.standard_normal(3)
    E = np.tile(uniaxial_strain(-0.01, d), (steps, 1))
    return Workload(f"cfg4_inst{i}", shape, vids, f, None, None, R, E)


def config5(steps: int = 100, n: int = 512, seed: int = 1005) -> Workload:
    """512^3 single-crystal pillar as config 2 (two variants, smooth plastic
    strain), mean strain ramped at -0.008% per step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    vids = [0, 3]
    R = np.eye(3)[None]
    f = _place_nuclei(rng, shape, vids, None, R, 8)
    eps_p = gaussian_plastic_strain(rng, shape, 8.0, 0.002)
    E = np.stack([uniaxial_strain(-0.00008 * (k + 1), D_10M10) for k in range(steps)])
    return Workload(f"cfg5_{n}c", shape, vids, f, eps_p, None, R, E)
