"""Seeded synthetic inputs for the anisotropic Gatenby-Gawlinski time step.

This module only draws input data: the per-cell tensor description
(theta, lambda1, lambda2) and the initial fields (u0, v0, w0), all as
float64 numpy arrays of shape (ny, nx), row-major with x fastest.  It holds
none of the method's arithmetic (no tensor assembly, no stencil, no update),
so that the CUDA path and the FP64 oracle can both consume exactly the same
bytes without sharing any code of the scheme itself.

The paper (Section 2 and Figure 2) states neither its initial data nor its
tensor fields, so these generators stand in for them:

* random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014); a uniform double
  is ``(z >> 11) * 2**-53``;
* a smooth field is a sum of 8 Fourier modes
  ``g = sum_m A_m cos(2 pi (k_m x + l_m y) + phi_m)`` with integer wave
  numbers in [-3, 3] (not both zero), ``A_m ~ U[0,1]/m`` and
  ``phi_m ~ U[0, 2 pi)``, normalised analytically to
  ``g_hat = (1 + g / sum_m A_m) / 2`` in [0, 1], so the field does not depend
  on the grid resolution;
* the initial datum is healthy tissue (u=1, v=0, w=0) with a tumour disk
  (u=0, v=1, w=0) of radius r centred at (0.5, 0.5), tested at cell centres
  with ``<=``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

MASK64 = (1 << 64) - 1

# Seed base of each workload: 1748 + 1000 * workload index.
SEED_PLAIN_128 = 1748
SEED_LAYERED_1024 = 2748
SEED_HETERO_8192 = 3748
SEED_ENSEMBLE = 4748
SEED_ADJOINT_2048 = 5748

FIELD_THETA = 1
FIELD_LAMBDA1 = 2
FIELD_LAMBDA2 = 3


class SplitMix64:
    """SplitMix64 counter-based generator (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


@dataclasses.dataclass
class FourierModes:
    k: List[int]
    l: List[int]
    amp: List[float]
    phase: List[float]


def draw_modes(seed: int, n_modes: int = 8, kmax: int = 3) -> FourierModes:
    rng = SplitMix64(seed)
    ks, ls, amps, phs = [], [], [], []
    for m in range(1, n_modes + 1):
        while True:
            k = rng.randint(-kmax, kmax)
            l = rng.randint(-kmax, kmax)
            if k != 0 or l != 0:
                break
        ks.append(k)
        ls.append(l)
        amps.append(rng.uniform() / m)
        phs.append(2.0 * math.pi * rng.uniform())
    return FourierModes(ks, ls, amps, phs)


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """Cell-centre coordinates (i + 1/2) * h, h = length / n."""
    h = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def smooth_field(nx: int, ny: int, seed: int, lx: float = 1.0, ly: float = 1.0) -> np.ndarray:
    """Normalised Fourier field g_hat in [0, 1] sampled at cell centres.

    Each mode is evaluated separably,
    cos(a + b) = cos(a) cos(b) - sin(a) sin(b) with a = 2 pi k x + phi and
    b = 2 pi l y, so a large grid costs two outer products per mode.
    """
    modes = draw_modes(seed)
    x = cell_centres(nx, lx)
    y = cell_centres(ny, ly)
    g = np.zeros((ny, nx), dtype=np.float64)
    for k, l, a, ph in zip(modes.k, modes.l, modes.amp, modes.phase):
        ax = 2.0 * math.pi * k * x + ph
        by = 2.0 * math.pi * l * y
        g += a * (np.outer(np.cos(by), np.cos(ax)) - np.outer(np.sin(by), np.sin(ax)))
    total = float(sum(modes.amp))
    return 0.5 * (1.0 + g / total)


def tumour_disk(nx: int, ny: int, radius: float, centre=(0.5, 0.5),
                lx: float = 1.0, ly: float = 1.0):
    """Initial datum: u=1, v=0, w=0 outside the disk, u=0, v=1, w=0 inside."""
    x = cell_centres(nx, lx)[None, :]
    y = cell_centres(ny, ly)[:, None]
    inside = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 <= radius * radius
    u0 = np.where(inside, 0.0, 1.0).astype(np.float64)
    v0 = np.where(inside, 1.0, 0.0).astype(np.float64)
    w0 = np.zeros((ny, nx), dtype=np.float64)
    return np.ascontiguousarray(u0), np.ascontiguousarray(v0), w0


@dataclasses.dataclass
class Problem:
    """One synthetic instance: grid, scalar rates and host input arrays."""
    name: str
    nx: int
    ny: int
    delta: float      # aggression rate (d in eq. 1)
    rho: float        # tumour growth rate (r in eq. 1)
    D: float          # tumour diffusion constant (alpha in eq. 1)
    c: float          # acid production / reabsorption rate (c in eq. 1)
    theta: np.ndarray
    lambda1: np.ndarray
    lambda2: np.ndarray
    u0: np.ndarray
    v0: np.ndarray
    w0: np.ndarray
    steps: int
    cfl: float = 0.9
    lx: float = 1.0
    ly: float = 1.0
    seed: int = 0

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def scalars(self) -> Dict[str, float]:
        return dict(delta=self.delta, rho=self.rho, D=self.D, c=self.c)


def heterogeneous_tensor(nx: int, ny: int, seed: int, lam_min: float, lam_max: float):
    """theta in [0, pi) and lambda1, lambda2 in [lam_min, lam_max], one seed each."""
    gt = smooth_field(nx, ny, seed ^ FIELD_THETA)
    g1 = smooth_field(nx, ny, seed ^ FIELD_LAMBDA1)
    g2 = smooth_field(nx, ny, seed ^ FIELD_LAMBDA2)
    theta = math.pi * gt
    l1 = lam_min + (lam_max - lam_min) * g1
    l2 = lam_min + (lam_max - lam_min) * g2
    return theta, l1, l2


def layered_tensor(nx: int, ny: int, seed: int):
    """Two half-planes split at x = 0.5 (theta = 0 left, pi/4 right), with
    lambda1 = 1 and lambda2 = 0.1 (ratio 10, lower diffusivity across the
    principal direction), each perturbed by a seeded smooth 10 % field."""
    x = cell_centres(nx)[None, :] * np.ones((ny, 1))
    gt = smooth_field(nx, ny, seed ^ FIELD_THETA)
    g1 = smooth_field(nx, ny, seed ^ FIELD_LAMBDA1)
    g2 = smooth_field(nx, ny, seed ^ FIELD_LAMBDA2)
    theta0 = np.where(x < 0.5, 0.0, math.pi / 4.0)
    theta = theta0 + 0.1 * (math.pi / 4.0) * (2.0 * gt - 1.0)
    l1 = 1.0 * (1.0 + 0.1 * (2.0 * g1 - 1.0))
    l2 = 0.1 * (1.0 + 0.1 * (2.0 * g2 - 1.0))
    return np.ascontiguousarray(theta), l1, l2


def plain_128(nx: int = 128, ny: Optional[int] = None, steps: int = 2000, seed: int = SEED_PLAIN_128) -> Problem:
    """128 x 128 cells, delta=12.5, rho=1, D=4e-5, c=70, lambda in [0.1, 1],
    disk r = 0.1, 2000 steps at CFL 0.9 (other sizes use the same fields)."""
    ny = nx if ny is None else ny
    th, l1, l2 = heterogeneous_tensor(nx, ny, seed, 0.1, 1.0)
    u0, v0, w0 = tumour_disk(nx, ny, 0.1)
    return Problem("plain_128", nx, ny, 12.5, 1.0, 4e-5, 70.0, th, l1, l2, u0, v0, w0, steps, seed=seed)


def layered_1024(delta: float = 12.5, nx: int = 1024, ny: Optional[int] = None, steps: int = 20000,
                 seed: int = SEED_LAYERED_1024) -> Problem:
    """Layered tissue, delta in {0.5, 12.5}, disk r = 0.05 on the interface."""
    ny = nx if ny is None else ny
    th, l1, l2 = layered_tensor(nx, ny, seed)
    u0, v0, w0 = tumour_disk(nx, ny, 0.05)
    return Problem(f"layered_1024_delta{delta}", nx, ny, delta, 1.0, 4e-5, 70.0, th, l1, l2,
                   u0, v0, w0, steps, seed=seed)


def hetero_8192(nx: int = 8192, ny: Optional[int] = None, steps: int = 5000, seed: int = SEED_HETERO_8192) -> Problem:
    """Fully heterogeneous tensor field, lambda in [0.01, 1]; the field is
    grid-independent, so a 512 x 512 instance samples the same tissue."""
    ny = nx if ny is None else ny
    th, l1, l2 = heterogeneous_tensor(nx, ny, seed, 0.01, 1.0)
    u0, v0, w0 = tumour_disk(nx, ny, 0.1)
    return Problem("hetero_8192", nx, ny, 12.5, 1.0, 4e-5, 70.0, th, l1, l2, u0, v0, w0, steps, seed=seed)


def adjoint_2048(nx: int = 2048, ny: Optional[int] = None, steps: int = 10000, seed: int = SEED_ADJOINT_2048,
                 target: bool = False) -> Problem:
    """Parameters of the 128 x 128 workload on a 2048 x 2048 grid.  With
    ``target=True`` the tensor field is drawn from seed + 1: the twin
    experiment whose final v is the misfit target."""
    ny = nx if ny is None else ny
    s = seed + 1 if target else seed
    th, l1, l2 = heterogeneous_tensor(nx, ny, s, 0.1, 1.0)
    u0, v0, w0 = tumour_disk(nx, ny, 0.1)
    return Problem("adjoint_2048" + ("_target" if target else ""), nx, ny, 12.5, 1.0, 4e-5, 70.0,
                   th, l1, l2, u0, v0, w0, steps, seed=s)


def growing_tumour(nx: int = 64, ny: Optional[int] = None, steps: int = 500, seed: int = SEED_PLAIN_128 + 7,
                   lx: float = 1.0, ly: float = 1.0) -> Problem:
    """Tumour cells in healthy tissue: U = 1 everywhere, V = 1 on a disk of
    radius 0.2, W = 0; tumour diffusion D = 0.2 well above the acid's
    lambda in [0.02, 0.08] (heterogeneous, seeded); delta = 3, rho = 1, c = 5.
    The tumour flux (mobility 1 - U) starts closed and opens as acid builds
    up and U falls inside the disk: the workload of the adaptive step."""
    ny = nx if ny is None else ny
    th, l1, l2 = heterogeneous_tensor(nx, ny, seed, 0.02, 0.08)
    u0, v0, w0 = tumour_disk(nx, ny, 0.2, centre=(0.5 * lx, 0.5 * ly), lx=lx, ly=ly)
    u0 = np.ones((ny, nx))
    return Problem("growing_tumour", nx, ny, 3.0, 1.0, 0.2, 5.0, th, l1, l2, u0, v0, w0, steps, lx=lx, ly=ly,
                   seed=seed)


ENSEMBLE_SIZES = (128, 256, 512, 1024)


def ensemble_specs(n_instances: int = 256, seed: int = SEED_ENSEMBLE):
    """Per-instance (nx, ny, delta, D) drawn independently: nx, ny uniform over
    {128, 256, 512, 1024}, delta ~ U[0.5, 20], D ~ logU[1e-5, 1e-3]."""
    rng = SplitMix64(seed)
    specs = []
    for _ in range(n_instances):
        nx = ENSEMBLE_SIZES[rng.randint(0, 3)]
        ny = ENSEMBLE_SIZES[rng.randint(0, 3)]
        delta = 0.5 + 19.5 * rng.uniform()
        D = 10.0 ** (-5.0 + 2.0 * rng.uniform())
        specs.append((nx, ny, delta, D))
    return specs


def ensemble_instance(index: int, spec, steps: int = 5000, seed: int = SEED_ENSEMBLE,
                      scale: int = 1) -> Problem:
    """Instance ``index`` of the ensemble (rho=1, c=70, lambda in [0.1, 1],
    disk r = 0.1).  ``scale`` divides both grid sizes (parity tests)."""
    nx, ny, delta, D = spec
    nx, ny = max(nx // scale, 1), max(ny // scale, 1)
    s = seed + 1 + index
    th, l1, l2 = heterogeneous_tensor(nx, ny, s, 0.1, 1.0)
    u0, v0, w0 = tumour_disk(nx, ny, 0.1)
    return Problem(f"ensemble_{index}", nx, ny, delta, 1.0, D, 70.0, th, l1, l2, u0, v0, w0, steps, seed=s)


def random_state(nx: int, ny: int, seed: int):
    """Smooth random fields in [0, 1] for u, v, w (parity of generic states)."""
    u = smooth_field(nx, ny, seed ^ 0x11)
    v = smooth_field(nx, ny, seed ^ 0x22)
    w = smooth_field(nx, ny, seed ^ 0x33)
    return u, v, w


def white_noise(nx: int, ny: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Cell-wise independent uniforms (rough data for operator tests), drawn
    with SplitMix64 vectorised over a counter: z_i = mix(seed + (i+1) * gamma)."""
    n = nx * ny
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (np.arange(1, n + 1, dtype=np.uint64) * gamma)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).reshape(ny, nx)
