"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle's tests.

This module holds no arithmetic of the method itself: it only draws random numbers and states the
workload shapes. Both sides (the CUDA library and the CPU oracle) receive the arrays made here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014). Element ``i`` of a stream with seed ``s`` is ``mix(s + (i + 1) * GAMMA)`` (mod 2**64),
so the stream is counter-based and can be produced in any order. The top 53 bits map to [0, 1).
Fields are filled in index order with x fastest, i.e. a C-ordered array of shape
``(N_z - 1, N_y - 1, N_x - 1)`` (3D) or ``(N_y - 1, N_x - 1)`` (2D); periodic fields keep every node,
``(N_z, N_y, N_x)`` or ``(N_y, N_x)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 20220923


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return ``count`` 64-bit outputs of SplitMix64 starting at stream position ``offset``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(shape: Sequence[int], lo: float, hi: float, seed: int) -> np.ndarray:
    """Field of i.i.d. uniform(lo, hi) values, C order (x fastest), float64."""
    n = int(np.prod(shape)) if len(shape) else 1
    return (lo + (hi - lo) * uniform01(seed, n)).reshape(tuple(shape))


def interior_shape(N: Sequence[int]) -> tuple:
    """Array shape of the interior nodal unknowns for intervals ``N = (N_x, N_y[, N_z])``."""
    return tuple(int(n) - 1 for n in reversed(N))


def field_shape(N: Sequence[int], bc: str = "dirichlet") -> tuple:
    """Array shape of the nodal unknowns: interior nodes (Dirichlet) or all N_a nodes (periodic)."""
    if bc == "periodic":
        return tuple(int(n) for n in reversed(N))
    if bc != "dirichlet":
        raise ValueError("bc must be 'dirichlet' or 'periodic'")
    return interior_shape(N)


@dataclass(frozen=True)
class Workload:
    """One synthetic workload shaped like the paper's 2D/3D experiments: unit square/cube,
    f(u) = flin u + fcub u^3 + flog atanh(u), boundary condition `bc`."""

    name: str
    N: tuple            # intervals per axis (N_x, N_y[, N_z]); unit domain -> h = 1/N
    D: float
    tau: float
    nsteps: int
    scheme: int         # 1 = ETDRK1 (EIFE1), 2 = ETDRK2 (EIFE2)
    u_lo: float
    u_hi: float
    seed: int = DEFAULT_SEED
    dtypes: tuple = field(default=("f64",))
    bc: str = "dirichlet"
    flin: float = 1.0
    fcub: float = -1.0
    flog: float = 0.0

    @property
    def h(self) -> tuple:
        return tuple(1.0 / n for n in self.N)

    @property
    def shape(self) -> tuple:
        return field_shape(self.N, self.bc)

    @property
    def unknowns(self) -> int:
        return int(np.prod(self.shape))

    def u0(self) -> np.ndarray:
        return uniform_field(self.shape, self.u_lo, self.u_hi, self.seed)


# The synthetic workloads (unit square/cube, homogeneous Dirichlet, f = u - u^3).
AC2D_64 = Workload("allen_cahn_2d_64x64_D1e-2_tau1e-2_etdrk2", (64, 64), 1e-2, 1e-2, 100, 2,
                   -0.9, 0.9, DEFAULT_SEED + 0, ("f64",))
AC2D_1024 = Workload("allen_cahn_2d_1024x1024_D1e-4_tau5e-3_etdrk2", (1024, 1024), 1e-4, 5e-3, 2000, 2,
                     -0.05, 0.05, DEFAULT_SEED + 1, ("f32", "f64"))
AC3D_256 = Workload("allen_cahn_3d_256cubed_D1e-3_tau1e-2_etdrk2", (256, 256, 256), 1e-3, 1e-2, 500, 2,
                    -0.9, 0.9, DEFAULT_SEED + 2, ("f32",))
AC3D_64 = Workload("allen_cahn_3d_64cubed_D1e-3_tau1e-2_etdrk2", (64, 64, 64), 1e-3, 1e-2, 500, 2,
                   -0.9, 0.9, DEFAULT_SEED + 2, ("f32", "f64"))

# Grain coarsening with the Flory-Huggins reaction (Example 5.3, Section 5.2): periodic unit cube,
# 128^3 mesh, eps = 0.01 (D = eps^2), theta = 0.8, theta_c = 1.6 (f = theta_c u - theta atanh u),
# tau = T / N_T = 20 / 2048, u0 uniform(-0.9, 0.9) per node.
GC3D_128 = Workload("grain_coarsening_3d_128cubed_periodic_flory_huggins_eps1e-2_tau5o512_etdrk2",
                    (128, 128, 128), 1e-4, 20.0 / 2048, 2048, 2, -0.9, 0.9, DEFAULT_SEED + 6, ("f32", "f64"),
                    "periodic", 1.6, 0.0, -0.8)
GC3D_32 = Workload("grain_coarsening_3d_32cubed_periodic_flory_huggins_eps1e-2_tau5o512_etdrk2",
                   (32, 32, 32), 1e-4, 20.0 / 2048, 64, 2, -0.9, 0.9, DEFAULT_SEED + 6, ("f32", "f64"),
                   "periodic", 1.6, 0.0, -0.8)

WORKLOADS = {w.name: w for w in (AC2D_64, AC2D_1024, AC3D_256, AC3D_64, GC3D_128, GC3D_32)}


@dataclass(frozen=True)
class BatchWorkload:
    """Many independent 2D Allen-Cahn problems of uneven size: per problem N_x and N_y drawn from
    `sizes`, D log-uniform in [d_lo, d_hi], u0 uniform(u_lo, u_hi); common tau and step count."""

    name: str
    count: int
    sizes: tuple
    d_lo: float
    d_hi: float
    tau: float
    nsteps: int
    u_lo: float = -0.9
    u_hi: float = 0.9
    seed: int = DEFAULT_SEED + 3

    def problems(self):
        r = uniform01(self.seed, 3 * self.count)
        ns = len(self.sizes)
        out = []
        for i in range(self.count):
            nx = self.sizes[min(int(r[3 * i] * ns), ns - 1)]
            ny = self.sizes[min(int(r[3 * i + 1] * ns), ns - 1)]
            D = float(np.exp(np.log(self.d_lo) + r[3 * i + 2] * (np.log(self.d_hi) - np.log(self.d_lo))))
            out.append(((nx, ny), D))
        return out

    def u0(self, i: int, shape) -> np.ndarray:
        return uniform_field(shape, self.u_lo, self.u_hi, self.seed + 1000 + i)


BATCH_2D_512 = BatchWorkload("batched_2d_512_allen_cahn_N64-384_D1e-4-1e-2_tau1e-2_etdrk2", 512,
                             (64, 96, 128, 192, 256, 384), 1e-4, 1e-2, 1e-2, 200)
BATCH_WORKLOADS = {BATCH_2D_512.name: BATCH_2D_512}


@dataclass(frozen=True)
class SnoWorkload:
    """Spectral-neural-operator coarse propagator at N x N: C channels, M x M retained sine modes,
    L layers, predicting `window` ETDRK2 steps of size tau. Training trajectories: u0 uniform(u_lo,
    u_hi), D log-uniform in [d_lo, d_hi], `traj_steps` steps, input/target pairs every `window`
    steps. Parareal runs: `batch` problems over `windows` windows."""

    name: str
    N: int = 256
    C: int = 32
    M: int = 24
    L: int = 4
    window: int = 50
    tau: float = 1e-2
    trajectories: int = 2000
    traj_steps: int = 200
    batch: int = 64
    windows: int = 4
    d_lo: float = 1e-4
    d_hi: float = 1e-2
    u_lo: float = -0.9
    u_hi: float = 0.9
    seed: int = DEFAULT_SEED + 5

    def D(self, i: int) -> float:
        r = float(uniform01(self.seed, 1, offset=i)[0])
        return float(np.exp(np.log(self.d_lo) + r * (np.log(self.d_hi) - np.log(self.d_lo))))

    def u0(self, i: int) -> np.ndarray:
        return uniform_field((self.N - 1, self.N - 1), self.u_lo, self.u_hi, self.seed + 7919 * (i + 1))

    def init_weights(self, seed_offset: int = 0) -> dict:
        """Seeded initial weights: uniform(-s, s) with s = 1 (lift), 1/C (mode mix), 1/sqrt(C)
        (pointwise), 0.1/sqrt(C) (projection); biases 0."""
        C, M, L = self.C, self.M, self.L
        sd = self.seed + 104729 + seed_offset
        return {
            "Wl": uniform_field((C, 2), -1.0, 1.0, sd),
            "bl": np.zeros(C),
            "Wm": uniform_field((L, M, M, C, C), -1.0 / C, 1.0 / C, sd + 1),
            "Wp": uniform_field((L, C, C), -1.0 / np.sqrt(C), 1.0 / np.sqrt(C), sd + 2),
            "bp": np.zeros((L, C)),
            "Wq": uniform_field((C,), -0.1 / np.sqrt(C), 0.1 / np.sqrt(C), sd + 3),
            "bq": np.zeros(()),
        }


SNO_256 = SnoWorkload("sno_parareal_2d_256_C32_M24_L4_w50_b64_allen_cahn")
SNO_WORKLOADS = {SNO_256.name: SNO_256}
