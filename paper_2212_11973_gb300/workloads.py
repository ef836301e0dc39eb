"""Seeded synthetic workloads shaped like the paper's (no method arithmetic here).

The paper evolves Hubbard models on cylinders CL W x L and ladders (main text,
"2D Hubbard model on the square lattice"; Fig. S1 geometries CL4x8 / CL6x12).
Every input is a physical model instance; the only random draws are the
batch parameters (splitmix64) and the random tensors of the kernel-level
parity tests.  Both the CUDA path and the oracle receive what this module
produces; it imports neither.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    Lx: int
    Wy: int
    periodic: bool
    t: float
    U: float
    mu: float
    form: int          # 1: U (n_up - 1/2)(n_dn - 1/2), mu = 0 is half filling
    D: int
    beta0: float
    dtau: float
    beta_end: float
    krylov: int = 8
    precision: int = 0  # 0 FP64, 1 split-BF16 x3, 2 split-BF16 x6

    @property
    def N(self) -> int:
        return self.Lx * self.Wy


# Chemical potential for 1/8 hole doping at U = 8 in the particle-hole
# symmetric form: n = 7/8 at beta = 10 on CL4x8 (FP64, D = 128, growth to
# beta = 1 then 1-TDVP steps of 0.05).  Measured n(mu): -2.4: 0.9038,
# -2.45: 0.8861, -2.5: 0.8693, -2.55: 0.8532, -2.7: 0.8087, -3.0: 0.7325;
# linear interpolation between -2.45 and -2.5 puts n = 7/8 at -2.483, frozen
# at -2.48 (n = 0.876 interpolated, inside 7/8 +- 0.005).
MU_EIGHTH_DOPING = -2.48

CLUSTER_2x2 = Workload("2x2 open cluster U=4 mu=0 D=64", 2, 2, False, 1.0, 4.0, 0.0, 1, 64, 0.01, 0.05, 4.0)
CLUSTER_2x2_FULL = replace(CLUSTER_2x2, name="2x2 open cluster U=4 mu=0 untruncated D=256", D=256)
CYL_4x8_D256 = Workload("CL4x8 U=8 1/8 doping D=256 FP64", 8, 4, True, 1.0, 8.0, MU_EIGHTH_DOPING, 1, 256, 0.01,
                        0.05, 10.0, 8, 0)
CYL_4x8_D512 = replace(CYL_4x8_D256, name="CL4x8 U=8 1/8 doping D=512 mixed", D=512, precision=2)
# The headline workload runs the exact-accumulation split (precision 3): the
# split-BF16 x6 mode misses the 1e-6 accuracy bar at this size (see bench.py
# --precision 2).
CYL_6x12_D1024 = Workload("CL6x12 U=8 1/8 doping D=1024 mixed (exact-split BF16 digits)", 12, 6, True, 1.0, 8.0,
                          MU_EIGHTH_DOPING, 1, 1024, 0.01, 0.05, 12.0, 8, 3)
LADDER_2x4 = Workload("2x4 ladder U=4 mu=-0.3 D=32", 4, 2, False, 1.0, 4.0, -0.3, 1, 32, 0.01, 0.05, 1.0)

BATCH_SEED = 2212119730


def splitmix64(seed: int):
    """splitmix64 (Steele, Lea, Flood 2014): yields 64-bit integers."""
    mask = (1 << 64) - 1
    x = seed & mask
    while True:
        x = (x + 0x9E3779B97F4A7C15) & mask
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        yield z ^ (z >> 31)


def batch_ladders(n: int = 64, seed: int = BATCH_SEED):
    """64 independent 2x8 ladders: U ~ U[2, 10], mu ~ U[-2, 0], D in {64, 96, 128}."""
    g = splitmix64(seed)
    out = []
    for i in range(n):
        u1 = (next(g) >> 11) * 2.0 ** -53
        u2 = (next(g) >> 11) * 2.0 ** -53
        out.append(Workload(f"ladder2x8[{i}]", 8, 2, False, 1.0, 2.0 + 8.0 * u1, -2.0 + 2.0 * u2, 1,
                            (64, 96, 128)[i % 3], 0.01, 0.05, 8.0, 8, 2))
    return out


# U(1)xU(1) bond charges (particle number, n_up - n_dn) of the Choi super-MPS
# within |n|, |s| <= 4; n + s is even for every local pair charge.
SECTOR_CHARGES = [(n, s) for n in range(-4, 5) for s in range(-4, 5) if (n + s) % 2 == 0]


def gaussian_sectors(total: int, width: float, allowed, seed: int = 0):
    """Sector table [(n, 2Sz, dim)] with dims ~ exp(-(n^2 + s^2) / (2 width^2)),
    summing to `total`, over the given allowed charges (sorted)."""
    allowed = sorted(allowed)
    w = np.array([np.exp(-(n * n + s * s) / (2.0 * width * width)) for n, s in allowed])
    dims = np.maximum(1, np.floor(w / w.sum() * total).astype(int))
    rng = np.random.default_rng(seed)
    while dims.sum() < total:
        dims[rng.integers(len(dims))] += 1
    while dims.sum() > total:
        i = int(np.argmax(dims))
        dims[i] -= 1
    return [(n, s, int(d)) for (n, s), d in zip(allowed, dims) if d > 0]


def random_vector(size: int, seed: int):
    """Standard-normal FP64 entries (numpy PCG64, seeded)."""
    return np.random.default_rng(seed).standard_normal(size)
