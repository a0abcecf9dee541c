"""Seeded synthetic inputs for the SFAC two-level Strang splitting workloads.

This module is shared by the CPU oracle, the tests and the benchmark. It holds
no arithmetic of the method itself: it only describes problem parameters and
draws initial fields.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the state
advances by the golden-gamma constant 0x9E3779B97F4A7C15 and each output is the
state passed through the variant-13 finaliser (xor-shift 30, multiply
0xBF58476D1CE4E5B9, xor-shift 27, multiply 0x94D049BB133111EB, xor-shift 31).
Output i of stream `seed` is mix(seed + (i + 1) * gamma) mod 2**64. A double in
[0, 1) is the top 53 bits times 2**-53. Fields are filled in memory order:
axis 1 (x^(1)) fastest, the layout of the paper's lexicographic ordering
(Sec. 2.1, the definition of the vector u below eq. (condition)).

Grids follow Sec. 2.1: m intervals per axis, h = (b - a) / m, interior nodes
x_i = a + i h for i = 1 .. m - 1, so n = m - 1 unknowns per axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with state `seed`."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2**-53."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float, hi: float, start: int = 0) -> np.ndarray:
    """lo + (hi - lo) * U with U from `uniform01`."""
    return lo + (hi - lo) * uniform01(seed, count, start)


@dataclass(frozen=True)
class Problem:
    """One SFAC problem: grid, fractional orders, interface width and step.

    n[l] is the number of interior unknowns along axis l+1 (n = m - 1 in the
    paper's notation), alpha[l] the Riesz order of that axis, [a, b] the
    domain side, eps the interface parameter and tau the time step.
    The field shape in memory is (n[d-1], ..., n[1], n[0]): axis 1 fastest.
    """

    n: tuple
    alpha: tuple
    eps: float
    tau: float
    a: float = -1.0
    b: float = 1.0
    steps: int = 1

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.n))

    @property
    def points(self) -> int:
        return int(np.prod(self.n))

    def h(self, axis: int) -> float:
        return (self.b - self.a) / (self.n[axis] + 1)

    def nodes(self, axis: int) -> np.ndarray:
        """Interior nodes x_i = a + i h, i = 1 .. n (Sec. 2.1)."""
        h = self.h(axis)
        return self.a + h * np.arange(1, self.n[axis] + 1, dtype=np.float64)

    def mesh(self):
        """Coordinate arrays x^(1), x^(2)[, x^(3)] broadcast to `shape`."""
        d = self.dim
        out = []
        for ax in range(d):
            x = self.nodes(ax)
            shp = [1] * d
            shp[d - 1 - ax] = self.n[ax]
            out.append(np.broadcast_to(x.reshape(shp), self.shape))
        return out


# ---------------------------------------------------------------------------
# The five synthetic workloads (2D/3D single grids, batched, serving).
# ---------------------------------------------------------------------------

CONFIG1 = Problem(n=(64, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01, steps=100)
CONFIG2 = Problem(n=(1024, 1024), alpha=(1.3, 1.7), eps=0.05, tau=1e-3, steps=1000)
CONFIG3 = Problem(n=(256, 256, 256), alpha=(1.2, 1.5, 1.8), eps=0.08, tau=2e-3, steps=500)


def config1_u0() -> np.ndarray:
    """2D n=64: u0 uniform in [-0.9, 0.9] from seed 0."""
    p = CONFIG1
    return uniform(0, p.points, -0.9, 0.9).reshape(p.shape)


def config2_u0(problem: Problem = CONFIG2) -> np.ndarray:
    """2D: u0 = 0.9 sin(pi x) sin(pi y) + U(-0.05, 0.05) noise from seed 1."""
    x1, x2 = problem.mesh()
    noise = uniform(1, problem.points, -0.05, 0.05).reshape(problem.shape)
    return 0.9 * np.sin(np.pi * x1) * np.sin(np.pi * x2) + noise


def config3_u0(problem: Problem = CONFIG3) -> np.ndarray:
    """3D: u0 uniform in [-1, 1] from seed 2."""
    return uniform(2, problem.points, -1.0, 1.0).reshape(problem.shape)


def random_field(problem: Problem, seed: int, lo: float = -0.9, hi: float = 0.9) -> np.ndarray:
    """u0 uniform in [lo, hi] from `seed`, in memory order."""
    return uniform(seed, problem.points, lo, hi).reshape(problem.shape)


def example1_problem(alpha, tau: float, m: int = 256) -> Problem:
    """Example 1 of Sec. 5: 2D, Omega = (0,2)^2, eps = 0.1, T = 1."""
    return Problem(n=(m - 1, m - 1), alpha=tuple(alpha), eps=0.1, tau=tau, a=0.0, b=2.0,
                   steps=int(round(1.0 / tau)))


def example1_u0(problem: Problem) -> np.ndarray:
    """Two Gaussian bumps centred at (2/3, 2/3) and (4/3, 4/3) (Example 1)."""
    x1, x2 = problem.mesh()
    return (0.5 * np.exp(-100.0 * ((x1 - 2 / 3) ** 2 + (x2 - 2 / 3) ** 2))
            + 0.5 * np.exp(-100.0 * ((x1 - 4 / 3) ** 2 + (x2 - 4 / 3) ** 2)))


def example2_problem(alpha, tau: float, m: int = 64) -> Problem:
    """Example 2 of Sec. 5: 3D, Omega = (0,1)^3, eps = 0.1, T = 1."""
    return Problem(n=(m - 1,) * 3, alpha=tuple(alpha), eps=0.1, tau=tau, a=0.0, b=1.0,
                   steps=int(round(1.0 / tau)))


def example2_u0(problem: Problem) -> np.ndarray:
    """Two Gaussian bumps centred at (3/8,3/8,3/8) and (5/8,5/8,5/8) (Example 2)."""
    x1, x2, x3 = problem.mesh()
    r1 = (x1 - 3 / 8) ** 2 + (x2 - 3 / 8) ** 2 + (x3 - 3 / 8) ** 2
    r2 = (x1 - 5 / 8) ** 2 + (x2 - 5 / 8) ** 2 + (x3 - 5 / 8) ** 2
    return 0.5 * np.exp(-500.0 * r1) + 0.5 * np.exp(-500.0 * r2)


# ---------------------------------------------------------------------------
# Batched workload: 512 independent 2D instances of uneven size and length.
# ---------------------------------------------------------------------------

BATCH_SIZES = (64, 128, 256, 512)


def batched_instances(count: int = 512, first_seed: int = 100, tau: float = 1e-3) -> list:
    """Instance i uses seed first_seed + i and draws, in this order from its
    own stream: n (one of 64/128/256/512), alpha_1, alpha_2 ~ U[1.1, 1.9],
    eps ~ U[0.02, 0.2], steps ~ U{50..500}. Its field u0 ~ U[-0.9, 0.9] comes
    from the same stream after those five draws."""
    out = []
    for i in range(count):
        seed = first_seed + i
        u = uniform01(seed, 5)
        n = BATCH_SIZES[min(int(u[0] * 4), 3)]
        a1 = 1.1 + 0.8 * u[1]
        a2 = 1.1 + 0.8 * u[2]
        eps = 0.02 + 0.18 * u[3]
        steps = 50 + min(int(u[4] * 451), 450)
        out.append((seed, Problem(n=(n, n), alpha=(a1, a2), eps=eps, tau=tau, steps=steps)))
    return out


def batched_u0(seed: int, problem: Problem) -> np.ndarray:
    return uniform(seed, problem.points, -0.9, 0.9, start=5).reshape(problem.shape)


# ---------------------------------------------------------------------------
# Serving workload: Poisson arrivals of 2D and 3D solves.
# ---------------------------------------------------------------------------

SERVE_2D_SIZES = (64, 128, 256, 512)
SERVE_3D_SIZES = (32, 64, 128)


@dataclass
class Request:
    rid: int
    arrival_s: float
    problem: Problem
    seed: int


def serving_stream(count: int = 2000, rate_hz: float = 200.0, arrival_seed: int = 7,
                   tau: float = 1e-3, sizes_2d: Sequence[int] = SERVE_2D_SIZES,
                   sizes_3d: Sequence[int] = SERVE_3D_SIZES,
                   steps_range=(100, 1000)) -> list:
    """Requests with exponential inter-arrival gaps (mean 1/rate_hz) drawn from
    stream `arrival_seed`; request r draws from stream 1_000_000 + r, in order:
    2D-or-3D (half each), the size, alpha per axis ~ U[1.1, 1.9],
    eps ~ U[0.02, 0.2] and steps ~ U{lo..hi}. Its u0 ~ U[-0.9, 0.9] uses the
    same stream after those draws (offset 16)."""
    gaps = -np.log1p(-uniform01(arrival_seed, count)) / rate_hz
    t = np.cumsum(gaps)
    out = []
    lo, hi = steps_range
    for r in range(count):
        seed = 1_000_000 + r
        u = uniform01(seed, 8)
        if u[0] < 0.5:
            n = sizes_2d[min(int(u[1] * len(sizes_2d)), len(sizes_2d) - 1)]
            dims = 2
        else:
            n = sizes_3d[min(int(u[1] * len(sizes_3d)), len(sizes_3d) - 1)]
            dims = 3
        alpha = tuple(1.1 + 0.8 * u[2 + k] for k in range(dims))
        eps = 0.02 + 0.18 * u[5]
        steps = lo + min(int(u[6] * (hi - lo + 1)), hi - lo)
        out.append(Request(r, float(t[r]), Problem(n=(n,) * dims, alpha=alpha, eps=eps,
                                                   tau=tau, steps=steps), seed))
    return out


def request_u0(req: Request) -> np.ndarray:
    return uniform(req.seed, req.problem.points, -0.9, 0.9, start=16).reshape(req.problem.shape)
