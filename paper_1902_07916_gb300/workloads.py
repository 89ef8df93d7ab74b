"""Seeded synthetic workloads (no arithmetic of the method lives here).

Each workload is a plain description of one integration: integrand,
parameters, box, k, n, trials, depth, sigma multiplier and seed.  The random
parameters of the Genz families are drawn with SplitMix64 (Steele, Lea and
Flood, OOPSLA 2014), implemented below, so the draw is the same on every
machine and every numpy version.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: a Weyl sequence with step 0x9E3779B97F4A7C15 passed through
    a two-multiply xor-shift finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        return a + (b - a) * ((self.next_u64() >> 11) * 2.0 ** -53)

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.next_u64() % (hi - lo + 1)


@dataclass
class Workload:
    name: str
    integrand: str
    dim: int
    lo: list
    hi: list
    k: int
    n: int
    trials: int
    depth: int
    sigma_multiplier: float
    seed: int
    params: list = field(default_factory=list)
    precision: str = "fp64"
    max_cells: int | None = None
    max_samples: int | None = None

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def level1_samples(self) -> int:
        return self.k ** self.dim * self.n * self.trials


def sin3d() -> Workload:
    """sin(x1+x2+x3) on [0,10]^3, k=4 (64 cells), n=1000, 5 trials, depth 2,
    m=2, seed 0: the small FP64 case the oracle runs in full."""
    return Workload("sin3d", "sin_sum", 3, [0.0] * 3, [10.0] * 3, 4, 1000, 5, 2, 2.0, 0)


def sin6d() -> Workload:
    """Eq. (1): sin(sum_{i<6} x_i) on [0,10]^6, k=4 (4096 cells), n=2^16,
    10 trials, depth 3, m=1.5."""
    return Workload("sin6d", "sin_sum", 6, [0.0] * 6, [10.0] * 6, 4, 1 << 16, 10, 3, 1.5, 0)


def gauss9d(sigma: float = 0.1) -> Workload:
    """Eq. (2): the normalised 9-D Gaussian of width sigma on [-1,1]^9, k=3
    (19683 cells), n=2^14, 8 trials, depth 4, m=2."""
    return Workload("gauss9d", "gauss_norm", 9, [-1.0] * 9, [1.0] * 9, 3, 1 << 14, 8, 4, 2.0,
                    0, [sigma])


def corner8d(seed: int = 0) -> Workload:
    """Genz corner peak (1 + sum a_i x_i)^-9 on [0,1]^8, a_i ~ U(0.5, 5) from
    the seed, k=4 (65536 cells), n=2^15, 16 trials, depth 5, m=1."""
    rng = SplitMix64(seed)
    a = [rng.uniform(0.5, 5.0) for _ in range(8)]
    return Workload("corner8d", "genz_corner", 8, [0.0] * 8, [1.0] * 8, 4, 1 << 15, 16, 5, 1.0,
                    seed, a)


GENZ_FAMILIES = ("genz_osc", "genz_prodpeak", "genz_gauss", "genz_corner")


def genz_batch(count: int = 512, seed: int = 0, trials: int = 8, m: float = 2.0,
               cap_level1: int = 1 << 31) -> list:
    """`count` independent Genz integrals on [0,1]^d: d ~ U{2..9},
    k ~ U{2..6}, n = 2^U{10..15}, depth ~ U{1..4}, a_i ~ U(1,10),
    u_i ~ U(0,1), family cycling through the four Genz integrands.  Integral
    j draws from SplitMix64(seed * 2^32 + j).  k is redrawn (then lowered)
    until k^d * n * trials <= cap_level1."""
    out = []
    for j in range(count):
        rng = SplitMix64(((seed & 0xFFFFFFFF) << 32) | j)
        fam = GENZ_FAMILIES[j % 4]
        d = rng.integer(2, 9)
        k = rng.integer(2, 6)
        n = 1 << rng.integer(10, 15)
        depth = rng.integer(1, 4)
        while k > 2 and k ** d * n * trials > cap_level1:
            k -= 1
        a = [rng.uniform(1.0, 10.0) for _ in range(d)]
        u = [rng.uniform(0.0, 1.0) for _ in range(d)]
        if fam == "genz_osc":
            params = [u[0]] + a
        elif fam == "genz_corner":
            params = a
        else:
            params = a + u
        out.append(Workload("genz%03d" % j, fam, d, [0.0] * d, [1.0] * d, k, n, trials, depth,
                            m, rng.next_u64(), params, precision="fp32_fp64acc"))
    return out


WORKLOADS = {"sin3d": sin3d, "sin6d": sin6d, "gauss9d": gauss9d, "corner8d": corner8d}
