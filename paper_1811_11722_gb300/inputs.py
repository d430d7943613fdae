"""Seeded synthetic inputs for the shifted rank-1 lattice rule.

This module only draws numbers and lays them out: SplitMix64 streams, shift
tables, polynomial term tables (coefficient + exponent row per monomial) and
prime lattice sizes.  It holds none of the rule's arithmetic (no indices,
transforms, integrand values or sums), so both the CUDA path and the CPU oracle
may consume what it produces.

Readings of the workloads (the paper fixes none of these draws):
  * SplitMix64 (Steele, Lea, Flood 2014) with 53-bit doubles u = (s >> 11) 2^-53.
  * Polynomials are a constant term c0 plus the stated number of random
    monomials; degree-1 monomials are c x_i, degree-2 are c x_i x_j (i <= j,
    squares allowed).  Variables (pairs) are drawn without replacement while
    the term count fits, else with replacement.  Sector-decomposed
    polynomials keep a nonzero constant after the monomial factors are pulled
    out (Sec. 2: sector functions are smooth on the closed cube), hence c0.
  * Draw order per problem: sizes, coefficients, variable indices, shifts.
  * Polynomial coefficients are rounded to the nearest float32 when drawn, so
    an FP32 evaluation and an FP64 evaluation integrate the identical
    integrand (rounding coefficients inside an FP32 kernel would otherwise
    move the integral by ~1e-7 relative).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def uniform_f32(self, lo: float, hi: float) -> float:
        """uniform_in rounded to the nearest float32 (exactly representable in both precisions)."""
        return float(np.float32(self.uniform_in(lo, hi)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] inclusive."""
        span = hi - lo + 1
        return lo + min(int(self.uniform() * span), span - 1)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def prev_prime(x: int) -> int:
    """Largest prime <= x (x >= 2)."""
    x = int(x)
    while not is_prime(x):
        x -= 1
    return x


def ladder_primes(e_lo: int = 20, e_hi: int = 52) -> List[int]:
    """Lattice-size ladder: the largest prime <= floor(2^(e/2)), e = e_lo..e_hi
    (2^10 .. 2^26 in sqrt(2) steps)."""
    return [prev_prime(math.isqrt(1 << e)) for e in range(e_lo, e_hi + 1)]


def batch_prime_table(count: int = 64, lo: float = 1e5, hi: float = 1e7) -> List[int]:
    """`count` log-spaced primes in [lo, hi]: largest prime <= lo (hi/lo)^(t/(count-1))."""
    out = []
    for t in range(count):
        v = int(math.floor(lo * (hi / lo) ** (t / (count - 1)) + 1e-9))
        out.append(prev_prime(v))
    return out


def pair_list(d: int):
    """All (i, j) with 0 <= i <= j < d in lexicographic order."""
    return [(i, j) for i in range(d) for j in range(i, d)]


def draw_indices(rng: SplitMix64, pool_size: int, count: int) -> List[int]:
    """`count` indices into a pool: partial Fisher-Yates without replacement
    while count <= pool_size, independent draws with replacement otherwise."""
    if count <= pool_size:
        pool = list(range(pool_size))
        for t in range(count):
            r = t + min(int(rng.uniform() * (pool_size - t)), pool_size - t - 1)
            pool[t], pool[r] = pool[r], pool[t]
        return pool[:count]
    return [min(int(rng.uniform() * pool_size), pool_size - 1) for _ in range(count)]


@dataclasses.dataclass
class Poly:
    """Polynomial as a term table: value = sum_t coef[t] * prod_i x_i^expo[t, i]."""
    coef: np.ndarray  # float64 [T]
    expo: np.ndarray  # uint8 [T, d]

    @property
    def nterms(self) -> int:
        return int(self.coef.shape[0])

    @property
    def degree(self) -> int:
        return int(self.expo.sum(axis=1).max()) if self.nterms else 0


@dataclasses.dataclass
class Problem:
    """One integration problem: lattice size, shift table, transform, integrand."""
    name: str
    d: int
    n: int
    m: int
    shifts: np.ndarray            # float64 [m, d] in [0, 1)
    transform: str                # "none" | "baker" | "korobov"
    alpha: int = 0                # Korobov weight
    kind: str = "sector"          # "const" | "separable_exp" | "sector" | "sector_deformed" | "trig"
    U: Optional[Poly] = None
    F: Optional[Poly] = None
    aU: int = -2
    aF: int = -1
    lam: float = 0.0
    c: Optional[np.ndarray] = None  # separable_exp: prod (1 + c_i z_i) exp(b_i z_i)
    b: Optional[np.ndarray] = None
    h: Optional[np.ndarray] = None  # trig: cos(2 pi h . z)
    precision: str = "fp64"         # "fp64" | "fp32"
    g: Optional[np.ndarray] = None  # generating vector (uint64 [d]) when attached
    gamma: Optional[np.ndarray] = None  # CBC product weights

    @property
    def evals(self) -> int:
        return self.n * self.m


def make_shifts(rng: SplitMix64, m: int, d: int) -> np.ndarray:
    return np.array([[rng.uniform() for _ in range(d)] for _ in range(m)], dtype=np.float64)


def random_poly(rng: SplitMix64, d: int, n_lin: int, n_quad: int, coef_lo=0.1, coef_hi=2.0,
                neg_quad: int = 0, neg_lo=-2.0, neg_hi=-0.5) -> Poly:
    """c0 + n_lin degree-1 monomials + n_quad degree-2 monomials.  The first
    `neg_quad` degree-2 coefficients are drawn from U(neg_lo, neg_hi)."""
    c0 = rng.uniform_f32(coef_lo, coef_hi)
    lin_c = [rng.uniform_f32(coef_lo, coef_hi) for _ in range(n_lin)]
    quad_c = [rng.uniform_f32(neg_lo, neg_hi) if t < neg_quad else rng.uniform_f32(coef_lo, coef_hi)
              for t in range(n_quad)]
    lin_v = draw_indices(rng, d, n_lin)
    pairs = pair_list(d)
    quad_v = [pairs[t] for t in draw_indices(rng, len(pairs), n_quad)]
    T = 1 + n_lin + n_quad
    coef = np.zeros(T, dtype=np.float64)
    expo = np.zeros((T, d), dtype=np.uint8)
    coef[0] = c0
    for t, (c, v) in enumerate(zip(lin_c, lin_v)):
        coef[1 + t] = c
        expo[1 + t, v] += 1
    for t, (c, (i, j)) in enumerate(zip(quad_c, quad_v)):
        coef[1 + n_lin + t] = c
        expo[1 + n_lin + t, i] += 1
        expo[1 + n_lin + t, j] += 1
    return Poly(coef, expo)


def product_weights(d: int) -> np.ndarray:
    """gamma_i = 1 / i^2, i = 1..d."""
    return np.array([1.0 / (i * i) for i in range(1, d + 1)], dtype=np.float64)


SEED_BASE = 0x5EED0000

N_C1 = 10007
N_C1_THROUGHPUT = 16777213
N_C2 = 16777213
N_C4 = 4194301
N_C5_MAX = 67108859
N_PILOT = 65537


def config1(n: int = N_C1, m: int = 10, seed: int = SEED_BASE + 1) -> Problem:
    """Plain rule, FP64: d=3, f = prod (1 + c_i x_i) exp(b_i x_i), c, b ~ U(0,1), Korobov 3."""
    rng = SplitMix64(seed)
    d = 3
    c = np.array([rng.uniform() for _ in range(d)])
    b = np.array([rng.uniform() for _ in range(d)])
    shifts = make_shifts(rng, m, d)
    return Problem("plain_fp64_separable_d3", d, n, m, shifts, "korobov", alpha=3,
                   kind="separable_exp", c=c, b=b, precision="fp64", gamma=product_weights(d))


def config2(n: int = N_C2, m: int = 32, seed: int = SEED_BASE + 2, precision: str = "fp32") -> Problem:
    """Single sector, FP32 evaluation / FP64 sums: d=6, U = c0 + 6 deg-1, F = c0 + 12 deg-2, baker."""
    rng = SplitMix64(seed)
    d = 6
    U = random_poly(rng, d, 6, 0)
    F = random_poly(rng, d, 0, 12)
    shifts = make_shifts(rng, m, d)
    return Problem("sector_fp32_d6", d, n, m, shifts, "baker", kind="sector", U=U, F=F,
                   aU=-2, aF=-1, precision=precision, gamma=product_weights(d))


def config3(count: int = 256, m: int = 16, seed: int = SEED_BASE + 3, transform: str = "baker",
            alpha: int = 0, precision: str = "fp32") -> List[Problem]:
    """Batched sectors: d ~ U{2..8}, T_U ~ U{4..10}, T_F ~ U{6..20}, n log-uniform in
    [1e5, 1e7] snapped to a 64-entry prime table, m = 16."""
    rng = SplitMix64(seed)
    table = batch_prime_table()
    lo, hi = math.log(1e5), math.log(1e7)
    probs = []
    for s in range(count):
        d = rng.randint(2, 8)
        tu = rng.randint(4, 10)
        tf = rng.randint(6, 20)
        v = math.exp(lo + (hi - lo) * rng.uniform())
        # snap to the largest table prime <= v (table[0] if v is below it)
        n = table[0]
        for p in table:
            if p <= v:
                n = p
        U = random_poly(rng, d, tu, 0)
        F = random_poly(rng, d, 0, tf)
        shifts = make_shifts(rng, m, d)
        probs.append(Problem(f"batch_sector_{s}", d, n, m, shifts, transform, alpha=alpha,
                             kind="sector", U=U, F=F, aU=-2, aF=-1, precision=precision,
                             gamma=product_weights(d)))
    return probs


def config3_shared(count: int = 32, d: int = 6, n: int = N_C2, m: int = 16, seed: int = SEED_BASE + 6,
                   transform: str = "baker", alpha: int = 0, precision: str = "fp32") -> List[Problem]:
    """Shared-lattice variant of configuration 3: `count` sectors of one dimension d
    on one lattice (n, m shifts) with configuration 3's term counts, T_U ~ U{4..10},
    T_F ~ U{6..20}; every problem carries the same shift table."""
    rng = SplitMix64(seed)
    shifts = make_shifts(rng, m, d)
    probs = []
    for s in range(count):
        tu = rng.randint(4, 10)
        tf = rng.randint(6, 20)
        U = random_poly(rng, d, tu, 0)
        F = random_poly(rng, d, 0, tf)
        probs.append(Problem(f"shared_sector_{s}", d, n, m, shifts, transform, alpha=alpha, kind="sector",
                             U=U, F=F, aU=-2, aF=-1, precision=precision, gamma=product_weights(d)))
    return probs


def config4(n: int = N_C4, m: int = 20, seed: int = SEED_BASE + 4, precision: str = "fp64",
            lam: float = 0.1) -> Problem:
    """Complex-valued sector: d=5, U = c0 + 5 deg-1, F = c0 + 10 deg-2 with 3 coefficients
    in U(-2,-0.5), contour deformation lambda = 0.1, Korobov 3."""
    rng = SplitMix64(seed)
    d = 5
    U = random_poly(rng, d, 5, 0)
    F = random_poly(rng, d, 0, 10, neg_quad=3)
    shifts = make_shifts(rng, m, d)
    return Problem("sector_deformed_d5", d, n, m, shifts, "korobov", alpha=3,
                   kind="sector_deformed", U=U, F=F, aU=-2, aF=-1, lam=lam,
                   precision=precision, gamma=product_weights(d))


def config5(n: int = N_C5_MAX, m: int = 16, seed: int = SEED_BASE + 5, precision: str = "fp32") -> Problem:
    """Control-variate sector: d=8, U = c0 + 8 deg-1, F = c0 + 24 deg-2, Korobov 3, m = 16."""
    rng = SplitMix64(seed)
    d = 8
    U = random_poly(rng, d, 8, 0)
    F = random_poly(rng, d, 0, 24)
    shifts = make_shifts(rng, m, d)
    return Problem("sector_cv_d8", d, n, m, shifts, "korobov", alpha=3, kind="sector",
                   U=U, F=F, aU=-2, aF=-1, precision=precision, gamma=product_weights(d))


def with_shifts(p: Problem, m: int, seed: int) -> Problem:
    """Same problem with a fresh shift table of m shifts from `seed`."""
    rng = SplitMix64(seed)
    return dataclasses.replace(p, m=m, shifts=make_shifts(rng, m, p.d))


def random_generating_vector(rng: SplitMix64, d: int, n: int) -> np.ndarray:
    """g_1 = 1 and g_i uniform in [1, n) (any such g is a valid lattice)."""
    g = [1] + [rng.randint(1, n - 1) for _ in range(d - 1)]
    return np.array(g, dtype=np.uint64)


def zbb_vertex_F() -> Poly:
    """Eq. (11): the Zbb vertex F / m_Z^2 in x0..x5 (16 monomials of degree 3)."""
    terms = [
        (+1, {3: 2, 5: 1}), (+1, {3: 2, 4: 1}), (+1, {2: 1, 3: 1, 5: 1}), (+1, {2: 1, 3: 1, 4: 1}),
        (+1, {1: 1, 3: 1, 5: 1}), (+1, {1: 1, 3: 1, 4: 1}), (+1, {1: 1, 3: 2}), (+1, {1: 1, 2: 1, 3: 1}),
        (+1, {0: 1, 3: 1, 4: 1}), (+1, {0: 1, 3: 2}), (+1, {0: 1, 2: 1, 3: 1}),
        (-1, {1: 1, 2: 1, 4: 1}), (-1, {0: 1, 1: 1, 5: 1}), (-1, {0: 1, 1: 1, 4: 1}),
        (-1, {0: 1, 1: 1, 2: 1}), (-1, {0: 1, 1: 1, 3: 1}),
    ]
    coef = np.array([c for c, _ in terms], dtype=np.float64)
    expo = np.zeros((len(terms), 6), dtype=np.uint8)
    for t, (_, e) in enumerate(terms):
        for i, k in e.items():
            expo[t, i] = k
    return Poly(coef, expo)
