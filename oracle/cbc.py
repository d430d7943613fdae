"""Fast component-by-component generating-vector search (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The criterion is the one the plain C search uses (``orc_cbc_plain``): the
shift-averaged worst-case error of a rank-1 lattice in the unanchored weighted
Sobolev space with product weights,
    e^2(g) = -1 + (1/n) sum_{k=0}^{n-1} prod_i (1 + gamma_i B2({k g_i / n})),
    B2(t) = t^2 - t + 1/6.
For prime n the candidate-by-point matrix B2({k z / n}) becomes circulant once
z and k are ordered by powers of a primitive root, so all candidates of one
dimension come from one cyclic convolution (Nuyens and Cools, Math. Comp. 2006).
numpy's FFT serves as that convolution; nothing else is reordered.
The FFT's rounding noise (~1e-16 n) can exceed the gaps between the best
candidates at large n, so the RERANK candidates with the smallest convolution
values are re-evaluated exactly, T(z) = sum_k p[k] B2({k z / n}) by the
oracle's compensated sum (the plain search's own criterion), and the smallest
T wins, ties to the smallest z.
"""
from __future__ import annotations

import numpy as np


def _factor(n: int):
    f, p = [], 2
    while p * p <= n:
        if n % p == 0:
            f.append(p)
            while n % p == 0:
                n //= p
        p += 1
    if n > 1:
        f.append(n)
    return f


def primitive_root(n: int) -> int:
    """Smallest generator of the multiplicative group mod the prime n."""
    if n == 2:
        return 1
    fac = _factor(n - 1)
    for w in range(2, n):
        if all(pow(w, (n - 1) // q, n) != 1 for q in fac):
            return w
    raise ValueError("no primitive root (n not prime?)")


def _powers(w: int, n: int, count: int) -> np.ndarray:
    """w^t mod n for t = 0..count-1, exact in int64 (n < 2^31)."""
    B = 1 << 12
    small = np.empty(B, dtype=np.int64)
    v = 1
    for t in range(B):
        small[t] = v
        v = v * w % n
    wB = v  # w^B
    nblk = (count + B - 1) // B
    big = np.empty(nblk, dtype=np.int64)
    v = 1
    for q in range(nblk):
        big[q] = v
        v = v * wB % n
    out = (big[:, None] * small[None, :]) % n
    return out.reshape(-1)[:count]


def _b2(t):
    return t * t - t + 1.0 / 6.0


RERANK = 32


def cbc_fast(d: int, n: int, gamma) -> np.ndarray:
    """CBC generating vector for prime n < 2^31 (g_1 = 1)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    if n < 5:
        raise ValueError("n must be a prime >= 5")
    g = [1]
    k = np.arange(n, dtype=np.int64)
    p = 1.0 + gamma[0] * _b2(k / n)
    if d == 1:
        return np.array(g, dtype=np.uint64)
    w = primitive_root(n)
    h = (n - 1) // 2
    perm = _powers(w, n, n - 1)                  # perm[t] = w^t mod n
    c = _b2(perm[:h] / n)                         # B2 is even about 1/2 and w^h = -1: period h
    M = 1
    while M < 2 * h - 1:
        M <<= 1
    c_hat = np.fft.rfft(c, M)
    # -b mod (n-1) for b = 0..n-2 gives k = w^(-b)
    neg = (-np.arange(n - 1, dtype=np.int64)) % (n - 1)
    kk = perm[neg]
    cand = np.minimum(perm[:h], n - perm[:h])     # z and n-z give the same error
    for s in range(1, d):
        q = p[kk]
        qf = q[:h] + q[h:2 * h]
        lin = np.fft.irfft(c_hat * np.fft.rfft(qf, M), M)
        T = lin[:h].copy()
        T[: M - h if M - h < h else h] += lin[h:2 * h][: min(h, M - h)]
        K = min(RERANK, h)
        top = np.argpartition(T, K - 1)[:K]
        from . import cbc_candidate
        pc = np.ascontiguousarray(p)
        best_t, z = None, None
        for zc in sorted(set(int(v) for v in cand[top])):
            tz = cbc_candidate(n, pc, zc)
            if best_t is None or tz < best_t:
                best_t, z = tz, zc
        g.append(z)
        p = p * (1.0 + gamma[s] * _b2(((k * z) % n) / n))
    return np.array(g, dtype=np.uint64)
