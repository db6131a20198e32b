"""The Bernoulli(p) coin theta_k of Algorithms 4 and 6 (FP64 oracle).

The paper draws theta_k with Prob(theta_k = 1) = p once per outer iteration and does
not name a generator.  Both sides of this project use the counter-based generator
Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), which each implements from its
published definition:

* state: four 64-bit counter words c and two 64-bit key words k;
* one round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 128-bit products),
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is bumped by
  the Weyl constants (k0 += W0, k1 += W1) mod 2^64;
* ten rounds.

The coin of outer iteration k for a problem with seed S is
theta_k = [ (w >> 11) < p * 2^53 ], w = first output word of
Philox4x64-10(counter = (k, 0, 0, 0), key = (S, 0)).  The comparison is exact in
double precision (p * 2^53 only scales the exponent), so p = 1 always gives 1 and the
schedule depends on (S, p, k) only: it is drawn on skipped iterations too.
"""

from __future__ import annotations

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(counter, key):
    """Ten-round Philox4x64 block for a 4-word counter and 2-word key (Python ints)."""
    c = [int(x) & MASK64 for x in counter]
    k = [int(x) & MASK64 for x in key]
    for rnd in range(10):
        if rnd > 0:
            k = [(k[0] + PHILOX_W0) & MASK64, (k[1] + PHILOX_W1) & MASK64]
        prod0 = PHILOX_M0 * c[0]
        prod1 = PHILOX_M1 * c[2]
        hi0, lo0 = prod0 >> 64, prod0 & MASK64
        hi1, lo1 = prod1 >> 64, prod1 & MASK64
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return c


def coin(seed: int, p: float, k: int) -> int:
    """theta_k in {0, 1} for problem seed ``seed`` and probability ``p``."""
    if not (0.0 < p <= 1.0):
        raise ValueError("p must lie in (0, 1]")
    w = philox4x64_10((k, 0, 0, 0), (seed, 0))[0]
    return 1 if (w >> 11) < p * 9007199254740992.0 else 0


def schedule(seed: int, p: float, K: int):
    """[theta_0, ..., theta_{K-1}]."""
    return [coin(seed, p, k) for k in range(K)]
