"""A seeded toy autoregressive model: conditional log-probabilities as inputs.

The sampler (Alg. 1) consumes log p_i(x_i | x_<i) from the caller's ansatz.
This stand-in makes them from a logistic model with pairwise couplings,
logit_i = b_i + sum_{j<i} w_ij x_j, and can restrict the samples to a
particle-number sector (probability zero once the remaining qubits can no
longer reach, or would exceed, the electron count), as the paper's ansatz
does for (N_e, S_z).  It holds none of the method's arithmetic.
"""

import math

import numpy as np


class ToyAutoregressive:
    def __init__(self, n_qubits: int, seed: int, n_electrons: int = None, scale: float = 1.5):
        rng = np.random.default_rng(seed)
        self.n = int(n_qubits)
        self.b = rng.normal(0.0, scale, self.n)
        self.w = np.tril(rng.normal(0.0, scale / 2, (self.n, self.n)), -1)
        self.ne = n_electrons

    def cond_logp(self, level: int, prefixes):
        """[(log p(x_level = 0 | x_<level), log p(1 | x_<level))] for each prefix (int bit vectors)."""
        out = []
        for x in prefixes:
            bits = np.array([(x >> j) & 1 for j in range(level)], dtype=np.float64)
            z = self.b[level] + float(self.w[level, :level] @ bits) if level else self.b[level]
            lp1 = -math.log1p(math.exp(-z)) if z > -700 else z
            lp0 = -math.log1p(math.exp(z)) if z < 700 else -z
            if self.ne is not None:
                ones = int(bits.sum())
                left = self.n - level - 1           # qubits after this one
                if ones + 1 > self.ne:             # a 1 here would exceed the count
                    lp0, lp1 = 0.0, -math.inf
                elif ones + left < self.ne:        # a 0 here could not reach the count
                    lp0, lp1 = -math.inf, 0.0
            out.append((lp0, lp1))
        return out

    def log_prob(self, x: int) -> float:
        """log p(x) = sum_i log p_i(x_i | x_<i)."""
        tot = 0.0
        for i in range(self.n):
            lp = self.cond_logp(i, [x & ((1 << i) - 1)])[0]
            tot += lp[(x >> i) & 1]
        return tot


def gumbel_noise(rng, size):
    """Gumbel(0) draws by inverse transform of uniform numbers: G = -log(-log U)."""
    u = rng.random(size)
    u = np.where(u == 0.0, np.nextafter(0.0, 1.0), u)
    return -np.log(-np.log(u))
