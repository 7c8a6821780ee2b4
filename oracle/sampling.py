"""Autoregressive sampling without replacement (oracle; test infrastructure).

Alg. 1 (ARGumbelTopK) of Sec. "Autoregressive sampling without replacement":
the partially sampled vectors x_<i keep their log-probability l and their
conditioned perturbed log-probability L~; per qubit each is extended by
x_i = 0 and 1 with l' = l + log p_i(x_i | x_<i), the unconditioned perturbed
value L' = l' + G (G a Gumbel(0) draw), Z = max of the two L', and the
conditioned value L~' = -log(exp(-L~) - exp(-Z) + exp(-L')); the extended
vectors are sorted by L~' in descending order and the first K kept.

The random numbers the method draws are inputs: ``gumbel[level]`` holds the
G values of that level, two per kept vector (x_i = 0 first, then 1, vectors
in the order they are kept).  The conditional log-probabilities come from the
caller's ansatz, ``cond_logp(level, prefixes) -> [(log p(0|x), log p(1|x))]``.

Readings (stated in the design notes): an extension with log-probability
-inf (an impossible outcome, e.g. outside the particle-number sector) is not
kept; the sort is stable, so equal L~' keep the order of the extensions
(vector order, x_i = 0 before 1).  The conditioned value is evaluated in an
algebraically identical form that keeps its digits: with T = L~ of the
parent, exp(-T) - exp(-Z) + exp(-L') = exp(-T) (1 + exp(T - Z) expm1(Z - L')),
so L~' = T - softplus(T - Z + log(expm1(Z - L'))) for L' < Z and L~' = T for
the larger extension (L' = Z); printed literally the expression cancels
exp(-Z) against exp(-L') and loses exp(-T) entirely once Z is far below T.
Bit vectors are Python ints (bit i = qubit i); arithmetic in FP64 with
``math``.
"""

import math


def conditioned_value(lt, Z, L):
    """L~' = -log(exp(-lt) - exp(-Z) + exp(-L)) in the form above."""
    if L >= Z:
        return lt
    v = (lt - Z) + math.log(math.expm1(Z - L))
    softplus = max(v, 0.0) + math.log1p(math.exp(-abs(v)))
    return lt - softplus


def ar_gumbel_topk(n_qubits: int, K: int, cond_logp, gumbel):
    """Alg. 1: returns [(x, l, L~)] in descending L~ after the last qubit."""
    kept = [(0, 0.0, 0.0)]
    for i in range(n_qubits):
        lp = cond_logp(i, [x for (x, _, _) in kept])
        g = gumbel[i]
        ext = []
        for p, (x, l, lt) in enumerate(kept):
            lc = [l + lp[p][0], l + lp[p][1]]
            L = [lc[0] + g[2 * p], lc[1] + g[2 * p + 1]]
            Z = max(L)
            for xi in (0, 1):
                if lc[xi] == -math.inf:
                    continue
                lt_c = conditioned_value(lt, Z, L[xi])
                ext.append((x | (xi << i), lc[xi], lt_c))
        ext.sort(key=lambda e: -e[2])
        kept = ext[:K]
    return kept
