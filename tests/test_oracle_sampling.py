"""The oracle's ARGumbelTopK (Alg. 1) pinned by what sampling without
replacement must produce, not by its own formula.

* K at least the number of possible outcomes: every outcome with p > 0 is
  returned exactly once (sampling without replacement exhausts the space).
* The particle-number sector: with zero probability outside it, every
  returned vector has the electron count and min(K, C(N, N_e)) are returned.
* Bounding property of the top-down construction: the kept extension with
  the larger unconditioned perturbed value inherits its parent's L~ (to
  rounding), the other one's L~ is below it.
* Gumbel-max trick: with K = 1 the returned vector is distributed as p(x)
  (empirical frequencies over 6000 seeded draws against the model's p(x)).
* Without replacement: with K = 2 the first two returned vectors (a, b)
  occur with probability p(a) p(b) / (1 - p(a)) (Eq. renorm_prob).
* A planted mistake (the unconditioned value kept instead of the
  conditioned one) breaks the without-replacement law.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from synth import ToyAutoregressive, gumbel_noise


def _draw(model, K, rng):
    """One run with fresh noise: level i gets 2 min(K, 2^i) Gumbel values (the widest it can need)."""
    g = [gumbel_noise(rng, 2 * min(K, 2 ** i)) for i in range(model.n)]
    return oracle.ar_gumbel_topk(model.n, K, model.cond_logp, g)


def test_exhausts_the_space():
    model = ToyAutoregressive(5, 1)
    out = _draw(model, 64, np.random.default_rng(0))
    assert sorted(x for x, _, _ in out) == list(range(32))
    for x, l, lt in out:
        assert abs(l - model.log_prob(x)) < 1e-12
    lts = [lt for _, _, lt in out]
    assert lts == sorted(lts, reverse=True)


def test_sector():
    model = ToyAutoregressive(8, 2, n_electrons=3)
    for K in (10, 56, 100):
        out = _draw(model, K, np.random.default_rng(K))
        assert len(out) == min(K, math.comb(8, 3))
        assert all(bin(x).count("1") == 3 for x, _, _ in out)
        assert len({x for x, _, _ in out}) == len(out)


def test_bounding_property():
    """Run the oracle for 1, 2, ..., N qubits on the same noise: every kept
    prefix's L~ equals the largest L~ among its two extensions one level on."""
    model = ToyAutoregressive(6, 3)
    rng = np.random.default_rng(5)
    noise = [gumbel_noise(rng, 2 * 2 ** i) for i in range(model.n)]
    prev = oracle.ar_gumbel_topk(1, 10 ** 6, model.cond_logp, noise)
    for n in range(2, model.n + 1):
        cur = oracle.ar_gumbel_topk(n, 10 ** 6, model.cond_logp, noise)
        by_parent = {}
        for x, l, lt in cur:
            by_parent.setdefault(x & ((1 << (n - 1)) - 1), []).append(lt)
        for x, l, lt in prev:
            kids = by_parent[x]
            assert abs(max(kids) - lt) <= 1e-12 * max(1.0, abs(lt))
            assert min(kids) <= lt
        prev = cur


def test_conditioned_value_is_the_printed_expression():
    """The stable form equals -log(exp(-T) - exp(-Z) + exp(-L)) evaluated with 50 digits,
    also where FP64 evaluation of the printed form loses every digit (Z far below T)."""
    import mpmath
    mpmath.mp.dps = 50
    rng = np.random.default_rng(23)
    from oracle.sampling import conditioned_value
    cases = [(-3.4657359027997265, -40.97809828410075, -48.8)]   # the printed form gives log(0) here
    for _ in range(400):
        T = rng.uniform(-60, 20)
        Z = T - rng.exponential(rng.choice([0.01, 1.0, 30.0]))
        L = Z - rng.exponential(rng.choice([1e-9, 0.1, 3.0, 50.0]))
        cases.append((T, Z, L))
    for T, Z, L in cases:
        exact = -mpmath.log(mpmath.exp(-mpmath.mpf(T)) - mpmath.exp(-mpmath.mpf(Z)) + mpmath.exp(-mpmath.mpf(L)))
        got = conditioned_value(T, Z, L)
        assert abs(got - float(exact)) <= 1e-13 * max(1.0, abs(float(exact))), (T, Z, L, got, float(exact))
    assert conditioned_value(1.5, -2.0, -2.0) == 1.5


def test_gumbel_max_frequencies():
    model = ToyAutoregressive(3, 7, scale=1.0)
    p = np.array([math.exp(model.log_prob(x)) for x in range(8)])
    rng = np.random.default_rng(11)
    M = 6000
    cnt = np.zeros(8)
    for _ in range(M):
        out = _draw(model, 1, rng)
        cnt[out[0][0]] += 1
    freq = cnt / M
    sigma = np.sqrt(p * (1 - p) / M)
    assert np.all(np.abs(freq - p) < 4.5 * sigma + 1e-3), (freq, p)


def _pair_law(draw_fn):
    model = ToyAutoregressive(3, 13, scale=1.2)
    p = np.array([math.exp(model.log_prob(x)) for x in range(8)])
    rng = np.random.default_rng(17)
    M = 20000
    cnt = {}
    for _ in range(M):
        out = draw_fn(model, rng)
        key = (out[0][0], out[1][0])
        cnt[key] = cnt.get(key, 0) + 1
    worst = 0.0
    for a, b in itertools.permutations(range(8), 2):
        want = p[a] * p[b] / (1.0 - p[a])
        got = cnt.get((a, b), 0) / M
        worst = max(worst, abs(got - want) / math.sqrt(want * (1 - want) / M))
    return worst


def test_without_replacement_law():
    assert _pair_law(lambda model, rng: _draw(model, 2, rng)) < 4.5


def test_planted_unconditioned_value_breaks_the_law(monkeypatch):
    def mutant(n_qubits, K, cond_logp, gumbel):
        kept = [(0, 0.0, 0.0)]
        for i in range(n_qubits):
            lp = cond_logp(i, [x for (x, _, _) in kept])
            g = gumbel[i]
            ext = []
            for p, (x, l, lt) in enumerate(kept):
                for xi in (0, 1):
                    lc = l + lp[p][xi]
                    ext.append((x | (xi << i), lc, lc + g[2 * p + xi]))   # L' instead of L~'
            ext.sort(key=lambda e: -e[2])
            kept = ext[:K]
        return kept
    monkeypatch.setattr(oracle, "ar_gumbel_topk", mutant)
    assert _pair_law(lambda model, rng: _draw(model, 2, rng)) > 4.5
