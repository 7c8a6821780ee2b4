"""Autoregressive sampling without replacement (Alg. 1) on the GPU against the oracle.

The same conditional log-probabilities (a seeded toy autoregressive model,
with and without a particle-number sector) and the same Gumbel draws go to
the oracle and to nqs_gumbel_topk_level; the sampled vectors must be the
oracle's, in the oracle's order (the L~ ordering is an exact FP64 decision on
both sides, with ties kept in extension order), with l and L~ within 1e-12
relative.  Covers K below, at and above the number of extensions, 70 and 130
qubits (two and three words), and a batch of 10^5 kept vectors.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from oracle.sampling import conditioned_value
from synth import ToyAutoregressive, gumbel_noise

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs


def _ints(x, W):
    words = x.cpu().numpy().view(np.uint64).reshape(-1, W)
    return [sum(int(r[w]) << (64 * w) for w in range(W)) for r in words]


@pytest.mark.parametrize("n,K,ne,seed", [(6, 64, None, 1), (10, 37, None, 2), (12, 200, 4, 3), (20, 1000, 6, 4),
                                          (70, 300, 10, 5), (130, 64, None, 6)])
def test_matches_oracle(n, K, ne, seed):
    model = ToyAutoregressive(n, seed, n_electrons=ne)
    rng = np.random.default_rng(seed)
    noise = [gumbel_noise(rng, 2 * min(K, 2 ** min(i, 40))) for i in range(n)]
    want = oracle.ar_gumbel_topk(n, K, model.cond_logp, noise)
    x, l, lt = nqs.ar_gumbel_topk(n, K, model.cond_logp, noise)
    W = (n + 63) // 64
    got = _ints(x, W)
    assert got == [w[0] for w in want]
    wl = np.array([w[1] for w in want]); wt = np.array([w[2] for w in want])
    assert np.all(np.abs(l.cpu().numpy() - wl) <= 1e-12 * np.maximum(1.0, np.abs(wl)))
    assert np.all(np.abs(lt.cpu().numpy() - wt) <= 1e-12 * np.maximum(1.0, np.abs(wt)))
    if ne is not None:
        assert all(bin(v).count("1") == ne for v in got)


def test_one_level_large_batch():
    """One qubit with 10^5 kept vectors (2 x 10^5 extensions, several sort tiles)."""
    n_par, K, level = 100_000, 70_000, 30
    rng = np.random.default_rng(9)
    px = rng.integers(0, 1 << 30, n_par, dtype=np.int64)
    pl = rng.normal(-20.0, 3.0, n_par)
    plt = pl + rng.gumbel(0.0, 1.0, n_par)
    lp = np.log(rng.dirichlet([1.0, 1.0], n_par))
    lp[rng.random(n_par) < 0.05, 1] = -np.inf
    g = rng.gumbel(0.0, 1.0, (n_par, 2))
    cx, cl, clt = nqs.gumbel_topk_level(40, level, torch.from_numpy(px[:, None]).cuda(), pl, plt, lp, g, K)
    # the oracle's step for one qubit, on the same parents
    ext = []
    for p in range(n_par):
        lc = [pl[p] + lp[p, 0], pl[p] + lp[p, 1]]
        L = [lc[0] + g[p, 0], lc[1] + g[p, 1]]
        Z = max(L)
        for xi in (0, 1):
            if lc[xi] == -math.inf:
                continue
            ext.append((int(px[p]) | (xi << level), lc[xi], conditioned_value(plt[p], Z, L[xi])))
    ext.sort(key=lambda e: -e[2])
    ext = ext[:K]
    assert cx.shape[0] == K
    assert cx[:, 0].cpu().numpy().tolist() == [e[0] for e in ext]
    assert np.abs(clt.cpu().numpy() - np.array([e[2] for e in ext])).max() <= 1e-11
