"""Autoregressive sampling without replacement (Alg. 1) on the GPU against the oracle.

The same conditional log-probabilities (a seeded toy autoregressive model,
with and without a particle-number sector) and the same Gumbel draws go to
the oracle and to nqs_gumbel_topk_level; the sampled vectors must be the
oracle's, in the oracle's order (the L~ ordering is an exact FP64 decision on
both sides, with ties kept in extension order), with l and L~ within 1e-12
relative.  Covers K below, at and above the number of extensions, 70 and 130
qubits (two and three words), one level of 10^5 kept vectors with parents in
L~ order and in arbitrary order (the bucket path), and a level whose equal
values overfill a bucket (the general radix-sort path).
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


def _one_level_oracle(px, pl, plt, lp, g, level, K):
    """The oracle's step for one qubit (the body of Alg. 1's loop), on the given parents."""
    ext = []
    for p in range(len(pl)):
        lc = [pl[p] + lp[p, 0], pl[p] + lp[p, 1]]
        L = [lc[0] + g[p, 0], lc[1] + g[p, 1]]
        Z = max(L)
        for xi in (0, 1):
            if lc[xi] == -math.inf:
                continue
            ext.append((int(px[p]) | (xi << level), lc[xi], conditioned_value(plt[p], Z, L[xi])))
    ext.sort(key=lambda e: -e[2])
    return ext[:K]


@pytest.mark.parametrize("K", [70_000, 300_000])
def test_one_level_sorted_parents(K):
    """10^5 parents in L~-descending order (the previous level's output), with
    runs of equal L~ among parents, equal perturbed values of both extensions
    (so both keep L~) and impossible outcomes."""
    n_par, level = 100_000, 31
    rng = np.random.default_rng(19)
    px = rng.integers(0, 1 << 31, n_par, dtype=np.int64)
    pl = rng.normal(-20.0, 3.0, n_par)
    plt = np.sort(pl + rng.gumbel(0.0, 1.0, n_par))[::-1].copy()
    plt[1000:1040] = plt[1000]
    plt[5000:5003] = plt[5000]
    lp = np.log(rng.dirichlet([1.0, 1.0], n_par))
    lp[rng.random(n_par) < 0.05, 1] = -np.inf
    g = rng.gumbel(0.0, 1.0, (n_par, 2))
    tie = rng.random(n_par) < 0.01
    g[tie, 1] = (pl[tie] + lp[tie, 0] + g[tie, 0]) - (pl[tie] + lp[tie, 1])
    g[~np.isfinite(g)] = 0.0
    want = _one_level_oracle(px, pl, plt, lp, g, level, K)
    cx, cl, clt = nqs.gumbel_topk_level(40, level, torch.from_numpy(px[:, None]).cuda(), pl, plt, lp, g, K)
    assert cx.shape[0] == len(want)
    assert cx[:, 0].cpu().numpy().tolist() == [e[0] for e in want]
    assert np.abs(cl.cpu().numpy() - np.array([e[1] for e in want])).max() <= 1e-12 * 40
    assert np.abs(clt.cpu().numpy() - np.array([e[2] for e in want])).max() <= 1e-11


def test_one_level_all_values_equal():
    """20,000 parents with one L~ and both extensions equally perturbed: all
    40,000 extensions keep that L~, so the order is the extension order (one
    bucket would hold them all: the general path takes over)."""
    n_par, level, K = 20_000, 15, 30_000
    rng = np.random.default_rng(29)
    px = rng.integers(0, 1 << 15, n_par, dtype=np.int64)
    pl = np.full(n_par, -7.0)
    plt = np.full(n_par, -6.5)
    lp = np.full((n_par, 2), math.log(0.5))
    g = np.repeat(rng.gumbel(0.0, 1.0, (n_par, 1)), 2, axis=1)
    want = _one_level_oracle(px, pl, plt, lp, g, level, K)
    cx, cl, clt = nqs.gumbel_topk_level(20, level, torch.from_numpy(px[:, None]).cuda(), pl, plt, lp, g, K)
    assert cx[:, 0].cpu().numpy().tolist() == [e[0] for e in want]
    assert np.all(clt.cpu().numpy() == -6.5)


def test_one_level_parent_without_outcomes():
    """A parent with both outcomes impossible: nothing of it is kept."""
    n_par, level, K = 5000, 12, 6000
    rng = np.random.default_rng(23)
    px = rng.integers(0, 1 << 12, n_par, dtype=np.int64)
    pl = rng.normal(-10.0, 2.0, n_par)
    plt = np.sort(pl + rng.gumbel(0.0, 1.0, n_par))[::-1].copy()
    lp = np.log(rng.dirichlet([1.0, 1.0], n_par))
    lp[17] = -np.inf
    g = rng.gumbel(0.0, 1.0, (n_par, 2))
    want = _one_level_oracle(px, pl, plt, lp, g, level, K)
    cx, cl, clt = nqs.gumbel_topk_level(20, level, torch.from_numpy(px[:, None]).cuda(), pl, plt, lp, g, K)
    assert cx[:, 0].cpu().numpy().tolist() == [e[0] for e in want]
    assert np.abs(clt.cpu().numpy() - np.array([e[2] for e in want])).max() <= 1e-11


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


def _table_run_async(n_qubits, K, lp_tab, g_tab, graph=False):
    """All levels through the device-count form (counts chained on the device),
    optionally captured once in a CUDA graph and replayed."""
    dev = "cuda"
    W = (n_qubits + 63) // 64
    lp = torch.from_numpy(lp_tab).to(dev)
    G = torch.from_numpy(g_tab).to(dev)
    lib = nqs.load_library()
    scratch = torch.empty(int(lib.nqs_gumbel_scratch_bytes(K)), dtype=torch.uint8, device=dev)
    bufs = [(torch.zeros((K, W), dtype=torch.int64, device=dev), torch.zeros(K, dtype=torch.float64, device=dev),
             torch.zeros(K, dtype=torch.float64, device=dev)) for _ in range(2)]
    counts = torch.zeros((n_qubits, 2), dtype=torch.int64, device=dev)
    one = torch.ones(1, dtype=torch.int64, device=dev)
    zero = torch.zeros(1, dtype=torch.float64, device=dev)

    def run():
        x, l, lt, n_dev, max_n = None, zero, zero, one, 1
        for i in range(n_qubits):
            out = bufs[i & 1]
            nqs.gumbel_topk_level_async(n_qubits, i, max_n, n_dev, x, l, lt, lp[i], G[i], K, out, scratch, counts[i])
            x, l, lt, n_dev = out[0], out[1], out[2], counts[i]
            max_n = min(K, 2 * max_n)

    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            run()   # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run()
        for b in bufs:
            for t in b:
                t.zero_()
        g.replay()
    else:
        run()
    torch.cuda.synchronize()
    k = int(counts[-1, 0].item())
    last = bufs[(n_qubits - 1) & 1]
    return last[0][:k].clone(), last[1][:k].clone(), last[2][:k].clone(), counts.cpu().numpy()


@pytest.mark.parametrize("graph", [False, True])
def test_device_count_form_matches_oracle(graph):
    """Levels chained on the device (and replayed from one CUDA graph): the
    oracle's samples in the oracle's order, for conditional log-probabilities
    given as a table (row r for the r-th kept prefix) with impossible outcomes."""
    n, K = 14, 300
    rng = np.random.default_rng(31)
    z = rng.normal(0.0, 2.0, (n, K))
    lp_tab = np.stack([-np.logaddexp(0.0, -z), -np.logaddexp(0.0, z)], axis=2)
    lp_tab[rng.random((n, K, 2)) < 0.03] = -np.inf
    g_tab = rng.gumbel(0.0, 1.0, (n, K, 2))
    want = oracle.ar_gumbel_topk(n, K, lambda i, pre: lp_tab[i, :len(pre)].tolist(),
                                 [g_tab[i].reshape(-1).tolist() for i in range(n)])
    x, l, lt, counts = _table_run_async(n, K, lp_tab, g_tab, graph=graph)
    assert np.all(counts[:, 1] == 1)
    assert _ints(x, 1) == [w[0] for w in want]
    wt = np.array([w[2] for w in want])
    assert np.all(np.abs(lt.cpu().numpy() - wt) <= 1e-12 * np.maximum(1.0, np.abs(wt)))


def test_device_count_form_equals_synchronous_form():
    """56 levels keeping 2 x 10^4 vectors: the device-count form and the
    synchronous form give the same children, bit for bit."""
    n, K = 56, 20_000
    rng = np.random.default_rng(37)
    z = rng.normal(0.0, 2.0, (n, K))
    lp_tab = np.stack([-np.logaddexp(0.0, -z), -np.logaddexp(0.0, z)], axis=2)
    g_tab = rng.gumbel(0.0, 1.0, (n, K, 2))
    xa, la, lta, counts = _table_run_async(n, K, lp_tab, g_tab)
    assert np.all(counts[:, 1] == 1)
    lp = torch.from_numpy(lp_tab).cuda()
    G = torch.from_numpy(g_tab).cuda()
    x, l, lt = None, torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(1, dtype=torch.float64,
                                                                                      device="cuda")
    for i in range(n):
        m = int(l.shape[0])
        x, l, lt = nqs.gumbel_topk_level(n, i, x, l, lt, lp[i, :m], G[i, :m], K)
    assert torch.equal(x, xa) and torch.equal(l, la) and torch.equal(lt, lta)


def test_device_count_form_reports_overflow():
    """A level whose extensions all share one value overfills a bucket: the
    device-count form keeps nothing there and says so in its status."""
    n_par, K = 20_000, 30_000
    dev = "cuda"
    rng = np.random.default_rng(41)
    px = torch.from_numpy(rng.integers(0, 1 << 15, n_par, dtype=np.int64)[:, None]).to(dev)
    pl = torch.full((n_par,), -7.0, dtype=torch.float64, device=dev)
    plt = torch.full((n_par,), -6.5, dtype=torch.float64, device=dev)
    lp = torch.full((n_par, 2), math.log(0.5), dtype=torch.float64, device=dev)
    g = torch.from_numpy(np.repeat(rng.gumbel(0.0, 1.0, (n_par, 1)), 2, axis=1)).to(dev)
    lib = nqs.load_library()
    scratch = torch.empty(int(lib.nqs_gumbel_scratch_bytes(n_par)), dtype=torch.uint8, device=dev)
    out = (torch.zeros((K, 1), dtype=torch.int64, device=dev), torch.zeros(K, dtype=torch.float64, device=dev),
           torch.zeros(K, dtype=torch.float64, device=dev))
    counts = torch.full((2,), 7, dtype=torch.int64, device=dev)
    n_dev = torch.tensor([n_par], dtype=torch.int64, device=dev)
    nqs.gumbel_topk_level_async(20, 15, n_par, n_dev, px, pl, plt, lp, g, K, out, scratch, counts)
    assert counts.cpu().tolist() == [0, 0]
