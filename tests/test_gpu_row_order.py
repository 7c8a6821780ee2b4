"""Row sums that do not depend on the order of a row's pairs (GPU required).

E_loc^var(x) = sum_j H_xj psi(x_j)/psi(x) (Eq. local_energy restricted to U)
and the adjoint's row sums are sums over a SET of pairs.  The library adds
each row's terms as exact fixed-point integers and rounds once, so a row's
result must be bitwise the same whatever order its pairs are listed in:

* the canonical lists (diagonal pair first, then ascending column);
* the lists as the LoopOverTerms search placed them (NQS_ROWS_UNSORTED: no
  row sort), which must hold the same pairs row by row;
* each row's pairs shuffled at random on the host.

Cases: a molecular 28-qubit batch (real H, real and complex log psi), a
random complex Hamiltonian (odd |Y|), and the star instance whose hub row is
long enough to be reduced by a whole block.  Both precisions; the adjoint
with stored and with recomputed matrix elements.
"""

import numpy as np
import pytest
import torch

from synth import config_instance, pack_ints, random_pauli_hamiltonian

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects


def _rows(pairs):
    rp, pj, pk = pairs
    rp = rp.cpu().numpy()
    j = pj.cpu().numpy().view(np.uint32).astype(np.int64)
    k = pk.cpu().numpy().view(np.uint32).astype(np.int64)
    return rp, j, k


def _shuffled(pairs, has_diag, seed):
    """The same CSR with every row's non-diagonal pairs in a random order."""
    rp, j, k = _rows(pairs)
    rng = np.random.default_rng(seed)
    perm = np.arange(len(j))
    for r in range(len(rp) - 1):
        a, b = rp[r] + (1 if has_diag and rp[r + 1] > rp[r] else 0), rp[r + 1]
        perm[a:b] = a + rng.permutation(b - a)
    dev = pairs[1].device
    return (pairs[0], torch.from_numpy(j[perm].astype(np.uint32).view(np.int32)).to(dev),
            torch.from_numpy(k[perm].astype(np.uint32).view(np.int32)).to(dev))


def _same_sets(sorted_pairs, other, has_diag, row_begin=0):
    rp, j, k = _rows(sorted_pairs)
    rq, j2, k2 = _rows(other)
    assert np.array_equal(rp, rq)
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        if has_diag and b > a:  # the diagonal pair leads the row in both
            assert j2[a] == row_begin + r and k2[a] == 0
            a += 1
        o = np.lexsort((k2[a:b], j2[a:b]))
        assert np.array_equal(j[a:b], j2[a:b][o]) and np.array_equal(k[a:b], k2[a:b][o])


def _run(batch, lre, lim, pairs, prec, g_re, g_im, store_h):
    hp = None
    n = int(pairs[1].numel())
    if store_h:
        hp = nqs.pair_h_buffer(n, prec, "cuda", batch.ham.complex)
    er, ei, hd = nqs.local_energy(batch, lre, lim, pairs, prec, hpair=hp)
    ev = nqs.variational_energy(batch, lre, er)
    gr, gi = nqs.local_energy_backward(batch, lre, lim, er, ei, hd, ev, g_re, g_im, None, pairs, prec, hpair=hp)
    batch.status()  # no device index or range check fired
    out = [er, hd, ev, gr]
    if ei is not None:
        out.append(ei)
    if gi is not None:
        out.append(gi)
    return [t.clone() for t in out]


def _check_orders(batch, lre, lim, prec, has_diag, seed):
    n = batch.n
    rng = np.random.default_rng(seed)
    g_re = rng.normal(0.0, 1.0, n)
    g_im = rng.normal(0.0, 1.0, n) if (lim is not None or batch.ham.complex) else None
    canon = nqs.coupled_pairs(batch)
    loose = nqs.coupled_pairs(batch, sort_rows=False)
    loose2 = nqs.coupled_pairs(batch, one_pass=False, sort_rows=False)
    _same_sets(canon, loose, has_diag)
    _same_sets(canon, loose2, has_diag)
    mixed = _shuffled(canon, has_diag, seed + 1)
    for store_h in (True, False):
        want = _run(batch, lre, lim, canon, prec, g_re, g_im, store_h)
        for other in (loose, loose2, mixed):
            got = _run(batch, lre, lim, other, prec, g_re, g_im, store_h)
            for x, y in zip(want, got):
                assert torch.equal(x, y)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("cplx_psi", [False, True])
def test_h28_row_order(prec, cplx_psi):
    inst = config_instance("h28", n_unq=3000, use_cache=False)
    ham, batch = gpu_objects(inst)
    lim = np.random.default_rng(7).uniform(-np.pi, np.pi, inst.n_unq) if cplx_psi else None
    _check_orders(batch, inst.logpsi_re, lim, prec, ham.info["has_diag"], seed=28)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_complex_h_row_order(prec):
    n, m = 20, 500
    x, z, c = random_pauli_hamiltonian(n, 400, 3, allow_odd_y=True, max_weight=4)
    ham = nqs.Hamiltonian(x, z, c, n)
    assert ham.complex
    ints = set()
    rng = __import__("random").Random(3)
    while len(ints) < m:
        ints.add(rng.getrandbits(n))
    batch = nqs.Batch(ham, to_dev_u(pack_ints(sorted(ints), n)))
    lre = np.random.default_rng(4).normal(0.0, 0.5, m)
    _check_orders(batch, lre, None, prec, ham.info["has_diag"], seed=20)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_star_long_row_order(prec):
    """The hub row (12001 pairs) is dealt to a whole block's warps."""
    n_qubits, n_two = 200, 12000
    rng = np.random.default_rng(41)
    pq = [(p, q) for p in range(n_qubits) for q in range(p + 1, n_qubits)]
    xs, zs, cs = [0], [0], [0.25]
    for p in range(n_qubits):
        xs.append(0); zs.append(1 << p); cs.append(rng.normal())
    for p, q in pq:
        m = (1 << p) | (1 << q)
        xs.append(m); zs.append(0); cs.append(rng.normal())
        xs.append(m); zs.append(m); cs.append(rng.normal())
    pick = rng.choice(len(pq), size=n_two, replace=False)
    samples = [0] + [(1 << pq[t][0]) | (1 << pq[t][1]) for t in pick]
    ham = nqs.Hamiltonian(pack_ints(xs, n_qubits), pack_ints(zs, n_qubits), np.array(cs), n_qubits)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(samples, n_qubits)))
    lre = rng.normal(0.0, 0.3, len(samples))
    _check_orders(batch, lre, None, prec, ham.info["has_diag"], seed=200)
