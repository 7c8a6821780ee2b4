"""Row order of the LoopOverTerms pair lists, and rows long enough to take the
block sort (GPU required).

The LoopOverTerms schedule finds each coupled pair once (from the sample
that has the pattern's highest qubit) and lists it in both rows; every row
then holds the diagonal pair first and the rest in ascending column index.

The star instance below has closed-form row lengths.  Qubits 0..N-1,
patterns {p, q} for every p < q (terms X_p X_q and Y_p Y_q) plus Z_p and
identity terms, and U = {0} plus two-qubit samples {p, q}.  Sample 0 couples
to every sample; sample {p, q} couples to itself, to 0, and to every other
sample sharing p or q, so its row holds deg(p) + deg(q) pairs, deg(p) being
the number of two-qubit samples containing p.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import config_instance, pack_ints, unpack_ints

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects, pair_set_gpu


def _rows_sorted(pairs, has_diag, row_begin=0):
    rp, pj, pk = pairs
    rp = rp.cpu().numpy()
    j = pj.cpu().numpy().view(np.uint32).astype(np.int64)
    k = pk.cpu().numpy().view(np.uint32).astype(np.int64)
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        if has_diag and b > a:
            assert k[a] == 0 and j[a] == row_begin + r, f"row {r}: diagonal pair not first"
            a += 1
        assert np.all(np.diff(j[a:b]) > 0), f"row {r}: columns not ascending"


@pytest.mark.parametrize("r0,r1", [(0, None), (17, 1234), (2990, 3000)])
def test_terms_rows_ascend_by_column(r0, r1):
    inst = config_instance("h28", n_unq=3000, use_cache=False)
    ham, batch = gpu_objects(inst)
    r1 = inst.n_unq if r1 is None else r1
    for one_pass in (True, False):
        pairs = nqs.coupled_pairs(batch, r0, r1, one_pass=one_pass)
        _rows_sorted(pairs, ham.info["has_diag"], r0)
    # the list of a row does not depend on the range it was listed in
    full = nqs.coupled_pairs(batch)
    part = nqs.coupled_pairs(batch, r0, r1)
    a, b = int(full[0][r0]), int(full[0][r1])
    assert torch.equal(part[1], full[1][a:b]) and torch.equal(part[2], full[2][a:b])


def _star(n_qubits, n_two, seed):
    rng = np.random.default_rng(seed)
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
    order = rng.permutation(len(samples))
    samples = [samples[t] for t in order]
    # the samples holding qubit 0 first: the rows of those samples then have
    # most of their columns in a narrow range at the start (clustered keys)
    samples = [v for v in samples if v & 1] + [v for v in samples if not v & 1]
    x = pack_ints(xs, n_qubits)
    z = pack_ints(zs, n_qubits)
    U = pack_ints(samples, n_qubits)
    logpsi = rng.normal(0.0, 0.3, len(samples))
    return x, z, np.array(cs), U, samples, logpsi


# 12000 two-qubit samples: sample 0's row (12001 pairs) is sorted in shared
# memory; all 19900: its row (19901 pairs) exceeds the shared-memory limit
# and is sorted in place.  Rows of samples holding qubit 0 have clustered
# columns and leave the warp sort for the block sort too.
@pytest.mark.parametrize("n_two", [12000, 19900])
def test_star_long_row(n_two):
    n_qubits = 200
    x, z, c, U, samples, logpsi = _star(n_qubits, n_two, seed=11 + n_two)
    ham = nqs.Hamiltonian(x, z, c, n_qubits)
    batch = nqs.Batch(ham, to_dev_u(U))
    pairs = nqs.coupled_pairs(batch)
    rp = pairs[0].cpu().numpy()
    deg = np.zeros(n_qubits, np.int64)
    for v in samples:
        if v:
            for b in range(n_qubits):
                if (v >> b) & 1:
                    deg[b] += 1
    want = np.array([len(samples) if v == 0 else sum(deg[b] for b in range(n_qubits) if (v >> b) & 1)
                     for v in samples])
    assert np.array_equal(np.diff(rp), want)
    _rows_sorted(pairs, ham.info["has_diag"])
    rows, j, k = pair_set_gpu(batch, pairs)
    xy = unpack_ints(ham.export()[0])
    hub = samples.index(0)
    assert sorted(j[rows == hub].tolist()) == list(range(len(samples)))
    sel = np.random.default_rng(3).choice(len(rows), 20000, replace=False)
    for t in sel:
        assert samples[rows[t]] ^ samples[j[t]] == xy[k[t]]
    # local energies and the adjoint of a few rows, the long one (one block,
    # warps dealt its rounds) included, against the oracle
    er, _, hd = nqs.local_energy(batch, logpsi, None, pairs, "fp64")
    ev = nqs.variational_energy(batch, logpsi, er)
    g = np.random.default_rng(5).normal(0.0, 1.0, len(samples))
    gr, _ = nqs.local_energy_backward(batch, logpsi, None, er, None, hd, ev, g, None, None, pairs, "fp64")
    # the same rows in FP32C (the long row is reduced by a whole block there too)
    er32, _, hd32 = nqs.local_energy(batch, logpsi, None, pairs, "fp32c")
    ev32 = nqs.variational_energy(batch, logpsi, er32)
    gr32, _ = nqs.local_energy_backward(batch, logpsi, None, er32, None, hd32, ev32, g, None, None, pairs, "fp32c")
    batch.status()  # no device index check fired
    ro = oracle.RowOracle(U, oracle.prepare_hamiltonian(x, z, c, n_qubits), logpsi)
    for r in [hub, 0, 1, len(samples) - 1]:
        want = ro.row(r)["eloc"]
        assert abs(er[r].item() - want.real) < 1e-9
        assert abs(er32[r].item() - want.real) < 1e-6
        eloc = np.zeros(len(samples), complex)
        eloc[r] = want
        g_want, _ = ro.row_vjp(r, eloc, 0.0, g_eloc_re=g, g_evar=0.0)
        assert abs(gr[r].item() - g_want) < 1e-9 * max(1.0, abs(g_want))
        assert abs(gr32[r].item() - g_want) < 1e-6 * max(1.0, abs(g_want))
    # one-pass and two-pass lists agree
    two = nqs.coupled_pairs(batch, one_pass=False)
    for a_, b_ in zip(pairs, two):
        assert torch.equal(a_, b_)
