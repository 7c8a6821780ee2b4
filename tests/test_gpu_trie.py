"""LoopOverTrie (Alg. 2C over the prefix trees of Alg. 3) on the GPU.

Pair sets are compared bit-exactly with the oracle (and with LoopOverTerms
at full size); a row's pairs must not depend on the row range; the trie
build must cope with batches whose samples share long prefixes, with dense
batches (every basis vector of a small space), with one and two samples, and
a search on a workspace without a tree must fail with NQS_ERR_ARG.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import config_instance, pack_ints, unpack_ints, random_pauli_hamiltonian

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects, pair_set_gpu, oracle_for


def _triples(batch, pairs, r0=0):
    r, j, k = pair_set_gpu(batch, pairs, r0)
    return sorted(zip(r.tolist(), j.tolist(), k.tolist()))


def _xy_ints(ham):
    xy, _, _, _ = ham.export()
    return unpack_ints(xy) if len(xy) else []


def _check_against_oracle(x, z, c, n, U_ints):
    ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
    ref = sorted(oracle.find_coupled_pairs(U_ints, ref_ham, "terms"))
    ham = nqs.Hamiltonian(x, z, c, n)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(U_ints, n)))
    pairs = nqs.coupled_pairs(batch, schedule="trie")
    r, j, k = pair_set_gpu(batch, pairs)
    assert sorted(zip(r.tolist(), j.tolist())) == ref
    xy = _xy_ints(ham)
    for (i, jj, kk) in zip(r.tolist(), j.tolist(), k.tolist()):
        assert U_ints[i] ^ U_ints[jj] == xy[kk]
    return ham, batch, pairs


def test_trie_h12_full_sector_and_energy():
    inst = config_instance("h12", use_cache=False)
    ref_ham = oracle_for(inst)
    ref = oracle.forward(inst.U, inst.logpsi_re, None, ref_ham)
    ham, batch = gpu_objects(inst)
    pairs = nqs.coupled_pairs(batch, schedule="trie")
    r, j, k = pair_set_gpu(batch, pairs)
    assert sorted(zip(r.tolist(), j.tolist())) == sorted(ref["pairs"])
    er, _, hd = nqs.local_energy(batch, inst.logpsi_re, None, pairs, "fp64")
    want = np.array([e.real for e in ref["eloc"]])
    assert np.abs(er.cpu().numpy() - want).max() < 1e-9


def test_trie_row_ranges_keep_row_order():
    inst = config_instance("h28", n_unq=3000, use_cache=False)
    ham, batch = gpu_objects(inst)
    rp, pj, pk = nqs.coupled_pairs(batch, schedule="trie")
    rp_h = rp.cpu().numpy()
    for (r0, r1) in [(0, 1), (1, 2), (777, 1500), (2999, 3000)]:
        q, qj, qk = nqs.coupled_pairs(batch, r0, r1, schedule="trie")
        a, b = rp_h[r0], rp_h[r1]
        assert torch.equal(qj, pj[a:b]) and torch.equal(qk, pk[a:b])
    two = nqs.coupled_pairs(batch, schedule="trie", one_pass=False)
    for x, y in zip((rp, pj, pk), two):
        assert torch.equal(x, y)
    # restaging invalidates the tree; the binding rebuilds it
    batch.restage(batch.U)
    again = nqs.coupled_pairs(batch, schedule="trie")
    for x, y in zip((rp, pj, pk), again):
        assert torch.equal(x, y)


def test_trie_shared_long_prefixes():
    # samples agree on the first 40 of 48 qubits: the tree is a long chain then a bush
    n = 48
    base = 0xA5A5A5A5A5 & ((1 << 40) - 1)
    U = [base | (v << 40) for v in range(256)]
    x, z, c = random_pauli_hamiltonian(n, 300, 11, allow_odd_y=False, max_weight=4)
    # add patterns that live in the top byte so that pairs exist
    extra = [(1 << 40) | (1 << 41), (1 << 44) | (1 << 47), (1 << 42) | (1 << 43) | (1 << 45) | (1 << 46)]
    xe = pack_ints(extra, n)
    x = np.concatenate([x, xe]); z = np.concatenate([z, np.zeros_like(xe)]); c = np.concatenate([c, [0.3, -0.2, 0.1]])
    _check_against_oracle(x, z, c, n, U)


def test_trie_dense_small_space():
    # every basis vector of 12 qubits: each sample couples through every pattern
    n = 12
    x, z, c = random_pauli_hamiltonian(n, 60, 12, allow_odd_y=False)
    _check_against_oracle(x, z, c, n, list(range(1 << n)))


def test_trie_one_and_two_samples():
    n = 20
    x, z, c = random_pauli_hamiltonian(n, 40, 13, allow_odd_y=False, max_weight=4)
    xs = unpack_ints(x)
    _check_against_oracle(x, z, c, n, [12345])
    _check_against_oracle(x, z, c, n, [12345, 12345 ^ xs[0]])


def test_trie_h56_matches_terms_full_size():
    inst = config_instance("h56")
    ham, batch = gpu_objects(inst)
    t = nqs.coupled_pairs(batch, schedule="terms")
    r = nqs.coupled_pairs(batch, schedule="trie")
    assert torch.equal(t[0], r[0])
    assert _triples(batch, t) == _triples(batch, r)
    a = torch.from_numpy(inst.logpsi_re).cuda()
    et = nqs.evaluate(batch, a, None, "fp32c", schedule="terms")
    ek = nqs.evaluate(batch, a, None, "fp32c", schedule="trie")
    assert (et["eloc_re"] - ek["eloc_re"]).abs().max().item() < 1e-6
    assert abs(et["evar"][0].item() - ek["evar"][0].item()) < 1e-9


@pytest.mark.device_status_error
def test_trie_without_tree_is_an_error():
    inst = config_instance("h28", n_unq=500, use_cache=False)
    ham, batch = gpu_objects(inst)
    lib = nqs.load_library()
    rp = torch.empty(batch.n + 1, dtype=torch.int64, device="cuda")
    import ctypes
    n = ctypes.c_int64()
    rc = lib.nqs_count_coupled_pairs(ham.handle, batch.U.data_ptr(), batch.n, batch.work.data_ptr(), 0,
                                     batch.n, 3, rp.data_ptr(), ctypes.byref(n), None)
    assert rc == -1
    assert b"nqs_stage_trie" in lib.nqs_last_error()
