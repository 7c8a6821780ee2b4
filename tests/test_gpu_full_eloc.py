"""The exact local energy (Eq. local_energy) on the GPU against the oracle.

nqs_full_candidates lists, for every sample x and every unique XY pattern k,
the candidate x XOR XY_k with its matrix element, and the distinct candidates
of the whole batch in numeric order; nqs_local_energy_full sums
H_xx' psi(x') / psi(x) over them.  Checked against oracle/candidates.py:

* the distinct candidate set, bit-exactly, and for every entry that its
  index names x XOR XY_k;
* every matrix element within 1e-12 (relative to max(1, |H|));
* the index of each candidate in U (or -1);
* E_loc within 1e-9 Ha (FP64), real and complex log-amplitudes;
* the eigenvector identity at 12 qubits (E_loc(x) = E_0 for the exact ground
  state) and, with psi = 0 outside U, equality with E_loc^var.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from synth import config_instance, pack_ints, unpack_ints, random_pauli_hamiltonian

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects

TOL64 = 1e-9


def _ints(rows_u64):
    return unpack_ints(np.ascontiguousarray(rows_u64.cpu().numpy()).view(np.uint64))


def _check_against_oracle(ham, batch, U_ints, ref_ham, fc, rng, cplx):
    n_xy = ham.info["n_xy"]
    rows, C = oracle.full_candidates(U_ints, ref_ham)
    got_c = _ints(fc.cand)
    assert got_c == C
    xy = unpack_ints(ham.export()[0])
    cid = fc.cand_id.cpu().numpy().view(np.uint32).astype(np.int64)
    hv = fc.hval.cpu().numpy()
    pos = {v: j for j, v in enumerate(U_ints)}
    in_u = fc.in_u.cpu().numpy()
    assert all(in_u[u] == pos.get(v, -1) for u, v in enumerate(C))
    for i, x in enumerate(U_ints):
        for k in range(n_xy):
            xp = x ^ xy[k]
            assert C[cid[i, k]] == xp
            want = oracle.matrix_element(x, xp, ref_ham)
            assert abs(hv[i, k] - want.real) <= 1e-12 * max(1.0, abs(want)), (i, k, hv[i, k], want)
    # E_loc with seeded log-amplitudes for U and for every candidate
    a = rng.normal(0.0, 0.5, len(U_ints))
    b = rng.uniform(-math.pi, math.pi, len(U_ints)) if cplx else None
    ca = rng.normal(0.0, 0.5, len(C))
    cb = rng.uniform(-math.pi, math.pi, len(C)) if cplx else None
    er, ei = nqs.local_energy_full(fc, a, b, ca, cb)
    batch.status()
    want = oracle.local_energy_full(U_ints, a, b, ref_ham, C, ca, cb)
    assert np.abs(er.cpu().numpy() - np.array([w.real for w in want])).max() <= TOL64
    if cplx:
        assert np.abs(ei.cpu().numpy() - np.array([w.imag for w in want])).max() <= TOL64


@pytest.mark.parametrize("seed,n,m,T,cplx", [(1, 6, 30, 40, False), (2, 12, 80, 150, True),
                                             (3, 40, 60, 200, False), (4, 70, 50, 150, True),
                                             (5, 130, 40, 120, False)])
def test_random_hamiltonians(seed, n, m, T, cplx):
    x, z, c = random_pauli_hamiltonian(n, T, seed, allow_odd_y=False, max_weight=4)
    rng = np.random.default_rng(seed)
    pyrng = __import__("random").Random(seed)
    ints = set()
    while len(ints) < min(m, 1 << n):
        ints.add(pyrng.getrandbits(n))
    U_ints = sorted(ints)
    ham = nqs.Hamiltonian(x, z, c, n)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(U_ints, n)))
    fc = nqs.full_candidates(batch)
    ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
    _check_against_oracle(ham, batch, U_ints, ref_ham, fc, rng, cplx)


def test_molecular_h28_subset():
    inst = config_instance("h28", n_unq=200, use_cache=False)
    ham, batch = gpu_objects(inst)
    fc = nqs.full_candidates(batch)
    ref_ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    _check_against_oracle(ham, batch, unpack_ints(inst.U), ref_ham, fc, np.random.default_rng(28), False)


def test_exact_ground_state_fixed_point_h12():
    from dense_ref import pauli_dense, sector_indices
    inst = config_instance("h12", use_cache=False)
    D = pauli_dense(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits, dense=False)
    sec = sector_indices(inst.meta["n_orb"], inst.n_alpha, inst.n_beta)
    evals, evecs = np.linalg.eigh(D[sec][:, sec].toarray().real)
    psi = np.zeros(1 << inst.n_qubits)
    psi[sec] = evecs[:, 0]
    keep = [s for s in sec if abs(psi[s]) > 1e-3]  # ratios psi(x')/psi(x) stay below ~1e3
    ham = nqs.Hamiltonian.from_instance(inst)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(keep, inst.n_qubits)))
    fc = nqs.full_candidates(batch)
    C = _ints(fc.cand)
    la = lambda v: math.log(abs(psi[v])) if psi[v] != 0.0 else -745.0
    lb = lambda v: math.pi if psi[v] < 0 else 0.0
    er, ei = nqs.local_energy_full(fc, [la(v) for v in keep], [lb(v) for v in keep],
                                   [la(v) for v in C], [lb(v) for v in C])
    batch.status()
    assert np.abs(er.cpu().numpy() - evals[0]).max() < TOL64
    assert np.abs(ei.cpu().numpy()).max() < TOL64


def test_restriction_to_batch_equals_surrogate():
    inst = config_instance("h28", n_unq=1500, use_cache=False)
    ham, batch = gpu_objects(inst)
    fc = nqs.full_candidates(batch)
    in_u = fc.in_u.cpu().numpy()
    ca = np.where(in_u >= 0, inst.logpsi_re[np.maximum(in_u, 0)], -745.0)
    er, _ = nqs.local_energy_full(fc, inst.logpsi_re, None, ca)
    ref = nqs.evaluate(batch, inst.logpsi_re, None, "fp64")
    batch.status()
    assert (er - ref["eloc_re"]).abs().max().item() < TOL64
    # the candidates in U are exactly the batch: every sample is its own diagonal candidate
    assert sorted(in_u[in_u >= 0].tolist()) == list(range(inst.n_unq))


def test_capacity_error_reports_the_count():
    import ctypes
    inst = config_instance("h28", n_unq=100, use_cache=False)
    ham, batch = gpu_objects(inst)
    lib = nqs.load_library()
    nbytes = lib.nqs_candidates_scratch_bytes(ham.handle, batch.n)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    n_xy = ham.info["n_xy"]
    cid = torch.empty((batch.n, n_xy), dtype=torch.int32, device="cuda")
    cand = torch.empty((4, 1), dtype=torch.int64, device="cuda")
    n = ctypes.c_int64()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.nqs_full_candidates(ham.handle, p(batch.U), batch.n, p(batch.work), p(scratch), scratch.numel(),
                                 p(cid), None, p(cand), None, 4, ctypes.byref(n), None)
    assert rc == -4 and n.value > 4
    fc = nqs.full_candidates(batch)
    assert fc.n_cand == n.value
    rc = lib.nqs_full_candidates(ham.handle, p(batch.U), batch.n, p(batch.work), p(scratch), 1000,
                                 p(cid), None, p(cand), None, 4, ctypes.byref(n), None)
    assert rc == -4


def _check_by_definition(ham, batch, U_ints_arr, fc):
    """Candidates = the distinct values of U_i XOR XY_k (numpy's unique), in
    numeric order; every entry's index into them; each candidate's index in U."""
    xy = ham.export()[0][:, 0]
    keys = (U_ints_arr[:, None] ^ xy[None, :]).reshape(-1)
    u, inv = np.unique(keys, return_inverse=True)
    got = np.ascontiguousarray(fc.cand.cpu().numpy()).view(np.uint64).reshape(-1)
    assert np.array_equal(got, u)
    cid = fc.cand_id.cpu().numpy().view(np.uint32).astype(np.int64).reshape(-1)
    assert np.array_equal(cid, inv.reshape(-1))
    order = np.argsort(U_ints_arr)
    pos = np.searchsorted(U_ints_arr[order], u)
    pos = np.minimum(pos, len(order) - 1)
    want_in_u = np.where(U_ints_arr[order][pos] == u, order[pos], -1)
    assert np.array_equal(fc.in_u.cpu().numpy(), want_in_u)


def test_deduplication_h56_300_samples():
    """13.8 M entries (300 samples x 46,163 patterns at 56 qubits): the
    deduplication checked against the definition, and a sample of matrix
    elements against the oracle."""
    inst = config_instance("h56")
    U = np.ascontiguousarray(inst.U[:300, 0])
    ham = nqs.Hamiltonian.from_instance(inst)
    batch = nqs.Batch(ham, to_dev_u(U[:, None]))
    fc = nqs.full_candidates(batch)
    batch.status()
    _check_by_definition(ham, batch, U, fc)
    ref_ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    xy = ham.export()[0][:, 0]
    hv = fc.hval.cpu().numpy()
    rng = np.random.default_rng(56)
    for _ in range(200):
        i, k = int(rng.integers(0, 300)), int(rng.integers(0, len(xy)))
        want = oracle.matrix_element(int(U[i]), int(U[i] ^ xy[k]), ref_ham)
        assert abs(hv[i, k] - want.real) <= 1e-12 * max(1.0, abs(want))


def test_one_candidate_shared_by_5000_entries():
    """5,000 samples each coupled to x' = 0 by its own pattern (U = the XY
    patterns): 5,000 entries share one candidate; the result is the
    definition's."""
    rng = np.random.default_rng(5)
    n = 24
    pats = np.unique(rng.integers(1, 1 << n, 6000, dtype=np.int64))[:5000].astype(np.uint64)
    x = pats[:, None].copy()
    z = rng.integers(0, 1 << n, (len(pats), 1), dtype=np.int64).astype(np.uint64) & ~x
    c = rng.normal(0.0, 1.0, len(pats))
    ham = nqs.Hamiltonian(x, z, c, n)
    batch = nqs.Batch(ham, to_dev_u(pats[:, None]))
    fc = nqs.full_candidates(batch)
    batch.status()
    _check_by_definition(ham, batch, pats, fc)
    assert int((fc.cand_id.cpu().numpy().reshape(-1) == 0).sum()) >= 5000   # candidate 0 is x' = 0
