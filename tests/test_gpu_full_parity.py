"""Every row of the full-size workloads against the oracle (GPU required).

The expected values were written by ``tests/golden/full_size.py``, which
calls ``oracle/`` only (RowOracle: LoopOverTerms per row, Alg. 2A; matrix
elements by the supplementary MatrixElement algorithm; E_loc^var by Eq.
local_energy restricted to U; E^var by Eq. variational_energy; correctly
rounded sums).  For every row of the 56-qubit batch (1e5 samples) and the
84-qubit batch (2e5 samples, two words per sample) this test checks, with the
one-pass LoopOverTerms search and canonical (sorted) rows, FP32C and FP64:

* the number of coupled pairs and a digest of the row's column set, exactly;
* for every pair, U_i XOR U_j equals the XY pattern the library names;
* E_loc^var: FP64 within 1e-9 Ha, FP32C within 1e-6 Ha of the oracle;
* E^var: FP64 within 1e-9 Ha, FP32C within 1e-6 Ha of the oracle's E^var;
* the workspace status word is clean (no device index check fired).

Rows of at least 1024 pairs (reduced by a whole block) and of more than 512
pairs (sorted by the block sort) are among them (295 at 56 qubits, the
Hartree-Fock row with 7,676 pairs the longest); the test asserts they occur.
The last test repeats the 56-qubit checks in the form bench.py times (the
no-wait search, rows left in search order).
"""

import importlib.util
import os

import numpy as np
import pytest
import torch

from synth import config_instance

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL64 = 1e-9
TOL32 = 1e-6

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import gpu_objects


def _golden_module():
    spec = importlib.util.spec_from_file_location("full_size", os.path.join(HERE, "golden", "full_size.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _load(name):
    fs = _golden_module()
    path = os.path.join(HERE, "golden", f"{name}_rows.npz")
    g = np.load(path)
    inst = config_instance(name)
    u_sha, xz_sha, l1 = fs.instance_digests(inst)
    assert str(g["u_sha"]) == u_sha, "the generator produced another sample batch than the golden file's"
    assert str(g["xz_sha"]) == xz_sha, "the generator produced other Pauli strings than the golden file's"
    assert abs(float(g["coef_l1"][0]) - l1) <= 1e-12 * l1
    return fs, g, inst


def _xor_rows(U, rows, cols):
    return U[rows] ^ U[cols]


def _spin_mask(n_words, parity):
    """Word masks of the even (parity 0, alpha) or odd (parity 1, beta) qubits."""
    m = 0x5555555555555555 if parity == 0 else 0xAAAAAAAAAAAAAAAA
    return np.full(n_words, m, dtype=np.uint64)


@pytest.mark.parametrize("name", ["h56", "h84"])
def test_every_row_against_oracle(name):
    fs, g, inst = _load(name)
    ham, batch = gpu_objects(inst)
    res = {p: nqs.evaluate(batch, inst.logpsi_re, None, p) for p in ("fp64", "fp32c")}
    batch.status()
    rp = res["fp32c"]["pairs"][0].cpu().numpy()
    pj = res["fp32c"]["pairs"][1].cpu().numpy().view(np.uint32)
    pk = res["fp32c"]["pairs"][2].cpu().numpy().view(np.uint32)
    # both precisions list the same pairs
    assert torch.equal(res["fp64"]["pairs"][1], res["fp32c"]["pairs"][1])
    lens = np.diff(rp)
    assert lens.sum() == int(g["n_pairs"][0])
    bad = np.nonzero(lens != g["count"])[0]
    assert len(bad) == 0, f"{len(bad)} rows differ in pair count, first {bad[:5]}"
    dig = fs.set_digest_np(rp, pj)
    bad = np.nonzero(dig != g["digest"])[0]
    assert len(bad) == 0, f"{len(bad)} rows differ in their column sets, first {bad[:5]}"
    # every pair's pattern index names U_i XOR U_j
    xy = ham.export()[0]
    U = np.ascontiguousarray(inst.U)
    rows = np.repeat(np.arange(inst.n_unq), lens)
    n_diag = 0
    for s0 in range(0, len(pj), 1 << 22):
        sl = slice(s0, s0 + (1 << 22))
        d = _xor_rows(U, rows[sl], pj[sl].astype(np.int64))
        assert np.array_equal(d, xy[pk[sl].astype(np.int64)])
        # a two-body H moves at most two electrons: |U_i XOR U_j| in {0, 2, 4}; and with
        # interleaved spin-orbitals (even qubits alpha, odd beta) both spin counts are kept
        pc = np.bitwise_count(d).sum(axis=1)
        assert np.isin(pc, (0, 2, 4)).all()
        cols = pj[sl].astype(np.int64)
        for mask in (_spin_mask(inst.n_words, 0), _spin_mask(inst.n_words, 1)):
            ni = np.bitwise_count(U[rows[sl]] & mask).sum(axis=1)
            nj = np.bitwise_count(U[cols] & mask).sum(axis=1)
            assert np.array_equal(ni, nj)
        n_diag += int((cols == rows[sl]).sum())
    # the diagonal pair of every row is listed exactly once
    assert n_diag == inst.n_unq
    # long rows: block-reduced (>= 1024 pairs) and block-sorted (> 512) ones are compared here too
    assert (lens >= 1024).sum() > 0 and (lens > 512).sum() > 0
    want = g["eloc"]
    for prec, tol in (("fp64", TOL64), ("fp32c", TOL32)):
        got = res[prec]["eloc_re"].cpu().numpy()
        err = np.abs(got - want)
        assert err.max() <= tol, (prec, int(err.argmax()), float(err.max()))
        ev = res[prec]["evar"][0].item()
        assert abs(ev - float(g["evar"][0])) <= tol, (prec, ev, float(g["evar"][0]))


def test_bench_step_configuration_h56():
    """The form bench.py times at 56 qubits: the no-wait search with rows left in
    search order and each pair packed in one 64-bit word, then E_loc^var, E^var and the adjoint on those lists.  Every row's
    pair count and column set against the oracle's, and E_loc^var / E^var bitwise
    equal to the canonical (sorted-row) path, which the test above holds to the
    oracle, in both precisions."""
    fs, g, inst = _load("h56")
    ham, batch = gpu_objects(inst)
    for prec, tol in (("fp64", TOL64), ("fp32c", TOL32)):
        ref = nqs.evaluate(batch, inst.logpsi_re, None, prec)
        total = int(ref["n_pairs"])
        rp, words, _ = nqs.coupled_pairs_async(batch, total + 1024, sort_rows=False, packed=True)
        er, ei, hd = nqs.local_energy(batch, inst.logpsi_re, None, (rp, words, None), prec)
        ev = nqs.variational_energy(batch, inst.logpsi_re, er)
        batch.status()
        rph = rp.cpu().numpy()
        assert int(rph[-1]) == int(g["n_pairs"][0])
        assert np.array_equal(np.diff(rph), g["count"])
        cols = (words[:total].cpu().numpy().view(np.uint64) >> np.uint64(32)).astype(np.uint32)
        dig = fs.set_digest_np(rph, cols)
        assert np.array_equal(dig, g["digest"])
        assert torch.equal(er, ref["eloc_re"]) and torch.equal(hd, ref["hdiag"])
        assert torch.equal(ev, ref["evar"])
        err = np.abs(er.cpu().numpy() - g["eloc"])
        assert err.max() <= tol, (prec, float(err.max()))
