"""Parity of the CUDA path with the CPU oracle (GPU required).

Pair lists are compared bit-exactly (as sets, plus the XY pattern of each
pair); energies within the tolerances stated per test:
  FP64 GPU path:  |dE_loc| <= 1e-9 Ha,  |dE^var| <= 1e-9 Ha
  FP32C GPU path: |dE_loc| <= 1e-6 Ha,  |dE^var| <= 1e-6 Ha
"""

import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from synth import (config_instance, pack_ints, unpack_ints, random_pauli_hamiltonian,
                   from_paper_string)

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects, pair_set_gpu, oracle_for

TOL64 = 1e-9
TOL32 = 1e-6
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_example.json")))


def _toy():
    xs = [sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "XY") for t in GOLD["terms"]["list"]]
    zs = [sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "YZ") for t in GOLD["terms"]["list"]]
    hs = np.array([t["h"] for t in GOLD["terms"]["list"]])
    U = pack_ints([from_paper_string(s) for s in GOLD["batch"]["U"]], 4)
    psi = np.array(GOLD["batch"]["psi"])
    return pack_ints(xs, 4), pack_ints(zs, 4), hs, U, psi


def _check_pairs(batch, pairs, ref_pairs, U_ints, xy_table, row_begin=0):
    rows, j, k = pair_set_gpu(batch, pairs, row_begin)
    got = sorted(zip(rows.tolist(), j.tolist()))
    assert len(set(got)) == len(got), "repeated pair"
    assert got == sorted(ref_pairs)
    for (i, jj, kk) in zip(rows[:5000], j[:5000], k[:5000]):
        assert U_ints[i] ^ U_ints[jj] == xy_table[kk]


def _xy_ints(ham):
    xy, _, _, _ = ham.export()
    return unpack_ints(xy) if len(xy) else []


def test_toy_example_worked_values():
    x, z, h, U, psi = _toy()
    ham = nqs.Hamiltonian(x, z, h, 4)
    batch = nqs.Batch(ham, to_dev_u(U))
    pairs = nqs.coupled_pairs(batch)
    rows, j, k = pair_set_gpu(batch, pairs)
    got = [sorted(j[rows == r].tolist()) for r in range(3)]
    assert got == [sorted(r) for r in GOLD["coupled_sets"]["rows"]]
    lre = np.log(np.abs(psi)); lim = np.where(psi < 0, np.pi, 0.0)
    for prec, tol in (("fp64", 1e-14), ("fp32c", 1e-12)):
        er, ei, hd = nqs.local_energy(batch, lre, lim, pairs, prec)
        assert np.allclose(er.cpu().numpy(), GOLD["local_energies"]["eloc"], atol=tol, rtol=0)
        assert np.abs(ei.cpu().numpy()).max() < 1e-12
        assert np.allclose(hd.cpu().numpy(), [0.8, 1.0, 1.0], atol=tol)
        ev = nqs.variational_energy(batch, lre, er)
        assert abs(ev[0].item() - 5.2 / 6.0) < tol


@pytest.mark.parametrize("seed,n,m,T", [(1, 6, 40, 30), (2, 10, 300, 120), (3, 20, 500, 400),
                                        (4, 70, 300, 200), (5, 130, 200, 150)])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_random_hamiltonians_match_definition(seed, n, m, T, prec):
    x, z, c = random_pauli_hamiltonian(n, T, seed, allow_odd_y=False, max_weight=4)
    rng = np.random.default_rng(seed)
    pyrng = __import__("random").Random(seed)
    ints = set()
    while len(ints) < m:
        ints.add(pyrng.getrandbits(n))
    Ui = sorted(ints)
    pyrng.shuffle(Ui)
    U = pack_ints(Ui, n)
    lre = rng.normal(0, 0.5, size=m)
    lim = np.where(rng.random(m) < 0.4, np.pi, 0.0)
    ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
    ref = oracle.forward(Ui, lre, lim, ref_ham)
    ham = nqs.Hamiltonian(x, z, c, n)
    batch = nqs.Batch(ham, to_dev_u(U))
    pairs = nqs.coupled_pairs(batch)
    _check_pairs(batch, pairs, ref["pairs"], Ui, _xy_ints(ham))
    er, ei, hd = nqs.local_energy(batch, lre, lim, pairs, prec)
    tol = TOL64 if prec == "fp64" else TOL32
    want = np.array(ref["eloc"])
    assert np.abs(er.cpu().numpy() - want.real).max() < tol
    assert np.abs(ei.cpu().numpy() - want.imag).max() < tol


@pytest.fixture(scope="module")
def h12():
    inst = config_instance("h12", use_cache=False)
    ref_ham = oracle_for(inst)
    ref = oracle.forward(inst.U, inst.logpsi_re, None, ref_ham)
    return inst, ref_ham, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_h12_whole_batch(h12, prec):
    inst, ref_ham, ref = h12
    ham, batch = gpu_objects(inst)
    pairs = nqs.coupled_pairs(batch)
    _check_pairs(batch, pairs, ref["pairs"], unpack_ints(inst.U), _xy_ints(ham))
    er, ei, hd = nqs.local_energy(batch, inst.logpsi_re, None, pairs, prec)
    tol = TOL64 if prec == "fp64" else TOL32
    want = np.array([e.real for e in ref["eloc"]])
    assert np.abs(er.cpu().numpy() - want).max() < tol
    ev = nqs.variational_energy(batch, inst.logpsi_re, er)
    assert abs(ev[0].item() - ref["e_var"].real) < tol


@pytest.fixture(scope="module")
def h28():
    inst = config_instance("h28", n_unq=3000, use_cache=False)
    ref_ham = oracle_for(inst)
    ref = oracle.forward(inst.U, inst.logpsi_re, None, ref_ham)
    return inst, ref_ham, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_h28_whole_batch(h28, prec):
    """3000 samples: many warps and row batches, a ragged last batch."""
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    pairs = nqs.coupled_pairs(batch)
    _check_pairs(batch, pairs, ref["pairs"], unpack_ints(inst.U), _xy_ints(ham))
    er, ei, hd = nqs.local_energy(batch, inst.logpsi_re, None, pairs, prec)
    tol = TOL64 if prec == "fp64" else TOL32
    want = np.array([e.real for e in ref["eloc"]])
    assert np.abs(er.cpu().numpy() - want).max() < tol
    ev = nqs.variational_energy(batch, inst.logpsi_re, er)
    assert abs(ev[0].item() - ref["e_var"].real) < tol


def test_row_ranges_and_chunks_agree(h28):
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    full = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c")
    chunked = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c", max_pairs=full["n_pairs"] // 7)
    assert len(chunked["chunks"]) >= 7
    # a row's pairs come out in the same order whatever the row range
    assert torch.equal(full["eloc_re"], chunked["eloc_re"])
    assert torch.equal(full["evar"], chunked["evar"])
    # a middle row range on its own
    r0, r1 = 1234, 2345
    pairs = nqs.coupled_pairs(batch, r0, r1)
    rows, j, k = pair_set_gpu(batch, pairs, r0)
    want = sorted((i, jj) for (i, jj) in ref["pairs"] if r0 <= i < r1)
    assert sorted(zip(rows.tolist(), j.tolist())) == want


def test_one_pass_equals_two_pass(h28):
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    a = nqs.coupled_pairs(batch, one_pass=True)
    b = nqs.coupled_pairs(batch, one_pass=False)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # a deliberately small first guess goes through the retry path
    batch2 = nqs.Batch(ham, batch.U)
    batch2._pair_guess = 100
    c = nqs.coupled_pairs(batch2)
    for x, y in zip(a, c):
        assert torch.equal(x, y)
    # sub-ranges: one-pass and two-pass give the same CSR and match the oracle rows
    for (r0, r1) in [(0, 7), (5, 1000), (2990, 3000)]:
        a = nqs.coupled_pairs(batch, r0, r1)
        b = nqs.coupled_pairs(batch, r0, r1, one_pass=False)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        rows, j, k = pair_set_gpu(batch, a, r0)
        want = sorted((i, jj) for (i, jj) in ref["pairs"] if r0 <= i < r1)
        assert sorted(zip(rows.tolist(), j.tolist())) == want


@pytest.mark.parametrize("schedule", ["batch", "auto", "trie"])
def test_batch_schedule_matches_terms(h28, schedule):
    """LoopOverBatch (Alg. 2B) and LoopOverTrie (Alg. 2C) list the same pairs;
    energies agree to rounding."""
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    for r0, r1 in [(0, inst.n_unq), (17, 1234)]:
        t = nqs.coupled_pairs(batch, r0, r1, schedule="terms")
        b = nqs.coupled_pairs(batch, r0, r1, schedule=schedule)
        assert torch.equal(t[0], b[0])  # same counts per row
        rt, jt, kt = pair_set_gpu(batch, t, r0)
        rb, jb, kb = pair_set_gpu(batch, b, r0)
        assert sorted(zip(rt.tolist(), jt.tolist(), kt.tolist())) == sorted(zip(rb.tolist(), jb.tolist(), kb.tolist()))
        # the diagonal pair leads each row in both schedules
        rp = b[0].cpu().numpy()
        assert np.all(jb[rp[:-1] - rp[0]] == np.arange(r0, r1))
    two = nqs.coupled_pairs(batch, schedule=schedule, one_pass=False)
    one = nqs.coupled_pairs(batch, schedule=schedule)
    for x, y in zip(one, two):
        assert torch.equal(x, y)
    eb = nqs.evaluate(batch, inst.logpsi_re, None, "fp64", schedule=schedule)
    want = np.array([e.real for e in ref["eloc"]])
    assert np.abs(eb["eloc_re"].cpu().numpy() - want).max() < TOL64


@pytest.mark.parametrize("schedule", ["batch", "trie"])
def test_batch_schedule_random_multiword(schedule):
    for n, seed in ((70, 4), (130, 5)):
        x, z, c = random_pauli_hamiltonian(n, 150, seed, allow_odd_y=False, max_weight=4)
        pyrng = __import__("random").Random(seed)
        Ui = set()
        while len(Ui) < 300:
            v = pyrng.getrandbits(n)
            Ui.add(v)
            Ui.add(v ^ (3 << 5))  # make some pairs couple through 2-bit patterns
        Ui = sorted(Ui)[:300]
        ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
        ref_pairs = oracle.find_coupled_pairs(Ui, ref_ham, "batch")
        ham = nqs.Hamiltonian(x, z, c, n)
        batch = nqs.Batch(ham, to_dev_u(pack_ints(Ui, n)))
        pairs = nqs.coupled_pairs(batch, schedule=schedule)
        _check_pairs(batch, pairs, ref_pairs, Ui, _xy_ints(ham))


def test_deterministic(h28):
    inst, _, _ = h28
    ham, batch = gpu_objects(inst)
    a = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c")
    b = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c")
    assert torch.equal(a["pairs"][1], b["pairs"][1]) and torch.equal(a["pairs"][2], b["pairs"][2])
    assert torch.equal(a["eloc_re"], b["eloc_re"]) and torch.equal(a["evar"], b["evar"])


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_backward_matches_oracle_vjp(prec):
    inst = config_instance("h12", use_cache=False)
    ref_ham = oracle_for(inst)
    rng = np.random.default_rng(12)
    lre = inst.logpsi_re
    lim = np.where(rng.random(inst.n_unq) < 0.3, np.pi, 0.0) + rng.normal(0, 0.2, inst.n_unq)
    gr = rng.normal(size=inst.n_unq); gi = rng.normal(size=inst.n_unq); gE = 0.37
    pairs_ref = oracle.find_coupled_pairs(inst.U, ref_ham)
    want_re, want_im = oracle.local_energy_vjp(inst.U, lre, lim, ref_ham, pairs_ref, gr, gi, gE)
    ham, batch = gpu_objects(inst)
    res = nqs.evaluate(batch, lre, lim, prec, keep_h=True)
    up = (torch.from_numpy(gr).cuda(), torch.from_numpy(gi).cuda(), torch.tensor([gE], dtype=torch.float64).cuda())
    g_re, g_im = nqs.local_energy_backward(batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"],
                                           res["evar"], *up, res["pairs"], prec)
    tol = TOL64 if prec == "fp64" else TOL32
    assert np.abs(g_re.cpu().numpy() - want_re).max() < tol
    assert np.abs(g_im.cpu().numpy() - want_im).max() < tol
    # the matrix elements stored by the forward call give the same bits
    h_re, h_im = nqs.local_energy_backward(batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"],
                                           res["evar"], *up, res["pairs"], prec, hpair=res["hpair"])
    assert torch.equal(h_re, g_re) and torch.equal(h_im, g_im)
    # closed form (no upstream on E_loc)
    c_re, c_im = nqs.local_energy_backward(batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"],
                                           res["evar"], None, None,
                                           torch.tensor([1.0], dtype=torch.float64).cuda(), None, prec)
    eloc_ref, _ = oracle.local_energy_var(inst.U, lre, lim, ref_ham, pairs_ref)
    ev_ref = oracle.variational_energy(lre, eloc_ref)
    w_re, w_im = oracle.energy_gradient_closed_form(lre, eloc_ref, ev_ref)
    assert np.abs(c_re.cpu().numpy() - w_re).max() < tol
    assert np.abs(c_im.cpu().numpy() - w_im).max() < tol


def test_autograd_function_and_finite_differences(h28):
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    lre = torch.from_numpy(inst.logpsi_re).cuda().requires_grad_(True)
    er, ei, ev = nqs.LocalEnergy.apply(batch, lre, None, "fp64", None)
    g = torch.from_numpy(np.random.default_rng(3).normal(size=inst.n_unq)).cuda()
    loss = ev + (g * er).sum() * 1e-3
    loss.backward()
    grad = lre.grad.detach().cpu().numpy()
    rng = np.random.default_rng(4)
    h = 1e-4
    base = inst.logpsi_re.copy()
    for y in rng.choice(inst.n_unq, size=6, replace=False):
        vals = []
        for sgn in (1, -1):
            l = base.copy(); l[y] += sgn * h
            res = nqs.evaluate(batch, l, None, "fp64")
            vals.append(res["evar"][0].item() + 1e-3 * float((g * res["eloc_re"]).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[y]) < 1e-6 * max(1.0, abs(fd)), (y, fd, grad[y])
    # recomputed pairs (memory cap) give the same gradient
    lre2 = torch.from_numpy(inst.logpsi_re).cuda().requires_grad_(True)
    er2, _, ev2 = nqs.LocalEnergy.apply(batch, lre2, None, "fp64", 20000)
    (ev2 + (g * er2).sum() * 1e-3).backward()
    assert torch.equal(lre2.grad, lre.grad)


def test_fp32c_vs_fp64_h56_full_size():
    """The 56-qubit batch of 1e5 peaked samples: sampled rows against the
    oracle, FP32C against FP64 on every row, E^var within 1e-6."""
    inst = config_instance("h56")
    ham, batch = gpu_objects(inst)
    r64 = nqs.evaluate(batch, inst.logpsi_re, None, "fp64")
    r32 = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c")
    assert r64["n_pairs"] == r32["n_pairs"]
    d = (r64["eloc_re"] - r32["eloc_re"]).abs().max().item()
    assert d < TOL32, d
    assert abs(r64["evar"][0].item() - r32["evar"][0].item()) < TOL32
    ro = oracle.RowOracle.from_instance(inst)
    rows, j, k = pair_set_gpu(batch, r32["pairs"])
    rng = np.random.default_rng(56)
    U_ints = ro.U
    xy = _xy_ints(ham)
    rp = r32["pairs"][0].cpu().numpy()
    for i in rng.choice(inst.n_unq, size=40, replace=False):
        rr = ro.row(int(i))
        got = sorted(j[rp[i]:rp[i + 1]].tolist())
        assert got == sorted(rr["j"])
        assert abs(r64["eloc_re"][i].item() - rr["eloc"].real) < TOL64
        assert abs(r32["eloc_re"][i].item() - rr["eloc"].real) < TOL32
    # pair symmetry over the whole list
    key = rows * inst.n_unq + j
    key_t = j * inst.n_unq + rows
    assert np.array_equal(np.sort(key), np.sort(key_t))
    # the reduction alone (E^var of the GPU's own E_loc by the oracle's formula); E^var against the
    # oracle's own E_loc of every row is checked in test_gpu_full_parity.py
    ev_ref = oracle.variational_energy(inst.logpsi_re, [complex(v) for v in r64["eloc_re"].cpu().numpy()])
    assert abs(ev_ref.real - r64["evar"][0].item()) < TOL64
    batch.status()


def test_error_paths():
    x, z, h, U, psi = _toy()
    ham = nqs.Hamiltonian(x, z, h, 4)
    dup = np.concatenate([U, U[:1]])
    with pytest.raises(nqs.NQSError) as e:
        nqs.Batch(ham, to_dev_u(dup))
    assert e.value.code == -5
    bad = U.copy(); bad[0, 0] |= np.uint64(1 << 9)
    with pytest.raises(nqs.NQSError) as e:
        nqs.Batch(ham, to_dev_u(bad))
    assert e.value.code == -1
    batch = nqs.Batch(ham, to_dev_u(U))
    rp = torch.empty(4, dtype=torch.int64, device="cuda")
    import ctypes
    n = ctypes.c_int64()
    lib = nqs.load_library()
    pj = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = lib.nqs_find_coupled_pairs(ham.handle, ctypes.c_void_p(batch.U.data_ptr()), 3,
                                    ctypes.c_void_p(batch.work.data_ptr()), 0, 3, 1, None, 0,
                                    ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(pj.data_ptr()),
                                    ctypes.c_void_p(pj.data_ptr()), 1, ctypes.byref(n), None)
    assert rc == -4 and n.value == 7
    # one-pass form with a scratch that is too small: capacity error, then the fill pass completes
    scratch = torch.empty(256 + 256 + 256 + 8, dtype=torch.uint8, device="cuda")
    rc = lib.nqs_find_coupled_pairs(ham.handle, ctypes.c_void_p(batch.U.data_ptr()), 3,
                                    ctypes.c_void_p(batch.work.data_ptr()), 0, 3, 1,
                                    ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                    ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(pj.data_ptr()),
                                    ctypes.c_void_p(pj.data_ptr()), 1, ctypes.byref(n), None)
    assert rc == -4 and n.value == 7


def test_edge_cases():
    # one sample; Hamiltonian without a diagonal pattern; only a diagonal pattern; no terms
    U = pack_ints([0b0110], 4)
    for xs, zs, cs, want in [([0b0011], [0], [1.0], 0.0), ([0], [0b0010], [2.0], -2.0),
                             ([], [], [], 0.0)]:
        ham = nqs.Hamiltonian(pack_ints(xs, 4) if xs else np.zeros((0, 1), np.uint64),
                              pack_ints(zs, 4) if zs else np.zeros((0, 1), np.uint64), np.array(cs), 4)
        batch = nqs.Batch(ham, to_dev_u(U))
        res = nqs.evaluate(batch, np.array([0.3]), None, "fp32c")
        assert res["eloc_re"][0].item() == want
    # 64 and 65 qubits (word boundary), samples using the top bits
    for n in (64, 65):
        x, z, c = random_pauli_hamiltonian(n, 50, 9, allow_odd_y=False, max_weight=3)
        Ui = [(1 << (n - 1)) | 5, (1 << (n - 1)) | 6, 3, 5, 6, (1 << (n - 2))]
        ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
        ref = oracle.forward(Ui, np.zeros(6), None, ref_ham)
        ham = nqs.Hamiltonian(x, z, c, n)
        batch = nqs.Batch(ham, to_dev_u(pack_ints(Ui, n)))
        res = nqs.evaluate(batch, np.zeros(6), None, "fp64")
        assert np.abs(res["eloc_re"].cpu().numpy() - np.array([e.real for e in ref["eloc"]])).max() < TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_stored_matrix_elements_h28(h28, prec):
    """hpair holds H of every pair (checked against the oracle on sampled pairs);
    the adjoint that reads it equals the one that recomputes, bitwise."""
    inst, ref_ham, ref = h28
    ham, batch = gpu_objects(inst)
    res = nqs.evaluate(batch, inst.logpsi_re, None, prec, keep_h=True)
    rp, pj, pk = res["pairs"]
    hp = res["hpair"]
    h = hp.double().cpu().numpy() if prec == "fp64" else hp.double().sum(dim=1).cpu().numpy()
    rows = np.repeat(np.arange(inst.n_unq), np.diff(rp.cpu().numpy()))
    jj = pj.cpu().numpy().view(np.uint32)
    Ui = unpack_ints(inst.U)
    rng = np.random.default_rng(2)
    for q in rng.choice(len(jj), 300, replace=False):
        want = oracle.matrix_element(Ui[rows[q]], Ui[int(jj[q])], ref_ham)
        assert abs(h[q] - want.real) < (1e-12 if prec == "fp64" else 1e-7) * max(1.0, abs(want))
    g = torch.from_numpy(np.random.default_rng(3).normal(0, 1e-3, inst.n_unq)).cuda()
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    a = torch.from_numpy(inst.logpsi_re).cuda()
    args = (batch, a, None, res["eloc_re"], None, res["hdiag"], res["evar"], g, None, gE, res["pairs"], prec)
    x, _ = nqs.local_energy_backward(*args)
    y, _ = nqs.local_energy_backward(*args, hpair=hp)
    assert torch.equal(x, y)


def test_cross_sector_pairs_have_vanishing_elements():
    """Samples from every particle-number sector of the 12-qubit molecule: the
    CUDA path lists the oracle's pairs (patterns do connect sectors) and the
    stored element of every cross-sector pair vanishes, because the molecular
    H conserves both spin counts."""
    inst = config_instance("h12")
    ref_ham = oracle_for(inst)
    scale = math.fsum(abs(float(c)) for c in inst.coef)
    rng = np.random.default_rng(17)
    U_ints = sorted(int(v) for v in rng.choice(1 << 12, size=400, replace=False))
    ham = nqs.Hamiltonian.from_instance(inst)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(U_ints, 12)))
    lre = np.random.default_rng(18).normal(0, 1, len(U_ints))
    res = nqs.evaluate(batch, lre, None, "fp64", keep_h=True)
    batch.status()
    rows, j, k = pair_set_gpu(batch, res["pairs"])
    want = sorted(oracle.find_coupled_pairs(U_ints, ref_ham, "terms"))
    assert sorted(zip(rows.tolist(), j.tolist())) == want
    h = res["hpair"].double().cpu().numpy()
    even = int("01" * 6, 2)
    cross = 0
    for q in range(len(j)):
        a, b = U_ints[rows[q]], U_ints[int(j[q])]
        if (bin(a & even).count("1") != bin(b & even).count("1")
                or bin(a & ~even).count("1") != bin(b & ~even).count("1")):
            cross += 1
            assert abs(h[q]) <= 1e-12 * scale
    assert cross > 0
