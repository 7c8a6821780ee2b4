"""FindCoupledPairs without a host wait (GPU required).

nqs_find_coupled_pairs_async enqueues the search and returns; the pair
total stays on the device.  Checked here:

* with room enough, the same row offsets and pair lists as the waiting call
  (bitwise, sorted rows; as sets row by row with NQS_ROWS_UNSORTED), for the
  LoopOverTerms one-pass form and the count + fill forms of LoopOverTerms,
  LoopOverBatch and LoopOverTrie, and the same E_loc^var, E^var and adjoint;
* with too little room, nothing is written, the energy and adjoint calls on
  the workspace leave their outputs alone, the status reports
  NQS_ERR_CAPACITY (-4) with valid row offsets, and the next call that fits
  clears the condition;
* a whole step (search, E_loc^var, E^var, adjoint) with no host wait gives
  the values of the waiting path.
"""

import numpy as np
import pytest
import torch

from synth import config_instance

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import gpu_objects


def _inst():
    return config_instance("h28", n_unq=3000, use_cache=False)


@pytest.mark.parametrize("schedule", ["terms", "batch", "trie"])
def test_async_matches_waiting_call(schedule):
    inst = _inst()
    ham, batch = gpu_objects(inst)
    rp, pj, pk = nqs.coupled_pairs(batch, schedule=schedule)
    total = int(pj.numel())
    arp, apj, apk = nqs.coupled_pairs_async(batch, total + 100, schedule=schedule)
    batch.status()
    assert torch.equal(arp, rp)
    assert int(arp[-1]) == total
    assert torch.equal(apj[:total], pj) and torch.equal(apk[:total], pk)
    # a sub-range of rows
    r0, r1 = 123, 2345
    rp2, pj2, pk2 = nqs.coupled_pairs(batch, r0, r1, schedule=schedule)
    arp2, apj2, apk2 = nqs.coupled_pairs_async(batch, int(pj2.numel()), r0, r1, schedule=schedule)
    batch.status()
    assert torch.equal(arp2, rp2)
    assert torch.equal(apj2, pj2) and torch.equal(apk2, pk2)


def test_async_terms_two_pass_and_unsorted():
    inst = _inst()
    ham, batch = gpu_objects(inst)
    rp, pj, pk = nqs.coupled_pairs(batch)
    total = int(pj.numel())
    # no scratch: count, capacity check, fill
    batch._scratch = None
    row_ptr = torch.empty(batch.n + 1, dtype=torch.int64, device="cuda")
    qj = torch.empty(total, dtype=torch.int32, device="cuda")
    qk = torch.empty(total, dtype=torch.int32, device="cuda")
    lib = nqs.load_library()
    rc = lib.nqs_find_coupled_pairs_async(batch.ham.handle, nqs._ptr(batch.U), batch.n, nqs._ptr(batch.work), 0,
                                          batch.n, nqs.SCHEDULES["terms"], None, 0, nqs._ptr(row_ptr),
                                          nqs._ptr(qj), nqs._ptr(qk), total, nqs._stream(None))
    assert rc == 0
    batch.status()
    assert torch.equal(row_ptr, rp) and torch.equal(qj, pj) and torch.equal(qk, pk)
    # rows left in search order hold the same pairs
    arp, apj, apk = nqs.coupled_pairs_async(batch, total, sort_rows=False)
    batch.status()
    assert torch.equal(arp, rp)
    r = rp.cpu().numpy()
    a_j, a_k = apj.cpu().numpy(), apk.cpu().numpy()
    w_j, w_k = pj.cpu().numpy(), pk.cpu().numpy()
    has_diag = ham.info["has_diag"]
    for i in range(batch.n):
        a, b = r[i] + (1 if has_diag else 0), r[i + 1]
        o = np.argsort(a_j[a:b].view(np.uint32), kind="stable")
        assert np.array_equal(a_j[a:b][o], w_j[a:b]) and np.array_equal(a_k[a:b][o], w_k[a:b])


def test_async_overflow_is_reported_and_cleared():
    inst = _inst()
    ham, batch = gpu_objects(inst)
    rp, pj, pk = nqs.coupled_pairs(batch)
    total = int(pj.numel())
    small = total // 2
    arp, apj, apk = nqs.coupled_pairs_async(batch, small)
    # nothing written to the pair buffers: fill them with a marker first, then search again
    apj.fill_(-7)
    apk.fill_(-7)
    arp, apj, apk = nqs.coupled_pairs_async(batch, small)
    # the energy and adjoint calls skip their rows: outputs keep their contents
    out = (torch.full((batch.n,), float("nan"), dtype=torch.float64, device="cuda"), None,
           torch.full((batch.n,), float("nan"), dtype=torch.float64, device="cuda"))
    er, _, hd = nqs.local_energy(batch, inst.logpsi_re, None, (arp, apj, apk), "fp32c", out=out)
    torch.cuda.synchronize()
    assert torch.isnan(er).all() and torch.isnan(hd).all()
    assert (apj == -7).all() and (apk == -7).all()
    with pytest.raises(nqs.NQSError) as err:
        batch.status()
    assert err.value.code == -4
    assert torch.equal(arp, rp)  # the offsets are valid: the caller sizes from them
    # a call that fits clears the condition
    arp, apj, apk = nqs.coupled_pairs_async(batch, int(arp[-1]))
    batch.status()
    assert torch.equal(apj, pj) and torch.equal(apk, pk)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_async_step_matches_waiting_step(prec):
    inst = _inst()
    ham, batch = gpu_objects(inst)
    g = np.random.default_rng(9).normal(0.0, 1.0, batch.n)
    pairs = nqs.coupled_pairs(batch)
    total = int(pairs[1].numel())
    hp = nqs.pair_h_buffer(total, prec, "cuda")
    er, ei, hd = nqs.local_energy(batch, inst.logpsi_re, None, pairs, prec, hpair=hp)
    ev = nqs.variational_energy(batch, inst.logpsi_re, er)
    gr, _ = nqs.local_energy_backward(batch, inst.logpsi_re, None, er, ei, hd, ev, g, None, [1.0], pairs, prec,
                                      hpair=hp)
    want = [er.clone(), hd.clone(), ev.clone(), gr.clone()]
    cap = total + 4096
    apairs = nqs.coupled_pairs_async(batch, cap, sort_rows=False)
    hp2 = nqs.pair_h_buffer(cap, prec, "cuda")
    er2, ei2, hd2 = nqs.local_energy(batch, inst.logpsi_re, None, apairs, prec, hpair=hp2)
    ev2 = nqs.variational_energy(batch, inst.logpsi_re, er2)
    gr2, _ = nqs.local_energy_backward(batch, inst.logpsi_re, None, er2, ei2, hd2, ev2, g, None, [1.0], apairs, prec,
                                       hpair=hp2)
    batch.status()
    for x, y in zip(want, [er2, hd2, ev2, gr2]):
        assert torch.equal(x, y)


def test_step_captured_in_a_cuda_graph():
    """Staging, the no-wait search, E_loc^var, E^var and the adjoint enqueue no host
    work, so a whole step can be captured once and replayed; a replay on new
    contents of the captured buffers (the batch in another order) gives the eager
    results bitwise."""
    inst = _inst()
    ham, batch = gpu_objects(inst)
    n = batch.n
    U_dev = batch.U.clone()
    a_dev = torch.from_numpy(np.asarray(inst.logpsi_re, dtype=np.float64)).cuda()
    g_dev = torch.from_numpy(np.random.default_rng(3).normal(0.0, 1.0, n)).cuda()
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    total = int(nqs.coupled_pairs(batch)[1].numel())
    cap = total + 2048
    hp = nqs.pair_h_buffer(cap, "fp32c", "cuda")
    out_e = (torch.zeros(n, dtype=torch.float64, device="cuda"), None,
             torch.zeros(n, dtype=torch.float64, device="cuda"))
    out_g = (torch.zeros(n, dtype=torch.float64, device="cuda"), None)
    out_v = torch.zeros(3, dtype=torch.float64, device="cuda")

    def step():
        batch.restage(U_dev)
        pairs = nqs.coupled_pairs_async(batch, cap, sort_rows=False)
        er, ei, hd = nqs.local_energy(batch, a_dev, None, pairs, "fp32c", out=out_e, hpair=hp)
        ev = nqs.variational_energy(batch, a_dev, er, out=out_v)
        nqs.local_energy_backward(batch, a_dev, None, er, ei, hd, ev, g_dev, None, gE, pairs, "fp32c",
                                  out=out_g, hpair=hp)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    perm = torch.from_numpy(np.random.default_rng(5).permutation(n)).cuda()
    U_perm, a_perm, g_perm = batch.U.clone()[perm], a_dev[perm], g_dev[perm]
    for Ux, ax, gx in ((batch.U.clone(), a_dev.clone(), g_dev.clone()), (U_perm, a_perm, g_perm)):
        U_dev.copy_(Ux)
        a_dev.copy_(ax)
        g_dev.copy_(gx)
        graph.replay()
        torch.cuda.synchronize()
        batch.status()
        got = [out_e[0].clone(), out_e[2].clone(), out_v.clone(), out_g[0].clone()]
        # eager reference on a fresh batch of the same contents
        ref = nqs.Batch(ham, Ux)
        pairs = nqs.coupled_pairs(ref)
        er, ei, hd = nqs.local_energy(ref, ax, None, pairs, "fp32c")
        ev = nqs.variational_energy(ref, ax, er)
        gr, _ = nqs.local_energy_backward(ref, ax, None, er, ei, hd, ev, gx, None, gE, pairs, "fp32c")
        ref.status()
        for x, y in zip(got, [er, hd, ev, gr]):
            assert torch.equal(x, y)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_packed_pairs(prec):
    """Pairs as one 64-bit word each (column << 32 | pattern), written by the no-wait
    search with no split pass: the same pairs row by row as the two-array form, and
    E_loc^var, E^var and the adjoint (stored and recomputed H) bitwise the same."""
    inst = _inst()
    ham, batch = gpu_objects(inst)
    g = np.random.default_rng(11).normal(0.0, 1.0, batch.n)
    canon = nqs.coupled_pairs(batch)
    total = int(canon[1].numel())
    cap = total + 512
    rp, words, none = nqs.coupled_pairs_async(batch, cap, sort_rows=False, packed=True)
    batch.status()
    assert none is None and words.dtype == torch.int64
    assert torch.equal(rp, canon[0])
    w = words[:total].cpu().numpy().view(np.uint64)
    cols, pats = (w >> np.uint64(32)).astype(np.int64), (w & np.uint64(0xFFFFFFFF)).astype(np.int64)
    r = rp.cpu().numpy()
    cj = canon[1].cpu().numpy().view(np.uint32).astype(np.int64)
    ck = canon[2].cpu().numpy().view(np.uint32).astype(np.int64)
    has_diag = ham.info["has_diag"]
    for i in range(batch.n):
        a, b = r[i], r[i + 1]
        if has_diag:
            assert cols[a] == i and pats[a] == 0
            a += 1
        o = np.lexsort((pats[a:b], cols[a:b]))
        assert np.array_equal(cols[a:b][o], cj[a:b]) and np.array_equal(pats[a:b][o], ck[a:b])
    for store_h in (True, False):
        res = []
        for pairs in (canon, (rp, words, None)):
            hp = nqs.pair_h_buffer(int(pairs[1].numel()), prec, "cuda") if store_h else None
            er, ei, hd = nqs.local_energy(batch, inst.logpsi_re, None, pairs, prec, hpair=hp)
            ev = nqs.variational_energy(batch, inst.logpsi_re, er)
            gr, _ = nqs.local_energy_backward(batch, inst.logpsi_re, None, er, ei, hd, ev, g, None, [1.0], pairs,
                                              prec, hpair=hp)
            batch.status()
            res.append([er.clone(), hd.clone(), ev.clone(), gr.clone()])
        for x, y in zip(*res):
            assert torch.equal(x, y)
    # the packed form needs rows left in search order and the one-pass search
    with pytest.raises(nqs.NQSError) as err:
        nqs.coupled_pairs_async(batch, cap, sort_rows=True, packed=True)
    assert err.value.code == -2


def test_async_count_only():
    """No pair buffers at all (capacity 0): the row offsets are still written and the
    status reports that the pairs did not fit."""
    inst = _inst()
    ham, batch = gpu_objects(inst)
    rp = nqs.coupled_pairs(batch)[0]
    nqs.coupled_pairs(batch, sort_rows=False)  # sizes the batch's scratch
    row_ptr = torch.empty(batch.n + 1, dtype=torch.int64, device="cuda")
    lib = nqs.load_library()
    for sched in (nqs.SCHEDULES["terms"], nqs.SCHEDULES["terms"] | nqs.ROWS_UNSORTED):
        rc = lib.nqs_find_coupled_pairs_async(batch.ham.handle, nqs._ptr(batch.U), batch.n, nqs._ptr(batch.work), 0,
                                              batch.n, sched, nqs._ptr(batch._scratch), batch._scratch.numel(),
                                              nqs._ptr(row_ptr), None, None, 0, nqs._stream(None))
        assert rc == 0
        with pytest.raises(nqs.NQSError) as err:
            batch.status()
        assert err.value.code == -4
        assert torch.equal(row_ptr, rp)
    # a call with room clears the condition
    nqs.coupled_pairs_async(batch, int(rp[-1]), sort_rows=False)
    batch.status()
