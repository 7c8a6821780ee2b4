"""Row sharding across ranks: block partition, E^var combination, gloo exchange.

The combination of block triples is checked against the oracle's E^var of
the whole batch (Eq. variational_energy), on one process and across two
gloo ranks (CPU, world size 2, 127.0.0.1).
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from synth import config_instance

nqs = pytest.importorskip("paper_2408_07625_gb300")
try:
    nqs.load_library()
    HAVE_LIB = True
except Exception:  # the library is built by the build step
    HAVE_LIB = False
needs_lib = pytest.mark.skipif(not HAVE_LIB, reason="libnqs.so not built")


def _block_triple(a, e):
    """[E_r, max_r, sum_r] of one block, straight from the definition."""
    if len(a) == 0:
        return [0.0, -np.inf, 0.0]
    m = float(np.max(a))
    w = np.exp(2.0 * (a - m))
    return [float(np.sum(w * e) / np.sum(w)), m, float(np.sum(w))]


@pytest.fixture(scope="module")
def h12_ref():
    inst = config_instance("h12", use_cache=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    ref = oracle.forward(inst.U, inst.logpsi_re, None, ham)
    eloc = np.array([e.real for e in ref["eloc"]])
    return inst, eloc, ref["e_var"].real, ref


def test_row_blocks_partition():
    from paper_2408_07625_gb300.sharding import row_blocks
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 500, size=1000)
    counts[17] = 20000  # one heavy row
    rp = np.concatenate([[0], np.cumsum(counts)])
    for ws in (1, 2, 3, 8):
        blocks = row_blocks(rp, ws)
        assert blocks[0][0] == 0 and blocks[-1][1] == 1000
        assert all(b[1] == c[0] for b, c in zip(blocks, blocks[1:]))
        work = [int(rp[r1] - rp[r0]) + 8 * (r1 - r0) for r0, r1 in blocks]
        ideal = (rp[-1] + 8 * 1000) / ws
        assert max(work) <= ideal + 20000 + 500 + 8  # off by at most the heaviest row
    tiny = row_blocks([0, 5], 4)  # fewer rows than ranks: some blocks are empty
    assert sum(r1 - r0 for r0, r1 in tiny) == 1 and tiny[-1][1] == 1


@needs_lib
def test_combine_host_matches_whole_batch(h12_ref):
    from paper_2408_07625_gb300.sharding import combine_parts
    inst, eloc, evar, _ = h12_ref
    a = inst.logpsi_re
    for cuts in ([0, 225], [0, 100, 225], [0, 1, 2, 224, 225], [0, 0, 50, 50, 225]):
        parts = torch.tensor([_block_triple(a[r0:r1], eloc[r0:r1]) for r0, r1 in zip(cuts, cuts[1:])],
                             dtype=torch.float64)
        out = combine_parts(parts)
        assert abs(out[0].item() - evar) < 1e-12
        assert out[1].item() == np.max(a)
        assert abs(out[2].item() - np.sum(np.exp(2 * (a - a.max())))) < 1e-12


def _rank_main(rank, ws, port, a, eloc, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2408_07625_gb300.sharding import combine_evar, row_blocks
    rp = np.arange(len(a) + 1) * 3  # equal work per row
    r0, r1 = row_blocks(rp, ws)[rank]
    part = torch.tensor(_block_triple(a[r0:r1], eloc[r0:r1]), dtype=torch.float64)
    out = combine_evar(part)
    q.put((rank, (r0, r1), out.tolist()))
    torch.distributed.destroy_process_group()


@needs_lib
def test_gloo_two_ranks_exchange(h12_ref):
    inst, eloc, evar, _ = h12_ref
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, inst.logpsi_re, eloc, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1][1] == res[1][1][0] and res[0][1][0] == 0 and res[1][1][1] == inst.n_unq
    for _, _, out in res:
        assert abs(out[0] - evar) < 1e-12
    assert res[0][2] == res[1][2]  # every rank holds the same triple


def _owner(bounds, row):
    return int(np.searchsorted(np.asarray(bounds), row, side="right") - 1)


def _exchange_main(rank, ws, port, bounds, records, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2408_07625_gb300.sharding import exchange_records
    m = len(records)
    mine = records[rank * m // ws:(rank + 1) * m // ws]   # this rank's search slice
    groups = [[] for _ in range(ws)]
    for rec in mine:  # routed as nqs_route_records does: to the owner of each endpoint row, once per owner
        owners = {_owner(bounds, rec[0]), _owner(bounds, rec[1])}
        for d in sorted(owners):
            groups[d].append(rec)
    counts = [len(g) for g in groups]
    flat = [r for g in groups for r in g]
    send = tuple(torch.tensor([r[c] for r in flat], dtype=torch.int32) for c in range(3))
    recv = exchange_records(send, counts)
    q.put((rank, sorted(zip(*(t.tolist() for t in recv)))))
    torch.distributed.destroy_process_group()


def test_gloo_record_exchange():
    """The all-to-all of the sharded search: every rank receives exactly the records
    (from every rank's search slice) that name one of its rows, once."""
    rng = np.random.default_rng(5)
    n, m, ws = 60, 500, 2
    i = rng.integers(0, n, m)
    j = (i + rng.integers(1, n, m)) % n
    records = [(int(a), int(b), int(k)) for a, b, k in zip(i, j, rng.integers(0, 1000, m))]
    bounds = [0, 23, n]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_exchange_main, args=(r, ws, port, bounds, records, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(ws):
        want = sorted(rec for rec in records if bounds[r] <= rec[0] < bounds[r + 1] or bounds[r] <= rec[1] < bounds[r + 1])
        assert res[r] == want
