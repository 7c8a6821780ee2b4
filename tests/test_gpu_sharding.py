"""Row-sharded evaluation on one GPU: the blocks of every rank run one after
another in one process (no collective), then their E^var triples are
combined on the device.  Local energies must equal the unsharded call
bitwise (a row's pairs do not depend on the row range), E^var and the
gradient must agree to rounding, and the device combination must match the
host one.
"""

import numpy as np
import pytest
import torch

from synth import config_instance

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from paper_2408_07625_gb300.sharding import row_blocks, combine_parts
    from gpu_helpers import gpu_objects


@pytest.mark.parametrize("ws", [2, 3, 8])
def test_sharded_rows_match_whole_batch(ws):
    inst = config_instance("h28", n_unq=3000, use_cache=False)
    ham, batch = gpu_objects(inst)
    a = torch.from_numpy(inst.logpsi_re).cuda()
    g = torch.from_numpy(np.random.default_rng(3).normal(0, 1e-3, inst.n_unq)).cuda()
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    full = nqs.evaluate(batch, a, None, "fp32c")
    gfull, _ = nqs.local_energy_backward(batch, a, None, full["eloc_re"], None, full["hdiag"], full["evar"],
                                         g, None, gE, full["pairs"], "fp32c")
    blocks = row_blocks(full["row_ptr"].cpu().numpy(), ws)
    er = torch.zeros_like(a); hd = torch.zeros_like(a)
    parts, pairs = [], []
    for r0, r1 in blocks:
        p = nqs.coupled_pairs(batch, r0, r1)
        pairs.append(p)
        nqs.local_energy(batch, a, None, p, "fp32c", r0, r1, (er, None, hd))
        parts.append(nqs.variational_energy(batch, a[r0:r1], er[r0:r1]))
    evar = combine_parts(torch.stack(parts))
    assert torch.equal(er, full["eloc_re"])
    assert abs(evar[0].item() - full["evar"][0].item()) < 1e-10
    assert evar[1].item() == full["evar"][1].item()
    gr = torch.zeros_like(a)
    for (r0, r1), p in zip(blocks, pairs):
        nqs.local_energy_backward(batch, a, None, er, None, hd, evar, g, None, gE, p, "fp32c", r0, r1,
                                  out=(gr, None))
    assert (gr - gfull).abs().max().item() <= 1e-12 * max(1.0, gfull.abs().max().item())


def test_device_combine_matches_host():
    rng = np.random.default_rng(5)
    for k in (1, 2, 7, 64):
        parts = np.stack([rng.normal(100, 5, k), rng.normal(0, 3, k), rng.uniform(0.5, 1e4, k)], axis=1)
        parts[0, 2] = 0.0  # an empty block is skipped
        if k == 1:
            parts[0, 2] = 3.0
        h = combine_parts(torch.from_numpy(parts))
        d = combine_parts(torch.from_numpy(parts).cuda())
        assert np.allclose(h.numpy(), d.cpu().numpy(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("ws,workload,n_unq", [(2, "h28", 3000), (3, "h28", 3000), (8, "h56", 20000)])
def test_sharded_search_matches_direct_search(ws, workload, n_unq):
    """The sharded FindCoupledPairs, emulated on one GPU: every rank's slice of the
    search's work items, routing of its records to the row owners, the all-to-all
    (concatenation of every slice's group for a rank) and the CSR assembly give each
    rank exactly the lists of searching its rows directly (bitwise); the slices
    together list every unordered pair once."""
    inst = config_instance(workload, n_unq=n_unq, use_cache=False)
    ham, batch = gpu_objects(inst)
    rp_all, _ = nqs.count_pairs(batch)
    blocks = row_blocks(rp_all.cpu().numpy(), ws)
    bounds = [b[0] for b in blocks] + [blocks[-1][1]]
    whole = nqs.half_pairs(batch)
    live = whole[0][:whole[3]].to(torch.int64) & 0xFFFFFFFF
    n_whole = int((live != 0xFFFFFFFF).sum().item())
    routed, n_parts_total = [], 0
    for p in range(ws):
        ri, rj, rk, ns = nqs.half_pairs(batch, part=p, n_parts=ws)
        rec = tuple(t[:ns].clone() for t in (ri, rj, rk)) + (ns,)
        n_parts_total += int(((rec[0].to(torch.int64) & 0xFFFFFFFF) != 0xFFFFFFFF).sum().item())
        oi, oj, ok, counts = nqs.route_records(rec, bounds)
        off = np.concatenate([[0], np.cumsum(counts)])
        routed.append([(oi[off[d]:off[d + 1]], oj[off[d]:off[d + 1]], ok[off[d]:off[d + 1]]) for d in range(ws)])
        batch.status()
    assert n_parts_total == n_whole
    for d, (r0, r1) in enumerate(blocks):
        recv = [torch.cat([routed[p][d][c] for p in range(ws)]) for c in range(3)]
        rp, pj, pk = nqs.pairs_from_records(batch, recv[0], recv[1], recv[2], r0, r1)
        rp_d, pj_d, pk_d = nqs.coupled_pairs(batch, r0, r1)
        assert torch.equal(rp, rp_d) and torch.equal(pj, pj_d) and torch.equal(pk, pk_d)
    batch.status()
