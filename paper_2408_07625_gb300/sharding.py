"""Sharding of one sample batch across ranks (one GPU per rank).

Rows of U are independent in E_loc^var and the adjoint: every rank stages
the whole batch (x' is looked up among all samples), owns a contiguous block
of rows balanced by pair counts, and computes its rows' local energies and
gradient.  FindCoupledPairs is sharded by work, not by rows: the oriented
search finds each unordered pair once, from either of its rows, so rank r
searches slice r of the search's work items (nqs_find_pairs_part) and the
records it finds are exchanged: each goes to the rank(s) owning its two rows
(nqs_route_records, then one all-to-all of record blocks), and every rank
builds its block's CSR lists from what it received (nqs_pairs_from_records),
identical to searching its rows directly.  E^var (Eq. variational_energy)
needs every row: each rank reduces its block to a triple [E_r, max_r, sum_r]
(nqs_variational_energy on its slices) and one all-gather of three doubles
per rank gives every rank the batch's triple (nqs_evar_combine), which the
adjoint of any block then takes as its E^var.
"""

import numpy as np
import torch
import torch.distributed as dist

from . import _check, _ptr, _stream, load_library


def row_blocks(row_ptr, world_size: int, row_cost: int = 8):
    """Contiguous row blocks [(r0, r1), ...] with about equal work each.

    ``row_ptr``: host int64 CSR offsets of the whole batch (n + 1 entries,
    from a count pass).  Work of a row = its pairs + ``row_cost``.
    """
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    cost = (rp - rp[0]) + row_cost * np.arange(n + 1, dtype=np.int64)
    total = int(cost[-1])
    bounds = [0]
    for r in range(1, world_size):
        b = int(np.searchsorted(cost, total * r / world_size, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world_size)]


def exchange_records(send, counts, group=None):
    """All-to-all of routed records: ``send`` = (i, j, k) tensors grouped by
    destination rank with ``counts[r]`` records for rank r; returns this
    rank's received (i, j, k), grouped by source rank."""
    ws = dist.get_world_size(group)
    if len(counts) != ws:
        raise ValueError("one count per rank")
    dev = send[0].device
    c_send = torch.tensor(counts, dtype=torch.int64, device=dev)
    c_recv = torch.empty(ws, dtype=torch.int64, device=dev)
    dist.all_to_all_single(c_recv, c_send, group=group)
    recv_counts = [int(v) for v in c_recv.cpu()]
    out = []
    for t in send:
        r = torch.empty(sum(recv_counts), dtype=t.dtype, device=dev)
        dist.all_to_all_single(r, t.contiguous(), output_split_sizes=recv_counts, input_split_sizes=list(counts),
                               group=group)
        out.append(r)
    return tuple(out)


def sharded_coupled_pairs(batch, bounds, rank: int, world_size: int, exchange=None, stream=None):
    """This rank's CSR lists (row_ptr, j, k) of rows [bounds[rank], bounds[rank + 1]) by the
    sharded search: slice ``rank`` of the work items, routing, exchange, assembly.
    ``exchange(send, counts)`` performs the all-to-all (default: ``exchange_records``
    on the default process group)."""
    from . import half_pairs, pairs_from_records, route_records
    rec = half_pairs(batch, stream=stream, part=rank, n_parts=world_size)
    oi, oj, ok, counts = route_records(rec, bounds, stream=stream)
    recv = (exchange or exchange_records)((oi, oj, ok), counts)
    return pairs_from_records(batch, recv[0], recv[1], recv[2], bounds[rank], bounds[rank + 1], stream=stream)


def combine_parts(parts: torch.Tensor, stream=None):
    """Triple of the whole batch from a [k, 3] tensor of block triples."""
    lib = load_library()
    parts = parts.contiguous()
    out = torch.empty(3, dtype=torch.float64, device=parts.device)
    if parts.is_cuda:
        _check(lib.nqs_evar_combine(_ptr(parts), int(parts.shape[0]), _ptr(out), _stream(stream)))
    else:
        _check(lib.nqs_evar_combine_host(_ptr(parts), int(parts.shape[0]), _ptr(out)))
    return out


def combine_evar(part: torch.Tensor, group=None, stream=None):
    """All-gather every rank's block triple and return the batch's triple."""
    ws = dist.get_world_size(group)
    parts = [torch.empty_like(part) for _ in range(ws)]
    dist.all_gather(parts, part.contiguous(), group=group)
    return combine_parts(torch.stack(parts), stream)
