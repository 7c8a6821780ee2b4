"""Row sharding of one sample batch across ranks (one GPU per rank).

Rows of U are independent in FindCoupledPairs, E_loc^var and the adjoint:
every rank stages the whole batch (x' is looked up among all samples), owns
a contiguous block of rows balanced by pair counts, and computes its rows'
pairs, local energies and gradient.  E^var (Eq. variational_energy) needs
every row: each rank reduces its block to a triple [E_r, max_r, sum_r]
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
