"""Shared helpers for the GPU parity tests (tests only)."""

import numpy as np
import torch

import oracle
import paper_2408_07625_gb300 as nqs


def to_dev_u(U):
    return torch.from_numpy(np.ascontiguousarray(U).view(np.int64)).cuda()


def gpu_objects(inst):
    ham = nqs.Hamiltonian.from_instance(inst)
    batch = nqs.Batch(ham, to_dev_u(inst.U))
    return ham, batch


def pair_set_gpu(batch, pairs, row_begin=0):
    """(i, j) pairs and the XY value of each pair from a CSR on the GPU."""
    rp, pj, pk = pairs
    rp = rp.cpu().numpy()
    j = pj.cpu().numpy().view(np.uint32).astype(np.int64)
    k = pk.cpu().numpy().view(np.uint32).astype(np.int64)
    rows = np.repeat(np.arange(row_begin, row_begin + len(rp) - 1), np.diff(rp))
    return rows, j, k


def oracle_for(inst):
    return oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
