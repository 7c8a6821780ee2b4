"""84 qubits (two 64-bit words per sample), 1.15e6 Pauli terms, 2e5 peaked samples.

Forward E^var in FP32C and FP64; sampled rows against the oracle (every row
is compared in test_gpu_full_parity.py); the adjoint
through the autograd function with the pair list recomputed in row chunks,
checked against central finite differences (h = 1e-4) at full size and against
the oracle's gradient on a 300-sample batch of the same Hamiltonian.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import config_instance, pack_ints, unpack_ints

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, gpu_objects, pair_set_gpu, oracle_for


@pytest.fixture(scope="module")
def h84():
    inst = config_instance("h84")
    ham, batch = gpu_objects(inst)
    return inst, ham, batch


def test_h84_forward_rows_and_precision(h84):
    inst, ham, batch = h84
    assert ham.n_words == 2
    r64 = nqs.evaluate(batch, inst.logpsi_re, None, "fp64")
    r32 = nqs.evaluate(batch, inst.logpsi_re, None, "fp32c")
    assert r64["n_pairs"] == r32["n_pairs"] > 0
    assert (r64["eloc_re"] - r32["eloc_re"]).abs().max().item() < 1e-6
    assert abs(r64["evar"][0].item() - r32["evar"][0].item()) < 1e-6
    ro = oracle.RowOracle.from_instance(inst)
    rp = r32["pairs"][0].cpu().numpy()
    j = r32["pairs"][1].cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(84)
    for i in rng.choice(inst.n_unq, size=12, replace=False):
        rr = ro.row(int(i))
        assert sorted(j[rp[i]:rp[i + 1]].tolist()) == sorted(rr["j"])
        assert abs(r64["eloc_re"][i].item() - rr["eloc"].real) < 1e-9
        assert abs(r32["eloc_re"][i].item() - rr["eloc"].real) < 1e-6


def test_h84_adjoint_chunked_vs_finite_differences(h84):
    inst, ham, batch = h84
    lre = torch.from_numpy(inst.logpsi_re).cuda().requires_grad_(True)
    n_pairs = nqs.count_pairs(batch)[1]
    er, ei, ev = nqs.LocalEnergy.apply(batch, lre, None, "fp64", n_pairs // 5)  # forces row chunks
    g = torch.from_numpy(np.random.default_rng(5).normal(size=inst.n_unq) * 1e-3).cuda()
    (ev + (g * er).sum()).backward()
    grad = lre.grad.detach().cpu().numpy()
    base = inst.logpsi_re.copy()
    h = 1e-4
    rng = np.random.default_rng(6)
    for y in rng.choice(inst.n_unq, size=5, replace=False):
        vals = []
        for sgn in (1, -1):
            l = base.copy(); l[y] += sgn * h
            res = nqs.evaluate(batch, l, None, "fp64")
            vals.append(res["evar"][0].item() + float((g * res["eloc_re"]).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[y]) < 2e-6 * max(1.0, abs(fd)), (y, fd, grad[y])


def test_h84_gradient_against_oracle_subset(h84):
    inst, ham, _ = h84
    rng = np.random.default_rng(7)
    # a connected subset: the 300 lowest-rank samples (they couple to each other)
    pick = np.argsort(inst.ranks, kind="stable")[:300]
    U = inst.U[pick]
    lre = inst.logpsi_re[pick]
    batch = nqs.Batch(ham, to_dev_u(U))
    ref_ham = oracle_for(inst)
    Ui = unpack_ints(U)
    pairs = oracle.find_coupled_pairs(Ui, ref_ham)
    assert len(pairs) > 600
    gr = rng.normal(size=300)
    want, _ = oracle.local_energy_vjp(Ui, lre, None, ref_ham, pairs, gr, None, 0.8)
    res = nqs.evaluate(batch, lre, None, "fp32c")
    got, _ = nqs.local_energy_backward(batch, lre, None, res["eloc_re"], None, res["hdiag"], res["evar"],
                                       torch.from_numpy(gr).cuda(), None,
                                       torch.tensor([0.8], dtype=torch.float64).cuda(), res["pairs"], "fp32c")
    assert np.abs(got.cpu().numpy() - want).max() < 1e-6
