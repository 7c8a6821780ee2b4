"""Complex Hamiltonians (strings with an odd number of Y) on the GPU (GPU required).

A string with an odd number of Y has the imaginary coefficient h i^{|Y|}
(Eq. pauli_melem), so H is complex Hermitian and the local energies are
complex even for real amplitudes.  Against the oracle (whose matrix elements
are pinned to Kronecker-product Pauli matrices, odd |Y| included):

* pair lists bit-exact (they depend on the XY patterns only);
* E_loc^var (real and imaginary parts) and E^var: FP64 within 1e-9 Ha,
  FP32C within 1e-6 Ha, for real and complex log-amplitudes;
* the stored per-pair matrix elements, and H_ij = conj(H_ji) over the lists;
* the adjoint (upstream on Re and Im E_loc and on E^var) against the oracle's
  vector-Jacobian product, with stored and recomputed matrix elements alike.
"""

import numpy as np
import pytest
import torch

import oracle
from synth import pack_ints, random_pauli_hamiltonian

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs
    from gpu_helpers import to_dev_u, pair_set_gpu

TOL = {"fp64": 1e-9, "fp32c": 1e-6}


def _instance(seed, n, m, T):
    x, z, c = random_pauli_hamiltonian(n, T, seed, allow_odd_y=True, max_weight=4)
    pyrng = __import__("random").Random(seed)
    ints = set()
    while len(ints) < m:
        ints.add(pyrng.getrandbits(n))
    Ui = sorted(ints)
    pyrng.shuffle(Ui)
    return x, z, c, Ui


CASES = [(1, 6, 40, 30), (2, 10, 300, 120), (3, 20, 500, 400), (4, 70, 300, 200), (5, 130, 200, 150)]


@pytest.mark.parametrize("seed,n,m,T", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("cplx_psi", [False, True])
def test_complex_h_forward(seed, n, m, T, prec, cplx_psi):
    x, z, c, Ui = _instance(seed, n, m, T)
    ham = nqs.Hamiltonian(x, z, c, n)
    assert ham.complex
    rng = np.random.default_rng(seed)
    lre = rng.normal(0, 0.5, size=m)
    lim = rng.uniform(-np.pi, np.pi, size=m) if cplx_psi else None
    ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
    ref = oracle.forward(Ui, lre, lim, ref_ham)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(Ui, n)))
    res = nqs.evaluate(batch, lre, lim, prec, keep_h=True)
    batch.status()
    rows, j, k = pair_set_gpu(batch, res["pairs"])
    assert sorted(zip(rows.tolist(), j.tolist())) == sorted(ref["pairs"])
    want = np.array(ref["eloc"])
    tol = TOL[prec]
    assert np.abs(res["eloc_re"].cpu().numpy() - want.real).max() < tol
    assert np.abs(res["eloc_im"].cpu().numpy() - want.imag).max() < tol
    assert abs(res["evar"][0].item() - ref["e_var"].real) < tol
    # stored matrix elements: the oracle's values, and Hermitian over the lists
    hp = res["hpair"].double().cpu().numpy().reshape(len(j), -1)
    h = hp[:, 0] + 1j * hp[:, 1] if prec == "fp64" else (hp[:, 0] + hp[:, 1]) + 1j * (hp[:, 2] + hp[:, 3])
    for q in np.random.default_rng(1).choice(len(j), min(300, len(j)), replace=False):
        w = oracle.matrix_element(Ui[rows[q]], Ui[j[q]], ref_ham)
        assert abs(h[q] - w) < (1e-12 if prec == "fp64" else 1e-7) * max(1.0, abs(w))
    index = {(int(a), int(b)): q for q, (a, b) in enumerate(zip(rows, j))}
    for (a, b), q in list(index.items())[:2000]:
        assert abs(h[q] - np.conj(h[index[(b, a)]])) < (1e-12 if prec == "fp64" else 1e-7) * max(1.0, abs(h[q]))


@pytest.mark.parametrize("seed,n,m,T", CASES[1:4])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_complex_h_adjoint(seed, n, m, T, prec):
    x, z, c, Ui = _instance(seed, n, m, T)
    rng = np.random.default_rng(seed + 100)
    lre = rng.normal(0, 0.5, size=m)
    lim = rng.uniform(-np.pi, np.pi, size=m)
    g_re = rng.normal(0, 1.0, size=m)
    g_im = rng.normal(0, 1.0, size=m)
    ref_ham = oracle.prepare_hamiltonian(x, z, c, n)
    pairs_ref = oracle.find_coupled_pairs(Ui, ref_ham, "terms")
    want_re, want_im = oracle.local_energy_vjp(Ui, lre, lim, ref_ham, pairs_ref, g_re, g_im, g_evar=0.7)
    ham = nqs.Hamiltonian(x, z, c, n)
    batch = nqs.Batch(ham, to_dev_u(pack_ints(Ui, n)))
    res = nqs.evaluate(batch, lre, lim, prec, keep_h=True)
    gE = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    args = (batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"], res["evar"], g_re, g_im, gE,
            res["pairs"], prec)
    gr, gi = nqs.local_energy_backward(*args)
    gr2, gi2 = nqs.local_energy_backward(*args, hpair=res["hpair"])
    batch.status()
    assert torch.equal(gr, gr2) and torch.equal(gi, gi2)
    tol = TOL[prec]
    scale = max(1.0, float(np.abs(want_re).max()), float(np.abs(want_im).max()))
    assert np.abs(gr.cpu().numpy() - want_re).max() < tol * scale
    assert np.abs(gi.cpu().numpy() - want_im).max() < tol * scale
