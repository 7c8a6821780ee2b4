"""Oracle pinned to dense matrices built without its bit arithmetic.

* Kronecker-product Pauli matrices (tests/dense_ref.py) for Eq. (pauli_melem)
  and MatrixElement, including strings with an odd number of Y (complex H).
* Exact diagonalisation at 12 qubits: with U = the whole (N_e, S_z) sector
  and psi its exact ground state, E_loc^var(x) = E_0 for every x and
  E^var = E_0 (eigenvector identity); E^var >= E_0 for any psi (variational
  bound); E^var is the Rayleigh quotient psi^T H_UU psi / psi^T psi.
* Slater-Condon diagonal energies from the integrals for H_xx.
* The Jordan-Wigner generator against direct fermionic action (8 qubits).
"""

import math

import numpy as np
import pytest

import oracle
from synth import (pack_ints, unpack_ints, random_pauli_hamiltonian, molecular_integrals,
                   jordan_wigner, hf_energy_from_integrals, config_instance,
                   all_sector_determinants)
from dense_ref import pauli_dense, fermion_dense, sector_indices


@pytest.mark.parametrize("seed,odd", [(1, True), (2, True), (3, False)])
def test_matrix_element_vs_kron(seed, odd):
    n = 5
    x, z, c = random_pauli_hamiltonian(n, 40, seed, allow_odd_y=odd)
    D = pauli_dense(x, z, c, n)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    for a in range(1 << n):
        for b in range(1 << n):
            h = oracle.matrix_element(a, b, ham)
            assert abs(h - D[a, b]) < 1e-12, (a, b, h, D[a, b])
            assert abs(oracle.matrix_element_all_terms(a, b, ham) - D[a, b]) < 1e-12


def test_pauli_element_single_terms_vs_kron():
    n = 4
    rng = np.random.default_rng(7)
    from dense_ref import pauli_string_matrix
    for _ in range(60):
        x = int(rng.integers(0, 1 << n)); z = int(rng.integers(0, 1 << n))
        t = oracle.PauliTerm(h=1.0, X=x & ~z, Y=x & z, Z=z & ~x)
        M = pauli_string_matrix(x, z, n).toarray()
        for a in range(1 << n):
            for b in range(1 << n):
                assert oracle.pauli_matrix_element(a, b, t) == pytest.approx(M[a, b], abs=0)


def test_jordan_wigner_vs_fermionic_action():
    h1, eri, _ = molecular_integrals(4, 99, irrep_bits=0)
    x, z, c = jordan_wigner(h1, eri)
    Hp = pauli_dense(x, z, c, 8)
    Hf = fermion_dense(h1, eri, 4)
    assert np.abs(Hp.imag).max() < 1e-12
    assert np.abs(Hp.real - Hf).max() < 1e-10


@pytest.fixture(scope="module")
def h12():
    inst = config_instance("h12", use_cache=False)
    D = pauli_dense(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits, dense=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    sec = sector_indices(inst.meta["n_orb"], inst.n_alpha, inst.n_beta)
    Hs = D[sec][:, sec].toarray()
    assert np.abs(Hs.imag).max() < 1e-12
    Hs = Hs.real
    evals, evecs = np.linalg.eigh(Hs)
    return inst, D, ham, sec, Hs, evals, evecs


def test_sector_batch_is_the_sector(h12):
    inst, D, ham, sec, Hs, evals, evecs = h12
    assert sorted(unpack_ints(inst.U)) == list(sec)


def test_exact_ground_state_fixed_point(h12):
    inst, D, ham, sec, Hs, evals, evecs = h12
    psi = evecs[:, 0]
    keep = np.abs(psi) > 1e-9
    U = list(sec[keep])
    lre = np.log(np.abs(psi[keep]))
    lim = np.where(psi[keep] < 0, np.pi, 0.0)
    res = oracle.forward(U, lre, lim, ham)
    E0 = evals[0]
    # only amplitudes that are not tiny: E_loc divides by psi(x)
    big = np.abs(psi[keep]) > 1e-4
    for e, b in zip(res["eloc"], big):
        if b:
            assert abs(e - E0) < 1e-9 * max(1.0, abs(E0))
    assert abs(res["e_var"] - E0) < 1e-10 * max(1.0, abs(E0))
    # the surrogate equals the full local energy when U holds the whole support
    full = (Hs @ psi)[keep] / psi[keep]
    assert np.allclose(full[big], E0, atol=1e-9 * abs(E0))


def test_rayleigh_quotient_and_variational_bound(h12):
    inst, D, ham, sec, Hs, evals, evecs = h12
    rng = np.random.default_rng(5)
    for trial in range(4):
        m = int(rng.integers(20, len(sec)))
        pick = np.sort(rng.choice(len(sec), size=m, replace=False))
        U = list(sec[pick])
        lre = rng.normal(0.0, 1.0, size=m)
        lim = np.where(rng.random(m) < 0.3, np.pi, 0.0)
        res = oracle.forward(U, lre, lim, ham)
        psi = np.exp(lre) * np.cos(lim)
        Huu = Hs[np.ix_(pick, pick)]
        rq = psi @ Huu @ psi / (psi @ psi)
        assert abs(res["e_var"].real - rq) < 1e-11 * max(1.0, abs(rq))
        assert abs(res["e_var"].imag) < 1e-11 * max(1.0, abs(rq))
        assert res["e_var"].real >= evals[0] - 1e-10
        # E_loc^var of every row is (H_UU psi)_x / psi_x
        want = (Huu @ psi) / psi
        for e, w in zip(res["eloc"], want):
            assert abs(e - w) < 1e-9 * max(1.0, abs(w))


def test_matrix_elements_vs_dense_12q(h12):
    inst, D, ham, sec, Hs, evals, evecs = h12
    rng = np.random.default_rng(11)
    Dd = D.tocsr()
    for _ in range(300):
        a = int(rng.choice(sec)); b = int(rng.choice(sec))
        assert abs(oracle.matrix_element(a, b, ham) - Dd[a, b]) < 1e-12
    # all pairs of the sector batch
    pairs = oracle.find_coupled_pairs(list(sec), ham, "terms")
    for (i, j) in pairs[:2000]:
        assert abs(oracle.matrix_element(int(sec[i]), int(sec[j]), ham) - Dd[sec[i], sec[j]]) < 1e-12
    # every nonzero of the sector block is a listed pair
    listed = set(pairs)
    nz = np.argwhere(np.abs(Hs) > 1e-13)
    for (i, j) in nz:
        assert (int(i), int(j)) in listed


@pytest.mark.parametrize("name", ["h12", "h28"])
def test_diagonal_vs_slater_condon(name):
    inst = config_instance(name, n_unq=None if name == "h12" else 300, use_cache=False)
    n_orb = inst.meta["n_orb"]
    h1, eri, _ = molecular_integrals(n_orb, 1000 + inst.n_qubits,
                                     irrep_bits=__import__("synth").CONFIGS[name][3])
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    for v in unpack_ints(inst.U)[:40]:
        occ_a = [p for p in range(n_orb) if (v >> (2 * p)) & 1]
        occ_b = [p for p in range(n_orb) if (v >> (2 * p + 1)) & 1]
        want = hf_energy_from_integrals(h1, eri, occ_a, occ_b)
        got = oracle.matrix_element(v, v, ham)
        assert abs(got - want) < 1e-10 * max(1.0, abs(want))
