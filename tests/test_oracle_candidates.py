"""The oracle's exact local energy (Eq. local_energy) pinned without its own formula.

* Dense matrix-vector products (Kronecker-product Pauli matrices from
  tests/dense_ref.py, no bit arithmetic): for any psi on the whole Hilbert
  space, E_loc(x) = (H psi)(x) / psi(x), including Hamiltonians with an odd
  number of Y (complex H) and complex psi.
* Every x' with H[x, x'] != 0 in the dense matrix is a candidate of x.
* Brute force over all 2^N basis vectors: the candidates of x are exactly
  the x' for which some term flips x into x'.
* Eigenvector identity at 12 qubits: with psi the exact ground state of the
  whole (N_e, S_z) sector, E_loc(x) = E_0 for every x of the sector
  (the surrogate E_loc^var needs U = the whole sector for this; the exact
  local energy needs only the candidates).
* Restricted to the candidates that lie in U, the sum is E_loc^var.
* A planted mistake (a candidate set that misses the diagonal pattern)
  fails the dense pin.
"""

import cmath
import math

import numpy as np
import pytest

import oracle
from synth import random_pauli_hamiltonian, config_instance, unpack_ints
from dense_ref import pauli_dense, sector_indices


def _random_state(n, rng, complex_psi):
    a = rng.normal(0.0, 0.7, 1 << n)
    b = rng.uniform(-math.pi, math.pi, 1 << n) if complex_psi else np.zeros(1 << n)
    return a, b


@pytest.mark.parametrize("seed,odd,cplx", [(1, False, False), (2, True, True), (3, False, True), (4, True, False)])
def test_full_local_energy_equals_dense_matvec(seed, odd, cplx):
    n = 6
    x, z, c = random_pauli_hamiltonian(n, 50, seed, allow_odd_y=odd, max_weight=4)
    D = pauli_dense(x, z, c, n)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    rng = np.random.default_rng(seed)
    a, b = _random_state(n, rng, cplx)
    psi = np.exp(a + 1j * b)
    Hpsi = D @ psi
    U = sorted(rng.choice(1 << n, size=20, replace=False).tolist())
    rows, C = oracle.full_candidates(U, ham)
    assert C == sorted(set(C))
    got = oracle.local_energy_full(U, a[U], b[U], ham, C, a[C], b[C])
    for i, xv in enumerate(U):
        want = Hpsi[xv] / psi[xv]
        assert abs(got[i] - want) < 1e-10 * max(1.0, abs(want)), (xv, got[i], want)
        cands = {xp for (xp, _, _) in rows[i]}
        support = set(np.flatnonzero(np.abs(D[xv]) > 1e-13).tolist())
        assert support <= cands
        for (xp, xy, h) in rows[i]:
            assert xp ^ xv == xy
            assert abs(h - D[xv, xp]) < 1e-12


def test_candidates_brute_force():
    n = 6
    x, z, c = random_pauli_hamiltonian(n, 30, 9, allow_odd_y=True, max_weight=3)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    flips = {t.XY for t in ham.terms}
    U = [0, 5, 17, 42, 63]
    rows, C = oracle.full_candidates(U, ham)
    allc = set()
    for i, xv in enumerate(U):
        want = {xp for xp in range(1 << n) if (xv ^ xp) in flips}
        assert {xp for (xp, _, _) in rows[i]} == want
        allc |= want
    assert C == sorted(allc)


def test_exact_ground_state_fixed_point_h12():
    inst = config_instance("h12", use_cache=False)
    D = pauli_dense(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits, dense=False)
    sec = sector_indices(inst.meta["n_orb"], inst.n_alpha, inst.n_beta)
    Hs = D[sec][:, sec].toarray().real
    evals, evecs = np.linalg.eigh(Hs)
    psi_sec = evecs[:, 0]
    psi = np.zeros(1 << inst.n_qubits)
    psi[sec] = psi_sec
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    keep = [s for s, p in zip(sec, psi_sec) if abs(p) > 1e-6]
    U = keep[:40]
    rows, C = oracle.full_candidates(U, ham)
    # log psi of the candidates; those outside the sector have psi = 0 -> a very negative log
    with np.errstate(divide="ignore"):
        a = np.where(np.abs(psi) > 0, np.log(np.abs(psi) + 1e-300), -745.0)
    b = np.where(psi < 0, math.pi, 0.0)
    got = oracle.local_energy_full(U, a[U], b[U], ham, C, a[C], b[C])
    for g in got:
        assert abs(g.real - evals[0]) < 1e-8 and abs(g.imag) < 1e-8


def test_restriction_to_batch_is_the_surrogate():
    inst = config_instance("h28", n_unq=120, use_cache=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    U = unpack_ints(inst.U)
    rows, C = oracle.full_candidates(U, ham)
    pos = {v: j for j, v in enumerate(U)}
    # psi = 0 outside U (log psi very negative): the full sum reduces to the one over U
    ca = np.array([inst.logpsi_re[pos[v]] if v in pos else -745.0 for v in C])
    full = oracle.local_energy_full(U, inst.logpsi_re, None, ham, C, ca)
    var, _ = oracle.local_energy_var(U, inst.logpsi_re, None, ham)
    for f, v in zip(full, var):
        assert abs(f - v) < 1e-9 * max(1.0, abs(v))


def test_planted_missing_diagonal_fails():
    n = 5
    x, z, c = random_pauli_hamiltonian(n, 30, 11, allow_odd_y=False, max_weight=3)
    D = pauli_dense(x, z, c, n)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    assert 0 in ham.xy_list
    rng = np.random.default_rng(1)
    a, b = _random_state(n, rng, False)
    psi = np.exp(a)
    want = (D @ psi)[3] / psi[3]
    # the mutant skips the XY = 0 pattern (the diagonal term)
    import oracle.candidates as oc
    terms = [h * cmath.exp(a[3 ^ xy] - a[3]) for xy in ham.xy_list if xy != 0
             for h in [oracle.matrix_element(3, 3 ^ xy, ham)]]
    mutant = math.fsum(t.real for t in terms)
    good = oc.local_energy_full([3], a[[3]], None, ham, list(range(1 << n)), a)[0]
    assert abs(good.real - want.real) < 1e-10
    assert abs(mutant - want.real) > 1e-6
