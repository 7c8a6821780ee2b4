"""Oracle pinned by invariants, brute force, closed forms and finite differences,
plus planted-mistake checks showing that the pins catch plausible bugs."""

import cmath
import math

import numpy as np
import pytest

import oracle
import oracle.energy as oe
import oracle.pairs as op
from synth import (pack_ints, unpack_ints, random_pauli_hamiltonian, config_instance,
                   popcount_rows)
from dense_ref import pauli_dense


def _random_batch(n, m, seed):
    rng = np.random.default_rng(seed)
    vals = rng.choice(1 << n, size=m, replace=False)
    return [int(v) for v in vals]


@pytest.mark.parametrize("seed,n,m,T,maxw", [(1, 6, 30, 25, None), (2, 8, 60, 40, 4),
                                             (3, 10, 120, 80, 4), (4, 3, 8, 12, None)])
def test_variants_agree_with_definition(seed, n, m, T, maxw):
    x, z, c = random_pauli_hamiltonian(n, T, seed, max_weight=maxw)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    U = _random_batch(n, m, seed + 100)
    ref = sorted(oracle.coupled_pairs_definition(U, ham))
    for method in ("terms", "batch", "trie"):
        assert sorted(oracle.find_coupled_pairs(U, ham, method)) == ref, method


def test_variants_agree_molecular_28q():
    inst = config_instance("h28", n_unq=400, use_cache=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    ref = sorted(oracle.find_coupled_pairs(inst.U, ham, "terms"))
    assert sorted(oracle.find_coupled_pairs(inst.U, ham, "batch")) == ref
    assert sorted(oracle.find_coupled_pairs(inst.U, ham, "trie")) == ref
    # two-body Hamiltonian: every coupled pair differs in 0, 2 or 4 bits
    U = unpack_ints(inst.U)
    assert {bin(U[i] ^ U[j]).count("1") for (i, j) in ref} <= {0, 2, 4}
    assert all((i, i) in set(ref) for i in range(len(U)))


@pytest.mark.parametrize("seed,odd", [(5, True), (6, False)])
def test_hermiticity_and_pair_symmetry(seed, odd):
    n = 8
    x, z, c = random_pauli_hamiltonian(n, 60, seed, allow_odd_y=odd, max_weight=4)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    U = _random_batch(n, 80, seed)
    pairs = set(oracle.find_coupled_pairs(U, ham, "terms"))
    for (i, j) in pairs:
        assert (j, i) in pairs
        hij = oracle.matrix_element(U[i], U[j], ham)
        hji = oracle.matrix_element(U[j], U[i], ham)
        assert abs(hij - hji.conjugate()) < 1e-13


def test_no_coupling_across_sectors():
    inst = config_instance("h12", use_cache=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    scale = math.fsum(abs(t.h) for t in ham.terms)
    U = _random_batch(12, 400, 17)  # all sectors mixed
    pairs = oracle.find_coupled_pairs(U, ham, "terms")
    even = int("01" * 6, 2)
    cross = 0
    for (i, j) in pairs:
        a, b = U[i], U[j]
        same = (bin(a & even).count("1") == bin(b & even).count("1")
                and bin(a & ~even).count("1") == bin(b & ~even).count("1"))
        if not same:
            cross += 1
            assert abs(oracle.matrix_element(a, b, ham)) <= 1e-12 * scale
    assert cross > 0  # patterns do list cross-sector pairs; their elements vanish


def test_closed_form_single_terms():
    n = 5
    U = [0b00000, 0b00001, 0b10110, 0b01011]
    l = np.array([0.3, -0.2, 0.7, 0.1])
    # H = Z_2: E_loc(x) = (-1)^{x_2}
    ham = oracle.prepare_hamiltonian(pack_ints([0], n), pack_ints([1 << 2], n), [1.0], n)
    el, _ = oracle.local_energy_var(U, l, None, ham)
    assert [e.real for e in el] == [(-1.0) ** ((u >> 2) & 1) for u in U]
    # H = X_0: couples 00000<->00001 only; E_loc = psi(x')/psi(x)
    ham = oracle.prepare_hamiltonian(pack_ints([1], n), pack_ints([0], n), [1.0], n)
    el, _ = oracle.local_energy_var(U, l, None, ham)
    assert el[0] == pytest.approx(math.exp(l[1] - l[0]), rel=1e-15)
    assert el[1] == pytest.approx(math.exp(l[0] - l[1]), rel=1e-15)
    assert el[2] == 0 and el[3] == 0
    # H = Y_0 Y_1 on 00000 <-> 00011 (x' with x'_0 = x'_1): <x|YY|x'> = i^2 (-1)^{x'_0 + x'_1}
    ham = oracle.prepare_hamiltonian(pack_ints([3], n), pack_ints([3], n), [1.0], n)
    assert oracle.matrix_element(0b00000, 0b00011, ham) == -1.0
    assert oracle.matrix_element(0b00011, 0b00000, ham) == -1.0
    assert oracle.matrix_element(0b00001, 0b00010, ham) == 1.0
    # H = Y_0: <0|Y|1> = -i, <1|Y|0> = +i
    ham = oracle.prepare_hamiltonian(pack_ints([1], n), pack_ints([1], n), [1.0], n)
    assert oracle.matrix_element(0, 1, ham) == -1j
    assert oracle.matrix_element(1, 0, ham) == 1j


def test_merging_and_zero_terms():
    n = 3
    # the same string twice sums; an exactly cancelling string is not a term
    x = pack_ints([1, 1, 2, 2], n)
    z = pack_ints([0, 0, 4, 4], n)
    ham = oracle.prepare_hamiltonian(x, z, [0.25, 0.5, 1.0, -1.0], n)
    assert len(ham.terms) == 1 and ham.terms[0].h == 0.75
    assert ham.xy_list == [1]


# --------------------------------------------------------------------------
# derivatives
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small12():
    inst = config_instance("h12", use_cache=False)
    ham = oracle.prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
    rng = np.random.default_rng(3)
    pick = np.sort(rng.choice(inst.n_unq, size=60, replace=False))
    U = [unpack_ints(inst.U)[i] for i in pick]
    return ham, U


def _loss(U, ham, lre, lim, gr, gi, gE):
    res = oracle.forward(U, lre, lim, ham)
    er = np.array([e.real for e in res["eloc"]])
    ei = np.array([e.imag for e in res["eloc"]])
    return float(gr @ er + gi @ ei + gE * res["e_var"].real)


def test_gradient_closed_form_vs_finite_differences(small12):
    ham, U = small12
    rng = np.random.default_rng(4)
    m = len(U)
    lre = rng.normal(0, 1, size=m)
    lim = np.where(rng.random(m) < 0.3, np.pi, 0.0)
    res = oracle.forward(U, lre, lim, ham)
    g_re, g_im = oracle.energy_gradient_closed_form(lre, res["eloc"], res["e_var"])
    assert abs(g_re.sum()) < 1e-12  # E^var is invariant under a global shift of log psi
    h = 1e-4
    zeros = np.zeros(m)
    for y in rng.choice(m, size=12, replace=False):
        for part, g in (("re", g_re), ("im", g_im)):
            lp, lm = lre.copy(), lre.copy()
            ip, im_ = lim.copy(), lim.copy()
            if part == "re":
                lp[y] += h; lm[y] -= h
            else:
                ip[y] += h; im_[y] -= h
            fd = (_loss(U, ham, lp, ip, zeros, zeros, 1.0) - _loss(U, ham, lm, im_, zeros, zeros, 1.0)) / (2 * h)
            assert abs(fd - g[y]) < 1e-6, (y, part, fd, g[y])


def test_general_vjp_vs_finite_differences_and_closed_form(small12):
    ham, U = small12
    rng = np.random.default_rng(8)
    m = len(U)
    lre = rng.normal(0, 0.7, size=m)
    lim = rng.normal(0, 1.0, size=m)  # general complex phases
    pairs = oracle.find_coupled_pairs(U, ham, "terms")
    gr = rng.normal(size=m); gi = rng.normal(size=m); gE = 0.7
    v_re, v_im = oracle.local_energy_vjp(U, lre, lim, ham, pairs, gr, gi, gE)
    h = 1e-4
    for y in rng.choice(m, size=10, replace=False):
        for part, v in (("re", v_re), ("im", v_im)):
            lp, lm = lre.copy(), lre.copy()
            ip, im_ = lim.copy(), lim.copy()
            if part == "re":
                lp[y] += h; lm[y] -= h
            else:
                ip[y] += h; im_[y] -= h
            fd = (_loss(U, ham, lp, ip, gr, gi, gE) - _loss(U, ham, lm, im_, gr, gi, gE)) / (2 * h)
            assert abs(fd - v[y]) < 2e-6 * max(1.0, abs(fd)), (y, part, fd, v[y])
    # with no upstream on E_loc the chain rule reduces to the closed form
    res = oracle.forward(U, lre, lim, ham)
    c_re, c_im = oracle.energy_gradient_closed_form(lre, res["eloc"], res["e_var"])
    v_re, v_im = oracle.local_energy_vjp(U, lre, lim, ham, pairs, None, None, 1.0)
    assert np.abs(v_re - c_re).max() < 1e-12
    assert np.abs(v_im - c_im).max() < 1e-12


def test_row_oracle_matches_whole_batch(small12):
    ham, U = small12
    rng = np.random.default_rng(9)
    m = len(U)
    lre = rng.normal(0, 1, size=m)
    lim = np.where(rng.random(m) < 0.5, np.pi, 0.0)
    res = oracle.forward(U, lre, lim, ham)
    ro = oracle.RowOracle(pack_ints(U, 12), ham, lre, lim)
    for i in range(m):
        r = ro.row(i)
        assert r["eloc"] == res["eloc"][i]
        assert sorted(r["j"]) == sorted(j for (a, j) in res["pairs"] if a == i)
    gr = rng.normal(size=m)
    v_re, v_im = oracle.local_energy_vjp(U, lre, lim, ham, res["pairs"], gr, None, 0.4)
    eloc = np.array(res["eloc"])
    for y in range(m):
        a, b = ro.row_vjp(y, eloc, res["e_var"], gr, None, 0.4)
        assert abs(a - v_re[y]) < 1e-12 and abs(b - v_im[y]) < 1e-12


# --------------------------------------------------------------------------
# planted mistakes (in the oracle, on the CPU): the pins above must notice them
# --------------------------------------------------------------------------

def _dense_error(ham, D, n, melem):
    return max(abs(melem(a, b, ham) - D[a, b]) for a in range(1 << n) for b in range(1 << n))


def test_planted_phase_mistakes_are_caught():
    n = 4
    x, z, c = random_pauli_hamiltonian(n, 30, 21, allow_odd_y=True)
    D = pauli_dense(x, z, c, n)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    assert _dense_error(ham, D, n, oracle.matrix_element) < 1e-12

    def phase_on_x(a, b, ham):  # uses x instead of x'
        return oe._csum(t.h * oe._I_POW[(t.Y.bit_count() + 2 * (a & t.YZ).bit_count()) % 4]
                        for t in ham.group(a ^ b))

    def no_i_power(a, b, ham):  # drops the i^|Y| factor
        return oe._csum(t.h * (-1) ** (b & t.YZ).bit_count() for t in ham.group(a ^ b))

    def yz_as_z(a, b, ham):  # uses Z instead of Y OR Z in the phase
        return oe._csum(t.h * oe._I_POW[(t.Y.bit_count() + 2 * (b & t.Z).bit_count()) % 4]
                        for t in ham.group(a ^ b))

    for bad in (phase_on_x, no_i_power, yz_as_z):
        assert _dense_error(ham, D, n, bad) > 1e-3, bad.__name__


def test_planted_energy_mistakes_are_caught(monkeypatch):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_example.json")))
    from synth import from_paper_string
    xs = [sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "XY") for t in gold["terms"]["list"]]
    zs = [sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "YZ") for t in gold["terms"]["list"]]
    hs = [t["h"] for t in gold["terms"]["list"]]
    ham = oracle.prepare_hamiltonian(pack_ints(xs, 4), pack_ints(zs, 4), hs, 4)
    U = [from_paper_string(s) for s in gold["batch"]["U"]]
    psi = np.array(gold["batch"]["psi"])
    lre, lim = np.log(np.abs(psi)), np.where(psi < 0, np.pi, 0.0)
    want = gold["local_energies"]["eloc"]

    def eloc_with(pairs_fn=None):
        pairs = oracle.find_coupled_pairs(U, ham, "terms")
        if pairs_fn:
            pairs = pairs_fn(pairs)
        el, _ = oracle.local_energy_var(U, lre, lim, ham, pairs)
        return [e.real for e in el]

    ok = eloc_with()
    assert np.allclose(ok, want, atol=1e-14)
    # dropped diagonal pairs
    assert not np.allclose(eloc_with(lambda p: [q for q in p if q[0] != q[1]]), want, atol=1e-3)
    # inverted amplitude ratio psi(x)/psi(x')
    orig_exp = cmath.exp
    monkeypatch.setattr(oe.cmath, "exp", lambda v: orig_exp(-v))
    assert not np.allclose(eloc_with(), want, atol=1e-3)
    monkeypatch.undo()
    # |psi| instead of |psi|^2 as weights in E^var
    el = [complex(e) for e in want]
    good = oracle.variational_energy(lre, el).real
    bad = oracle.variational_energy(lre / 2.0, el).real
    assert abs(good - 5.2 / 6.0) < 1e-14 and abs(bad - 5.2 / 6.0) > 1e-3


def test_planted_trie_mistake_is_caught(monkeypatch):
    n = 8
    x, z, c = random_pauli_hamiltonian(n, 40, 31, max_weight=4)
    ham = oracle.prepare_hamiltonian(x, z, c, n)
    U = _random_batch(n, 60, 32)
    ref = sorted(oracle.coupled_pairs_definition(U, ham))
    assert sorted(oracle.find_coupled_pairs(U, ham, "trie")) == ref

    def wrong_child(x, tree_u, tree_xy, n_bits):  # XY child indexed by x'_i instead of x_i ^ x'_i
        frontier = [(tree_u[0], tree_xy[0])]
        for i in range(n_bits):
            nxt = []
            for (un, xyn) in frontier:
                for bit in (0, 1):
                    nu, nxy = un.children[bit], xyn.children[bit]
                    if nu is not None and nxy is not None:
                        nxt.append((nu, nxy))
            frontier = nxt
        return [un.leaf_of for un, _ in frontier], [xyn.leaf_of for _, xyn in frontier]

    monkeypatch.setattr(op, "couple_via_prefix_tree", wrong_child)
    assert sorted(op.find_coupled_pairs(U, ham, "trie")) != ref
