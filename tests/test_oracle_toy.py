"""Oracle pinned to the paper's worked toy example (values in tests/golden)."""

import json
import os

import numpy as np
import pytest

import oracle
from synth import from_paper_string, pack_ints

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_example.json")))
N = GOLD["n_qubits"]


def paper_dec(s):
    """The paper's decimal value of a bit string (x_0 most significant)."""
    return int(s, 2)


def toy_pauli():
    """Symplectic (x, z) masks of the toy terms from their Pauli letters."""
    xs, zs, hs = [], [], []
    for t in GOLD["terms"]["list"]:
        x = sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "XY")
        z = sum(1 << i for i, ch in enumerate(t["pauli"]) if ch in "YZ")
        xs.append(x), zs.append(z), hs.append(t["h"])
    return pack_ints(xs, N), pack_ints(zs, N), np.array(hs)


@pytest.fixture(scope="module")
def ham():
    x, z, h = toy_pauli()
    return oracle.prepare_hamiltonian(x, z, h, N)


@pytest.fixture(scope="module")
def batch():
    U = [from_paper_string(s) for s in GOLD["batch"]["U"]]
    psi = np.array(GOLD["batch"]["psi"])
    lre = np.log(np.abs(psi))
    lim = np.where(psi < 0, np.pi, 0.0)
    return U, lre, lim


def test_bit_order_convention():
    for s, d in zip(GOLD["batch"]["U"], GOLD["batch"]["U_dec"]):
        assert paper_dec(s) == d
    for row in GOLD["table"]["rows"]:
        assert paper_dec(row["XY"]) == row["XY_dec"]


def test_table_y_xy_yz(ham):
    # terms keep input order inside each XY group; map back by coefficient+pattern
    by_l = {}
    for row in GOLD["table"]["rows"]:
        by_l[row["l"]] = row
    x, z, h = toy_pauli()
    for l, t in enumerate(GOLD["terms"]["list"]):
        term = oracle.PauliTerm(h=t["h"], X=0, Y=0, Z=0)
        xi = int(x[l, 0]); zi = int(z[l, 0])
        term = oracle.PauliTerm(h=t["h"], X=xi & ~zi, Y=xi & zi, Z=zi & ~xi)
        row = by_l[l]
        assert term.Y == from_paper_string(row["Y"])
        assert term.XY == from_paper_string(row["XY"])
        assert term.YZ == from_paper_string(row["YZ"])


def test_unique_xy_and_groups(ham):
    assert ham.xy_list == [from_paper_string(s) for s in GOLD["unique_xy"]["strings"]]
    hs = [t["h"] for t in GOLD["terms"]["list"]]
    for m, members in enumerate(GOLD["unique_xy"]["P_XY"]):
        assert ham.nums[m] == len(members)
        got = [t.h for t in ham.terms[ham.starts[m]: ham.starts[m] + ham.nums[m]]]
        assert got == [hs[l] for l in members]


def test_xor_table(batch):
    U, _, _ = batch
    for i, row in enumerate(GOLD["xor_table_dec"]["rows"]):
        for j, d in enumerate(row):
            from synth import to_paper_string
            assert paper_dec(to_paper_string(U[i] ^ U[j], N)) == d


@pytest.mark.parametrize("method", ["definition", "terms", "batch", "trie"])
def test_coupled_sets(ham, batch, method):
    U, _, _ = batch
    if method == "definition":
        pairs = oracle.coupled_pairs_definition(U, ham)
    else:
        pairs = oracle.find_coupled_pairs(U, ham, method)
    rows = [sorted(j for (i, j) in pairs if i == r) for r in range(len(U))]
    assert rows == [sorted(r) for r in GOLD["coupled_sets"]["rows"]]


def test_matrix_elements(ham, batch):
    U, _, _ = batch
    for e in GOLD["matrix_elements"]["entries"]:
        h = oracle.matrix_element(U[e["i"]], U[e["j"]], ham)
        assert h.imag == 0.0
        assert h.real == pytest.approx(e["H"], abs=1e-15)
        h2 = oracle.matrix_element_all_terms(U[e["i"]], U[e["j"]], ham)
        assert h2 == pytest.approx(h, abs=1e-15)


def test_local_energies(ham, batch):
    U, lre, lim = batch
    res = oracle.forward(U, lre, lim, ham)
    for got, want in zip(res["eloc"], GOLD["local_energies"]["eloc"]):
        assert got.real == pytest.approx(want, abs=1e-14)
        assert abs(got.imag) < 1e-15


def test_variational_energy(ham, batch):
    U, lre, lim = batch
    res = oracle.forward(U, lre, lim, ham)
    psi = GOLD["batch"]["psi"]
    el = GOLD["local_energies"]["eloc"]
    # Eq. (variational_energy) evaluated by hand on the printed values
    want = sum(p * p * e for p, e in zip(psi, el)) / sum(p * p for p in psi)
    assert res["e_var"].real == pytest.approx(want, abs=1e-14)
    assert want == pytest.approx(5.2 / 6.0, abs=1e-15)


def test_find_a_in_b_example(ham, batch):
    U, _, _ = batch
    A = [U[i] ^ U[j] for i in range(3) for j in range(3)]  # row-major candidates XY?
    B = ham.xy_list
    mask, ptr = oracle.find_a_in_b_pointers(A, B)
    g = GOLD["find_a_in_b"]
    assert paper_dec(__import__("synth").to_paper_string(A[g["member_index"]], N)) == g["member_dec"]
    assert mask[g["member_index"]] is True
    assert mask[g["non_member_index"]] is False
    # the member at candidate index 1 is the second member overall
    assert ptr[sum(mask[: g["member_index"]])] == g["member_pointer"]
    # the coupled-pair pointer array of the paper's figures, row-major
    assert ptr == [0, 2, 1, 2, 0, 1, 0]


def test_prefix_tree_figure_node_counts():
    vals = [from_paper_string(s) for s in GOLD["prefix_tree_figure"]["set"]]
    tree = oracle.construct_prefix_tree(vals, 6)
    depth = {id(tree[0]): 0}
    counts = [0] * 7
    counts[0] = 1
    stack = [tree[0]]
    while stack:
        node = stack.pop()
        for ch in node.children:
            if ch is not None:
                depth[id(ch)] = depth[id(node)] + 1
                counts[depth[id(ch)]] += 1
                stack.append(ch)
    assert counts == [1, 2, 3, 4, 5, 5, 5]
    assert len(tree) == sum(counts)
    levels = oracle.prefix_tree_levels(vals, 6)
    assert [len(lv["up"]) for lv in levels] == counts
    # 110110 and 111001 share their first two levels, not the third
    a, b = vals[2], vals[3]
    assert levels[2]["to_node"][2] == levels[2]["to_node"][3]
    assert levels[3]["to_node"][2] != levels[3]["to_node"][3]


def test_prefix_tree_levels_toy(batch):
    U, _, _ = batch
    levels = oracle.prefix_tree_levels(U, N)
    g = GOLD["prefix_tree_levels"]
    assert levels[2]["to_node"][0] == g["to_node_level2_of_x0"]
    assert levels[2]["up"][2] == (g["level2_node2_value"], g["level2_node2_parent"])
    assert levels[2]["down"][0] == (g["level2_node0_child0"], g["level2_node0_child1"])
    assert all(lv == 0 for lv in levels[0]["to_node"])
    # every leaf maps back to its vector
    tree = oracle.construct_prefix_tree(U, N)
    leaves = sorted(n.leaf_of for n in tree if n.leaf_of is not None)
    assert leaves == [0, 1, 2]
