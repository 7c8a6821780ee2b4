"""FindCoupledPairs (oracle; test infrastructure).

All functions return, for a sample x of the unique batch U, the indices j of
the samples x' = U[j] with x XOR x' in the set of unique XY patterns (the set
SC_x of Sec. "Unique XY").  Bit vectors are Python ints, bit i = qubit i =
the paper's x_i.
"""

import numpy as np

from .hamiltonian import PreparedHamiltonian, _as_int_list


# --------------------------------------------------------------------------
# definition
# --------------------------------------------------------------------------

def coupled_pairs_definition(U, ham: PreparedHamiltonian):
    """All ordered (i, j) with U_i XOR U_j = XY^(l) for some term l.

    Straight from Eq. (pauli_melem): term l couples x to x' exactly when
    x XOR x' = XY^(l).  Loops over every term (not the unique set); the
    diagonal (i, i) is included when a term has XY = 0.  Cost O(N_unq^2 N_T).
    """
    U = _as_int_list(U)
    xy_terms = [t.XY for t in ham.terms]
    out = []
    if ham.n_qubits <= 64 and xy_terms:
        arr = np.array(xy_terms, dtype=np.uint64)
        for i, x in enumerate(U):
            for j, xp in enumerate(U):
                if np.any(arr == np.uint64(x ^ xp)):
                    out.append((i, j))
    else:
        for i, x in enumerate(U):
            for j, xp in enumerate(U):
                if any((x ^ xp) == xy for xy in xy_terms):
                    out.append((i, j))
    return out


# --------------------------------------------------------------------------
# Alg. 2A: loop over unique XY
# --------------------------------------------------------------------------

def couple_via_unique_xy(x: int, u_index: dict, xy_list):
    """Alg. 2A (LoopOverTerms): for XY in the unique set, x' = x XOR XY, keep x' if in U.

    ``u_index`` maps each sample of U to its position (the membership test).
    Returns the positions j in the order of ``xy_list``.
    """
    sc = []
    for xy in xy_list:
        xp = x ^ xy
        j = u_index.get(xp)
        if j is not None:
            sc.append(j)
    return sc


# --------------------------------------------------------------------------
# Alg. 2B: loop over the batch
# --------------------------------------------------------------------------

def couple_all_to_all(x: int, U, xy_set):
    """Alg. 2B (LoopOverBatch): for x' in U, keep x' if x XOR x' is a unique XY."""
    sc = []
    for j, xp in enumerate(U):
        if (x ^ xp) in xy_set:
            sc.append(j)
    return sc


def find_a_in_b_pointers(A, B):
    """FindAInB semantics (Sec. "FindAInB implementation"): the mask ``A in B``
    and, for the members of A in their original order, their positions in B
    (B holds no repeats)."""
    pos = {b: k for k, b in enumerate(B)}
    mask = [a in pos for a in A]
    ptr = [pos[a] for a in A if a in pos]
    return mask, ptr


# --------------------------------------------------------------------------
# Alg. 3: prefix tree; Alg. 2C: loop over the tree
# --------------------------------------------------------------------------

class _Node:
    __slots__ = ("value", "parent", "children", "leaf_of")

    def __init__(self, value, parent):
        self.value = value
        self.parent = parent
        self.children = [None, None]
        self.leaf_of = None


def construct_prefix_tree(values, n_bits: int):
    """Alg. 3 (ConstructPrefixTree): insert every vector bit by bit x_0..x_{N-1}.

    Returns the node list; node 0 is the root (value None).  Each leaf also
    records the position of the vector that ends there, which is how the
    coupled vectors are read back at the end of Alg. 2C.
    """
    tree = [_Node(None, None)]
    for pos, x in enumerate(values):
        cur = tree[0]
        for i in range(n_bits):
            b = (x >> i) & 1
            if cur.children[b] is None:
                node = _Node(b, cur)
                cur.children[b] = node
                tree.append(node)
            cur = cur.children[b]
        cur.leaf_of = pos
    return tree


def couple_via_prefix_tree(x: int, tree_u, tree_xy, n_bits: int):
    """Alg. 2C (LoopOverTrie) for one x.

    Keeps the list of pairs (node of T^U, node of T^XY) whose prefixes x'_{<i}
    and XY_{<i} = x_{<i} XOR x'_{<i} both exist; at level i each pair is
    extended by the two possible bits x'_i, the XY node moving to its child
    x_i XOR x'_i.  Returns (positions j of x' in U, positions m of XY in the
    unique set), in the order the leaves come out.
    """
    frontier = [(tree_u[0], tree_xy[0])]
    for i in range(n_bits):
        xi = (x >> i) & 1
        nxt = []
        for (un, xyn) in frontier:
            for bit in (0, 1):
                nu = un.children[bit]
                nxy = xyn.children[xi ^ bit]
                if nu is not None and nxy is not None:
                    nxt.append((nu, nxy))
        frontier = nxt
    return [un.leaf_of for un, _ in frontier], [xyn.leaf_of for _, xyn in frontier]


def prefix_tree_levels(values, n_bits: int):
    """Per-level arrays of the GPU trie layout (Sec. "Prefix tree data structures").

    Nodes of level i are the distinct prefixes of length i, numbered in
    lexicographic order of the prefix read x_0 first (the reading that
    reproduces the paper's worked values).  Returns a list over levels of
    dicts with ``to_node`` (T_->i: node of each vector), ``up`` (T_i-up:
    (value, parent) per node, None at the root) and ``down`` (T_i-down:
    (child0, child1) per node, None when absent).
    """
    vals = list(values)

    def prefix_key(v, i):
        return tuple((v >> b) & 1 for b in range(i))

    levels = []
    for i in range(n_bits + 1):
        keys = sorted({prefix_key(v, i) for v in vals})
        index = {k: n for n, k in enumerate(keys)}
        to_node = [index[prefix_key(v, i)] for v in vals]
        if i == 0:
            up = [(None, None)]
        else:
            prev = levels[i - 1]["index"]
            up = [(k[-1], prev[k[:-1]]) for k in keys]
        levels.append({"index": index, "to_node": to_node, "up": up})
    for i in range(n_bits + 1):
        n_nodes = len(levels[i]["up"])
        down = [[None, None] for _ in range(n_nodes)]
        if i < n_bits:
            for node, (val, parent) in enumerate(levels[i + 1]["up"]):
                down[parent][val] = node
        levels[i]["down"] = [tuple(d) for d in down]
    return levels


# --------------------------------------------------------------------------
# driver over the whole batch
# --------------------------------------------------------------------------

def find_coupled_pairs(U, ham: PreparedHamiltonian, method: str = "terms"):
    """All coupled ordered pairs (i, j) of the batch, row by row.

    method: "terms" (Alg. 2A), "batch" (Alg. 2B) or "trie" (Alg. 2C).
    The pairs of row i appear contiguously, rows in increasing i; inside a
    row the order is the algorithm's own.
    """
    U = _as_int_list(U)
    out = []
    if method == "terms":
        u_index = {x: j for j, x in enumerate(U)}
        if len(u_index) != len(U):
            raise ValueError("U holds repeated samples")
        for i, x in enumerate(U):
            out.extend((i, j) for j in couple_via_unique_xy(x, u_index, ham.xy_list))
    elif method == "batch":
        xy_set = set(ham.xy_list)
        for i, x in enumerate(U):
            out.extend((i, j) for j in couple_all_to_all(x, U, xy_set))
    elif method == "trie":
        n = ham.n_qubits
        tree_u = construct_prefix_tree(U, n)
        tree_xy = construct_prefix_tree(ham.xy_list, n)
        for i, x in enumerate(U):
            js, _ = couple_via_prefix_tree(x, tree_u, tree_xy, n)
            out.extend((i, j) for j in js)
    else:
        raise ValueError(f"unknown method {method!r}")
    return out
