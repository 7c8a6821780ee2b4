"""Hamiltonian arithmetic and preparation (oracle; test infrastructure).

Follows Sec. "Hamiltonian arithmetic" (Eq. pauli_melem), Sec. "Unique XY",
Eq. (xy_to_yz_set) and Sec. "Preparation" (Fig. ham_prep).
"""

import dataclasses
import math

import numpy as np


def _as_int_list(a):
    """uint64 [n, W] array (bit i of word w = qubit 64w+i) or iterable of ints -> ints."""
    if isinstance(a, np.ndarray):
        a = np.asarray(a, dtype=np.uint64)
        if a.ndim == 1:
            a = a[:, None]
        out = []
        for row in a:
            v = 0
            for w in range(a.shape[1] - 1, -1, -1):
                v = (v << 64) | int(row[w])
            out.append(v)
        return out
    return [int(v) for v in a]


@dataclasses.dataclass(frozen=True)
class PauliTerm:
    """One Hamiltonian term (h_l, X^(l), Y^(l), Z^(l)) of Sec. "Hamiltonian arithmetic".

    X, Y and Z are the bit vectors of the positions that carry that Pauli
    operator (mutually exclusive).
    """
    h: float
    X: int
    Y: int
    Z: int

    @property
    def XY(self) -> int:
        """XY^(l) = X^(l) OR Y^(l): the qubits the term flips."""
        return self.X | self.Y

    @property
    def YZ(self) -> int:
        """YZ^(l) = Y^(l) OR Z^(l): the qubits whose value enters the phase."""
        return self.Y | self.Z


# i**a for a = 0..3, exact
_I_POW = (complex(1, 0), complex(0, 1), complex(-1, 0), complex(0, -1))


def pauli_matrix_element(x: int, xp: int, term: PauliTerm) -> complex:
    """<x| P^(l) |x'> by Eq. (pauli_melem).

    Zero unless x XOR x' equals XY^(l); otherwise exp(i phi) with
    phi = (pi/2)|Y^(l)| + pi |x' AND YZ^(l)|.  Since phi is an integer
    multiple of pi/2, exp(i phi) = i^(|Y| + 2|x' & YZ|) exactly.
    """
    if (x ^ xp) != term.XY:
        return complex(0.0, 0.0)
    a = term.Y.bit_count() + 2 * (xp & term.YZ).bit_count()
    return _I_POW[a % 4]


@dataclasses.dataclass
class PreparedHamiltonian:
    """The tensors of Fig. (ham_prep).

    ``terms`` are grouped by XY in the order of ``xy_list`` (unique XY in
    order of first appearance, as in the toy example); ``starts[m]`` and
    ``nums[m]`` locate the set P_{XY_m} inside ``terms``.
    """
    n_qubits: int
    terms: list
    xy_list: list
    starts: list
    nums: list
    xy_index: dict

    def group(self, xy: int):
        """The set P_XY of Eq. (xy_to_yz_set) as a list of terms (empty if XY is absent)."""
        m = self.xy_index.get(xy)
        if m is None:
            return []
        return self.terms[self.starts[m]: self.starts[m] + self.nums[m]]


def prepare_hamiltonian(x_mask, z_mask, coef, n_qubits: int) -> PreparedHamiltonian:
    """Build the grouped representation from symplectic Pauli strings.

    Input encoding: qubit i carries X if (x_i, z_i) = (1, 0), Y if (1, 1) and
    Z if (0, 1).  Reading of the paper (its Hamiltonian has distinct terms):
    identical strings are one term whose coefficient is the (correctly
    rounded) sum, and a term whose coefficient is exactly zero is not a term
    of H, so it contributes no XY pattern.
    """
    xs = _as_int_list(x_mask)
    zs = _as_int_list(z_mask)
    cs = [float(c) for c in np.asarray(coef, dtype=np.float64).ravel()]
    if not (len(xs) == len(zs) == len(cs)):
        raise ValueError("mask and coefficient lengths differ")
    limit = 1 << int(n_qubits)
    acc = {}
    order = []
    for x, z, c in zip(xs, zs, cs):
        if x >= limit or z >= limit:
            raise ValueError("Pauli mask has bits beyond n_qubits")
        key = (x, z)
        if key not in acc:
            acc[key] = []
            order.append(key)
        acc[key].append(c)
    raw_terms = []
    for (x, z) in order:
        h = math.fsum(acc[(x, z)])
        if h == 0.0:
            continue
        raw_terms.append(PauliTerm(h=h, X=x & ~z, Y=x & z, Z=z & ~x))

    xy_list, groups = [], {}
    for t in raw_terms:
        if t.XY not in groups:
            groups[t.XY] = []
            xy_list.append(t.XY)
        groups[t.XY].append(t)
    terms, starts, nums = [], [], []
    for xy in xy_list:
        starts.append(len(terms))
        nums.append(len(groups[xy]))
        terms.extend(groups[xy])
    xy_index = {xy: m for m, xy in enumerate(xy_list)}
    return PreparedHamiltonian(int(n_qubits), terms, xy_list, starts, nums, xy_index)
