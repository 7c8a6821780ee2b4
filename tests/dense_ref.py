"""Independent dense references for pinning the oracle (tests only).

* ``pauli_dense``: the Hamiltonian matrix built from 2x2 Pauli matrices with
  Kronecker products (no bit arithmetic), basis index = sum_i x_i 2^i.
* ``fermion_dense``: the second-quantised Hamiltonian of Eq. (fermionic_qc)
  applied directly to occupation-number states, with the fermionic sign
  (-1)^(number of occupied modes below the acted-on mode); no Pauli algebra.
"""

import numpy as np
import scipy.sparse as sp

_I = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)


def _to_int(row):
    row = np.atleast_1d(np.asarray(row, dtype=np.uint64))
    v = 0
    for w in range(row.shape[0] - 1, -1, -1):
        v = (v << 64) | int(row[w])
    return v


def pauli_string_matrix(x, z, n):
    """Sparse matrix of one Pauli string (qubit 0 = least significant index bit)."""
    m = sp.identity(1, dtype=complex, format="csr")
    for q in range(n - 1, -1, -1):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        P = _I if (xb, zb) == (0, 0) else _X if (xb, zb) == (1, 0) else _Y if (xb, zb) == (1, 1) else _Z
        m = sp.kron(m, sp.csr_matrix(P), format="csr")
    return m


def pauli_dense(x_mask, z_mask, coef, n, dense=True):
    H = sp.csr_matrix((1 << n, 1 << n), dtype=complex)
    for xr, zr, c in zip(x_mask, z_mask, coef):
        H = H + float(c) * pauli_string_matrix(_to_int(xr), _to_int(zr), n)
    return H.toarray() if dense else H


def _annihilate(state, mode):
    if not (state >> mode) & 1:
        return None, 0
    sign = -1 if bin(state & ((1 << mode) - 1)).count("1") % 2 else 1
    return state ^ (1 << mode), sign


def _create(state, mode):
    if (state >> mode) & 1:
        return None, 0
    sign = -1 if bin(state & ((1 << mode) - 1)).count("1") % 2 else 1
    return state | (1 << mode), sign


def _apply(ops, state):
    """Apply a product of ladder operators (rightmost first) to a basis state."""
    sign = 1
    for (kind, mode) in reversed(ops):
        state, s = (_create if kind == "+" else _annihilate)(state, mode)
        if state is None:
            return None, 0
        sign *= s
    return state, sign


def fermion_dense(h1, eri, n_orb):
    """H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs, interleaved spins."""
    N = 2 * n_orb
    dim = 1 << N
    H = np.zeros((dim, dim))
    for st in range(dim):
        for p in range(n_orb):
            for q in range(n_orb):
                if h1[p, q] == 0:
                    continue
                for s in (0, 1):
                    out, sg = _apply([("+", 2 * p + s), ("-", 2 * q + s)], st)
                    if out is not None:
                        H[out, st] += h1[p, q] * sg
        for p in range(n_orb):
            for q in range(n_orb):
                for r in range(n_orb):
                    for s_ in range(n_orb):
                        v = eri[p, q, r, s_]
                        if v == 0:
                            continue
                        for s in (0, 1):
                            for t in (0, 1):
                                out, sg = _apply([("+", 2 * p + s), ("+", 2 * r + t),
                                                  ("-", 2 * s_ + t), ("-", 2 * q + s)], st)
                                if out is not None:
                                    H[out, st] += 0.5 * v * sg
    return H


def sector_indices(n_orb, n_a, n_b):
    """Basis indices with n_a electrons on even qubits and n_b on odd qubits."""
    out = []
    for st in range(1 << (2 * n_orb)):
        a = bin(st & int("01" * n_orb, 2)).count("1")
        b = bin(st & int("10" * n_orb, 2)).count("1")
        if a == n_a and b == n_b:
            out.append(st)
    return np.array(out, dtype=np.int64)
