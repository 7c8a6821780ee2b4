"""Full local energy: coupled candidates outside the batch (oracle; test infrastructure).

The exact local energy of Eq. (local_energy) sums over every x' with
H_xx' != 0, not only over the sampled batch U (the surrogate E_loc^var of
Sec. "Streamlined local energy calculations" keeps only x' in U).  Term l
of the Hamiltonian couples x to x' exactly when x XOR x' = XY^(l)
(Eq. pauli_melem), so the x' that can have H_xx' != 0 are the candidates
x XOR XY for the unique XY patterns of the Hamiltonian (Sec. "Unique XY");
evaluating the ansatz on them is the O(N_unq N_T) cost the paper's
surrogate avoids.

Reading (stated in the design notes): a candidate is generated for every
unique XY pattern, whether or not its matrix element cancels to zero for
that x (the same combinatorial notion of "coupled" as the pair lists); a
zero matrix element adds nothing to the sum.  The candidates of the whole
batch are deduplicated, and the unique set is listed in increasing numeric
order of the bit vectors (qubit 0 the least significant bit).

Bit vectors are Python ints (bit i = qubit i); sums use ``math.fsum``.
"""

import cmath
import math

import numpy as np

from .hamiltonian import PreparedHamiltonian, _as_int_list
from .energy import matrix_element, _csum, _logpsi


def full_candidates(U, ham: PreparedHamiltonian):
    """Candidates of every x in U: x XOR XY for each unique XY pattern.

    Returns (rows, C): rows[i] is the list of (x', XY, H_xx') for sample i in
    the order of ``ham.xy_list``, H by MatrixElement (supplementary
    algorithm); C is the sorted list of the distinct x' over the whole batch.
    """
    U = _as_int_list(U)
    rows = []
    seen = set()
    for x in U:
        r = []
        for xy in ham.xy_list:
            xp = x ^ xy
            r.append((xp, xy, matrix_element(x, xp, ham)))
            seen.add(xp)
        rows.append(r)
    return rows, sorted(seen)


def local_energy_full(U, logpsi_re, logpsi_im, ham: PreparedHamiltonian, C, logpsi_c_re, logpsi_c_im=None):
    """E_loc(x) = sum over x' coupled to x of H_xx' psi(x') / psi(x) (Eq. local_energy).

    psi(x) = exp(l(x)) for x in U (``logpsi_*``) and for every candidate in
    C (``logpsi_c_*``, same order as C).  Returns a list of complex values.
    """
    U = _as_int_list(U)
    l_u = _logpsi(logpsi_re, logpsi_im, len(U))
    l_c = _logpsi(logpsi_c_re, logpsi_c_im, len(C))
    lc = {x: l for x, l in zip(C, l_c)}
    out = []
    for x, lx in zip(U, l_u):
        terms = []
        for xy in ham.xy_list:
            xp = x ^ xy
            h = matrix_element(x, xp, ham)
            terms.append(h * cmath.exp(lc[xp] - lx))
        out.append(_csum(terms))
    return out
