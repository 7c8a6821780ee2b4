"""CPU FP64 oracle for the sampled-space local energy (test infrastructure).

This package is the slow, plain reference that the CUDA library is checked
against.  It is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path
(``paper_2408_07625_gb300``) never imports, calls or falls back to it, and it
shares no code with that path; both read inputs from the separate ``synth``
generator only.

Representation: every N-bit vector is a Python int with bit i = qubit i, so
no word splitting is involved; floating point is Python float (IEEE FP64)
and complex; sums use ``math.fsum`` (correctly rounded) on real and imaginary
parts separately.

Modules and the passages they follow:

* ``hamiltonian`` -- Hamiltonian arithmetic, Sec. "Hamiltonian arithmetic"
  (Eq. pauli_melem), the unique-XY sets P_XY (Eq. xy_to_yz_set) and the
  grouped storage of Sec. "Preparation" (Fig. ham_prep).
* ``pairs`` -- FindCoupledPairs: the definition, LoopOverTerms (Alg. 2A),
  LoopOverBatch (Alg. 2B), the prefix tree (Alg. 3) and LoopOverTrie
  (Alg. 2C).
* ``energy`` -- MatrixElement (supplementary algorithm "Calculating the
  Hamiltonian matrix element"), the surrogate local energy (Eq. local_energy
  restricted to U), the variational energy (Eq. variational_energy) and its
  derivatives with respect to log psi.
* ``rows`` -- the same quantities for a chosen subset of rows of a large
  batch (LoopOverTerms per row), used for sampled checks at full size.
* ``sampling`` -- autoregressive sampling without replacement, Alg. 1
  (ARGumbelTopK), with the random numbers passed in.
* ``sr`` -- the quantum geometric tensor of Eq. (qgt_definition) on the most
  probable samples and the regularised (min-SR) step.
* ``candidates`` -- the exact local energy of Eq. (local_energy): the
  coupled candidates x XOR XY of every sample (inside or outside U),
  deduplicated over the batch, and the sum over them.

Every function has at least one pin in ``tests/test_oracle_*.py`` that does
not reuse the oracle's own formula (paper's worked example, dense Kronecker
matrices, exact diagonalisation, Slater-Condon energies, brute force,
finite differences).
"""

from .hamiltonian import (PauliTerm, PreparedHamiltonian, prepare_hamiltonian,
                          pauli_matrix_element)
from .pairs import (coupled_pairs_definition, couple_via_unique_xy, couple_all_to_all,
                    construct_prefix_tree, couple_via_prefix_tree, find_coupled_pairs,
                    find_a_in_b_pointers, prefix_tree_levels)
from .energy import (matrix_element, matrix_element_all_terms, local_energy_var,
                     variational_energy, energy_gradient_closed_form,
                     local_energy_vjp, forward)
from .rows import RowOracle
from .candidates import full_candidates, local_energy_full
from .sampling import ar_gumbel_topk
from .sr import top_probable, sr_weights, qgt, centred, sample_gram, min_sr_step

__all__ = [
    "PauliTerm", "PreparedHamiltonian", "prepare_hamiltonian", "pauli_matrix_element",
    "coupled_pairs_definition", "couple_via_unique_xy", "couple_all_to_all",
    "construct_prefix_tree", "couple_via_prefix_tree", "find_coupled_pairs",
    "find_a_in_b_pointers", "prefix_tree_levels",
    "matrix_element", "matrix_element_all_terms", "local_energy_var", "variational_energy",
    "energy_gradient_closed_form", "local_energy_vjp", "forward", "RowOracle",
    "full_candidates", "local_energy_full", "ar_gumbel_topk",
    "top_probable", "sr_weights", "qgt", "centred", "sample_gram", "min_sr_step",
]
