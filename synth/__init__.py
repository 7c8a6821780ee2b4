"""Seeded synthetic inputs for the sampled-space local-energy path.

This package produces the *inputs* of the method and nothing else: qubit
Hamiltonians obtained from synthetic molecular integrals through the
Jordan-Wigner mapping (the paper obtains them from OpenFermion, Sec. "General
setup"), peaked batches of unique sampled determinants, and log-amplitudes.
It holds none of the method's own arithmetic (no pair search, matrix element,
local energy or energy reduction), so that both the CPU oracle and the CUDA
library can consume the same instances without sharing code.

Bit layout of every N-bit vector: qubit i is bit (i % 64) of 64-bit word
(i // 64); a batch is a ``uint64`` array of shape ``[n, W]`` with
``W = ceil(N / 64)``.  The paper prints bit strings with x_0 first; the
helpers ``from_paper_string``/``to_paper_string`` convert.
"""

from .bits import (n_words, pack_ints, unpack_ints, from_paper_string,
                   to_paper_string, popcount_rows)
from .molecular import (molecular_integrals, jordan_wigner, hf_energy_from_integrals,
                        pauli_to_xyz)
from .samples import (peaked_samples, all_sector_determinants, rank_quotas,
                      excitation_rank)
from .instances import (Instance, config_instance, CONFIGS, batched_instances,
                        random_pauli_hamiltonian)
from .ansatz import ToyAutoregressive, gumbel_noise

__all__ = [
    "n_words", "pack_ints", "unpack_ints", "from_paper_string", "to_paper_string",
    "popcount_rows", "molecular_integrals", "jordan_wigner", "hf_energy_from_integrals",
    "pauli_to_xyz", "peaked_samples", "all_sector_determinants", "rank_quotas",
    "excitation_rank", "Instance", "config_instance", "CONFIGS", "batched_instances",
    "random_pauli_hamiltonian", "ToyAutoregressive", "gumbel_noise",
]
