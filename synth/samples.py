"""Peaked batches of unique sampled determinants.

The paper's wave functions are peaked around the Hartree-Fock determinant
(Sec. "Autoregressive neural quantum states"); its batches hold N_unq unique
determinants drawn without replacement (Sec. "Sampling without replacement").
A sampler and a trained ansatz are outside the hot path, so a batch is drawn
here from a fixed rule instead:

* excitation rank k (number of electrons moved out of the Hartree-Fock
  orbitals) carries weight 0.1^k, k <= k_max;
* quotas are assigned from rank 0 upwards: n_k = min(count_k,
  round(rem * w_k / sum_{j=k..k_max} w_j)) with rem the samples still to
  place, so that ranks that are too small are filled completely and the
  remainder moves up;
* within a rank, determinants are uniform without replacement over the fixed
  (N_e, S_z) sector;
* the batch is returned in a seeded random order.
"""

import itertools
import math

import numpy as np

from .bits import pack_ints


def _rank_count(n_orb, n_a, n_b, ka, kb):
    va, vb = n_orb - n_a, n_orb - n_b
    return math.comb(n_a, ka) * math.comb(va, ka) * math.comb(n_b, kb) * math.comb(vb, kb)


def _rank_splits(n_orb, n_a, n_b, k):
    out = []
    for ka in range(0, k + 1):
        kb = k - ka
        c = _rank_count(n_orb, n_a, n_b, ka, kb)
        if c > 0:
            out.append((ka, kb, c))
    return out


def rank_quotas(n_orb, n_a, n_b, n_unq, k_max=6, decay=0.1):
    """Per-rank sample counts following the rule in the module docstring."""
    counts = [sum(c for _, _, c in _rank_splits(n_orb, n_a, n_b, k)) for k in range(k_max + 1)]
    w = [decay ** k for k in range(k_max + 1)]
    rem = int(n_unq)
    quotas = []
    for k in range(k_max + 1):
        share = w[k] / sum(w[k:])
        nk = min(counts[k], int(round(rem * share)))
        quotas.append(nk)
        rem -= nk
    if rem > 0:
        raise ValueError("sector too small for the requested number of unique samples")
    return quotas, counts


def _det_int(occ_a, occ_b):
    v = 0
    for p in occ_a:
        v |= 1 << (2 * int(p))
    for p in occ_b:
        v |= 1 << (2 * int(p) + 1)
    return v


def _excite(hf_a, vir_a, hf_b, vir_b, ra, aa, rb, ab):
    occ_a = (set(hf_a) - set(ra)) | set(aa)
    occ_b = (set(hf_b) - set(rb)) | set(ab)
    return _det_int(occ_a, occ_b)


def excitation_rank(v: int, n_a: int, n_b: int) -> int:
    """Number of electrons outside the Hartree-Fock orbitals of determinant v."""
    hf = _det_int(range(n_a), range(n_b))
    return bin(v & ~hf).count("1")


def peaked_samples(n_orb: int, n_a: int, n_b: int, n_unq: int, seed: int,
                   k_max: int = 6, decay: float = 0.1):
    """Unique determinants around Hartree-Fock.

    Returns (values: list of Python ints, ranks: int64 array), both in the
    same seeded random order.
    """
    rng = np.random.default_rng(seed)
    quotas, counts = rank_quotas(n_orb, n_a, n_b, n_unq, k_max, decay)
    hf_a, hf_b = list(range(n_a)), list(range(n_b))
    vir_a, vir_b = list(range(n_a, n_orb)), list(range(n_b, n_orb))
    values, ranks = [], []
    for k, nk in enumerate(quotas):
        if nk == 0:
            continue
        splits = _rank_splits(n_orb, n_a, n_b, k)
        chosen = []
        if nk == counts[k]:
            for ka, kb, _ in splits:
                for ra in itertools.combinations(hf_a, ka):
                    for aa in itertools.combinations(vir_a, ka):
                        for rb in itertools.combinations(hf_b, kb):
                            for ab in itertools.combinations(vir_b, kb):
                                chosen.append(_excite(hf_a, vir_a, hf_b, vir_b, ra, aa, rb, ab))
        else:
            probs = np.array([c for _, _, c in splits], dtype=float)
            probs /= probs.sum()
            seen = set()
            while len(chosen) < nk:
                ka, kb, _ = splits[rng.choice(len(splits), p=probs)]
                ra = rng.choice(n_a, size=ka, replace=False) if ka else []
                aa = rng.choice(vir_a, size=ka, replace=False) if ka else []
                rb = rng.choice(n_b, size=kb, replace=False) if kb else []
                ab = rng.choice(vir_b, size=kb, replace=False) if kb else []
                v = _excite(hf_a, vir_a, hf_b, vir_b, list(ra), list(aa), list(rb), list(ab))
                if v not in seen:
                    seen.add(v)
                    chosen.append(v)
        values.extend(chosen)
        ranks.extend([k] * len(chosen))
    perm = rng.permutation(len(values))
    values = [values[i] for i in perm]
    ranks = np.asarray(ranks, dtype=np.int64)[perm]
    return values, ranks


def all_sector_determinants(n_orb: int, n_a: int, n_b: int):
    """Every determinant with n_a alpha and n_b beta electrons (sorted ints)."""
    out = []
    for occ_a in itertools.combinations(range(n_orb), n_a):
        for occ_b in itertools.combinations(range(n_orb), n_b):
            out.append(_det_int(occ_a, occ_b))
    return sorted(out)


def pack_samples(values, n_qubits):
    return pack_ints(values, n_qubits)
