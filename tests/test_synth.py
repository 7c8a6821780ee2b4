"""The seeded input generator: determinism, sectors, quotas, term counts."""

import numpy as np
import pytest

from synth import (config_instance, rank_quotas, excitation_rank, unpack_ints, pack_ints,
                   popcount_rows, from_paper_string, to_paper_string, n_words)


def test_pack_roundtrip_multiword():
    vals = [0, 1, (1 << 63), (1 << 64) | 5, (1 << 83) | (1 << 70) | 3]
    arr = pack_ints(vals, 84)
    assert arr.shape == (5, 2)
    assert unpack_ints(arr) == vals
    assert list(popcount_rows(arr)) == [bin(v).count("1") for v in vals]
    assert n_words(64) == 1 and n_words(65) == 2
    assert to_paper_string(from_paper_string("0110"), 4) == "0110"
    with pytest.raises(ValueError):
        pack_ints([1 << 12], 12)


def test_quota_rule_matches_configured_batches():
    q, c = rank_quotas(28, 7, 7, 100_000)
    assert q == [1, 294, 30429, 62355, 6235, 624, 62] and sum(q) == 100_000
    q, c = rank_quotas(14, 5, 5, 10_000)
    assert q == [1, 90, 2745, 6448, 645, 65, 6]
    q, c = rank_quotas(42, 10, 10, 200_000)
    assert q[:3] == [1, 640, 147040] and sum(q) == 200_000


def test_peaked_batch_28q():
    inst = config_instance("h28", n_unq=2000, use_cache=False)
    vals = unpack_ints(inst.U)
    assert len(set(vals)) == len(vals) == 2000
    even = int("01" * 14, 2)
    for v in vals:
        assert bin(v & even).count("1") == 5 and bin(v & ~even).count("1") == 5
    ranks = [excitation_rank(v, 5, 5) for v in vals]
    assert ranks == list(inst.ranks)
    q, _ = rank_quotas(14, 5, 5, 2000)
    assert np.bincount(inst.ranks, minlength=7).tolist() == q
    # log psi = -2k + N(0, 0.3)
    resid = inst.logpsi_re + 2.0 * inst.ranks
    assert abs(resid.mean()) < 0.05 and 0.25 < resid.std() < 0.35
    again = config_instance("h28", n_unq=2000, use_cache=False)
    assert np.array_equal(again.U, inst.U) and np.array_equal(again.coef, inst.coef)


def test_term_counts_track_the_configs():
    inst = config_instance("h28", n_unq=100, use_cache=False)
    assert 1.2e4 < inst.n_terms < 1.8e4  # config: ~1.5e4 Pauli terms
    assert np.all(np.bitwise_count(inst.x_mask).sum(axis=1) <= 4)
    assert len(np.unique(np.concatenate([inst.x_mask, inst.z_mask], axis=1), axis=0)) == inst.n_terms


def test_samples_beyond_64_qubits():
    from synth.samples import peaked_samples
    vals, ranks = peaked_samples(42, 10, 10, 3000, 7)
    assert all(v > 0 and v < (1 << 84) for v in vals)
    even = int("01" * 42, 2)
    assert all(bin(v & even).count("1") == 10 and bin(v & ~even).count("1") == 10 for v in vals)
    assert any(v >> 64 for v in vals)
