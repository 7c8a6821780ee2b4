"""Stochastic reconfiguration on the most probable samples (GPU required).

The sample-space Gram matrix T = Obar Obar^T of min-SR is formed on the
tensor cores (tcgen05) from a bf16 hi + lo split of Obar with FP32
accumulation.  Tolerance, from that arithmetic: each value keeps a relative
error of at most 2^-18 after the split and the dropped lo lo term is below
2^-18 |v_i v_j|, so each product is off by at most ~3 * 2^-18 |v_i v_j|;
FP32 accumulation over a CTA's K range adds less at these sizes.  Summed and
bounded by Cauchy-Schwarz (sum |v_ik v_jk| <= sqrt(T_ii T_jj)):
    |T_ij - T_ij(oracle)| <= 5e-5 sqrt(T_ii T_jj).
The solve is FP64; the step delta_p = sum_x sqrt(w_x) y_x (O_xp - m_p) takes
FP32 factors (the mean, the scaled solution, the products: a few roundings of
2^-24 each) summed with compensation, so given the GPU's own T it must equal
Obar^T y from the oracle's Obar and eps within 1e-6 sum_x |sqrt(w_x) y_x|
|O_xp - m_p| per entry (the terms cancel, so the bound is on their
magnitudes, not on delta's), y solving the system the kernel factorises:
T + lambda I + c u u^T with u = sqrt(w), c = tr T / n (u is a null vector of
the exact T that Obar^T annihilates, so the step is that of T + lambda I).
The selection of the most probable samples is exact.
"""

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2408_07625_gb300 as nqs


@pytest.mark.parametrize("n,P,seed", [(1, 64, 1), (7, 1000, 2), (100, 4097, 3), (128, 64, 4), (100, 200_000, 5)])
def test_gram_and_step_match_oracle(n, P, seed):
    rng = np.random.default_rng(seed)
    O = (rng.normal(0.0, 1.0, (n, P)) + rng.normal(0.0, 0.5, P)[None, :]).astype(np.float32)  # a shared mean
    a = rng.normal(0.0, 0.7, n)
    eloc = rng.normal(-5.0, 1.0, n)
    E = -5.1
    Ot = torch.from_numpy(O).cuda()
    T_ref = oracle.sample_gram(O.astype(np.float64), a)
    lam = 0.1 * max(1e-12, float(np.trace(T_ref)) / n)
    delta, T = nqs.sr_step(Ot, a, eloc, E, lam, want_T=True)
    T = T.cpu().numpy()
    d = np.sqrt(np.outer(np.diag(T_ref), np.diag(T_ref)))
    assert np.all(np.abs(T - T_ref) <= 5e-5 * d + 1e-30), float(np.max(np.abs(T - T_ref) / (d + 1e-300)))
    assert np.abs(T - T.T).max() == 0.0
    Ob = oracle.centred(O.astype(np.float64), a)
    w = oracle.sr_weights(a)
    eps = np.sqrt(w) * (eloc - E)
    u = np.sqrt(w)
    y = np.linalg.solve(T + lam * np.eye(n) + (np.trace(T) / n) * np.outer(u, u), eps)
    want = Ob.T @ y
    mag = np.abs(Ob).T @ np.abs(y)
    got = delta.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-6 * mag + 1e-300), float(np.max(np.abs(got - want) / (mag + 1e-300)))
    # and against the oracle's own step (its T in FP64): within the Gram tolerance propagated
    ref, _ = oracle.min_sr_step(O.astype(np.float64), a, eloc, E, lam)
    assert np.abs(got - ref.real).max() <= 1e-3 * max(1e-30, np.abs(ref).max())


def test_small_lambda_matches_oracle():
    """lambda far below the Gram's rounding (1e-6 of its mean eigenvalue): the centred T
    is singular along sqrt(w), so T + lambda I is only as definite as the rounding lets
    it be; the step must still equal the oracle's FP64 step.  Weights of similar size
    keep T's other eigenvalues within a small factor, so the Gram tolerance carries
    over to delta as a relative 1e-3."""
    rng = np.random.default_rng(21)
    n, P = 100, 200_000
    O = (rng.normal(0.0, 1.0, (n, P)) + rng.normal(0.0, 0.5, P)[None, :]).astype(np.float32)
    a = rng.normal(0.0, 0.2, n)
    eloc = rng.normal(-5.0, 1.0, n)
    E = -5.1
    T_ref = oracle.sample_gram(O.astype(np.float64), a)
    lam = 1e-6 * float(np.trace(T_ref)) / n
    delta = nqs.sr_step(torch.from_numpy(O).cuda(), a, eloc, E, lam)[0].cpu().numpy()
    ref, _ = oracle.min_sr_step(O.astype(np.float64), a, eloc, E, lam)
    assert np.abs(delta - ref.real).max() <= 1e-3 * np.abs(ref).max()


def test_top_probable():
    rng = np.random.default_rng(9)
    a = np.round(rng.normal(0.0, 2.0, 100_000), 2)   # many ties
    idx = nqs.sr_top(a, 100).cpu().numpy().tolist()
    assert idx == oracle.top_probable(a, 100)
