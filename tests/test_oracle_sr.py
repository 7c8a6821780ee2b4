"""The oracle's QGT and min-SR step pinned without their own formulas.

* QGT of an explicit state: for psi_theta(x) = exp(sum_p theta_p f_p(x) +
  i sum_p theta_p g_p(x)) on all 2^4 basis vectors (samples = the whole
  space, weights = the normalised Born probabilities), S of Eq.
  (qgt_definition) equals <d_p psi^|d_q psi^> - <d_p psi^|psi^><psi^|d_q psi^>
  computed from the normalised state vector and central finite differences
  of it in theta (no log-derivatives involved).
* S is Hermitian positive semi-definite; one sample gives S = 0.
* min-SR: Obar^H (T + lambda I)^{-1} eps equals (S + lambda I)^{-1} g with
  g = Obar^H eps, solved directly in parameter space (push-through identity).
* The most probable samples are the largest log-amplitudes (ties by index).
* A planted mistake (no centring) breaks the finite-difference pin.
"""

import math

import numpy as np

import oracle


def _state(theta, F, G):
    return np.exp(F @ theta + 1j * (G @ theta))


def test_qgt_of_explicit_state_vs_finite_differences():
    rng = np.random.default_rng(3)
    P, D = 5, 16
    F = rng.normal(0, 0.6, (D, P)); G = rng.normal(0, 0.6, (D, P))
    theta = rng.normal(0, 0.5, P)
    psi = _state(theta, F, G)
    nrm = lambda v: v / np.linalg.norm(v)
    h = 1e-5
    dpsi = np.zeros((P, D), dtype=complex)
    for p in range(P):
        e = np.zeros(P); e[p] = h
        dpsi[p] = (nrm(_state(theta + e, F, G)) - nrm(_state(theta - e, F, G))) / (2 * h)
    ph = nrm(psi)
    S_fd = dpsi.conj() @ dpsi.T - np.outer(dpsi.conj() @ ph, ph.conj() @ dpsi.T)
    O = F + 1j * G                       # d log psi / d theta_p, per basis vector
    S = oracle.qgt(O, np.log(np.abs(psi)))
    assert np.abs(S - S_fd).max() < 1e-8
    assert np.abs(S - S.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(S).min() > -1e-12


def test_one_sample_gives_zero():
    O = np.random.default_rng(1).normal(size=(1, 6))
    assert np.abs(oracle.qgt(O, np.zeros(1))).max() == 0.0


def test_min_sr_push_through():
    rng = np.random.default_rng(7)
    n, P = 12, 40
    O = rng.normal(size=(n, P)) + 1j * rng.normal(size=(n, P))
    a = rng.normal(0, 1, n)
    eloc = rng.normal(-3, 1, n) + 1j * rng.normal(0, 0.1, n)
    E = 0.3 - 2.0
    lam = 1e-3
    delta, T = oracle.min_sr_step(O, a, eloc, E, lam)
    Ob = oracle.centred(O, a)
    w = oracle.sr_weights(a)
    g = Ob.conj().T @ (np.sqrt(w) * (eloc - E))
    S = oracle.qgt(O, a)
    assert np.abs(Ob.conj().T @ Ob - S).max() < 1e-12
    want = np.linalg.solve(S + lam * np.eye(P), g)
    assert np.abs(delta - want).max() < 1e-8 * max(1.0, np.abs(want).max())
    assert np.abs(T - T.conj().T).max() < 1e-13


def test_top_probable():
    a = np.array([0.5, 2.0, -1.0, 2.0, 1.5])
    assert oracle.top_probable(a, 3) == [1, 3, 4]


def test_planted_uncentred_qgt_fails():
    rng = np.random.default_rng(3)
    P, D = 4, 16
    F = rng.normal(0, 0.6, (D, P)); G = rng.normal(0, 0.6, (D, P))
    theta = rng.normal(0, 0.5, P)
    psi = _state(theta, F, G)
    O = F + 1j * G
    w = oracle.sr_weights(np.log(np.abs(psi)))
    S_bad = (w[:, None, None] * O.conj()[:, :, None] * O[:, None, :]).sum(axis=0)   # no centring
    S = oracle.qgt(O, np.log(np.abs(psi)))
    assert np.abs(S_bad - S).max() > 1e-3
