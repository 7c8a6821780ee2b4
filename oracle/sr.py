"""Stochastic reconfiguration on the most probable samples (oracle; test infrastructure).

Sec. "ANQS-tailored stochastic reconfiguration": the quantum geometric tensor
of Eq. (qgt_definition), estimated with the renormalised probabilities
w(x) = p(x) / sum_y p(y), p = |psi|^2, over the N_SR unique samples of highest
probability, and the SR step nabla E -> S^{-1} nabla E regularised as in
min-SR.  With O_xp = d log psi(x) / d theta_p for the N_SR samples:

    S_pq = sum_x w_x conj(O_xp) O_xq - conj(m_p) m_q,   m = sum_x w_x O_x,

i.e. S = Obar^H Obar with Obar_x = sqrt(w_x) (O_x - m).  The energy gradient
of Eq. (grad_def) with renormalised probabilities is g = Obar^H eps with
eps_x = sqrt(w_x) (E_loc(x) - E).  min-SR solves in sample space:

    T = Obar Obar^H  (N_SR x N_SR),   delta = Obar^H (T + lambda I)^{-1} eps,

which equals (S + lambda I)^{-1} g (push-through identity).

Arrays: O is [n_sr, n_params] (real or complex); logpsi_re gives p; FP64.
"""

import math

import numpy as np


def top_probable(logpsi_re, n_sr):
    """Indices of the n_sr samples of highest probability (ties: lower index first)."""
    a = np.asarray(logpsi_re, dtype=np.float64)
    order = sorted(range(len(a)), key=lambda i: (-a[i], i))
    return order[:n_sr]


def sr_weights(logpsi_re):
    a = np.asarray(logpsi_re, dtype=np.float64)
    p = [math.exp(2.0 * (v - a.max())) for v in a]
    s = math.fsum(p)
    return np.array([v / s for v in p])


def qgt(O, logpsi_re):
    """S_pq of Eq. (qgt_definition) with renormalised probabilities, summed term by term."""
    O = np.asarray(O)
    w = sr_weights(logpsi_re)
    n, P = O.shape
    m = [complex(math.fsum((w[x] * O[x, p]).real for x in range(n)), math.fsum((w[x] * O[x, p]).imag for x in range(n)))
         for p in range(P)]
    S = np.zeros((P, P), dtype=complex)
    for p in range(P):
        for q in range(P):
            t = [w[x] * np.conj(O[x, p]) * O[x, q] for x in range(n)]
            S[p, q] = complex(math.fsum(v.real for v in t), math.fsum(v.imag for v in t)) - np.conj(m[p]) * m[q]
    return S


def centred(O, logpsi_re):
    """Obar_x = sqrt(w_x) (O_x - m)."""
    O = np.asarray(O)
    w = sr_weights(logpsi_re)
    m = (w[:, None] * O).sum(axis=0)
    return np.sqrt(w)[:, None] * (O - m[None, :])


def sample_gram(O, logpsi_re):
    """T = Obar Obar^H (the sample-space Gram matrix of min-SR)."""
    Ob = centred(O, logpsi_re)
    return Ob @ Ob.conj().T


def min_sr_step(O, logpsi_re, eloc, e_var, lam):
    """delta = Obar^H (T + lambda I)^{-1} eps, eps_x = sqrt(w_x) (E_loc(x) - E)."""
    Ob = centred(O, logpsi_re)
    w = sr_weights(logpsi_re)
    eps = np.sqrt(w) * (np.asarray(eloc) - e_var)
    T = Ob @ Ob.conj().T
    x = np.linalg.solve(T + lam * np.eye(T.shape[0]), eps)
    return Ob.conj().T @ x, T
