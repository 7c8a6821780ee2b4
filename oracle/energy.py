"""Matrix elements, surrogate local energies, variational energy and their
derivatives (oracle; test infrastructure).

Amplitudes are given as log psi = l = a + i b per sample (b may be absent),
so psi(x') / psi(x) = exp(l(x') - l(x)) and the Born weight is
p(x) = |psi(x)|^2 = exp(2 a(x)) up to a constant that cancels.
"""

import cmath
import math

import numpy as np

from .hamiltonian import PreparedHamiltonian, pauli_matrix_element, _as_int_list, _I_POW
from .pairs import find_coupled_pairs


def _csum(values):
    """Correctly rounded sum of complex values (real and imaginary separately)."""
    vals = list(values)
    return complex(math.fsum(v.real for v in vals), math.fsum(v.imag for v in vals))


def matrix_element(x: int, xp: int, ham: PreparedHamiltonian) -> complex:
    """MatrixElement (supplementary algorithm "Calculating the Hamiltonian matrix element").

    XY = x XOR x'; for each term of P_XY, phi = (pi/2)|Y| + pi|x' AND YZ| and
    H_xx' += h exp(i phi).  The terms of P_XY all satisfy x XOR x' = XY, so
    exp(i phi) = i^(|Y| + 2|x' & YZ|) exactly.
    """
    contrib = []
    for t in ham.group(x ^ xp):
        a = t.Y.bit_count() + 2 * (xp & t.YZ).bit_count()
        contrib.append(t.h * _I_POW[a % 4])
    return _csum(contrib)


def matrix_element_all_terms(x: int, xp: int, ham: PreparedHamiltonian) -> complex:
    """H_xx' = sum over *all* terms of h_l <x|P^(l)|x'> (Eq. jw_hamiltonian with
    Eq. pauli_melem), without the grouping by XY."""
    return _csum(t.h * pauli_matrix_element(x, xp, t) for t in ham.terms)


def _logpsi(logpsi_re, logpsi_im, n):
    re = [float(v) for v in np.asarray(logpsi_re, dtype=np.float64).ravel()]
    if logpsi_im is None:
        im = [0.0] * n
    else:
        im = [float(v) for v in np.asarray(logpsi_im, dtype=np.float64).ravel()]
    if len(re) != n or len(im) != n:
        raise ValueError("log psi length differs from the batch")
    return [complex(a, b) for a, b in zip(re, im)]


def local_energy_var(U, logpsi_re, logpsi_im, ham: PreparedHamiltonian, pairs=None):
    """E_loc^var(x) = sum over x' in SC_x of H_xx' psi(x') / psi(x).

    This is Eq. (local_energy) with the sum restricted to the sampled batch
    (the surrogate of Sec. "Streamlined local energy calculations"; the three
    steps of Fig. scatter_local_energies).  ``pairs`` defaults to the
    LoopOverTerms pair list.  Returns (eloc: list of complex, hvals: dict
    (i, j) -> H_ij).
    """
    U = _as_int_list(U)
    n = len(U)
    l = _logpsi(logpsi_re, logpsi_im, n)
    if pairs is None:
        pairs = find_coupled_pairs(U, ham, "terms")
    rows = [[] for _ in range(n)]
    hvals = {}
    for (i, j) in pairs:
        h = matrix_element(U[i], U[j], ham)
        hvals[(i, j)] = h
        rows[i].append(h * cmath.exp(l[j] - l[i]))
    return [_csum(r) for r in rows], hvals


def variational_energy(logpsi_re, eloc):
    """E^var = sum_x E_loc^var(x) p(x) / sum_x p(x), p = |psi|^2 (Eq. variational_energy).

    The weights are exp(2 (a - max a)); the common factor cancels.  Returns
    the complex value (its imaginary part vanishes for Hermitian H up to
    rounding).
    """
    a = [float(v) for v in np.asarray(logpsi_re, dtype=np.float64).ravel()]
    amax = max(a)
    p = [math.exp(2.0 * (ai - amax)) for ai in a]
    norm = math.fsum(p)
    num = _csum(pi * e for pi, e in zip(p, eloc))
    return num / norm


def energy_gradient_closed_form(logpsi_re, eloc, e_var):
    """dE^var/d Re l_y = 2 w_y (Re E_loc(y) - E), dE^var/d Im l_y = 2 w_y Im E_loc(y),
    w_y = p(y) / sum p.

    Follows from Eq. (variational_energy) with p = |psi|^2 = exp(2 Re l) and
    the Hermiticity of H; it is the same structure as Eq. (grad_def) with the
    renormalised probabilities in place of sample frequencies.
    """
    a = np.asarray(logpsi_re, dtype=np.float64).ravel()
    p = np.exp(2.0 * (a - a.max()))
    w = p / math.fsum(p)
    er = np.array([e.real for e in eloc])
    ei = np.array([e.imag for e in eloc])
    E = float(np.real(e_var))
    return 2.0 * w * (er - E), 2.0 * w * ei


def local_energy_vjp(U, logpsi_re, logpsi_im, ham: PreparedHamiltonian, pairs,
                     g_eloc_re=None, g_eloc_im=None, g_evar=0.0):
    """Vector-Jacobian product of L = sum_x [gr(x) Re E_loc(x) + gi(x) Im E_loc(x)]
    + g_E Re E^var with respect to (Re l, Im l), by the plain chain rule.

    With T = H_xx' exp(l(x') - l(x)) for each listed pair (x, x'),
    d E_loc(x) / d Re l(y) = sum over pairs of T (delta_{x'y} - delta_{xy}) =: D_xy
    and d E_loc(x) / d Im l(y) = i D_xy.  E^var = sum_x w_x Re E_loc(x) adds
    g_E [w_x to the upstream of Re E_loc(x)] and g_E 2 w_y (Re E_loc(y) - E)
    through the weights.  Scatters over every pair into its column.
    """
    U = _as_int_list(U)
    n = len(U)
    l = _logpsi(logpsi_re, logpsi_im, n)
    gr = np.zeros(n) if g_eloc_re is None else np.asarray(g_eloc_re, dtype=np.float64).copy()
    gi = np.zeros(n) if g_eloc_im is None else np.asarray(g_eloc_im, dtype=np.float64).copy()
    eloc, _ = local_energy_var(U, logpsi_re, logpsi_im, ham, pairs)
    e_var = variational_energy(logpsi_re, eloc).real
    a = np.array([v.real for v in l])
    p = np.exp(2.0 * (a - a.max()))
    w = p / math.fsum(p)
    gr_eff = gr + float(g_evar) * w

    da = [[] for _ in range(n)]
    db = [[] for _ in range(n)]
    for (x, xp) in pairs:
        T = matrix_element(U[x], U[xp], ham) * cmath.exp(l[xp] - l[x])
        for (y, sgn) in ((xp, 1.0), (x, -1.0)):
            D = sgn * T
            da[y].append(gr_eff[x] * D.real + gi[x] * D.imag)
            db[y].append(-gr_eff[x] * D.imag + gi[x] * D.real)
    g_re = np.array([math.fsum(v) for v in da])
    g_im = np.array([math.fsum(v) for v in db])
    g_re += float(g_evar) * 2.0 * w * (np.array([e.real for e in eloc]) - e_var)
    return g_re, g_im


def forward(U, logpsi_re, logpsi_im, ham: PreparedHamiltonian, method: str = "terms"):
    """Pairs, matrix elements, E_loc^var and E^var for a whole batch."""
    pairs = find_coupled_pairs(U, ham, method)
    eloc, hvals = local_energy_var(U, logpsi_re, logpsi_im, ham, pairs)
    e_var = variational_energy(logpsi_re, eloc)
    return {"pairs": pairs, "H": hvals, "eloc": eloc, "e_var": e_var}
