"""Oracle quantities for selected rows of a large batch (test infrastructure).

At the paper's sizes (1e4-2e5 unique samples, up to ~1e6 terms) the whole
oracle takes too long, so full-size checks compare a sample of rows.  Each
row is computed exactly as in ``energy``: its coupled set by LoopOverTerms
(Alg. 2A), its matrix elements by MatrixElement, its local energy by the
restricted Eq. (local_energy).
"""

import cmath
import math

import numpy as np

from .hamiltonian import PreparedHamiltonian, _as_int_list, prepare_hamiltonian
from .pairs import couple_via_unique_xy
from .energy import matrix_element, _csum


class RowOracle:
    def __init__(self, U, ham: PreparedHamiltonian, logpsi_re, logpsi_im=None):
        self.U = _as_int_list(U)
        self.n = len(self.U)
        self.ham = ham
        self.u_index = {x: j for j, x in enumerate(self.U)}
        if len(self.u_index) != self.n:
            raise ValueError("U holds repeated samples")
        re = np.asarray(logpsi_re, dtype=np.float64).ravel()
        im = np.zeros(self.n) if logpsi_im is None else np.asarray(logpsi_im, dtype=np.float64).ravel()
        self.l = [complex(a, b) for a, b in zip(re, im)]
        self.a = re

    @classmethod
    def from_instance(cls, inst):
        ham = prepare_hamiltonian(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)
        return cls(inst.U, ham, inst.logpsi_re, inst.logpsi_im)

    def coupled(self, i):
        """SC_{x_i} as positions j (Alg. 2A order)."""
        return couple_via_unique_xy(self.U[i], self.u_index, self.ham.xy_list)

    def row(self, i):
        """Coupled positions, matrix elements and E_loc^var of row i."""
        js = self.coupled(i)
        x = self.U[i]
        hs = [matrix_element(x, self.U[j], self.ham) for j in js]
        eloc = _csum(h * cmath.exp(self.l[j] - self.l[i]) for h, j in zip(hs, js))
        return {"j": js, "H": hs, "eloc": eloc}

    def weights(self):
        """Normalised Born weights w = p / sum p with p = exp(2 (a - max a))."""
        p = np.exp(2.0 * (self.a - self.a.max()))
        return p / math.fsum(p)

    def row_vjp(self, y, eloc_all, e_var, g_eloc_re=None, g_eloc_im=None, g_evar=0.0, w=None):
        """(d/d Re l_y, d/d Im l_y) of the loss of ``energy.local_energy_vjp``.

        Column y of D collects the pairs (x, y): by Eq. (pauli_melem) these are
        the x with x XOR y an XY pattern, i.e. the coupled set of y itself.
        ``eloc_all`` is the full E_loc^var (complex array) the loss is
        evaluated at.
        """
        if w is None:
            w = self.weights()
        gr = np.zeros(self.n) if g_eloc_re is None else np.asarray(g_eloc_re, dtype=np.float64)
        gi = np.zeros(self.n) if g_eloc_im is None else np.asarray(g_eloc_im, dtype=np.float64)
        gr_eff = lambda x: gr[x] + float(g_evar) * w[x]
        r = self.row(y)
        da, db = [], []
        hyy = complex(0.0, 0.0)
        for h, x in zip(r["H"], r["j"]):
            if x == y:
                hyy = h
                continue
            T = matrix_element(self.U[x], self.U[y], self.ham) * cmath.exp(self.l[y] - self.l[x])
            da.append(gr_eff(x) * T.real + gi[x] * T.imag)
            db.append(-gr_eff(x) * T.imag + gi[x] * T.real)
        Dyy = -(complex(eloc_all[y]) - hyy)
        da.append(gr_eff(y) * Dyy.real + gi[y] * Dyy.imag)
        db.append(-gr_eff(y) * Dyy.imag + gi[y] * Dyy.real)
        g_re = math.fsum(da) + float(g_evar) * 2.0 * w[y] * (complex(eloc_all[y]).real - float(np.real(e_var)))
        g_im = math.fsum(db)
        return g_re, g_im
