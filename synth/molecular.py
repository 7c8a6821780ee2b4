"""Synthetic molecular integrals and their Jordan-Wigner qubit Hamiltonian.

The second-quantised Hamiltonian is the one of Eq. (fermionic_qc) written in
chemists' notation over spatial orbitals p, q, r, s and spins sigma, tau:

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,st} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}

Spin-orbitals are interleaved: qubit 2p is p-alpha, qubit 2p+1 is p-beta, so
the Hartree-Fock determinant with n_alpha = n_beta occupies the first n_e
qubits, as the paper's basis section states.

The Jordan-Wigner mapping (Eq. jw_hamiltonian) is written from its definition
a+_j = Z_0..Z_{j-1} (X_j - i Y_j)/2.  Internally every operator is kept as a
real combination of monomials X^x Z^z (x, z bit masks; Z applied first), whose
product rule is (X^a Z^b)(X^c Z^d) = (-1)^{|b & c|} X^{a^c} Z^{b^d}.  In that
basis a+_j = 1/2 (X^{e_j} Z^{m_j} + X^{e_j} Z^{m_j ^ e_j}) and
a_j = 1/2 (X^{e_j} Z^{m_j} - X^{e_j} Z^{m_j ^ e_j}) with e_j the unit mask of
qubit j and m_j the mask of all qubits below j.  At the end a monomial is
converted to a Pauli string: X^x Z^z = (-i)^{|x & z|} P(x, z), where P(x, z)
carries Y on x & z, X on x & ~z and Z on z & ~x (the symplectic encoding the
library takes).
"""

import numpy as np

from .bits import n_words


# --------------------------------------------------------------------------
# integrals
# --------------------------------------------------------------------------

def molecular_integrals(n_orb: int, seed: int, irrep_bits: int = 0,
                        sigma: float = 0.5):
    """Random real integrals shaped like a small molecule's.

    * h_pq symmetric; diagonal h_pp = -10 + 2p (ascending orbital energies so
      that the lowest orbitals form a dominant Hartree-Fock determinant),
      off-diagonal N(0, sigma).
    * (pq|rs) with the 8-fold permutational symmetry of real orbitals;
      Coulomb-like (pp|qq) = 1 + |N(0, sigma)|, every other canonical entry
      N(0, sigma), copied to its 8 images.
    * Optional abelian point-group labels: each spatial orbital gets an irrep
      in Z_2^irrep_bits; an integral is kept only when the product (XOR) of
      its orbitals' irreps is the totally symmetric one, as point-group
      symmetry does for real molecules.  This brings the Pauli-term counts
      close to those of the paper's molecules.

    Returns (h1 [n,n], eri [n,n,n,n], irreps [n]).
    """
    rng = np.random.default_rng(seed)
    n = int(n_orb)
    irreps = (rng.integers(0, 1 << irrep_bits, size=n) if irrep_bits > 0
              else np.zeros(n, dtype=np.int64))

    h1 = np.zeros((n, n))
    for p in range(n):
        h1[p, p] = -10.0 + 2.0 * p
        for q in range(p):
            v = rng.normal(0.0, sigma)
            if irreps[p] != irreps[q]:
                v = 0.0
            h1[p, q] = h1[q, p] = v

    eri = np.zeros((n, n, n, n))
    # canonical representatives: p>=q, r>=s, pq>=rs (pair index)
    for p in range(n):
        for q in range(p + 1):
            pq = p * (p + 1) // 2 + q
            for r in range(n):
                for s in range(r + 1):
                    rs = r * (r + 1) // 2 + s
                    if rs > pq:
                        continue
                    if p == q and r == s:
                        v = 1.0 + abs(rng.normal(0.0, sigma))
                    else:
                        v = rng.normal(0.0, sigma)
                    if irreps[p] ^ irreps[q] ^ irreps[r] ^ irreps[s]:
                        v = 0.0
                    for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                        eri[a, b, c, d] = v
    return h1, eri, irreps


def hf_energy_from_integrals(h1, eri, occ_alpha, occ_beta) -> float:
    """Slater-Condon diagonal energy of a determinant from the integrals.

    E = sum_{i occ} h_ii + 1/2 sum_{i,j occ} [(ii|jj) - delta_{s_i s_j} (ij|ji)]
    (spin-orbital sum).  Used only as an independent check of the mapping.
    """
    so = [(p, 0) for p in occ_alpha] + [(p, 1) for p in occ_beta]
    e = 0.0
    for (p, s) in so:
        e += h1[p, p]
    for (p, s) in so:
        for (q, t) in so:
            e += 0.5 * eri[p, p, q, q]
            if s == t:
                e -= 0.5 * eri[p, q, q, p]
    return float(e)


# --------------------------------------------------------------------------
# Jordan-Wigner in the X^x Z^z monomial basis, vectorised over index tuples
# --------------------------------------------------------------------------

def _unit_and_below(idx: np.ndarray, W: int):
    """Unit mask e_j and below-mask m_j (bits < j) for each index j: [n, W]."""
    idx = np.asarray(idx, dtype=np.int64)
    n = idx.size
    e = np.zeros((n, W), dtype=np.uint64)
    m = np.zeros((n, W), dtype=np.uint64)
    word = idx // 64
    bit = (idx % 64).astype(np.uint64)
    one = np.uint64(1)
    for w in range(W):
        sel = word == w
        e[sel, w] = one << bit[sel]
        m[sel, w] = (one << bit[sel]) - one
        m[word > w, w] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return e, m


def _ladder(idx, dagger: bool, W: int):
    """a+_j (dagger) or a_j as two monomials per index: x,z [n,2,W], c [n,2]."""
    e, m = _unit_and_below(idx, W)
    n = e.shape[0]
    x = np.stack([e, e], axis=1)
    z = np.stack([m, m ^ e], axis=1)
    c = np.empty((n, 2))
    c[:, 0] = 0.5
    c[:, 1] = 0.5 if dagger else -0.5
    return x, z, c


def _mul(A, B):
    """Product of monomial sums, tuple-wise: (X^a Z^b)(X^c Z^d) = (-1)^{|b&c|} X^{a^c} Z^{b^d}."""
    xa, za, ca = A
    xb, zb, cb = B
    n, a, W = xa.shape
    b = xb.shape[1]
    x = xa[:, :, None, :] ^ xb[:, None, :, :]
    z = za[:, :, None, :] ^ zb[:, None, :, :]
    par = np.bitwise_count(za[:, :, None, :] & xb[:, None, :, :]).sum(axis=-1) & 1
    c = ca[:, :, None] * cb[:, None, :] * (1.0 - 2.0 * par)
    return x.reshape(n, a * b, W), z.reshape(n, a * b, W), c.reshape(n, a * b)


def _reduce(x, z, c):
    """Merge identical monomials (sum coefficients); x,z [M,W], c [M]."""
    if x.shape[0] == 0:
        return x, z, c
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    csum = np.bincount(inv.ravel(), weights=c, minlength=uniq.shape[0])
    W = x.shape[1]
    return uniq[:, :W].copy(), uniq[:, W:].copy(), csum


def jordan_wigner(h1, eri, n_qubits: int = None, ecore: float = 0.0,
                  drop_tol: float = 1e-12, chunk: int = 40000):
    """Qubit Hamiltonian (Eq. jw_hamiltonian) of the integrals' fermionic H.

    Returns (x_mask [T,W] uint64, z_mask [T,W] uint64, coef [T] float64): the
    symplectic Pauli encoding (Y where both bits are set) with real
    coefficients; terms are unique and sorted by (x, z).
    """
    n = h1.shape[0]
    N = 2 * n if n_qubits is None else int(n_qubits)
    W = n_words(N)
    parts_x, parts_z, parts_c = [], [], []

    # identity / core constant
    parts_x.append(np.zeros((1, W), dtype=np.uint64))
    parts_z.append(np.zeros((1, W), dtype=np.uint64))
    parts_c.append(np.array([float(ecore)]))

    # one-body: h_pq a+_{p s} a_{q s}
    pp, qq = np.nonzero(h1)
    P = np.concatenate([2 * pp, 2 * pp + 1])
    Q = np.concatenate([2 * qq, 2 * qq + 1])
    v = np.concatenate([h1[pp, qq], h1[pp, qq]])
    if P.size:
        A = _mul(_ladder(P, True, W), _ladder(Q, False, W))
        c = A[2] * v[:, None]
        x, z, c = _reduce(A[0].reshape(-1, W), A[1].reshape(-1, W), c.ravel())
        parts_x.append(x), parts_z.append(z), parts_c.append(c)

    # two-body: 1/2 (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
    p_, q_, r_, s_ = np.nonzero(eri)
    vals = eri[p_, q_, r_, s_]
    spin_P, spin_R = [], []
    Ps, Qs, Rs, Ss, Vs = [], [], [], [], []
    for sg in (0, 1):
        for tg in (0, 1):
            Pi = 2 * p_ + sg
            Qi = 2 * q_ + sg
            Ri = 2 * r_ + tg
            Si = 2 * s_ + tg
            keep = (Pi != Ri) & (Qi != Si)
            Ps.append(Pi[keep]), Qs.append(Qi[keep]), Rs.append(Ri[keep]), Ss.append(Si[keep])
            Vs.append(0.5 * vals[keep])
    Ps = np.concatenate(Ps); Qs = np.concatenate(Qs)
    Rs = np.concatenate(Rs); Ss = np.concatenate(Ss); Vs = np.concatenate(Vs)
    for a in range(0, Ps.size, chunk):
        sl = slice(a, a + chunk)
        A = _ladder(Ps[sl], True, W)
        A = _mul(A, _ladder(Rs[sl], True, W))
        A = _mul(A, _ladder(Ss[sl], False, W))
        A = _mul(A, _ladder(Qs[sl], False, W))
        c = A[2] * Vs[sl][:, None]
        x, z, c = _reduce(A[0].reshape(-1, W), A[1].reshape(-1, W), c.ravel())
        parts_x.append(x), parts_z.append(z), parts_c.append(c)

    x, z, c = _reduce(np.concatenate(parts_x), np.concatenate(parts_z), np.concatenate(parts_c))

    # X^x Z^z = (-i)^{|x&z|} P(x,z): even |x&z| -> real factor (-1)^{|x&z|/2};
    # odd |x&z| monomials are antisymmetric and cancel for a real symmetric H.
    ny = np.bitwise_count(x & z).sum(axis=1)
    odd = (ny & 1) == 1
    if odd.any() and np.abs(c[odd]).max() > 1e-9:
        raise AssertionError("imaginary Pauli coefficients in a real Hamiltonian")
    coef = c * np.where((ny // 2) % 2 == 1, -1.0, 1.0)
    keep = (~odd) & (np.abs(coef) > drop_tol)
    return x[keep], z[keep], coef[keep]


def pauli_to_xyz(x_mask: np.ndarray, z_mask: np.ndarray):
    """Symplectic (x, z) -> the paper's exclusive (X, Y, Z) position masks."""
    x_mask = np.asarray(x_mask, dtype=np.uint64)
    z_mask = np.asarray(z_mask, dtype=np.uint64)
    return x_mask & ~z_mask, x_mask & z_mask, z_mask & ~x_mask
