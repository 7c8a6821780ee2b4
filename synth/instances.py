"""Named, seeded workload instances shaped like the paper's molecules.

Seeds: integrals 1000+N, samples 2000+N, log-amplitudes 3000+N (numpy PCG64).
Instances are deterministic functions of their name; large ones are cached as
``.npz`` files under ``$NQS_CACHE`` (default ``<repo>/.cache``).
"""

import dataclasses
import math
import os
import time

import numpy as np

from .bits import n_words, pack_ints
from .molecular import molecular_integrals, jordan_wigner
from .samples import peaked_samples, all_sector_determinants

_GEN_VERSION = 3


@dataclasses.dataclass
class Instance:
    name: str
    n_qubits: int
    n_alpha: int
    n_beta: int
    x_mask: np.ndarray          # [T, W] uint64 (symplectic Pauli encoding)
    z_mask: np.ndarray          # [T, W] uint64
    coef: np.ndarray            # [T] float64
    U: np.ndarray               # [n_unq, W] uint64, unique, caller order
    ranks: np.ndarray           # [n_unq] excitation rank of each sample
    logpsi_re: np.ndarray       # [n_unq] float64
    logpsi_im: np.ndarray       # [n_unq] float64 (zeros for real amplitudes)
    meta: dict

    @property
    def n_words(self):
        return n_words(self.n_qubits)

    @property
    def n_unq(self):
        return int(self.U.shape[0])

    @property
    def n_terms(self):
        return int(self.coef.shape[0])


# name -> (n_orb, n_alpha, n_beta, irrep_bits, n_unq or None for the full sector)
CONFIGS = {
    "h12": (6, 2, 2, 2, None),
    "h28": (14, 5, 5, 2, 10_000),
    "h56": (28, 7, 7, 2, 100_000),
    "h84": (42, 10, 10, 2, 200_000),
}


def _cache_dir():
    d = os.environ.get("NQS_CACHE")
    if not d:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".cache")
    os.makedirs(d, exist_ok=True)
    return d


def _hamiltonian(n_orb, irrep_bits, seed):
    h1, eri, irreps = molecular_integrals(n_orb, seed, irrep_bits=irrep_bits)
    x, z, c = jordan_wigner(h1, eri, 2 * n_orb)
    return x, z, c, h1, eri, irreps


def config_instance(name: str, n_unq: int = None, use_cache: bool = True,
                    complex_phase: bool = False) -> Instance:
    """Build (or load) a named instance.

    ``n_unq`` overrides the configured batch size (a smaller peaked batch of
    the same Hamiltonian); ``complex_phase`` gives every amplitude a seeded
    random sign (imaginary part 0 or pi).
    """
    n_orb, n_a, n_b, irrep_bits, cfg_unq = CONFIGS[name]
    N = 2 * n_orb
    n_unq = cfg_unq if n_unq is None else int(n_unq)
    key = f"{name}_u{n_unq}_v{_GEN_VERSION}"
    path = os.path.join(_cache_dir(), key + ".npz")
    if use_cache and os.path.exists(path):
        d = np.load(path, allow_pickle=False)
        inst = Instance(name, N, n_a, n_b, d["x"], d["z"], d["c"], d["U"], d["ranks"],
                        d["lre"], d["lim"], {"n_orb": n_orb, "cached": True})
    else:
        t0 = time.time()
        x, z, c, h1, eri, irreps = _hamiltonian(n_orb, irrep_bits, 1000 + N)
        t_ham = time.time() - t0
        rng_l = np.random.default_rng(3000 + N)
        if n_unq is None:
            vals = all_sector_determinants(n_orb, n_a, n_b)
            ranks = np.zeros(len(vals), dtype=np.int64)
            U = pack_ints(vals, N)
            lre = rng_l.normal(0.0, 1.0, size=len(vals))
        else:
            vals, ranks = peaked_samples(n_orb, n_a, n_b, n_unq, 2000 + N)
            U = pack_ints(vals, N)
            lre = -2.0 * ranks + rng_l.normal(0.0, 0.3, size=len(vals))
        lim = np.zeros_like(lre)
        inst = Instance(name, N, n_a, n_b, x, z, c, U, ranks, lre, lim,
                        {"n_orb": n_orb, "cached": False, "t_ham_s": t_ham})
        if use_cache:
            np.savez(path, x=x, z=z, c=c, U=U, ranks=ranks, lre=lre, lim=lim)
    if complex_phase:
        rng_p = np.random.default_rng(4000 + N)
        inst.logpsi_im = np.where(rng_p.random(inst.n_unq) < 0.5, 0.0, math.pi)
    return inst


def batched_instances(n_inst: int = 64, seed: int = 5000, use_cache: bool = True):
    """Uneven instances: N uniform in {20,28,36,44,56}, n_alpha = n_beta =
    ceil(N/8), |U| = round(10^U(3,5)) capped at half the sector's size.

    Returns a list of Instance.  Instances of the same N share that N's
    Hamiltonian (integrals seed 1000+N); every instance has its own peaked
    batch (samples seed 6000+t) and log-amplitudes (seed 7000+t).
    """
    path = os.path.join(_cache_dir(), f"batched_{n_inst}_s{seed}_v{_GEN_VERSION}.npz")
    rng = np.random.default_rng(seed)
    plan = []
    for t in range(n_inst):
        N = int(rng.choice([20, 28, 36, 44, 56]))
        ne = math.ceil(N / 8)
        sector = math.comb(N // 2, ne) ** 2
        plan.append((N, ne, min(int(round(10 ** rng.uniform(3, 5))), sector // 2)))
    cached = np.load(path, allow_pickle=False) if use_cache and os.path.exists(path) else None
    hams, out, save = {}, [], {}
    for t, (N, ne, n_unq) in enumerate(plan):
        n_orb = N // 2
        if N not in hams:
            if cached is not None:
                hams[N] = (cached[f"x{N}"], cached[f"z{N}"], cached[f"c{N}"])
            else:
                x, z, c, _, _, _ = _hamiltonian(n_orb, 2, 1000 + N)
                hams[N] = (x, z, c)
                save.update({f"x{N}": x, f"z{N}": z, f"c{N}": c})
        x, z, c = hams[N]
        if cached is not None:
            U, ranks, lre = cached[f"U{t}"], cached[f"r{t}"], cached[f"l{t}"]
        else:
            vals, ranks = peaked_samples(n_orb, ne, ne, n_unq, 6000 + t)
            U = pack_ints(vals, N)
            rng_l = np.random.default_rng(7000 + t)
            lre = -2.0 * ranks + rng_l.normal(0.0, 0.3, size=len(vals))
            save.update({f"U{t}": U, f"r{t}": ranks, f"l{t}": lre})
        out.append(Instance(f"b{t}_N{N}", N, ne, ne, x, z, c, U, ranks, lre,
                            np.zeros_like(lre), {"n_orb": n_orb, "batched": True}))
    if cached is None and use_cache:
        np.savez(path, **save)
    return out


def random_pauli_hamiltonian(n_qubits: int, n_terms: int, seed: int,
                             allow_odd_y: bool = True, max_weight: int = None):
    """Random Pauli strings with real coefficients (a Hermitian operator).

    Each qubit of a string is I, X, Y or Z uniformly (restricted to
    ``max_weight`` non-identity positions if given).  With
    ``allow_odd_y=False`` strings with an odd number of Y are redrawn, which
    makes the operator real symmetric.  Strings may repeat.
    """
    rng = np.random.default_rng(seed)
    xs, zs, cs = [], [], []
    while len(cs) < n_terms:
        ops = rng.integers(0, 4, size=n_qubits)  # 0 I, 1 X, 2 Y, 3 Z
        if max_weight is not None:
            nz = np.flatnonzero(ops)
            if nz.size > max_weight:
                drop = rng.choice(nz, size=nz.size - max_weight, replace=False)
                ops[drop] = 0
        if not allow_odd_y and (ops == 2).sum() % 2 == 1:
            continue
        x = sum(1 << i for i in range(n_qubits) if ops[i] in (1, 2))
        z = sum(1 << i for i in range(n_qubits) if ops[i] in (2, 3))
        xs.append(x), zs.append(z), cs.append(rng.normal())
    return pack_ints(xs, n_qubits), pack_ints(zs, n_qubits), np.asarray(cs)

