"""Expected per-row results of the full-size workloads, written by the oracle.

Run as a script, this module computes with ``oracle/`` alone (inputs from
``synth``), for every row i of a named workload (h56: 1e5 samples, h84: 2e5):

* the size of the coupled set SC_{x_i} (Eq. pauli_melem: the x' in U with
  x_i XOR x' an XY pattern of the merged Hamiltonian), diagonal included;
* a digest of that set: the sum, modulo 2^64, of a 64-bit mixing function of
  every column index j in it (order-independent, so any listing order gives
  the same value);
* E_loc^var(x_i) in FP64 (Eq. local_energy restricted to U, correctly
  rounded sums), and
* E^var over the whole batch (Eq. variational_energy);

and stores them in ``tests/golden/<name>_rows.npz`` together with digests of
the integer inputs (U and the Pauli masks) and the sum of |h_l|, so that a
test can tell when the generator produced a different instance.

The GPU test (``tests/test_gpu_full_parity.py``) recomputes the same digest
from the library's pair list with ``set_digest_np``.

    python tests/golden/full_size.py h56 --procs 8
    python tests/golden/full_size.py h84 --procs 8

A process pool with the ``spawn`` start method splits the rows into
contiguous blocks; every worker rebuilds the row oracle from the cached
instance.
"""

import argparse
import hashlib
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

_M64 = (1 << 64) - 1


def mix64_py(j: int) -> int:
    """SplitMix64's finaliser applied to j + 1 (Python ints, mod 2^64)."""
    z = (j + 1 + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def mix64_np(j: np.ndarray) -> np.ndarray:
    """The same function on a uint64 array (numpy wraps modulo 2^64)."""
    with np.errstate(over="ignore"):
        z = j.astype(np.uint64) + np.uint64(1 + 0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def set_digest_py(cols) -> int:
    return sum(mix64_py(int(j)) for j in cols) & _M64


def set_digest_np(row_ptr: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Per-row digests of a CSR list (row_ptr int64 [rows + 1], cols uint32)."""
    rows = len(row_ptr) - 1
    m = mix64_np(cols)
    out = np.zeros(rows, dtype=np.uint64)
    lens = np.diff(row_ptr)
    nz = np.nonzero(lens > 0)[0]
    if len(nz):
        with np.errstate(over="ignore"):
            out[nz] = np.add.reduceat(m, row_ptr[nz].astype(np.int64), dtype=np.uint64)
    return out


def instance_digests(inst):
    """Digests of the integer inputs and the coefficient mass of an instance."""
    u = hashlib.sha256(np.ascontiguousarray(inst.U).tobytes()).hexdigest()
    xz = hashlib.sha256(np.ascontiguousarray(inst.x_mask).tobytes() +
                        np.ascontiguousarray(inst.z_mask).tobytes()).hexdigest()
    return u, xz, math.fsum(np.abs(inst.coef).tolist())


_RO = None


def _init(name):
    global _RO
    sys.path.insert(0, ROOT)
    import oracle
    from synth import config_instance
    _RO = oracle.RowOracle.from_instance(config_instance(name))


def _block(bounds):
    r0, r1 = bounds
    cnt = np.zeros(r1 - r0, np.int64)
    dig = np.zeros(r1 - r0, np.uint64)
    el = np.zeros(r1 - r0, np.float64)
    for i in range(r0, r1):
        r = _RO.row(i)
        cnt[i - r0] = len(r["j"])
        dig[i - r0] = np.uint64(set_digest_py(r["j"]))
        el[i - r0] = r["eloc"].real
    return r0, cnt, dig, el


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["h28", "h56", "h84"])
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    ap.add_argument("--block", type=int, default=500)
    args = ap.parse_args(argv)
    sys.path.insert(0, ROOT)
    import oracle
    from synth import config_instance
    t0 = time.time()
    inst = config_instance(args.name)   # builds the cache the workers read
    n = inst.n_unq
    blocks = [(r, min(r + args.block, n)) for r in range(0, n, args.block)]
    cnt = np.zeros(n, np.int64)
    dig = np.zeros(n, np.uint64)
    el = np.zeros(n, np.float64)
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs, initializer=_init, initargs=(args.name,)) as pool:
        done = 0
        for r0, c, d, e in pool.imap_unordered(_block, blocks):
            cnt[r0:r0 + len(c)] = c
            dig[r0:r0 + len(c)] = d
            el[r0:r0 + len(c)] = e
            done += len(c)
            if done % 20000 < args.block:
                print(f"{args.name}: {done}/{n} rows, {time.time() - t0:.0f} s", flush=True)
    evar = oracle.variational_energy(inst.logpsi_re, [complex(v) for v in el])
    u_sha, xz_sha, coef_l1 = instance_digests(inst)
    path = os.path.join(HERE, f"{args.name}_rows.npz")
    np.savez_compressed(path, count=cnt.astype(np.int32), digest=dig, eloc=el,
                        evar=np.array([evar.real, evar.imag]), n_pairs=np.array([int(cnt.sum())]),
                        u_sha=np.array(u_sha), xz_sha=np.array(xz_sha), coef_l1=np.array([coef_l1]))
    print(f"{args.name}: {n} rows, {int(cnt.sum())} pairs, E^var = {evar.real!r}, "
          f"{time.time() - t0:.0f} s -> {path}")


if __name__ == "__main__":
    main()
